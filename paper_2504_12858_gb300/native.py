"""Thin ctypes binding of the CUDA library declared in ``include/gp.h``.

Argument marshalling only: every step of the particle update runs in the
library's kernels.  PyTorch supplies device memory (the context arena and the
workspaces of the stand-alone calls) and the CUDA stream.  ``load()`` raises if
the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgp.so")

GP_DEVICE_PTR = 1
STATUS = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_CAPACITY", 3: "GP_ERR_HASH_FULL",
          4: "GP_ERR_CUDA", 5: "GP_ERR_STATE", 6: "GP_ERR_TIMEOUT"}


class gp_domain(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class gp_growth_law(C.Structure):
    _fields_ = [("nterms", C.c_int32), ("a", C.c_double * 2), ("b", C.c_double * 2),
                ("T_liquidus", C.c_double)]


class gp_thermal_analytic(C.Structure):
    _fields_ = [("T0", C.c_double), ("G", C.c_double * 3), ("x_ref", C.c_double * 3),
                ("Tdot", C.c_double)]


class gp_thermal_grid(C.Structure):
    _fields_ = [("T", C.c_void_p), ("n", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3), ("frame_vel", C.c_double * 3), ("flags", C.c_int32)]


class gp_solute_grid(C.Structure):
    _fields_ = [("w", C.c_void_p), ("n", C.c_int32 * 3), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3), ("frame_vel", C.c_double * 3), ("T_m", C.c_double),
                ("m_L", C.c_double), ("flags", C.c_int32)]


class gp_voxel_grid(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("spacing", C.c_double * 3), ("n", C.c_int32 * 3)]


class gp_memory(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("reached_capacity", C.c_int64),
                ("claim_blocks", C.c_int64), ("max_grains", C.c_int32),
                ("max_nuclei", C.c_int32), ("grid_nodes", C.c_int64),
                ("tape_steps", C.c_int64), ("arena", C.c_void_p),
                ("arena_bytes", C.c_size_t), ("solute_nodes", C.c_int64),
                ("tape_checkpoint_every", C.c_int64)]


STATS_FIELDS = ["step", "n_live", "n_active", "n_frozen", "n_grains", "n_reached",
                "particle_steps", "n_frozen_new", "n_spawned", "n_claims_lost", "n_clipped",
                "n_clamped", "n_nucleated", "n_claim_blocks", "error_flags", "n_melted",
                "n_walkback"]


class gp_stats_t(C.Structure):
    _fields_ = [(f, C.c_int64) for f in STATS_FIELDS] + [("reserved", C.c_int64 * 3)]


class gp_launch_config(C.Structure):
    _fields_ = [("build_ctas_per_sm", C.c_int32), ("advance_ctas_per_sm", C.c_int32),
                ("emit_ctas_per_sm", C.c_int32), ("graph_steps", C.c_int32)]


class gp_kernel_prof(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("units", C.c_double), ("bytes_per_unit", C.c_double)]


# name -> (restype, argtypes); every exported entry point of include/gp.h
_P = C.c_void_p
SIGNATURES = {
    "gp_arena_bytes": (C.c_int, [C.POINTER(gp_domain), C.c_double, C.POINTER(gp_memory),
                                 C.POINTER(C.c_size_t)]),
    "gp_create": (C.c_int, [C.POINTER(gp_domain), C.c_double, C.c_double,
                            C.POINTER(gp_growth_law), C.POINTER(gp_memory), _P, C.POINTER(_P)]),
    "gp_destroy": (C.c_int, [_P]),
    "gp_last_error": (C.c_char_p, [_P]),
    "gp_add_grains": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int32, C.POINTER(C.c_int32)]),
    "gp_seed_shell": (C.c_int, [_P, C.c_int64, _P, C.c_int32, C.c_double]),
    "gp_set_thermal_analytic": (C.c_int, [_P, C.POINTER(gp_thermal_analytic)]),
    "gp_set_thermal_grid": (C.c_int, [_P, C.POINTER(gp_thermal_grid)]),
    "gp_set_solute_grid": (C.c_int, [_P, C.POINTER(gp_solute_grid)]),
    "gp_set_melting": (C.c_int, [_P, C.c_int32]),
    "gp_set_periodic": (C.c_int, [_P, C.c_int32]),
    "gp_set_obstacle_store": (C.c_int, [_P, C.c_int32]),
    "gp_inspect_order": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, _P, C.POINTER(C.c_int64),
                                   _P, C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_uint32)]),
    "gp_nucleation_sites": (C.c_int, [_P, C.c_int64, _P, _P, _P]),
    "gp_step": (C.c_int, [_P, C.c_int32]),
    "gp_grain_map": (C.c_int, [_P, C.POINTER(gp_voxel_grid), _P, C.c_int32]),
    "gp_stats": (C.c_int, [_P, C.POINTER(gp_stats_t)]),
    "gp_get_particles": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, _P,
                                   C.POINTER(C.c_int64)]),
    "gp_load_particles": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, C.c_int64]),
    "gp_add_sites": (C.c_int, [_P, C.c_int64, _P, _P, C.c_int32, C.c_int32]),
    "gp_get_reached": (C.c_int, [_P, C.c_int64, _P, _P, C.POINTER(C.c_int64)]),
    "gp_save": (C.c_int, [_P, _P, C.c_size_t, C.POINTER(C.c_size_t)]),
    "gp_load": (C.c_int, [_P, _P, C.c_size_t]),
    "gp_checkpoint_check": (C.c_int, [_P, C.c_size_t, C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64)]),
    "gp_profile": (C.c_int, [_P, C.c_int32]),
    "gp_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(gp_kernel_prof),
                                  C.POINTER(C.c_int32)]),
    "gp_hash_workspace_bytes": (C.c_int, [C.c_int64, C.POINTER(gp_domain), C.c_double,
                                          C.POINTER(C.c_size_t)]),
    "gp_hash_build": (C.c_int, [_P, C.c_int64, C.POINTER(gp_domain), C.c_double, _P, _P, _P, _P,
                                C.POINTER(C.c_int64), _P, C.c_size_t, _P]),
    "gp_contact": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(gp_domain), C.c_double, _P, _P,
                             C.c_int64, C.POINTER(C.c_int64), _P, C.c_size_t, _P]),
    "gp_hash_build_static": (C.c_int, [_P, C.c_int64, C.POINTER(gp_domain), C.c_double, _P, _P,
                                       _P, _P, C.POINTER(C.c_int64), _P]),
    "gp_selftest_wait": (C.c_int, [C.c_int32, C.c_uint32, _P]),
    "gp_tape_begin": (C.c_int, [_P]),
    "gp_adjoint": (C.c_int, [_P, _P, C.c_int64, C.c_int32, C.POINTER(C.c_double)]),
    "gp_batch_arena_bytes": (C.c_int, [C.c_int32, C.POINTER(gp_domain), C.c_double,
                                       C.POINTER(gp_memory), C.POINTER(C.c_size_t)]),
    "gp_batch_create": (C.c_int, [C.c_int32, C.POINTER(gp_domain), C.c_double, C.c_double,
                                  C.POINTER(gp_growth_law), C.POINTER(gp_memory), _P,
                                  C.POINTER(_P)]),
    "gp_run_set_thermal_analytic": (C.c_int, [_P, C.c_int32, C.POINTER(gp_thermal_analytic)]),
    "gp_run_add_grains": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, C.c_int32,
                                    C.POINTER(C.c_int32)]),
    "gp_run_nucleation_sites": (C.c_int, [_P, C.c_int32, C.c_int64, _P, _P, _P,
                                          C.POINTER(C.c_int32)]),
    "gp_run_grain_map": (C.c_int, [_P, C.c_int32, C.POINTER(gp_voxel_grid), _P, C.c_int32]),
    "gp_run_counts": (C.c_int, [_P, C.c_int32, _P, _P]),
    "gp_grain_table": (C.c_int, [_P, C.c_int64, _P, _P, C.POINTER(C.c_int64)]),
    "gp_get_launch_config": (C.c_int, [_P, C.POINTER(gp_launch_config)]),
    "gp_set_launch_config": (C.c_int, [_P, C.POINTER(gp_launch_config)]),
    "gp_autotune": (C.c_int, [_P, C.c_int32, C.POINTER(gp_launch_config)]),
}
GP_STATIC_SCRATCH_MAX_POINTS = 262144

_lib = None


class GPError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load():
    """Loads libgp.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "or python -m paper_2504_12858_gb300.build")
    L = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """Host pointer of a numpy array (None -> NULL)."""
    if a is None:
        return None
    return a.ctypes.data_as(C.c_void_p)


def _dptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def checkpoint_check(data: bytes) -> dict:
    """Host-only check of a checkpoint (``gp_checkpoint_check``): its step counter and
    particle count; raises GPError (GP_ERR_ARG) if it is not an intact checkpoint."""
    data = bytes(data)
    step, n = C.c_int64(0), C.c_int64(0)
    st = load().gp_checkpoint_check(data, len(data), C.byref(step), C.byref(n))
    if st != 0:
        raise GPError(st, "not an intact checkpoint")
    return {"step": int(step.value), "n_particles": int(n.value)}


def domain(lo, hi):
    d = gp_domain()
    d.lo[:] = [float(v) for v in lo]
    d.hi[:] = [float(v) for v in hi]
    return d


def growth_law(a, b, T_L):
    g = gp_growth_law()
    g.nterms = len(a)
    a = list(a) + [0.0] * (2 - len(a))
    b = list(b) + [0.0] * (2 - len(b))
    g.a[:] = a
    g.b[:] = b
    g.T_liquidus = float(T_L)
    return g


class Sim:
    """One simulation context (``gp_create`` ... ``gp_destroy``).

    Device memory is a torch uint8 tensor (the arena); the stream is a torch CUDA
    stream whose handle is passed to the library.
    """

    def __init__(self, lo, hi, h, dt, a, b, T_L, capacity, reached_capacity=0,
                 claim_blocks=0, max_grains=0, max_nuclei=0, grid_nodes=0, tape_steps=0,
                 stream=None, device="cuda", solute_nodes=0, tape_checkpoint_every=0,
                 arena_fill=None):
        self.lo, self.hi = tuple(lo), tuple(hi)
        self._open([(lo, hi)], False, h, dt, a, b, T_L, capacity, reached_capacity,
                   claim_blocks, max_grains, max_nuclei, grid_nodes, tape_steps, stream, device,
                   solute_nodes, tape_checkpoint_every, arena_fill)

    def _open(self, domains, batch, h, dt, a, b, T_L, capacity, reached_capacity, claim_blocks,
              max_grains, max_nuclei, grid_nodes, tape_steps, stream, device, solute_nodes=0,
              tape_checkpoint_every=0, arena_fill=None):
        import torch
        self._torch = torch
        L = load()
        self.h, self.dt = float(h), float(dt)
        self.nruns = len(domains)
        self._doms = (gp_domain * self.nruns)(*[domain(lo, hi) for lo, hi in domains])
        self._law = growth_law(a, b, T_L)
        mem = gp_memory()
        mem.capacity = int(capacity)
        mem.reached_capacity = int(reached_capacity)
        mem.claim_blocks = int(claim_blocks)
        mem.max_grains = int(max_grains)
        mem.max_nuclei = int(max_nuclei)
        mem.grid_nodes = int(grid_nodes)
        mem.tape_steps = int(tape_steps)
        mem.solute_nodes = int(solute_nodes)
        mem.tape_checkpoint_every = int(tape_checkpoint_every)
        nb = C.c_size_t(0)
        if batch:
            self._check(L.gp_batch_arena_bytes(self.nruns, self._doms, self.h, C.byref(mem),
                                               C.byref(nb)))
        else:
            self._check(L.gp_arena_bytes(self._doms, self.h, C.byref(mem), C.byref(nb)))
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        self.arena = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)
        if arena_fill is not None:  # tests: a known byte where the library must write first
            self.arena.fill_(int(arena_fill))
            torch.cuda.synchronize(self.device)
        mem.arena = self.arena.data_ptr()
        mem.arena_bytes = nb.value
        self.arena_bytes = int(nb.value)
        self._mem = mem
        h_ = C.c_void_p()
        with torch.cuda.device(self.device):
            if batch:
                self._check(L.gp_batch_create(self.nruns, self._doms, self.h, self.dt,
                                              C.byref(self._law), C.byref(mem),
                                              C.c_void_p(self.stream.cuda_stream), C.byref(h_)))
            else:
                self._check(L.gp_create(self._doms, self.h, self.dt, C.byref(self._law),
                                        C.byref(mem), C.c_void_p(self.stream.cuda_stream),
                                        C.byref(h_)))
        self._h = h_

    # -- plumbing --------------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            msg = ""
            h = getattr(self, "_h", None)
            if h:
                msg = (load().gp_last_error(h) or b"").decode()
            raise GPError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            load().gp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls (same names as the C ABI) ---------------------------------------------
    def gp_add_grains(self, pos, quat, nucleate=True) -> int:
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        first = C.c_int32(0)
        self._check(load().gp_add_grains(self._h, pos.shape[0], _ptr(pos), _ptr(quat),
                                         1 if nucleate else 0, C.byref(first)))
        return int(first.value)

    def gp_seed_shell(self, grains, n0, ell0=0.0):
        g = np.ascontiguousarray(grains, np.int32).reshape(-1)
        self._check(load().gp_seed_shell(self._h, g.size, _ptr(g), int(n0), float(ell0)))

    def gp_set_thermal_analytic(self, T0, G, xref, Tdot):
        th = gp_thermal_analytic()
        th.T0 = float(T0)
        th.G[:] = [float(v) for v in G]
        th.x_ref[:] = [float(v) for v in xref]
        th.Tdot = float(Tdot)
        self._check(load().gp_set_thermal_analytic(self._h, C.byref(th)))

    def gp_set_thermal_grid(self, T, origin, spacing, vel=(0.0, 0.0, 0.0)):
        """T: numpy (host) or torch CUDA tensor of shape (nz, ny, nx), float32."""
        th = gp_thermal_grid()
        keep = T
        if hasattr(T, "data_ptr") and getattr(T, "is_cuda", False):
            assert T.dtype == self._torch.float32 and T.is_contiguous()
            th.T = T.data_ptr()
            th.flags = GP_DEVICE_PTR
        else:
            keep = np.ascontiguousarray(T, np.float32)
            th.T = keep.ctypes.data
            th.flags = 0
        nz, ny, nx = keep.shape
        th.n[:] = [nx, ny, nz]
        th.origin[:] = [float(v) for v in origin]
        th.spacing[:] = [float(v) for v in spacing]
        th.frame_vel[:] = [float(v) for v in vel]
        self._check(load().gp_set_thermal_grid(self._h, C.byref(th)))

    def gp_set_periodic(self, axes):
        """Periodic axes, a bit per axis (1 = x, 2 = y, 4 = z)."""
        self._check(load().gp_set_periodic(self._h, int(axes)))

    def gp_set_obstacle_store(self, mode=1):
        """0 off, 1 automatic (default), 2 a flush every step with FROZEN particles."""
        self._check(load().gp_set_obstacle_store(self._h, int(mode)))

    def gp_inspect_order(self, which=0):
        """Ordering of the next step (which = 0) or the obstacle store (1): dict of
        keys_in, keys_sorted, src (uint32 numpy), table (nseg, 4) uint32 and stamp."""
        L = load()
        n, nseg, stamp = C.c_int64(0), C.c_int64(0), C.c_uint32(0)
        self._check(L.gp_inspect_order(self._h, int(which), 0, None, None, None, C.byref(n),
                                       None, 0, C.byref(nseg), C.byref(stamp)))
        m = int(n.value)
        out = dict(keys_in=np.zeros(m, np.uint32), keys_sorted=np.zeros(m, np.uint32),
                   src=np.zeros(m, np.uint32), table=np.zeros((int(nseg.value), 4), np.uint32))
        self._check(L.gp_inspect_order(self._h, int(which), m, _ptr(out["keys_in"]),
                                       _ptr(out["keys_sorted"]), _ptr(out["src"]), C.byref(n),
                                       _ptr(out["table"]), int(nseg.value), C.byref(nseg),
                                       C.byref(stamp)))
        out["stamp"] = int(stamp.value)
        return out

    def gp_set_melting(self, enable=True):
        self._check(load().gp_set_melting(self._h, 1 if enable else 0))

    def gp_set_solute_grid(self, w, origin, spacing, T_m, m_L, vel=(0.0, 0.0, 0.0)):
        """w: numpy (host) or torch CUDA float32 tensor of shape (nz, ny, nx)."""
        sg = gp_solute_grid()
        keep = w
        if hasattr(w, "data_ptr") and getattr(w, "is_cuda", False):
            assert w.dtype == self._torch.float32 and w.is_contiguous()
            sg.w = w.data_ptr()
            sg.flags = GP_DEVICE_PTR
        else:
            keep = np.ascontiguousarray(w, np.float32)
            sg.w = keep.ctypes.data
            sg.flags = 0
        nz, ny, nx = keep.shape
        sg.n[:] = [nx, ny, nz]
        sg.origin[:] = [float(v) for v in origin]
        sg.spacing[:] = [float(v) for v in spacing]
        sg.frame_vel[:] = [float(v) for v in vel]
        sg.T_m = float(T_m)
        sg.m_L = float(m_L)
        self._check(load().gp_set_solute_grid(self._h, C.byref(sg)))

    def gp_nucleation_sites(self, pos, dTn, quat):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        dTn = np.ascontiguousarray(dTn, np.float64).reshape(-1)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        self._check(load().gp_nucleation_sites(self._h, pos.shape[0], _ptr(pos), _ptr(dTn),
                                               _ptr(quat)))

    def gp_step(self, n=1):
        self._check(load().gp_step(self._h, int(n)))

    def gp_stats(self) -> dict:
        s = gp_stats_t()
        self._check(load().gp_stats(self._h, C.byref(s)))
        return {f: int(getattr(s, f)) for f in STATS_FIELDS}

    def gp_get_particles(self) -> dict:
        L = load()
        n = C.c_int64(0)
        self._check(L.gp_get_particles(self._h, 0, None, None, None, None, None, None,
                                       C.byref(n)))
        m = int(n.value)
        out = dict(grain=np.zeros(m, np.int32), site=np.zeros((m, 3), np.int32),
                   dir=np.zeros(m, np.int8), ell=np.zeros(m, np.float32),
                   state=np.zeros(m, np.uint8), x=np.zeros((m, 3), np.float32))
        self._check(L.gp_get_particles(self._h, m, _ptr(out["grain"]), _ptr(out["site"]),
                                       _ptr(out["dir"]), _ptr(out["ell"]), _ptr(out["state"]),
                                       _ptr(out["x"]), C.byref(n)))
        return out

    def gp_load_particles(self, grain, site, dir, ell, state, step):
        grain = np.ascontiguousarray(grain, np.int32)
        site = np.ascontiguousarray(site, np.int32).reshape(-1, 3)
        dir = np.ascontiguousarray(dir, np.int8)
        ell = np.ascontiguousarray(ell, np.float32)
        state = np.ascontiguousarray(state, np.uint8)
        self._check(load().gp_load_particles(self._h, grain.size, _ptr(grain), _ptr(site),
                                             _ptr(dir), _ptr(ell), _ptr(state), int(step)))

    def gp_add_sites(self, grain, site, reached, claimed):
        grain = np.ascontiguousarray(grain, np.int32)
        site = np.ascontiguousarray(site, np.int32).reshape(-1, 3)
        self._check(load().gp_add_sites(self._h, grain.size, _ptr(grain), _ptr(site),
                                        1 if reached else 0, 1 if claimed else 0))

    def gp_get_reached(self):
        L = load()
        n = C.c_int64(0)
        self._check(L.gp_get_reached(self._h, 0, None, None, C.byref(n)))
        m = int(n.value)
        g = np.zeros(m, np.int32)
        s = np.zeros((m, 3), np.int32)
        self._check(L.gp_get_reached(self._h, m, _ptr(g), _ptr(s), C.byref(n)))
        return g, s

    def gp_save(self) -> bytes:
        """Checkpoint of the context between steps (``gp_save``), as bytes."""
        L = load()
        n = C.c_size_t(0)
        self._check(L.gp_save(self._h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(max(int(n.value), 1))
        self._check(L.gp_save(self._h, buf, int(n.value), C.byref(n)))
        return buf.raw[:int(n.value)]

    def gp_load(self, data: bytes):
        """Loads a checkpoint of ``gp_save`` into this new context (``gp_load``)."""
        data = bytes(data)
        self._check(load().gp_load(self._h, data, len(data)))

    def gp_grain_map(self, origin, spacing, n, out=None):
        """Host numpy result, or into a torch CUDA int32 tensor ``out``."""
        g = gp_voxel_grid()
        g.origin[:] = [float(v) for v in origin]
        g.spacing[:] = [float(v) for v in spacing]
        g.n[:] = [int(v) for v in n]
        if out is not None:
            self._check(load().gp_grain_map(self._h, C.byref(g), _dptr(out), GP_DEVICE_PTR))
            return out
        res = np.zeros((int(n[2]), int(n[1]), int(n[0])), np.int32)
        self._check(load().gp_grain_map(self._h, C.byref(g), _ptr(res), 0))
        return res

    def gp_tape_begin(self):
        self._check(load().gp_tape_begin(self._h))

    def gp_adjoint(self, seed):
        """seed: dL/d ell of the live particles in store order (numpy float32 or a
        torch CUDA float32 tensor).  Returns dL/d(a0, b0, a1, b1, Gx, Gy, Gz, Tdot)."""
        g = (C.c_double * 8)()
        if hasattr(seed, "data_ptr") and getattr(seed, "is_cuda", False):
            self._check(load().gp_adjoint(self._h, _dptr(seed), seed.numel(), GP_DEVICE_PTR, g))
        else:
            sd = np.ascontiguousarray(seed, np.float32)
            self._check(load().gp_adjoint(self._h, _ptr(sd), sd.size, 0, g))
        return np.array(list(g))

    def gp_profile(self, enable=True):
        self._check(load().gp_profile(self._h, 1 if enable else 0))

    def gp_profile_read(self) -> list:
        L = load()
        n = C.c_int32(0)
        buf = (gp_kernel_prof * 32)()
        self._check(L.gp_profile_read(self._h, 32, buf, C.byref(n)))
        return [dict(name=buf[i].name.decode(), launches=int(buf[i].launches),
                     total_ms=float(buf[i].total_ms), units=float(buf[i].units),
                     bytes_per_unit=float(buf[i].bytes_per_unit)) for i in range(n.value)]


class Batch(Sim):
    """A batch context (``gp_batch_create``): ``domains`` is a list of (lo, hi) per
    run; the run-level calls take the run index first."""

    def __init__(self, domains, h, dt, a, b, T_L, capacity, reached_capacity=0,
                 claim_blocks=0, max_grains=0, max_nuclei=0, stream=None, device="cuda",
                 arena_fill=None):
        self.domains = [(tuple(lo), tuple(hi)) for lo, hi in domains]
        self._open(self.domains, True, h, dt, a, b, T_L, capacity, reached_capacity,
                   claim_blocks, max_grains, max_nuclei, 0, 0, stream, device,
                   arena_fill=arena_fill)

    def gp_run_set_thermal_analytic(self, run, T0, G, xref, Tdot):
        th = gp_thermal_analytic()
        th.T0 = float(T0)
        th.G[:] = [float(v) for v in G]
        th.x_ref[:] = [float(v) for v in xref]
        th.Tdot = float(Tdot)
        self._check(load().gp_run_set_thermal_analytic(self._h, int(run), C.byref(th)))

    def gp_run_add_grains(self, run, pos, quat, nucleate=True) -> int:
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        first = C.c_int32(0)
        self._check(load().gp_run_add_grains(self._h, int(run), pos.shape[0], _ptr(pos),
                                             _ptr(quat), 1 if nucleate else 0, C.byref(first)))
        return int(first.value)

    def gp_run_nucleation_sites(self, run, pos, dTn, quat) -> int:
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        dTn = np.ascontiguousarray(dTn, np.float64).reshape(-1)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        first = C.c_int32(0)
        self._check(load().gp_run_nucleation_sites(self._h, int(run), pos.shape[0], _ptr(pos),
                                                   _ptr(dTn), _ptr(quat), C.byref(first)))
        return int(first.value)

    def gp_run_grain_map(self, run, origin, spacing, n):
        g = gp_voxel_grid()
        g.origin[:] = [float(v) for v in origin]
        g.spacing[:] = [float(v) for v in spacing]
        g.n[:] = [int(v) for v in n]
        res = np.zeros((int(n[2]), int(n[1]), int(n[0])), np.int32)
        self._check(load().gp_run_grain_map(self._h, int(run), C.byref(g), _ptr(res), 0))
        return res

    def gp_get_launch_config(self) -> dict:
        cfg = gp_launch_config()
        self._check(load().gp_get_launch_config(self._h, C.byref(cfg)))
        return {f: int(getattr(cfg, f)) for f, _ in gp_launch_config._fields_}

    def gp_set_launch_config(self, **kw):
        cfg = gp_launch_config()
        cur = self.gp_get_launch_config()
        cur.update(kw)
        for f, v in cur.items():
            setattr(cfg, f, int(v))
        self._check(load().gp_set_launch_config(self._h, C.byref(cfg)))

    def gp_autotune(self, trial_steps=2) -> dict:
        cfg = gp_launch_config()
        self._check(load().gp_autotune(self._h, int(trial_steps), C.byref(cfg)))
        return {f: int(getattr(cfg, f)) for f, _ in gp_launch_config._fields_}

    def gp_run_counts(self):
        live = np.zeros(self.nruns, np.int64)
        active = np.zeros(self.nruns, np.int64)
        self._check(load().gp_run_counts(self._h, self.nruns, _ptr(live), _ptr(active)))
        return live, active


def gp_selftest_wait(which, spin_limit, stream=None):
    """Runs one bounded device wait on a word nothing publishes; returns the status
    (GP_ERR_TIMEOUT = 6 when the wait gave up, as it must)."""
    import torch
    s = stream or torch.cuda.current_stream()
    return int(load().gp_selftest_wait(int(which), int(spin_limit), C.c_void_p(s.cuda_stream)))


def grain_table(sim):
    """(nucleus positions (n, 3) float32, run (n,) int32) of every grain of a context."""
    L = load()
    n = C.c_int64(0)
    sim._check(L.gp_grain_table(sim._h, 0, None, None, C.byref(n)))
    m = int(n.value)
    c3 = np.zeros((m, 3), np.float32)
    run = np.zeros(m, np.int32)
    sim._check(L.gp_grain_table(sim._h, m, _ptr(c3), _ptr(run), C.byref(n)))
    return c3, run


def _workspace(n, lo, hi, h, device):
    import torch
    L = load()
    d = domain(lo, hi)
    nb = C.c_size_t(0)
    st = L.gp_hash_workspace_bytes(int(n), C.byref(d), float(h), C.byref(nb))
    if st:
        raise GPError(st, "workspace size")
    return d, torch.empty(max(int(nb.value), 256), dtype=torch.uint8, device=device)


def gp_hash_build(x3, lo, hi, h, stream=None):
    """Stand-alone spatial hash of a (n, 3) float32 CUDA tensor.

    Returns (keys_sorted uint32 as int64 numpy, ids_sorted, cell_keys, cell_start)."""
    import torch
    L = load()
    n = x3.shape[0]
    dev = x3.device
    d, ws = _workspace(n, lo, hi, h, dev)
    ks = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ids = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    ck = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cs = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    nc = C.c_int64(0)
    s = stream or torch.cuda.current_stream(dev)
    st = L.gp_hash_build(_dptr(x3), n, C.byref(d), float(h), _dptr(ks), _dptr(ids), _dptr(ck),
                         _dptr(cs), C.byref(nc), _dptr(ws), ws.numel(), C.c_void_p(s.cuda_stream))
    if st:
        raise GPError(st, "gp_hash_build")
    s.synchronize()
    u = lambda t, m: t[:m].cpu().numpy().view(np.uint32)
    return (u(ks, n), ids[:n].cpu().numpy(), u(ck, nc.value), cs[:nc.value].cpu().numpy())


def gp_contact(x3, grain, state, lo, hi, h, want_pairs=False, pair_cap=None, stream=None):
    """Stand-alone contact search on CUDA tensors; returns freeze (and sorted pairs)."""
    import torch
    L = load()
    n = x3.shape[0]
    dev = x3.device
    d, ws = _workspace(n, lo, hi, h, dev)
    fr = torch.zeros(max(n, 1), dtype=torch.uint8, device=dev)
    cap = int(pair_cap if pair_cap is not None else 8 * max(n, 1))
    pairs = torch.zeros((cap, 2), dtype=torch.int32, device=dev) if want_pairs else None
    npairs = C.c_int64(0)
    s = stream or torch.cuda.current_stream(dev)
    st = L.gp_contact(_dptr(x3), _dptr(grain), _dptr(state), n, C.byref(d), float(h), _dptr(fr),
                      _dptr(pairs), cap if want_pairs else 0,
                      C.byref(npairs) if want_pairs else None, _dptr(ws), ws.numel(),
                      C.c_void_p(s.cuda_stream))
    if st:
        raise GPError(st, "gp_contact")
    s.synchronize()
    f = fr[:n].cpu().numpy()
    if not want_pairs:
        return f
    m = int(npairs.value)
    p = pairs[:min(m, cap)].cpu().numpy()
    order = np.lexsort((p[:, 1], p[:, 0]))
    return f, p[order], m
