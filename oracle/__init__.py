"""FP64 CPU oracle of the grain-envelope particle step: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and it
imports nothing from the CUDA package.

``build()`` compiles ``gp_oracle.cpp`` with g++ (``-ffp-contract=off`` so the
binary32 predicates are evaluated exactly as written).  ``Oracle`` wraps one
simulation; module-level functions wrap the stand-alone binary32 hash / contact
references.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.cpp")
_LIB = os.path.join(_HERE, "libgp_oracle.so")
_lock = threading.Lock()
_lib = None

P_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
P_F = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
P_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
P_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
P_I8 = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
P_U8 = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
P_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _opt(ptr_type):
    """ndpointer that also accepts None (NULL)."""
    def from_param(cls, obj):
        if obj is None:
            return None
        return ptr_type.from_param(obj)
    return type("Opt" + ptr_type.__name__, (ptr_type,), {"from_param": classmethod(from_param)})


def lib():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    oD, oF, oI32, oU32, oI8, oU8 = (_opt(P_D), _opt(P_F), _opt(P_I32), _opt(P_U32),
                                    _opt(P_I8), _opt(P_U8))
    sig = {
        "go_create": (vp, [P_D, P_D, d, d, C.c_int, P_D, P_D, d]),
        "go_destroy": (None, [vp]),
        "go_set_thermal_analytic": (None, [vp, d, P_D, P_D, d]),
        "go_set_thermal_grid": (None, [vp, P_F, P_I32, P_D, P_D, P_D]),
        "go_set_solute_grid": (None, [vp, P_F, P_I32, P_D, P_D, P_D, d, d]),
        "go_set_melting": (None, [vp, C.c_int]),
        "go_set_reach_tol": (None, [vp, d]),
        "go_set_periodic": (None, [vp, C.c_int]),
        "go_add_grains": (i64, [vp, i64, P_D, P_D, C.c_int]),
        "go_seed_shell": (None, [vp, i64, P_I32, i32, d, C.c_int]),
        "go_nucleation_sites": (None, [vp, i64, P_D, P_D, P_D]),
        "go_step": (None, [vp, i32]),
        "go_num_particles": (i64, [vp]),
        "go_num_grains": (i64, [vp]),
        "go_get_step": (i64, [vp]),
        "go_set_step": (None, [vp, i64]),
        "go_get_particles": (None, [vp, oI32, oI32, oI8, oD, oU8, oD]),
        "go_load_particles": (None, [vp, i64, P_I32, P_I32, P_I8, P_D, P_U8]),
        "go_num_reached": (i64, [vp]),
        "go_get_reached": (None, [vp, P_I32, P_I32]),
        "go_add_reached": (None, [vp, i64, P_I32, P_I32]),
        "go_num_claimed": (i64, [vp]),
        "go_get_claimed": (None, [vp, P_I32, P_I32]),
        "go_add_claimed": (None, [vp, i64, P_I32, P_I32]),
        "go_get_stats": (None, [vp, P_I64]),
        "go_get_grain": (None, [vp, i32, P_D, P_D]),
        "go_undercooling": (d, [vp, P_D, d]),
        "go_velocity": (d, [vp, d]),
        "go_is_outer": (C.c_int, [P_I32, C.c_int]),
        "go_grain_map": (None, [vp, P_D, P_D, P_I32, P_I32]),
        "go_grain_map_bruteforce": (None, [vp, P_D, P_D, P_I32, P_I32]),
        "go_contact_f64": (None, [vp, P_U8, C.c_int]),
        "go_hash_build_f32": (i64, [P_F, i64, P_D, P_D, d, oU32, oI32, oU32, oI32]),
        "go_cell_keys_f32": (None, [P_F, i64, P_D, P_D, d, P_U32]),
        "go_contact_f32": (i64, [P_F, P_I32, P_U8, i64, P_D, P_D, d, oU8, oI32, i64]),
        "go_contact_bruteforce_f32": (i64, [P_F, P_I32, P_U8, i64, d, oU8, oI32, i64]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _d3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


STAT_NAMES = ("steps", "particle_steps", "frozen", "spawned", "claims_lost", "clipped",
              "clamped", "nucleated", "reached", "melted", "walkback")


class Oracle:
    """One FP64 simulation (plain sequential reference of the whole step)."""

    def __init__(self, lo, hi, h, dt, a, b, TL):
        L = lib()
        a, b = list(a), list(b)
        nterms = len(a)
        assert nterms in (1, 2) and len(b) == nterms
        a = a + [0.0] * (2 - nterms)
        b = b + [0.0] * (2 - nterms)
        self.h, self.dt = float(h), float(dt)
        self.lo, self.hi = _d3(lo), _d3(hi)
        self._p = L.go_create(self.lo, self.hi, self.h, self.dt, nterms,
                              np.array(a, np.float64), np.array(b, np.float64), float(TL))

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().go_destroy(p)
            self._p = None

    # --- set-up -------------------------------------------------------------------
    def set_thermal_analytic(self, T0, G, xref, Tdot):
        lib().go_set_thermal_analytic(self._p, float(T0), _d3(G), _d3(xref), float(Tdot))

    def set_thermal_grid(self, T, origin, spacing, vel=(0.0, 0.0, 0.0)):
        T = np.ascontiguousarray(T, dtype=np.float32)
        nz, ny, nx = T.shape
        lib().go_set_thermal_grid(self._p, T.reshape(-1), np.array([nx, ny, nz], np.int32),
                                  _d3(origin), _d3(spacing), _d3(vel))

    def set_solute_grid(self, w, origin, spacing, Tm, mL, vel=(0.0, 0.0, 0.0)):
        """Local liquidus T_m + m_L w(x) from a node-centred composition grid (nz, ny, nx)."""
        w = np.ascontiguousarray(w, dtype=np.float32)
        nz, ny, nx = w.shape
        lib().go_set_solute_grid(self._p, w.reshape(-1), np.array([nx, ny, nz], np.int32),
                                 _d3(origin), _d3(spacing), _d3(vel), float(Tm), float(mL))

    def set_periodic(self, axes):
        """Periodic axes, a bit per axis (1 = x, 2 = y, 4 = z)."""
        lib().go_set_periodic(self._p, int(axes))

    def set_melting(self, on=True):
        """Melting walk-back pass at the start of every step (Sec. 2.1.3)."""
        lib().go_set_melting(self._p, 1 if on else 0)

    def set_reach_tol(self, tol):
        """Tolerance of the reached-target test (default 2^-20 of a spacing)."""
        lib().go_set_reach_tol(self._p, float(tol))

    def add_grains(self, pos, quat, nucleate=True) -> int:
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        return int(lib().go_add_grains(self._p, pos.shape[0], pos.reshape(-1),
                                       quat.reshape(-1), 1 if nucleate else 0))

    def seed_shell(self, grains, n0, ell0=0.0, interior=False):
        g = np.ascontiguousarray(grains, np.int32).reshape(-1)
        lib().go_seed_shell(self._p, g.size, g, int(n0), float(ell0), 1 if interior else 0)

    def nucleation_sites(self, pos, dTn, quat):
        pos = np.ascontiguousarray(pos, np.float64).reshape(-1, 3)
        dTn = np.ascontiguousarray(dTn, np.float64).reshape(-1)
        quat = np.ascontiguousarray(quat, np.float64).reshape(-1, 4)
        lib().go_nucleation_sites(self._p, pos.shape[0], pos.reshape(-1), dTn,
                                  quat.reshape(-1))

    def step(self, n=1):
        lib().go_step(self._p, int(n))

    # --- state ----------------------------------------------------------------------
    @property
    def n_particles(self) -> int:
        return int(lib().go_num_particles(self._p))

    @property
    def n_grains(self) -> int:
        return int(lib().go_num_grains(self._p))

    @property
    def step_index(self) -> int:
        return int(lib().go_get_step(self._p))

    def set_step(self, n):
        lib().go_set_step(self._p, int(n))

    def particles(self) -> dict:
        n = self.n_particles
        out = dict(grain=np.zeros(n, np.int32), site=np.zeros((n, 3), np.int32),
                   dir=np.zeros(n, np.int8), ell=np.zeros(n, np.float64),
                   state=np.zeros(n, np.uint8), x=np.zeros((n, 3), np.float64))
        lib().go_get_particles(self._p, out["grain"], out["site"].reshape(-1), out["dir"],
                               out["ell"], out["state"], out["x"].reshape(-1))
        return out

    def load_particles(self, grain, site, dir, ell, state):
        n = len(grain)
        lib().go_load_particles(self._p, n, np.ascontiguousarray(grain, np.int32),
                                np.ascontiguousarray(site, np.int32).reshape(-1),
                                np.ascontiguousarray(dir, np.int8),
                                np.ascontiguousarray(ell, np.float64),
                                np.ascontiguousarray(state, np.uint8))

    def reached(self):
        n = int(lib().go_num_reached(self._p))
        g = np.zeros(n, np.int32)
        s = np.zeros((n, 3), np.int32)
        lib().go_get_reached(self._p, g, s.reshape(-1))
        return g, s

    def add_reached(self, grain, site):
        g = np.ascontiguousarray(grain, np.int32)
        lib().go_add_reached(self._p, g.size, g,
                             np.ascontiguousarray(site, np.int32).reshape(-1))

    def claimed(self):
        n = int(lib().go_num_claimed(self._p))
        g = np.zeros(n, np.int32)
        s = np.zeros((n, 3), np.int32)
        lib().go_get_claimed(self._p, g, s.reshape(-1))
        return g, s

    def add_claimed(self, grain, site):
        g = np.ascontiguousarray(grain, np.int32)
        lib().go_add_claimed(self._p, g.size, g,
                             np.ascontiguousarray(site, np.int32).reshape(-1))

    def stats(self) -> dict:
        out = np.zeros(len(STAT_NAMES), np.int64)
        lib().go_get_stats(self._p, out)
        return dict(zip(STAT_NAMES, (int(v) for v in out)))

    def grain(self, g):
        c = np.zeros(3)
        R = np.zeros(9)
        lib().go_get_grain(self._p, int(g), c, R)
        return c, R.reshape(3, 3)

    def undercooling(self, x, t) -> float:
        return float(lib().go_undercooling(self._p, _d3(x), float(t)))

    def velocity(self, dT) -> float:
        return float(lib().go_velocity(self._p, float(dT)))

    def grain_map(self, origin, spacing, n, bruteforce=False):
        n = np.ascontiguousarray(n, np.int32).reshape(3)
        out = np.zeros(int(n[0]) * int(n[1]) * int(n[2]), np.int32)
        f = lib().go_grain_map_bruteforce if bruteforce else lib().go_grain_map
        f(self._p, _d3(origin), _d3(spacing), n, out)
        return out.reshape(int(n[2]), int(n[1]), int(n[0]))

    def contact_flags(self, bruteforce=False):
        out = np.zeros(self.n_particles, np.uint8)
        lib().go_contact_f64(self._p, out, 1 if bruteforce else 0)
        return out


def is_outer(site, k) -> bool:
    return bool(lib().go_is_outer(np.ascontiguousarray(site, np.int32).reshape(3), int(k)))


def hash_build_f32(x, lo, hi, h):
    """Binary32 cell keys + stable sort + cell starts (reference of the CUDA hash)."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    n = x.shape[0]
    ks = np.zeros(n, np.uint32)
    ids = np.zeros(n, np.int32)
    ck = np.zeros(max(n, 1), np.uint32)
    cs = np.zeros(max(n, 1), np.int32)
    nc = lib().go_hash_build_f32(x.reshape(-1), n, _d3(lo), _d3(hi), float(h), ks, ids, ck, cs)
    return ks, ids, ck[:nc].copy(), cs[:nc].copy()


def cell_keys_f32(x, lo, hi, h):
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    out = np.zeros(x.shape[0], np.uint32)
    lib().go_cell_keys_f32(x.reshape(-1), x.shape[0], _d3(lo), _d3(hi), float(h), out)
    return out


def contact_f32(x, grain, state, lo, hi, h, want_pairs=False, bruteforce=False):
    """Binary32 contact flags (and sorted i<j pair list) by cell list or exhaustively."""
    x = np.ascontiguousarray(x, np.float32).reshape(-1, 3)
    n = x.shape[0]
    grain = np.ascontiguousarray(grain, np.int32)
    state = np.ascontiguousarray(state, np.uint8)
    fr = np.zeros(n, np.uint8)
    L = lib()
    if bruteforce:
        npairs = L.go_contact_bruteforce_f32(x.reshape(-1), grain, state, n, float(h), fr, None, 0)
    else:
        npairs = L.go_contact_f32(x.reshape(-1), grain, state, n, _d3(lo), _d3(hi), float(h),
                                  fr, None, 0)
    if not want_pairs:
        return fr
    pairs = np.zeros((max(npairs, 1), 2), np.int32)
    if bruteforce:
        L.go_contact_bruteforce_f32(x.reshape(-1), grain, state, n, float(h), None,
                                    pairs.reshape(-1), npairs)
        pairs = pairs[:npairs]
        order = np.lexsort((pairs[:, 1], pairs[:, 0]))
        pairs = pairs[order]
    else:
        L.go_contact_f32(x.reshape(-1), grain, state, n, _d3(lo), _d3(hi), float(h), None,
                         pairs.reshape(-1), npairs)
        pairs = pairs[:npairs]
    return fr, pairs
