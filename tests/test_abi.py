"""CPU checks of the C ABI: the library builds, loads without a GPU and exports
every entry point that include/gp.h declares; the binding declares them all."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "gp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_entry_points()
    for required in ["gp_create", "gp_destroy", "gp_add_grains", "gp_set_thermal_analytic",
                     "gp_set_thermal_grid", "gp_nucleation_sites", "gp_step", "gp_grain_map",
                     "gp_get_particles", "gp_stats", "gp_last_error", "gp_hash_build",
                     "gp_contact"]:
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2504_12858_gb300 import build, native
    build.build()
    L = native.load()
    for name in declared_entry_points():
        assert hasattr(L, name), name
    assert set(declared_entry_points()) == set(native.SIGNATURES)


def test_arena_size_query_needs_no_gpu():
    import ctypes as C
    from paper_2504_12858_gb300 import native
    L = native.load()
    d = native.domain((0, 0, 0), (200e-6, 200e-6, 200e-6))
    m = native.gp_memory()
    m.capacity = 100000
    nb = C.c_size_t(0)
    assert L.gp_arena_bytes(C.byref(d), 2e-6, C.byref(m), C.byref(nb)) == 0
    assert nb.value > 100000 * 64
    # domain of more than 4000 lattice spacings along the diagonal is refused
    d2 = native.domain((0, 0, 0), (10e-3, 10e-3, 10e-3))
    assert L.gp_arena_bytes(C.byref(d2), 2e-6, C.byref(m), C.byref(nb)) == 1
    m.capacity = 0
    assert L.gp_arena_bytes(C.byref(d), 2e-6, C.byref(m), C.byref(nb)) == 1


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2504_12858_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "gp_oracle" not in txt, f


def test_checkpoint_check_needs_no_gpu():
    # the host-only check of gp_checkpoint_check refuses what is not an intact checkpoint
    # (the round trip through gp_save / gp_load is a GPU test)
    import ctypes as C

    import numpy as np
    from paper_2504_12858_gb300 import native
    L = native.load()
    step, n = C.c_int64(-1), C.c_int64(-1)
    assert L.gp_checkpoint_check(None, 0, C.byref(step), C.byref(n)) == 1
    magic = b"GPCKPT\x00\x01"
    g = np.random.default_rng(3)
    for data in (b"", magic, magic + bytes(4096), bytes(g.integers(0, 256, 4096, np.uint8))):
        assert L.gp_checkpoint_check(data, len(data), C.byref(step), C.byref(n)) == 1
        with pytest.raises(native.GPError):
            native.checkpoint_check(data)
    assert (step.value, n.value) == (-1, -1)        # outputs untouched on a refusal
