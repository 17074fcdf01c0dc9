"""gp_hash_build_static: the spatial hash for callers that cannot allocate.

Callers embedded in a host code that owns and budgets all device memory (or that
must not pay the synchronisation of an allocation) can neither pass a workspace
nor let the library call cudaMalloc; this entry point draws its scratch from a
static device array of the library instead.  These tests call it through the C
ABI and require results identical to those of gp_hash_build (the workspace
variant) on consecutive calls that reuse the shared array, unchanged free device
memory across further calls, and a clean refusal of inputs above its size limit.
The file sorts last so that a run stopping at its first failure has already run
every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2504_12858_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2504_12858_gb300 import build, native  # noqa: E402

build.build()
LIB = native.load()
DEV = torch.device("cuda:0")


def _static_hash(x, lo, hi, h):
    n = x.shape[0]
    d = native.domain(lo, hi)
    out = [torch.full((max(n, 1),), -7, dtype=torch.int32, device=DEV) for _ in range(4)]
    nc = C.c_int64(-1)
    stream = torch.cuda.current_stream(DEV)
    st = LIB.gp_hash_build_static(C.c_void_p(x.data_ptr()), n, C.byref(d), float(h),
                                  *[C.c_void_p(t.data_ptr()) for t in out], C.byref(nc),
                                  C.c_void_p(stream.cuda_stream))
    if st:
        return st, None
    m = int(nc.value)
    ks, ids, ck, cs = (t.cpu().numpy() for t in out)
    return st, (ks[:n].view(np.uint32), ids[:n], ck[:m].view(np.uint32), cs[:m])


CASES = [
    # (n, lo, hi, h, seed): different sizes and grids so each call leaves different
    # contents in the shared scratch array for the next one
    (200003, (0.0, 0.0, 0.0), (300e-6, 200e-6, 100e-6), 2e-6, 1),
    (4097, (-1e-5, 2e-5, 0.0), (5e-5, 9e-5, 3e-5), 1e-6, 2),
    (262144, (0.0, 0.0, 0.0), (80e-6, 80e-6, 80e-6), 2e-6, 3),
]


def test_static_scratch_hash_equals_workspace_hash_on_consecutive_calls():
    for n, lo, hi, h, seed in CASES + CASES[:1]:
        g = inputs.rng(seed)
        lo_a, hi_a = np.array(lo), np.array(hi)
        x = (lo_a + g.random((n, 3)) * (hi_a - lo_a)).astype(np.float32)
        x[: n // 10] = x[n // 10: 2 * (n // 10)]          # duplicates: stable order
        xd = torch.from_numpy(x).to(DEV)
        st, got = _static_hash(xd, lo, hi, h)
        assert st == 0, native.STATUS.get(st, st)
        ref = native.gp_hash_build(xd, lo, hi, h)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b)


def test_static_scratch_call_allocates_no_device_memory():
    n, lo, hi, h, seed = CASES[0]
    g = inputs.rng(seed)
    x = (np.array(lo) + g.random((n, 3)) * (np.array(hi) - np.array(lo))).astype(np.float32)
    xd = torch.from_numpy(x).to(DEV)
    d = native.domain(lo, hi)
    out = [torch.empty(n, dtype=torch.int32, device=DEV) for _ in range(4)]
    nc = C.c_int64(-1)
    stream = torch.cuda.current_stream(DEV)
    args = [C.c_void_p(xd.data_ptr()), n, C.byref(d), float(h),
            *[C.c_void_p(t.data_ptr()) for t in out], C.byref(nc), C.c_void_p(stream.cuda_stream)]
    assert LIB.gp_hash_build_static(*args) == 0          # warm-up: module and address set up
    torch.cuda.synchronize(DEV)
    free0, _ = torch.cuda.mem_get_info(DEV)
    for _ in range(3):
        assert LIB.gp_hash_build_static(*args) == 0
    torch.cuda.synchronize(DEV)
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 == free0


def test_static_scratch_refuses_inputs_above_its_limit():
    n = native.GP_STATIC_SCRATCH_MAX_POINTS + 1
    x = torch.zeros((n, 3), dtype=torch.float32, device=DEV)
    st, _ = _static_hash(x, (0, 0, 0), (1e-4, 1e-4, 1e-4), 2e-6)
    assert st == 2                                     # GP_ERR_CAPACITY
    # and the entry point still works afterwards
    st, got = _static_hash(x[:1000], (0, 0, 0), (1e-4, 1e-4, 1e-4), 2e-6)
    assert st == 0 and len(got[2]) == 1
