"""hoszp_mean_noalloc through the C ABI, against hoszp_mean.

The no-allocation entry point serves callers that may not allocate device
memory when they call (their device memory belongs to a host framework's pool,
or a cudaMalloc's implicit synchronization is unaffordable in their loop), so
it cannot use a context's workspace; its scratch is a static device array.
This file sorts last so that a run stopping at the first failure has run every
other test before it; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build

    build.build()
    L = hz.load_library()
    f = L.hoszp_mean_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    return hz, f


def call_noalloc(f, c):
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(ctypes.c_void_p(c.data_ptr()), c.numel(), ctypes.c_void_p(out.data_ptr()),
           ctypes.c_void_p(st.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, float(out.item()), int(st.item())


def test_mean_noalloc_matches_mean_twice(lib):
    hz, f = lib
    for seed, n in ((3, 1_000_003), (4, 777_777)):  # two calls in a row
        x = torch.from_numpy(datagen.sines_1d(n, seed=seed)).cuda()
        c = hz.compress(x, eb=1e-3, mode="rel")
        expected = hz.mean(c)
        rc, got, st = call_noalloc(f, c)
        assert rc == 0 and st == 0
        assert abs(got - expected) <= REL_TOL * max(abs(expected), 1e-300)


def test_mean_noalloc_rejects_streams_beyond_its_scratch(lib):
    hz, f = lib
    n = (1 << 28) + 64  # one block more than the scratch bounds
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    c = hz.compress(x, eb=0.1)
    del x
    rc, got, st = call_noalloc(f, c)
    assert rc == 0 and hz.STATUS[st] == "CAPACITY"
    assert np.isnan(got)  # a refused stream's result is NaN, never a stale or partial mean
    # and a valid call afterwards still works
    y = torch.from_numpy(datagen.sines_1d(100_000, seed=9)).cuda()
    cy = hz.compress(y, eb=1e-3, mode="rel")
    rc, got, st = call_noalloc(f, cy)
    assert rc == 0 and st == 0 and abs(got - hz.mean(cy)) <= REL_TOL * abs(hz.mean(cy))


def test_mean_noalloc_allocates_no_device_memory(lib):
    """After a first call (which loads the kernels), further calls leave the
    device's free memory unchanged: the scratch is the static array."""
    hz, f = lib
    x = torch.from_numpy(datagen.sines_1d(2_000_000, seed=21)).cuda()
    c = hz.compress(x, eb=1e-4, mode="rel")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (ctypes.c_void_p(c.data_ptr()), c.numel(), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(st.data_ptr()), stream)
    assert f(*args) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert f(*args) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert int(st.item()) == 0 and abs(float(out.item()) - hz.mean(c)) <= REL_TOL * abs(hz.mean(c))
