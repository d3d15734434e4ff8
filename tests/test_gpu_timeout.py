"""Failure detection without a GPU fault: the library's bounded waits, run on a
flag that nothing sets (hoszp_selftest_wait through the C ABI), give up with
HOSZP_ERR_TIMEOUT in the context's status word, and the context then serves
ordinary calls again. The look-back wait is given a few hundred polls, the
mbarrier wait one millisecond: nothing spins without a limit."""
import ctypes
import time

import numpy as np
import pytest

import datagen
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build

    build.build()
    O.build()
    return hz


@pytest.mark.parametrize("which,limit", [(0, 300), (1, 1_000_000)])
def test_bounded_wait_gives_up_and_context_stays_usable(hz, which, limit):
    ctx = hz.Context(0)
    x = datagen.sines_1d(70_001, seed=41)
    c = hz.compress(torch.from_numpy(x).cuda(), eb=1e-3, mode="rel", ctx=ctx)
    oc = O.compress(x, eb=1e-3, mode="rel")
    L = hz.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    assert L.hoszp_selftest_wait(ctx.handle, which, limit, stream) == 0
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert hz.STATUS[ctx.status()] == "TIMEOUT"
    assert ctx.status() == 0  # read and cleared
    # the same context keeps working, with the oracle's results
    assert np.array_equal(hz.negate(c, ctx=ctx).cpu().numpy(), O.negate(oc))
    assert np.array_equal(hz.mul_scalar(c, 2.5, ctx=ctx).cpu().numpy(), O.mul_scalar(oc, 2.5))
    m = hz.mean(c, ctx=ctx)
    assert abs(m - O.mean(oc)) <= 1e-12 * abs(O.mean(oc))
    # limits outside the documented range are argument errors, launched nothing
    assert L.hoszp_selftest_wait(ctx.handle, which, 0, stream) == -1
    assert L.hoszp_selftest_wait(ctx.handle, 2, 1, stream) == -1
