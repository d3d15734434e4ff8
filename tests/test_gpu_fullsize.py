"""The benchmark's full-size workload, in the benchmark's launch configuration
(default context, the same calls and arguments as bench.py's step): two
512^3 Gaussian random fields, relative bound 1e-4, B at A's absolute bound.
Every produced stream is compared with the oracle's byte for byte, the
decompressed field value for value, and mean and
variance against the oracle's exact integer sums (within 1e-12)."""
import numpy as np
import pytest

import datagen
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SHAPE = (512, 512, 512)


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build

    build.build()
    O.build()
    return hz


@pytest.fixture(scope="module")
def work(hz):
    A = datagen.grf(SHAPE, seed=1).reshape(-1)
    B = datagen.grf(SHAPE, seed=2).reshape(-1)
    ctx = hz.Context(0)
    xa, xb = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ca = hz.compress(xa, eb=1e-4, mode="rel", dims=SHAPE, ctx=ctx)
    e = hz.header(ca)["eps_q"]
    cb = hz.compress(xb, eb=e, dims=SHAPE, ctx=ctx)
    oa = O.compress(A, dims=SHAPE, eb=1e-4, mode="rel")
    ob = O.compress(B, dims=SHAPE, eb=float(e))
    return dict(A=A, ctx=ctx, ca=ca, cb=cb, oa=oa, ob=ob)


def host(t):
    return t.cpu().numpy()


def test_compress_full_size(hz, work):
    assert np.array_equal(host(work["ca"]), work["oa"])
    assert np.array_equal(host(work["cb"]), work["ob"])


def test_metadata_operators_full_size(hz, work):
    ctx, ca, oa = work["ctx"], work["ca"], work["oa"]
    assert np.array_equal(host(hz.negate(ca, ctx=ctx)), O.negate(oa))
    assert np.array_equal(host(hz.add_scalar(ca, 0.5, ctx=ctx)), O.add_scalar(oa, 0.5))


def test_mul_and_add_full_size(hz, work):
    ctx, ca, cb, oa, ob = work["ctx"], work["ca"], work["cb"], work["oa"], work["ob"]
    assert np.array_equal(host(hz.mul_scalar(ca, 3.14, ctx=ctx)), O.mul_scalar(oa, 3.14))
    assert np.array_equal(host(hz.add(ca, cb, ctx=ctx)), O.add(oa, ob))


def test_decompress_full_size(hz, work):
    x = host(hz.decompress(work["ca"], ctx=work["ctx"]))
    n = x.size
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([rng.integers(0, n, 1 << 20), [0, 63, 64, n - 65, n - 1]]))
    q = O.decode_q(work["oa"])
    e = O.header(work["oa"])["eps_q"]
    want = np.array([O.dequantize(int(q[i]), e) for i in idx[:20000]], dtype=np.float32)
    assert np.array_equal(x[idx[:20000]], want)
    # every value against the oracle's full decompression
    ref = O.decompress(work["oa"])
    assert np.array_equal(x, ref)
    # the error bound of Eq. 3 holds on the sample
    A = work["A"]
    assert np.all(np.abs(A[idx].astype(np.float64) - x[idx]) <= float(e) * (1 + 2.0 ** -20)
                  + np.spacing(np.abs(x[idx])))


def test_mean_var_full_size(hz, work):
    ctx, ca, oa = work["ctx"], work["ca"], work["oa"]
    m, v = hz.mean(ca, ctx=ctx), hz.var(ca, ctx=ctx)
    om, ov = O.mean(oa), O.var(oa)
    assert abs(m - om) <= 1e-12 * max(abs(om), 1e-300)
    assert abs(v - ov) <= 1e-12 * abs(ov)
