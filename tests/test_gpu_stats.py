"""Scalar subtraction, standard deviation, block-wise means, covariance,
multiplication by the scalar itself and the Hadamard product (Sec. V-A, V-B,
V-C, V-D) on the CUDA path against the oracle, through the C ABI.

Bit-exact: produced streams and block-wise means (exact block sums, the same
two FP64 operations). Within 1e-12 relative: standard deviation and
covariance (exact integer sums, FP64 finish)."""
import numpy as np
import pytest

import datagen
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL_TOL = 1e-12


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build

    build.build()
    O.build()
    return hz


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def close(a, b, tol=REL_TOL):
    return abs(a - b) <= tol * max(abs(b), 1e-300)


CASES = datagen.small_cases()


@pytest.mark.parametrize("name", list(CASES.keys()))
@pytest.mark.parametrize("eb,mode", [(1e-2, "rel"), (1e-4, "rel"), (0.05, "abs")])
def test_small_cases(hz, name, eb, mode):
    x = CASES[name]
    c = hz.compress(dev(x), eb=eb, mode=mode, dims=(x.size,))
    oc = O.compress(x, dims=(x.size,), eb=eb, mode=mode)
    assert np.array_equal(host(c), oc)
    for s in (0.5, -3.25, 0.0):
        assert np.array_equal(host(hz.sub_scalar(c, s)), O.sub_scalar(oc, s)), s
    assert np.array_equal(host(hz.block_means(c)), O.block_means(oc))
    # negated input: sign bits set at zero magnitudes (position 0, tail, zeros)
    assert np.array_equal(host(hz.block_means(hz.negate(c))), O.block_means(O.negate(oc)))
    if x.size > 0:
        assert close(hz.std(c), O.std(oc))
        assert close(hz.var(hz.negate(c)), O.var(oc))


@pytest.mark.parametrize("shape", [(64, 48, 37), (100, 50, 50), (449, 45, 23)])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_grf_shapes(hz, shape, rel):
    x = datagen.grf(shape, seed=11).reshape(-1)
    c = hz.compress(dev(x), eb=rel, mode="rel", dims=shape)
    oc = O.compress(x, dims=shape, eb=rel, mode="rel")
    assert np.array_equal(host(c), oc)
    assert np.array_equal(host(hz.block_means(c)), O.block_means(oc))
    assert np.array_equal(host(hz.sub_scalar(c, 0.25)), O.sub_scalar(oc, 0.25))
    assert close(hz.std(c), O.std(oc))


def test_sub_scalar_inplace_and_errors(hz):
    x = datagen.sines_1d(40_000, seed=3)
    c = hz.compress(dev(x), eb=1e-3, mode="rel")
    oc = host(c)
    w = c.clone()
    hz.sub_scalar(w, 1.5, inplace=True)
    assert np.array_equal(host(w), O.sub_scalar(oc, 1.5))
    hz.add_scalar(w, 1.5, inplace=True)
    assert np.array_equal(np.delete(host(w), range(56, 60)), np.delete(oc, range(56, 60)))
    big = hz.compress(dev(np.full(64, 8e5, np.float32)), eb=0.1)
    with pytest.raises(hz.HoszpError) as ex:
        hz.sub_scalar(big, 1e9)
    assert ex.value.name in ("RANGE", "OVERFLOW")


def test_widest_rates(hz):
    # deltas near 2^31 (rates up to 31): decode, variance, std, block means
    n = 64 * 37 + 11
    x = np.where(np.arange(n) % 2 == 0, 4194304.0, -4194304.0).astype(np.float32)
    x[200:400] = 7.0
    c = hz.compress(dev(x), eb=0.5)
    m = hz.mul_scalar(c, 120.0)
    z = hz.add(m, m)
    om = O.mul_scalar(O.compress(x, eb=0.5), 120.0)
    oz = O.add(om, om)
    assert np.array_equal(host(z), oz)
    for t, o in ((m, om), (z, oz), (hz.negate(z), O.negate(oz))):
        assert np.array_equal(host(hz.decompress(t)), O.decompress(o))
        assert np.array_equal(host(hz.block_means(t)), O.block_means(o))
        assert close(hz.var(t), O.var(o))
        assert close(hz.std(t), O.std(o))
        assert close(hz.mean(t), O.mean(o))


def test_mixed_rates_every_width(hz):
    # blocks of every rate 0..31 side by side in one warp's 16 blocks
    rng = np.random.default_rng(5)
    n = 64 * 512 + 17
    q = np.zeros(n, np.int64)
    for b in range((n + 63) // 64):
        r = b % 32
        lo = b * 64
        hi = min(n, lo + 64)
        if r == 0:
            q[lo:hi] = rng.integers(-1000, 1000)
            continue
        d = rng.integers(-(1 << (r - 1)), 1 << (r - 1), hi - lo)
        d[0] = rng.integers(-(1 << 20), 1 << 20)
        q[lo:hi] = np.cumsum(d)
    q = np.clip(q, -(1 << 22), 1 << 22)
    x = (q.astype(np.float64) * 2 * 0.5).astype(np.float32)  # eps = 0.5: bins of width 1
    c = hz.compress(dev(x), eb=0.5)
    oc = O.compress(x, eb=0.5)
    assert np.array_equal(host(c), oc)
    for t, o in ((c, oc), (hz.mul_scalar(c, 50.0), O.mul_scalar(oc, 50.0))):
        assert np.array_equal(host(t), o)
        assert np.array_equal(host(hz.decompress(t)), O.decompress(o))
        assert np.array_equal(host(hz.block_means(t)), O.block_means(o))
        assert close(hz.var(t), O.var(o))
        assert close(hz.std(t), O.std(o))


@pytest.mark.parametrize("name", [k for k in CASES.keys() if CASES[k].size > 0])
def test_cov_small_cases(hz, name):
    x = CASES[name]
    y = (x[::-1].copy() * np.float32(-0.75) + np.float32(0.125)).astype(np.float32)
    for eb_a, eb_b in ((0.05, 0.05), (0.05, 0.013)):  # equal and different bounds
        c = hz.compress(dev(x), eb=eb_a, dims=(x.size,))
        d = hz.compress(dev(y), eb=eb_b, dims=(y.size,))
        oc, od = host(c), host(d)
        assert np.array_equal(oc, O.compress(x, dims=(x.size,), eb=eb_a))
        assert np.array_equal(od, O.compress(y, dims=(y.size,), eb=eb_b))
        assert close(hz.cov(c, d), O.cov(oc, od))
        assert close(hz.cov(d, c), O.cov(od, oc))
        assert close(hz.cov(hz.negate(c), d), O.cov(O.negate(oc), od))
    assert hz.cov(c, c) == hz.var(c)  # S_AA = S2 exactly, then the same FP64 steps


@pytest.mark.parametrize("shape", [(64, 48, 37), (449, 45, 23), (256, 256, 128)])
def test_cov_grf_pairs(hz, shape):
    # (256, 256, 128): 512 super-tiles, several per CTA range
    x = datagen.grf(shape, seed=21).reshape(-1)
    y = datagen.grf(shape, seed=22).reshape(-1)
    y = (0.6 * x + 0.8 * y).astype(np.float32)  # correlated
    c = hz.compress(dev(x), eb=1e-4, mode="rel", dims=shape)
    e = float(O.header(host(c))["eps_q"])
    d = hz.compress(dev(y), eb=e, dims=shape)  # the same bound
    oc, od = host(c), host(d)
    assert np.array_equal(od, O.compress(y, dims=shape, eb=e))
    assert close(hz.cov(c, d), O.cov(oc, od))
    m = hz.mul_scalar(d, 7.5)
    assert close(hz.cov(c, m), O.cov(oc, O.mul_scalar(od, 7.5)))
    f = hz.compress(dev(y), eb=1e-3, mode="rel", dims=shape)  # another bound
    assert close(hz.cov(c, f), O.cov(oc, host(f)))


def test_cov_wide_rates_and_errors(hz):
    n = 64 * 37 + 11
    x = np.where(np.arange(n) % 2 == 0, 4194304.0, -4194304.0).astype(np.float32)
    x[200:400] = 7.0
    c = hz.compress(dev(x), eb=0.5)
    m = hz.mul_scalar(c, 120.0)  # rates near 30, qbound about 5e8
    y = (1000.0 * np.sin(0.013 * np.arange(n)) + 0.5 * np.cos(0.7 * np.arange(n))).astype(np.float32)
    d = hz.compress(dev(y), eb=0.5)
    om, od = host(m), host(d)
    assert close(hz.cov(m, d), O.cov(om, od))
    assert close(hz.cov(m, hz.negate(m)), O.cov(om, O.negate(om)))
    z = hz.add(m, m)  # the widest rates: deltas near 2^31
    oz = host(z)
    assert close(hz.cov(z, d), O.cov(oz, od))
    assert close(hz.cov(m, z), O.cov(om, oz))
    assert close(hz.cov(z, hz.negate(z)), O.cov(oz, O.negate(oz)))
    g = hz.compress(dev(x), eb=1.0)  # another bound
    assert close(hz.cov(c, g), O.cov(host(c), host(g)))
    with pytest.raises(hz.HoszpError) as ex:  # different lengths
        hz.cov(c, hz.compress(dev(np.ones(n + 1, np.float32)), eb=0.5))
    assert ex.value.name == "MISMATCH"


@pytest.mark.parametrize("name", list(CASES.keys()))
def test_mul_scalar_exact_small_cases(hz, name):
    x = CASES[name]
    c = hz.compress(dev(x), eb=0.05, dims=(x.size,))
    oc = host(c)
    for s in (3.14, -0.37, 2.5, 1e-3, 1.0, -1.0, 0.0):
        assert np.array_equal(host(hz.mul_scalar_exact(c, s)), O.mul_scalar_exact(oc, s)), s
    assert np.array_equal(host(hz.mul_scalar_exact(c, 1.0)), oc)  # identity, byte for byte


def test_mul_scalar_exact_grf_and_wide(hz):
    shape = (449, 45, 23)
    x = datagen.grf(shape, seed=31).reshape(-1)
    c = hz.compress(dev(x), eb=1e-4, mode="rel", dims=shape)
    oc = host(c)
    for s in (3.14, -123.456, 7e-4):
        assert np.array_equal(host(hz.mul_scalar_exact(c, s)), O.mul_scalar_exact(oc, s)), s
    n = 64 * 37 + 11  # deltas near 2^31 after the product
    w = np.where(np.arange(n) % 2 == 0, 4194304.0, -4194304.0).astype(np.float32)
    cw = hz.compress(dev(w), eb=0.5)
    ow = host(cw)
    for s in (120.0, -127.9, 0.999):
        assert np.array_equal(host(hz.mul_scalar_exact(cw, s)), O.mul_scalar_exact(ow, s)), s
    with pytest.raises(hz.HoszpError) as ex:
        hz.mul_scalar_exact(cw, 1000.0)
    assert ex.value.name == "OVERFLOW"


@pytest.mark.parametrize("name", list(CASES.keys()))
def test_hadamard_small_cases(hz, name):
    x = CASES[name]
    y = (x[::-1].copy() * np.float32(-0.75) + np.float32(0.125)).astype(np.float32)
    c = hz.compress(dev(x), eb=0.05, dims=(x.size,))
    d = hz.compress(dev(y), eb=0.05, dims=(y.size,))
    oc, od = host(c), host(d)
    assert np.array_equal(host(hz.hadamard(c, d)), O.hadamard(oc, od))
    assert np.array_equal(host(hz.hadamard(hz.negate(c), d)), O.hadamard(O.negate(oc), od))


def test_hadamard_grf_constant_and_errors(hz):
    shape = (449, 45, 23)
    x = datagen.grf(shape, seed=41).reshape(-1)
    y = datagen.grf(shape, seed=42).reshape(-1)
    c = hz.compress(dev(x), eb=1e-3, mode="rel", dims=shape)
    e = float(O.header(host(c))["eps_q"])
    d = hz.compress(dev(y), eb=e, dims=shape)
    oc, od = host(c), host(d)
    z = hz.hadamard(c, d)
    assert np.array_equal(host(z), O.hadamard(oc, od))
    # a constant field s: the scalar multiplication by s, byte for byte
    s = np.float32(3.14)
    k = hz.compress(dev(np.full(x.size, s, np.float32)), eb=e, dims=shape)
    assert np.array_equal(host(hz.hadamard(c, k)), host(hz.mul_scalar(c, float(s))))
    # large products: q_A up to 2^22, q_B up to 100
    n = 64 * 37 + 11
    w = np.where(np.arange(n) % 2 == 0, 4194304.0, -4194304.0).astype(np.float32)
    v = (100.0 * np.sin(0.05 * np.arange(n))).astype(np.float32)
    cw, cv = hz.compress(dev(w), eb=0.5), hz.compress(dev(v), eb=0.5)
    assert np.array_equal(host(hz.hadamard(cw, cv)), O.hadamard(host(cw), host(cv)))
    with pytest.raises(hz.HoszpError) as ex:
        hz.hadamard(cw, cw)  # 2^44: beyond the integer range
    assert ex.value.name == "OVERFLOW"
    with pytest.raises(hz.HoszpError) as ex:
        hz.hadamard(c, hz.compress(dev(y), eb=2 * e, dims=shape))
    assert ex.value.name == "MISMATCH"
