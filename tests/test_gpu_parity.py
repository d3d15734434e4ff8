"""CUDA path against the oracle, element by element, through the C ABI.

Bit-exact: compressed bytes, decoded floats, every produced stream.
Within 1e-12 relative: mean and variance (exact integer sums, FP64 finish).
"""
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
def test_codec_and_ops_small(hz, name, eb, mode):
    x = CASES[name]
    c = hz.compress(dev(x), eb=eb, mode=mode, dims=(x.size,))
    oc = O.compress(x, dims=(x.size,), eb=eb, mode=mode)
    assert np.array_equal(host(c), oc)
    assert np.array_equal(host(hz.decompress(c)), O.decompress(oc))
    assert np.array_equal(host(hz.negate(c)), O.negate(oc))
    assert np.array_equal(host(hz.add_scalar(c, 0.5)), O.add_scalar(oc, 0.5))
    for s in (3.14, -0.37, 1e-3):
        assert np.array_equal(host(hz.mul_scalar(c, s)), O.mul_scalar(oc, s)), s
    y = (x[::-1].copy() * np.float32(0.5)).astype(np.float32)
    e = float(O.header(oc)["eps_q"])
    cy = hz.compress(dev(y), eb=e, dims=(y.size,))
    ocy = O.compress(y, dims=(y.size,), eb=e)
    assert np.array_equal(host(cy), ocy)
    assert np.array_equal(host(hz.add(c, cy)), O.add(oc, ocy))
    assert np.array_equal(host(hz.sub(c, cy)), O.sub(oc, ocy))
    # negated input: sign bits set at zero magnitudes (position 0, tail, zeros)
    assert np.array_equal(host(hz.add(hz.negate(c), cy)), O.add(O.negate(oc), ocy))
    assert np.array_equal(host(hz.sub(cy, hz.negate(c))), O.sub(ocy, O.negate(oc)))
    if x.size > 0:
        assert close(hz.mean(c), O.mean(oc))
        assert close(hz.var(c), O.var(oc))


@pytest.fixture(scope="module")
def config1(hz):
    x = datagen.sines_1d(1 << 20, seed=0)
    c = hz.compress(dev(x), eb=1e-3, mode="rel")
    oc = O.compress(x, eb=1e-3, mode="rel")
    return x, c, oc


def test_config1_sines_2p20(hz, config1):
    x, c, oc = config1
    assert np.array_equal(host(c), oc)
    assert np.array_equal(host(hz.decompress(c)), O.decompress(oc))
    assert np.array_equal(host(hz.negate(c)), O.negate(oc))
    assert np.array_equal(host(hz.add_scalar(c, 0.5)), O.add_scalar(oc, 0.5))
    assert np.array_equal(host(hz.mul_scalar(c, 2.5)), O.mul_scalar(oc, 2.5))
    assert close(hz.mean(c), O.mean(oc))
    assert close(hz.var(c), O.var(oc))


def test_inplace_negate_and_add_scalar(hz, config1):
    _, c, oc = config1
    w = c.clone()
    hz.negate(w, inplace=True)
    assert np.array_equal(host(w), O.negate(oc))
    hz.add_scalar(w, -1.25, inplace=True)
    assert np.array_equal(host(w), O.add_scalar(O.negate(oc), -1.25))


def test_add_sub_widest_rates(hz):
    # deltas near 2^31: alternating +-2^22 bins scaled by 120 (q' ~ 5e8), then
    # summed with itself (qbound 1.007e9 <= HOSZP_QLIM): rates up to 31
    n = 64 * 37 + 11
    x = np.where(np.arange(n) % 2 == 0, 4194304.0, -4194304.0).astype(np.float32)
    x[200:400] = 7.0  # a few constant blocks in between
    c, oc = hz.compress(dev(x), eb=0.5), O.compress(x, eb=0.5)
    assert np.array_equal(host(c), oc)
    m, om = hz.mul_scalar(c, 120.0), O.mul_scalar(oc, 120.0)
    assert np.array_equal(host(m), om)
    z, oz = hz.add(m, m), O.add(om, om)
    assert np.array_equal(host(z), oz)
    assert int(O.header(oz)["qbound"]) > (1 << 29)
    assert np.array_equal(host(hz.sub(m, hz.negate(m))), oz)
    assert np.array_equal(host(hz.sub(m, m)), O.sub(om, om))


def test_theorem1_add_negate_is_zero(hz, config1):
    _, c, _ = config1
    z = hz.add(c, hz.negate(c))
    h = hz.header(z)
    assert h["nnc"] == 0 and h["R"] == 0
    assert not host(hz.decompress(z)).any()


@pytest.mark.parametrize("shape,rel", [((64, 80, 91), 1e-3), ((33, 47, 29), 1e-5),
                                        ((100, 500, 50), 1e-4)])
def test_grf_3d(hz, shape, rel):
    x = datagen.grf(shape, seed=5)
    y = datagen.grf(shape, seed=6)
    c = hz.compress(dev(x), eb=rel, mode="rel")
    oc = O.compress(x, eb=rel, mode="rel")
    assert np.array_equal(host(c), oc)
    e = float(O.header(oc)["eps_q"])
    cy, ocy = hz.compress(dev(y), eb=e), O.compress(y, eb=e)
    assert np.array_equal(host(cy), ocy)
    assert np.array_equal(host(hz.add(c, cy)), O.add(oc, ocy))
    assert np.array_equal(host(hz.sub(c, cy)), O.sub(oc, ocy))
    assert np.array_equal(host(hz.decompress(c)), O.decompress(oc))
    assert np.array_equal(host(hz.mul_scalar(c, -1.5)), O.mul_scalar(oc, -1.5))
    assert close(hz.mean(c), O.mean(oc)) and close(hz.var(c), O.var(oc))


def test_land_mask_fill_values(hz):
    x = datagen.lat_bands_2d(180, 360, seed=3)
    for rel in (1e-2, 1e-4, 1e-6):
        c = hz.compress(dev(x), eb=rel, mode="rel")
        oc = O.compress(x, eb=rel, mode="rel")
        assert np.array_equal(host(c), oc)
        assert np.array_equal(host(hz.mul_scalar(c, 0.75)), O.mul_scalar(oc, 0.75))
        assert close(hz.mean(c), O.mean(oc)) and close(hz.var(c), O.var(oc))


def test_wide_rates_and_quantizer_edges(hz):
    rng = np.random.default_rng(7)
    e = np.float32(0.5)
    # exact bin edges, their neighbours, values near the quantizer's range limit
    k = rng.integers(-4_000_000, 4_000_000, 20_000)
    edges = ((2 * k - 1) * 0.5).astype(np.float32)
    x = np.concatenate([edges, np.nextafter(edges, np.float32(np.inf)),
                        np.nextafter(edges, np.float32(-np.inf)),
                        rng.uniform(-8.3e6, 8.3e6, 30_000).astype(np.float32),
                        np.float32([8388606.0, -8388606.0, 8388605.4])]).astype(np.float32)
    c = hz.compress(dev(x), eb=float(e))
    oc = O.compress(x, eb=float(e))
    assert np.array_equal(host(c), oc)
    assert O.header(oc)["R"] > 0
    assert np.array_equal(host(hz.decompress(c)), O.decompress(oc))
    # 8388606.5 / (2 * 0.5) rounds to 8388607 = HOSZP_QMAX_COMPRESS + 1
    over = np.float32([1.0, 8388606.5])
    with pytest.raises(O.OracleError) as eo:
        O.compress(over, eb=0.5)
    assert eo.value.name == "RANGE"
    with pytest.raises(hz.HoszpError) as eg:
        hz.compress(dev(over), eb=0.5)
    assert eg.value.name == "RANGE"


def test_errors_reported(hz):
    HE = hz.HoszpError
    with pytest.raises(HE) as ex:
        hz.compress(dev(np.array([1.0, np.nan] * 100, np.float32)), eb=0.1)
    assert ex.value.name == "NONFINITE"
    with pytest.raises(HE) as ex:
        hz.compress(dev(np.array([1.0, np.inf] * 100, np.float32)), eb=0.1, mode="rel")
    assert ex.value.name == "NONFINITE"
    with pytest.raises(HE) as ex:
        hz.compress(dev(np.full(100, 1e10, np.float32)), eb=1e-3)
    assert ex.value.name == "RANGE"
    with pytest.raises(HE) as ex:
        hz.compress(dev(np.ones(10, np.float32)), eb=-1.0)
    assert ex.value.name == "ARG"
    x = np.ones(1000, np.float32)
    c = hz.compress(dev(x), eb=0.1)
    bad = c.clone()
    bad[0] ^= 1
    with pytest.raises(HE) as ex:
        hz.decompress(bad, n=1000)
    assert ex.value.name == "FORMAT"
    with pytest.raises(HE) as ex:
        hz.add(c, hz.compress(dev(x), eb=0.2))
    assert ex.value.name == "MISMATCH"
    with pytest.raises(HE) as ex:
        hz.mean(hz.compress(dev(np.zeros(0, np.float32)), eb=0.1, dims=(0,)))
    assert ex.value.name == "ARG"
    big = hz.compress(dev(np.full(64, 8e5, np.float32)), eb=0.1)
    with pytest.raises(HE) as ex:
        hz.mul_scalar(big, 1000.0)
    assert ex.value.name == "OVERFLOW"
    with pytest.raises(HE) as ex:
        hz.add_scalar(big, 1e9)
    assert ex.value.name in ("RANGE", "OVERFLOW")
    # a stream whose rate section disagrees with its header
    c2 = hz.compress(dev(datagen.sines_1d(5000, seed=1)), eb=1e-3)
    corrupt = c2.clone()
    corrupt[64] = (int(corrupt[64]) + 1) % 20 + 1
    with pytest.raises(HE) as ex:
        hz.mean(corrupt)
    assert ex.value.name == "FORMAT"
    # too small an output buffer
    xs = dev(datagen.sines_1d(50_000, seed=2))
    small = torch.empty(2_000, dtype=torch.uint8, device="cuda")
    with pytest.raises(HE) as ex:
        hz.compress(xs, eb=1e-4, mode="rel", out=small)
    assert ex.value.name == "CAPACITY"
    # the context stays usable after errors
    assert np.array_equal(host(hz.compress(dev(x), eb=0.1)), O.compress(x, eb=0.1))


def test_repeated_calls_are_deterministic(hz, config1):
    x, c, oc = config1
    for _ in range(3):
        assert np.array_equal(host(hz.compress(dev(x), eb=1e-3, mode="rel")), oc)
        assert close(hz.var(c), O.var(oc))


def test_sums_words_and_sharded_finish(hz, config1):
    """hoszp_sums gives the oracle's exact sums; finishing them with
    hoszp_finish_sums (the multi-rank path) gives the kernels' mean and variance
    bit for bit, also for the sums of two shards of whole blocks."""
    from paper_2408_11971_gb300 import sharded

    x, c, oc = config1
    s = sharded.from_words(hz.sums(c))
    s1, s2, n, e = O.sums(oc)
    assert (s.s1, s.s2, s.n) == (s1, s2, n)
    eq = float(hz.header(c)["eps_q"])
    m, v = sharded.finish(s, eq)
    assert m == hz.mean(c) and v == hz.var(c)
    cut = 64 * 5000
    p = [hz.compress(dev(x[:cut]), eb=eq), hz.compress(dev(x[cut:]), eb=eq)]
    t = sharded.from_words(hz.sums(p[0])) + sharded.from_words(hz.sums(p[1]))
    assert (t.s1, t.s2, t.n) == (s1, s2, n)
    assert sharded.finish(t, eq) == (hz.mean(c), hz.var(c))
    # the finish's own edge: no values
    with pytest.raises(RuntimeError, match="ARG"):
        hz.finish_sums([0, 0, 0, 0, 0], eq)


@pytest.mark.parametrize("eb,mode", [(0.1, "abs"), (1e-3, "rel"), (1e-5, "rel")])
def test_mul_scalar_every_requantization_width(hz, eb, mode):
    """Scalars from below the bin width to 1e5: the 32-bit, 64-bit and 128-bit
    requantizations (picked from the header's bound of |q| and the scalar's
    bin), rates growing by up to 17 bits, a tail of 43 values."""
    x = datagen.grf((47_147,), seed=5)
    c = hz.compress(dev(x), eb=eb, mode=mode)
    oc = O.compress(x, eb=eb, mode=mode)
    assert np.array_equal(host(c), oc)
    for s in (3.14, -2.5, 0.3, 1e-7, 123.456, -7.5e3, 1e5):
        for gpu_op, orc_op in ((hz.mul_scalar, O.mul_scalar),
                               (hz.mul_scalar_exact, O.mul_scalar_exact)):
            try:
                want = orc_op(oc, s)
            except O.OracleError as ex:
                with pytest.raises(RuntimeError, match=ex.name):
                    gpu_op(c, s)
                continue
            assert np.array_equal(host(gpu_op(c, s)), want), (s, orc_op.__name__)


def test_concat_shards_into_the_field_stream(hz):
    """hoszp_concat joins the GPU streams of consecutive shards into the stream
    of the whole field, byte for byte the oracle's (Sec. VI-B5), for 1-D and
    3-D shapes, shards of one block, a ragged last shard and a single shard;
    and refuses what is not one field."""
    g = datagen.grf((20, 48, 63), seed=12)  # 60480 values: 945 blocks
    x = g.reshape(-1)
    eps = float(O.header(O.compress(x, eb=1e-4, mode="rel"))["eps_q"])
    whole = O.compress(g, eb=eps)
    for cuts in ([0, 64 * 400, x.size], [0, 64, 128, 64 * 900, x.size], [0, x.size],
                 [0, 64 * 100, 64 * 200, 64 * 300, 64 * 940, x.size]):
        parts = [hz.compress(dev(x[a:b]), eb=eps) for a, b in zip(cuts, cuts[1:])]
        assert np.array_equal(host(hz.concat(parts, g.shape)), whole), cuts
    a = hz.compress(dev(x[:64 * 10]), eb=eps)
    with pytest.raises(RuntimeError, match="MISMATCH"):  # another bound
        hz.concat([a, hz.compress(dev(x[64 * 10:]), eb=2 * eps)], (x.size,))
    with pytest.raises(RuntimeError, match="MISMATCH"):  # a ragged shard before the last
        hz.concat([hz.compress(dev(x[:100]), eb=eps), hz.compress(dev(x[100:]), eb=eps)],
                  (x.size,))
    with pytest.raises(RuntimeError, match="ARG"):  # the shape disagrees with the values
        hz.concat([a, hz.compress(dev(x[64 * 10:]), eb=eps)], (x.size + 1,))
    bad = a.clone()
    bad[0] ^= 1  # magic
    with pytest.raises(RuntimeError, match="FORMAT"):
        hz.concat([bad, a], (64 * 20,))
    b = hz.compress(dev(x[64 * 10:]), eb=eps)
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="CAPACITY"):
        hz.concat([a, b], (x.size,), out=small)


@pytest.mark.parametrize("kind", ["sines", "grf", "mask", "const"])
def test_compress_output_sizes(hz, kind):
    """Compression into the library's bound and into a buffer of exactly the
    stream's size gives the oracle's bytes (constant runs, no constant block,
    land mask, a constant field); one 16-byte unit less is CAPACITY."""
    if kind == "sines":
        x = datagen.sines_1d(300_017, seed=17)  # about 20 % constant runs
    elif kind == "grf":
        x = datagen.grf((24, 48, 50), seed=18).reshape(-1)  # no constant block
    elif kind == "mask":
        x = datagen.lat_bands_2d(180, 360, seed=19).reshape(-1)
    else:
        x = np.full(70_001, np.float32(2.5), np.float32)
    want = O.compress(x, eb=1e-4, mode="rel")
    assert np.array_equal(host(hz.compress(dev(x), eb=1e-4, mode="rel")), want)
    exact = torch.empty(want.size, dtype=torch.uint8, device="cuda")
    got = hz.compress(dev(x), eb=1e-4, mode="rel", out=exact)
    assert np.array_equal(host(got), want)
    small = torch.empty(want.size - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(RuntimeError, match="CAPACITY"):
        hz.compress(dev(x), eb=1e-4, mode="rel", out=small)
