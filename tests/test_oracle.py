"""The oracle against what the paper and mathematics fix (no GPU).

Pins: the paper's printed worked examples (tests/golden/paper_examples.json),
exact rational arithmetic for Eq. 3 and the operators, brute force on small
inputs, the error-bound invariant, the constant-block and bit-width rules,
Theorem 1 identities, and the textbook mean/variance.
"""
import json
import math
import os
import statistics
from fractions import Fraction

import numpy as np
import pytest

import datagen
import oracle as O
from streamfmt import parse, values, block_deltas

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_examples.json")))
L = 64


def bin_search_q(x, e):
    """Brute force: the integer k whose bin [(2k-1)e, (2k+1)e) holds x (exact)."""
    X, E = Fraction(float(x)), Fraction(float(e))
    k = int(X / (2 * E))  # start near, then walk
    while not ((2 * k - 1) * E <= X):
        k -= 1
    while not (X < (2 * k + 1) * E):
        k += 1
    return k


def eq3_fraction(x, e):
    X, E = Fraction(float(x)), Fraction(float(e))
    return math.floor((X + E) / (2 * E))


# ---------------------------------------------------------------- paper examples
def test_worked_example_quantize_lorenzo_signs():
    g = GOLD["quantize_lorenzo"]
    x = np.array(g["A1"], np.float32)
    c = O.compress(x, dims=(2, 2), eb=g["eps_inferred"])
    s = parse(c)
    assert list(values(s)) == g["q"]
    assert list(O.decode_q(c)) == g["q"]
    assert s["outlier"][0] == g["outlier"]
    d = block_deltas(s)[0, :4]
    assert list(d) == g["P_signed"]
    signs = [int((int(s["sign"][0]) >> i) & 1) for i in range(4)]
    assert signs == g["signs"]
    assert list(np.abs(d)) == g["P_magnitude"]


def test_worked_example_fixed_length():
    g = GOLD["fixed_length"]
    x = np.array(GOLD["quantize_lorenzo"]["A1"], np.float32)
    s = parse(O.compress(x, dims=(4,), eb=0.01))
    assert int(s["rate"][0]) == g["bits_per_value"]
    mags = np.abs(block_deltas(s)[0, :4])
    assert list(mags) == g["P"]
    # the stored planes, repacked element-major (first value in the high bits)
    word = 0
    for m in mags:
        word = (word << g["bits_per_value"]) | int(m)
    assert word == int(g["C_hex"], 16)


def test_worked_example_scalar_multiplication():
    g = GOLD["scalar_multiplication"]
    e = O.eps_q(0.01)
    assert O.quantize_scalar(g["s"], e) == g["rho_s"]
    q = np.array(GOLD["quantize_lorenzo"]["q"])
    assert list(q * g["rho_s"]) == g["q_times_rho"]
    c = O.compress(np.array(GOLD["quantize_lorenzo"]["A1"], np.float32), dims=(2, 2), eb=0.01)
    m = O.mul_scalar(c, g["s"])
    s = parse(m)
    assert list(values(s)) == g["q_after"]
    assert s["outlier"][0] == g["outlier_after"]
    d = block_deltas(s)[0, :4]
    assert list(np.abs(d)) == g["P_magnitude_after"]
    assert [int((int(s["sign"][0]) >> i) & 1) for i in range(4)] == g["signs_after"]


def test_worked_example_scalar_addition_reading():
    g = GOLD["scalar_addition"]
    e = O.eps_q(0.01)
    # Eq. 3 gives 34; the paper prints 33 = floor(s / 2e) (see the golden note)
    rho = O.quantize_scalar(g["s"], e)
    assert rho == eq3_fraction(g["s"], e) == 34
    assert math.floor(Fraction(g["s"]) / Fraction(2, 100)) == g["rho_s_printed"]
    c = O.compress(np.array(GOLD["quantize_lorenzo"]["A1"], np.float32), dims=(2, 2), eb=0.01)
    a = O.add_scalar(c, g["s"])
    s0, s1 = parse(c), parse(a)
    assert s1["outlier"][0] == GOLD["quantize_lorenzo"]["outlier"] + rho
    # predicted values and signs are untouched (proof of Theorem 1)
    assert np.array_equal(s0["sign"], s1["sign"]) and np.array_equal(s0["plane"], s1["plane"])


def test_worked_example_mean():
    g = GOLD["mean"]
    c = O.compress(np.array(GOLD["quantize_lorenzo"]["A1"], np.float32), dims=(2, 2), eb=0.01)
    s1, _, n, e = O.sums(c)
    assert s1 == g["sum"] and n == g["n"]
    assert O.mean(c) == pytest.approx(g["mean"], rel=1e-7)  # eps_q = float32(0.01)


def test_table6_block_length_64():
    g = GOLD["constant_blocks_table6"]
    for k, tb in g["total_blocks"].items():
        assert g["values"][k] == 64 * tb
    x = np.arange(64 * 3 + 5, dtype=np.float32)
    assert parse(O.compress(x, eb=0.5))["nb"] == 4


# ---------------------------------------------------------------- quantizer
def test_eps_q_is_largest_float_not_above_eps():
    rng = np.random.default_rng(5)
    for eps in list(10.0 ** rng.uniform(-30, 30, 300)) + [0.01, 1e-3, 0.1, 1.0, 3.0]:
        f = O.eps_q(eps)
        assert float(f) <= eps
        assert float(np.nextafter(f, np.float32(np.inf))) > eps


@pytest.mark.parametrize("seed", range(4))
def test_quantize_matches_bin_search(seed):
    rng = np.random.default_rng(seed)
    e = np.float32(10.0 ** rng.uniform(-6, 2))
    xs = (rng.standard_normal(300) * float(e) * 10 ** rng.uniform(0, 5)).astype(np.float32)
    # exact bin edges and their float neighbours
    ks = rng.integers(-1000, 1000, 60)
    edges = [np.float32((2 * int(k) - 1) * float(e)) for k in ks]
    xs = np.concatenate([xs, edges, np.nextafter(edges, np.float32(np.inf)),
                         np.nextafter(edges, np.float32(-np.inf)), [0.0, -0.0, e, -e]]
                        ).astype(np.float32)
    for x in xs:
        q = O.quantize(x, e)
        assert q == bin_search_q(x, e) == eq3_fraction(x, e), (x, e)


def test_quantize_power_of_two_edges():
    e = np.float32(0.5)  # bins of width 1 centred on integers, edges at k + 1/2
    for x, q in [(1.5, 2), (-0.5, 0), (2.5, 3), (-1.5, -1), (0.49999997, 0), (-0.50000006, -1)]:
        assert O.quantize(np.float32(x), e) == q


def test_quantize_range_limit():
    e = np.float32(1.0)
    top = 8388606  # the quantizer's range: |q| <= 2^23 - 2
    assert O.quantize(np.float32(2 * top), e) == top
    with pytest.raises(O.OracleError) as ex:
        O.quantize(np.float32(2 * top + 2), e)
    assert ex.value.name == "RANGE"


def nearest_f32(exact: Fraction) -> np.float32:
    """The float32 nearest to a rational, ties to the even significand; found by
    comparing exact distances of the float32 neighbours of a first guess (the
    guess may be one step off after its double rounding)."""
    guess = np.float32(float(exact))
    cands = [guess]
    for _ in range(2):
        cands += [np.nextafter(cands[-1], np.float32(-np.inf))]
    up = guess
    for _ in range(2):
        up = np.nextafter(up, np.float32(np.inf))
        cands.append(up)
    cands = [c for c in cands if np.isfinite(c)]
    dist = [abs(Fraction(float(c)) - exact) for c in cands]
    best = min(dist)
    tied = [c for c, d in zip(cands, dist) if d == best]
    return min(tied, key=lambda c: int(np.array(c).view(np.uint32)) & 1)


def test_dequantize_is_correctly_rounded():
    """Reverse quantization (proof of Theorem 1): 2e*q rounded once to float32,
    over the whole stream range |q| <= 2^30 - 1 that operator outputs reach."""
    rng = np.random.default_rng(9)
    cases = []
    for _ in range(600):
        e = np.float32(10.0 ** rng.uniform(-8, 3))
        top = int(rng.choice([1 << 23, 1 << 25, (1 << 30) - 1]))
        cases.append((int(rng.integers(-top, top + 1)), e))
    # ties at |q| >= 2^24: 2e a power of two and q odd above 2^24, so the
    # product needs 25 significant bits and lies halfway between two floats
    for q in (16777217, 16777219, -16777217, -16777219, (1 << 30) - 1, -((1 << 30) - 1),
              (1 << 25) + 2, (1 << 25) + 6, 33554435):
        cases.append((q, np.float32(0.5)))
        cases.append((q, np.float32(2.0 ** -20)))
    # e whose significand is odd and wide (no power of two), large q
    for q in ((1 << 30) - 1, (1 << 29) + 12345, -(1 << 28) - 7):
        cases.append((q, np.float32(0.1)))
        cases.append((q, np.float32(1e-7)))
    for q, e in cases:
        exact = Fraction(q) * 2 * Fraction(float(e))
        got = O.dequantize(q, e)
        want = nearest_f32(exact)
        assert got == want and np.signbit(got) == np.signbit(want), (q, float(e), got, want)
    # the double rounding of float(q) * 2e is what this must not do: it differs
    # on some of these cases, so the pin does tell the two apart
    twice = sum(np.float32(np.float32(q) * np.float32(2 * e)) != nearest_f32(
        Fraction(q) * 2 * Fraction(float(e))) for q, e in cases)
    assert twice > 0


# ---------------------------------------------------------------- codec
def _check_stream(x, c):
    """Brute-force quantization, decoding by the test's own reader, size formula,
    rate and constant-block rules, error bound."""
    s = parse(c)
    e = s["eps_q"]
    n = x.size
    assert s["magic"] == 0x505A5348 and s["block"] == 64 and s["n"] == n
    raw = 64 + (s["nb"] + 15) // 16 * 16 + (4 * s["nb"] + 15) // 16 * 16 + 8 * s["nnc"] + 8 * s["R"]
    assert s["size"] == len(c) == (raw + 15) // 16 * 16
    assert not c[raw:].any()  # end padding is zero
    idx = np.random.default_rng(1).choice(n, size=min(n, 400), replace=False) if n else []
    qs = values(s)
    for i in idx:
        assert qs[i] == eq3_fraction(x[i], e)
    assert np.array_equal(qs, O.decode_q(c))
    # rate rule: bit length of the largest |delta| in the block; 0 <=> constant block
    qpad = np.concatenate([qs, np.repeat(qs[-1:], (-n) % L)]) if n else qs
    blocks = qpad.reshape(-1, L)
    for b in range(s["nb"]):
        ln = min(L, n - b * L)
        dmax = int(np.max(np.abs(np.diff(blocks[b, :ln])))) if ln > 1 else 0
        assert int(s["rate"][b]) == dmax.bit_length()
        assert (s["rate"][b] == 0) == bool(np.all(blocks[b, :ln] == blocks[b, 0]))
        assert s["outlier"][b] == blocks[b, 0]
    assert s["nnc"] == int(np.count_nonzero(s["rate"])) and s["R"] == int(s["rate"].sum())
    assert s["qbound"] == (int(np.max(np.abs(qs))) if n else 0)
    # error bound: |x - x'| <= eps_q + ulp(x')/2 (Eq. 3 bin, then float rounding)
    xr = O.decompress(c)
    if n:
        err = np.abs(xr.astype(np.float64) - x.astype(np.float64))
        half_ulp = np.spacing(np.abs(xr)).astype(np.float64) / 2
        assert np.all(err <= float(e) + half_ulp)
        assert float(e) <= s["eps"]


@pytest.mark.parametrize("name", list(datagen.small_cases().keys()))
def test_codec_small_cases(name):
    x = datagen.small_cases()[name]
    for eb in (1e-2, 1e-4):
        c = O.compress(x, dims=(x.size,), eb=eb, mode="rel")
        _check_stream(x, c)


def test_codec_abs_modes_and_shapes():
    g = datagen.grf((20, 30, 11), seed=3)
    c = O.compress(g, eb=1e-3)
    s = parse(c)
    assert s["ndims"] == 3 and s["dims"] == [20, 30, 11]
    _check_stream(g.reshape(-1), c)


def test_relative_bound_uses_value_range():
    x = datagen.sines_1d(10_000, seed=4)
    c = O.compress(x, eb=1e-3, mode="rel")
    eps = 1e-3 * (float(x.max()) - float(x.min()))
    assert parse(c)["eps"] == eps
    assert float(parse(c)["eps_q"]) == float(O.eps_q(eps))


def test_constant_runs_give_constant_blocks():
    x = datagen.sines_1d(1 << 16, seed=2, const_frac=0.2)
    s = parse(O.compress(x, eb=1e-3, mode="rel"))
    frac = 1 - s["nnc"] / s["nb"]
    assert 0.12 < frac < 0.3


# ---------------------------------------------------------------- operators (Theorem 1)
@pytest.fixture(scope="module")
def pair():
    a = datagen.sines_1d(30_011, seed=7)
    b = datagen.sines_1d(30_011, seed=8)
    ca = O.compress(a, eb=1e-3)
    cb = O.compress(b, eb=1e-3)
    return ca, cb


def test_negate(pair):
    ca, _ = pair
    ng = O.negate(ca)
    assert np.array_equal(O.decode_q(ng), -O.decode_q(ca))
    assert np.array_equal(O.decompress(ng), -O.decompress(ca))
    assert np.array_equal(O.negate(ng), ca)  # involution, byte for byte
    s0, s1 = parse(ca), parse(ng)
    assert np.array_equal(s1["sign"], ~s0["sign"])  # every sign bit inverted
    assert np.array_equal(s1["plane"], s0["plane"]) and np.array_equal(s1["rate"], s0["rate"])


def test_add_scalar(pair):
    ca, _ = pair
    e = parse(ca)["eps_q"]
    for s in (0.5, -3.25, 0.0, 1e-9):
        out = O.add_scalar(ca, s)
        rho = bin_search_q(s, e)
        assert rho == eq3_fraction(s, e) == O.quantize_scalar(s, e)
        assert np.array_equal(O.decode_q(out), O.decode_q(ca) + rho)
        assert parse(out)["qbound"] == parse(ca)["qbound"] + abs(rho)
        xr = O.decompress(out)
        q = O.decode_q(ca) + rho
        assert np.array_equal(xr, (q.astype(np.float32) * np.float32(2 * e)).astype(np.float32))


def test_mul_scalar(pair):
    ca, _ = pair
    e = parse(ca)["eps_q"]
    q = O.decode_q(ca)
    idx = np.random.default_rng(3).choice(q.size, 300, replace=False)
    for s in (3.14, -0.5, 2.0, 1e-5, 0.0):
        rho = eq3_fraction(s, e)
        out = O.mul_scalar(ca, s)
        q2 = O.decode_q(out)
        for i in idx:  # Eq. 3 applied to (2e q)(2e rho), exactly
            prod = 2 * Fraction(float(e)) * int(q[i]) * rho
            assert q2[i] == math.floor(prod + Fraction(1, 2))
        _check_stream_q(out, q2)


def _check_stream_q(c, q):
    s = parse(c)
    assert np.array_equal(values(s), q)
    assert s["qbound"] == (int(np.max(np.abs(q))) if q.size else 0)


def test_add_fields(pair):
    ca, cb = pair
    z = O.add(ca, cb)
    assert np.array_equal(O.decode_q(z), O.decode_q(ca) + O.decode_q(cb))
    assert parse(z)["qbound"] == parse(ca)["qbound"] + parse(cb)["qbound"]
    # commutative, and A + (-A) is the all-constant zero stream
    assert np.array_equal(O.add(cb, ca), z)
    zero = parse(O.add(ca, O.negate(ca)))
    assert zero["nnc"] == 0 and zero["R"] == 0 and not zero["outlier"].any()
    # the identity of Fig. 7: decompressing the homomorphic sum equals
    # dequantizing the sum of the decompressed fields' bins
    xa, xb = O.decompress(ca), O.decompress(cb)
    e = parse(ca)["eps_q"]
    qa = np.array([eq3_fraction(v, e) for v in xa[:200]])
    assert np.array_equal(qa, O.decode_q(ca)[:200])


def test_sub_fields(pair):
    ca, cb = pair
    z = O.sub(ca, cb)
    qa, qb = values(parse(ca)), values(parse(cb))  # independent parser
    assert np.array_equal(values(parse(z)), qa - qb)
    assert parse(z)["qbound"] == parse(ca)["qbound"] + parse(cb)["qbound"]
    # A - B is A + (-B) byte for byte (both re-encode q_A - q_B canonically)
    assert np.array_equal(z, O.add(ca, O.negate(cb)))
    # anti-commutative at the bin level, and A - A is the all-constant zero stream
    assert np.array_equal(values(parse(O.sub(cb, ca))), qb - qa)
    zero = parse(O.sub(ca, ca))
    assert zero["nnc"] == 0 and zero["R"] == 0 and not zero["outlier"].any()


def test_negate_metadata_equals_reencode_up_to_zero_signs(pair):
    ca, _ = pair
    ng = parse(O.negate(ca))
    x = O.decompress(ca)
    ref = parse(O.compress(-x, eb=float(parse(ca)["eps_q"])))
    assert np.array_equal(ng["rate"], ref["rate"]) and np.array_equal(ng["plane"], ref["plane"])
    assert np.array_equal(ng["outlier"], ref["outlier"])
    # signs agree wherever the magnitude is non-zero
    j = 0
    for b in range(ng["nb"]):
        r = int(ng["rate"][b])
        if r == 0:
            continue
        nz = 0
        base = int(np.sum(ng["rate"][:b]))
        for p in range(r):
            nz |= int(ng["plane"][base + p])
        assert (int(ng["sign"][j]) & nz) == (int(ref["sign"][j]) & nz)
        j += 1


def test_mean_and_variance_textbook(pair):
    ca, _ = pair
    q = [int(v) for v in O.decode_q(ca)]
    e = Fraction(float(parse(ca)["eps_q"]))
    n = len(q)
    mean_exact = Fraction(sum(q), n) * 2 * e
    assert O.mean(ca) == float(mean_exact)
    # the paper's two-pass form: sum (q - mean)^2 / n, then times (2e)^2
    mq = Fraction(sum(q), n)
    var_q = sum((Fraction(v) - mq) ** 2 for v in q) / n
    assert O.var(ca) == float(var_q * 4 * e * e)
    assert statistics.pvariance(q) == pytest.approx(float(var_q), rel=1e-12)
    # and the float64 two-pass variance of the decompressed values, within rounding
    xr = O.decompress(ca).astype(np.float64)
    assert O.var(ca) == pytest.approx(float(np.var(xr)), rel=1e-6)
    assert O.mean(ca) == pytest.approx(float(np.mean(xr)), rel=1e-6, abs=1e-9)


# ---------------------------------------------------------------- errors
def test_errors():
    x = np.ones(100, np.float32)
    with pytest.raises(O.OracleError) as ex:
        O.compress(np.array([1.0, np.nan], np.float32), eb=0.1)
    assert ex.value.name == "NONFINITE"
    with pytest.raises(O.OracleError) as ex:
        O.compress(np.array([1.0, np.inf], np.float32), eb=0.1, mode="rel")
    assert ex.value.name == "NONFINITE"
    with pytest.raises(O.OracleError) as ex:
        O.compress(np.array([1e10], np.float32), eb=1e-3)
    assert ex.value.name == "RANGE"
    with pytest.raises(O.OracleError) as ex:
        O.compress(x, eb=-1.0)
    assert ex.value.name == "ARG"
    c = O.compress(x, eb=0.1)
    bad = c.copy()
    bad[0] ^= 1
    with pytest.raises(O.OracleError) as ex:
        O.decompress(bad)
    assert ex.value.name == "FORMAT"
    with pytest.raises(O.OracleError) as ex:
        O.add(c, O.compress(x, eb=0.2))
    assert ex.value.name == "MISMATCH"
    with pytest.raises(O.OracleError) as ex:
        O.add(c, O.compress(np.ones(101, np.float32), eb=0.1))
    assert ex.value.name == "MISMATCH"
    with pytest.raises(O.OracleError) as ex:
        O.mean(O.compress(np.zeros(0, np.float32), dims=(0,), eb=0.1))
    assert ex.value.name == "ARG"
    big = O.compress(np.full(64, 8e5, np.float32), eb=0.1)  # q = 4e6
    with pytest.raises(O.OracleError) as ex:
        O.mul_scalar(big, 1000.0)
    assert ex.value.name == "OVERFLOW"
    with pytest.raises(O.OracleError) as ex:
        O.add_scalar(big, 1e9)
    assert ex.value.name in ("RANGE", "OVERFLOW")


# ---------------------------------------------------------------- scalar subtraction, std,
# block-wise means, covariance (Sec. V-A, V-B, V-D)
def test_sub_scalar(pair):
    ca, _ = pair
    e = parse(ca)["eps_q"]
    q = values(parse(ca))
    for s in (0.5, -3.25, 0.0, 1e-9, 123.456):
        rho = bin_search_q(s, e)
        assert rho == eq3_fraction(s, e)
        out = O.sub_scalar(ca, s)
        so = parse(out)
        assert np.array_equal(values(so), q - rho)  # O' = O - rho_s, deltas untouched
        assert so["qbound"] == parse(ca)["qbound"] + abs(rho)
        assert np.array_equal(so["sign"], parse(ca)["sign"])
        assert np.array_equal(so["plane"], parse(ca)["plane"])
        # subtracting after adding the same scalar restores every byte but the bound
        back = O.sub_scalar(O.add_scalar(ca, s), s)
        assert np.array_equal(np.delete(back, range(56, 60)), np.delete(ca, range(56, 60)))


def test_sub_scalar_differs_from_adding_the_negated_scalar_only_at_ties():
    # Eq. 3 rounds half up: at s = (2k + 1) eps the bins of s and -s are not opposite
    x = np.array(GOLD["quantize_lorenzo"]["A1"], np.float32)
    c = O.compress(x, dims=(2, 2), eb=0.01)
    e = parse(c)["eps_q"]
    s_tie = float(np.float32(3) * e)  # exactly 3 eps_q
    assert eq3_fraction(s_tie, e) == 2 and eq3_fraction(-s_tie, e) == -1
    assert np.array_equal(values(parse(O.sub_scalar(c, s_tie))), values(parse(c)) - 2)
    assert np.array_equal(values(parse(O.add_scalar(c, -s_tie))), values(parse(c)) - 1)
    s = 0.3  # not a tie: both readings agree
    assert np.array_equal(values(parse(O.sub_scalar(c, s))), values(parse(O.add_scalar(c, -s))))


def test_std():
    e = 0.01
    k = 37
    x = np.where(np.arange(1000) % 2 == 0, 2 * k * e, -2 * k * e).astype(np.float32)
    c = O.compress(x, eb=e)
    q = values(parse(c))
    assert set(q.tolist()) == {k, -k}
    ea = Fraction(float(parse(c)["eps_q"]))
    assert O.std(c) == float(2 * ea * k)  # alternating +-k: std = 2 eps k exactly
    assert O.std(O.compress(np.full(300, 1.5, np.float32), eb=e)) == 0.0
    xs = datagen.sines_1d(20_000, seed=5)
    cs = O.compress(xs, eb=1e-3, mode="rel")
    assert O.std(cs) ** 2 == pytest.approx(O.var(cs), rel=1e-15)
    assert O.std(cs) == pytest.approx(float(np.std(O.decompress(cs).astype(np.float64))), rel=1e-6)


def test_block_means(pair):
    ca, _ = pair
    s = parse(ca)
    q = values(s)
    e2 = 2.0 * float(s["eps_q"])
    bm = O.block_means(ca)
    nb = (q.size + L - 1) // L
    assert bm.shape == (nb,) and nb * L > q.size  # the pair has a ragged last block
    for b in range(nb):
        blk = [int(v) for v in q[b * L:(b + 1) * L]]
        assert bm[b] == (float(sum(blk)) / len(blk)) * e2
    # length-weighted average of the block means is the mean, within rounding
    w = np.array([min(L, q.size - b * L) for b in range(nb)], np.float64)
    assert float(np.sum(bm * w) / q.size) == pytest.approx(O.mean(ca), rel=1e-12)
    # the paper's worked block (Sec. V-B): sum -8 over 4 values, mean -0.04
    g = GOLD["mean"]
    c = O.compress(np.array(GOLD["quantize_lorenzo"]["A1"], np.float32), dims=(2, 2), eb=0.01)
    assert O.block_means(c)[0] == pytest.approx(g["mean"], rel=1e-7)


def test_cov(pair):
    ca, cb = pair
    qa = [int(v) for v in values(parse(ca))]
    qb = [int(v) for v in values(parse(cb))]
    sab, s1a, s1b, n = O.cov_sums(ca, cb)
    assert (sab, s1a, s1b, n) == (sum(a * b for a, b in zip(qa, qb)), sum(qa), sum(qb), len(qa))
    ea = 2 * Fraction(float(parse(ca)["eps_q"]))
    eb = 2 * Fraction(float(parse(cb)["eps_q"]))
    ma, mb = Fraction(sum(qa), n), Fraction(sum(qb), n)
    two_pass = sum((a - ma) * (b - mb) for a, b in zip(qa, qb)) / n
    assert O.cov(ca, cb) == float(ea * eb * two_pass)
    assert O.cov(ca, cb) == O.cov(cb, ca)
    assert O.cov(ca, ca) == O.var(ca)  # covariance with itself is the variance
    assert O.cov(ca, O.negate(ca)) == -O.var(ca)
    xa = O.decompress(ca).astype(np.float64)
    xb = O.decompress(cb).astype(np.float64)
    assert O.cov(ca, cb) == pytest.approx(float(np.cov(xa, xb, bias=True)[0, 1]), rel=1e-6)
    # different error bounds are allowed: each side scales by its own 2 eps
    cc = O.compress(datagen.sines_1d(30_011, seed=8), eb=3e-3)
    qc = [int(v) for v in values(parse(cc))]
    ec = 2 * Fraction(float(parse(cc)["eps_q"]))
    mc = Fraction(sum(qc), n)
    assert O.cov(ca, cc) == float(ea * ec * sum((a - ma) * (c - mc) for a, c in zip(qa, qc)) / n)
    with pytest.raises(O.OracleError) as ex:
        O.cov(ca, O.compress(np.ones(101, np.float32), eb=0.1))
    assert ex.value.name == "MISMATCH"


def test_mul_scalar_exact(pair):
    """q' = floor(q s + 1/2) with s itself (no quantization of the scalar)."""
    ca, _ = pair
    q = values(parse(ca))
    idx = np.random.default_rng(4).choice(q.size, 300, replace=False)
    for s in (3.14, -0.5, 2.0, 1e-5, 0.37, -7.25):
        out = O.mul_scalar_exact(ca, s)
        q2 = values(parse(out))
        for i in idx:  # exact rational rounding, half up
            assert q2[i] == math.floor(Fraction(int(q[i])) * Fraction(s) + Fraction(1, 2))
        _check_stream_q(out, q2)
    # special cases that reduce to known streams
    assert np.array_equal(O.mul_scalar_exact(ca, 1.0), ca)  # identity, byte for byte
    assert np.array_equal(values(parse(O.mul_scalar_exact(ca, 2.0))), 2 * q)
    assert np.array_equal(values(parse(O.mul_scalar_exact(ca, -1.0))), -q)
    assert np.array_equal(values(parse(O.mul_scalar_exact(ca, 0.0))), 0 * q)
    # a scalar below eps does not zero the field (the paper's rho_s would be 0)
    e = float(parse(ca)["eps_q"])
    assert eq3_fraction(e / 4, e) == 0
    small = values(parse(O.mul_scalar_exact(ca, 1000.0 * e)))
    assert np.array_equal(small, [math.floor(Fraction(int(v)) * Fraction(1000.0 * e) + Fraction(1, 2))
                                  for v in q])
    with pytest.raises(O.OracleError) as ex:
        O.mul_scalar_exact(O.compress(np.full(64, 8e5, np.float32), eb=0.1), 1000.0)
    assert ex.value.name == "OVERFLOW"


def test_hadamard(pair):
    """Hadamard product (Sec. V-C): q' = floor(2 eps q_A q_B + 1/2)."""
    ca, _ = pair
    e = float(parse(ca)["eps_q"])
    b = datagen.sines_1d(30_011, seed=9)
    cb = O.compress(b, eb=e)  # the same bound
    qa, qb = values(parse(ca)), values(parse(cb))
    z = O.hadamard(ca, cb)
    qz = values(parse(z))
    idx = np.random.default_rng(6).choice(qa.size, 400, replace=False)
    E2 = 2 * Fraction(e)
    for i in idx:  # Eq. 3 applied to (2e q_A)(2e q_B), exactly
        assert qz[i] == math.floor(E2 * int(qa[i]) * int(qb[i]) + Fraction(1, 2))
    _check_stream_q(z, qz)
    zr = O.hadamard(cb, ca)  # commutative: the same sections (the header takes A's fields)
    assert np.array_equal(zr[64:], z[64:]) and np.array_equal(values(parse(zr)), qz)
    # a constant field s reduces it to the scalar multiplication by s (q_B = rho_s)
    s = 3.14
    cs = O.compress(np.full(qa.size, s, np.float32), eb=e)
    assert set(values(parse(cs)).tolist()) == {eq3_fraction(np.float32(s), e)}
    assert np.array_equal(O.hadamard(ca, cs), O.mul_scalar(ca, float(np.float32(s))))
    with pytest.raises(O.OracleError) as ex:
        O.hadamard(ca, O.compress(b, eb=2 * e))
    assert ex.value.name == "MISMATCH"
    big = O.compress(np.full(64, 8e5, np.float32), eb=0.1)  # q = 4e6: q^2 0.2 = 3.2e12
    with pytest.raises(O.OracleError) as ex:
        O.hadamard(big, big)
    assert ex.value.name == "OVERFLOW"


# ---------------------------------------------------------------- shard streams joined
def test_concat_of_shards_is_the_whole_field_stream():
    """Sec. VI-B5 (the nodes' streams gathered at a root): the streams of
    consecutive shards of whole blocks, compressed with one bound, join into
    exactly the stream of the whole field; the last shard may be ragged."""
    x = datagen.sines_1d(64 * 700 + 37, seed=8)
    eps = 1e-3 * float(x.max() - x.min())
    whole = O.compress(x, eb=eps)
    for cuts in ([0, 64 * 300, x.size], [0, 64, 64 * 2, 64 * 650, x.size], [0, x.size]):
        parts = [O.compress(np.ascontiguousarray(x[a:b]), eb=eps) for a, b in zip(cuts, cuts[1:])]
        assert np.array_equal(O.concat(parts, (x.size,)), whole)
    # a 3-D field split along its slowest axis keeps its shape in the header
    g = datagen.grf((8, 16, 32), seed=2)
    e = 1e-3 * float(g.max() - g.min())
    parts = [O.compress(np.ascontiguousarray(g[:5]).reshape(-1), eb=e),
             O.compress(np.ascontiguousarray(g[5:]).reshape(-1), eb=e)]
    assert np.array_equal(O.concat(parts, (8, 16, 32)), O.compress(g, eb=e))


def test_concat_refuses_what_is_not_one_field():
    x = datagen.sines_1d(64 * 20, seed=9)
    a = O.compress(x[:64 * 10], eb=0.01)
    b = O.compress(x[64 * 10:], eb=0.01)
    with pytest.raises(O.OracleError) as ex:  # different bounds
        O.concat([a, O.compress(x[64 * 10:], eb=0.02)], (x.size,))
    assert ex.value.name == "MISMATCH"
    with pytest.raises(O.OracleError) as ex:  # a shard before the last is ragged
        O.concat([O.compress(x[:100], eb=0.01), O.compress(x[100:], eb=0.01)], (x.size,))
    assert ex.value.name == "MISMATCH"
    with pytest.raises(O.OracleError) as ex:  # the shape disagrees with the values
        O.concat([a, b], (x.size + 1,))
    assert ex.value.name == "ARG"
