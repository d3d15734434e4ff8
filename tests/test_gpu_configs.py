"""The other workload shapes at full size, through the C ABI, against the oracle.

- A 449x449x235 Gaussian random field (47,376,235 values: the last block holds
  43) at relative bounds 1e-2 and 1e-5: compression, decompression (every
  value), negation, scalar addition, scalar multiplication, field + field
  addition (B at A's absolute bound), mean and variance.
- The other two 3-D shapes of the workload, 100x500x500 (25 M values) at
  relative bound 1e-3 and 256x384x384 (37.7 M) at 1e-4, through every
  operator as above, and the 512x512x512 field at relative bounds 1e-2, 1e-3
  and 1e-5 (compression, every decompressed value, mean and variance).
- One 1800x3600 latitude-banded variable with its 30 % land mask at 1e35, at
  relative bound 1e-6 (wide rates next to constant land blocks): mean,
  variance and scalar multiplication.
- 64 fields of the batched workload's generator (log-uniform sizes, 1-D/2-D/3-D
  fields, per-field relative bounds) through one batch plan: every batched
  result equals the oracle's for its field.
Streams bit for bit; mean and variance within 1e-12 relative (exact integer
sums, FP64 finish).
"""
import numpy as np
import pytest

import datagen
import oracle as O

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


SHAPE = (449, 449, 235)


@pytest.fixture(scope="module")
def grf449():
    A = datagen.grf(SHAPE, seed=21).reshape(-1)
    B = datagen.grf(SHAPE, seed=22).reshape(-1)
    assert A.size == 47_376_235 and A.size % 64 == 43
    return A, B


def every_operator(hz, A, B, shape, rel):
    ctx = hz.Context(0)
    ca = hz.compress(dev(A), eb=rel, mode="rel", dims=shape, ctx=ctx)
    oa = O.compress(A, dims=shape, eb=rel, mode="rel")
    assert np.array_equal(host(ca), oa)
    e = float(O.header(oa)["eps_q"])
    cb = hz.compress(dev(B), eb=e, dims=shape, ctx=ctx)
    ob = O.compress(B, dims=shape, eb=e)
    assert np.array_equal(host(cb), ob)
    assert np.array_equal(host(hz.decompress(ca, ctx=ctx)), O.decompress(oa))
    assert np.array_equal(host(hz.negate(ca, ctx=ctx)), O.negate(oa))
    assert np.array_equal(host(hz.add_scalar(ca, 0.5, ctx=ctx)), O.add_scalar(oa, 0.5))
    assert np.array_equal(host(hz.mul_scalar(ca, 3.14, ctx=ctx)), O.mul_scalar(oa, 3.14))
    assert np.array_equal(host(hz.add(ca, cb, ctx=ctx)), O.add(oa, ob))
    assert close(hz.mean(ca, ctx=ctx), O.mean(oa)) and close(hz.var(ca, ctx=ctx), O.var(oa))


@pytest.mark.parametrize("rel", [1e-2, 1e-5])
def test_grf_449x449x235_every_operator(hz, grf449, rel):
    A, B = grf449
    every_operator(hz, A, B, SHAPE, rel)  # every decompressed value, the 43-value tail included


@pytest.mark.parametrize("shape,rel", [((100, 500, 500), 1e-3), ((256, 384, 384), 1e-4)])
def test_grf_other_shapes_every_operator(hz, shape, rel):
    A = datagen.grf(shape, seed=31).reshape(-1)
    B = datagen.grf(shape, seed=32).reshape(-1)
    every_operator(hz, A, B, shape, rel)


@pytest.fixture(scope="module")
def grf512():
    return datagen.grf((512, 512, 512), seed=1).reshape(-1)


@pytest.mark.parametrize("rel", [1e-2, 1e-3, 1e-5])
def test_grf_512_other_bounds(hz, grf512, rel):
    shape = (512, 512, 512)
    ctx = hz.Context(0)
    c = hz.compress(dev(grf512), eb=rel, mode="rel", dims=shape, ctx=ctx)
    oc = O.compress(grf512, dims=shape, eb=rel, mode="rel")
    assert np.array_equal(host(c), oc)
    assert np.array_equal(host(hz.decompress(c, ctx=ctx)), O.decompress(oc))
    assert close(hz.mean(c, ctx=ctx), O.mean(oc)) and close(hz.var(c, ctx=ctx), O.var(oc))


def test_land_mask_1800x3600_at_1e6(hz):
    x = datagen.lat_bands_2d(1800, 3600, seed=3)
    assert np.mean(x == np.float32(1e35)) > 0.2
    c = hz.compress(dev(x.reshape(-1)), eb=1e-6, mode="rel", dims=x.shape)
    oc = O.compress(x.reshape(-1), dims=x.shape, eb=1e-6, mode="rel")
    assert np.array_equal(host(c), oc)
    rates = host(c)[64:64 + (x.size + 63) // 64]
    assert (rates == 0).mean() > 0.1 and rates.max() >= 8  # constant land, wide coasts
    assert close(hz.mean(c), O.mean(oc)) and close(hz.var(c), O.var(oc))
    for s in (0.75, 3.14):
        assert np.array_equal(host(hz.mul_scalar(c, s)), O.mul_scalar(oc, s)), s


def test_batched_generator_fields(hz):
    specs, gen = datagen.field_set_batched(64, seed=4, lo=1e4, hi=1e6)
    xs = [np.ascontiguousarray(gen(i).reshape(-1)) for i in range(len(specs))]
    rels = [r for _, r, _ in specs]
    cs = [hz.compress(dev(x), eb=r, mode="rel") for x, r in zip(xs, rels)]
    ocs = [O.compress(x, eb=r, mode="rel") for x, r in zip(xs, rels)]
    for c, oc in zip(cs, ocs):
        assert np.array_equal(host(c), oc)
    b = hz.Batch([c.clone() for c in cs])
    m, v = host(b.mean()), host(b.var())
    outs = b.decompress()
    for f, oc in enumerate(ocs):
        assert close(m[f], O.mean(oc)) and close(v[f], O.var(oc)), f
        assert np.array_equal(host(outs[f]), O.decompress(oc)), f
