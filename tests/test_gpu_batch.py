"""Batched execution over many resident streams, against the single-stream
operators and the oracle (through the C ABI).

Each batched result must equal the single-stream operator on that field:
bit-identical doubles for mean / variance (same exact integer sums, same FP64
finish), identical bytes for in-place negation / scalar addition, and within
1e-12 of the oracle.
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


def uneven_fields(seed=11):
    """Fields of uneven sizes (1 value .. 2e5, ragged tails, constant fields),
    each with its own relative bound."""
    rng = np.random.default_rng(seed)
    sizes = [1, 63, 64, 65, 4096, 4097, 50_000, 200_003, 7, 130_000]
    sizes += [int(v) for v in np.exp(rng.uniform(np.log(10), np.log(80_000), 22))]
    xs, ebs = [], []
    for i, n in enumerate(sizes):
        kind = i % 4
        if kind == 0:
            x = datagen.sines_1d(n, seed=100 + i) if n >= 64 else rng.normal(size=n).astype(np.float32)
        elif kind == 1:
            x = datagen.grf((n,), seed=200 + i) if n >= 2 else np.float32([0.5] * n)
        elif kind == 2:
            x = np.full(n, np.float32(rng.normal()), np.float32)  # constant field
        else:
            x = (rng.normal(size=n) * 10 ** rng.uniform(-2, 3)).astype(np.float32)
        xs.append(np.ascontiguousarray(x, np.float32))
        ebs.append(float(10 ** rng.uniform(-5, -2)))
    return xs, ebs


@pytest.fixture(scope="module")
def fields(hz):
    xs, ebs = uneven_fields()
    cs = [hz.compress(dev(x), eb=e, mode="rel") for x, e in zip(xs, ebs)]
    ocs = [O.compress(x, eb=e, mode="rel") for x, e in zip(xs, ebs)]
    for c, oc in zip(cs, ocs):
        assert np.array_equal(host(c), oc)
    return xs, ebs, cs, ocs


def test_batch_reductions(hz, fields):
    _, _, cs, ocs = fields
    work = [c.clone() for c in cs]
    b = hz.Batch(work)
    m, v = host(b.mean()), host(b.var())
    for f, (c, oc) in enumerate(zip(work, ocs)):
        assert m[f] == hz.mean(c) and v[f] == hz.var(c), f
        assert close(m[f], O.mean(oc)) and close(v[f], O.var(oc)), f
    # repeated launches reuse the per-field accumulators (reset in-kernel)
    assert np.array_equal(host(b.mean()), m) and np.array_equal(host(b.var()), v)


def test_batch_decompress(hz, fields):
    """One launch decompresses every field: bit for bit the single-stream
    decompression and the oracle's."""
    _, _, cs, ocs = fields
    b = hz.Batch([c.clone() for c in cs])
    outs = b.decompress()
    for f, (c, oc) in enumerate(zip(cs, ocs)):
        got = host(outs[f])
        assert np.array_equal(got, host(hz.decompress(c))), f
        assert np.array_equal(got, O.decompress(oc)), f
    again = b.decompress()  # repeated launches
    for f in range(len(cs)):
        assert np.array_equal(host(again[f]), host(outs[f])), f


def test_batch_in_place_operators(hz, fields):
    _, _, cs, ocs = fields
    work = [c.clone() for c in cs]
    b = hz.Batch(work)
    b.negate()
    torch.cuda.synchronize()
    b.check()
    neg = [O.negate(oc) for oc in ocs]
    for f in range(len(work)):
        assert np.array_equal(host(work[f]), neg[f]), f
    b.add_scalar(0.37)
    torch.cuda.synchronize()
    b.check()
    for f in range(len(work)):
        assert np.array_equal(host(work[f]), O.add_scalar(neg[f], 0.37)), f
    m = host(b.mean())
    for f in range(len(work)):
        assert close(m[f], O.mean(O.add_scalar(neg[f], 0.37))), f


def test_batch_graph_capture(hz, fields):
    _, _, cs, ocs = fields
    work = [c.clone() for c in cs]
    b = hz.Batch(work)
    out = torch.zeros(len(work), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up outside capture
        b.negate(stream=s)
        b.negate(stream=s)
        b.mean(out=out, stream=s, sync=False)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b.negate(stream=s)
        b.mean(out=out, stream=s, sync=False)
    torch.cuda.synchronize()
    ref = np.array([O.mean(oc) for oc in ocs])
    for rep in range(4):
        g.replay()
        torch.cuda.synchronize()
        sign = -1.0 if rep % 2 == 0 else 1.0
        got = host(out)
        for f in range(len(work)):
            assert close(got[f], sign * ref[f]) or (ref[f] == 0 and got[f] == 0), (rep, f)
    b.check()
    for f in range(len(work)):  # an even number of negations
        assert np.array_equal(host(work[f]), ocs[f]), f


def _run_op(hz, b, op, cs):
    """Runs op (0 mean, 1 var, 2 decompress) on plan b; True when every field
    equals the single-stream operator bit for bit."""
    if op == 0:
        got = host(b.mean())
        return all(got[f] == hz.mean(c) for f, c in enumerate(cs))
    if op == 1:
        got = host(b.var())
        return all(got[f] == hz.var(c) for f, c in enumerate(cs))
    outs = b.decompress()
    return all(np.array_equal(host(o), host(hz.decompress(c))) for o, c in zip(outs, cs))


def low_rate_fields(rel):
    """GRFs of uneven sizes (1-D, 2-D, 3-D, ragged tails) at one coarse relative
    bound, so every rate stays small and the rate-specialised shapes exist."""
    shapes = [(5000,), (70_001,), (64,), (999,), (300, 211), (37, 41, 23), (123_457,)]
    return [datagen.grf(sh, seed=300 + i).reshape(-1) for i, sh in enumerate(shapes)]


def test_batch_autotune(hz, fields):
    _, _, cs, ocs = fields
    b = hz.Batch([c.clone() for c in cs])
    outs = [torch.empty(hz.header(c)["n"], dtype=torch.float32, device="cuda") for c in cs]
    picks = b.tune(outs=outs)
    for op in ("mean", "var"):
        p = picks[op]
        assert p["stages"] in (4, 8) and p["ctas_per_sm"] in (1, 2), p
        assert p["warps_per_group"] in (4, 8, 16) and p["plane_groups"] in (1, 2, 4), p
    assert picks["decompress"]["warps_per_group"] in (4, 8), picks
    m = host(b.mean())
    for f, oc in enumerate(ocs):
        assert close(m[f], O.mean(oc)), f
    for f, oc in enumerate(ocs):  # the tuner's own decompression runs wrote the outputs
        assert np.array_equal(host(outs[f]), O.decompress(oc)), f


def test_batch_every_shape_uneven(hz, fields):
    """Every launch shape the tuner may pick gives the single-stream results."""
    _, _, cs, _ = fields
    b = hz.Batch([c.clone() for c in cs])
    for op in range(3):
        n = b.shapes(op)
        assert n >= (6 if op < 2 else 2), (op, n)
        for i in range(n):
            b.set_shape(op, i)
            assert _run_op(hz, b, op, cs), (op, i, b.config(op))
    with pytest.raises(hz.HoszpError):
        b.set_shape(0, b.shapes(0))


@pytest.mark.parametrize("rel", [1e-2, 1e-3])
def test_batch_every_shape_rate_specialised(hz, rel):
    """A plan whose header bounds keep every rate small offers rate-specialised
    decodes (fewer plane groups) for variance and decompression; each shape
    gives the single-stream results bit for bit."""
    xs = low_rate_fields(rel)
    cs = [hz.compress(dev(x), eb=rel, mode="rel") for x in xs]
    b = hz.Batch(cs)
    for op in range(3):
        groups = set()
        for i in range(b.shapes(op)):
            b.set_shape(op, i)
            groups.add(b.config(op)["plane_groups"])
            assert _run_op(hz, b, op, cs), (op, i, b.config(op))
        assert min(groups) < 4, (op, groups)  # a specialised shape was offered


def test_batch_errors(hz, fields):
    _, _, cs, _ = fields
    bad = cs[4].clone()
    bad[0] ^= 0xFF  # magic
    with pytest.raises(hz.HoszpError) as e:
        hz.Batch([cs[0], bad])
    assert e.value.name == "FORMAT"
    empty = hz.compress(dev(np.zeros(0, np.float32)), eb=0.1)
    with pytest.raises(hz.HoszpError) as e:
        hz.Batch([cs[0], empty])
    assert e.value.name == "ARG"
    # a scalar that leaves the integer range: no field changes, status RANGE
    work = [c.clone() for c in cs[:3]]
    b = hz.Batch(work)
    b.add_scalar(1e30)
    torch.cuda.synchronize()
    assert b.status() == -5  # RANGE
    for f in range(3):
        assert torch.equal(work[f], cs[f])
