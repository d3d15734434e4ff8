"""Batched producing operators through the C ABI: scalar multiplication,
element-wise addition and subtraction over a batch plan, and compression of
many fields, each in one launch over all fields' tiles. Every field's stream
must equal the single-stream call's and the oracle's byte for byte; a captured
CUDA graph of the batched multiplication replays to the same streams."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def field_set(seed=5):
    """Uneven fields: one value, ragged tails, a constant field, whole tiles,
    sines with constant runs, GRFs; each with its own relative bound."""
    rng = np.random.default_rng(seed)
    sizes = [1, 63, 65, 4096, 4097, 70_001, 131_072, 9, 200_003, 33_333]
    sizes += [int(v) for v in np.exp(rng.uniform(np.log(100), np.log(60_000), 14))]
    xs, rels = [], []
    for i, n in enumerate(sizes):
        kind = i % 3
        if kind == 0 and n >= 64:
            x = datagen.sines_1d(n, seed=300 + i)
        elif kind == 1 and n >= 2:
            x = datagen.grf((n,), seed=400 + i)
        else:
            x = np.full(n, np.float32(rng.normal()), np.float32)
        xs.append(np.ascontiguousarray(x, np.float32))
        rels.append(float(10 ** rng.uniform(-5, -2)))
    return xs, rels


@pytest.fixture(scope="module")
def plan_inputs(hz):
    xs, rels = field_set()
    ca = [hz.compress(dev(x), eb=r, mode="rel") for x, r in zip(xs, rels)]
    oa = [O.compress(x, eb=r, mode="rel") for x, r in zip(xs, rels)]
    for c, o in zip(ca, oa):
        assert np.array_equal(host(c), o)
    # B: other values on the same shapes, at A's absolute bound field by field
    ys = [(x[::-1] * np.float32(0.7) + np.float32(0.1)).astype(np.float32) for x in xs]
    es = [float(O.header(o)["eps_q"]) for o in oa]
    cb = [hz.compress(dev(y), eb=e) for y, e in zip(ys, es)]
    ob = [O.compress(y, eb=e) for y, e in zip(ys, es)]
    return xs, rels, ca, oa, cb, ob


@pytest.mark.parametrize("s", [3.14, -0.37, 250.0, 1e-6])
def test_batch_mul_scalar(hz, plan_inputs, s):
    _, _, ca, oa, _, _ = plan_inputs
    b = hz.Batch([c.clone() for c in ca])
    got = b.mul_scalar(s)
    for f, (c, o) in enumerate(zip(ca, oa)):
        want = O.mul_scalar(o, s)
        assert np.array_equal(host(got[f]), want), f
        assert np.array_equal(host(hz.mul_scalar(c, s)), want), f


@pytest.mark.parametrize("subtract", [False, True])
def test_batch_add_sub(hz, plan_inputs, subtract):
    _, _, ca, oa, cb, ob = plan_inputs
    A = hz.Batch([c.clone() for c in ca])
    B = hz.Batch([c.clone() for c in cb])
    got = A.add(B, subtract=subtract)
    for f in range(len(ca)):
        want = O.sub(oa[f], ob[f]) if subtract else O.add(oa[f], ob[f])
        assert np.array_equal(host(got[f]), want), f


@pytest.mark.parametrize("mode", ["rel", "abs"])
def test_batch_compress(hz, plan_inputs, mode):
    xs, rels, _, _, _, _ = plan_inputs
    ebs = rels if mode == "rel" else [0.01 * (1 + i % 3) for i in range(len(xs))]
    got = hz.batch_compress([dev(x) for x in xs], ebs, mode=mode)
    for f, (x, e) in enumerate(zip(xs, ebs)):
        want = O.compress(x, dims=(x.size,), eb=e, mode=mode)
        assert np.array_equal(host(got[f]), want), f
        assert np.array_equal(host(hz.compress(dev(x), eb=e, mode=mode, dims=(x.size,))), want), f


def test_batch_mul_scalar_graph_capture(hz, plan_inputs):
    """The batched multiplication's three launches, captured in a CUDA graph
    through the C ABI (pointer tables made before the capture), replay to the
    oracle's streams."""
    import ctypes

    _, _, ca, oa, _, _ = plan_inputs
    b = hz.Batch([c.clone() for c in ca])
    outs = [torch.zeros(hz.compress_bound(hz.header(c)["n"]), dtype=torch.uint8, device="cuda")
            for c in ca]
    ptrs = torch.tensor([o.data_ptr() for o in outs], dtype=torch.int64, device="cuda")
    caps = torch.tensor([o.numel() for o in outs], dtype=torch.int64, device="cuda")
    sizes = torch.zeros(len(outs), dtype=torch.int64, device="cuda")
    L = hz.load_library()
    s = torch.cuda.Stream()

    def call():
        return L.hoszp_batch_mul_scalar(b.handle, 2.5, ctypes.c_void_p(ptrs.data_ptr()),
                                        ctypes.c_void_p(caps.data_ptr()),
                                        ctypes.c_void_p(sizes.data_ptr()),
                                        ctypes.c_void_p(s.cuda_stream))

    with torch.cuda.stream(s):  # the first call grows the workspace, outside the capture
        assert call() == 0
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        assert call() == 0
    for o in outs:
        o.zero_()
    sizes.zero_()
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        b.check()
        n = sizes.cpu().tolist()
        for f, o in enumerate(oa):
            assert np.array_equal(host(outs[f][: int(n[f])]), O.mul_scalar(o, 2.5)), f


def test_batch_produce_errors(hz, plan_inputs):
    xs, rels, ca, oa, cb, _ = plan_inputs
    A = hz.Batch([c.clone() for c in ca[:4]])
    other = [hz.compress(dev(x), eb=0.123) for x in xs[:4]]  # other bounds
    B = hz.Batch(other)
    with pytest.raises(hz.HoszpError) as e:
        A.add(B)
    assert e.value.name == "MISMATCH"
    # an output too small for its field: CAPACITY, size 0, other fields intact
    outs = [torch.empty(hz.compress_bound(hz.header(c)["n"]), dtype=torch.uint8, device="cuda")
            for c in ca[:4]]
    outs[3] = torch.empty(64, dtype=torch.uint8, device="cuda")
    got, sizes = A.mul_scalar(3.0, outs=outs, sync=False)
    torch.cuda.synchronize()
    assert A.status() != 0
    n = sizes.cpu().tolist()
    assert n[3] == 0
    for f in range(3):
        assert np.array_equal(host(outs[f][: int(n[f])]), O.mul_scalar(oa[f], 3.0)), f
