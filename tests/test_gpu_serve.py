"""Serving loop on the GPU, through the C ABI: a mixed stream of requests
over resident streams, admitted as slots and memory free up, gives for every
request exactly the result of the same call made alone (streams byte for byte,
mean and variance bit for bit); a tight HBM budget delays requests but never
exceeds the arena; errors come back per request."""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_11971_gb300 as hz
    from paper_2408_11971_gb300 import build

    build.build()
    return hz


@pytest.fixture(scope="module")
def fields(hz):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()  # noqa: E731
    x1 = datagen.sines_1d(1 << 20, seed=21)
    x2 = (datagen.sines_1d(1 << 20, seed=22) * np.float32(0.5)).astype(np.float32)
    g1 = datagen.grf((64, 80, 91), seed=3)
    g2 = datagen.grf((64, 80, 91), seed=4)
    c1 = hz.compress(dev(x1), eb=1e-3, mode="rel")
    e1 = hz.header(c1)["eps_q"]
    c2 = hz.compress(dev(x2), eb=e1)
    c3 = hz.compress(dev(g1), eb=1e-3, mode="rel", dims=(64, 80, 91))
    e3 = hz.header(c3)["eps_q"]
    c4 = hz.compress(dev(g2), eb=e3, dims=(64, 80, 91))
    return [c1, c2, c3, c4]


PAIRS = [(0, 1), (2, 3), (1, 0), (3, 2)]


def alone(hz, streams, op, a, b, s):
    if op == "mean":
        return hz.mean(streams[a])
    if op == "var":
        return hz.var(streams[a])
    if op == "negate":
        return hz.negate(streams[a])
    if op == "add_scalar":
        return hz.add_scalar(streams[a], s)
    if op == "mul_scalar":
        return hz.mul_scalar(streams[a], s)
    if op == "add":
        return hz.add(streams[a], streams[b])
    if op == "sub":
        return hz.sub(streams[a], streams[b])
    return hz.decompress(streams[a])


def make_requests(rng, n):
    ops = []
    for i in range(n):
        u = rng.random()
        if u < 0.4:
            op = "mean" if rng.random() < 0.5 else "var"
        elif u < 0.7:
            op = "add_scalar" if rng.random() < 0.5 else "mul_scalar"
        elif u < 0.9:
            op = "add" if rng.random() < 0.5 else "sub"
        else:
            op = "decompress"
        a, b = PAIRS[int(rng.integers(len(PAIRS)))]
        s = float(rng.choice([0.5, -1.25, 3.14, 0.01]))
        ops.append((i, op, a, b, s))
    return ops


def drain(srv, n, keep=None, timeout_s=60.0):
    import time

    got = []
    t_end = time.time() + timeout_s
    while len(got) < n and time.time() < t_end:
        for c in srv.poll(64, wait_us=20000):
            if keep is not None:
                keep(c)
            got.append(c)
    return got


def test_mixed_stream_same_as_alone(hz, fields):
    rng = np.random.default_rng(5)
    reqs = make_requests(rng, 240)
    expect = {i: alone(hz, fields, op, a, b, s) for i, op, a, b, s in reqs}
    torch.cuda.synchronize()
    srv = hz.Server(0, slots=4, hbm_budget=2 << 30, max_n=1 << 21)
    ids = [srv.register(c) for c in fields]
    t0 = srv.now_us() + 2000
    gaps = rng.exponential(100.0, len(reqs))  # about 10,000 requests per second
    arrival = t0 + np.cumsum(gaps).astype(np.int64)
    for (i, op, a, b, s), t in zip(reqs, arrival):
        srv.submit(op, ids[a], ids[b], s, tag=i, arrival_us=int(t))
    bad = []

    def check(c):
        i, op, a, b, s = reqs[c["tag"]]
        if c["status"] != 0:
            bad.append((i, op, c["status"]))
        elif op in ("mean", "var"):
            if c["value"] != expect[i]:
                bad.append((i, op, c["value"], expect[i]))
        else:
            out = srv.output(c)
            if not torch.equal(out, expect[i]):
                bad.append((i, op, "differs"))
            srv.release(c)
        assert c["arrival_us"] <= c["start_us"] <= c["done_us"]

    got = drain(srv, len(reqs), keep=check)
    st = srv.stats()
    srv.close()
    assert len(got) == len(reqs)
    assert not bad, bad[:5]
    assert st["completed"] == len(reqs) and st["pending"] == 0 and st["in_flight"] == 0
    assert st["arena_in_use"] == 0
    assert st["max_in_flight"] >= 2  # requests overlapped on the device


def test_tight_budget_delays_but_never_exceeds(hz, fields):
    probe = hz.Server(0, slots=2, hbm_budget=1 << 30, max_n=1 << 21)
    ws = probe.stats()["workspace_bytes"]
    probe.close()
    n = hz.header(fields[0])["n"]
    srv = hz.Server(0, slots=2, hbm_budget=ws + 6 * n, max_n=1 << 21)  # room for one field of floats
    sid = srv.register(fields[0])
    ref = hz.decompress(fields[0])
    for i in range(12):
        srv.submit("decompress", sid, tag=i)
        srv.submit("mean", sid, tag=100 + i)
    m = hz.mean(fields[0])
    seen = []

    def check(c):
        assert c["status"] == 0
        if c["op"] == hz.Server.OPS["decompress"]:
            assert torch.equal(srv.output(c), ref)
            srv.release(c)
        else:
            assert c["value"] == m
        seen.append(c["tag"])

    got = drain(srv, 24, keep=check)
    st = srv.stats()
    srv.close()
    assert len(got) == 24 and sorted(seen) == sorted(list(range(12)) + [100 + i for i in range(12)])
    assert st["arena_peak"] <= st["arena_bytes"] < 2 * 4 * n


def test_request_errors(hz, fields):
    srv = hz.Server(0, slots=2, hbm_budget=1 << 30, max_n=1 << 21)
    a = srv.register(fields[0])
    c = srv.register(fields[2])
    with pytest.raises(hz.HoszpError):
        srv.submit("mean", 99)
    srv.submit("add", a, c, tag=7)  # different n and eps: MISMATCH on the device
    srv.submit("mean", a, tag=8)
    got = {x["tag"]: x for x in drain(srv, 2)}
    srv.close()
    assert got[7]["status"] == -4 and not got[7]["d_out"]
    assert got[8]["status"] == 0
