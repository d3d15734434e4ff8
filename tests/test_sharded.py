"""A field split into shards of whole blocks across ranks (gloo, world size 2,
on the CPU): the exact sums of the shards, added by one all-reduce, equal the
sums of the whole field, and every rank holds the same five words for the
library's finish (hoszp_finish_sums, tested on a GPU). The shards' sums come
from the oracle (no GPU here); on a GPU the same words come from hoszp_sums."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _field():
    import datagen

    return datagen.sines_1d(200_003, seed=31)  # ragged tail: 3125 blocks + 3 values


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle as O
    from paper_2408_11971_gb300 import sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = _field()
    eps = 1e-3 * float(x.max() - x.min())
    nb = (x.size + 63) // 64
    cut = [0, 1000 * 64, x.size][rank:rank + 2]  # shard 0: 1000 blocks, shard 1: the rest
    shard = np.ascontiguousarray(x[cut[0]:cut[1]])
    s1, s2, n, e = O.sums(O.compress(shard, eb=eps))
    tot = sharded.allreduce(sharded.Sums(s1, s2, n))
    q.put((rank, tot.s1, tot.s2, tot.n, sharded.to_words(tot), float(e), nb))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_combine_exact_sums():
    import multiprocessing as mp

    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = _field()
    eps = 1e-3 * float(x.max() - x.min())
    whole = O.compress(x, eb=eps)
    s1, s2, n, e = O.sums(whole)
    for rank, t1, t2, tn, words, eq, nb in got:
        assert (t1, t2, tn) == (s1, s2, n)  # exact, whatever the split
        assert eq == float(e)
    # every rank hands the library's finish the same five words (the device
    # finish of those words is compared with hoszp_mean / hoszp_var on a GPU)
    assert got[0][4] == got[1][4]


def test_sums_words_roundtrip():
    from paper_2408_11971_gb300 import sharded

    for s1, s2, n in [(0, 0, 1), (-5, 25, 3), (-(1 << 100) - 7, (1 << 120) + 3, 1 << 40),
                      ((1 << 126) - 1, (1 << 128) - 1, 5)]:
        w = [s1 & (2**64 - 1), (s1 >> 64) & (2**64 - 1), s2 & (2**64 - 1), s2 >> 64, n]
        s = sharded.from_words(w)
        assert (s.s1, s.s2, s.n) == (s1, s2, n)
        assert sharded._from_limbs(sharded._to_limbs(s)) == s


def _reduce_rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import datagen
    import oracle as O
    from paper_2408_11971_gb300 import sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = datagen.sines_1d(50_011, seed=100 + rank)  # each node's own field, one shape
    c = torch.from_numpy(O.compress(x, eb=2e-3))  # one absolute bound for all nodes

    def add(a, b):  # the oracle's homomorphic addition stands in for hoszp_add here
        return torch.from_numpy(O.add(a.numpy(), b.numpy()))

    out = sharded.reduce_sum(c, add=add)
    q.put((rank, None if out is None else out.numpy().tobytes()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [3, 4])
def test_reduce_sum_binomial_tree(world):
    """The sum of the nodes' compressed fields, added along a binomial tree of
    homomorphic additions (Sec. VI-B5), is the stream of the summed integers:
    byte for byte the same as adding the streams one after another."""
    import multiprocessing as mp

    import datagen
    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_reduce_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(got[r] is None for r in range(1, world))
    cs = [O.compress(datagen.sines_1d(50_011, seed=100 + r), eb=2e-3) for r in range(world)]
    chain = cs[0]
    for c in cs[1:]:
        chain = O.add(chain, c)
    assert got[0] == chain.tobytes()
    qsum = sum(O.decode_q(c).astype(np.int64) for c in cs)
    assert np.array_equal(O.decode_q(np.frombuffer(got[0], np.uint8)), qsum)


def _gather_rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import datagen
    import oracle as O
    from paper_2408_11971_gb300 import sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = datagen.grf((12, 40, 63), seed=7)  # 30240 values: 472 blocks and a ragged one
    x = g.reshape(-1)
    eps = 1e-3 * float(x.max() - x.min())
    cuts = [0, 64 * 101, 64 * 300, 64 * 400][:world] + [x.size]  # whole blocks but the last
    c = torch.from_numpy(O.compress(np.ascontiguousarray(x[cuts[rank]:cuts[rank + 1]]), eb=eps))

    def concat(parts, dims):  # the oracle's join stands in for hoszp_concat here
        return torch.from_numpy(O.concat([p.numpy() for p in parts], dims))

    out, offsets = sharded.gather_stream(c, g.shape, concat=concat)
    q.put((rank, None if out is None else out.numpy().tobytes(), offsets, c.numel()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gather_stream_assembles_the_whole_field(world):
    """Shards of one field compressed on the ranks are assembled on rank 0 into
    the stream of the whole field, byte for byte the oracle's compression of it
    (Sec. VI-B5); every rank gets the exclusive scan of the shard sizes."""
    import multiprocessing as mp

    import datagen
    import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_gather_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    got = {r: (s, off, nb) for r, s, off, nb in (q.get(timeout=60) for _ in ps)}
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(got[r][0] is None for r in range(1, world))
    g = datagen.grf((12, 40, 63), seed=7)
    eps = 1e-3 * float(g.max() - g.min())
    assert got[0][0] == O.compress(g, eb=eps).tobytes()
    sizes = [got[r][2] for r in range(world)]
    want = [sum(sizes[:r]) for r in range(world)]
    assert all(got[r][1] == want for r in range(world))
