"""Reductions over compressed data held by several devices or processes (one
per rank).

Sum of fields (the distributed experiment of Sec. VI-B5: every node compresses
its data and the streams are summed at a root): `reduce_sum` adds the ranks'
streams of one field shape with the homomorphic element-wise addition (Sec.
V-C) along a binomial tree -- log2(P) rounds; in round k a rank whose bit k is
set sends its partial stream to the rank 2^k below it, which adds -- so no
stream is ever decompressed and the root receives the stream of the sum. The
result does not depend on the tree: q-sums are exact and the encoding of a
q-field is unique.

Stream of a field whose shards live on the ranks: `gather_stream` assembles
the shards' streams into the field's stream on rank 0 (the sections laid end
to end under one header; nothing is decoded).

Mean and variance of one field whose compressed shards live on the ranks:

Each rank holds a stream of whole blocks of the field, compressed with the same
absolute bound (the same eps_q bits). The library returns each shard's exact
integer sums (hoszp_sums: S1 = sum q, S2 = sum q^2, n; Sec. V-B); the ranks add
them with one all-reduce of 32-bit limbs held in int64 -- exact and independent
of the order of addition -- and every rank finishes mean and variance on its
device with the library's hoszp_finish_sums, the same FP64 steps as the
single-stream kernels, so a sharded field gives the same double as the whole
field on one device.
"""
from __future__ import annotations

from dataclasses import dataclass

MASK64 = (1 << 64) - 1
_LIMBS = 8  # S1 and S2 as four 32-bit limbs each


@dataclass
class Sums:
    s1: int  # sum of q (signed)
    s2: int  # sum of q^2
    n: int

    def __add__(self, o: "Sums") -> "Sums":
        return Sums(self.s1 + o.s1, self.s2 + o.s2, self.n + o.n)


def from_words(w) -> Sums:
    """The five words written by hoszp_sums."""
    s1 = int(w[0]) | (int(w[1]) << 64)
    if s1 >> 127:
        s1 -= 1 << 128
    return Sums(s1, int(w[2]) | (int(w[3]) << 64), int(w[4]))


def _to_limbs(s: Sums):
    s1 = s.s1 & ((1 << 128) - 1)  # two's complement; the sum is taken modulo 2^128
    out = [(s1 >> (32 * k)) & 0xFFFFFFFF for k in range(4)]
    out += [(s.s2 >> (32 * k)) & 0xFFFFFFFF for k in range(4)]
    return out + [s.n]


def _from_limbs(v) -> Sums:
    s1 = sum(int(v[k]) << (32 * k) for k in range(4)) & ((1 << 128) - 1)
    if s1 >> 127:
        s1 -= 1 << 128
    s2 = sum(int(v[4 + k]) << (32 * k) for k in range(4))
    return Sums(s1, s2, int(v[_LIMBS]))


def allreduce(s: Sums, group=None) -> Sums:
    """Exact sum of every rank's Sums (torch.distributed, any backend). Each
    32-bit limb sum stays exact in int64 for up to 2^31 ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor(_to_limbs(s), dtype=torch.int64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return _from_limbs(t.cpu().tolist())


def to_words(s: Sums):
    """The five words of hoszp_sums for combined sums (S1 as a 128-bit two's
    complement integer, S2 as 128-bit unsigned, n)."""
    s1 = s.s1 & ((1 << 128) - 1)
    return [s1 & MASK64, s1 >> 64, s.s2 & MASK64, (s.s2 >> 64) & MASK64, s.n]


def finish(s: Sums, eps_q: float, device: int = 0, ctx=None):
    """(mean, population variance) of combined sums, finished on the device by
    the library (hoszp_finish_sums) with the single-stream kernels' FP64 steps."""
    if s.n == 0:
        raise ValueError("empty field")
    from . import _binding as B

    return B.finish_sums(to_words(s), eps_q, device=device, ctx=ctx)


def mean_var(c_local, eps_q: float, group=None, ctx=None):
    """Mean and variance of the field whose shard on this rank is the stream
    c_local (a CUDA uint8 tensor); collective over `group`."""
    from . import _binding as B

    s = from_words(B.sums(c_local, ctx=ctx))
    return finish(allreduce(s, group), eps_q, device=c_local.device.index or 0, ctx=ctx)


def _send_stream(t, dst, group=None):
    import torch
    import torch.distributed as dist

    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    dist.send(n, dst, group=group)
    dist.send(t.contiguous(), dst, group=group)


def _recv_stream(src, device, group=None):
    import torch
    import torch.distributed as dist

    n = torch.zeros(1, dtype=torch.int64, device=device)
    dist.recv(n, src, group=group)
    t = torch.empty(int(n.item()), dtype=torch.uint8, device=device)
    dist.recv(t, src, group=group)
    return t


def reduce_sum(c_local, group=None, add=None):
    """Sum of the fields whose streams (uint8 tensors, one per rank, the same n
    and eps_q) the ranks hold, by a binomial tree of homomorphic additions.
    Returns the stream of the sum on rank 0 and None elsewhere. `add(a, b)`
    adds two streams (default: the library's hoszp_add on the tensors' device;
    the tensors travel on that device, so use a backend that can carry it)."""
    import torch.distributed as dist

    if add is None:
        from . import _binding as B

        add = B.add
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    cur = c_local
    step = 1
    while step < world:
        if rank % (2 * step) == step:  # send to the partner below and stop
            _send_stream(cur, rank - step, group)
            return None
        if rank % (2 * step) == 0 and rank + step < world:
            other = _recv_stream(rank + step, cur.device, group)
            cur = add(cur, other)
        step *= 2
    return cur


def gather_stream(c_local, dims, group=None, concat=None):
    """The stream of a field whose consecutive shards (whole blocks each but the
    last; one bound) the ranks hold in rank order, assembled on rank 0 (Sec.
    VI-B5: the nodes' compressed data gathered at a root). One all-gather of
    the shards' byte counts gives each rank its byte offset in the gathered
    bytes (an exclusive scan, returned with the result); the shards then travel
    to rank 0, which joins their sections under one header with `concat`
    (default: the library's hoszp_concat on the tensors' device). Returns
    (stream or None, offsets) -- the stream on rank 0, None elsewhere."""
    import torch
    import torch.distributed as dist

    if concat is None:
        from . import _binding as B

        concat = B.concat
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    dev = c_local.device
    mine = torch.tensor([c_local.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(sizes, mine, group=group)
    sizes = [int(t.item()) for t in sizes]
    offsets = [0]
    for s in sizes[:-1]:
        offsets.append(offsets[-1] + s)
    if rank != 0:
        dist.send(c_local.contiguous(), 0, group=group)
        return None, offsets
    parts = [c_local]
    for r in range(1, world):
        t = torch.empty(sizes[r], dtype=torch.uint8, device=dev)
        dist.recv(t, r, group=group)
        parts.append(t)
    return concat(parts, dims), offsets
