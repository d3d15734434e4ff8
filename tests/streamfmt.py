"""Independent reader of the stream layout (header, rates, outliers, sign words,
bit planes), written with numpy for the tests. It restates the layout from the
format definition and shares nothing with the oracle or the library."""
from __future__ import annotations

import numpy as np

L = 64
HDR = 64


def _a16(v):
    return (v + 15) // 16 * 16


def parse(c) -> dict:
    c = np.asarray(c, dtype=np.uint8)
    h = c[:HDR].tobytes()
    magic = int.from_bytes(h[0:4], "little")
    n = int.from_bytes(h[24:32], "little")
    nnc = int.from_bytes(h[40:48], "little")
    R = int.from_bytes(h[48:56], "little")
    nb = (n + L - 1) // L
    o_out = HDR + _a16(nb)
    o_sign = o_out + _a16(4 * nb)
    o_plane = o_sign + 8 * nnc
    size = _a16(o_plane + 8 * R)
    return dict(
        magic=magic,
        version=int.from_bytes(h[4:6], "little"),
        ndims=h[7],
        dims=[int.from_bytes(h[8 + 4 * i:12 + 4 * i], "little") for i in range(3)],
        eps_q=np.frombuffer(h[20:24], np.float32)[0],
        n=n,
        eps=np.frombuffer(h[32:40], np.float64)[0],
        nnc=nnc,
        R=R,
        qbound=int.from_bytes(h[56:60], "little"),
        block=int.from_bytes(h[60:64], "little"),
        nb=nb,
        size=size,
        rate=c[HDR:HDR + nb].copy(),
        outlier=c[o_out:o_out + 4 * nb].view(np.int32).copy(),
        sign=c[o_sign:o_sign + 8 * nnc].view(np.uint64).copy(),
        plane=c[o_plane:o_plane + 8 * R].view(np.uint64).copy(),
    )


def block_deltas(s: dict) -> np.ndarray:
    """Signed deltas (nb x 64, int64) read from sign words and bit planes."""
    nb = s["nb"]
    d = np.zeros((nb, L), np.int64)
    si = pi = 0
    bits = np.arange(L, dtype=np.uint64)
    for b in range(nb):
        r = int(s["rate"][b])
        if r == 0:
            continue
        sign = (s["sign"][si] >> bits) & np.uint64(1)
        si += 1
        mag = np.zeros(L, np.int64)
        for p in range(r):
            mag |= (((s["plane"][pi] >> bits) & np.uint64(1)).astype(np.int64) << p)
            pi += 1
        d[b] = np.where(sign == 1, -mag, mag)
    return d


def values(s: dict) -> np.ndarray:
    """Quantized integers q: outlier + running sum of deltas 1..63 per block."""
    n, nb = s["n"], s["nb"]
    d = block_deltas(s)
    d[:, 0] = 0
    q = s["outlier"].astype(np.int64)[:, None] + np.cumsum(d, axis=1)
    return q.reshape(-1)[:n]
