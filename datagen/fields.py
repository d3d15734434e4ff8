"""Generators (numpy PCG64, seeded). See the package docstring."""
from __future__ import annotations

import numpy as np

# 3-D shapes: Hurricane (100x500x500) and Miranda (256x384x384) of Table 3, a
# 512^3 cube, and 449x449x235 whose size leaves a 43-value tail block.
GRF_SHAPES = [(100, 500, 500), (256, 384, 384), (512, 512, 512), (449, 449, 235)]
REL_BOUNDS = [1e-2, 1e-3, 1e-4, 1e-5]


def _constant_runs(x: np.ndarray, rng: np.random.Generator, frac: float) -> np.ndarray:
    """Overwrite runs of 64..4096 values with the run's first value until about
    `frac` of the array is covered (exactly constant stretches, like the
    constant blocks counted in Table 6)."""
    n = x.size
    covered = np.zeros(n, bool)
    target = int(frac * n)
    done = 0
    while done < target:
        L = int(rng.integers(64, 4097))
        s = int(rng.integers(0, max(1, n - L)))
        e = min(n, s + L)
        x[s:e] = x[s]
        done += int((~covered[s:e]).sum())
        covered[s:e] = True
    return x


def sines_1d(n: int = 1 << 20, seed: int = 0, const_frac: float = 0.2,
             noise: float = 0.01) -> np.ndarray:
    """Sum of 8 sines (amplitude U(0.5,2), frequency log-uniform in [1,2000]
    cycles per field, phase U(0,2pi)) plus N(0, noise^2) noise, with about
    `const_frac` of the values in exactly constant runs."""
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64) / max(n, 1)
    A = rng.uniform(0.5, 2.0, 8)
    f = np.exp(rng.uniform(np.log(1.0), np.log(2000.0), 8))
    ph = rng.uniform(0, 2 * np.pi, 8)
    x = np.zeros(n, np.float64)
    for k in range(8):
        x += A[k] * np.sin(2 * np.pi * f[k] * i + ph[k])
    x += rng.normal(0.0, noise, n)
    x = x.astype(np.float32)
    if const_frac > 0 and n >= 128:
        x = _constant_runs(x, rng, const_frac)
    return x


def grf(shape, seed: int = 0, spectral_slope: float = -5.0 / 3.0) -> np.ndarray:
    """Gaussian random field with a power-law energy spectrum E(k) ~ k^slope
    (Kolmogorov -5/3 by default): white noise filtered in Fourier space by
    |k|^((slope - (d-1)) / 2), d = number of dimensions, then scaled to zero mean
    and unit variance. float32."""
    import scipy.fft as sfft

    shape = tuple(int(s) for s in shape)
    d = len(shape)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape, dtype=np.float32)
    W = sfft.rfftn(w, workers=-1)
    del w
    ks = [np.fft.fftfreq(s).astype(np.float32) for s in shape[:-1]]
    ks.append(np.fft.rfftfreq(shape[-1]).astype(np.float32))
    k2 = np.zeros(W.shape, np.float32)
    for ax, k in enumerate(ks):
        sh = [1] * d
        sh[ax] = k.size
        k2 += (k.reshape(sh)) ** 2
    k2.flat[0] = 1.0
    expo = (spectral_slope - (d - 1)) / 4.0  # amplitude = |k|^((slope-(d-1))/2) = (k^2)^expo
    W *= np.power(k2, np.float32(expo))
    del k2
    W.flat[0] = 0.0
    x = sfft.irfftn(W, s=shape, workers=-1).astype(np.float32)
    del W
    x -= np.float32(x.mean(dtype=np.float64))
    sd = float(x.std(dtype=np.float64))
    if sd > 0:
        x /= np.float32(sd)
    return x


def _smooth_noise_2d(ny: int, nx: int, rng: np.random.Generator, scale: float) -> np.ndarray:
    import scipy.fft as sfft

    w = rng.standard_normal((ny, nx), dtype=np.float32)
    W = sfft.rfft2(w, workers=-1)
    ky = np.fft.fftfreq(ny).astype(np.float32).reshape(-1, 1)
    kx = np.fft.rfftfreq(nx).astype(np.float32).reshape(1, -1)
    W *= np.exp(-(ky ** 2 + kx ** 2) / np.float32(2 * scale ** 2))
    s = sfft.irfft2(W, s=(ny, nx), workers=-1).astype(np.float32)
    s -= s.mean()
    sd = s.std()
    return s / sd if sd > 0 else s


def lat_bands_2d(ny: int = 1800, nx: int = 3600, seed: int = 0, land_frac: float = 0.3,
                 fill: float = 1e35, amp: float | None = None) -> np.ndarray:
    """Latitude-banded climate-like field A cos(3 phi) + B cos(9 phi) plus smooth
    noise, with a spatially coherent land mask (about `land_frac` of the points,
    a thresholded smooth noise) set to the fill value `fill` (CESM-style 1e35),
    which produces constant blocks. `amp` scales the non-fill values (default:
    log-uniform in [1e28, 1e34], so that a value-range-relative bound leaves a
    mix of bit widths next to the 1e35 fill)."""
    rng = np.random.default_rng(seed)
    phi = np.linspace(-np.pi / 2, np.pi / 2, ny, dtype=np.float64).reshape(-1, 1)
    A, B = rng.uniform(0.5, 1.5), rng.uniform(0.1, 0.5)
    base = A * np.cos(3 * phi) + B * np.cos(9 * phi)
    x = (base + 0.2 * _smooth_noise_2d(ny, nx, rng, 0.02)).astype(np.float64)
    if amp is None:
        amp = float(np.exp(rng.uniform(np.log(1e28), np.log(1e34))))
    x = (x * amp).astype(np.float32)
    mask_src = _smooth_noise_2d(ny, nx, rng, 0.01)
    thr = np.quantile(mask_src, 1.0 - land_frac)
    x[mask_src > thr] = np.float32(fill)
    return x


def field_set_batched(count: int = 4096, seed: int = 0, lo: float = 1e4, hi: float = 1e7,
                      max_total: int | None = None):
    """Sizes log-uniform in [lo, hi] and relative bounds log-uniform in
    [1e-5, 1e-2] for a batch of uneven fields; returns a list of (n, rel) and a
    generator callback gen(i) -> float32 field of n values (a 1-D, 2-D or 3-D
    smooth random field, chosen per field)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), count)).astype(np.int64)
    rels = np.exp(rng.uniform(np.log(1e-5), np.log(1e-2), count))
    kinds = rng.integers(1, 4, count)
    if max_total is not None:
        keep = np.cumsum(sizes) <= max_total
        sizes, rels, kinds = sizes[keep], rels[keep], kinds[keep]
    spec = [(int(n), float(r), int(k)) for n, r, k in zip(sizes, rels, kinds)]

    def gen(i: int) -> np.ndarray:
        n, _, kind = spec[i]
        if kind == 1 or n < 4096:
            return sines_1d(n, seed=seed * 100003 + i, const_frac=0.1)
        if kind == 2:
            nx = int(np.sqrt(n))
            return grf((n // nx, nx), seed=seed * 100003 + i).reshape(-1)[:n].copy() \
                if (n // nx) * nx == n else np.concatenate(
                    [grf((n // nx, nx), seed=seed * 100003 + i).reshape(-1),
                     np.zeros(n - (n // nx) * nx, np.float32)])
        c = max(2, int(round(n ** (1 / 3))))
        base = grf((c, c, c), seed=seed * 100003 + i).reshape(-1)
        reps = -(-n // base.size)
        return np.tile(base, reps)[:n].copy()

    return spec, gen


def small_cases(seed: int = 0):
    """Small named inputs for parity tests: sizes that span several tiles and a
    ragged tail, all-constant fields, wide bit widths and special values."""
    rng = np.random.default_rng(seed)
    cases = {}
    cases["empty"] = np.zeros(0, np.float32)
    cases["one"] = np.array([0.3], np.float32)
    cases["tail_63"] = rng.standard_normal(63).astype(np.float32)
    cases["tail_65"] = rng.standard_normal(65).astype(np.float32)
    cases["sines_50k"] = sines_1d(50_003, seed=seed + 1)
    cases["noise_wide"] = (rng.standard_normal(40_000) * 1000).astype(np.float32)
    cases["all_const"] = np.full(10_000, 1.25, np.float32)
    cases["all_zero"] = np.zeros(9_999, np.float32)
    cases["ramp"] = np.arange(20_000, dtype=np.float32) * np.float32(0.01)
    cases["grf_2d"] = grf((130, 77), seed=seed + 2).reshape(-1)
    cases["alternating"] = np.where(np.arange(12_345) % 2 == 0, 1.0, -1.0).astype(np.float32)
    return cases
