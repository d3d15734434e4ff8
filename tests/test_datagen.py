"""The seeded input generators against the recipes they state: determinism,
the Gaussian random field's normalisation and energy spectrum E(k) ~ k^-5/3,
the share of exactly constant runs in the sines, the land-mask share of the
latitude bands, and the size and bound ranges of the batched field set."""
import numpy as np

import datagen


def test_deterministic_per_seed():
    a = datagen.grf((40, 30, 20), seed=5)
    assert np.array_equal(a, datagen.grf((40, 30, 20), seed=5))
    assert not np.array_equal(a, datagen.grf((40, 30, 20), seed=6))
    s = datagen.sines_1d(70_000, seed=3)
    assert np.array_equal(s, datagen.sines_1d(70_000, seed=3))
    assert not np.array_equal(s, datagen.sines_1d(70_000, seed=4))


def _shell_slope(x: np.ndarray, kmin: float, kmax: float) -> float:
    """Least-squares slope of log E(k) against log k, E(k) the spectral energy
    summed over shells of unit width in |k| (integer wavenumbers)."""
    X = np.fft.fftn(x.astype(np.float64))
    P = np.abs(X) ** 2
    grids = np.meshgrid(*[np.fft.fftfreq(s) * s for s in x.shape], indexing="ij")
    kk = np.sqrt(sum(g ** 2 for g in grids))
    shells = np.rint(kk).astype(np.int64).ravel()
    E = np.bincount(shells, weights=P.ravel())
    k = np.arange(E.size)
    sel = (k >= kmin) & (k <= kmax)
    return float(np.polyfit(np.log(k[sel]), np.log(E[sel]), 1)[0])


def test_grf_normalised_and_kolmogorov_spectrum():
    for shape, kmax in (((96, 96, 96), 30), ((512, 512), 150)):
        x = datagen.grf(shape, seed=1)
        assert x.dtype == np.float32 and x.shape == shape
        assert abs(float(x.mean(dtype=np.float64))) < 1e-6
        assert abs(float(x.std(dtype=np.float64)) - 1.0) < 1e-5
        slope = _shell_slope(x, 3, kmax)
        assert abs(slope - (-5.0 / 3.0)) < 0.15, (shape, slope)
    # another slope is honoured too (the filter, not a fixed spectrum)
    y = datagen.grf((512, 512), seed=2, spectral_slope=-3.0)
    assert abs(_shell_slope(y, 3, 150) - (-3.0)) < 0.15


def test_sines_constant_run_share():
    n = 1 << 20
    x = datagen.sines_1d(n, seed=0)
    assert x.dtype == np.float32 and x.size == n and np.isfinite(x).all()
    assert float(np.abs(x).max()) < 8 * 2.0 + 0.1  # 8 sines of amplitude <= 2, small noise
    same = float(np.mean(x[1:] == x[:-1]))
    assert 0.17 < same < 0.27, same
    y = datagen.sines_1d(n, seed=0, const_frac=0.0)
    assert float(np.mean(y[1:] == y[:-1])) < 1e-3


def test_lat_bands_land_mask_share():
    x = datagen.lat_bands_2d(180, 360, seed=4)
    assert x.shape == (180, 360) and x.dtype == np.float32
    land = x == np.float32(1e35)
    assert abs(float(land.mean()) - 0.3) < 0.01
    sea = np.abs(x[~land])
    assert np.isfinite(sea).all() and float(sea.max()) < 1e35
    # the fill is spatially coherent: most land points have a land neighbour to the east
    assert float(np.mean(land[:, 1:][land[:, :-1]])) > 0.9


def test_batched_field_set_ranges():
    spec, gen = datagen.field_set_batched(count=64, seed=7, lo=1e3, hi=1e5)
    assert len(spec) == 64
    for n, rel, kind in spec:
        assert 1e3 <= n <= 1e5 and 1e-5 <= rel <= 1e-2 and kind in (1, 2, 3)
    for i in range(0, 64, 9):
        x = gen(i)
        assert x.dtype == np.float32 and x.size == spec[i][0] and np.isfinite(x).all()
    capped, _ = datagen.field_set_batched(count=64, seed=7, lo=1e3, hi=1e5, max_total=200_000)
    assert sum(n for n, _, _ in capped) <= 200_000 and capped == spec[:len(capped)]


def test_small_cases_cover_the_edges():
    c = datagen.small_cases()
    assert c["empty"].size == 0 and c["one"].size == 1
    assert c["tail_63"].size == 63 and c["tail_65"].size == 65
    assert np.unique(c["all_const"]).size == 1 and not c["all_zero"].any()
    assert all(v.dtype == np.float32 for v in c.values())
