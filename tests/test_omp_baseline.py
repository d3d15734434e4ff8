"""The all-core CPU baseline (the oracle's arithmetic with an OpenMP loop over
blocks) gives the oracle's results byte for byte: it is timed as a baseline,
so it must compute the same thing."""
import numpy as np
import pytest

import datagen
import oracle as O
from oracle import omp


@pytest.mark.parametrize("field", ["sines", "grf3d", "mask"])
def test_omp_baseline_equals_oracle(field):
    if field == "sines":
        x = datagen.sines_1d(200_003, seed=13)
    elif field == "grf3d":
        x = datagen.grf((24, 40, 37), seed=3).reshape(-1)
    else:
        x = datagen.lat_bands_2d(90, 180, seed=2).reshape(-1)
    assert omp.threads() >= 1
    for eb, mode in ((1e-3, "rel"), (1e-5, "rel"), (0.05, "abs")):
        try:
            oc = O.compress(x, eb=eb, mode=mode)
        except O.OracleError as ex:  # the fill value is out of range at this bound
            with pytest.raises(O.OracleError) as ex2:
                omp.compress(x, eb=eb, mode=mode)
            assert ex2.value.name == ex.name
            continue
        c = omp.compress(x, eb=eb, mode=mode)
        assert np.array_equal(c, oc)
        assert np.array_equal(omp.decompress(c), O.decompress(oc))
        assert np.array_equal(omp.negate(c), O.negate(oc))
        assert np.array_equal(omp.add_scalar(c, 0.5), O.add_scalar(oc, 0.5))
        assert np.array_equal(omp.mul_scalar(c, 3.14), O.mul_scalar(oc, 3.14))
        e = float(O.header(oc)["eps_q"])
        y = x[::-1].copy()
        cy = O.compress(y, eb=e)
        assert np.array_equal(omp.add(c, cy), O.add(oc, cy))
        assert omp.sums(c) == O.sums(oc)
        assert omp.mean(c) == O.mean(oc) and omp.var(c) == O.var(oc)
