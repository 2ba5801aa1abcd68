"""The adaptive time step of the oracle's time loop against Eq. sencondt with the
energy-change driver: dt_1 = dt_init, and for n >= 2
    dt_n = max(dt_min, dt_max / sqrt(1 + zeta X'^2)),  X' = |E^{n-1} - E^{n-2}| / dt_{n-1},
computed here from the energies the loop reports (E^0 the initial energy); every
step is accepted without a retry in this run, so zeta keeps its value."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S


@pytest.mark.parametrize("dim,n,elastic", [(2, (12, 12), True), (1, (48,), False)])
def test_energy_driven_dt_sequence_follows_the_predictor(dim, n, elastic):
    cf = S.coefficients() if elastic else S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    op = S.options(sub=(2,) * dim, overlap=1, dt_mode="energy", dt_max=0.5, zeta=50.0)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    c, e = S.initial_fields(dim, n, 0.18, 5)
    steps = 6
    rc, X, infos, e0 = O.simulate(c, e, steps)
    assert rc == 0
    assert all(i["retries"] == 0 for i in infos)
    dts = [i["dt"] for i in infos]
    energies = [e0] + [i["energy"] for i in infos]
    assert dts[0] == op["dt_init"]
    for k in range(1, steps):
        xd = abs(energies[k] - energies[k - 1]) / dts[k - 1]
        want = max(op["dt_min"], op["dt_max"] / math.sqrt(1.0 + op["zeta"] * xd * xd))
        assert dts[k] == pytest.approx(want, rel=1e-13), (k, dts[k], want)
    # the steps are taken: time advances by the sum of the dt, energy does not increase
    assert infos[-1]["t"] == pytest.approx(sum(dts), rel=1e-14)
    assert np.all(np.diff(energies) <= 1e-12 * abs(energies[0]))
