"""The oracle's Newton line search against its definition (Sec. 4): from X with
residual F and Newton direction S (the GMRES solution of J S = -F), the accepted
iterate is X + lambda S for the largest lambda in 1, 1/2, 1/4, ... whose trial
lies in the domain of the logarithms (c, c eta and c (4 - 3 eta) in (0, 1)) and
satisfies ||F(X + lambda S)||^2 <= (1 - 2 alpha lambda) ||F(X)||^2.  One Newton
iteration is observed by allowing one and accepting any decrease."""
import numpy as np
import pytest

import oracle
import synthetic as S


def _in_domain(X, nf):
    c, e = X[0::nf], X[1::nf]
    return all(np.all((v > 0) & (v < 1)) for v in (c, c * e, c * (4 - 3 * e)))


@pytest.mark.parametrize("dt,lam_expected", [(1.0, 1.0), (100.0, 0.5)])
def test_accepted_step_is_the_first_admissible_halving(dt, lam_expected):
    dim, n = 2, (16, 16)
    cf = S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    op = S.options(sub=(2, 2), overlap=1, newton_maxit=1, newton_rtol=1 - 1e-9, newton_atol=0.0)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    # a dilute state: the long step (dt = 100) overshoots c = 0 somewhere
    c, e = S.initial_fields(dim, n, 0.012, 3, c_amp=0.01)
    X0 = O.interleave(c, e)
    cb = float(np.mean(c))
    F0 = O.residual(X0, X0, cb, dt)
    rc, X1, info = O.newton_step(X0, cb, dt)
    assert rc == 0 and info["newton_its"] == 1
    tol = max(op["gmres_rtol"] * np.linalg.norm(F0), op["gmres_atol"])
    rcs, Sd, its, res = O.linear_solve(X0, X0, cb, dt, -F0, tol)
    assert rcs == 0
    d = X1 - X0
    lam = float(d @ Sd / (Sd @ Sd))
    assert lam == pytest.approx(lam_expected, rel=1e-12)
    assert np.linalg.norm(d - lam * Sd) <= 1e-13 * np.linalg.norm(d)
    alpha = op["ls_alpha"]
    f0 = np.linalg.norm(F0)

    def admissible(l):
        Xt = X0 + l * Sd
        if not _in_domain(Xt, O.nf):
            return False
        ft = np.linalg.norm(O.residual(Xt, X0, cb, dt))
        return np.isfinite(ft) and ft ** 2 <= (1 - 2 * alpha * l) * f0 ** 2

    assert admissible(lam)
    # every larger candidate was rejected
    l = 1.0
    while l > lam * 1.5:
        assert not admissible(l)
        l *= 0.5
    if lam_expected < 1.0:
        assert not _in_domain(X0 + Sd, O.nf)  # the full step leaves the domain
