"""The oracle's GMRES(m) against its defining property (Sec. 4; Saad and Schultz):
with the right preconditioner M^-1 = P RAS^-1 and x_0 = 0, the iterate after k
Arnoldi steps of one cycle is x_k = M^-1 y_k, where y_k minimises ||b - A M^-1 y||
over the Krylov space K_k(A M^-1, b); a restart starts the same construction
from the true residual of the previous cycle.  The Krylov spaces are built here
explicitly (power basis, QR) and the minimisation is a dense least-squares solve,
independent of the Arnoldi recurrence, the Gram-Schmidt rule and the Givens
rotations the oracle uses."""
import numpy as np
import pytest

import oracle
import synthetic as S


def _setup(dim, n, sub, restart, maxit):
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=1, gmres_restart=restart, gmres_maxit=maxit)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    c0, e0, u0 = S.random_fields(dim, n, 51, u_amp=0.01)
    c1 = c0 * (1 + 0.03 * np.sin(np.arange(c0.size)))
    X1, X0 = O.interleave(c1, e0, u0), O.interleave(c0, e0, u0)
    cb, dt = float(np.mean(c0)), 0.1
    A = O.jacobian_scipy(X1, X0, cb, dt).toarray()

    def M(v):
        rc, z = O.precond_apply(X1, X0, cb, dt, v)
        assert rc == 0
        return z

    return O, X1, X0, cb, dt, A, M


def _gmres_cycle(A, M, r0, k):
    """argmin over x in M^-1 K_k(A M^-1, r0) of ||r0 - A x||"""
    K = np.zeros((r0.size, k))
    v = r0 / np.linalg.norm(r0)
    for i in range(k):
        K[:, i] = v
        v = A @ M(v)
        v /= np.linalg.norm(v)
    Q = np.linalg.qr(K)[0]
    MQ = np.stack([M(Q[:, i]) for i in range(k)], axis=1)
    c = np.linalg.lstsq(A @ MQ, r0, rcond=None)[0]
    return MQ @ c


@pytest.mark.parametrize("dim,n,sub,k", [(2, (8, 6), (2, 2), 6), (1, (24,), (3,), 5), (3, (4, 4, 4), (2, 2, 1), 5)])
def test_one_cycle_iterate_is_the_minimal_residual_one(dim, n, sub, k):
    O, X1, X0, cb, dt, A, M = _setup(dim, n, sub, 30, k)
    b = np.random.default_rng(12).standard_normal(A.shape[0])
    rc, x, its, res = O.linear_solve(X1, X0, cb, dt, b, 1e-300)
    assert rc == 0 and its == k
    want = _gmres_cycle(A, M, b, k)
    assert np.linalg.norm(x - want) <= 1e-7 * np.linalg.norm(want)
    assert res == pytest.approx(np.linalg.norm(b - A @ want), rel=1e-7)


def test_restart_continues_from_the_true_residual():
    k1, k2 = 4, 3
    O, X1, X0, cb, dt, A, M = _setup(2, (8, 6), (2, 2), k1, k1 + k2)
    b = np.random.default_rng(13).standard_normal(A.shape[0])
    rc, x, its, res = O.linear_solve(X1, X0, cb, dt, b, 1e-300)
    assert rc == 0 and its == k1 + k2
    x1 = _gmres_cycle(A, M, b, k1)
    want = x1 + _gmres_cycle(A, M, b - A @ x1, k2)
    assert np.linalg.norm(x - want) <= 1e-7 * np.linalg.norm(want)
    # the residual never increases from one cycle to the next
    assert np.linalg.norm(b - A @ want) <= np.linalg.norm(b - A @ x1) * (1 + 1e-12)
