"""Pins of the oracle's model with three order parameters (App. A; row f2).

The model is checked against what the mathematics fixes, not against itself:
  * with eta_1 = eta_2 = eta_3 it is the reduced model of the main text: the
    energy, the DVD derivative (G_c, and sum_j G_eta_j = G_eta) and whole NKS
    steps agree with the (separately pinned) one-order-parameter oracle;
  * the discrete chain rule of the DVD construction holds exactly (exact Psi
    quotients): sum_p G . (X1 - X0) = E(X1) - E(X0) without elasticity, and
    pointwise for the local terms;
  * the analytic-by-complex-step Jacobian equals central differences of the
    residual;
  * on asymmetric states the steps conserve mass and do not increase the
    energy (Theorem 3.2), and permuting eta_1, eta_2, eta_3 permutes the result.
These tests run on the CPU only; tests/test_gpu_model3.py holds the CUDA path to them.
"""
import numpy as np
import pytest

import oracle
import synthetic as S


def _cf(n_eta, **over):
    return S.coefficients(n_eta=n_eta, **over)


def _state3(dim, n, seed, u_amp=0.0):
    c, eta = S.initial_fields3(dim, n, 0.18, seed, eta_amp=0.05)
    N = c.size
    u = None
    if u_amp:
        u = u_amp * (2.0 * S.uniform01(seed + 7, dim * N).reshape(dim, N) - 1.0)
    return c, eta, u


@pytest.mark.parametrize("elastic", [True, False])
def test_energy_reduces_to_the_reduced_model(elastic):
    dim, n, h = 2, (9, 7), 0.25
    over = {} if elastic else {"Lscale": 0.0}
    O1 = oracle.Problem(dim, n, h, _cf(1, **over))
    O3 = oracle.Problem(dim, n, h, _cf(3, **over))
    c, eta, u = _state3(dim, n, 3, u_amp=0.01 if elastic else 0.0)
    e = eta[0]
    cb = float(c.mean())
    X1 = O1.interleave(c, e, u)
    X3 = O3.interleave(c, np.stack([e, e, e]), u)
    E1, p1 = O1.energy(X1, cb, parts=True)
    E3, p3 = O3.energy(X3, cb, parts=True)
    assert np.allclose(p3, p1, rtol=1e-13, atol=1e-12 * np.abs(p1).max())
    assert E3 == pytest.approx(E1, rel=1e-13)


@pytest.mark.parametrize("j", [0, 1, 2])
def test_gibbs_energy_has_the_four_sublattice_symmetry(j):
    """The four FCC sublattices are equivalent, so E_G(c, eta_1..eta_4) is invariant
    under exchanging any eta_j with eta_4 = 4 - sum (the three pairings phi_i then
    permute and change sign in pairs).  Pins the phi_i and the sublattice sum; the
    gradient energy (eta_1..eta_3 only) is left out."""
    dim, n, h = 2, (7, 6), 0.25
    O3 = oracle.Problem(dim, n, h, _cf(3, Lscale=0.0))
    c, eta, _ = _state3(dim, n, 51)
    eta = 1.0 + 3.0 * (eta - 0.1)  # spread the order parameters: |eta_i - 1| up to 0.15
    e4 = 4.0 - eta.sum(axis=0)
    swapped = eta.copy()
    swapped[j] = e4
    _, pa = O3.energy(O3.interleave(c, eta), 0.0, parts=True)
    _, pb = O3.energy(O3.interleave(c, swapped), 0.0, parts=True)
    assert pb[0] == pytest.approx(pa[0], rel=1e-13)
    assert pb[1] == pytest.approx(pa[1], rel=1e-13)
    # and the energy does depend on the order parameters individually
    _, pc = O3.energy(O3.interleave(c, eta[[0, 0, 2]]), 0.0, parts=True)
    assert abs(pc[0] - pa[0]) > 1e-6 * abs(pa[0])


@pytest.mark.parametrize("S_order", [10, 0])
def test_dvd_derivative_reduces_to_the_reduced_model(S_order):
    dim, n, h = 2, (8, 6), 0.25
    O1 = oracle.Problem(dim, n, h, _cf(1, S=S_order))
    O3 = oracle.Problem(dim, n, h, _cf(3, S=S_order))
    c0, eta0, u0 = _state3(dim, n, 5, u_amp=0.01)
    c1, eta1, u1 = _state3(dim, n, 6, u_amp=0.01)
    cb = float(c0.mean())
    a1 = O1.interleave(c1, eta1[0], u1)
    a0 = O1.interleave(c0, eta0[0], u0)
    b1 = O3.interleave(c1, np.stack([eta1[0]] * 3), u1)
    b0 = O3.interleave(c0, np.stack([eta0[0]] * 3), u0)
    # the exact quotient (Psi(y1) - Psi(y0)) / (y1 - y0) cancels digits when y1 and y0
    # are close, and the two implementations round their logarithms differently
    tol = 1e-12 if S_order > 0 else 1e-10
    for which in (1, 2, 4, 8):
        gc1, ge1 = O1.dvd_G(a1, a0, cb, which)
        gc3, ge3 = O3.dvd_G(b1, b0, cb, which)
        sc = max(np.abs(gc1).max(), 1e-300)
        assert np.abs(gc3 - gc1).max() <= tol * sc, which
        se = max(np.abs(ge1).max(), 1e-300)
        assert np.abs(ge3.sum(axis=0) - ge1).max() <= tol * se + 1e-14, which
        # the three order parameters stay symmetric
        assert np.abs(ge3[0] - ge3[1]).max() <= 1e-12 * se + 1e-14
        assert np.abs(ge3[0] - ge3[2]).max() <= 1e-12 * se + 1e-14


def test_discrete_chain_rule_exact_quotients():
    """sum_p [G_c dc + sum_j G_eta_j deta_j] h^d = E(X1) - E(X0) (no elasticity,
    exact Psi quotients); the local terms (G^1 + G^2) also pointwise."""
    dim, n, h = 2, (8, 7), 0.25
    O3 = oracle.Problem(dim, n, h, _cf(3, S=0, Lscale=0.0))
    c0, eta0, _ = _state3(dim, n, 11)
    c1, eta1, _ = _state3(dim, n, 12)
    X0 = O3.interleave(c0, eta0)
    X1 = O3.interleave(c1, eta1)
    gc, ge = O3.dvd_G(X1, X0, 0.0, 15)
    lhs = (np.sum(gc * (c1 - c0)) + np.sum(ge * (eta1 - eta0))) * h ** dim
    E1, p1 = O3.energy(X1, 0.0, parts=True)
    E0, p0 = O3.energy(X0, 0.0, parts=True)
    assert lhs == pytest.approx(E1 - E0, rel=1e-9, abs=1e-12 * abs(E0))
    # local terms point by point: single-point energies from a one-point grid
    gc3, ge3 = O3.dvd_G(X1, X0, 0.0, 3)
    P1 = oracle.Problem(1, (1,), h, _cf(3, S=0, Lscale=0.0))
    for p in range(0, c0.size, 7):
        y1 = P1.interleave(np.array([c1[p]]), eta1[:, p:p + 1])
        y0 = P1.interleave(np.array([c0[p]]), eta0[:, p:p + 1])
        _, q1 = P1.energy(y1, 0.0, parts=True)
        _, q0 = P1.energy(y0, 0.0, parts=True)
        dE = (q1[0] + q1[1] - q0[0] - q0[1]) / h
        dG = gc3[p] * (c1[p] - c0[p]) + np.dot(ge3[:, p], eta1[:, p] - eta0[:, p])
        assert dG == pytest.approx(dE, rel=1e-9, abs=1e-13)


@pytest.mark.parametrize("dim,n", [(2, (5, 4)), (1, (7,))])
def test_jacobian_matches_central_differences(dim, n):
    h, dt = 0.25, 0.05
    O3 = oracle.Problem(dim, n, h, _cf(3))
    c0, eta0, u0 = _state3(dim, n, 21, u_amp=0.01)
    c1, eta1, u1 = _state3(dim, n, 22, u_amp=0.01)
    cb = float(c0.mean())
    X0 = O3.interleave(c0, eta0, u0)
    X1 = O3.interleave(c1, eta1, u1)
    for mode in (0, 1):
        J = O3.jacobian_scipy(X1, X0, cb, dt, mode).toarray()
        Jfd = np.zeros_like(J)
        for i in range(X1.size):
            step = 1e-6 * max(1.0, abs(X1[i]))
            Xp, Xm = X1.copy(), X1.copy()
            Xp[i] += step
            Xm[i] -= step
            Jfd[:, i] = (O3.residual(Xp, X0, cb, dt, mode) - O3.residual(Xm, X0, cb, dt, mode)) / (2 * step)
        scale = np.abs(J).max()
        if mode == 0:
            assert np.abs(J - Jfd).max() <= 1e-6 * scale
        else:
            # the displacement-only system: c and eta rows are identity rows, the
            # displacement rows are the derivative of the displacement residual
            rows = np.arange(X1.size).reshape(-1, O3.nf)
            fixed, disp = rows[:, :O3.ku].ravel(), rows[:, O3.ku:].ravel()
            assert np.array_equal(J[fixed], np.eye(X1.size)[fixed])
            assert np.abs(J[disp] - Jfd[disp]).max() <= 1e-6 * scale


def test_symmetric_steps_follow_the_reduced_model():
    dim, n, h = 2, (12, 10), 0.25
    op = S.options(sub=(2, 2), overlap=1, newton_rtol=1e-12)
    O1 = oracle.Problem(dim, n, h, _cf(1), op)
    O3 = oracle.Problem(dim, n, h, _cf(3), op)
    c, e = S.initial_fields(dim, n, 0.18, 4)
    rc1, X1, inf1, e01 = O1.simulate(c, e, 2)
    rc3, X3, inf3, e03 = O3.simulate(c, np.stack([e, e, e]), 2)
    assert rc1 == 0 and rc3 == 0
    ca, ea, ua = O1.split(X1)
    cb_, eb, ub = O3.split(X3)
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(cb_, ca) <= 1e-9 and rel(ub, ua) <= 1e-8
    for j in range(3):
        assert rel(eb[j], ea) <= 1e-9
    assert np.abs(eb[0] - eb[1]).max() <= 1e-12 and np.abs(eb[0] - eb[2]).max() <= 1e-12
    assert e03 == pytest.approx(e01, rel=1e-12)
    for a, b in zip(inf1, inf3):
        assert b["energy"] == pytest.approx(a["energy"], rel=1e-10)


def test_asymmetric_steps_conserve_mass_and_dissipate_energy():
    dim, n, h = 2, (12, 12), 0.25
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy")
    O3 = oracle.Problem(dim, n, h, _cf(3), op)
    c, eta, _ = _state3(dim, n, 31)
    rc, X, infos, e0 = O3.simulate(c, eta, 3)
    assert rc == 0
    m0 = c.sum() * h ** dim
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    _, eF, _ = O3.split(X)
    assert np.abs(eF[0] - eF[1]).max() > 1e-6  # the order parameters evolve apart


def test_permuting_the_order_parameters_permutes_the_step():
    dim, n, h = 2, (10, 8), 0.25
    op = S.options(sub=(2, 2), overlap=1, newton_rtol=1e-12)
    O3 = oracle.Problem(dim, n, h, _cf(3), op)
    c, eta, _ = _state3(dim, n, 41)
    rc, X, _, _ = O3.simulate(c, eta, 1)
    perm = [2, 0, 1]
    rcp, Xp, _, _ = O3.simulate(c, eta[perm], 1)
    assert rc == 0 and rcp == 0
    cA, eA, uA = O3.split(X)
    cB, eB, uB = O3.split(Xp)
    assert np.linalg.norm(cB - cA) <= 1e-9 * np.linalg.norm(cA)
    assert np.linalg.norm(eB - eA[perm]) <= 1e-9 * np.linalg.norm(eA)
    assert np.linalg.norm(uB - uA) <= 1e-8 * np.linalg.norm(uA)


def test_three_order_parameters_with_neumann_boundaries():
    """The two next rows together: three order parameters on a grid with
    homogeneous Neumann boundaries conserve mass, obey the energy law, and keep
    the permutation symmetry of the order parameters."""
    dim, n, h = 2, (10, 9), 0.25
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy", newton_rtol=1e-12)
    O3 = oracle.Problem(dim, n, h, _cf(3), op, neumann=True)
    c, eta, _ = _state3(dim, n, 61)
    rc, X, infos, e0 = O3.simulate(c, eta, 3)
    assert rc == 0
    m0 = c.sum() * h ** dim
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    perm = [1, 2, 0]
    rcp, Xp, _, _ = O3.simulate(c, eta[perm], 3)
    assert rcp == 0
    _, eA, _ = O3.split(X)
    _, eB, _ = O3.split(Xp)
    assert np.linalg.norm(eB - eA[perm]) <= 1e-8 * np.linalg.norm(eA)
