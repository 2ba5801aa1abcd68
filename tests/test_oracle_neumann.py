"""Pins of the oracle's homogeneous Neumann boundaries (Eq. boundaryequ; row f3).

On the cell-centred grid of Sec. 3 the Neumann conditions are mirror ghost
cells, so the fixed standard is the periodic problem on the mirrored domain:
a state on n cells, reflected across each boundary face into a periodic grid
of 2n cells, stays mirror-symmetric, and its first n cells are the Neumann
solution.  Checked for energies (the mirrored energy is 2^d times the Neumann
one) and for whole NKS steps in 1-D and 2-D without elasticity.  The traction-
free displacement rows are the exact variation of the discrete elastic energy:
-F_u equals its finite differences (on periodic grids too, where it is the
divergence form).  Mass conservation, the energy law and the Jacobian against
central differences hold with elasticity.  The projection removes the whole null
space of the traction-free displacement block (its dimension counted by an SVD),
so the displacement does not depend on the Schwarz decomposition.
"""
import numpy as np
import pytest

import oracle
import synthetic as S


def _cf():
    return S.coefficients(Lscale=0.0)


def _mirror(f, n):
    """Reflect a field on n cells (x-fastest) across every boundary face into 2n cells."""
    a = np.asarray(f).reshape(tuple(reversed(n)))
    for ax in range(a.ndim):
        a = np.concatenate([a, np.flip(a, axis=ax)], axis=ax)
    return a.reshape(-1)


def _restrict(f, n):
    """The first n cells of every axis of a mirrored field on 2n cells."""
    big = tuple(reversed([2 * m for m in n]))
    a = np.asarray(f).reshape(big)
    return a[tuple(slice(0, m) for m in reversed(n))].reshape(-1)


@pytest.mark.parametrize("dim,n", [(1, (14,)), (2, (9, 7))])
def test_energy_of_the_mirrored_state(dim, n):
    c, e = S.initial_fields(dim, n, 0.18, 3, c_amp=0.02, eta_amp=0.05)
    On = oracle.Problem(dim, n, 0.25, _cf(), neumann=True)
    Op = oracle.Problem(dim, tuple(2 * m for m in n), 0.25, _cf())
    En, pn = On.energy(On.interleave(c, e), 0.0, parts=True)
    Ep, pp = Op.energy(Op.interleave(_mirror(c, n), _mirror(e, n)), 0.0, parts=True)
    assert np.allclose(pp, 2 ** dim * pn, rtol=1e-12, atol=1e-12 * abs(En))
    # the Neumann gradient energy has no boundary-face terms: it differs from the
    # periodic energy of the same (unmirrored) state
    Oq = oracle.Problem(dim, n, 0.25, _cf())
    _, pq = Oq.energy(Oq.interleave(c, e), 0.0, parts=True)
    assert abs(pq[3] - pn[3]) > 1e-6 * abs(pn[3])


@pytest.mark.parametrize("dim,n,sub", [(1, (16,), (2,)), (2, (10, 8), (2, 2))])
def test_steps_equal_the_mirrored_periodic_steps(dim, n, sub):
    op = S.options(sub=sub, overlap=1, newton_rtol=1e-12)
    c, e = S.initial_fields(dim, n, 0.18, 5, c_amp=0.02, eta_amp=0.05)
    On = oracle.Problem(dim, n, 0.25, _cf(), op, neumann=True)
    n2 = tuple(2 * m for m in n)
    Op = oracle.Problem(dim, n2, 0.25, _cf(), dict(op, sub=tuple(2 * s for s in sub)))
    rcn, Xn, infn, en0 = On.simulate(c, e, 3, dt_replay=[0.01, 0.02, 0.04])
    rcp, Xp, infp, ep0 = Op.simulate(_mirror(c, n), _mirror(e, n), 3, dt_replay=[0.01, 0.02, 0.04])
    assert rcn == 0 and rcp == 0
    cn, en, _ = On.split(Xn)
    cp, ep, _ = Op.split(Xp)
    assert np.linalg.norm(_restrict(cp, n) - cn) <= 1e-9 * np.linalg.norm(cn)
    assert np.linalg.norm(_restrict(ep, n) - en) <= 1e-9 * np.linalg.norm(en)
    for a, b in zip(infn, infp):
        assert b["energy"] == pytest.approx(2 ** dim * a["energy"], rel=1e-10)


def test_mass_and_energy_law_with_neumann_boundaries():
    dim, n = 2, (12, 10)
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy")
    O = oracle.Problem(dim, n, 0.25, _cf(), op, neumann=True)
    c, e = S.initial_fields(dim, n, 0.18, 7, c_amp=0.02, eta_amp=0.05)
    rc, X, infos, e0 = O.simulate(c, e, 4)
    assert rc == 0
    m0 = c.sum() * 0.25 ** dim
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)


def test_jacobian_matches_central_differences_with_neumann_boundaries():
    dim, n, dt = 2, (5, 4), 0.05
    O = oracle.Problem(dim, n, 0.25, _cf(), neumann=True)
    c0, e0 = S.initial_fields(dim, n, 0.18, 8, c_amp=0.03, eta_amp=0.05)
    c1, e1 = S.initial_fields(dim, n, 0.18, 9, c_amp=0.03, eta_amp=0.05)
    X0, X1 = O.interleave(c0, e0), O.interleave(c1, e1)
    cb = float(c0.mean())
    J = O.jacobian_scipy(X1, X0, cb, dt).toarray()
    fd = np.zeros_like(J)
    for i in range(X1.size):
        xp, xm = X1.copy(), X1.copy()
        xp[i] += 1e-6
        xm[i] -= 1e-6
        fd[:, i] = (O.residual(xp, X0, cb, dt) - O.residual(xm, X0, cb, dt)) / 2e-6
    assert np.abs(J - fd).max() <= 1e-6 * np.abs(J).max()


@pytest.mark.parametrize("neumann", [True, False])
def test_displacement_rows_are_the_variation_of_the_elastic_energy(neumann):
    """F_u = -dE_3/du (per unit volume): the traction-free rows under Neumann, the
    divergence form on periodic grids."""
    dim, n, h = 2, (6, 5), 0.25
    O = oracle.Problem(dim, n, h, S.coefficients(), neumann=neumann)
    c, e = S.initial_fields(dim, n, 0.18, 12, c_amp=0.03, eta_amp=0.05)
    u = 0.01 * (2.0 * S.uniform01(13, dim * c.size).reshape(dim, c.size) - 1.0)
    cb = float(c.mean())
    X = O.interleave(c, e, u)
    F = O.residual(X, X, cb, 1.0, mode=1)
    Fu = O.split(F)[2]
    grad = np.zeros_like(u)
    for I in range(dim):
        for p in range(c.size):
            up, um = u.copy(), u.copy()
            up[I, p] += 1e-6
            um[I, p] -= 1e-6
            ep = O.energy(O.interleave(c, e, up), cb, parts=True)[1][2]
            em = O.energy(O.interleave(c, e, um), cb, parts=True)[1][2]
            grad[I, p] = (ep - em) / 2e-6 / h ** dim
    assert np.abs(Fu + grad).max() <= 1e-6 * np.abs(grad).max()


def test_elastic_steps_with_neumann_boundaries():
    dim, n = 2, (12, 10)
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy")
    O = oracle.Problem(dim, n, 0.25, S.coefficients(), op, neumann=True)
    c, e = S.initial_fields(dim, n, 0.18, 14, c_amp=0.02, eta_amp=0.05)
    rc, X, infos, e0 = O.simulate(c, e, 3)
    assert rc == 0
    m0 = c.sum() * 0.25 ** dim
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    dt = 0.05
    c0, e0_ = S.initial_fields(dim, (5, 4), 0.18, 15, c_amp=0.03, eta_amp=0.05)
    Os = oracle.Problem(dim, (5, 4), 0.25, S.coefficients(), neumann=True)
    u0 = 0.01 * (2.0 * S.uniform01(16, dim * c0.size).reshape(dim, c0.size) - 1.0)
    X0 = Os.interleave(c0, e0_, u0)
    X1 = X0 * (1.0 + 0.01 * np.sin(np.arange(X0.size)))
    cb = float(c0.mean())
    for mode in (0, 1):
        J = Os.jacobian_scipy(X1, X0, cb, dt, mode).toarray()
        fd = np.zeros_like(J)
        for i in range(X1.size):
            xp, xm = X1.copy(), X1.copy()
            xp[i] += 1e-6
            xm[i] -= 1e-6
            fd[:, i] = (Os.residual(xp, X0, cb, dt, mode) - Os.residual(xm, X0, cb, dt, mode)) / 2e-6
        rows = np.arange(X1.size).reshape(-1, Os.nf)
        check = rows.ravel() if mode == 0 else rows[:, Os.ku:].ravel()
        assert np.abs(J[check] - fd[check]).max() <= 1e-6 * np.abs(J).max(), mode


def _displacement_block(O, X, cb):
    """J_uu of the displacement-only system (mode 1) as a dense matrix, components
    one after another"""
    J = O.jacobian_scipy(X, X, cb, 1.0, mode=1).toarray()
    idx = np.concatenate([np.arange(O.N) * O.nf + O.ku + I for I in range(O.dim)])
    return J[np.ix_(idx, idx)]


@pytest.mark.parametrize("dim,n,rot", [(2, (12, 10), 1), (2, (11, 10), 0), (2, (9, 7), 0), (3, (6, 4, 4), 3),
                                       (3, (5, 4, 4), 1)])
def test_projection_removes_the_null_space_of_the_traction_free_block(dim, n, rot):
    """The displacement block under traction-free boundaries is singular: besides
    the d translations, one discrete rotation for every pair of axes that both have
    an even number of cells (rot) has zero strain.  Counted by the SVD of the
    oracle's block (no mode written out here), and the projected Schwarz output
    z = P M^-1 r has no component in that null space."""
    op = S.options(sub=tuple([2] * dim), overlap=1)
    O = oracle.Problem(dim, n, 0.25, S.coefficients(), op, neumann=True)
    c, e = S.initial_fields(dim, n, 0.18, 21, c_amp=0.03, eta_amp=0.05)
    u = 0.01 * (2.0 * S.uniform01(22, dim * c.size).reshape(dim, c.size) - 1.0)
    X = O.interleave(c, e, u)
    cb = float(c.mean())
    A = _displacement_block(O, X, cb)
    U, s, Vt = np.linalg.svd(A)
    null = Vt[s <= 1e-12 * s[0]]
    assert len(null) == dim + rot
    r = np.sin(np.arange(X.size) * 0.7)
    rc, z = O.precond_apply(X, X, cb, 1.0, r)
    assert rc == 0
    zu = np.concatenate(list(O.split(z)[2]))
    assert np.abs(null @ zu).max() <= 1e-12 * np.linalg.norm(zu)


def test_elastic_neumann_steps_do_not_depend_on_the_decomposition():
    """With the whole null space projected out, the displacement after a few steps
    is fixed by the equations alone: two Schwarz decompositions agree to 1e-9
    (an unprojected rotation would be left where each Krylov process put it)."""
    dim, n = 2, (16, 12)
    c, e = S.initial_fields(dim, n, 0.18, 23, c_amp=0.03, eta_amp=0.05)
    out = []
    for sub in [(2, 2), (4, 3)]:
        O = oracle.Problem(dim, n, 0.25, S.coefficients(), S.options(sub=sub, overlap=1, newton_rtol=1e-12),
                           neumann=True)
        rc, X, infos, e0 = O.simulate(c, e, 3, dt_replay=[0.01] * 3)
        assert rc == 0
        out.append(O.split(X))
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(out[0][0], out[1][0]) <= 1e-9
    for I in range(dim):
        assert rel(out[0][2][I], out[1][2][I]) <= 1e-9, I
