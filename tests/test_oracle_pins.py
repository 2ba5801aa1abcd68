"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with an
independent statement (App. A's four-sublattice construction, the DVD identity
of Eq. DVD, summation by parts, the closed form of Psi_S's remainder, a
Fourier analysis of the linearised scheme, finite differences, the defining
property of ILU(0), a dense direct solve, conservation and symmetry laws).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _psi(z):
    return z * math.log(z) + (1 - z) * math.log(1 - z)


# ---------------------------------------------------------------------------
# constants and coefficient inputs
# ---------------------------------------------------------------------------

def test_dimensionless_constants_follow_printed_values():
    dE, Lm = GOLD["Delta_E_J_per_m3"]["value"], GOLD["length_scale_m"]["value"]
    assert S.COEFFS["gamma_c"] == pytest.approx(GOLD["gamma_c_J_per_m"]["value"] / (dE * Lm ** 2), rel=1e-14)
    assert S.COEFFS["gamma_eta"] == pytest.approx(GOLD["gamma_eta_J_per_m"]["value"] / (dE * Lm ** 2), rel=1e-14)
    theta = 8.314462618 * GOLD["T_K"]["value"] / (GOLD["V_m_m3_per_mol"]["value"] * dE)
    assert S.COEFFS["theta"] == pytest.approx(theta, rel=1e-14)
    assert S.COEFFS["eps0"] == GOLD["eps0"]["value"]
    assert S.COEFFS["kappa"] == GOLD["kappa"]["value"]
    assert S.COEFFS["S"] == GOLD["S"]["value"]
    assert S.OPTS["dt_init"] == GOLD["dt_1"]["value"] and S.OPTS["zeta"] == GOLD["zeta"]["value"]
    assert S.OPTS["dt_min"] == GOLD["dt_min"]["value"] and S.OPTS["dt_max"] == GOLD["dt_max"]["value"]


def test_stored_gibbs_coefficients_put_wells_where_printed():
    """The stored (L0, U1, U4) make the printed wells stationary and common-tangent."""
    from oracle import fit_coefficients as fc
    cf = S.coefficients(C11=0.0, C12=0.0, C44=0.0, gamma_c=0.0, gamma_eta=0.0)
    r = fc.conditions(cf)
    assert np.all(np.abs(r) < 1e-5), r
    # the ordered well is a minimum along eta at fixed c
    c, e = GOLD["well_ordered"]["c"], GOLD["well_ordered"]["eta"]
    f = [fc.gibbs_density(c, e + s, cf) for s in (-1e-3, 0.0, 1e-3)]
    assert f[0] > f[1] and f[2] > f[1]


# ---------------------------------------------------------------------------
# Gibbs energy: App. A construction E_dis + E_ord(eta_i) - E_ord(1,1,1)
# ---------------------------------------------------------------------------

def _gibbs_appendix_A(cf, c, eta):
    """App. A with eta_1 = eta_2 = eta_3 = eta and eta_4 = 4 - 3 eta (sum eta_i = 4)."""
    th = cf["theta"]
    L, U1, U4 = cf["L"], cf["U1"], cf["U4"]

    def e_ord(etas):
        e1, e2, e3 = etas[:3]
        phis = [1 - (e1 + e2) / 2, 1 - (e1 + e3) / 2, 1 - (e2 + e3) / 2]
        sp2 = sum(p * p for p in phis)
        ref = 6 * U1 * c * c * sp2
        ideal = th / 4 * sum(_psi(c * ei) for ei in etas)
        ex = -2 * U1 * c * c * sp2 + 12 * U4 * (1 - 2 * c) * c * c * sp2 - 48 * U4 * c ** 3 * phis[0] * phis[1] * phis[2]
        return ref + ideal + ex

    e_dis = cf["dE0"] * c + th * _psi(c) + c * (1 - c) * sum(L[i] * (2 * c - 1) ** i for i in range(4))
    return e_dis + e_ord([eta, eta, eta, 4 - 3 * eta]) - e_ord([1.0, 1.0, 1.0, 1.0])


@pytest.mark.parametrize("w", [0.0, 1.0])
def test_homogeneous_energy_is_appendix_A_gibbs_plus_main_text_psi(w):
    cf = S.coefficients(L=[-150.0, 20.0, -8.0, 3.0], U1=-19.0, U4=4.0, dE0=0.7, w_psi=w,
                        C11=0.0, C12=0.0, C44=0.0)
    P = oracle.Problem(1, (3,), 1.0, cf)
    rng = np.random.default_rng(3)
    for _ in range(20):
        c = rng.uniform(0.05, 0.24)
        eta = rng.uniform(0.01, 0.99)
        X = P.interleave(np.full(3, c), np.full(3, eta))
        dens = P.energy(X, c) / 3.0
        # App. A cancels theta Psi(c); the main text's E_2 keeps it with weight w
        ref = _gibbs_appendix_A(cf, c, eta) + w * cf["theta"] * _psi(c)
        assert dens == pytest.approx(ref, rel=1e-13, abs=1e-12)


def test_appendix_B_chemical_potential_matches_energy_derivative():
    """App. B's dE_G/dc = M0 + M1 c + M2 c^2 + M3 c^3 + M4 c^4 + RT/4 phi'_c (with w = 0)
    against a central difference of the oracle's energy density."""
    cf = S.coefficients(L=[-150.0, 20.0, -8.0, 3.0], U1=-19.0, U4=4.0, dE0=0.7, w_psi=0.0,
                        C11=0.0, C12=0.0, C44=0.0)
    L, U1, U4, th = cf["L"], cf["U1"], cf["U4"], cf["theta"]
    P = oracle.Problem(1, (3,), 1.0, cf)

    def dens(c, e):
        return P.energy(P.interleave(np.full(3, c), np.full(3, e)), c) / 3.0

    for c, e in [(0.12, 0.3), (0.2, 0.05), (0.17, 0.8)]:
        phi = 1 - e
        M0 = cf["dE0"] + L[0] - L[1] + L[2] - L[3]
        M1 = -(2 * L[0] - 6 * L[1] + 10 * L[2] - 14 * L[3]) + 24 * U1 * phi ** 2 + 72 * U4 * phi ** 2
        M2 = -(6 * L[1] - 24 * L[2] + 54 * L[3]) - 216 * U4 * phi ** 2 - 144 * U4 * phi ** 3
        M3 = -(16 * L[2] - 80 * L[3])
        M4 = -40 * L[3]
        dpsi = lambda z: math.log(z / (1 - z))
        phic = 3 * e * dpsi(c * e) + (4 - 3 * e) * dpsi(c * (4 - 3 * e))
        mu_B = M0 + M1 * c + M2 * c ** 2 + M3 * c ** 3 + M4 * c ** 4 + th / 4 * phic
        M5 = -(24 * U1 * c * c + 72 * U4 * (1 - 2 * c) * c * c)
        M6 = 144 * U4 * c ** 3
        phie = 3 * c * dpsi(c * e) - 3 * c * dpsi(c * (4 - 3 * e))
        nu_B = M5 * phi + M6 * phi ** 2 + th / 4 * phie
        s = 1e-6
        mu_fd = (dens(c + s, e) - dens(c - s, e)) / (2 * s)
        nu_fd = (dens(c, e + s) - dens(c, e - s)) / (2 * s)
        assert mu_fd == pytest.approx(mu_B, rel=1e-7, abs=1e-7)
        assert nu_fd == pytest.approx(nu_B, rel=1e-7, abs=1e-7)


# ---------------------------------------------------------------------------
# Psi_S (Sec. 3): closed form of the truncated quotient
# ---------------------------------------------------------------------------

def test_psiS_matches_exact_quotient_within_taylor_remainder():
    rng = np.random.default_rng(0)
    Sord = 10
    for _ in range(400):
        yb = rng.uniform(0.003, 0.95)
        m = min(yb, 1 - yb)
        r = rng.uniform(0.01, 0.9)
        de = r * m * rng.choice([-1, 1])
        y1, y2 = yb - de, yb + de
        exact = (_psi(y1) - _psi(y2)) / (y1 - y2)
        approx = oracle.psi_quot(y1, y2, Sord)
        bound = r ** (2 * Sord) / (2 * Sord * (2 * Sord + 1) * (1 - r * r))
        rounding = 1e-15 * (abs(_psi(y1)) + abs(_psi(y2))) / abs(y1 - y2) * 8 + 1e-14 * abs(exact)
        assert abs(approx - exact) <= bound + rounding, (y1, y2, approx, exact, bound)
        # the oracle's S <= 0 mode is the exact quotient of Eq. D2
        assert oracle.psi_quot(y1, y2, 0) == pytest.approx(exact, rel=1e-12, abs=1e-12)


def test_psiS_reduces_to_log_derivative_at_equal_arguments():
    for y in (0.01, 0.2, 0.5, 0.9):
        assert oracle.psi_quot(y, y, 10) == pytest.approx(math.log(y / (1 - y)), rel=1e-15, abs=1e-15)
        # d/dy1 Psi_S[y, y] = Psi''(y)/2
        assert oracle.psi_quot_d1(y, y, 10) == pytest.approx(0.5 * (1 / y + 1 / (1 - y)), rel=1e-14)


def test_psiS_first_argument_derivative_matches_difference_quotient():
    rng = np.random.default_rng(1)
    for _ in range(100):
        y1 = rng.uniform(0.01, 0.9)
        y2 = y1 * rng.uniform(0.7, 1.3)
        s = 1e-7 * y1
        fd = (oracle.psi_quot(y1 + s, y2, 10) - oracle.psi_quot(y1 - s, y2, 10)) / (2 * s)
        assert oracle.psi_quot_d1(y1, y2, 10) == pytest.approx(fd, rel=2e-6, abs=1e-6)


# ---------------------------------------------------------------------------
# DVD identity (Eq. DVD, Eq. localsum1-2): h^d sum G^K . dV = dE_K
# ---------------------------------------------------------------------------

def _pair(P, dim, n, seed, du=0.0):
    c0, e0, u0 = S.random_fields(dim, n, seed, u_amp=du)
    rng = np.random.default_rng(seed + 100)
    c1 = c0 * (1 + 0.05 * rng.uniform(-1, 1, c0.shape))
    e1 = e0 * (1 + 0.05 * rng.uniform(-1, 1, e0.shape))
    u1 = u0 * (1 + 0.05 * rng.uniform(-1, 1, u0.shape))
    return P.interleave(c1, e1, u1), P.interleave(c0, e0, u0), (c1, e1, c0, e0)


@pytest.mark.parametrize("dim,n", [(1, (11,)), (2, (7, 6)), (3, (5, 4, 6))])
@pytest.mark.parametrize("term,part", [(1, 0), (2, 1), (8, 3)])
def test_dvd_identity_exact_quotient(dim, n, term, part):
    cf = S.coefficients(S=0, C11=0.0, C12=0.0, C44=0.0, L=[-150.0, 20.0, -8.0, 3.0], U4=4.0, dE0=0.3)
    P = oracle.Problem(dim, n, 0.25, cf)
    X1, X0, (c1, e1, c0, e0) = _pair(P, dim, n, 7 + dim)
    cb = c0.mean()
    gc, ge = P.dvd_G(X1, X0, cb, which=term)
    lhs = (np.sum(gc * (c1 - c0)) + np.sum(ge * (e1 - e0))) * 0.25 ** dim
    dE = P.energy(X1, cb, parts=True)[1][part] - P.energy(X0, cb, parts=True)[1][part]
    assert lhs == pytest.approx(dE, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("dim,n", [(2, (6, 8)), (3, (4, 6, 5))])
def test_dvd_identity_elastic_term_at_equilibrium(dim, n):
    """G^3 satisfies the identity when u is in equilibrium at both levels (Eq. localsum1)."""
    cf = S.coefficients()
    op = S.options(sub=(1, 1, 1), overlap=0, subsolver=0, u0_rtol=1e-14, u0_atol=1e-15, u0_maxit=30,
                   gmres_maxit=2000, gmres_rtol=1e-10)
    P = oracle.Problem(dim, n, 0.25, cf, op)
    _, _, (c1, e1, c0, e0) = _pair(P, dim, n, 21)
    cb = c0.mean()
    c1 = c1 - c1.mean() + cb          # same mass at both levels
    rc0, X0, _ = P.equilibrate(P.interleave(c0, e0), cb)
    rc1, X1, _ = P.equilibrate(P.interleave(c1, e1), cb)
    assert rc0 == 0 and rc1 == 0
    gc, _ = P.dvd_G(X1, X0, cb, which=4)
    lhs = np.sum(gc * (c1 - c0)) * 0.25 ** dim
    dE = P.energy(X1, cb, parts=True)[1][2] - P.energy(X0, cb, parts=True)[1][2]
    assert lhs == pytest.approx(dE, rel=1e-9, abs=1e-12)
    # <eps, eps^el> = 0 at equilibrium (Theorem 3.1 proof) <=> E3 = -<eps0 (c - cbar) tr sigma>/2
    F = P.residual(X1, X1, cb, 1.0, mode=1)
    assert np.max(np.abs(F)) < 1e-9 * max(1.0, np.max(np.abs(P.residual(P.interleave(c1, e1), P.interleave(c1, e1), cb, 1.0, mode=1))))


# ---------------------------------------------------------------------------
# flux operator: summation by parts (Eq. summation) and semi-positivity (Eq. neq:02)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(1, (9,)), (2, (6, 7)), (3, (4, 5, 6))])
def test_summation_by_parts_and_mass_telescoping(dim, n):
    cf = S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    P = oracle.Problem(dim, n, 0.25, cf)
    X1, X0, (c1, e1, c0, e0) = _pair(P, dim, n, 31)
    cb, dt = c0.mean(), 0.07
    F = P.residual(X1, X0, cb, dt)[0::P.nf]
    G, _ = P.dvd_G(X1, X0, cb)
    # F_c = (c1 - c0)/dt - D M D G  =>  A11 G := -D M D G = F_c - (c1 - c0)/dt
    AG = F - (c1 - c0) / dt
    shape = tuple(reversed(n))
    Gg, cg = G.reshape(shape), c0.reshape(shape)
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(G.shape)
    pg = phi.reshape(shape)
    mob = S.COEFFS["kappa"] * cg * (1 - cg)
    rhs = 0.0
    for J in range(dim):
        ax = dim - 1 - J
        Mh = 0.5 * (mob + np.roll(mob, -1, axis=ax))
        rhs += np.sum(Mh * (np.roll(pg, -1, axis=ax) - pg) * (np.roll(Gg, -1, axis=ax) - Gg)) / 0.25 ** 2
    lhs = np.sum(phi * AG)
    assert lhs == pytest.approx(rhs, rel=1e-10, abs=1e-10)
    assert np.sum(G * AG) >= -1e-10 * np.sum(np.abs(G * AG))
    # telescoping: sum_i (D M D G)_i = 0, so the mass moves only by sum (c1 - c0)
    assert abs(np.sum(AG)) <= 1e-11 * np.sum(np.abs(AG))


# ---------------------------------------------------------------------------
# steady states
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n", [(2, (8, 8)), (3, (6, 6, 6))])
def test_constant_disordered_state_is_exact_steady_solution(dim, n):
    """c = const, eta = 1, u = 0: F = 0 exactly for any dt; Newton takes no iteration."""
    P = oracle.Problem(dim, n, 0.25, S.coefficients(), S.options(sub=(2, 2, 2)))
    N = int(np.prod(n))
    X = P.interleave(np.full(N, 0.17), np.full(N, 1.0))
    for dt in (0.01, 2.0):
        F = P.residual(X, X, 0.17, dt)
        assert np.all(F == 0.0)
        rc, X1, info = P.newton_step(X, 0.17, dt)
        assert rc == 0 and info["newton_its"] == 0 and np.array_equal(X1, X)


# ---------------------------------------------------------------------------
# linear growth rate of one Fourier mode (linearised NSOA-1 is the trapezoidal rule)
# ---------------------------------------------------------------------------

def _B_h(cf, s):
    """Elastic symbol: u in equilibrium with a composition mode of symbol s_J = sin(k_J h)/h;
    returns the coefficient B with G^3_c = B * c_hat (cubic Hooke law, eigenstrain eps0 c I)."""
    d = len(s)
    C11, C12, C44, e0 = cf["C11"], cf["C12"], cf["C44"], cf["eps0"]
    lam = C11 + (d - 1) * C12
    A = np.zeros((d, d))
    for I in range(d):
        for K in range(d):
            if I == K:
                A[I, I] = C11 * s[I] ** 2 + C44 * sum(s[J] ** 2 for J in range(d) if J != I)
            else:
                A[I, K] = (C12 + C44) * s[I] * s[K]
    rhs = e0 * lam * np.asarray(s)
    v = np.linalg.lstsq(A, rhs, rcond=None)[0]
    return -e0 * lam * (np.dot(s, v) - d * e0)


@pytest.mark.parametrize("dim,n,kidx,field", [(2, (16, 16), (1, 2), "c"), (2, (16, 16), (3, 0), "eta"),
                                              (3, (8, 8, 8), (1, 1, 2), "c"), (1, (32,), (3,), "c")])
def test_linear_amplification_factor(dim, n, kidx, field):
    cf = S.coefficients()
    op = S.options(sub=(2, 2, 2), overlap=1, newton_rtol=1e-7, newton_atol=0.0, gmres_rtol=1e-7,
                   gmres_atol=1e-30, u0_rtol=1e-13, u0_atol=1e-30, u0_maxit=30)
    P = oracle.Problem(dim, n, 0.25, cf, op)
    h, cbar, dt, amp = 0.25, 0.18, 0.05, 1e-6
    grids = np.meshgrid(*[np.arange(m) for m in reversed(n)], indexing="ij")
    xs = list(reversed(grids))
    k = [2 * math.pi * kidx[J] / (n[J] * h) for J in range(dim)]
    mode = np.cos(sum(k[J] * xs[J] * h for J in range(dim))).reshape(-1)
    c = np.full(P.N, cbar) + (amp * mode if field == "c" else 0.0)
    eta = np.ones(P.N) + (amp * mode if field == "eta" else 0.0)
    rc, X0, _ = P.equilibrate(P.interleave(c, eta), cbar)
    assert rc == 0
    rc, X1, info = P.newton_step(X0, cbar, dt)
    assert rc == 0
    f = 0 if field == "c" else 1
    base = cbar if field == "c" else 1.0
    a0 = np.dot(X0[f::P.nf] - base, mode)
    a1 = np.dot(X1[f::P.nf] - base, mode)
    lam_h = sum(4 / h ** 2 * math.sin(k[J] * h / 2) ** 2 for J in range(dim))
    L, U1, U4, th, w = cf["L"], cf["U1"], cf["U4"], cf["theta"], cf["w_psi"]
    psi2 = 1 / cbar + 1 / (1 - cbar)
    if field == "c":
        M1 = -(2 * L[0] - 6 * L[1] + 10 * L[2] - 14 * L[3])
        M2 = -(6 * L[1] - 24 * L[2] + 54 * L[3])
        M3, M4 = -(16 * L[2] - 80 * L[3]), -40 * L[3]
        fcc = M1 + 2 * M2 * cbar + 3 * M3 * cbar ** 2 + 4 * M4 * cbar ** 3 + th * (w + 1) * psi2
        s = [math.sin(k[J] * h) / h for J in range(dim)]
        B = _B_h(cf, s) if dim > 0 else 0.0
        sigma = -cf["kappa"] * cbar * (1 - cbar) * lam_h * (fcc + cf["gamma_c"] * lam_h + B)
    else:
        M5 = -(24 * U1 * cbar ** 2 + 72 * U4 * (1 - 2 * cbar) * cbar ** 2)
        fee = -M5 + 3 * th * cbar ** 2 * psi2
        sigma = -(fee + 3 * cf["gamma_eta"] * lam_h)
    expect = (1 + dt * sigma / 2) / (1 - dt * sigma / 2)
    assert a1 / a0 == pytest.approx(expect, rel=2e-5, abs=1e-6)


# ---------------------------------------------------------------------------
# Jacobian against central differences; structural pattern size
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,nnz_pt", [(1, (7,), 22), (2, (5, 5), 64), (3, (5, 5, 5), 130)])
def test_jacobian_matches_central_differences(dim, n, nnz_pt):
    cf = S.coefficients()
    P = oracle.Problem(dim, n, 0.25, cf)
    X1, X0, (c1, e1, c0, e0) = _pair(P, dim, n, 41, du=0.01)
    cb, dt = c0.mean(), 0.3
    J = P.jacobian_scipy(X1, X0, cb, dt).toarray()
    assert np.count_nonzero(P.jacobian(X1, X0, cb, dt)[2] != 0.0) <= P.N * nnz_pt
    assert len(P.jacobian(X1, X0, cb, dt)[2]) == P.N * nnz_pt
    n_unk = len(X1)
    Jfd = np.zeros_like(J)
    for j in range(n_unk):
        s = 1e-6 * max(abs(X1[j]), 1e-3)
        Xp, Xm = X1.copy(), X1.copy()
        Xp[j] += s
        Xm[j] -= s
        Jfd[:, j] = (P.residual(Xp, X0, cb, dt) - P.residual(Xm, X0, cb, dt)) / (2 * s)
    scale = np.max(np.abs(J))
    assert np.max(np.abs(J - Jfd)) <= 1e-6 * scale


# ---------------------------------------------------------------------------
# ILU(0), RAS and GMRES
# ---------------------------------------------------------------------------

def test_ilu0_reproduces_matrix_on_its_pattern():
    """The defining property of ILU(0): (L U)_ij = A_ij for every (i, j) in the pattern of A."""
    cf = S.coefficients()
    P = oracle.Problem(2, (6, 6), 0.25, cf)
    X1, X0, (c1, e1, c0, e0) = _pair(P, 2, (6, 6), 51, du=0.01)
    rp, ci, v = P.jacobian(X1, X0, c0.mean(), 0.1)
    rc, w = oracle.ilu0(rp, ci, v)
    assert rc == 0
    n = len(rp) - 1
    A = np.zeros((n, n))
    Lm, Um = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for jj in range(rp[i], rp[i + 1]):
            j = ci[jj]
            A[i, j] = v[jj]
            if j < i:
                Lm[i, j] = w[jj]
            else:
                Um[i, j] = w[jj]
    LU = Lm @ Um
    mask = A != 0
    for i in range(n):
        mask[i, ci[rp[i]:rp[i + 1]]] = True
    assert np.max(np.abs((LU - A)[mask])) <= 1e-10 * np.max(np.abs(A))
    # and it is not the exact LU (fill was dropped)
    assert np.max(np.abs(LU - A)) > 1e-8 * np.max(np.abs(A))


def _null_modes(n, dim):
    """Sign patterns of the centred-difference null space per component."""
    grids = np.meshgrid(*[np.arange(m) for m in reversed(n)], indexing="ij")
    xs = [g.reshape(-1) for g in reversed(grids)]
    modes = []
    for m in range(1 << dim):
        if any((m >> J) & 1 and n[J] % 2 for J in range(dim)):
            continue
        sg = np.ones(len(xs[0]))
        for J in range(dim):
            if (m >> J) & 1:
                sg = sg * (-1.0) ** xs[J]
        modes.append(sg / np.linalg.norm(sg))
    return modes


def _project_u(P, x, dim, n):
    x = x.copy()
    for I in range(dim):
        col = x[2 + I::P.nf]
        for m in _null_modes(n, dim):
            col = col - np.dot(col, m) * m
        x[2 + I::P.nf] = col
    return x


@pytest.mark.parametrize("dim,n,sub", [(2, (6, 6), (2, 2)), (2, (7, 6), (2, 3)), (3, (4, 4, 4), (2, 2, 1))])
def test_gmres_ras_solution_matches_dense_solve(dim, n, sub):
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=1, gmres_maxit=3000, gmres_restart=30)
    P = oracle.Problem(dim, n, 0.25, cf, op)
    X1, X0, (c1, e1, c0, e0) = _pair(P, dim, n, 61, du=0.01)
    cb, dt = c0.mean(), 0.2
    J = P.jacobian_scipy(X1, X0, cb, dt).toarray()
    rng = np.random.default_rng(7)
    b = rng.standard_normal(len(X1))
    b[0::P.nf] -= b[0::P.nf].mean()          # consistent: sum b_c = 0 (mass)
    b = _project_u(P, b, dim, n)             # consistent: b_u orthogonal to the null modes
    xd = np.linalg.lstsq(J, b, rcond=None)[0]
    xd = _project_u(P, xd, dim, n)
    rc, x, its, res = P.linear_solve(X1, X0, cb, dt, b, 1e-13 * np.linalg.norm(b))
    assert rc == 0 and res <= 1e-13 * np.linalg.norm(b) * 1.0001
    assert abs(x[0::P.nf].sum()) < 1e-12 * np.abs(x[0::P.nf]).sum()
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_single_subdomain_exact_solver_converges_in_one_iteration():
    cf = S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    op = S.options(sub=(1, 1), overlap=0, subsolver=1)
    P = oracle.Problem(2, (6, 5), 0.25, cf, op)
    X1, X0, (c1, e1, c0, e0) = _pair(P, 2, (6, 5), 71)
    b = np.random.default_rng(9).standard_normal(len(X1))
    b[0::2] -= b[0::2].mean()
    rc, x, its, res = P.linear_solve(X1, X0, c0.mean(), 0.2, b, 1e-10 * np.linalg.norm(b))
    assert rc == 0 and its == 1 and res <= 1e-10 * np.linalg.norm(b)


def test_ras_with_full_overlap_single_subdomain_ilu_is_plain_ilu():
    """With one subdomain the RAS sweep is one ILU(0) solve of the whole Jacobian."""
    cf = S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    op = S.options(sub=(1, 1), overlap=0, project=0)
    P = oracle.Problem(2, (6, 6), 0.25, cf, op)
    X1, X0, (c1, e1, c0, e0) = _pair(P, 2, (6, 6), 81)
    rp, ci, v = P.jacobian(X1, X0, c0.mean(), 0.2)
    r = np.random.default_rng(2).standard_normal(len(X1))
    rc, z = P.precond_apply(X1, X0, c0.mean(), 0.2, r)
    rc2, w = oracle.ilu0(rp, ci, v)
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    n = len(rp) - 1
    M = sp.csr_matrix((w, ci, rp), shape=(n, n))
    Lm = sp.tril(M, -1) + sp.eye(n)
    Um = sp.triu(M)
    y = sla.spsolve_triangular(Lm.tocsr(), r, lower=True)
    ref = sla.spsolve_triangular(Um.tocsr(), y, lower=False)
    assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)


# ---------------------------------------------------------------------------
# time stepping: mass, energy law (Theorem 3.2), symmetry, dt predictor
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,n,sub,mode,steps", [(2, (16, 16), (2, 2), "energy", 6),
                                                  (2, (12, 10), (3, 2), "solution", 5),
                                                  (3, (8, 8, 8), (2, 2, 2), "fixed", 3)])
def test_mass_conservation_and_energy_decay(dim, n, sub, mode, steps):
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=1, dt_mode=mode)
    P = oracle.Problem(dim, n, 0.25, cf, op)
    c, e = S.initial_fields(dim, n, 0.18, 5)
    rc, X, infos, e0 = P.simulate(c, e, steps)
    assert rc == 0
    m0 = c.sum() * 0.25 ** dim
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    if mode != "fixed":
        assert all(i["dt"] >= op["dt_min"] - 1e-15 for i in infos)


def test_sphere_particle_state_and_oracle_steps():
    """The single-particle state of Sec. 5.1: two phases only, the lattice count of
    the ball within 10% of its volume, symmetric under axis swaps and reflections
    through the centre; and the oracle's adaptive steps from it, with the Hooke
    tensor scaled by L = 0 (no elasticity), 1 and 3, conserve mass and do not
    increase the energy (Theorem 3.2)."""
    n, h, r = (16, 16, 16), 0.25, 1.6
    c, e = S.sphere_fields(3, n, h, r)
    inside = c == 0.238
    assert np.all(e[inside] == 0.01) and np.all(c[~inside] == 0.1375) and np.all(e[~inside] == 0.99)
    assert abs(inside.sum() - 4.0 / 3.0 * math.pi * (r / h) ** 3) <= 0.1 * 4.0 / 3.0 * math.pi * (r / h) ** 3
    c3 = c.reshape(16, 16, 16)
    assert np.array_equal(c3, c3.transpose(1, 0, 2)) and np.array_equal(c3, c3.transpose(2, 1, 0))
    core = c3[1:, 1:, 1:]  # points 1..15: the centre is point 8 on every axis
    assert np.array_equal(core, core[::-1, ::-1, ::-1])
    for L in (0.0, 1.0, 3.0):
        n2 = (12, 12, 12)
        c, e = S.sphere_fields(3, n2, h, 1.0)
        P = oracle.Problem(3, n2, h, S.coefficients(Lscale=L), S.options(sub=(2, 2, 2), overlap=1, dt_mode="energy"))
        rc, X, infos, e0 = P.simulate(c, e, 2)
        assert rc == 0
        m0 = c.sum() * h ** 3
        E = [e0] + [i["energy"] for i in infos]
        for i in infos:
            assert abs(i["mass"] - m0) <= 1e-12 * m0
        for a, b in zip(E[:-1], E[1:]):
            assert b <= a + 1e-12 * abs(a)


def test_shift_and_axis_swap_symmetry():
    cf = S.coefficients()
    n = (12, 12)
    op = S.options(sub=(2, 2), overlap=1, newton_rtol=1e-12)
    P = oracle.Problem(2, n, 0.25, cf, op)
    c, e = S.initial_fields(2, n, 0.18, 11)
    rc, X, _, _ = P.simulate(c, e, 2)
    cF, eF, uF = P.split(X)
    # shift by (3, 5) cells
    sh = lambda f: np.roll(f.reshape(12, 12), (5, 3), axis=(0, 1)).reshape(-1)
    rc2, X2, _, _ = P.simulate(sh(c), sh(e), 2)
    c2, e2, u2 = P.split(X2)
    assert np.linalg.norm(c2 - sh(cF)) <= 1e-9 * np.linalg.norm(cF)
    assert np.linalg.norm(e2 - sh(eF)) <= 1e-9 * np.linalg.norm(eF)
    # transpose (cubic Hooke tensor is symmetric under the axis swap)
    tr = lambda f: f.reshape(12, 12).T.reshape(-1)
    rc3, X3, _, _ = P.simulate(tr(c), tr(e), 2)
    c3, e3, u3 = P.split(X3)
    assert np.linalg.norm(c3 - tr(cF)) <= 1e-9 * np.linalg.norm(cF)
    assert np.linalg.norm(u3[0] - tr(uF[1])) <= 1e-8 * np.linalg.norm(uF)
    assert np.linalg.norm(u3[1] - tr(uF[0])) <= 1e-8 * np.linalg.norm(uF)


def test_dt_predictor_formula():
    """Eq. sencondt: max(dt_min, dt_max / sqrt(1 + zeta X'^2))."""
    assert oracle.dt_predict(0.01, 2.0, 100.0, 0.0) == 2.0
    assert oracle.dt_predict(0.01, 2.0, 100.0, 1.0) == pytest.approx(2.0 / math.sqrt(101.0), rel=1e-15)
    assert oracle.dt_predict(0.01, 2.0, 100.0, 1e4) == 0.01


def test_divergence_triggers_retry_with_smaller_dt():
    """A Newton limit of one iteration with an unreachable tolerance forces every
    attempt to fail: the step retries max_retries times and reports divergence."""
    cf = S.coefficients()
    op = S.options(sub=(2, 2), overlap=1, newton_maxit=1, newton_rtol=1e-30, newton_atol=0.0, max_retries=3)
    P = oracle.Problem(2, (8, 8), 0.25, cf, op)
    c, e = S.initial_fields(2, (8, 8), 0.18, 2)
    rc, X, infos, _ = P.simulate(c, e, 1)
    assert rc == oracle.ORC_EDIVERGED
    assert infos[0]["retries"] == 3
    assert infos[0]["dt"] == pytest.approx(0.01 / 2 ** 1.5, rel=1e-12)


# ---------------------------------------------------------------------------
# Schwarz preconditioner types (Sec. 4, Table 2) against their definitions
# ---------------------------------------------------------------------------

def _boxes(n, sub, delta):
    """Box decomposition: per axis, box s owns [s n / sub, (s+1) n / sub) and is
    extended by delta cells per side (periodic), or is the whole axis when the
    extension would cover it; yields (points, owned mask) with x fastest."""
    import itertools
    per_axis = []
    for nn, sb in zip(n, sub):
        ax = []
        for s in range(sb):
            o0, o1 = s * nn // sb, (s + 1) * nn // sb
            if o1 - o0 + 2 * delta >= nn:
                cells = list(range(nn))
            else:
                cells = [(o0 - delta + t) % nn for t in range(o1 - o0 + 2 * delta)]
            ax.append([(c, o0 <= c < o1) for c in cells])
        per_axis.append(ax)
    for combo in itertools.product(*[range(len(a)) for a in per_axis[::-1]]):
        combo = combo[::-1]
        cells = [per_axis[J][combo[J]] for J in range(len(n))]
        pts, own = [], []
        for idx in itertools.product(*[range(len(c)) for c in cells[::-1]]):
            idx = idx[::-1]
            p, stride, ok = 0, 1, True
            for J in range(len(n)):
                c, o = cells[J][idx[J]]
                p += c * stride
                stride *= n[J]
                ok = ok and o
            pts.append(p)
            own.append(ok)
        yield np.array(pts), np.array(own)


@pytest.mark.parametrize("dim,n,sub,delta", [(1, (13,), (3,), 2), (2, (9, 8), (2, 2), 1), (2, (10, 9), (3, 2), 2)])
def test_schwarz_types_match_their_definitions(dim, n, sub, delta):
    """left-RAS, classical AS and right-RAS (exact subdomain solves, no projection)
    against z = sum_i E_i (owned | all) A_i^-1 (all | owned) restrictions of r,
    formed with dense inverses of J restricted to each overlapped box."""
    cf = S.coefficients()
    c0, e0, u0 = S.random_fields(dim, n, 31, u_amp=0.01)
    c1 = c0 * 1.01
    O0 = oracle.Problem(dim, n, 0.25, cf, S.options(sub=sub, overlap=delta))
    nf = O0.nf
    X1, X0 = O0.interleave(c1, e0, u0), O0.interleave(c0, e0, u0)
    cb, dt = float(np.mean(c0)), 0.05
    J = O0.jacobian_scipy(X1, X0, cb, dt, 0).toarray()
    r = np.random.default_rng(4).standard_normal(J.shape[0])
    want = {"left-ras": np.zeros_like(r), "as": np.zeros_like(r), "right-ras": np.zeros_like(r)}
    for pts, own in _boxes(n, sub, delta):
        idx = (pts[:, None] * nf + np.arange(nf)[None, :]).reshape(-1)
        own_u = np.repeat(own, nf)
        A = J[np.ix_(idx, idx)]
        x = np.linalg.solve(A, r[idx])
        want["left-ras"][idx[own_u]] = x[own_u]
        want["as"][idx] += x
        want["right-ras"][idx] += np.linalg.solve(A, np.where(own_u, r[idx], 0.0))
    for var, zw in want.items():
        O = oracle.Problem(dim, n, 0.25, cf, S.options(sub=sub, overlap=delta, subsolver=1, project=0,
                                                       ras_variant=var))
        rc, z = O.precond_apply(X1, X0, cb, dt, r)
        assert rc == 0
        assert np.linalg.norm(z - zw) <= 1e-11 * np.linalg.norm(zw), var


def test_schwarz_types_coincide_without_overlap():
    """delta = 0: the three types are block Jacobi (Table 2's classical AS, delta = 0)."""
    dim, n = 2, (9, 8)
    cf = S.coefficients()
    c0, e0, u0 = S.random_fields(dim, n, 33, u_amp=0.01)
    zs = []
    for var in ("left-ras", "as", "right-ras"):
        O = oracle.Problem(dim, n, 0.25, cf, S.options(sub=(3, 2), overlap=0, ras_variant=var))
        X = O.interleave(c0, e0, u0)
        r = np.random.default_rng(5).standard_normal(X.size)
        rc, z = O.precond_apply(X, X, float(np.mean(c0)), 0.05, r)
        assert rc == 0
        zs.append(z)
    assert np.array_equal(zs[0], zs[1]) and np.array_equal(zs[0], zs[2])
