"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Operator level: energy/mass, the residual F, the Jacobian action, the Schwarz
preconditioner and the GMRES solve, element by element on seeded inputs whose
grids span several subdomains with ragged sizes.  Time-step level: the fields
after whole NKS steps, relative L2 per field <= 1e-8 (the tolerance of the
FP64 method), mass to 1e-12 and a non-increasing energy.  Full size: one step
of the 1024^2 workload checked by the oracle's own residual on the GPU result.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nks():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as m
    return m


def soa(c, e, u=None):
    parts = [c, e] + ([] if u is None else list(np.asarray(u)))
    return np.concatenate(parts)


def split_soa(X, N, nf):
    Y = X.reshape(nf, N)
    return Y[0], Y[1], (Y[2:] if nf > 2 else None)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _pair(dim, n, seed, du=0.01):
    c0, e0, u0 = S.random_fields(dim, n, seed, u_amp=du)
    rng = np.random.default_rng(seed + 1)
    c1 = c0 * (1 + 0.04 * rng.uniform(-1, 1, c0.shape))
    c1 += c0.mean() - c1.mean()  # same mass at both levels, as every Newton iterate has
    e1 = e0 * (1 + 0.04 * rng.uniform(-1, 1, e0.shape))
    u1 = u0 * (1 + 0.04 * rng.uniform(-1, 1, u0.shape))
    return (c1, e1, u1), (c0, e0, u0)


# (dim, grid, subdomains, overlap, elastic): ragged tiles of the stencil kernels and
# unequal Schwarz boxes; 1-D and the elasticity-free model (nf = 2) included
CASES = [(2, (37, 29), (3, 2), 1, True), (2, (40, 36), (2, 3), 2, True), (3, (11, 10, 9), (2, 2, 2), 1, True),
         (1, (61,), (3,), 2, True), (2, (35, 33), (2, 2), 1, False), (3, (9, 11, 10), (2, 2, 2), 1, False)]


@pytest.mark.parametrize("dim,n,sub,ov,elastic", CASES)
def test_operators_match_oracle(nks, dim, n, sub, ov, elastic):
    cf = S.coefficients() if elastic else S.coefficients(Lscale=0.0)
    op = S.options(sub=sub, overlap=ov)
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 100 + dim)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    N, nf = P.N, P.nf
    cb = float(np.sum(c0) / N)
    if nf == 2:
        u1 = u0 = None
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)
    to_soa = lambda Xo: soa(*O.split(Xo)) if nf > 2 else soa(*O.split(Xo)[:2])
    dt = 0.07
    # energy and mass
    parts, mass = P.eval_energy(X1g)
    e_o, parts_o = O.energy(X1o, cb, parts=True)
    assert parts[4] == pytest.approx(e_o, rel=1e-13, abs=1e-11)
    assert np.allclose(parts[:4], parts_o, rtol=1e-12, atol=1e-11)
    assert mass == pytest.approx(O.mass(X1o), rel=1e-14)
    # residual (full and displacement-only systems)
    for mode in (0, 1):
        Fg = P.eval_residual(X1g, X0g, dt, mode)
        Fo = to_soa(O.residual(X1o, X0o, cb, dt, mode))
        for f in range(nf):
            a, b = Fg[f * N:(f + 1) * N], Fo[f * N:(f + 1) * N]
            assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-30) + 1e-300, (mode, f)
    # Jacobian action against the oracle's assembled Jacobian
    v = np.random.default_rng(5).standard_normal(nf * N)
    vo = O.interleave(*split_soa(v, N, nf))
    for mode in (0, 1):
        Jv = P.apply_jacobian(X1g, X0g, dt, v, mode)
        Jo = to_soa(O.jacobian_scipy(X1o, X0o, cb, dt, mode) @ vo)
        for f in range(nf):
            a, b = Jv[f * N:(f + 1) * N], Jo[f * N:(f + 1) * N]
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), (mode, f)
    # Schwarz preconditioner with the projection
    r = np.random.default_rng(6).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, dt, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, dt, O.interleave(*split_soa(r, N, nf)))
    assert rc == 0
    assert rel(z, to_soa(zo)) <= 1e-9
    assert abs(z[:N].sum()) <= 1e-11 * np.abs(z[:N]).sum()
    # GMRES solve
    b = -P.eval_residual(X1g, X0g, dt, 0)
    tol = 1e-11 * np.linalg.norm(b)
    x, its, res = P.linear_solve(X1g, X0g, dt, b, tol)
    assert res <= tol
    rc, xo, its_o, res_o = O.linear_solve(X1o, X0o, cb, dt, O.interleave(*split_soa(b, N, nf)), tol)
    assert rel(x, to_soa(xo)) <= 1e-8
    assert abs(its - its_o) <= max(2, its_o // 5)
    P.destroy()


@pytest.mark.parametrize("dim,n,sub,ov,elastic", CASES)
def test_mixed_operators_match_oracle(nks, dim, n, sub, ov, elastic):
    """The mixed-precision forms as the solver applies them: the FP32 Jacobian action
    (FP32 vectors, coefficients and arithmetic) and the FP32 Schwarz sweeps, against
    the FP64 oracle within FP32 rounding of the largest term of each row."""
    cf = S.coefficients() if elastic else S.coefficients(Lscale=0.0)
    op = S.options(sub=sub, overlap=ov, precision="mixed")
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 200 + dim)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    N, nf = P.N, P.nf
    cb = float(np.sum(c0) / N)
    if nf == 2:
        u1 = u0 = None
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)
    to_soa = lambda Xo: soa(*O.split(Xo)) if nf > 2 else soa(*O.split(Xo)[:2])
    dt = 0.07
    v = np.random.default_rng(7).standard_normal(nf * N)
    vo = O.interleave(*split_soa(v, N, nf))
    for mode in (0, 1):
        Jv = P.apply_jacobian(X1g, X0g, dt, v, mode)
        Jm = O.jacobian_scipy(X1o, X0o, cb, dt, mode)
        Jo = to_soa(Jm @ vo)
        # scale of the row terms: |J| |v|
        scale = to_soa(abs(Jm) @ np.abs(vo))
        err = np.abs(Jv - Jo)
        assert np.all(err <= 1e-5 * scale + 1e-30), (mode, float(np.max(err / (scale + 1e-300))))
        assert rel(Jv, Jo) <= 1e-5, mode
    r = np.random.default_rng(8).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, dt, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, dt, O.interleave(*split_soa(r, N, nf)))
    assert rc == 0
    assert rel(z, to_soa(zo)) <= 1e-4
    P.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("variant", ["left-ras", "as"])
@pytest.mark.parametrize("dim,n,sub,ov", [(3, (36, 36, 36), (2, 2, 2), 1), (2, (232, 232), (2, 2), 2)])
def test_preconditioner_with_box_vectors_in_global_memory(nks, dim, n, sub, ov, variant, precision):
    """Boxes too large for their vector to sit in shared memory (20^3 x 5 fields,
    120^2 x 4 fields): both sweeps then keep it in global scratch; the Schwarz
    application still matches the oracle's (restricted and overlapped prolongation)."""
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=ov, precision=precision, ras_variant=variant)
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 300 + dim)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    N, nf = P.N, P.nf
    cb = float(np.sum(c0) / N)
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)
    r = np.random.default_rng(9).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, 0.07, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, 0.07, O.interleave(*split_soa(r, N, nf)))
    assert rc == 0
    assert rel(z, soa(*O.split(zo))) <= (1e-10 if precision == "fp64" else 1e-4)
    P.destroy()


def _run_both(nks, dim, n, cbar, seed, steps, op, cf=None, dt=0.01):
    cf = cf or S.coefficients()
    c, e = S.initial_fields(dim, n, cbar, seed)
    P = nks.Problem(dim, n, 0.25, c, e, cf, op)
    infos = [P.step(dt) for _ in range(steps)]
    cg, eg, ug = P.get_fields()
    O = oracle.Problem(dim, n, 0.25, cf, dict(op, newton_rtol=1e-12))
    rc, X, oinf, e0 = O.simulate(c, e, steps, dt_replay=[i["dt"] for i in infos])
    assert rc == 0
    co, eo, uo = O.split(X)
    return P, (c, e), (cg, eg, ug), (co, eo, uo), infos, oinf, e0


def test_config_2d64_ten_steps(nks):
    cfg = S.CONFIGS["2d64"]
    op = S.options(**cfg["opts"])
    P, (c, e), (cg, eg, ug), (co, eo, uo), infos, oinf, e0 = _run_both(nks, 2, cfg["n"], cfg["cbar"], cfg["seed"],
                                                                        cfg["steps"], op)
    assert rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8
    assert rel(ug, uo) <= 1e-8
    m0 = c.sum() * 0.25 ** 2
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
        assert i["newton_its"] >= 1
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    for gi, oi in zip(infos, oinf):
        assert gi["energy"] == pytest.approx(oi["energy"], rel=1e-10)
        assert abs(gi["gmres_its"] - oi["gmres_its"]) <= max(3, oi["gmres_its"] // 5)
    P.destroy()


def test_3d_small_three_steps(nks):
    op = S.options(sub=(2, 2, 2), overlap=1)
    P, _, (cg, eg, ug), (co, eo, uo), infos, oinf, _ = _run_both(nks, 3, (16, 14, 12), 0.18, 9, 3, op)
    assert rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8 and rel(ug, uo) <= 1e-8
    P.destroy()


def test_adaptive_steps_replayed_by_oracle(nks):
    cf = S.coefficients()
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy")
    c, e = S.initial_fields(2, (32, 32), 0.2, 4)
    P = nks.Problem(2, (32, 32), 0.25, c, e, cf, op)
    infos = [P.step() for _ in range(6)]
    assert infos[0]["dt"] == 0.01
    assert all(i["dt"] >= 0.01 - 1e-15 for i in infos)
    cg, eg, ug = P.get_fields()
    O = oracle.Problem(2, (32, 32), 0.25, cf, dict(op, newton_rtol=1e-12))
    rc, X, oinf, _ = O.simulate(c, e, 6, dt_replay=[i["dt"] for i in infos])
    co, eo, uo = O.split(X)
    assert rc == 0 and rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8
    P.destroy()


@pytest.mark.parametrize("L", [0.0, 1.0, 3.0])
def test_sphere_particle_steps_replayed_by_oracle(nks, L):
    """The single-particle state of Sec. 5.1 (sharp interface, Hooke tensor x L;
    L = 0 is the model without elasticity): adaptive steps on the GPU, replayed by
    the oracle with the same step sizes."""
    n, h = (16, 16, 16), 0.25
    cf = S.coefficients(Lscale=L)
    op = S.options(sub=(2, 2, 2), overlap=1, dt_mode="energy")
    c, e = S.sphere_fields(3, n, h, 1.6)
    P = nks.Problem(3, n, h, c, e, cf, op)
    infos = [P.step() for _ in range(3)]
    cg, eg, ug = P.get_fields()
    O = oracle.Problem(3, n, h, cf, dict(op, newton_rtol=1e-12))
    rc, X, oinf, e0 = O.simulate(c, e, 3, dt_replay=[i["dt"] for i in infos])
    co, eo, uo = O.split(X)
    assert rc == 0 and rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8
    if L:
        assert rel(ug, uo) <= 1e-8
    else:
        assert ug is None and uo is None
    for gi, oi in zip(infos, oinf):
        assert gi["energy"] == pytest.approx(oi["energy"], rel=1e-10)
    P.destroy()


def test_full_size_sphere_80_step_checked_by_oracle_residual(nks):
    """One step of the 80^3 single-particle workload (Sec. 5.1), checked by the
    oracle's residual of the GPU result."""
    cfg = S.CONFIGS["3d80sphere"]
    cf = S.config_coefficients(cfg)
    op = S.options(**cfg["opts"])
    n, h = cfg["n"], cfg["h"]
    c, e = S.config_fields(cfg)
    P = nks.Problem(3, n, h, c, e, cf, op)
    _, _, u0 = P.get_fields()
    info = P.step()
    assert info["status"] == 0 and info["dt"] == 0.01
    cg, eg, ug = P.get_fields()
    O = oracle.Problem(3, n, h, cf, op)
    cb = float(np.sum(c) / c.size)
    X0 = O.interleave(c, e, u0)
    X1 = O.interleave(cg, eg, ug)
    F = O.residual(X1, X0, cb, info["dt"])
    F0 = O.residual(X0, X0, cb, info["dt"])
    assert np.linalg.norm(F) <= 1e-9 * np.linalg.norm(F0)
    # the mass h^3 sum(c), summed exactly: over 512,000 near-constant values a
    # plain running sum (the oracle's) drifts by about 1e-11 relative
    m0 = math.fsum(c) * h ** 3
    assert abs(info["mass"] - m0) <= 1e-12 * m0
    assert info["energy"] <= O.energy(X0, cb)
    P.destroy()


def test_initial_equilibrium_with_mixed_inner_solves(nks):
    """u0_mixed = 1 in FP64 mode: the equilibrium's GMRES runs in the mixed form but
    its Newton residual is FP64, so u0 meets the same tolerance as the all-FP64
    solve (checked with the oracle's residual), and the FP64 steps that follow
    agree with the all-FP64 run."""
    n, h = (40, 36), 0.25
    cf = S.coefficients()
    c, e = S.initial_fields(2, n, 0.18, 6)
    O = oracle.Problem(2, n, h, cf, S.options(sub=(2, 3), overlap=2))
    cb = float(np.sum(c) / c.size)
    F00 = np.linalg.norm(O.residual(O.interleave(c, e), O.interleave(c, e), cb, 1.0, 1))
    runs = {}
    for um in (0, 1):
        op = S.options(sub=(2, 3), overlap=2, u0_mixed=um, dt_mode="energy")
        P = nks.Problem(2, n, h, c, e, cf, op)
        _, _, u0 = P.get_fields()
        X0 = O.interleave(c, e, u0)
        assert np.linalg.norm(O.residual(X0, X0, cb, 1.0, mode=1)) <= 1e-11 * F00
        infos = [P.step() for _ in range(2)]
        runs[um] = (u0, P.get_fields(), infos)
        P.destroy()
    (ua, (ca, ea, wa), ia), (ub, (cb_, eb, wb), ib) = runs[0], runs[1]
    assert rel(ub, ua) <= 1e-9
    assert rel(cb_, ca) <= 1e-9 and rel(eb, ea) <= 1e-9 and rel(wb, wa) <= 1e-8
    assert [i["dt"] for i in ia] == pytest.approx([i["dt"] for i in ib], rel=1e-9)


def test_checkpoint_resume_is_bitwise(nks):
    cf = S.coefficients()
    op = S.options(sub=(2, 2), overlap=1, dt_mode="solution")
    c, e = S.initial_fields(2, (24, 24), 0.18, 3)
    A = nks.Problem(2, (24, 24), 0.25, c, e, cf, op)
    for _ in range(2):
        A.step()
    blob = A.get_state()
    ref = [A.step() for _ in range(2)]
    ca, ea, ua = A.get_fields()
    B = nks.Problem(2, (24, 24), 0.25, c, e, cf, op)
    B.set_state(blob)
    got = [B.step() for _ in range(2)]
    cb_, eb_, ub_ = B.get_fields()
    assert np.array_equal(ca, cb_) and np.array_equal(ea, eb_) and np.array_equal(ua, ub_)
    assert [r["dt"] for r in ref] == [g["dt"] for g in got]
    A.destroy()
    B.destroy()


def test_steady_state_and_invalid_inputs(nks):
    cf = S.coefficients()
    op = S.options(sub=(2, 2), overlap=1)
    N = 16 * 16
    P = nks.Problem(2, (16, 16), 0.25, np.full(N, 0.17), np.full(N, 1.0), cf, op)
    info = P.step(0.5)
    assert info["newton_its"] == 0
    c, e, u = P.get_fields()
    assert np.all(c == 0.17) and np.all(e == 1.0)
    P.destroy()
    with pytest.raises(nks.NksError) as ei:
        nks.Problem(2, (16, 16), 0.25, np.full(N, 0.3), np.full(N, 0.0), cf, op)
    assert ei.value.code == nks.NKS_EDOMAIN
    with pytest.raises(nks.NksError) as ei:
        nks.Problem(2, (16, 16), 0.25, np.full(N, 0.17), np.full(N, 0.5), cf, S.options(sub=(1, 1), overlap=1))
    assert ei.value.code == nks.NKS_EINVAL


def test_three_order_parameter_pointwise_derivative_matches_oracle(nks):
    """The CUDA path's pointwise DVD derivative of the model with three order
    parameters (closed polynomial quotients, Simpson's rule, dual-number
    derivatives; a host function of the library) against the oracle's
    (Gauss-Legendre quotients), and its derivative block against central
    differences of the oracle's G."""
    rng = np.random.default_rng(0)
    cf = S.coefficients(n_eta=3)
    O = oracle.Problem(1, (1,), 0.25, cf)
    pack = lambda x: O.interleave(np.array([x[0]]), np.asarray(x[1:]).reshape(3, 1))
    for _ in range(25):
        c0, c1 = 0.12 + 0.1 * rng.random(2)
        e0 = 0.6 + 0.8 * rng.random(3)
        e1 = e0 + 0.05 * rng.standard_normal(3)
        x1, x0 = np.array([c1, *e1]), np.array([c0, *e0])
        G, dG = nks.model3_point(cf, x1, x0)
        gc, ge = O.dvd_G(pack(x1), pack(x0), 0.0, 3)
        Go = np.array([gc[0], *ge[:, 0]])
        assert np.abs(G - Go).max() <= 1e-13 * np.abs(Go).max()
        fd = np.zeros((4, 4))
        for b in range(4):
            xp, xm = x1.copy(), x1.copy()
            xp[b] += 1e-6
            xm[b] -= 1e-6
            gp, gm = O.dvd_G(pack(xp), pack(x0), 0.0, 3), O.dvd_G(pack(xm), pack(x0), 0.0, 3)
            fd[:, b] = (np.array([gp[0][0], *gp[1][:, 0]]) - np.array([gm[0][0], *gm[1][:, 0]])) / 2e-6
        assert np.abs(dG - fd).max() <= 1e-7 * np.abs(fd).max()


def test_size_limits_are_refused_before_any_allocation(nks):
    """The largest sizes: (2 + d) N at or above 2^31 would overflow the kernels'
    32-bit field offsets, and n_z x slots above 65535 the 3-D launch grid; both
    are refused by validation, before any device memory is touched."""
    cf = S.coefficients()
    op = S.options(sub=(2, 2, 2), overlap=1)
    with pytest.raises(nks.NksError) as ei:
        nks.Batch(3, (800, 800, 800), 0.25, 1, cf, op)  # 5 x 512e6 > 2^31
    assert ei.value.code == nks.NKS_EINVAL
    with pytest.raises(nks.NksError) as ei:
        nks.Batch(3, (16, 16, 4096), 0.25, 16, cf, op)  # n_z x slots = 65536
    assert ei.value.code == nks.NKS_EINVAL
    with pytest.raises(nks.NksError) as ei:
        nks.Batch(2, (64, 2), 0.25, 1, cf, S.options(sub=(2, 1), overlap=1))  # fewer than 3 cells
    assert ei.value.code == nks.NKS_EINVAL


def test_full_size_2d1024_step_checked_by_oracle_residual(nks):
    cfg = S.CONFIGS["2d1024"]
    cf = S.coefficients()
    op = S.options(**cfg["opts"])
    n = cfg["n"]
    c, e = S.initial_fields(2, n, cfg["cbar"], cfg["seed"])
    P = nks.Problem(2, n, 0.25, c, e, cf, op)
    _, _, u0 = P.get_fields()
    info = P.step()
    assert info["status"] == 0 and info["dt"] == 0.01
    cg, eg, ug = P.get_fields()
    O = oracle.Problem(2, n, 0.25, cf, op)
    cb = float(np.sum(c) / c.size)
    X0 = O.interleave(c, e, u0)
    X1 = O.interleave(cg, eg, ug)
    # u0 is the oracle's equilibrium too: its displacement residual vanishes
    Fu0 = O.residual(X0, X0, cb, 1.0, mode=1)
    assert np.linalg.norm(Fu0) <= 1e-9 * np.linalg.norm(O.residual(O.interleave(c, e), O.interleave(c, e), cb, 1.0, 1))
    F = O.residual(X1, X0, cb, info["dt"])
    F0 = O.residual(X0, X0, cb, info["dt"])
    assert np.linalg.norm(F) <= 1e-9 * np.linalg.norm(F0)
    m0 = O.mass(X0)
    assert abs(info["mass"] - m0) <= 1e-12 * m0
    assert info["energy"] <= O.energy(X0, cb)
    P.destroy()


# ---------------------------------------------------------------------------
# mixed precision: FP32 Schwarz factors/sweeps and Krylov basis, FP64 residual,
# update, logarithms, energy and mass; results must still match the FP64 oracle
# ---------------------------------------------------------------------------

def test_mixed_precision_config_2d64_matches_fp64_oracle(nks):
    cfg = S.CONFIGS["2d64"]
    op = S.options(**dict(cfg["opts"], precision="mixed"))
    P, (c, e), (cg, eg, ug), (co, eo, uo), infos, oinf, e0 = _run_both(nks, 2, cfg["n"], cfg["cbar"], cfg["seed"],
                                                                        cfg["steps"], op)
    assert rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8 and rel(ug, uo) <= 1e-8
    m0 = c.sum() * 0.25 ** 2
    E = [e0] + [i["energy"] for i in infos]
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
    for a, b in zip(E[:-1], E[1:]):
        assert b <= a + 1e-12 * abs(a)
    P.destroy()


def test_mixed_precision_3d_small(nks):
    op = S.options(sub=(2, 2, 2), overlap=1, precision="mixed")
    P, _, (cg, eg, ug), (co, eo, uo), infos, oinf, _ = _run_both(nks, 3, (16, 14, 12), 0.18, 9, 3, op)
    assert rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8 and rel(ug, uo) <= 1e-8
    P.destroy()


def test_full_size_3d128_fp64_and_mixed_steps(nks):
    """One step of the 3-D 128^3 workload in FP64 and in mixed precision: both solve
    the oracle's equations (its residual on the GPU result) and agree with each other."""
    cfg = S.CONFIGS["3d128"]
    cf = S.coefficients()
    n = cfg["n"]
    c, e = S.initial_fields(3, n, cfg["cbar"], cfg["seed"])
    out = {}
    for prec in ("fp64", "mixed"):
        op = S.options(**dict(cfg["opts"], precision=prec))
        P = nks.Problem(3, n, 0.25, c, e, cf, op)
        _, _, u0 = P.get_fields()
        info = P.step()
        assert info["status"] == 0
        out[prec] = (u0, P.get_fields(), info)
        P.destroy()
    O = oracle.Problem(3, n, 0.25, cf, S.options(**cfg["opts"]))
    cb = float(np.sum(c) / c.size)
    for prec in ("fp64", "mixed"):
        u0, (cg, eg, ug), info = out[prec]
        X0 = O.interleave(c, e, u0)
        X1 = O.interleave(cg, eg, ug)
        F = O.residual(X1, X0, cb, info["dt"])
        F0 = O.residual(X0, X0, cb, info["dt"])
        assert np.linalg.norm(F) <= 1e-9 * np.linalg.norm(F0), prec
        m0 = O.mass(X0)
        assert abs(info["mass"] - m0) <= 1e-12 * m0
        assert info["energy"] <= O.energy(X0, cb)
    (_, (c64, e64, u64), _), (_, (c32, e32, u32), _) = out["fp64"], out["mixed"]
    assert rel(c32, c64) <= 1e-8 and rel(e32, e64) <= 1e-8 and rel(u32, u64) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sweep_copy_timeout_is_reported_and_the_problem_recovers(nks, prec):
    """Failure detection without a GPU fault: with a factor copy withheld, every
    sweep block's bounded mbarrier wait expires (about a second); the solve
    returns NKS_ETIMEOUT, the state stays at X^n, the context stays usable and
    the next step matches a fresh problem bit for bit."""
    import time
    dim, n = 2, (24, 20)
    op = S.options(sub=(2, 2), overlap=1, precision=prec)
    c, e = S.initial_fields(dim, n, 0.18, 3)
    P = nks.Problem(dim, n, 0.25, c, e, S.coefficients(), op)
    before = P.get_fields()
    P.debug_withhold_copy(True)
    t0 = time.time()
    with pytest.raises(nks.NksError) as ex:
        P.step(0.01)
    assert ex.value.code == 5, ex.value  # NKS_ETIMEOUT
    assert "bulk copy" in str(ex.value)
    assert time.time() - t0 < 60
    after = P.get_fields()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    P.debug_withhold_copy(False)
    P.step(0.01)
    Q = nks.Problem(dim, n, 0.25, c, e, S.coefficients(), op)
    Q.step(0.01)
    for a, b in zip(P.get_fields(), Q.get_fields()):
        assert np.array_equal(a, b)
    P.destroy()
    Q.destroy()


@pytest.mark.parametrize("variant", ["as", "right-ras"])
@pytest.mark.parametrize("dim,n,sub,ov", [(2, (37, 29), (3, 2), 1), (2, (40, 36), (2, 3), 2),
                                          (3, (11, 10, 9), (2, 2, 2), 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_schwarz_types_match_oracle(nks, variant, dim, n, sub, ov, prec):
    """Classical AS and right-RAS (Sec. 4, Table 2): the preconditioner with the
    projection against the oracle's, and a GMRES solve; overlaps summed in box order."""
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=ov, ras_variant=variant, precision=prec)
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 300 + dim)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    N, nf = P.N, P.nf
    cb = float(np.sum(c0) / N)
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)
    to_soa = lambda Xo: soa(*O.split(Xo))
    dt = 0.07
    r = np.random.default_rng(16).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, dt, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, dt, O.interleave(*split_soa(r, N, nf)))
    assert rc == 0
    assert rel(z, to_soa(zo)) <= (1e-9 if prec == "fp64" else 1e-4)
    assert abs(z[:N].sum()) <= (1e-11 if prec == "fp64" else 1e-5) * np.abs(z[:N]).sum()
    b = -P.eval_residual(X1g, X0g, dt, 0)
    tol = 1e-9 * np.linalg.norm(b)
    x, its, res = P.linear_solve(X1g, X0g, dt, b, tol)
    assert res <= tol
    rc, xo, its_o, res_o = O.linear_solve(X1o, X0o, cb, dt, O.interleave(*split_soa(b, N, nf)), tol)
    assert rel(x, to_soa(xo)) <= 1e-6
    if prec == "fp64":
        assert abs(its - its_o) <= max(2, its_o // 5)
    P.destroy()


def test_classical_as_without_overlap_config_2d64(nks):
    """The paper's choice (Table 2): classical AS, delta = 0, ILU(0)-reuse; ten
    steps of the 64^2 workload against the oracle."""
    cfg = S.CONFIGS["2d64"]
    op = S.options(**dict(cfg["opts"], overlap=0, ras_variant="as"))
    P, (c, e), (cg, eg, ug), (co, eo, uo), infos, oinf, e0 = _run_both(nks, 2, cfg["n"], cfg["cbar"], cfg["seed"],
                                                                        cfg["steps"], op)
    assert rel(cg, co) <= 1e-8 and rel(eg, eo) <= 1e-8 and rel(ug, uo) <= 1e-8
    m0 = c.sum() * 0.25 ** 2
    for i in infos:
        assert abs(i["mass"] - m0) <= 1e-12 * m0
