"""The model with three order parameters (App. A; n_eta = 3) in the CUDA path,
against the FP64 oracle's model of App. A (itself pinned in
tests/test_oracle_three_eta.py by its reduction to the reduced model, the DVD
chain rule and finite differences).

Operator level, element by element on ragged grids (1-D, 2-D, 3-D, with and
without elasticity, periodic and Neumann): energy, residual, Jacobian action
(FP64 and the mixed form), the Schwarz preconditioner (ILU(0) of the 166-slot
3-D pattern) and the GMRES solve.  Steps: ten fixed-dt NKS steps against the
oracle's, mass to 1e-12 and a non-increasing energy (Theorem 3.2).  Reduction:
with eta_1 = eta_2 = eta_3 the GPU solves the reduced model (every eta_j equal
to the reduced model's eta).  Batches: each slot equals its run alone, bit for
bit.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def soa(c, eta, u=None):
    return np.concatenate([c, np.asarray(eta).reshape(-1)] + ([] if u is None else [np.asarray(u).reshape(-1)]))


def _state(dim, n, seed, elastic, u_amp=0.01):
    """(c, eta[3, N], u) with the order parameters spread over (0.1, 0.9) so that the
    coupling between them is exercised"""
    c, eta = S.initial_fields3(dim, n, 0.18, seed, c_amp=0.04, eta_mean=0.5, eta_amp=0.4)
    N = c.size
    u = u_amp * (2.0 * S.uniform01(seed + 5, dim * N).reshape(dim, N) - 1.0) if elastic else None
    return c, eta, u


def _pair(dim, n, seed, elastic):
    (c0, e0, u0) = _state(dim, n, seed, elastic)
    rng = np.random.default_rng(seed + 1)
    c1 = c0 * (1 + 0.04 * rng.uniform(-1, 1, c0.shape))
    c1 += c0.mean() - c1.mean()
    e1 = e0 * (1 + 0.04 * rng.uniform(-1, 1, e0.shape))
    u1 = None if u0 is None else u0 * (1 + 0.04 * rng.uniform(-1, 1, u0.shape))
    return (c1, e1, u1), (c0, e0, u0)


# (dim, grid, subdomains, overlap, elastic, neumann)
CASES = [(2, (21, 18), (2, 2), 1, True, False), (3, (10, 9, 8), (2, 2, 2), 1, True, False),
         (1, (45,), (3,), 2, True, False), (2, (19, 17), (2, 2), 1, False, False),
         (3, (9, 10, 8), (2, 2, 2), 1, False, False), (2, (20, 16), (2, 2), 1, True, True),
         (3, (8, 8, 6), (2, 2, 2), 1, True, True)]


@pytest.mark.parametrize("dim,n,sub,ov,elastic,neumann", CASES)
def test_model3_operators_match_oracle(nks, dim, n, sub, ov, elastic, neumann):
    cf = S.coefficients(n_eta=3) if elastic else S.coefficients(n_eta=3, Lscale=0.0)
    op = S.options(sub=sub, overlap=ov, gmres_maxit=6000)
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 600 + dim, elastic)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op, neumann=neumann)
    O = oracle.Problem(dim, n, 0.25, cf, op, neumann=neumann)
    N, nf = P.N, P.nf
    assert (P.ne, nf, O.nf) == (3, 4 + (dim if elastic else 0), nf)
    cb = float(np.sum(c0) / N)
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)

    def to_soa(Xo):
        c, e, u = O.split(Xo)
        return soa(c, e, u)

    def split_soa(v):
        Y = v.reshape(nf, N)
        return Y[0], Y[1:4], (Y[4:] if nf > 4 else None)

    dt = 0.07
    parts, mass = P.eval_energy(X1g)
    e_o, parts_o = O.energy(X1o, cb, parts=True)
    assert parts[4] == pytest.approx(e_o, rel=1e-13, abs=1e-11)
    assert np.allclose(parts[:4], parts_o, rtol=1e-12, atol=1e-11)
    assert mass == pytest.approx(O.mass(X1o), rel=1e-14)
    for mode in (0, 1):
        Fg = P.eval_residual(X1g, X0g, dt, mode)
        Fo = to_soa(O.residual(X1o, X0o, cb, dt, mode))
        for f in range(nf):
            a, b = Fg[f * N:(f + 1) * N], Fo[f * N:(f + 1) * N]
            assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-30) + 1e-300, (mode, f)
    v = np.random.default_rng(25).standard_normal(nf * N)
    vo = O.interleave(*split_soa(v))
    for mode in (0, 1):
        Jv = P.apply_jacobian(X1g, X0g, dt, v, mode)
        Jo = to_soa(O.jacobian_scipy(X1o, X0o, cb, dt, mode) @ vo)
        for f in range(nf):
            a, b = Jv[f * N:(f + 1) * N], Jo[f * N:(f + 1) * N]
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b)), (mode, f)
    r = np.random.default_rng(26).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, dt, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, dt, O.interleave(*split_soa(r)))
    assert rc == 0
    assert rel(z, to_soa(zo)) <= 1e-9
    assert abs(z[:N].sum()) <= 1e-11 * np.abs(z[:N]).sum()
    b = -P.eval_residual(X1g, X0g, dt, 0)
    tol = 1e-11 * np.linalg.norm(b)
    x, its, res = P.linear_solve(X1g, X0g, dt, b, tol)
    assert res <= tol
    rc, xo, its_o, res_o = O.linear_solve(X1o, X0o, cb, dt, O.interleave(*split_soa(b)), tol)
    assert rc == 0
    assert rel(x, to_soa(xo)) <= 1e-8
    assert abs(its - its_o) <= max(2, its_o // 5)
    P.destroy()


@pytest.mark.parametrize("dim,n,sub,ov,elastic,neumann", [CASES[0], CASES[1], CASES[5], CASES[6]])
def test_model3_mixed_operators_match_oracle(nks, dim, n, sub, ov, elastic, neumann):
    """FP32 Jacobian action within 1e-5 of |J| |v| per row; FP32 Schwarz sweep within 1e-4."""
    cf = S.coefficients(n_eta=3)
    op = S.options(sub=sub, overlap=ov, precision="mixed")
    (c1, e1, u1), (c0, e0, u0) = _pair(dim, n, 700 + dim, elastic)
    P = nks.Problem(dim, n, 0.25, c0, e0, cf, op, neumann=neumann)
    O = oracle.Problem(dim, n, 0.25, cf, op, neumann=neumann)
    N, nf = P.N, P.nf
    cb = float(np.sum(c0) / N)
    X1g, X0g = soa(c1, e1, u1), soa(c0, e0, u0)
    X1o, X0o = O.interleave(c1, e1, u1), O.interleave(c0, e0, u0)
    to_soa = lambda Xo: soa(*O.split(Xo))
    split_soa = lambda v: (v.reshape(nf, N)[0], v.reshape(nf, N)[1:4], v.reshape(nf, N)[4:])
    dt = 0.07
    v = np.random.default_rng(27).standard_normal(nf * N)
    vo = O.interleave(*split_soa(v))
    for mode in (0, 1):
        Jv = P.apply_jacobian(X1g, X0g, dt, v, mode)
        Jm = O.jacobian_scipy(X1o, X0o, cb, dt, mode)
        Jo = to_soa(Jm @ vo)
        scale = to_soa(abs(Jm) @ np.abs(vo))
        err = np.abs(Jv - Jo)
        assert np.all(err <= 1e-5 * scale + 1e-30), (mode, float(np.max(err / (scale + 1e-300))))
    r = np.random.default_rng(28).standard_normal(nf * N)
    z = P.apply_preconditioner(X1g, X0g, dt, r)
    rc, zo = O.precond_apply(X1o, X0o, cb, dt, O.interleave(*split_soa(r)))
    assert rc == 0
    assert rel(z, to_soa(zo)) <= 1e-4
    P.destroy()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("dim,n,sub", [(2, (32, 28), (2, 2)), (3, (12, 12, 10), (2, 2, 2))])
def test_model3_steps_match_oracle(nks, dim, n, sub, precision):
    """Ten fixed-dt steps (dt = 0.01) from the App. A recipe (each eta_j drawn on its
    own): fields within 1e-8 of the oracle's, energy per step within 1e-10, mass to
    1e-12, energy non-increasing."""
    cf = S.coefficients(n_eta=3)
    op = S.options(sub=sub, overlap=1, precision=precision, newton_rtol=1e-12)
    c, e = S.initial_fields3(dim, n, 0.18, 33, eta_amp=0.05)
    P = nks.Problem(dim, n, 0.25, c, e, cf, op)
    E0, m0 = P.energy(), P.mass()
    infos = [P.step(0.01) for _ in range(10)]
    cg, eg, ug = P.get_fields()
    P.destroy()
    assert eg.shape == (3, c.size)
    O = oracle.Problem(dim, n, 0.25, cf, op)
    rc, X, oinf, e0 = O.simulate(c, e, 10, dt_replay=[0.01] * 10)
    assert rc == 0
    co, eo, uo = O.split(X)
    assert rel(cg, co) <= 1e-8, rel(cg, co)
    for j in range(3):
        assert rel(eg[j], eo[j]) <= 1e-8, (j, rel(eg[j], eo[j]))
    for I in range(dim):
        assert rel(ug[I], uo[I]) <= 1e-8, (I, rel(ug[I], uo[I]))
    assert E0 == pytest.approx(e0, rel=1e-10)
    prev = E0
    for gi, oi in zip(infos, oinf):
        assert gi["status"] == 0
        assert gi["energy"] == pytest.approx(oi["energy"], rel=1e-10)
        assert abs(gi["mass"] - m0) <= 1e-12 * abs(m0)
        assert gi["energy"] <= prev + 1e-12 * abs(prev)
        prev = gi["energy"]
    # the three order parameters were drawn independently and stay distinct
    assert rel(eg[0], eg[1]) > 1e-3


def test_equal_order_parameters_solve_the_reduced_model(nks):
    """eta_1 = eta_2 = eta_3 = eta: the three-parameter GPU solver follows the reduced
    model's GPU solver (adaptive steps replayed), each eta_j equal to its eta."""
    dim, n = 2, (32, 24)
    op = S.options(sub=(2, 2), overlap=1, newton_rtol=1e-12)
    c, e = S.initial_fields(dim, n, 0.18, 35)
    R = nks.Problem(dim, n, 0.25, c, e, S.coefficients(), dict(op, dt_mode="energy"))
    infos = [R.step() for _ in range(5)]
    cr, er, ur = R.get_fields()
    R.destroy()
    T = nks.Problem(dim, n, 0.25, c, np.stack([e, e, e]), S.coefficients(n_eta=3), op)
    tinf = [T.step(i["dt"]) for i in infos]
    ct, et, ut = T.get_fields()
    T.destroy()
    assert rel(ct, cr) <= 1e-9
    for j in range(3):
        assert rel(et[j], er) <= 1e-9, j
    for I in range(dim):
        assert rel(ut[I], ur[I]) <= 1e-9, I
    for a, b in zip(tinf, infos):
        assert a["energy"] == pytest.approx(b["energy"], rel=1e-11)


def test_model3_batch_slots_equal_their_runs_alone(nks):
    dim, n = 2, (24, 20)
    cf = S.coefficients(n_eta=3)
    op = S.options(sub=(2, 2), overlap=1, precision="mixed", dt_mode="energy")
    fields = [S.initial_fields3(dim, n, cb, sd, eta_amp=0.05) for cb, sd in [(0.15, 41), (0.2, 42), (0.17, 43)]]
    c = np.stack([f[0] for f in fields])
    e = np.stack([f[1] for f in fields])
    B = nks.Batch(dim, n, 0.25, 3, cf, op, c=c, eta=e)
    binfo = [B.step() for _ in range(3)]
    for i in range(3):
        P = nks.Problem(dim, n, 0.25, c[i], e[i], cf, op)
        infos = [P.step() for _ in range(3)]
        cg, eg, ug = P.get_fields()
        P.destroy()
        cb_, eb, ub = B.get_fields(i)
        assert np.array_equal(cg, cb_) and np.array_equal(eg, eb) and np.array_equal(ug, ub)
        for s in range(3):
            for key in ("dt", "energy", "mass", "newton_its", "gmres_its"):
                assert binfo[s][i][key] == infos[s][key], (i, s, key)
    B.destroy()
