"""Batches (nks_create_batch): several same-shape problems stepped by one kernel
launch per solver phase.  Each slot keeps its own Newton / GMRES iteration,
step size and retries, and converged slots are masked out of later launches,
so every slot must reproduce, bit for bit, the run of the same problem alone:
same fields, same step sizes, same iteration counts.  Slots load, unload and
reload independently (the serving path), and the batch result is also checked
against the FP64 oracle."""
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


def _fields(dim, n, cbars, seeds):
    cs, es = zip(*[S.initial_fields(dim, n, cb, sd) for cb, sd in zip(cbars, seeds)])
    return np.stack(cs), np.stack(es)


def _alone(nks, dim, n, c, e, op, steps, dt=None):
    P = nks.Problem(dim, n, 0.25, c, e, S.coefficients(), op)
    infos = [P.step(dt or 0.0) for _ in range(steps)]
    out = P.get_fields()
    P.destroy()
    return infos, out


def _same(a, b):
    ca, ea, ua = a
    cb, eb, ub = b
    assert np.array_equal(ca, cb) and np.array_equal(ea, eb)
    assert (ua is None and ub is None) or np.array_equal(ua, ub)


KEYS = ("dt", "t", "energy", "mass", "newton_its", "gmres_its", "retries", "status")


@pytest.mark.parametrize("dim,n,sub,prec", [(2, (24, 20), (2, 2), "fp64"), (2, (24, 20), (2, 2), "mixed"),
                                            (3, (9, 10, 8), (2, 2, 2), "fp64"), (3, (9, 10, 8), (2, 2, 2), "mixed")])
def test_batch_slots_equal_their_runs_alone(nks, dim, n, sub, prec):
    op = S.options(sub=sub, overlap=1, precision=prec, dt_mode="energy")
    cbars, seeds = [0.14, 0.2, 0.17, 0.23], [11, 12, 13, 14]
    c, e = _fields(dim, n, cbars, seeds)
    B = nks.Batch(dim, n, 0.25, 4, S.coefficients(), op, c=c, eta=e)
    steps = 3
    binfo = [B.step() for _ in range(steps)]
    for i in range(4):
        infos, fields = _alone(nks, dim, n, c[i], e[i], op, steps)
        _same(B.get_fields(i), fields)
        for s in range(steps):
            for k in KEYS:
                assert binfo[s][i][k] == infos[s][k], (i, s, k)
    B.destroy()


def test_batch_slots_load_unload_and_active_mask(nks):
    dim, n = 2, (20, 22)
    op = S.options(sub=(2, 2), overlap=1, dt_mode="energy")
    c, e = _fields(dim, n, [0.15, 0.21, 0.18], [21, 22, 23])
    B = nks.Batch(dim, n, 0.25, 3, S.coefficients(), op)
    assert not any(B.loaded(i) for i in range(3))
    B.load(1, c[0], e[0])
    r1 = B.step()
    assert r1[0] is None and r1[2] is None and r1[1]["status"] == 0
    B.load(2, c[1], e[1])             # joins while slot 1 is mid-run
    r2 = B.step(active=[0, 1, 1])
    assert r2[0] is None and r2[1]["status"] == 0 and r2[2]["status"] == 0
    B.step(active=[0, 0, 1])          # slot 1 waits one step
    B.step()
    # slot 1: three steps; slot 2: three steps, as when run alone
    _same(B.get_fields(1), _alone(nks, dim, n, c[0], e[0], op, 3)[1])
    _same(B.get_fields(2), _alone(nks, dim, n, c[1], e[1], op, 3)[1])
    B.unload(1)
    B.load(0, c[2], e[2])
    B.step(dt=0.02)
    _same(B.get_fields(0), _alone(nks, dim, n, c[2], e[2], op, 1, dt=0.02)[1])
    # a checkpoint of one slot restores into another slot of the batch
    blob = B.get_state(2)
    B.set_state(1, blob)
    B.step(active=[0, 1, 1])
    _same(B.get_fields(1), B.get_fields(2))
    B.destroy()


def test_batch_against_fp64_oracle(nks):
    dim, n = 2, (24, 24)
    op = S.options(sub=(2, 2), overlap=1)
    c, e = _fields(dim, n, [0.16, 0.22], [31, 32])
    B = nks.Batch(dim, n, 0.25, 2, S.coefficients(), op, c=c, eta=e)
    steps = 4
    for _ in range(steps):
        B.step(dt=0.01)
    for i in range(2):
        O = oracle.Problem(dim, n, 0.25, S.coefficients(), dict(op, newton_rtol=1e-12))
        rc, X, oinf, e0 = O.simulate(c[i], e[i], steps, dt_replay=[0.01] * steps)
        assert rc == 0
        co, eo, uo = O.split(X)
        cg, eg, ug = B.get_fields(i)
        for a, b in ((cg, co), (eg, eo), (ug, uo)):
            assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b)
        m0 = c[i].sum() * 0.25 ** 2
        assert abs(B.mass(i) - m0) <= 1e-12 * m0
    B.destroy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(nks, prec):
    """GMRES iterations replayed from captured CUDA graphs give the same bits as
    the same kernels launched one by one; the launch counters agree too."""
    dim, n = 2, (24, 20)
    c, e = _fields(dim, n, [0.16, 0.2, 0.18], [41, 42, 43])
    out = {}
    for graphs in (0, 1):
        op = S.options(sub=(2, 2), overlap=1, precision=prec, dt_mode="energy", graphs=graphs)
        B = nks.Batch(dim, n, 0.25, 3, S.coefficients(), op, c=c, eta=e)
        B.reset_stats()
        infos = [B.step() for _ in range(3)]
        out[graphs] = ([B.get_fields(i) for i in range(3)], infos, B.get_stats())
        B.destroy()
    for i in range(3):
        _same(out[0][0][i], out[1][0][i])
    assert out[0][1] == out[1][1]
    assert out[0][2]["kernel_launches"] == out[1][2]["kernel_launches"]
