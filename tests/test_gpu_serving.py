"""Serving (nks_server_*) and the decomposition autotuner (nks_autotune).

Serving: requests of several grid shapes arrive while others run; same-shape
requests share a batch and join it in free slots between batch steps.  Every
result must be bitwise the result of the same request run alone, whether it
ran in a mix (several shape groups at once, slots reused) or alone by the
memory budget (one slot at a time)."""
import threading
import time

import numpy as np
import pytest

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


SIDE2, SIDE3 = 16, 8


def _req_opts(dim, n, base):
    side = SIDE3 if dim == 3 else SIDE2
    sub = tuple(max(2, (n[J] + side // 2) // side) for J in range(dim))
    return dict(base, sub=sub)


def _alone(nks, dim, n, c, e, op, steps):
    P = nks.Problem(dim, n, 0.25, c, e, S.coefficients(), op)
    for _ in range(steps):
        P.step()
    out = P.get_fields()
    P.destroy()
    return out


REQS = [(2, (32, 32), 0.15, 3), (2, (40, 36), 0.2, 4), (2, (32, 32), 0.22, 2), (3, (16, 16, 16), 0.18, 2),
        (2, (40, 36), 0.12, 3), (2, (32, 32), 0.17, 5), (3, (16, 16, 16), 0.2, 3)]


def _run_server(nks, base, **server_kw):
    srv = nks.Server(S.coefficients(), base, box_side_2d=SIDE2, box_side_3d=SIDE3, **server_kw)
    fields = []
    ids = []

    def submit(i):
        dim, n, cb, steps = REQS[i]
        c, e = S.initial_fields(dim, n, cb, 500 + i)
        fields.append((i, c, e))
        ids.append((i, srv.submit(dim, n, 0.25, c, e, steps)))

    for i in range(4):
        submit(i)
    time.sleep(0.05)  # the rest arrive while the first are running
    for i in range(4, len(REQS)):
        submit(i)
    res = {i: srv.wait(rid) for i, rid in ids}
    srv.destroy()
    return res, {i: (c, e) for i, c, e in fields}


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_served_results_equal_alone_in_the_mix(nks, prec):
    base = S.options(precision=prec, dt_mode="energy", overlap=1)
    res, fields = _run_server(nks, base, max_slots=2, max_groups=4)
    for i, (dim, n, cb, steps) in enumerate(REQS):
        r, (c, e, u) = res[i]
        assert r["status"] == 0 and r["steps"] == steps, r
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        ca, ea, ua = _alone(nks, dim, n, *fields[i], _req_opts(dim, n, base), steps)
        assert np.array_equal(c, ca) and np.array_equal(e, ea) and np.array_equal(u, ua), i


def test_memory_budget_bounds_admission(nks):
    """A budget of one 3-D slot: a 3-D request runs only with nothing else on the
    device, the reserved bytes never exceed the budget, results stay bitwise."""
    base = S.options(precision="mixed", dt_mode="energy", overlap=1)
    per = {}
    for dim, n, _, _ in REQS:
        B = nks.Batch(dim, n, 0.25, 1, S.coefficients(), _req_opts(dim, n, base))
        per[(dim, n)] = B.device_bytes()
        B.destroy()
    budget = per[(3, (16, 16, 16))]
    assert budget == max(per.values())
    srv = nks.Server(S.coefficients(), base, box_side_2d=SIDE2, box_side_3d=SIDE3, max_slots=4, max_groups=4,
                     mem_budget=budget)
    seen, stop = [], [False]

    def poll():
        while not stop[0]:
            st = srv.status()
            seen.append(st["bytes_reserved"] <= st["mem_budget"])
            time.sleep(0.002)

    th = threading.Thread(target=poll)
    th.start()
    ids, fields = [], {}
    for i, (dim, n, cb, steps) in enumerate(REQS):
        c, e = S.initial_fields(dim, n, cb, 700 + i)
        fields[i] = (c, e)
        ids.append((i, srv.submit(dim, n, 0.25, c, e, steps)))
    res = {i: srv.wait(rid) for i, rid in ids}
    stop[0] = True
    th.join()
    srv.destroy()
    assert seen and all(seen)
    spans = {i: (r["t_admit"], r["t_done"]) for i, (r, _) in res.items()}
    for i, (dim, n, cb, steps) in enumerate(REQS):
        r, (c, e, u) = res[i]
        assert r["status"] == 0
        if dim == 3:
            a0, d0 = spans[i]
            for k, (a1, d1) in spans.items():
                if k != i:
                    assert d1 <= a0 + 1e-9 or a1 >= d0 - 1e-9, (i, k)
        ca, ea, _ = _alone(nks, dim, n, *fields[i], _req_opts(dim, n, base), steps)
        assert np.array_equal(c, ca) and np.array_equal(e, ea), i


def test_concurrent_submitters(nks):
    """submit and wait from several host threads at once"""
    base = S.options(precision="mixed", dt_mode="energy", overlap=1)
    srv = nks.Server(S.coefficients(), base, box_side_2d=SIDE2, box_side_3d=SIDE3, max_slots=3)
    out, errs = {}, []

    def client(k):
        try:
            dim, n, cb, steps = REQS[k]
            c, e = S.initial_fields(dim, n, cb, 900 + k)
            rid = srv.submit(dim, n, 0.25, c, e, steps)
            out[k] = (srv.wait(rid), c, e)
        except Exception as ex:  # pragma: no cover - reported below
            errs.append(ex)

    th = [threading.Thread(target=client, args=(k,)) for k in range(len(REQS))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    srv.destroy()
    assert not errs
    for k, ((r, (c, e, u)), c0, e0) in out.items():
        dim, n, cb, steps = REQS[k]
        assert r["status"] == 0
        ca, ea, _ = _alone(nks, dim, n, c0, e0, _req_opts(dim, n, base), steps)
        assert np.array_equal(c, ca) and np.array_equal(e, ea), k


def test_autotune_picks_the_fastest_valid_decomposition(nks):
    dim, n = 2, (48, 40)
    c, e = S.initial_fields(dim, n, 0.18, 7)
    cands = [((2, 2), 1), ((3, 2), 1), ((4, 4), 2), ((1, 1), 1)]  # the last box does not fit the grid
    op, table, chosen = nks.autotune(dim, n, 0.25, c, e, S.coefficients(), S.options(), candidates=cands)
    times = [t for _, _, t in table]
    assert times[3] == -1.0
    valid = [i for i in range(3) if times[i] > 0]
    assert valid and chosen == min(valid, key=lambda i: times[i])
    assert tuple(op["sub"]) == cands[chosen][0] and op["overlap"] == cands[chosen][1]
    # the built-in candidate list
    op2, table2, chosen2 = nks.autotune(dim, n, 0.25, c, e, S.coefficients(), S.options())
    assert chosen2 >= 0 and all(o >= 1 for o in op2["sub"])


def test_served_results_match_the_oracle(nks):
    """Requests served in a mix (two shape groups, slots shared) against the FP64
    oracle run of each request alone: fixed dt so the oracle takes the same step
    sizes; relative L2 per field <= 1e-8 and energy, mass after the last step."""
    import oracle
    base = S.options(precision="mixed", dt_mode="fixed", overlap=1)
    reqs = [(2, (32, 32), 0.15, 3, 701), (3, (16, 16, 16), 0.2, 2, 702), (2, (40, 36), 0.12, 3, 703),
            (2, (32, 32), 0.22, 2, 704)]
    srv = nks.Server(S.coefficients(), base, box_side_2d=SIDE2, box_side_3d=SIDE3, max_slots=2, max_groups=4)
    init = [S.initial_fields(dim, n, cb, seed) for dim, n, cb, _, seed in reqs]
    ids = [srv.submit(dim, n, 0.25, c, e, steps) for (dim, n, _, steps, _), (c, e) in zip(reqs, init)]
    served = [srv.wait(rid) for rid in ids]
    srv.destroy()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    for (dim, n, _, steps, _), (c0, e0), (r, (c, e, u)) in zip(reqs, init, served):
        assert r["status"] == 0 and r["steps"] == steps, r
        op = dict(_req_opts(dim, n, base), precision="fp64", newton_rtol=1e-12)
        O = oracle.Problem(dim, n, 0.25, S.coefficients(), op)
        rc, X, infos, _ = O.simulate(c0, e0, steps)
        assert rc == 0
        co, eo, uo = O.split(X)
        assert rel(c, co) <= 1e-8 and rel(e, eo) <= 1e-8, (n, rel(c, co), rel(e, eo))
        for I in range(dim):
            assert rel(u[I], uo[I]) <= 1e-8, (n, I, rel(u[I], uo[I]))
        assert r["energy"] == pytest.approx(infos[-1]["energy"], rel=1e-10)
        assert r["mass"] == pytest.approx(infos[-1]["mass"], rel=1e-12)
        assert r["t"] == pytest.approx(sum(i["dt"] for i in infos), rel=1e-14)
