"""Full-size parity after several time steps: the CUDA path against the FP64
oracle's run of the same workload.

The oracle's references (``tests/golden/full_<workload>.json``, written by
``tests/golden/make_full_size.py``, which calls only the oracle) hold, for the
first steps of the 2-D 1024^2 and 3-D 128^3 workloads and of the 3-D 128^3
workload with three order parameters (App. A), the step sizes the
oracle's adaptive controller chose (Sec. 4, Eq. sencondt), the energy and mass
after every step, and for every field of the final state its L2 norm, a
256-row seeded sign sketch and its values at 1024 seeded points.  Here the
GPU solver, FP64 and mixed precision, replays those step sizes from the same
initial state in the workload's own launch configuration (at the references'
Newton tolerance), and:

  * the relative L2 error per field, estimated as |S x_gpu - S x_oracle| /
    |x_oracle| (Johnson-Lindenstrauss: with 256 rows the estimate lies within
    0.7..1.3 of the true value except with probability < 1e-6), is <= 1e-8;
  * at the sampled points the error is <= 1e-8 of the field's RMS value;
  * energy matches to 1e-10 and mass to 1e-12 after every step, the energy
    does not increase (Theorem 3.2) and the mass stays at its initial value.
"""
import json
import os

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
WORKLOADS = ["3d128", "2d1024", "3d128eta3"]


@pytest.fixture(scope="module")
def nks():
    import torch
    assert torch.cuda.is_available()
    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as m
    return m


def golden(name):
    with open(os.path.join(HERE, "golden", "full_%s.json" % name)) as fh:
        return json.load(fh)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", WORKLOADS)
def test_full_size_steps_match_the_oracle(nks, name, precision):
    G = golden(name)
    cfg = S.CONFIGS[name]
    op = S.options(**cfg["opts"])
    op["precision"] = precision
    # the references' Newton tolerance (eps_r = 1e-12): at the workload's 1e-10 the
    # 1024^2 displacement is settled only to ~3e-7 relative, since the displacement
    # rows carry about 1e-12 of ||F|| and the GMRES cap leaves them last to converge
    op["newton_rtol"] = G["newton_rtol"]
    c, e = S.config_fields(cfg)
    P = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg), op)
    E0 = P.energy()
    assert E0 == pytest.approx(G["energy0"], rel=1e-10)
    m0 = P.mass()
    prevE = E0
    for st in G["per_step"]:
        info = P.step(st["dt"])
        assert info["status"] == 0
        assert info["energy"] == pytest.approx(st["energy"], rel=1e-10)
        assert abs(info["mass"] - st["mass"]) <= 1e-12 * abs(st["mass"])
        assert abs(info["mass"] - m0) <= 1e-12 * abs(m0)
        assert info["energy"] <= prevE + 1e-12 * abs(prevE)
        prevE = info["energy"]
    cg, eg, ug = P.get_fields()
    P.destroy()
    fields = {"c": cg, "eta": eg} if eg.ndim == 1 else {"c": cg, **{"eta%d" % (j + 1): eg[j] for j in range(len(eg))}}
    if ug is not None:
        for I in range(len(ug)):
            fields["u%d" % (I + 1)] = ug[I]
    assert sorted(fields) == sorted(G["fields"])
    names = list(G["fields"])
    sk = S.sign_sketch([fields[f] for f in names], G["sketch"]["k"], G["sketch"]["seed"])
    idx = np.array(G["samples"]["index"], dtype=np.int64)
    for i, f in enumerate(names):
        ref = G["fields"][f]
        est = np.linalg.norm(sk[i] - np.array(ref["sketch"])) / ref["norm"]
        rms = ref["norm"] / np.sqrt(c.size)
        pt = np.max(np.abs(fields[f][idx] - np.array(ref["at_samples"]))) / rms
        print("%s %s %s: rel L2 (sketch) %.2e, max sampled %.2e" % (name, precision, f, est, pt))
        assert est <= 1e-8, (f, est)
        assert pt <= 1e-8, (f, pt)


def test_3d256_mixed_two_steps(nks):
    """The 256^3 workload (mixed precision, 16^3 Schwarz boxes): the oracle's full
    run does not fit the host (its CSR Jacobian, Schwarz factors and Krylov basis
    need about 140 GB), so two adaptive steps are checked by what holds at any
    size: mass to 1e-12, a non-increasing energy, the FP64 solver replaying the
    same dt within 1e-8 per field, and the oracle's residual of the FP64 result's
    last step (its defining equation F(X^{n+1}; X^n) = 0, Eq. NSOA-1) below
    1e-9 of the residual at the step's start."""
    import oracle
    cfg = S.CONFIGS["3d256"]
    op = S.options(**cfg["opts"])
    assert op["precision"] == "mixed"
    c, e = S.config_fields(cfg)
    cf = S.config_coefficients(cfg)
    P = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, cf, op)
    E0, m0 = P.energy(), P.mass()
    infos = [P.step() for _ in range(2)]
    mixed = P.get_fields()
    P.destroy()
    prev = E0
    for i in infos:
        assert i["status"] == 0
        assert abs(i["mass"] - m0) <= 1e-12 * abs(m0)
        assert i["energy"] <= prev + 1e-12 * abs(prev)
        prev = i["energy"]
    Q = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, cf, dict(op, precision="fp64"))
    Q.step(infos[0]["dt"])
    X1 = Q.get_fields()
    Q.step(infos[1]["dt"])
    X2 = Q.get_fields()
    Q.destroy()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(mixed[0], X2[0]) <= 1e-8 and rel(mixed[1], X2[1]) <= 1e-8
    for I in range(3):
        assert rel(mixed[2][I], X2[2][I]) <= 1e-8
    O = oracle.Problem(cfg["dim"], cfg["n"], cfg["h"], cf)
    cbar0 = float(np.sum(c) / c.size)
    Y1 = O.interleave(X1[0], X1[1], X1[2])
    Y2 = O.interleave(X2[0], X2[1], X2[2])
    dt = infos[1]["dt"]
    f0 = np.linalg.norm(O.residual(Y1, Y1, cbar0, dt))
    f2 = np.linalg.norm(O.residual(Y2, Y1, cbar0, dt))
    print("3d256: |F(X2; X1)| / |F(X1; X1)| = %.2e" % (f2 / f0))
    assert f2 <= 1e-9 * f0
