"""Writes the full-size oracle references of the parity tests.

    python tests/golden/make_full_size.py 3d128 5      # -> tests/golden/full_3d128.json
    python tests/golden/make_full_size.py 2d1024 5     # -> tests/golden/full_2d1024.json
    python tests/golden/make_full_size.py 3d128eta3 3  # -> tests/golden/full_3d128eta3.json

For a workload of ``synthetic.CONFIGS`` this runs the FP64 oracle (``oracle/``,
nothing else computes) from the workload's initial state for the given number
of adaptive time steps, with the Newton tolerance of the parity references
(eps_r = 1e-12; the workload's own solver settings otherwise), and stores:

  * per step: dt, energy, mass, Newton and GMRES iterations (the dt list is
    what the GPU tests replay);
  * per field of the final state (c, eta or eta_1..eta_3, u_1..u_d): its L2 norm, a 256-row
    seeded sign sketch (``synthetic.sign_sketch``: |S a - S b| estimates the
    L2 distance |a - b|), and its values at 1024 seeded points
    (``synthetic.sample_points``).

The fields themselves (tens of MB) are not stored.  Runs take tens of minutes
on a few cores (OMP_NUM_THREADS sets the oracle's threads).
"""
import json
import os
import platform
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic as S  # noqa: E402

PARITY_RTOL = 1e-12  # Newton tolerance of the oracle's parity references


def oracle_hash():
    try:
        return subprocess.check_output(["git", "-C", ROOT, "log", "-1", "--format=%h", "--", "oracle/nks_oracle.c"],
                                       text=True).strip()
    except Exception:
        return None


def main(workload, steps):
    cfg = S.CONFIGS[workload]
    op = S.options(**cfg["opts"])
    op["newton_rtol"] = PARITY_RTOL
    op["precision"] = "fp64"
    c, e = S.config_fields(cfg)
    cf = S.config_coefficients(cfg)
    O = oracle.Problem(cfg["dim"], cfg["n"], cfg["h"], cf, op)
    t0 = time.time()
    rc, X, infos, e0 = O.simulate(c, e, steps)
    wall = time.time() - t0
    if rc != 0:
        raise SystemExit("oracle failed: rc %d" % rc)
    cx, ex, ux = O.split(X)
    # one order parameter: "eta"; three (App. A): "eta1".."eta3"
    fields = {"c": cx, "eta": ex} if ex.ndim == 1 else {"c": cx, **{"eta%d" % (j + 1): ex[j] for j in range(len(ex))}}
    if ux is not None:
        for I in range(cfg["dim"]):
            fields["u%d" % (I + 1)] = ux[I]
    names = list(fields)
    sk = S.sign_sketch([fields[f] for f in names])
    idx = S.sample_points(c.size)
    out = {
        "_source": "FP64 oracle (oracle/nks_oracle.c, commit %s), written by tests/golden/make_full_size.py" % oracle_hash(),
        "workload": workload, "desc": cfg["desc"], "steps": steps,
        "newton_rtol": PARITY_RTOL, "energy0": e0,
        "oracle_threads": oracle.num_threads(), "wall_s": wall, "host": platform.machine(),
        "per_step": [{k: i[k] for k in ("dt", "energy", "mass", "newton_its", "gmres_its")} for i in infos],
        "sketch": {"k": 256, "seed": 7}, "samples": {"count": int(idx.size), "seed": 11, "index": idx.tolist()},
        "fields": {f: {"norm": float(np.linalg.norm(fields[f])), "sketch": sk[i].tolist(),
                       "at_samples": fields[f][idx].tolist()} for i, f in enumerate(names)},
    }
    path = os.path.join(HERE, "full_%s.json" % workload)
    with open(path, "w") as fh:
        fh.write("{\n" + ",\n".join("%s: %s" % (json.dumps(key), json.dumps(val)) for key, val in out.items()) + "\n}\n")
    print(path, "%.0f s" % wall, [(i["newton_its"], i["gmres_its"], i["dt"]) for i in infos])


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 5)
