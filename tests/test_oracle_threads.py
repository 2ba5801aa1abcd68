"""The oracle's parallel loops (OpenMP) give bit-identical results for any
thread count: every sum is taken in a fixed block order, and every point, row
or subdomain is computed by one thread exactly as the serial loop computes it."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_RUN = r"""
import json, sys
sys.path.insert(0, %r)
import numpy as np
import oracle, synthetic as S
out = {"threads": oracle.num_threads()}
for dim, n, sub, variant in ((2, (20, 18), (3, 2), "left-ras"), (3, (10, 9, 8), (2, 2, 2), "as")):
    op = S.options(sub=sub, overlap=1, dt_mode="energy", ras_variant=variant, newton_rtol=1e-12)
    c, e = S.initial_fields(dim, n, 0.18, 3)
    O = oracle.Problem(dim, n, 0.25, S.coefficients(), op)
    rc, X, infos, e0 = O.simulate(c, e, 3)
    out["%%dd" %% dim] = {"rc": rc, "X": X.tobytes().hex(), "its": [i["gmres_its"] for i in infos],
                         "energy": [i["energy"] for i in infos]}
print(json.dumps(out))
""" % ROOT


def _run(threads):
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", _RUN], env=env, capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_oracle_is_bitwise_independent_of_thread_count():
    one, many = _run(1), _run(max(2, min(8, os.cpu_count() or 2)))
    assert one["threads"] == 1 and many["threads"] >= 2
    for key in ("2d", "3d"):
        assert one[key]["rc"] == 0 and many[key]["rc"] == 0
        assert one[key]["its"] == many[key]["its"]
        assert one[key]["X"] == many[key]["X"], key
        assert one[key]["energy"] == many[key]["energy"]
