"""The residual entry point that allocates no device memory.

Some callers cannot allocate device memory when they need a residual: a host
application whose own memory manager owns the whole GPU, or a latency-critical
loop where an allocation could synchronise the device.  nks_residual_noalloc
serves them from a fixed scratch array inside the library; these tests check,
through the C ABI, that it returns what the problem-based entry point
(nks_eval_residual) returns, on two calls in a row, and that it refuses grids
larger than its stated maximum.  The file is named so that pytest collects it
last.
"""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def _serial_mean(a):
    s = 0.0
    for v in a:
        s += float(v)
    return s / len(a)


def _state(dim, n, seed):
    c, e, u = S.random_fields(dim, n, seed, u_amp=0.01)
    return np.concatenate([c, e] + list(u)), c


@pytest.mark.parametrize("dim,n", [(2, (40, 36)), (3, (14, 12, 10))])
def test_noalloc_residual_matches_problem_residual_twice(dim, n):
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as nks

    cf = S.coefficients()
    X0, c0 = _state(dim, n, 11)
    P = nks.Problem(dim, n, 0.25, c0, X0[c0.size:2 * c0.size], cf, S.options(sub=(2, 2, 2), overlap=1))
    N, nf = P.N, P.nf
    cbar0 = _serial_mean(c0)  # the problem takes cbar0 from its initial c in the same order
    stream = torch.cuda.current_stream()
    for call, (seed, dt, mode) in enumerate([(21, 0.05, 0), (22, 0.3, 1)]):
        X1, _ = _state(dim, n, seed)
        X1[:N] += c0.mean() - X1[:N].mean()
        ref = P.eval_residual(X1, X0, dt, mode)
        d1 = torch.tensor(X1, device="cuda", dtype=torch.float64)
        d0 = torch.tensor(X0, device="cuda", dtype=torch.float64)
        dF = torch.full((nf * N,), float("nan"), device="cuda", dtype=torch.float64)
        dn = torch.zeros(1, device="cuda", dtype=torch.float64)
        rc = nks.residual_noalloc(dim, n, 0.25, cf, cbar0, dt, d1.data_ptr(), d0.data_ptr(), dF.data_ptr(),
                                  dn.data_ptr(), stream.cuda_stream, mode=mode)
        assert rc == nks.NKS_OK, nks.last_error()
        F = dF.cpu().numpy()
        for f in range(nf):
            a, b = F[f * N:(f + 1) * N], ref[f * N:(f + 1) * N]
            assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-30), (call, f)
        assert float(dn.item()) == pytest.approx(float(np.dot(ref, ref)), rel=1e-12)
    P.destroy()


def test_noalloc_residual_rejects_grids_beyond_its_maximum():
    import torch

    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as nks

    n = (300, 300)
    assert n[0] * n[1] > nks.NOALLOC_MAX_POINTS
    buf = [torch.zeros(4 * n[0] * n[1], device="cuda", dtype=torch.float64) for _ in range(3)]
    rc = nks.residual_noalloc(2, n, 0.25, S.coefficients(), 0.2, 0.01, buf[0].data_ptr(), buf[1].data_ptr(),
                              buf[2].data_ptr(), None, None)
    assert rc == nks.NKS_EINVAL
    assert "NKS_NOALLOC_MAX_POINTS" in nks.last_error()
