"""The residual entry point that allocates no device memory.

Some callers cannot allocate device memory when they need a residual: a host
application whose own memory manager owns the whole GPU, or a latency-critical
loop where an allocation could synchronise the device.  nks_residual_noalloc
serves them from a fixed scratch array inside the library; these tests check,
through the C ABI, that it returns what the problem-based entry point
(nks_eval_residual) and the FP64 oracle return, on two calls in a row, with and
without elasticity and at its largest accepted grid, that the device's free
memory does not move across a call, and that it refuses grids larger than its
stated maximum.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu


def _serial_mean(a):
    s = 0.0
    for v in a:
        s += float(v)
    return s / len(a)


def _state(dim, n, seed, elastic=True):
    c, e, u = S.random_fields(dim, n, seed, u_amp=0.01)
    return np.concatenate([c, e] + (list(u) if elastic else [])), c


def _nks():
    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as nks
    return nks


def _close(a, b, tol=1e-12):
    return np.max(np.abs(a - b)) <= tol * max(np.max(np.abs(b)), 1e-30)


# (dim, grid, elastic): 3-D and 2-D with elasticity, the model without it (nf = 2), and the
# largest grid the entry point accepts (256^2 = NKS_NOALLOC_MAX_POINTS points)
CASES = [(2, (40, 36), True), (3, (14, 12, 10), True), (2, (37, 29), False), (2, (256, 256), True)]


@pytest.mark.parametrize("dim,n,elastic", CASES)
def test_noalloc_residual_matches_problem_and_oracle_twice(dim, n, elastic):
    import torch

    nks = _nks()
    cf = S.coefficients() if elastic else S.coefficients(C11=0.0, C12=0.0, C44=0.0)
    X0, c0 = _state(dim, n, 11, elastic)
    N = c0.size
    nf = 2 + (dim if elastic else 0)
    assert X0.size == nf * N
    if n == (256, 256):
        assert N == nks.NOALLOC_MAX_POINTS
    sub = tuple(max(2, v // 32) for v in n)  # Schwarz boxes of at most 32 + 2 cells per axis
    P = nks.Problem(dim, n, 0.25, c0, X0[N:2 * N], cf, S.options(sub=sub, overlap=1))
    assert P.nf == nf
    O = oracle.Problem(dim, n, 0.25, cf)
    cbar0 = _serial_mean(c0)  # the problem takes cbar0 from its initial c in the same order
    stream = torch.cuda.current_stream()
    dF = torch.full((nf * N,), float("nan"), device="cuda", dtype=torch.float64)
    dn = torch.zeros(1, device="cuda", dtype=torch.float64)
    free_after = []
    for call, (seed, dt, mode) in enumerate([(21, 0.05, 0), (22, 0.3, 1)]):
        X1, _ = _state(dim, n, seed, elastic)
        X1[:N] += c0.mean() - X1[:N].mean()
        ref = P.eval_residual(X1, X0, dt, mode)
        Fo = O.residual(O.interleave(X1[:N], X1[N:2 * N], X1[2 * N:].reshape(-1, N) if elastic else None),
                        O.interleave(X0[:N], X0[N:2 * N], X0[2 * N:].reshape(-1, N) if elastic else None),
                        cbar0, dt, mode).reshape(N, nf).T.reshape(-1)
        d1 = torch.tensor(X1, device="cuda", dtype=torch.float64)
        d0 = torch.tensor(X0, device="cuda", dtype=torch.float64)
        dF.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = nks.residual_noalloc(dim, n, 0.25, cf, cbar0, dt, d1.data_ptr(), d0.data_ptr(), dF.data_ptr(),
                                  dn.data_ptr(), stream.cuda_stream, mode=mode)
        assert rc == nks.NKS_OK, nks.last_error()
        torch.cuda.synchronize()
        free_after.append((free_before, torch.cuda.mem_get_info()[0]))
        F = dF.cpu().numpy()
        for f in range(nf):
            a, b, o = F[f * N:(f + 1) * N], ref[f * N:(f + 1) * N], Fo[f * N:(f + 1) * N]
            assert _close(a, b), (call, f)
            assert _close(a, o, 1e-11), (call, f)
        if mode == 1 and not elastic:
            assert not F.any()  # the displacement-only system is empty
        assert float(dn.item()) == pytest.approx(float(np.dot(ref, ref)), rel=1e-12, abs=1e-300)
    # the second call (scratch set up by the first) leaves the device's free memory unchanged
    assert free_after[1][0] == free_after[1][1], free_after
    P.destroy()


def test_noalloc_residual_rejects_grids_beyond_its_maximum():
    import torch

    nks = _nks()
    buf = [torch.zeros(4 * 300 * 300, device="cuda", dtype=torch.float64) for _ in range(3)]
    for n in [(300, 300), (257, 256), (70000, 3)]:
        rc = nks.residual_noalloc(2, n, 0.25, S.coefficients(), 0.2, 0.01, buf[0].data_ptr(), buf[1].data_ptr(),
                                  buf[2].data_ptr(), None, None)
        assert rc == nks.NKS_EINVAL, n
        assert "NKS_NOALLOC_MAX_POINTS" in nks.last_error()
    # an axis so long that the product of the sides would overflow is refused by the per-axis check
    rc = nks.residual_noalloc(3, (2 ** 30, 2 ** 30, 2 ** 30), 0.25, S.coefficients(), 0.2, 0.01, buf[0].data_ptr(),
                              buf[1].data_ptr(), buf[2].data_ptr(), None, None)
    assert rc == nks.NKS_EINVAL
