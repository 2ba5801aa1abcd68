"""The oracle's Schwarz preconditioner with its ILU(0) subdomain solver and the
projection, against the definitions of Sec. 4 built here from dense matrices:

    z = P sum_i R_i^0T (L_i U_i)^-1 R_i^delta r     (left-RAS)

with A_i = J restricted to the overlapped box i (periodic boxes wrap; Neumann
boxes stop at the boundary), L_i U_i its ILU(0) factorisation on the stored
pattern of A_i (textbook row-by-row elimination, unit L, no fill), and P the
orthogonal projection that removes the mean of z_c and, from the displacement,
its component in the null space of the discrete strain: on periodic grids the
sign patterns prod_J (-1)^{x_J} over the axes with an even number of cells (the
constant included), with Neumann boundaries the d translations and, for every
pair of axes I < J with an even number of cells each, the discrete rotation
u_I = -S(x_J), u_J = S(x_I), S(x) = floor((x + 1) / 2) - n / 4.  P is formed
here as a least-squares projection onto those modes, not as the oracle's
one-mode-at-a-time subtraction.
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
import synthetic as S


def _axis_cells(nn, sb, s, delta, neumann):
    o0, o1 = s * nn // sb, (s + 1) * nn // sb
    if neumann:
        cells = list(range(max(0, o0 - delta), min(nn, o1 + delta)))
    elif o1 - o0 + 2 * delta >= nn:
        cells = list(range(nn))
    else:
        cells = [(o0 - delta + t) % nn for t in range(o1 - o0 + 2 * delta)]
    return [(c, o0 <= c < o1) for c in cells]


def _boxes(n, sub, delta, neumann):
    """(points, owned mask) per box, boxes and their points with x fastest"""
    axes = [[_axis_cells(nn, sb, s, delta, neumann) for s in range(sb)] for nn, sb in zip(n, sub)]
    for combo in itertools.product(*[range(len(a)) for a in axes[::-1]]):
        cells = [axes[J][s] for J, s in enumerate(combo[::-1])]
        pts, own = [], []
        for idx in itertools.product(*[range(len(c)) for c in cells[::-1]]):
            p, stride, ok = 0, 1, True
            for J, t in enumerate(idx[::-1]):
                c, o = cells[J][t]
                p += c * stride
                stride *= n[J]
                ok = ok and o
            pts.append(p)
            own.append(ok)
        yield np.array(pts), np.array(own)


def _ilu0(A, pattern):
    """ILU(0) on `pattern`: for each row i, for each k < i of its pattern in order,
    l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for the j > k of row i's pattern"""
    A = A.copy()
    n = A.shape[0]
    for i in range(n):
        for k in np.nonzero(pattern[i, :i])[0]:
            A[i, k] /= A[k, k]
            js = k + 1 + np.nonzero(pattern[i, k + 1:])[0]
            A[i, js] -= A[i, k] * A[k, js]
    return A


def _coords(n):
    N = int(np.prod(n))
    p = np.arange(N)
    out, stride = [], 1
    for nn in n:
        out.append((p // stride) % nn)
        stride *= nn
    return out


def _null_modes(n, neumann):
    """displacement null modes as (d, N) arrays (one per mode)"""
    d, N = len(n), int(np.prod(n))
    x = _coords(n)
    modes = []
    if not neumann:
        even = [J for J in range(d) if n[J] % 2 == 0]
        for I in range(d):
            for m in range(1 << len(even)):
                sg = np.ones(N)
                for b, J in enumerate(even):
                    if m & (1 << b):
                        sg *= np.where(x[J] % 2, -1.0, 1.0)
                md = np.zeros((d, N))
                md[I] = sg
                modes.append(md)
    else:
        for I in range(d):
            md = np.zeros((d, N))
            md[I] = 1.0
            modes.append(md)
        stair = [(x[J] + 1) // 2 - n[J] / 4.0 for J in range(d)]
        for I in range(d):
            for J in range(I + 1, d):
                if n[I] % 2 or n[J] % 2:
                    continue
                md = np.zeros((d, N))
                md[I] = -stair[J]
                md[J] = stair[I]
                modes.append(md)
    return modes


def _project(z, n, nf, ku, neumann):
    N = int(np.prod(n))
    Z = z.reshape(N, nf).copy()
    Z[:, 0] -= Z[:, 0].mean()
    if nf > ku:
        U = Z[:, ku:].T.reshape(-1)  # (d N) stacked displacement
        Phi = np.stack([m.reshape(-1) for m in _null_modes(n, neumann)], axis=1)
        coef = np.linalg.lstsq(Phi, U, rcond=None)[0]
        U = U - Phi @ coef
        Z[:, ku:] = U.reshape(len(n), N).T
    return Z.reshape(-1)


CASES = [(2, (12, 10), (2, 2), 1, False), (2, (11, 10), (3, 2), 2, False), (3, (6, 6, 4), (2, 2, 2), 1, False),
         (2, (12, 10), (2, 2), 1, True), (3, (6, 5, 4), (2, 2, 2), 1, True), (1, (15,), (3,), 2, False)]


@pytest.mark.parametrize("dim,n,sub,delta,neumann", CASES)
def test_left_ras_ilu0_and_projection_match_their_definitions(dim, n, sub, delta, neumann):
    cf = S.coefficients()
    op = S.options(sub=sub, overlap=delta, subsolver=0, project=1, ras_variant="left-ras")
    O = oracle.Problem(dim, n, 0.25, cf, op, neumann=neumann)
    nf, ku = O.nf, O.ku
    c0, e0, u0 = S.random_fields(dim, n, 41, u_amp=0.01)
    c1 = c0 * (1 + 0.02 * np.cos(np.arange(c0.size)))
    X1, X0 = O.interleave(c1, e0, u0), O.interleave(c0, e0, u0)
    cb, dt = float(np.mean(c0)), 0.07
    Jsp = O.jacobian_scipy(X1, X0, cb, dt, 0)
    r = np.random.default_rng(6).standard_normal(Jsp.shape[0])
    z = np.zeros_like(r)
    for pts, own in _boxes(n, sub, delta, neumann):
        idx = (pts[:, None] * nf + np.arange(nf)[None, :]).reshape(-1)
        Ab = Jsp[idx][:, idx]
        pattern = np.zeros(Ab.shape, bool)
        rows = np.repeat(np.arange(Ab.shape[0]), np.diff(Ab.indptr))
        pattern[rows, Ab.indices] = True
        LU = _ilu0(Ab.toarray(), pattern)
        y = sla.solve_triangular(LU, r[idx], lower=True, unit_diagonal=True)
        x = sla.solve_triangular(LU, y, lower=False)
        own_u = np.repeat(own, nf)
        z[idx[own_u]] = x[own_u]
    want = _project(z, n, nf, ku, neumann)
    rc, got = O.precond_apply(X1, X0, cb, dt, r)
    assert rc == 0
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


@pytest.mark.parametrize("neumann", [False, True])
def test_projection_output_is_orthogonal_to_the_null_modes(neumann):
    """P z has zero c-mean and no component along any displacement null mode"""
    dim, n = 3, (6, 6, 4)
    cf = S.coefficients()
    O = oracle.Problem(dim, n, 0.25, cf, S.options(sub=(2, 2, 2), overlap=1), neumann=neumann)
    c0, e0, u0 = S.random_fields(dim, n, 43, u_amp=0.01)
    X = O.interleave(c0, e0, u0)
    r = np.random.default_rng(8).standard_normal(X.size)
    rc, z = O.precond_apply(X, X, float(np.mean(c0)), 0.05, r)
    assert rc == 0
    N = int(np.prod(n))
    Z = z.reshape(N, O.nf)
    assert abs(Z[:, 0].sum()) <= 1e-12 * np.abs(Z[:, 0]).sum()
    U = Z[:, O.ku:].T
    for m in _null_modes(n, neumann):
        assert abs(np.sum(m * U)) <= 1e-12 * np.linalg.norm(m) * np.linalg.norm(U)
