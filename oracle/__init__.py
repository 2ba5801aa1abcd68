"""FP64 CPU oracle for the per-time-step Newton-Krylov-Schwarz solve of the
DVD scheme NSOA-1 of arXiv 2209.08001 (Huang & Yang, "Parallel energy stable
phase field simulations of Ni-based alloys system").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA path (``paper_2209_08001_gb300``);
neither imports the other.  The arithmetic lives in ``nks_oracle.c`` (plain
serial C, compiled with ``-ffp-contract=off``); this module only builds it,
marshals arrays and converts between the product's field-by-field layout and
the paper's point-interleaved unknown vector (Sec. 4).  Loops over independent
points, rows, subdomains and vector entries run on all host threads (OpenMP,
``OMP_NUM_THREADS`` to limit them); every sum is taken in a fixed block order,
so results do not depend on the thread count.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  energy / mass / G^1 / G^2 / G^4 .... pinned (App. A construction, DVD identity,
                                        summation by parts, closed forms)
  Psi_S ............................... pinned (exact quotient + tail bound)
  G^3 / elastic residual .............. pinned (DVD identity at equilibrium,
                                        Fourier symbol of the equilibrium)
  Jacobian ............................ pinned (central finite differences)
  ILU(0) / RAS / GMRES ................ pinned (ILU(0) defining property,
                                        dense LU, 1-subdomain exact solve)
  Newton / time stepping .............. pinned (steady states, linear growth
                                        rate, mass, energy law, symmetries)
  physical coefficient values ......... parity unpinned (the CALPHAD and
                                        elastic constants are not printed)
  Neumann boundaries .................. pinned (mirrored periodic problem without
                                        elasticity; -F_u = dE_3/du; mass, energy
                                        law, central differences; projection vs
                                        the SVD null space of the displacement
                                        block)
  three order parameters (n_eta = 3) .. pinned (reduction to the pinned reduced
                                        model, four-sublattice symmetry of E_G,
                                        exact discrete chain rule, central
                                        differences, mass, energy law,
                                        permutations)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nks_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ORC_OK, ORC_EINVAL, ORC_EDOMAIN, ORC_EDIVERGED, ORC_EPIVOT = 0, 1, 2, 4, 7


def build(force: bool = False) -> str:
    """Compile nks_oracle.c into liboracle.so (plain gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("neumann", ctypes.c_int)]


class _Coeffs(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("gamma_c", ctypes.c_double), ("gamma_eta", ctypes.c_double),
                ("theta", ctypes.c_double), ("w_psi", ctypes.c_double), ("dE0", ctypes.c_double),
                ("L", ctypes.c_double * 4), ("U1", ctypes.c_double), ("U4", ctypes.c_double),
                ("eps0", ctypes.c_double), ("C11", ctypes.c_double), ("C12", ctypes.c_double),
                ("C44", ctypes.c_double), ("S", ctypes.c_int), ("n_eta", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int),
                ("ls_alpha", ctypes.c_double), ("ls_lambda_min", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("gmres_rtol", ctypes.c_double), ("gmres_atol", ctypes.c_double),
                ("sub", ctypes.c_int * 3), ("overlap", ctypes.c_int), ("subsolver", ctypes.c_int),
                ("reuse", ctypes.c_int), ("project", ctypes.c_int),
                ("dt_init", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("zeta", ctypes.c_double), ("dt_mode", ctypes.c_int), ("zeta_persist", ctypes.c_int),
                ("max_retries", ctypes.c_int),
                ("u0_rtol", ctypes.c_double), ("u0_atol", ctypes.c_double), ("u0_maxit", ctypes.c_int),
                ("variant", ctypes.c_int)]


class StepInfo(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("t", ctypes.c_double), ("energy", ctypes.c_double),
                ("mass", ctypes.c_double), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double),
                ("retries", ctypes.c_int), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)
_P = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        g, k, o = ctypes.POINTER(_Grid), ctypes.POINTER(_Coeffs), ctypes.POINTER(_Opts)
        si = ctypes.POINTER(StepInfo)
        sig = {
            "orc_nfields": (ctypes.c_int, [g, k]),
            "orc_num_threads": (ctypes.c_int, []),
            "orc_set_threads": (None, [ctypes.c_int]),
            "orc_energy": (ctypes.c_double, [g, k, ctypes.c_double, _D, _D]),
            "orc_mass": (ctypes.c_double, [g, k, _D]),
            "orc_psi_quot": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "orc_psi_quot_d1": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_int]),
            "orc_dvd_G": (None, [g, k, ctypes.c_double, _D, _D, ctypes.c_int, _D, _D]),
            "orc_residual": (None, [g, k, ctypes.c_double, ctypes.c_double, _D, _D, ctypes.c_int, _D]),
            "orc_jacobian_new": (_P, [g, k, ctypes.c_double, ctypes.c_double, _D, _D, ctypes.c_int]),
            "orc_csr_n": (ctypes.c_long, [_P]),
            "orc_csr_nnz": (ctypes.c_long, [_P]),
            "orc_csr_copy": (None, [_P, _L, _L, _D]),
            "orc_csr_free": (None, [_P]),
            "orc_ilu0": (ctypes.c_int, [ctypes.c_long, _L, _L, _D]),
            "orc_ilu0_solve": (None, [ctypes.c_long, _L, _L, _D, _D, _D]),
            "orc_equilibrate": (ctypes.c_int, [g, k, o, ctypes.c_double, _D, si]),
            "orc_newton_step": (ctypes.c_int, [g, k, o, ctypes.c_double, ctypes.c_double, _D, _D, si]),
            "orc_precond_apply": (ctypes.c_int, [g, k, o, ctypes.c_double, ctypes.c_double, _D, _D, _D, _D]),
            "orc_linear_solve": (ctypes.c_int, [g, k, o, ctypes.c_double, ctypes.c_double, _D, _D, ctypes.c_int,
                                                _D, _D, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _D]),
            "orc_dt_predict": (ctypes.c_double, [ctypes.c_double] * 4),
            "orc_simulate": (ctypes.c_int, [g, k, o, _D, ctypes.c_int, _D, si, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling
# --------------------------------------------------------------------------

def _ptr(a):
    return a.ctypes.data_as(_D)


def make_grid(dim, n, h, neumann=False):
    G = _Grid()
    G.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for J in range(3):
        G.n[J] = int(nn[J]) if J < dim else 1
    G.h = float(h)
    G.neumann = 1 if neumann else 0
    return G


def make_coeffs(cf: dict):
    """cf: the coefficient dict of ``synthetic.coefficients`` (C_ij before the
    Lscale factor).  The Hooke constants enter multiplied by Lscale (Sec. 5.1)."""
    K = _Coeffs()
    K.kappa, K.gamma_c, K.gamma_eta = cf["kappa"], cf["gamma_c"], cf["gamma_eta"]
    K.theta, K.w_psi, K.dE0 = cf["theta"], cf["w_psi"], cf["dE0"]
    for i in range(4):
        K.L[i] = cf["L"][i]
    K.U1, K.U4, K.eps0 = cf["U1"], cf["U4"], cf["eps0"]
    s = cf.get("Lscale", 1.0)
    K.C11, K.C12, K.C44 = cf["C11"] * s, cf["C12"] * s, cf["C44"] * s
    K.S = int(cf["S"])
    K.n_eta = int(cf.get("n_eta", 1))
    return K


def make_opts(op: dict):
    O = _Opts()
    O.newton_rtol, O.newton_atol, O.newton_maxit = op["newton_rtol"], op["newton_atol"], op["newton_maxit"]
    O.ls_alpha, O.ls_lambda_min = op["ls_alpha"], op["ls_lambda_min"]
    O.gmres_restart, O.gmres_maxit = op["gmres_restart"], op["gmres_maxit"]
    O.gmres_rtol, O.gmres_atol = op["gmres_rtol"], op["gmres_atol"]
    sub = list(op["sub"]) + [1] * (3 - len(op["sub"]))
    for J in range(3):
        O.sub[J] = int(sub[J])
    O.overlap, O.subsolver = op["overlap"], op.get("subsolver", 0)
    O.reuse, O.project = op["ilu_reuse"], op.get("project", 1)
    O.dt_init, O.dt_min, O.dt_max, O.zeta = op["dt_init"], op["dt_min"], op["dt_max"], op["zeta"]
    O.dt_mode = {"fixed": 0, "solution": 1, "energy": 2}[op["dt_mode"]]
    O.zeta_persist, O.max_retries = op["zeta_persist"], op["max_retries"]
    O.u0_rtol, O.u0_atol, O.u0_maxit = op["u0_rtol"], op["u0_atol"], op["u0_maxit"]
    O.variant = RAS_VARIANTS[op.get("ras_variant", "left-ras")]
    return O


# Schwarz preconditioner types of Sec. 4 / Table 2
RAS_VARIANTS = {"left-ras": 0, "as": 1, "right-ras": 2}


class Problem:
    """Grid + coefficients + options bundle; converts SoA fields <-> interleaved X."""

    def __init__(self, dim, n, h, coeffs: dict, opts: dict | None = None, neumann=False):
        """neumann: homogeneous Neumann boundaries (Eq. boundaryequ) instead of
        periodic ones: mirror ghost cells for c and eta, traction-free displacement
        rows as the exact variation of the discrete elastic energy."""
        self.dim, self.n, self.h = dim, tuple(n[:dim]), h
        self.G = make_grid(dim, n, h, neumann)
        self.K = make_coeffs(coeffs)
        self.opts = opts
        self.O = make_opts(opts) if opts is not None else None
        self.N = int(np.prod(self.n))
        self.nf = lib().orc_nfields(ctypes.byref(self.G), ctypes.byref(self.K))
        self.ne = 3 if self.K.n_eta == 3 else 1  # order parameters per point
        self.ku = 1 + self.ne                    # first displacement field

    # SoA (c, eta, u[d, N]) <-> point-interleaved X (Sec. 4); with three order
    # parameters eta is (3, N)
    def interleave(self, c, eta, u=None):
        X = np.zeros((self.N, self.nf))
        X[:, 0] = c
        X[:, 1:self.ku] = np.asarray(eta).reshape(self.ne, self.N).T
        if self.nf > self.ku and u is not None:
            X[:, self.ku:] = np.asarray(u).reshape(self.dim, self.N).T
        return np.ascontiguousarray(X.reshape(-1))

    def split(self, X):
        Y = np.asarray(X).reshape(self.N, self.nf)
        u = Y[:, self.ku:].T.copy() if self.nf > self.ku else None
        eta = Y[:, 1].copy() if self.ne == 1 else Y[:, 1:self.ku].T.copy()
        return Y[:, 0].copy(), eta, u

    def _g(self):
        return ctypes.byref(self.G), ctypes.byref(self.K)

    def energy(self, X, cbar0, parts=False):
        X = np.ascontiguousarray(X, dtype=np.float64)
        pr = np.zeros(4)
        e = lib().orc_energy(*self._g(), cbar0, _ptr(X), _ptr(pr))
        return (e, pr) if parts else e

    def mass(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64)
        return lib().orc_mass(*self._g(), _ptr(X))

    def dvd_G(self, X1, X0, cbar0, which=15):
        X1 = np.ascontiguousarray(X1, dtype=np.float64)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        gc, ge = np.zeros(self.N), np.zeros(self.N * self.ne)
        lib().orc_dvd_G(*self._g(), cbar0, _ptr(X1), _ptr(X0), which, _ptr(gc), _ptr(ge))
        return gc, (ge if self.ne == 1 else ge.reshape(3, self.N))

    def residual(self, X1, X0, cbar0, dt, mode=0):
        X1 = np.ascontiguousarray(X1, dtype=np.float64)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        F = np.zeros(self.N * self.nf)
        lib().orc_residual(*self._g(), cbar0, dt, _ptr(X1), _ptr(X0), mode, _ptr(F))
        return F

    def jacobian(self, X1, X0, cbar0, dt, mode=0):
        """Analytic dF/dX1 as (indptr, indices, data) of a CSR matrix."""
        X1 = np.ascontiguousarray(X1, dtype=np.float64)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        L = lib()
        h = L.orc_jacobian_new(*self._g(), cbar0, dt, _ptr(X1), _ptr(X0), mode)
        n, nnz = L.orc_csr_n(h), L.orc_csr_nnz(h)
        rp, ci, v = np.zeros(n + 1, np.int64), np.zeros(nnz, np.int64), np.zeros(nnz)
        L.orc_csr_copy(h, rp.ctypes.data_as(_L), ci.ctypes.data_as(_L), _ptr(v))
        L.orc_csr_free(h)
        return rp, ci, v

    def jacobian_scipy(self, X1, X0, cbar0, dt, mode=0):
        import scipy.sparse as sp
        rp, ci, v = self.jacobian(X1, X0, cbar0, dt, mode)
        n = len(rp) - 1
        return sp.csr_matrix((v, ci, rp), shape=(n, n))

    def equilibrate(self, X, cbar0):
        X = np.ascontiguousarray(X, dtype=np.float64).copy()
        info = StepInfo()
        rc = lib().orc_equilibrate(*self._g(), ctypes.byref(self.O), cbar0, _ptr(X), ctypes.byref(info))
        return rc, X, info.as_dict()

    def newton_step(self, X0, cbar0, dt):
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        X = np.zeros_like(X0)
        info = StepInfo()
        rc = lib().orc_newton_step(*self._g(), ctypes.byref(self.O), cbar0, dt, _ptr(X0), _ptr(X),
                                   ctypes.byref(info))
        return rc, X, info.as_dict()

    def precond_apply(self, X1, X0, cbar0, dt, r):
        X1 = np.ascontiguousarray(X1, dtype=np.float64)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.zeros_like(r)
        rc = lib().orc_precond_apply(*self._g(), ctypes.byref(self.O), cbar0, dt, _ptr(X1), _ptr(X0),
                                     _ptr(r), _ptr(z))
        return rc, z

    def linear_solve(self, X1, X0, cbar0, dt, b, tol, mode=0):
        X1 = np.ascontiguousarray(X1, dtype=np.float64)
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        its, res = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = lib().orc_linear_solve(*self._g(), ctypes.byref(self.O), cbar0, dt, _ptr(X1), _ptr(X0), mode,
                                    _ptr(b), _ptr(x), tol, ctypes.byref(its), ctypes.byref(res))
        return rc, x, its.value, res.value

    def simulate(self, c, eta, nsteps, dt_replay=None):
        """Runs nsteps NKS time steps from (c, eta, u = equilibrium).  Returns
        (rc, X_final, [step info dicts], energy at level 0)."""
        X = self.interleave(c, eta)
        infos = (StepInfo * max(nsteps, 1))()
        e0 = ctypes.c_double(0.0)
        rp = None
        if dt_replay is not None:
            rp = np.ascontiguousarray(dt_replay, dtype=np.float64)
        rc = lib().orc_simulate(*self._g(), ctypes.byref(self.O), _ptr(X), nsteps,
                                _ptr(rp) if rp is not None else None, infos, ctypes.byref(e0))
        return rc, X, [infos[i].as_dict() for i in range(nsteps)], e0.value


def num_threads() -> int:
    """Host threads the oracle's parallel loops use."""
    return int(lib().orc_num_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's later parallel loops (n <= 0: all processors)."""
    lib().orc_set_threads(int(n))


def psi_quot(y1, y2, S):
    return lib().orc_psi_quot(float(y1), float(y2), int(S))


def psi_quot_d1(y1, y2, S):
    return lib().orc_psi_quot_d1(float(y1), float(y2), int(S))


def dt_predict(dt_min, dt_max, zeta, Xd):
    return lib().orc_dt_predict(float(dt_min), float(dt_max), float(zeta), float(Xd))


def ilu0(rp, ci, v):
    """ILU(0) of a CSR matrix with sorted columns; returns (rc, factored values)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int64)
    w = np.ascontiguousarray(v, dtype=np.float64).copy()
    rc = lib().orc_ilu0(len(rp) - 1, rp.ctypes.data_as(_L), ci.ctypes.data_as(_L), _ptr(w))
    return rc, w
