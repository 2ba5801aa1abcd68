"""GB300 Newton-Krylov-Schwarz solver for the DVD scheme of arXiv 2209.08001.

Thin ctypes binding over ``libnks.so`` (the C ABI of ``include/nks.h``): every
function here only marshals arguments; all arithmetic of the time step runs in
the library's CUDA kernels.  There is no CPU fallback: importing works without
a GPU (so the build can be checked), but any call raises if the library or a
CUDA device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnks.so")

NKS_OK, NKS_EINVAL, NKS_EDOMAIN, NKS_ENOMEM, NKS_EDIVERGED, NKS_ETIMEOUT, NKS_ECUDA, NKS_EPIVOT = range(8)
NKS_FP64, NKS_MIXED = 0, 1
# Schwarz preconditioner types (Sec. 4, Table 2)
RAS_VARIANTS = {"left-ras": 0, "as": 1, "right-ras": 2}
DT_MODES = {"fixed": 0, "solution": 1, "energy": 2}
KERNEL_CLASSES = ["residual", "jacobian_action", "schwarz_apply", "assembly_ilu0", "gs_dots", "gs_update",
                  "projection", "energy_mass", "vector_ops", "hessenberg", "true_residual_jv"]


class NksError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("nks error %d: %s" % (code, msg))
        self.code = code


class nks_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double), ("bc", ctypes.c_int)]


NKS_PERIODIC, NKS_NEUMANN = 0, 1


class nks_coeffs(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("gamma_c", ctypes.c_double), ("gamma_eta", ctypes.c_double),
                ("theta", ctypes.c_double), ("w_psi", ctypes.c_double), ("dE0", ctypes.c_double),
                ("L", ctypes.c_double * 4), ("U1", ctypes.c_double), ("U4", ctypes.c_double),
                ("eps0", ctypes.c_double), ("C11", ctypes.c_double), ("C12", ctypes.c_double),
                ("C44", ctypes.c_double), ("Lscale", ctypes.c_double), ("S", ctypes.c_int), ("n_eta", ctypes.c_int)]


class nks_opts(ctypes.Structure):
    _fields_ = [("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
                ("ls_alpha", ctypes.c_double), ("ls_lambda_min", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("gmres_rtol", ctypes.c_double), ("gmres_atol", ctypes.c_double),
                ("sub", ctypes.c_int * 3), ("overlap", ctypes.c_int), ("ilu_reuse", ctypes.c_int),
                ("precision", ctypes.c_int),
                ("dt_init", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("zeta", ctypes.c_double), ("dt_mode", ctypes.c_int), ("zeta_persist", ctypes.c_int),
                ("max_retries", ctypes.c_int), ("u0_rtol", ctypes.c_double), ("u0_atol", ctypes.c_double),
                ("u0_maxit", ctypes.c_int), ("timing", ctypes.c_int), ("graphs", ctypes.c_int),
                ("ras_variant", ctypes.c_int), ("u0_mixed", ctypes.c_int)]


class nks_server_opts(ctypes.Structure):
    _fields_ = [("opts", nks_opts), ("mem_budget", ctypes.c_size_t), ("max_slots", ctypes.c_int),
                ("max_groups", ctypes.c_int), ("box_side_2d", ctypes.c_int), ("box_side_3d", ctypes.c_int)]


class nks_request_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("steps", ctypes.c_int),
                ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int), ("retries", ctypes.c_int),
                ("points", ctypes.c_longlong), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t", ctypes.c_double), ("energy", ctypes.c_double),
                ("mass", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nks_server_state(ctypes.Structure):
    _fields_ = [("waiting", ctypes.c_int), ("groups", ctypes.c_int), ("in_flight", ctypes.c_int),
                ("bytes_reserved", ctypes.c_size_t), ("mem_budget", ctypes.c_size_t)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class nks_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class nks_step_info(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("t", ctypes.c_double), ("energy", ctypes.c_double),
                ("mass", ctypes.c_double), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double),
                ("retries", ctypes.c_int), ("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


NCLASS = 11


class nks_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong * NCLASS), ("ms", ctypes.c_double * NCLASS),
                ("newton_its", ctypes.c_longlong), ("gmres_its", ctypes.c_longlong),
                ("steps", ctypes.c_longlong), ("retries", ctypes.c_longlong),
                ("factor_bytes", ctypes.c_longlong), ("schwarz_points", ctypes.c_double),
                ("schwarz_bytes", ctypes.c_double), ("schwarz_flops", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("reorth", ctypes.c_longlong), ("cgs_bytes", ctypes.c_double)]

    def as_dict(self):
        return {"launches": {KERNEL_CLASSES[i]: self.launches[i] for i in range(NCLASS)},
                "ms": {KERNEL_CLASSES[i]: self.ms[i] for i in range(NCLASS)},
                "newton_its": self.newton_its, "gmres_its": self.gmres_its, "steps": self.steps,
                "retries": self.retries, "factor_bytes": self.factor_bytes,
                "schwarz_points": self.schwarz_points, "schwarz_bytes": self.schwarz_bytes,
                "schwarz_flops": self.schwarz_flops, "kernel_launches": self.kernel_launches,
                "reorth": self.reorth, "cgs_bytes": self.cgs_bytes}


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_P = ctypes.c_void_p


def load():
    """Load libnks.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libnks.so is missing: run `python -c 'import __graft_entry__ as g; g.build()'` "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "nks_default_opts": (None, [ctypes.POINTER(nks_opts)]),
        "nks_create_problem": (ctypes.c_int, [ctypes.POINTER(nks_grid), _D, _D, ctypes.POINTER(nks_coeffs),
                                              ctypes.POINTER(nks_opts), ctypes.POINTER(nks_allocator), _P, pp]),
        "nks_step": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(nks_step_info)]),
        "nks_energy": (ctypes.c_int, [_P, _D]),
        "nks_mass": (ctypes.c_int, [_P, _D]),
        "nks_get_fields": (ctypes.c_int, [_P, _D, _D, _D]),
        "nks_state_size": (ctypes.c_size_t, [_P]),
        "nks_get_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
        "nks_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
        "nks_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(nks_stats)]),
        "nks_reset_stats": (ctypes.c_int, [_P]),
        "nks_destroy": (None, [_P]),
        "nks_last_error": (ctypes.c_char_p, [_P]),
        "nks_eval_residual": (ctypes.c_int, [_P, _D, _D, ctypes.c_double, ctypes.c_int, _D]),
        "nks_apply_jacobian": (ctypes.c_int, [_P, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D]),
        "nks_apply_preconditioner": (ctypes.c_int, [_P, _D, _D, ctypes.c_double, _D, _D]),
        "nks_linear_solve": (ctypes.c_int, [_P, _D, _D, ctypes.c_double, ctypes.c_int, _D, _D, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int), _D]),
        "nks_eval_energy": (ctypes.c_int, [_P, _D, _D, _D]),
        "nks_residual_noalloc": (ctypes.c_int, [ctypes.POINTER(nks_grid), ctypes.POINTER(nks_coeffs),
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int, _P, _P, _P, _P, _P]),
        "nks_create_batch": (ctypes.c_int, [ctypes.POINTER(nks_grid), ctypes.c_int, _D, _D, ctypes.POINTER(nks_coeffs),
                                            ctypes.POINTER(nks_opts), ctypes.POINTER(nks_allocator), _P, pp]),
        "nks_batch_size": (ctypes.c_int, [_P]),
        "nks_batch_load": (ctypes.c_int, [_P, ctypes.c_int, _D, _D]),
        "nks_batch_unload": (ctypes.c_int, [_P, ctypes.c_int]),
        "nks_batch_loaded": (ctypes.c_int, [_P, ctypes.c_int]),
        "nks_batch_step": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _D, ctypes.POINTER(nks_step_info)]),
        "nks_batch_energy": (ctypes.c_int, [_P, ctypes.c_int, _D]),
        "nks_batch_mass": (ctypes.c_int, [_P, ctypes.c_int, _D]),
        "nks_batch_get_fields": (ctypes.c_int, [_P, ctypes.c_int, _D, _D, _D]),
        "nks_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
        "nks_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
        "nks_device_bytes": (ctypes.c_size_t, [_P]),
        "nks_debug_withhold_copy": (ctypes.c_int, [_P, ctypes.c_int]),
        "nks_model3_point": (ctypes.c_int, [ctypes.POINTER(nks_coeffs), _D, _D, _D, _D]),
        "nks_server_default_opts": (None, [ctypes.POINTER(nks_server_opts)]),
        "nks_server_create": (ctypes.c_int, [ctypes.POINTER(nks_coeffs), ctypes.POINTER(nks_server_opts), pp]),
        "nks_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(nks_grid), _D, _D, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_longlong)]),
        "nks_server_wait": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.POINTER(nks_request_result), _D, _D, _D,
                                           ctypes.c_double]),
        "nks_server_status": (ctypes.c_int, [_P, ctypes.POINTER(nks_server_state)]),
        "nks_server_destroy": (None, [_P]),
        "nks_autotune": (ctypes.c_int, [ctypes.POINTER(nks_grid), _D, _D, ctypes.POINTER(nks_coeffs),
                                        ctypes.POINTER(nks_opts), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(nks_opts), _D, ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names the binding expects libnks.so to export (all of include/nks.h)."""
    return ["nks_default_opts", "nks_create_problem", "nks_step", "nks_energy", "nks_mass", "nks_get_fields",
            "nks_state_size", "nks_get_state", "nks_set_state", "nks_get_stats", "nks_reset_stats", "nks_destroy",
            "nks_last_error", "nks_eval_residual", "nks_apply_jacobian", "nks_apply_preconditioner",
            "nks_linear_solve", "nks_eval_energy", "nks_residual_noalloc", "nks_create_batch", "nks_batch_size",
            "nks_batch_load", "nks_batch_unload", "nks_batch_loaded", "nks_batch_step", "nks_batch_energy",
            "nks_batch_mass", "nks_batch_get_fields", "nks_batch_get_state", "nks_batch_set_state",
            "nks_device_bytes", "nks_debug_withhold_copy", "nks_model3_point", "nks_autotune",
            "nks_server_default_opts", "nks_server_create", "nks_server_submit", "nks_server_wait",
            "nks_server_status", "nks_server_destroy"]


def _ptr(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_grid(dim, n, h, neumann=False):
    g = nks_grid()
    g.dim = dim
    nn = list(n) + [1] * (3 - len(n))
    for J in range(3):
        g.n[J] = int(nn[J]) if J < dim else 1
    g.h = float(h)
    g.bc = NKS_NEUMANN if neumann else NKS_PERIODIC
    return g


def make_coeffs(cf: dict):
    k = nks_coeffs()
    for name in ("kappa", "gamma_c", "gamma_eta", "theta", "w_psi", "dE0", "U1", "U4", "eps0", "C11", "C12", "C44"):
        setattr(k, name, float(cf[name]))
    for i in range(4):
        k.L[i] = float(cf["L"][i])
    k.Lscale = float(cf.get("Lscale", 1.0))
    k.S = int(cf["S"])
    k.n_eta = int(cf.get("n_eta", 1))
    return k


def _layout(dim, coeffs: dict):
    """(order parameters, fields per point) of a model: c, eta_1..eta_ne and, with
    elasticity, u_1..u_d."""
    ne = 3 if int(coeffs.get("n_eta", 1)) == 3 else 1
    elastic = any(coeffs[k] != 0.0 for k in ("C11", "C12", "C44")) and coeffs.get("Lscale", 1.0) != 0.0
    return ne, 1 + ne + (dim if elastic else 0)


def _eta_out(ne, N):
    """host array for n_eta order-parameter fields: (N,) for one, (3, N) for three"""
    return np.empty(N) if ne == 1 else np.empty((ne, N))


def make_opts(op: dict, timing=False):
    o = nks_opts()
    load().nks_default_opts(ctypes.byref(o))
    for name in ("newton_rtol", "newton_atol", "ls_alpha", "ls_lambda_min", "gmres_rtol", "gmres_atol", "dt_init",
                 "dt_min", "dt_max", "zeta", "u0_rtol", "u0_atol"):
        if name in op:
            setattr(o, name, float(op[name]))
    for name in ("newton_maxit", "gmres_restart", "gmres_maxit", "overlap", "ilu_reuse", "zeta_persist",
                 "max_retries", "u0_maxit", "graphs", "u0_mixed"):
        if name in op:
            setattr(o, name, int(op[name]))
    if "sub" in op:
        sub = list(op["sub"]) + [1] * (3 - len(op["sub"]))
        for J in range(3):
            o.sub[J] = int(sub[J])
    if "dt_mode" in op:
        o.dt_mode = DT_MODES[op["dt_mode"]] if isinstance(op["dt_mode"], str) else int(op["dt_mode"])
    if "precision" in op:
        o.precision = {"fp64": NKS_FP64, "mixed": NKS_MIXED}.get(op["precision"], op["precision"])
    if "ras_variant" in op:
        o.ras_variant = RAS_VARIANTS.get(op["ras_variant"], op["ras_variant"])
    o.timing = 1 if timing else 0
    return o


def last_error(p=None):
    m = load().nks_last_error(p)
    return m.decode() if m else ""


def _check(rc, p=None):
    if rc != NKS_OK:
        raise NksError(rc, last_error(p))
    return rc


class Problem:
    """One simulation resident on the current CUDA device (``nks_problem``)."""

    def __init__(self, dim, n, h, c, eta, coeffs: dict, opts: dict, stream=None, allocator=None, timing=False,
                 neumann=False):
        """neumann: homogeneous Neumann boundaries (mirror ghost cells, traction-free
        displacement rows) instead of periodic ones."""
        L = load()
        self.dim, self.n = dim, tuple(n[:dim])
        self.N = int(np.prod(self.n))
        self._grid = make_grid(dim, n, h, neumann)
        self._coeffs = make_coeffs(coeffs)
        self._opts = make_opts(opts, timing)
        self.ne, self.nf = _layout(dim, coeffs)
        self.ku = 1 + self.ne  # first displacement field
        c, eta = _c64(c), _c64(eta)
        assert c.size == self.N and eta.size == self.ne * self.N
        self._alloc = allocator
        handle = ctypes.c_void_p()
        rc = L.nks_create_problem(ctypes.byref(self._grid), _ptr(c), _ptr(eta), ctypes.byref(self._coeffs),
                                  ctypes.byref(self._opts), ctypes.byref(allocator) if allocator else None,
                                  ctypes.c_void_p(stream) if stream else None, ctypes.byref(handle))
        _check(rc, None)
        self._h = handle

    def __del__(self):
        self.destroy()

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().nks_destroy(h)
            self._h = None

    # -- the time step
    def step(self, dt=0.0):
        info = nks_step_info()
        rc = load().nks_step(self._h, float(dt), ctypes.byref(info))
        _check(rc, self._h)
        return info.as_dict()

    def energy(self):
        v = ctypes.c_double()
        _check(load().nks_energy(self._h, ctypes.byref(v)), self._h)
        return v.value

    def mass(self):
        v = ctypes.c_double()
        _check(load().nks_mass(self._h, ctypes.byref(v)), self._h)
        return v.value

    def get_fields(self):
        """(c, eta, u): eta is (N,) with one order parameter, (3, N) with three;
        u is (d, N) or None without elasticity."""
        c, eta = np.empty(self.N), _eta_out(self.ne, self.N)
        u = np.empty((self.nf - self.ku, self.N)) if self.nf > self.ku else None
        _check(load().nks_get_fields(self._h, _ptr(c), _ptr(eta), _ptr(u) if u is not None else None), self._h)
        return c, eta, u

    def get_state(self) -> bytes:
        L = load()
        n = L.nks_state_size(self._h)
        buf = ctypes.create_string_buffer(n)
        _check(L.nks_get_state(self._h, buf, n), self._h)
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().nks_set_state(self._h, buf, len(blob)), self._h)

    def get_stats(self):
        s = nks_stats()
        _check(load().nks_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def reset_stats(self):
        _check(load().nks_reset_stats(self._h), self._h)

    def device_bytes(self):
        return int(load().nks_device_bytes(self._h))

    # -- operator-level entry points (state arrays: fields one after another)
    def eval_residual(self, X1, X0, dt, mode=0):
        X1, X0 = _c64(X1), _c64(X0)
        F = np.empty(self.nf * self.N)
        _check(load().nks_eval_residual(self._h, _ptr(X1), _ptr(X0), float(dt), int(mode), _ptr(F)), self._h)
        return F

    def apply_jacobian(self, X1, X0, dt, v, mode=0):
        X1, X0, v = _c64(X1), _c64(X0), _c64(v)
        out = np.empty(self.nf * self.N)
        _check(load().nks_apply_jacobian(self._h, _ptr(X1), _ptr(X0), float(dt), int(mode), _ptr(v), _ptr(out)),
               self._h)
        return out

    def apply_preconditioner(self, X1, X0, dt, r):
        X1, X0, r = _c64(X1), _c64(X0), _c64(r)
        z = np.empty(self.nf * self.N)
        _check(load().nks_apply_preconditioner(self._h, _ptr(X1), _ptr(X0), float(dt), _ptr(r), _ptr(z)), self._h)
        return z

    def linear_solve(self, X1, X0, dt, b, tol, mode=0):
        X1, X0, b = _c64(X1), _c64(X0), _c64(b)
        x = np.empty(self.nf * self.N)
        its, res = ctypes.c_int(), ctypes.c_double()
        _check(load().nks_linear_solve(self._h, _ptr(X1), _ptr(X0), float(dt), int(mode), _ptr(b), _ptr(x),
                                       float(tol), ctypes.byref(its), ctypes.byref(res)), self._h)
        return x, its.value, res.value

    def debug_withhold_copy(self, on=True):
        """Testing hook: the Schwarz sweeps withhold a factor copy (their bounded
        waits expire; the next solve fails with NKS_ETIMEOUT)."""
        _check(load().nks_debug_withhold_copy(self._h, 1 if on else 0), self._h)

    def eval_energy(self, X):
        X = _c64(X)
        parts, mass = np.empty(5), ctypes.c_double()
        _check(load().nks_eval_energy(self._h, _ptr(X), _ptr(parts), ctypes.byref(mass)), self._h)
        return parts, mass.value


class Batch:
    """nb same-shape problems stepped together (``nks_create_batch``): one kernel
    launch per solver phase for all slots; each slot keeps its own Newton/GMRES
    iteration and step size.  c, eta: (nb, N) arrays, or None for empty slots."""

    def __init__(self, dim, n, h, nb, coeffs: dict, opts: dict, c=None, eta=None, stream=None, allocator=None,
                 timing=False, neumann=False):
        L = load()
        self.dim, self.n, self.nb = dim, tuple(n[:dim]), int(nb)
        self.N = int(np.prod(self.n))
        self._grid = make_grid(dim, n, h, neumann)
        self._coeffs = make_coeffs(coeffs)
        self._opts = make_opts(opts, timing)
        self.ne, self.nf = _layout(dim, coeffs)
        self.ku = 1 + self.ne
        cp = ep = None
        if c is not None:
            c, eta = _c64(c).reshape(-1), _c64(eta).reshape(-1)
            assert c.size == self.N * self.nb and eta.size == self.ne * self.N * self.nb
            cp, ep = _ptr(c), _ptr(eta)
        self._alloc = allocator
        handle = ctypes.c_void_p()
        rc = L.nks_create_batch(ctypes.byref(self._grid), self.nb, cp, ep, ctypes.byref(self._coeffs),
                                ctypes.byref(self._opts), ctypes.byref(allocator) if allocator else None,
                                ctypes.c_void_p(stream) if stream else None, ctypes.byref(handle))
        _check(rc, None)
        self._h = handle

    def __del__(self):
        self.destroy()

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().nks_destroy(h)
            self._h = None

    def load(self, slot, c, eta):
        c, eta = _c64(c), _c64(eta)
        assert c.size == self.N and eta.size == self.ne * self.N
        _check(load().nks_batch_load(self._h, int(slot), _ptr(c), _ptr(eta)), self._h)

    def unload(self, slot):
        _check(load().nks_batch_unload(self._h, int(slot)), self._h)

    def loaded(self, slot):
        return bool(load().nks_batch_loaded(self._h, int(slot)))

    def step(self, active=None, dt=None):
        """One step of the active loaded slots; returns one info dict per slot
        (None for slots not stepped)."""
        act = None
        if active is not None:
            a = (ctypes.c_int * self.nb)(*[1 if x else 0 for x in active])
            act = ctypes.cast(a, ctypes.POINTER(ctypes.c_int))
        dtp = None
        if dt is not None:
            d = np.full(self.nb, float(dt)) if np.isscalar(dt) else _c64(dt)
            dtp = _ptr(d)
        infos = (nks_step_info * self.nb)()
        stepped = [load().nks_batch_loaded(self._h, i) and (active is None or bool(active[i]))
                   for i in range(self.nb)]
        _check(load().nks_batch_step(self._h, act, dtp, infos), self._h)
        return [infos[i].as_dict() if stepped[i] else None for i in range(self.nb)]

    def energy(self, slot):
        v = ctypes.c_double()
        _check(load().nks_batch_energy(self._h, int(slot), ctypes.byref(v)), self._h)
        return v.value

    def mass(self, slot):
        v = ctypes.c_double()
        _check(load().nks_batch_mass(self._h, int(slot), ctypes.byref(v)), self._h)
        return v.value

    def get_fields(self, slot):
        c, eta = np.empty(self.N), _eta_out(self.ne, self.N)
        u = np.empty((self.nf - self.ku, self.N)) if self.nf > self.ku else None
        _check(load().nks_batch_get_fields(self._h, int(slot), _ptr(c), _ptr(eta),
                                           _ptr(u) if u is not None else None), self._h)
        return c, eta, u

    def get_state(self, slot) -> bytes:
        L = load()
        n = L.nks_state_size(self._h)
        buf = ctypes.create_string_buffer(n)
        _check(L.nks_batch_get_state(self._h, int(slot), buf, n), self._h)
        return buf.raw

    def set_state(self, slot, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(load().nks_batch_set_state(self._h, int(slot), buf, len(blob)), self._h)

    def get_stats(self):
        s = nks_stats()
        _check(load().nks_get_stats(self._h, ctypes.byref(s)), self._h)
        return s.as_dict()

    def reset_stats(self):
        _check(load().nks_reset_stats(self._h), self._h)

    def device_bytes(self):
        return int(load().nks_device_bytes(self._h))


def model3_point(coeffs: dict, x1, x0):
    """Pointwise DVD derivative of the model with three order parameters and its
    derivative block (nks_model3_point): x1, x0 = (c, eta_1, eta_2, eta_3) at
    levels n+1 and n; returns (G[4], dG[4, 4]) with dG[a, b] = dG_a/dx1_b."""
    k = make_coeffs(dict(coeffs, n_eta=3))
    x1, x0 = _c64(x1).reshape(4), _c64(x0).reshape(4)
    G, dG = np.empty(4), np.empty(16)
    rc = load().nks_model3_point(ctypes.byref(k), _ptr(x1), _ptr(x0), _ptr(G), _ptr(dG))
    if rc != NKS_OK:
        raise NksError(rc, "nks_model3_point: invalid arguments")
    return G, dG.reshape(4, 4)


def autotune(dim, n, h, c, eta, coeffs: dict, opts: dict, candidates=None, dt_trial=0.01, neumann=False):
    """Pick the Schwarz decomposition (sub, overlap) with the shortest time step
    (nks_autotune).  candidates: list of (sub tuple, overlap) or None for the
    built-in list.  Returns (opts dict with the choice, [(sub, overlap, seconds)])."""
    L = load()
    g, k, o = make_grid(dim, n, h, neumann), make_coeffs(coeffs), make_opts(opts)
    c, eta = _c64(c), _c64(eta)
    if candidates is not None:
        flat = []
        for sub, ov in candidates:
            sub = list(sub) + [1] * (3 - len(sub))
            flat += [int(sub[0]), int(sub[1]), int(sub[2]), int(ov)]
        arr = (ctypes.c_int * len(flat))(*flat)
        cp, nc = ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)), len(candidates)
    else:
        cp, nc = None, 0
    best = nks_opts()
    times = np.full(max(nc, 64), -1.0)
    chosen = ctypes.c_int(-1)
    _check(L.nks_autotune(ctypes.byref(g), _ptr(c), _ptr(eta), ctypes.byref(k), ctypes.byref(o), cp, nc,
                          float(dt_trial), ctypes.byref(best), _ptr(times), ctypes.byref(chosen)), None)
    out = dict(opts)
    out["sub"] = tuple(best.sub[J] for J in range(dim))
    out["overlap"] = best.overlap
    if candidates is not None:
        table = [(tuple(sub), ov, float(times[i])) for i, (sub, ov) in enumerate(candidates)]
    else:
        table = [(None, None, float(t)) for t in times if t != -1.0]
    return out, table, chosen.value


class Server:
    """Request loop for many simulations on the current device (nks_server_*):
    same-shape requests share a batch, admitted into free slots between batch
    steps; shape groups run on their own streams and worker threads."""

    def __init__(self, coeffs: dict, opts: dict = None, mem_budget=0, max_slots=16, max_groups=8, box_side_2d=32,
                 box_side_3d=16):
        L = load()
        so = nks_server_opts()
        L.nks_server_default_opts(ctypes.byref(so))
        if opts:
            so.opts = make_opts(dict(opts))
        so.mem_budget = int(mem_budget)
        so.max_slots, so.max_groups = int(max_slots), int(max_groups)
        so.box_side_2d, so.box_side_3d = int(box_side_2d), int(box_side_3d)
        self._coeffs = make_coeffs(coeffs)
        self.ne = 3 if self._coeffs.n_eta == 3 else 1
        h = ctypes.c_void_p()
        _check(L.nks_server_create(ctypes.byref(self._coeffs), ctypes.byref(so), ctypes.byref(h)), None)
        self._h = h
        self._shape = {}

    def submit(self, dim, n, h, c, eta, steps, neumann=False):
        g = make_grid(dim, n, h, neumann)
        c, eta = _c64(c), _c64(eta)
        assert eta.size == self.ne * c.size
        rid = ctypes.c_longlong()
        _check(load().nks_server_submit(self._h, ctypes.byref(g), _ptr(c), _ptr(eta), int(steps), ctypes.byref(rid)),
               None)
        self._shape[rid.value] = (dim, int(np.prod(n[:dim])))
        return rid.value

    def wait(self, rid, timeout=-1.0):
        """(result dict, (c, eta, u)) of a finished request."""
        dim, N = self._shape.pop(rid)
        c, eta, u = np.empty(N), _eta_out(self.ne, N), np.empty((dim, N))
        r = nks_request_result()
        _check(load().nks_server_wait(self._h, int(rid), ctypes.byref(r), _ptr(c), _ptr(eta), _ptr(u),
                                      float(timeout)), None)
        return r.as_dict(), (c, eta, u)

    def status(self):
        st = nks_server_state()
        _check(load().nks_server_status(self._h, ctypes.byref(st)), None)
        return {k: getattr(st, k) for k, _ in st._fields_}

    def destroy(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().nks_server_destroy(h)
            self._h = None

    def __del__(self):
        self.destroy()


NOALLOC_MAX_POINTS = 65536


def residual_noalloc(dim, n, h, coeffs: dict, cbar0, dt, X1_ptr, X0_ptr, F_ptr, fnorm2_ptr=None, stream=None,
                     mode=0, neumann=False):
    """F(X1; X0, dt) on caller-owned device arrays (raw pointers) without any
    device allocation (nks_residual_noalloc).  Returns the status code."""
    g, k = make_grid(dim, n, h, neumann), make_coeffs(coeffs)
    return load().nks_residual_noalloc(ctypes.byref(g), ctypes.byref(k), float(cbar0), float(dt), int(mode),
                                       X1_ptr, X0_ptr, F_ptr, fnorm2_ptr, stream)


def torch_allocator():
    """An nks_allocator backed by PyTorch's caching allocator on the current device."""
    import torch

    def _alloc(nbytes, ctx):
        return torch.cuda.caching_allocator_alloc(int(nbytes))

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    a = nks_allocator()
    a.alloc = ALLOC_FN(_alloc)
    a.free = FREE_FN(_free)
    a.ctx = None
    a._keep = (a.alloc, a.free)
    return a
