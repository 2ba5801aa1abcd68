"""Seeded synthetic inputs for the NKS solve of the DVD scheme (arXiv 2209.08001).

This module is the only code shared by the oracle-side tests and the callers of
the CUDA path.  It holds no arithmetic of the method: only random draws
(SplitMix64), grid sizes, coefficient values, solver settings, the five
workload descriptions, and a seeded random projection (``sign_sketch``) and
point sample (``sample_points``) for comparing full-size fields.

Workload recipe (the paper's own workloads are synthetic initial states,
Sec. 5.1-5.3; no dataset is involved):
  * periodic grid, h = 0.25 (Sec. 5.1);
  * c = cbar + U(-0.005, 0.005), eta = 0.1 + U(-0.01, 0.01), one SplitMix64
    stream per seed, all c draws in x-fastest point order, then all eta draws.
    The order-parameter mean 0.1 is the paper's random initial state (Sec. 5.3);
    a zero-mean eta would put c*eta outside (0, 1) where Psi is undefined;
  * u is not drawn: it is the mechanical equilibrium of the initial c.

The single-particle workload (Sec. 5.1) is deterministic instead: a sphere of
gamma' (c = 0.238, eta = 0.01) of radius 7.5 at the centre of an 80^3 box of
gamma matrix (c = 0.1375, eta = 0.99), the Hooke tensor scaled by L = 1.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of SplitMix64 (Steele, Lea & Flood 2014):
    state_i = seed + (i+1) * 0x9E3779B97F4A7C15, then the two xor-shift-multiply
    rounds and a final xor-shift."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """u = (x >> 11) * 2^-53 in [0, 1)."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def sign_sketch(fields, k: int = 256, seed: int = 7) -> np.ndarray:
    """Seeded random projection for comparing large fields without storing them:
    row i of the k x N matrix S has entries (1 - 2 b_ij)/sqrt(k), b_ij the bits
    (least significant first) of SplitMix64 outputs with seed (seed << 20) + i.
    Returns S x for every array x in `fields` (shape (len(fields), k)).  For any
    vector v, |S v| estimates |v|: |S v|^2 / |v|^2 concentrates like chi^2_k / k
    (Johnson-Lindenstrauss), so |S a - S b| estimates the L2 distance |a - b|."""
    X = [np.ascontiguousarray(x, dtype=np.float64).ravel() for x in fields]
    N = X[0].size
    words = (N + 63) // 64
    out = np.zeros((len(X), k))
    for i in range(k):
        bits = np.unpackbits(splitmix64((seed << 20) + i, words).view(np.uint8), bitorder="little")[:N]
        sg = 1.0 - 2.0 * bits.astype(np.float64)
        for f, x in enumerate(X):
            out[f, i] = np.dot(sg, x)
    return out / math.sqrt(k)


def sample_points(N: int, count: int = 1024, seed: int = 11) -> np.ndarray:
    """`count` distinct seeded point indices in [0, N), sorted."""
    u = uniform01(seed, 4 * count + 64)
    idx = np.unique((u * N).astype(np.int64))
    return np.sort(idx[:count]) if idx.size >= count else idx


def initial_fields(dim: int, n, cbar: float, seed: int, c_amp: float = 0.005,
                   eta_mean: float = 0.1, eta_amp: float = 0.01):
    """(c, eta) as flat float64 arrays in x-fastest order."""
    N = int(np.prod(n[:dim]))
    u = uniform01(seed, 2 * N)
    c = cbar + c_amp * (2.0 * u[:N] - 1.0)
    eta = eta_mean + eta_amp * (2.0 * u[N:] - 1.0)
    return c, eta


def initial_fields3(dim: int, n, cbar: float, seed: int, c_amp: float = 0.005, eta_mean: float = 0.1,
                    eta_amp: float = 0.01):
    """(c, eta[3, N]) for the model with three order parameters (App. A): the
    reduced model's recipe with each eta_j drawn independently (all c draws,
    then eta_1, eta_2, eta_3, in x-fastest order)."""
    N = int(np.prod(n[:dim]))
    u = uniform01(seed, 4 * N)
    c = cbar + c_amp * (2.0 * u[:N] - 1.0)
    eta = eta_mean + eta_amp * (2.0 * u[N:].reshape(3, N) - 1.0)
    return c, eta


def sphere_fields(dim: int, n, h: float, radius: float, inside=(0.238, 0.01), outside=(0.1375, 0.99)):
    """(c, eta) of one spherical particle (Sec. 5.1) as flat float64 arrays in
    x-fastest order: grid point i of an axis sits at x_i = i h, the centre at
    (n // 2) h on every axis; points with |x - centre| < radius take `inside`,
    the rest `outside`."""
    axes = [(np.arange(n[J]) - n[J] // 2) * h for J in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first: ravel is x-fastest
    r2 = sum(g * g for g in grids).ravel()
    isin = r2 < radius * radius
    c = np.where(isin, inside[0], outside[0]).astype(np.float64)
    eta = np.where(isin, inside[1], outside[1]).astype(np.float64)
    return c, eta


def random_fields(dim: int, n, seed: int, c_range=(0.10, 0.24), eta_range=(0.05, 0.95), u_amp=0.0):
    """Independent random (c, eta, u) for operator-level tests; c*eta and
    c*(4 - 3 eta) stay inside (0, 1)."""
    N = int(np.prod(n[:dim]))
    u = uniform01(seed, (2 + dim) * N)
    c = c_range[0] + (c_range[1] - c_range[0]) * u[:N]
    eta = eta_range[0] + (eta_range[1] - eta_range[0]) * u[N:2 * N]
    disp = u_amp * (2.0 * u[2 * N:].reshape(dim, N) - 1.0)
    return c, eta, disp


# ---------------------------------------------------------------------------
# coefficients (dimensionless; App. A scaling by V_m dE and L = 1.5 nm)
# ---------------------------------------------------------------------------

# theta = R T / (V_m dE), T = 1037 K, V_m dE = 1.48e-5 * 3.3e7 J/mol
THETA_1037K = 8.314462618 * 1037.0 / (1.48e-5 * 3.3e7)
# gamma~ = gamma / (dE * L^2): 2.5e-9 / (3.3e7 * 1.5e-9^2) and 6.0e-12 / (...)
GAMMA_C = 2.5e-9 / (3.3e7 * (1.5e-9) ** 2)
GAMMA_ETA = 6.0e-12 / (3.3e7 * (1.5e-9) ** 2)

COEFFS = dict(
    kappa=0.008,            # App. A
    gamma_c=GAMMA_C,        # 33.67
    gamma_eta=GAMMA_ETA,    # 0.0808
    theta=THETA_1037K,      # 17.654
    w_psi=1.0,              # theta*Psi(c) kept in E_2 as in the main text
    dE0=0.0,                # (E0_Al - E0_Ni)/(V_m dE): drops out of the dynamics
    # written by `python -m oracle.fit_coefficients` (wells of App. A at 1037 K)
    L=[-173.2736992, 0.0, 0.0, 0.0],
    U1=-19.77084797,
    U4=3.857829558,
    eps0=0.049,             # App. A
    # builder-chosen cubic Hooke constants / dE (not printed in the paper)
    C11=6000.0, C12=4000.0, C44=3000.0,
    Lscale=1.0,             # multiplier of the Hooke tensor (Sec. 5.1)
    S=10,                   # Taylor order of Psi_S (Sec. 5)
)


def coefficients(**over) -> dict:
    cf = dict(COEFFS)
    cf["L"] = list(COEFFS["L"])
    cf.update(over)
    return cf


# ---------------------------------------------------------------------------
# solver settings
# ---------------------------------------------------------------------------

OPTS = dict(
    newton_rtol=1e-10, newton_atol=1e-12, newton_maxit=20,
    ls_alpha=1e-4, ls_lambda_min=2.0 ** -10,
    gmres_restart=30, gmres_maxit=300, gmres_rtol=1e-6, gmres_atol=1e-14,
    sub=(4, 4, 1), overlap=1, subsolver=0, ilu_reuse=1, project=1,
    dt_init=0.01, dt_min=0.01, dt_max=2.0, zeta=100.0, dt_mode="fixed",
    zeta_persist=0, max_retries=8,
    u0_rtol=1e-12, u0_atol=1e-13, u0_maxit=10,
    # the initial mechanical equilibrium's inner GMRES in the mixed form (its Newton
    # residual and tolerance stay FP64); the time steps keep `precision`
    u0_mixed=1,
    precision="fp64",
)


def options(**over) -> dict:
    op = dict(OPTS)
    op.update(over)
    return op


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

CONFIGS = {
    "2d64": dict(
        desc="2D 64x64 periodic FP64, 10 fixed-dt DVD steps (dt=0.01), Newton tol 1e-10, "
             "GMRES(30), RAS 4x4 subdomains overlap 1, ILU(0)",
        dim=2, n=(64, 64), h=0.25, cbar=0.16, seed=0, steps=10,
        opts=dict(dt_mode="fixed", sub=(4, 4), overlap=1, precision="fp64")),
    "2d1024": dict(
        desc="2D 1024x1024 periodic FP64, 200 adaptive DVD steps (energy-change dt driver), "
             "GMRES(30), RAS 16x16 subdomains overlap 2, ILU(0)-reuse",
        dim=2, n=(1024, 1024), h=0.25, cbar=0.20, seed=1, steps=200,
        opts=dict(dt_mode="energy", sub=(16, 16), overlap=2, precision="fp64")),
    "3d128": dict(
        desc="3D 128^3 periodic, 50 adaptive DVD steps, FP64 beside mixed precision, "
             "RAS 8x8x8 subdomains overlap 1",
        dim=3, n=(128, 128, 128), h=0.25, cbar=0.18, seed=2, steps=50,
        opts=dict(dt_mode="energy", sub=(8, 8, 8), overlap=1, precision="fp64")),
    "3d128eta3": dict(
        desc="3D 128^3 periodic, three order parameters (App. A, eta_1..eta_3 drawn independently), "
             "50 adaptive DVD steps, FP64 beside mixed precision, RAS 8x16x16 subdomains overlap 1",
        dim=3, n=(128, 128, 128), h=0.25, cbar=0.18, seed=2, steps=50, init="three", coeffs=dict(n_eta=3),
        opts=dict(dt_mode="energy", sub=(8, 16, 16), overlap=1, precision="fp64")),
    "3d256": dict(
        desc="3D 256^3 periodic mixed precision, 100 adaptive DVD steps, RAS 16x16x16 subdomains overlap 1",
        dim=3, n=(256, 256, 256), h=0.25, cbar=0.22, seed=3, steps=100,
        opts=dict(dt_mode="energy", sub=(16, 16, 16), overlap=1, precision="mixed")),
    "3d80sphere": dict(
        desc="3D 80^3 single gamma' particle of radius 7.5 at the centre (Sec. 5.1; inside c=0.238, eta=0.01, "
             "outside c=0.1375, eta=0.99), Hooke tensor x L=1, FP64, adaptive dt (zeta=100, dt in [0.01, 2]), "
             "RAS 5x5x5 subdomains overlap 1, periodic",
        dim=3, n=(80, 80, 80), h=0.25, init="sphere", radius=7.5, coeffs=dict(Lscale=1.0), seed=0, steps=100,
        opts=dict(dt_mode="energy", sub=(5, 5, 5), overlap=1, precision="fp64")),
}


def config_fields(cfg: dict, seed_offset: int = 0):
    """Initial (c, eta) of a workload: the particle of Sec. 5.1, the seeded random
    state (seed + seed_offset), or with three order parameters its App. A form
    (eta of shape (3, N))."""
    if cfg.get("init") == "sphere":
        return sphere_fields(cfg["dim"], cfg["n"], cfg["h"], cfg["radius"])
    if cfg.get("init") == "three":
        return initial_fields3(cfg["dim"], cfg["n"], cfg["cbar"], cfg["seed"] + seed_offset)
    return initial_fields(cfg["dim"], cfg["n"], cfg["cbar"], cfg["seed"] + seed_offset)


def config_coefficients(cfg: dict) -> dict:
    """Coefficients of a workload (the defaults with its overrides)."""
    return coefficients(**cfg.get("coeffs", {}))


def serving_requests(count: int = 256, seed: int = 4, rate: float = 1.0):
    """Request stream of the serving workload: Poisson arrivals (exponential
    gaps, mean 1/rate seconds), 2-D or 3-D with probability 1/2, side length
    log-uniform in [64, 512] (2-D) or [32, 96] (3-D) rounded down to a multiple
    of 16, mean composition U(0.10, 0.25), per-request field seed."""
    u = uniform01(seed, 5 * count).reshape(count, 5)
    reqs = []
    t = 0.0
    for i in range(count):
        t += -math.log(1.0 - u[i, 0]) / rate
        if u[i, 1] < 0.5:
            dim, lo, hi = 2, 64, 512
        else:
            dim, lo, hi = 3, 32, 96
        side = int(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u[i, 2]))
        side = max(lo, (side // 16) * 16)
        reqs.append(dict(id=i, arrival=t, dim=dim, n=tuple([side] * dim), h=0.25,
                         cbar=0.10 + 0.15 * u[i, 3], seed=int(1000 + i)))
    return reqs
