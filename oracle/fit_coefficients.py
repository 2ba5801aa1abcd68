"""Derivation of the builder-chosen Gibbs-energy coefficients (L0, U1, U4).

The paper takes E0_Al, E0_Ni, L_0..L_3, U_1 and U_4 "from the CALPHAD
database" (App. A) and prints none of them.  It does print the two wells of
E_G at T = 1037 K: the disordered phase at (c, eta) = (0.137, 1) and the
ordered phase at (0.229, 0.02) (App. A, discussion of the free-energy
contour).  This script chooses the dimensionless set (L1 = L2 = L3 = 0,
dE0 = 0) for which

  1. dE/deta = 0 at the ordered well (the disordered well eta = 1 is
     stationary for any coefficients),
  2. dE/dc is equal at both wells (equal chemical potential), and
  3. the two wells share a common tangent,

with E = e1 + e2 the homogeneous Gibbs energy density of the oracle.  The
conditions are linear in (L0, U1, U4), so one 3x3 solve fixes them.  Only the
oracle is called.  The printed values are the ones stored in
``synthetic.COEFFS``.

Run:  python -m oracle.fit_coefficients
"""
import numpy as np

import oracle

R_GAS = 8.314462618          # J / (mol K)
T_K = 1037.0                 # App. A: contour plot temperature (reading of the paper)
VM_DE = 1.48e-5 * 3.3e7      # V_m * Delta E, J / mol (App. A)
WELL_DIS = (0.137, 1.0)      # App. A
WELL_ORD = (0.229, 0.02)     # App. A


def _coeffs(theta, w, L0=0.0, U1=0.0, U4=0.0):
    return dict(kappa=0.008, gamma_c=0.0, gamma_eta=0.0, theta=theta, w_psi=w, dE0=0.0,
                L=[L0, 0.0, 0.0, 0.0], U1=U1, U4=U4, eps0=0.049, C11=0.0, C12=0.0, C44=0.0, S=10)


def gibbs_density(c, eta, cf):
    """Homogeneous e1 + e2 per unit volume from the oracle's discrete energy."""
    P = oracle.Problem(1, (3,), 1.0, cf)
    X = P.interleave(np.full(3, c), np.full(3, eta))
    return P.energy(X, c) / 3.0


def conditions(cf, step=1e-6):
    def f(c, e):
        return gibbs_density(c, e, cf)

    def fc(c, e):
        return (f(c + step, e) - f(c - step, e)) / (2 * step)

    def fe(c, e):
        return (f(c, e + step) - f(c, e - step)) / (2 * step)

    (ca, ea), (cb, eb) = WELL_DIS, WELL_ORD
    ea = ea - 1e-9  # keep c (4 - 3 eta) strictly inside (0, 1) for the difference quotient
    return np.array([fe(cb, eb), fc(ca, ea) - fc(cb, eb), f(cb, eb) - f(ca, ea) - fc(cb, eb) * (cb - ca)])


def fit(w=1.0):
    theta = R_GAS * T_K / VM_DE
    base = conditions(_coeffs(theta, w))
    A = np.zeros((3, 3))
    for j, name in enumerate(("L0", "U1", "U4")):
        A[:, j] = conditions(_coeffs(theta, w, **{name: 1.0})) - base
    x = np.linalg.solve(A, -base)
    return theta, dict(L0=x[0], U1=x[1], U4=x[2])


if __name__ == "__main__":
    theta, par = fit(1.0)
    print("theta = %.10g" % theta)
    for k, v in par.items():
        print("%s = %.10g" % (k, v))
