// nks_model3.cuh -- pointwise part of the DVD derivative for the model with
// three order parameters (App. A: eta_1, eta_2, eta_3, eta_4 = 4 - sum) and
// its exact derivative block, for host and device code.
//
// Energy (scaled like the reduced model): E_1 = dis(c) + a(c) S(eta) + b(c) T(eta),
//   dis(c) = dE0 c + c(1-c) sum_i L_i (2c-1)^i = sum_{k=1..5} m_k c^k,
//   a(c) = (4 U1 + 12 U4) c^2 - 24 U4 c^3,  b(c) = -48 U4 c^3,
//   S = phi_1^2 + phi_2^2 + phi_3^2,  T = phi_1 phi_2 phi_3,
//   phi_1 = 1 - (eta_1+eta_2)/2, phi_2 = 1 - (eta_1+eta_3)/2, phi_3 = 1 - (eta_2+eta_3)/2;
// E_2 = theta { w Psi(c) + 1/4 sum_{i=1..4} Psi(c eta_i) }.
// DVD derivative (the discrete chain rule term by term): a product f(c) g(eta)
// gives G_c += f[c1, c0] (g(eta^0) + g(eta^1))/2 and G_eta_j += (f(c0) + f(c1))/2
// g_j with f[., .] the polynomial quotient (closed form in powers of c1, c0) and
// g_j the average-vector-field gradient of g: for the quadratic S its gradient
// at the midpoint, for the cubic T Simpson's rule along the segment (both
// exact); the logarithms use the Psi_S quotients of Sec. 3 with p_i = c eta_i.
// For eta_1 = eta_2 = eta_3 this is the reduced model's G_c and sum_j G_eta_j.
//
// The derivative block d(G_c, G_eta_1..3)/d(c1, eta_1..3 at level n+1) comes
// from evaluating the same code on forward-mode dual numbers (exact to rounding).
#pragma once

#include <math.h>

#include "nks_internal.cuh"

namespace nks {

#define NKS_HD __host__ __device__ __forceinline__

// forward-mode dual number: value and the derivatives along (c1, eta_1, eta_2, eta_3)
struct Dual4 {
    double v, d[4];
};

NKS_HD Dual4 dual(double v)
{
    Dual4 r;
    r.v = v;
    for (int i = 0; i < 4; i++) r.d[i] = 0.0;
    return r;
}
NKS_HD Dual4 dual_seed(double v, int i)
{
    Dual4 r = dual(v);
    r.d[i] = 1.0;
    return r;
}
NKS_HD Dual4 operator+(const Dual4 &a, const Dual4 &b)
{
    Dual4 r;
    r.v = a.v + b.v;
    for (int i = 0; i < 4; i++) r.d[i] = a.d[i] + b.d[i];
    return r;
}
NKS_HD Dual4 operator-(const Dual4 &a, const Dual4 &b)
{
    Dual4 r;
    r.v = a.v - b.v;
    for (int i = 0; i < 4; i++) r.d[i] = a.d[i] - b.d[i];
    return r;
}
NKS_HD Dual4 operator*(const Dual4 &a, const Dual4 &b)
{
    Dual4 r;
    r.v = a.v * b.v;
    for (int i = 0; i < 4; i++) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
NKS_HD Dual4 operator/(const Dual4 &a, const Dual4 &b)
{
    Dual4 r;
    const double ib = 1.0 / b.v;
    r.v = a.v * ib;
    for (int i = 0; i < 4; i++) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
NKS_HD Dual4 operator+(const Dual4 &a, double b) { return a + dual(b); }
NKS_HD Dual4 operator+(double a, const Dual4 &b) { return dual(a) + b; }
NKS_HD Dual4 operator-(const Dual4 &a, double b) { return a - dual(b); }
NKS_HD Dual4 operator-(double a, const Dual4 &b) { return dual(a) - b; }
NKS_HD Dual4 operator*(const Dual4 &a, double b)
{
    Dual4 r;
    r.v = a.v * b;
    for (int i = 0; i < 4; i++) r.d[i] = a.d[i] * b;
    return r;
}
NKS_HD Dual4 operator*(double a, const Dual4 &b) { return b * a; }
NKS_HD Dual4 logd(const Dual4 &a)
{
    Dual4 r;
    r.v = log(a.v);
    const double ia = 1.0 / a.v;
    for (int i = 0; i < 4; i++) r.d[i] = a.d[i] * ia;
    return r;
}
NKS_HD double logd(double a) { return log(a); }

// Psi_S[y1, y0] of Sec. 3: ln(ybar/(1-ybar)) + sum_{k=1}^{S-1} (a^2k - b^2k)/(2k(2k+1)),
// ybar = (y1+y0)/2, delta = (y0-y1)/2, a = delta/(1-ybar), b = delta/ybar (Horner in a^2, b^2)
template <typename T>
NKS_HD T psiS3(const DCoef &k, const T &y1, const T &y0)
{
    const T yb = 0.5 * (y1 + y0), de = 0.5 * (y0 - y1);
    const T a = de / (1.0 - yb), b = de / yb;
    const T A = a * a, B = b * b;
    T sA = A * 0.0, sB = B * 0.0;
    for (int kk = k.S - 1; kk >= 1; kk--) {
        sA = (sA + k.ser_c[kk]) * A;
        sB = (sB + k.ser_c[kk]) * B;
    }
    return logd(yb / (1.0 - yb)) + (sA - sB);
}

template <typename T>
NKS_HD void phis3(const T e[3], T f[3])
{
    f[0] = 1.0 - 0.5 * (e[0] + e[1]);
    f[1] = 1.0 - 0.5 * (e[0] + e[2]);
    f[2] = 1.0 - 0.5 * (e[1] + e[2]);
}

// gradient of T = phi_1 phi_2 phi_3 with respect to eta_1..eta_3
template <typename T>
NKS_HD void gradT3(const T e[3], T g[3])
{
    T f[3];
    phis3(e, f);
    g[0] = -0.5 * (f[2] * (f[0] + f[1]));
    g[1] = -0.5 * (f[1] * (f[0] + f[2]));
    g[2] = -0.5 * (f[0] * (f[1] + f[2]));
}

// G^1 + G^{2,S} of the three-parameter model at one point: G = (G_c, G_eta_1..3);
// level n+1 values of type T, level n values plain
template <typename T>
NKS_HD void model3_point(const DCoef &k, const T &c1, const T e1[3], double c0, const double e0[3], T G[4])
{
    const T zero = c1 * 0.0;
    // monomial coefficients of dis(c): dis = sum_{k=1..5} m_k c^k
    const double *L = k.L;
    const double m[6] = {0.0, k.dE0 + L[0] - L[1] + L[2] - L[3], -L[0] + 3.0 * L[1] - 5.0 * L[2] + 7.0 * L[3],
                         -2.0 * L[1] + 8.0 * L[2] - 18.0 * L[3], -4.0 * L[2] + 20.0 * L[3], -8.0 * L[3]};
    // powers of c1 and c0 for the closed quotients q_n = sum_{j<n} c1^j c0^(n-1-j)
    T p1[5];
    p1[0] = zero + 1.0;
    for (int i = 1; i < 5; i++) p1[i] = p1[i - 1] * c1;
    double p0[5];
    p0[0] = 1.0;
    for (int i = 1; i < 5; i++) p0[i] = p0[i - 1] * c0;
    T q[6];
    for (int n = 1; n <= 5; n++) {
        T s = zero;
        for (int j = 0; j < n; j++) s = s + p1[j] * p0[n - 1 - j];
        q[n] = s;
    }
    const double aa = 4.0 * k.U1 + 12.0 * k.U4, ab = -24.0 * k.U4, bb = -48.0 * k.U4;
    T dis_q = zero;
    for (int n = 1; n <= 5; n++) dis_q = dis_q + m[n] * q[n];
    const T a_q = aa * q[2] + ab * q[3], b_q = bb * q[3];
    const T a1 = aa * p1[2] + ab * (p1[2] * c1), b1 = bb * (p1[2] * c1);
    const double a0 = aa * c0 * c0 + ab * c0 * c0 * c0, b0 = bb * c0 * c0 * c0;
    // S, T at both levels, their discrete gradients along the segment
    T f1[3], eh[3], em[3], g1[3], gm[3];  // phi at n+1; midpoint; dT/deta at n, midpoint, n+1
    double f0[3];
    phis3(e1, f1);
    {
        const double q0[3] = {1.0 - 0.5 * (e0[0] + e0[1]), 1.0 - 0.5 * (e0[0] + e0[2]), 1.0 - 0.5 * (e0[1] + e0[2])};
        for (int i = 0; i < 3; i++) f0[i] = q0[i];
    }
    const T S1 = f1[0] * f1[0] + f1[1] * f1[1] + f1[2] * f1[2];
    const double S0 = f0[0] * f0[0] + f0[1] * f0[1] + f0[2] * f0[2];
    const T T1 = f1[0] * f1[1] * f1[2];
    const double T0 = f0[0] * f0[1] * f0[2];
    for (int j = 0; j < 3; j++) eh[j] = 0.5 * (e1[j] + e0[j]);
    T fh[3];
    phis3(eh, fh);
    // dS/deta at the midpoint (S is quadratic: exact)
    const T Sg[3] = {-1.0 * (fh[0] + fh[1]), -1.0 * (fh[0] + fh[2]), -1.0 * (fh[1] + fh[2])};
    // Simpson along the segment for the quadratic dT/deta_j (exact)
    T e0t[3];
    for (int j = 0; j < 3; j++) e0t[j] = zero + e0[j];
    gradT3(e0t, em);
    gradT3(eh, gm);
    gradT3(e1, g1);
    T Tg[3];
    for (int j = 0; j < 3; j++) Tg[j] = (em[j] + 4.0 * gm[j] + g1[j]) * (1.0 / 6.0);
    G[0] = dis_q + a_q * (0.5 * (S1 + S0)) + b_q * (0.5 * (T1 + T0));
    for (int j = 0; j < 3; j++) G[1 + j] = 0.5 * (a1 + a0) * Sg[j] + 0.5 * (b1 + b0) * Tg[j];
    // G^{2,S}
    const T e14 = 4.0 - e1[0] - e1[1] - e1[2];
    const double e04 = 4.0 - e0[0] - e0[1] - e0[2];
    const T E1[4] = {e1[0], e1[1], e1[2], e14};
    const double E0[4] = {e0[0], e0[1], e0[2], e04};
    T Qp[4];
    for (int i = 0; i < 4; i++) Qp[i] = psiS3(k, c1 * E1[i], zero + c0 * E0[i]);
    const T ch = 0.5 * (c1 + c0);
    T gc = 4.0 * k.w_psi * psiS3(k, c1, zero + c0);
    for (int i = 0; i < 4; i++) gc = gc + 0.5 * (E1[i] + E0[i]) * Qp[i];
    const double t4 = 0.25 * k.theta;
    G[0] = G[0] + t4 * gc;
    for (int j = 0; j < 3; j++) G[1 + j] = G[1 + j] + t4 * ch * (Qp[j] - Qp[3]);
}

// G and its derivative block dG[a * 4 + b] = dG_a / dx_b, x = (c1, eta_1..3 at level n+1)
NKS_HD void model3_block(const DCoef &k, const double x1[4], const double x0[4], double G[4], double dG[16])
{
    const Dual4 c1 = dual_seed(x1[0], 0);
    const Dual4 e1[3] = {dual_seed(x1[1], 1), dual_seed(x1[2], 2), dual_seed(x1[3], 3)};
    const double e0[3] = {x0[1], x0[2], x0[3]};
    Dual4 g[4];
    model3_point(k, c1, e1, x0[0], e0, g);
    for (int a = 0; a < 4; a++) {
        G[a] = g[a].v;
        for (int b = 0; b < 4; b++) dG[a * 4 + b] = g[a].d[b];
    }
}

#undef NKS_HD

}  // namespace nks
