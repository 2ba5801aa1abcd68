// nks_stencil.cu -- DVD residual, Jacobian action and energy/mass reductions.
//
// The residual of the scheme NSOA-1 (Sec. 3) is evaluated in two passes so
// that the expensive pointwise part (three Psi_S series with logarithms,
// App. B polynomials, FP64) runs once per point:
//   pass A: G_c = G^1_c + G^{2,S}_c + G^3_c + G^4_c and G_eta at each point,
//           F_eta = (eta1 - eta0)/dt + G_eta, the pointwise derivatives
//           of G^1 + G^{2,S} (reused by the Jacobian action), and the stress
//           sigma(eps^el(u1, c1)) at each point;
//   pass B: F_c = (c1 - c0)/dt - D M D G_c (flux form with level-n edge
//           mobilities) and F_u = sum_J Dhat_J sigma_IJ, plus ||F||^2 partials.
// The Jacobian action J v has an FP64 two-pass form and an FP32 tiled form
// (mixed-precision Arnoldi vectors).
#include <math.h>

#include <algorithm>

#include "nks_internal.cuh"
#include "nks_model3.cuh"

namespace nks {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int threads = kThreads)
{
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

// index of the stress component (I, J), I <= J, in the packed array
__host__ __device__ inline int scomp(int d, int I, int J)
{
    if (I > J) {
        int t = I;
        I = J;
        J = t;
    }
    if (I == J) return I;
    // off-diagonals after the d diagonal entries: (0,1), (0,2), (1,2)
    return d + (I == 0 ? J - 1 : 2);
}

// Psi_S[y1, y0] of Sec. 3 and its derivative in y1.  With ybar = (y1 + y0)/2,
// delta = (y0 - y1)/2, a = delta/(1 - ybar), b = delta/ybar:
//   Psi_S = ln(ybar/(1 - ybar)) + sum_{k=1}^{S-1} (a^2k - b^2k) / (2k(2k+1))
//   dPsi_S/dy1 = 1/2 [1/ybar + 1/(1-ybar) + sum_k (a^2k/(1-ybar) + b^2k/ybar)/(2k+1)]
//              - 1/2 [sum_k (a^(2k-1)/(1-ybar) - b^(2k-1)/ybar)/(2k+1)]
// Series by Horner in a^2, b^2 with the coefficient tables of DCoef.
__device__ inline void psiS_d1(const DCoef &k, double y1, double y0, double &q, double &d1)
{
    const double yb = 0.5 * (y1 + y0), de = 0.5 * (y0 - y1);
    const double iy = 1.0 / yb, iz = 1.0 / (1.0 - yb);
    const double a = de * iz, b = de * iy;
    const double A = a * a, B = b * b;
    double sAc = 0.0, sBc = 0.0, tAe = 0.0, tBe = 0.0;
    for (int kk = k.S - 1; kk >= 1; kk--) {
        sAc = (sAc + k.ser_c[kk]) * A;
        sBc = (sBc + k.ser_c[kk]) * B;
        tAe = tAe * A + k.ser_e[kk];
        tBe = tBe * B + k.ser_e[kk];
    }
    q = log(yb * iz) + (sAc - sBc);
    d1 = 0.5 * (iy + iz + iz * A * tAe + iy * B * tBe) - 0.5 * (iz * a * tAe - iy * b * tBe);
}

struct PointG {
    double gc, ge;              // G^1 + G^{2,S}
    double dcc, dce, dec, dee;  // d(G_c, G_eta)/d(c1, eta1)
};

// G^1 (App. B, polynomial part) + G^{2,S} (Eq. D2-1) at one point, with derivatives.
__device__ inline PointG pointG(const DCoef &k, double c1, double e1, double c0, double e0)
{
    PointG r;
    const double f1 = 1.0 - e1, f0 = 1.0 - e0;
    const double ch = 0.5 * (c1 + c0), fh = 0.5 * (f1 + f0), eh = 0.5 * (e1 + e0);
    // App. B: M1(phi) = m1a + m1b phi^2, M2(phi) = m2a + m2b phi^2 + m2c phi^3
    const double M1_0 = k.m1a + k.m1b * f0 * f0, M1_1 = k.m1a + k.m1b * f1 * f1;
    const double M2_0 = k.m2a + f0 * f0 * (k.m2b + k.m2c * f0), M2_1 = k.m2a + f1 * f1 * (k.m2b + k.m2c * f1);
    const double c1s = c1 * c1, c0s = c0 * c0, c10 = c1 * c0;
    const double Q3 = c1s + c10 + c0s;
    const double Q4 = (c1 + c0) * (c1s + c0s);
    const double Q5 = c1s * c1s + c1s * c10 + c10 * c10 + c10 * c0s + c0s * c0s;
    const double gc1 = 0.5 * (M1_0 + M1_1) * ch + (M2_0 + M2_1) * (1.0 / 6.0) * Q3 + 0.25 * k.M3 * Q4 +
                       0.2 * k.M4 * Q5 + k.M0;
    // M5(c) = -(24 U1 c^2 + 72 U4 (1 - 2c) c^2), M6(c) = 144 U4 c^3
    const double M5_0 = -c0s * (24.0 * k.U1 + 72.0 * k.U4 * (1.0 - 2.0 * c0));
    const double M5_1 = -c1s * (24.0 * k.U1 + 72.0 * k.U4 * (1.0 - 2.0 * c1));
    const double M6_0 = 144.0 * k.U4 * c0s * c0, M6_1 = 144.0 * k.U4 * c1s * c1;
    const double P3 = f1 * f1 + f1 * f0 + f0 * f0;
    const double ge1 = 0.5 * (M5_0 + M5_1) * fh + (M6_0 + M6_1) * (1.0 / 6.0) * P3;
    // derivatives of G^1
    const double g1c_c = 0.25 * (M1_0 + M1_1) + (M2_0 + M2_1) * (1.0 / 6.0) * (2.0 * c1 + c0) +
                         0.25 * k.M3 * (3.0 * c1s + 2.0 * c10 + c0s) +
                         0.2 * k.M4 * (4.0 * c1s * c1 + 3.0 * c1s * c0 + 2.0 * c1 * c0s + c0s * c0);
    const double g1c_e = -(k.m1b * f1 * ch + (2.0 * k.m2b * f1 + 3.0 * k.m2c * f1 * f1) * (1.0 / 6.0) * Q3);
    const double dM5 = -(48.0 * k.U1 * c1 + 72.0 * k.U4 * (2.0 * c1 - 6.0 * c1s));
    const double dM6 = 432.0 * k.U4 * c1s;
    const double g1e_c = 0.5 * dM5 * fh + dM6 * (1.0 / 6.0) * P3;
    const double g1e_e = -(0.25 * (M5_0 + M5_1) + (M6_0 + M6_1) * (1.0 / 6.0) * (2.0 * f1 + f0));
    // G^{2,S}: p = c eta, q = c (4 - 3 eta)
    const double p1 = c1 * e1, p0 = c0 * e0;
    const double q1 = c1 * (4.0 - 3.0 * e1), q0 = c0 * (4.0 - 3.0 * e0);
    double Qc = 0.0, Dc = 0.0, Qp, Dp, Qq, Dq;
    if (k.w_psi != 0.0) psiS_d1(k, c1, c0, Qc, Dc);
    psiS_d1(k, p1, p0, Qp, Dp);
    psiS_d1(k, q1, q0, Qq, Dq);
    const double t4 = 0.25 * k.theta;
    const double eph = 4.0 - 3.0 * eh;
    const double gc2 = t4 * (4.0 * k.w_psi * Qc + 3.0 * eh * Qp + eph * Qq);
    const double ge2 = t4 * 3.0 * ch * (Qp - Qq);
    const double g2c_c = t4 * (4.0 * k.w_psi * Dc + 3.0 * eh * e1 * Dp + eph * (4.0 - 3.0 * e1) * Dq);
    const double g2c_e = t4 * (1.5 * (Qp - Qq) + 3.0 * c1 * (eh * Dp - eph * Dq));
    const double g2e_c = t4 * 3.0 * (0.5 * (Qp - Qq) + ch * (e1 * Dp - (4.0 - 3.0 * e1) * Dq));
    const double g2e_e = t4 * 3.0 * ch * c1 * (Dp + 3.0 * Dq);
    r.gc = gc1 + gc2;
    r.ge = ge1 + ge2;
    r.dcc = g1c_c + g2c_c;
    r.dce = g1c_e + g2c_e;
    r.dec = g1e_c + g2e_c;
    r.dee = g1e_e + g2e_e;
    return r;
}

__device__ inline bool in_domain(double c, double e)
{
    const double p = c * e, q = c * (4.0 - 3.0 * e);
    return c > 0.0 && c < 1.0 && p > 0.0 && p < 1.0 && q > 0.0 && q < 1.0;
}

// three order parameters: c and the four site fractions c eta_i (eta_4 = 4 - sum)
__device__ inline bool in_domain3(double c, const double (&e)[3])
{
    bool ok = c > 0.0 && c < 1.0;
    const double e4 = 4.0 - e[0] - e[1] - e[2];
    for (int i = 0; i < 4; i++) {
        const double q = c * (i < 3 ? e[i] : e4);
        ok = ok && q > 0.0 && q < 1.0;
    }
    return ok;
}

// symmetric gradient of the displacement at (x, y, z): Du[I][J] = Dhat_J u_I
template <typename TV>
__device__ inline void grad_u(const DGrid &g, const TV *U /* field 2 plane */, int x, int y, int z,
                              double (&Du)[3][3])
{
    const double i2h = g.i2h;
    for (int I = 0; I < g.dim; I++)
        for (int J = 0; J < g.dim; J++)
            Du[I][J] = ((double)U[I * g.N + nbrJ(g, x, y, z, J, +1)] - (double)U[I * g.N + nbrJ(g, x, y, z, J, -1)]) * i2h;
}

// sigma = C : (sym(Du) - s I) for the cubic Hooke law, packed by scomp()
__device__ inline void hooke_packed(const DGrid &g, const DCoef &k, const double (&Du)[3][3], double s,
                                    double *sig, long long p)
{
    const int d = g.dim;
    double tr = 0.0;
    for (int I = 0; I < d; I++) tr += Du[I][I] - s;
    for (int I = 0; I < d; I++) {
        const double eII = Du[I][I] - s;
        sig[(long long)I * g.N + p] = k.C11 * eII + k.C12 * (tr - eII);
        for (int J = I + 1; J < d; J++)
            sig[(long long)scomp(d, I, J) * g.N + p] = k.C44 * (Du[I][J] + Du[J][I]);
    }
}

// ---------------------------------------------------------------------------

__global__ void k_mobility(DGrid g, DCoef k, Bat bt, const double *__restrict__ c0, double *__restrict__ mob)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    c0 = shift(c0, io);
    mob = shift(mob, io);
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    int x, y, z;
    coords_of(g, p, x, y, z);
    const double a = c0[p] * (1.0 - c0[p]);
    for (int J = 0; J < g.dim; J++) {
        const double cb = c0[nbrJ(g, x, y, z, J, +1)];
        mob[J * g.N + p] = k.kappa * 0.5 * (a + cb * (1.0 - cb));  // M_{p + e_J/2} (Sec. 3)
    }
}

// tr eps^el of the level-n state (used by G^3 at n + 1/2)
__global__ void k_trace0(DGrid g, DCoef k, Bat bt, const double *__restrict__ isc, const double *__restrict__ X0,
                         double *__restrict__ tr0)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    X0 = shift(X0, io);
    tr0 = shift(tr0, io);
    const double cbar0 = shift(isc, io)[I_CBAR0];
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    int x, y, z;
    coords_of(g, p, x, y, z);
    const double *U = X0 + (1 + k.ne) * g.N;
    double tr = 0.0;
    for (int K = 0; K < g.dim; K++)
        tr += (U[K * g.N + nbrJ(g, x, y, z, K, +1)] - U[K * g.N + nbrJ(g, x, y, z, K, -1)]) * g.i2h;
    tr0[p] = tr - g.dim * k.eps0 * (X0[p] - cbar0);
}

// NE: order parameters (1: the reduced model; 3: App. A, whose pointwise part
// and its 4 x 4 derivative block come from model3_block)
template <int NE>
__global__ void k_res_a(DGrid g, DCoef k, Bat bt, const double *__restrict__ isc, int mode,
                        const double *__restrict__ X1, const double *__restrict__ X0, const double *__restrict__ tr0,
                        double *__restrict__ Gc, double *__restrict__ sig, double *__restrict__ part,
                        double *__restrict__ F, int *__restrict__ flag)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    X1 = shift(X1, io);
    X0 = shift(X0, io);
    tr0 = shift(tr0, io);
    Gc = shift(Gc, io);
    sig = shift(sig, io);
    part = shift(part, io);
    F = shift(F, io);
    flag = shift(flag, io);
    const double idt = shift(isc, io)[I_IDT], cbar0 = shift(isc, io)[I_CBAR0];
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= g.N) return;
    int x, y, z;
    coords_of(g, p, x, y, z);
    const long long N = g.N;
    const double c1 = X1[p];
    double e1[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < NE; j++) e1[j] = X1[(1 + j) * N + p];
    if (!(NE == 3 ? in_domain3(c1, e1) : in_domain(c1, e1[0]))) atomicOr(flag, 1);
    double Du[3][3];
    if (k.elastic) {
        grad_u(g, X1 + (1 + NE) * N, x, y, z, Du);
        hooke_packed(g, k, Du, k.eps0 * (c1 - cbar0), sig, p);
    }
    if (mode != 0) {
#pragma unroll
        for (int j = 0; j < NE; j++) F[(1 + j) * N + p] = 0.0;
        return;
    }
    const double c0 = X0[p];
    double e0[3] = {0.0, 0.0, 0.0}, ge[3] = {0.0, 0.0, 0.0}, gc;
#pragma unroll
    for (int j = 0; j < NE; j++) e0[j] = X0[(1 + j) * N + p];
    if constexpr (NE == 3) {
        const double x1[4] = {c1, e1[0], e1[1], e1[2]}, x0[4] = {c0, e0[0], e0[1], e0[2]};
        double G[4], dG[16];
        model3_block(k, x1, x0, G, dG);
        gc = G[0];
#pragma unroll
        for (int j = 0; j < 3; j++) ge[j] = G[1 + j];
#pragma unroll
        for (int a = 0; a < 16; a++) part[a * N + p] = dG[a];
    } else {
        const PointG G = pointG(k, c1, e1[0], c0, e0[0]);
        gc = G.gc;
        ge[0] = G.ge;
        part[p] = G.dcc;
        part[N + p] = G.dce;
        part[2 * N + p] = G.dec;
        part[3 * N + p] = G.dee;
    }
    if (k.elastic) {
        // G^3_c = -eps0 sum_I sigma_II(eps^el_{n+1/2}) = -eps0 lam (tr1 + tr0)/2
        double tr1 = -g.dim * k.eps0 * (c1 - cbar0);
        for (int K = 0; K < g.dim; K++) tr1 += Du[K][K];
        gc += -k.eps0 * k.lam * 0.5 * (tr1 + tr0[p]);
    }
    // G^4 = (-gamma_c D^2 c_h, -3 gamma_eta D^2 eta_h), D^2 = sum_J D+_J D-_J; with three
    // order parameters -gamma_eta D^2 eta_j,h, the eta_j rows carrying the kinetic factor 3
    const double ih2 = g.ih2;
    double lc = 0.0, le[3] = {0.0, 0.0, 0.0};
    const double chp = c1 + c0;
    for (int J = 0; J < g.dim; J++) {
        const long long pp = nbrJ(g, x, y, z, J, +1), pm = nbrJ(g, x, y, z, J, -1);
        lc += (X1[pp] + X0[pp]) + (X1[pm] + X0[pm]) - 2.0 * chp;
#pragma unroll
        for (int j = 0; j < NE; j++) {
            const long long o = (1 + j) * N;
            le[j] += (X1[o + pp] + X0[o + pp]) + (X1[o + pm] + X0[o + pm]) - 2.0 * (e1[j] + e0[j]);
        }
    }
    gc += -k.gamma_c * 0.5 * lc * ih2;
    Gc[p] = gc;
    if constexpr (NE == 3) {
#pragma unroll
        for (int j = 0; j < 3; j++)
            F[(1 + j) * N + p] = (e1[j] - e0[j]) * idt + k.keta * (ge[j] - k.gamma_eta * 0.5 * le[j] * ih2);
    } else {
        ge[0] += -3.0 * k.gamma_eta * 0.5 * le[0] * ih2;
        F[N + p] = (e1[0] - e0[0]) * idt + ge[0];
    }
}

__global__ void __launch_bounds__(kRedThreads) k_res_b(DGrid g, DCoef k, Bat bt, const double *__restrict__ isc,
                                                       int mode, const double *__restrict__ X1,
                                                       const double *__restrict__ X0, const double *__restrict__ Gc,
                                                       const double *__restrict__ mob, const double *__restrict__ sig,
                                                       double *__restrict__ F, double *__restrict__ partials)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    X1 = shift(X1, io);
    X0 = shift(X0, io);
    Gc = shift(Gc, io);
    mob = shift(mob, io);
    sig = shift(sig, io);
    F = shift(F, io);
    partials = shift(partials, io);
    const double idt = shift(isc, io)[I_IDT];
    const long long N = g.N;
    const double ih2 = g.ih2, i2h = g.i2h;
    double acc[1] = {0.0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords_of(g, p, x, y, z);
        double fc = 0.0;
        if (mode == 0) {
            double flux = 0.0;
            const double G0 = Gc[p];
            for (int J = 0; J < g.dim; J++) {
                const long long pp = nbrJ(g, x, y, z, J, +1), pm = nbrJ(g, x, y, z, J, -1);
                flux += mob[J * N + p] * (Gc[pp] - G0) - mob[J * N + pm] * (G0 - Gc[pm]);
            }
            fc = (X1[p] - X0[p]) * idt - flux * ih2;
        }
        F[p] = fc;
        double s = fc * fc;
        for (int j = 0; j < k.ne; j++) {
            const double fe = F[(1 + j) * N + p];
            s += fe * fe;
        }
        if (k.elastic) {
            const long long ou = (long long)(1 + k.ne) * N;
            // F_uI = sum_J Dhat_J sigma_IJ on a periodic grid; with Neumann boundaries the
            // exact variation -dE_3/du of the discrete elastic energy, which differs only
            // where the neighbour is the mirrored cell itself: its sigma enters with the
            // opposite sign (traction-free rows)
            for (int I = 0; I < g.dim; I++) {
                double div = 0.0;
                for (int J = 0; J < g.dim; J++) {
                    const int cmp = scomp(g.dim, I, J);
                    const long long pp = nbrJ(g, x, y, z, J, +1), pm = nbrJ(g, x, y, z, J, -1);
                    const double sp = pp == p ? -1.0 : 1.0, sm = pm == p ? -1.0 : 1.0;
                    div += (sp * sig[cmp * N + pp] - sm * sig[cmp * N + pm]) * i2h;
                }
                F[ou + I * N + p] = div;
                s += div * div;
            }
        }
        acc[0] += s;
    }
    block_reduce_store<1>(acc, partials);
}

// Jacobian action J v: the linearisation of the residual at the current Newton
// iterate applied to v,
//   dG_c      = dcc v_c + dce v_eta - 1/2 gamma_c Lap_h v_c - 1/2 eps0 lam (tr Dhat v_u - d eps0 v_c)
//   sigma     = C : (sym Dhat v_u - eps0 v_c I)
//   (J v)_c   = v_c/dt - div_h(M^n grad_h dG_c)          (edge mobilities at level n)
//   (J v)_eta = v_eta/dt + dec v_c + dee v_eta - 3/2 gamma_eta Lap_h v_eta
//   (J v)_u_I = sum_J Dhat_J sigma_IJ,
// with the pointwise derivatives (dcc, dce, dec, dee) of the last residual
// evaluation (part).  With NE = 3 order parameters the pointwise block is 4 x 4
// (part[(a * 4 + b) N + p] = dG_a/dx_b, x = (c, eta_1..eta_3)), dG_c sums over the
// three eta_j, and the eta_j rows carry the kinetic factor keta = 3 on the
// pointwise block (their Laplacian weight is the same 3/2 gamma_eta).  mode 1 (displacement-only system) keeps the identity on the
// c and eta rows.  With zsum != nullptr the action is applied to P v instead of v,
// where P removes the mean m = zsum[0] / N of v_c (the null modes of v_u are
// annihilated by J): every use of v_c reads v_c - m, except the Laplacian, which
// a constant shift leaves unchanged.
// Indices are 32-bit (the problem constructor checks nf N < 2^31).
//
// GB300 executes FP64 at 1/64 of the FP32 rate, so the FP64 form is organised to
// do each FP64 operation once: two passes over the grid (dG_c and sigma written
// once per point, then the flux and divergence forms), constants folded on the
// host (JvConst).  The FP32 form (mixed precision: Arnoldi vectors, FP32 copies
// of the coefficients) is one tiled kernel that recomputes dG_c and sigma on a
// one-point halo in shared memory instead of writing them out.

// per-operator constants with the grid spacings folded in, in the arithmetic
// type of the kernel (converted once on the host: on GB300 a double-to-float
// conversion per use would occupy the FP64 pipe)
template <typename T>
struct JvConst {
    T gc;        // 1/2 gamma_c / h^2
    T ge;        // 3/2 gamma_eta / h^2
    T ih2;       // 1/h^2
    T el_t;      // 1/2 eps0 lam / (2h)  (times the undivided trace)
    T el_c;      // 1/2 eps0 lam d eps0
    T ab, b, c4; // (C11 - C12)/(2h), C12/(2h), C44/(2h)
    T ls;        // lam eps0
    T i2h;       // 1/(2h)
    T invN;      // 1/N: the mean of v_c is zsum / N
    T keta;      // kinetic factor of the eta rows (three order parameters: 3)
    int mode;
};

template <typename T>
static JvConst<T> jv_const(const DGrid &g, const DCoef &k, int mode)
{
    JvConst<T> c;
    const double i2h = 0.5 / g.h, ih2 = 1.0 / (g.h * g.h);
    c.gc = (T)(0.5 * k.gamma_c * ih2);
    c.ge = (T)(1.5 * k.gamma_eta * ih2);
    c.ih2 = (T)ih2;
    c.el_t = (T)(0.5 * k.eps0 * k.lam * i2h);
    c.el_c = (T)(0.5 * k.eps0 * k.lam * g.dim * k.eps0);
    c.ab = (T)((k.C11 - k.C12) * i2h);
    c.b = (T)(k.C12 * i2h);
    c.c4 = (T)(k.C44 * i2h);
    c.ls = (T)(k.lam * k.eps0);
    c.i2h = (T)i2h;
    c.invN = (T)(1.0 / (double)g.N);
    c.keta = (T)k.keta;
    c.mode = mode;
    return c;
}

// neighbour offsets of point (x, y, z) along each axis, 32-bit: periodic, or
// (bc, Neumann) the point itself beyond a boundary (mirror ghost)
template <int D>
__device__ __forceinline__ void nbr_offsets(const int (&c3)[3], const int (&nn)[3], int p, int (&im)[3], int (&ip)[3],
                                            int bc)
{
    int st = 1;
#pragma unroll
    for (int J = 0; J < D; J++) {
        im[J] = p + (c3[J] == 0 ? (bc ? 0 : (nn[J] - 1) * st) : -st);
        ip[J] = p + (c3[J] == nn[J] - 1 ? (bc ? 0 : -(nn[J] - 1) * st) : st);
        st *= nn[J];
    }
}

// dG_c and sigma at one point; T is the arithmetic type
template <int D, bool EL, int NE, typename T, typename TV, typename TC>
__device__ __forceinline__ void jv_point(const JvConst<T> &c, int mode, int N, int idx, const int (&im)[3],
                                         const int (&ip)[3], const TV *__restrict__ v, const TC *__restrict__ part,
                                         T m, T &dg, T (&sg)[EL ? D * (D + 1) / 2 : 1])
{
    constexpr int KU = 1 + NE;  // first displacement field
    const T v0 = (T)v[idx], vc = v0 - m;
    T trd = (T)0;
    if constexpr (EL) {
        T Dd[D][D];
#pragma unroll
        for (int I = 0; I < D; I++)
#pragma unroll
            for (int J = 0; J < D; J++) Dd[I][J] = (T)v[(KU + I) * N + ip[J]] - (T)v[(KU + I) * N + im[J]];
#pragma unroll
        for (int I = 0; I < D; I++) trd += Dd[I][I];
        // sigma_II = (C11 - C12) e_II + C12 tr e - lam eps0 v_c;  sigma_IJ = C44 (D_IJ + D_JI)
        const T common = c.b * trd - c.ls * vc;
#pragma unroll
        for (int I = 0; I < D; I++) {
            sg[I] = c.ab * Dd[I][I] + common;
#pragma unroll
            for (int J = I + 1; J < D; J++) sg[scomp(D, I, J)] = c.c4 * (Dd[I][J] + Dd[J][I]);
        }
    }
    if (mode == 0) {
        T sn = (T)0;
#pragma unroll
        for (int J = 0; J < D; J++) sn += (T)v[ip[J]] + (T)v[im[J]];
        const T lc = sn - (T)(2 * D) * v0;
        dg = (T)part[idx] * vc;
#pragma unroll
        for (int j = 1; j <= NE; j++) dg += (T)part[j * N + idx] * (T)v[j * N + idx];
        dg -= c.gc * lc;
        if constexpr (EL) dg += c.el_c * vc - c.el_t * trd;
    }
}

// ---- FP64: two passes --------------------------------------------------------

// grid: (x tiles, y tiles, n_z x instances); the instance is blockIdx.z / n_z
template <int D>
__device__ __forceinline__ bool grid_point(const DGrid &g, int (&c3)[3], int &p)
{
    c3[0] = blockIdx.x * blockDim.x + threadIdx.x;
    c3[1] = D >= 2 ? (int)(blockIdx.y * blockDim.y + threadIdx.y) : 0;
    c3[2] = D == 3 ? (int)(blockIdx.z % g.n[2]) : 0;
    if (c3[0] >= g.n[0] || c3[1] >= g.n[1]) return false;
    p = c3[0] + g.n[0] * (c3[1] + g.n[1] * c3[2]);
    return true;
}

template <int D, bool EL, int NE>
__global__ void __launch_bounds__(256) k_jv64_a(DGrid g, JvConst<double> c, Bat bt, const double *__restrict__ part,
                                                const double *__restrict__ v, double *__restrict__ dG,
                                                double *__restrict__ sig, const double *__restrict__ zsum)
{
    long long io;
    if (!inst_off(bt, blockIdx.z / g.n[2], io)) return;
    part = shift(part, io);
    v = shift(v, io);
    dG = shift(dG, io);
    sig = shift(sig, io);
    const double m = zsum ? shift(zsum, io)[0] * c.invN : 0.0;
    int c3[3], p;
    if (!grid_point<D>(g, c3, p)) return;
    const int nn[3] = {g.n[0], g.n[1], g.n[2]};
    const int N = (int)g.N;
    int im[3], ip[3];
    nbr_offsets<D>(c3, nn, p, im, ip, g.bc);
    double dg = 0.0, sg[EL ? D * (D + 1) / 2 : 1];
    jv_point<D, EL, NE, double, double, double>(c, c.mode, N, p, im, ip, v, part, m, dg, sg);
    if (c.mode == 0) dG[p] = dg;
    if constexpr (EL) {
#pragma unroll
        for (int q = 0; q < D * (D + 1) / 2; q++) sig[q * N + p] = sg[q];
    }
}

template <int D, bool EL, int NE>
__global__ void __launch_bounds__(256) k_jv64_b(DGrid g, JvConst<double> c, Bat bt, const double *__restrict__ isc,
                                                const double *__restrict__ part, const double *__restrict__ mob,
                                                const double *__restrict__ v, const double *__restrict__ dG,
                                                const double *__restrict__ sig, double *__restrict__ Jv,
                                                const double *__restrict__ zsum)
{
    constexpr int KU = 1 + NE;
    long long io;
    if (!inst_off(bt, blockIdx.z / g.n[2], io)) return;
    part = shift(part, io);
    mob = shift(mob, io);
    v = shift(v, io);
    dG = shift(dG, io);
    sig = shift(sig, io);
    Jv = shift(Jv, io);
    const double idt = shift(isc, io)[I_IDT];
    const double m = zsum ? shift(zsum, io)[0] * c.invN : 0.0;
    int c3[3], p;
    if (!grid_point<D>(g, c3, p)) return;
    const int nn[3] = {g.n[0], g.n[1], g.n[2]};
    const int N = (int)g.N;
    int im[3], ip[3];
    nbr_offsets<D>(c3, nn, p, im, ip, g.bc);
    const double vc = v[p] - m;
    double ve[NE], je[NE], jc;
#pragma unroll
    for (int j = 0; j < NE; j++) ve[j] = v[(1 + j) * N + p];
    if (c.mode == 0) {
        const double G0 = dG[p];
        double flux = 0.0, sn[NE];
#pragma unroll
        for (int j = 0; j < NE; j++) sn[j] = 0.0;
#pragma unroll
        for (int J = 0; J < D; J++) {
            flux += mob[J * N + p] * (dG[ip[J]] - G0) - mob[J * N + im[J]] * (G0 - dG[im[J]]);
#pragma unroll
            for (int j = 0; j < NE; j++) sn[j] += v[(1 + j) * N + ip[J]] + v[(1 + j) * N + im[J]];
        }
        jc = vc * idt - flux * c.ih2;
#pragma unroll
        for (int j = 0; j < NE; j++) {
            const double *pr = part + (size_t)(1 + j) * KU * N + p;  // row 1 + j of the pointwise block
            if constexpr (NE == 1) {
                je[j] = ve[j] * idt + pr[0] * vc + pr[N] * ve[j] - c.ge * (sn[j] - (2 * D) * ve[j]);
            } else {
                double pw = pr[0] * vc;
#pragma unroll
                for (int i = 0; i < NE; i++) pw += pr[(size_t)(1 + i) * N] * ve[i];
                je[j] = ve[j] * idt + c.keta * pw - c.ge * (sn[j] - (2 * D) * ve[j]);
            }
        }
    } else {
        jc = vc;
#pragma unroll
        for (int j = 0; j < NE; j++) je[j] = ve[j];
    }
    Jv[p] = jc;
#pragma unroll
    for (int j = 0; j < NE; j++) Jv[(1 + j) * N + p] = je[j];
    if constexpr (EL) {
        // as the residual: the mirrored neighbour's stress enters with the opposite sign
#pragma unroll
        for (int I = 0; I < D; I++) {
            double div = 0.0;
#pragma unroll
            for (int J = 0; J < D; J++) {
                const int q = scomp(D, I, J) * N;
                div += (ip[J] == p ? -sig[q + ip[J]] : sig[q + ip[J]]) - (im[J] == p ? -sig[q + im[J]] : sig[q + im[J]]);
            }
            Jv[(KU + I) * N + p] = div * c.i2h;
        }
    }
}

// ---- FP32: one tiled kernel --------------------------------------------------

template <int D>
struct JvTile;
template <>
struct JvTile<1> {
    static constexpr int TX = 256, TY = 1, TZ = 1;
};
template <>
struct JvTile<2> {
    static constexpr int TX = 32, TY = 8, TZ = 1;
};
template <>
struct JvTile<3> {
    static constexpr int TX = 16, TY = 4, TZ = 4;
};

template <int D, bool EL, int NE>
__global__ void __launch_bounds__(256) k_jv32(DGrid g, JvConst<float> c, Bat bt, const double *__restrict__ isc,
                                              const float *__restrict__ part, const float *__restrict__ mob,
                                              const float *__restrict__ v, float *__restrict__ Jv,
                                              const double *__restrict__ zsum)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    part = shift(part, io);
    mob = shift(mob, io);
    v = shift(v, io);
    Jv = shift(Jv, io);
    constexpr int TX = JvTile<D>::TX, TY = JvTile<D>::TY, TZ = JvTile<D>::TZ;
    constexpr int HX = TX + 2, HY = D >= 2 ? TY + 2 : 1, HZ = D == 3 ? TZ + 2 : 1;
    constexpr int NH = HX * HY * HZ;
    constexpr int NS = EL ? D * (D + 1) / 2 : 1;
    __shared__ float sG[NH];
    __shared__ float sS[NS][EL ? NH : 1];
    const int nn[3] = {g.n[0], g.n[1], g.n[2]};
    const int N = (int)g.N;
    const int tx_n = (nn[0] + TX - 1) / TX, ty_n = (nn[1] + TY - 1) / TY;
    int b = blockIdx.x;
    const int x0 = (b % tx_n) * TX;
    b /= tx_n;
    const int y0 = (b % ty_n) * TY;
    const int z0 = (b / ty_n) * TZ;
    const int sh[3] = {1, HX, HX * HY};
    // per-block scalars (one double-to-float conversion each, not one per thread)
    __shared__ float sidt, sm;
    if (threadIdx.x == 0) {
        sidt = (float)shift(isc, io)[I_IDT];
        sm = zsum ? (float)(shift(zsum, io)[0] * (double)c.invN) : 0.f;
    }
    __syncthreads();
    const float m = sm, idt = sidt;

    // tile + halo: dG_c and sigma
    for (int q = threadIdx.x; q < NH; q += blockDim.x) {
        const int hx = q % HX, hy = (q / HX) % HY, hz = q / (HX * HY);
        int c3[3] = {x0 - 1 + hx, D >= 2 ? y0 - 1 + hy : 0, D == 3 ? z0 - 1 + hz : 0};
        if (c3[0] > nn[0] || c3[1] > nn[1] || c3[2] > nn[2]) continue;  // beyond a ragged tile: never read
        // periodic wrap, or with Neumann boundaries the mirror ghost's cell (a halo cell
        // beyond the grid holds the boundary cell's values)
#pragma unroll
        for (int J = 0; J < 3; J++) c3[J] = g.bc ? (c3[J] < 0 ? 0 : (c3[J] >= nn[J] ? nn[J] - 1 : c3[J])) : wrapi(c3[J], nn[J]);
        const int idx = c3[0] + nn[0] * (c3[1] + nn[1] * c3[2]);
        int im[3], ip[3];
        nbr_offsets<D>(c3, nn, idx, im, ip, g.bc);
        float dg = 0.f, sg[NS];
        jv_point<D, EL, NE, float, float, float>(c, c.mode, N, idx, im, ip, v, part, m, dg, sg);
        sG[q] = dg;
        if constexpr (EL) {
#pragma unroll
            for (int s = 0; s < NS; s++) sS[s][q] = sg[s];
        }
    }
    __syncthreads();

    const float ih2 = c.ih2, ge = c.ge, i2h = c.i2h;
    for (int t = threadIdx.x; t < TX * TY * TZ; t += blockDim.x) {
        const int tx = t % TX, ty = (t / TX) % TY, tz = t / (TX * TY);
        const int c3[3] = {x0 + tx, y0 + ty, z0 + tz};
        if (c3[0] >= nn[0] || c3[1] >= nn[1] || c3[2] >= nn[2]) continue;
        const int p = c3[0] + nn[0] * (c3[1] + nn[1] * c3[2]);
        int im[3], ip[3];
        nbr_offsets<D>(c3, nn, p, im, ip, g.bc);
        const int hq = (tx + 1) + (D >= 2 ? HX * (ty + 1) : 0) + (D == 3 ? HX * HY * (tz + 1) : 0);
        constexpr int KU = 1 + NE;
        const float vc = v[p] - m;
        float ve[NE], je[NE], jc;
#pragma unroll
        for (int j = 0; j < NE; j++) ve[j] = v[(1 + j) * N + p];
        if (c.mode == 0) {
            const float G0 = sG[hq];
            float flux = 0.f, sn[NE];
#pragma unroll
            for (int j = 0; j < NE; j++) sn[j] = 0.f;
#pragma unroll
            for (int J = 0; J < D; J++) {
                flux += mob[J * N + p] * (sG[hq + sh[J]] - G0) - mob[J * N + im[J]] * (G0 - sG[hq - sh[J]]);
#pragma unroll
                for (int j = 0; j < NE; j++) sn[j] += v[(1 + j) * N + ip[J]] + v[(1 + j) * N + im[J]];
            }
            jc = vc * idt - flux * ih2;
#pragma unroll
            for (int j = 0; j < NE; j++) {
                const float *pr = part + (size_t)(1 + j) * KU * N + p;
                if constexpr (NE == 1) {
                    je[j] = ve[j] * idt + pr[0] * vc + pr[N] * ve[j] - ge * (sn[j] - (float)(2 * D) * ve[j]);
                } else {
                    float pw = pr[0] * vc;
#pragma unroll
                    for (int i = 0; i < NE; i++) pw += pr[(size_t)(1 + i) * N] * ve[i];
                    je[j] = ve[j] * idt + c.keta * pw - ge * (sn[j] - (float)(2 * D) * ve[j]);
                }
            }
        } else {
            jc = vc;
#pragma unroll
            for (int j = 0; j < NE; j++) je[j] = ve[j];
        }
        Jv[p] = jc;
#pragma unroll
        for (int j = 0; j < NE; j++) Jv[(1 + j) * N + p] = je[j];
        if constexpr (EL) {
            // the mirrored neighbour's stress enters with the opposite sign (Neumann)
#pragma unroll
            for (int I = 0; I < D; I++) {
                float div = 0.f;
#pragma unroll
                for (int J = 0; J < D; J++) {
                    const int s = scomp(D, I, J);
                    const float a = sS[s][hq + sh[J]], b = sS[s][hq - sh[J]];
                    div += (ip[J] == p ? -a : a) - (im[J] == p ? -b : b);
                }
                Jv[(KU + I) * N + p] = div * i2h;
            }
        }
    }
}

// ---- FP32, 3-D: 2.5-D z-marching form ------------------------------------------
//
// A block owns a JZ_TX x JZ_TY column of points and marches along z over zc planes.
// The input v streams through a ring of five planes in shared memory (every field,
// with a two-cell halo in x and y), each plane loaded once by cp.async while the
// block works on the planes below it; dG_c and sigma are formed once per halo cell
// and plane into a ring of three planes, from which the flux and divergence forms
// of the plane take their neighbours.  Per output point the block reads v once
// (plus the halo share), the pointwise block and the mobilities once, and writes
// J v once; dG_c and sigma never leave shared memory.
//
// Halo cells beyond the grid hold the wrapped (periodic) or mirrored (Neumann:
// the boundary cell itself) values; with Neumann boundaries a stage-1 cell or
// plane beyond the grid takes the values of the boundary cell, as in the tiled form.
constexpr int JZ_TX = 32, JZ_TY = 8;
constexpr int JZ_VX = JZ_TX + 4, JZ_VY = JZ_TY + 4, JZ_VP = JZ_VX * JZ_VY;  // v tile, 2-cell halo
constexpr int JZ_SX = JZ_TX + 2, JZ_SY = JZ_TY + 2, JZ_SP = JZ_SX * JZ_SY;  // dG / sigma tile, 1-cell halo
constexpr int JZ_NV = 5;                                                   // v ring planes
// threads per block: every dG / sigma cell of a plane in one pass (340 of 352); the
// first 256 form J v on the plane
constexpr int JZ_THREADS = 352;
static_assert(JZ_THREADS >= JZ_SP && JZ_THREADS >= JZ_TX * JZ_TY && 2 * JZ_THREADS >= JZ_VP, "tile shapes");

__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// coordinate a of an axis of n cells seen from a halo cell (|overhang| <= 2):
// periodic wrap, or the mirror ghost's cell (clamp) with Neumann boundaries
__device__ __forceinline__ int halo_coord(int a, int n, int bc)
{
    if (bc) return a < 0 ? 0 : (a >= n ? n - 1 : a);
    return a < 0 ? a + n : (a >= n ? a - n : a);
}

// resident blocks of k_jv32_z on the device (set with the kernel's attributes)
template <bool EL, int NE>
struct JzOcc {
    static int resident;
};
template <bool EL, int NE>
int JzOcc<EL, NE>::resident = 0;

template <int NF>
static size_t jv32z_smem(int ns)
{
    return sizeof(float) * ((size_t)JZ_NV * NF * JZ_VP + (size_t)3 * (1 + ns) * JZ_SP);
}

template <bool EL, int NE>
__global__ void __launch_bounds__(JZ_THREADS) k_jv32_z(DGrid g, JvConst<float> c, Bat bt, const double *__restrict__ isc,
                                                const float *__restrict__ part, const float *__restrict__ mob,
                                                const float *__restrict__ v, float *__restrict__ Jv,
                                                const double *__restrict__ zsum, int zc)
{
    constexpr int KU = 1 + NE, NF = KU + (EL ? 3 : 0), NS = EL ? 6 : 1;
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    part = shift(part, io);
    mob = shift(mob, io);
    v = shift(v, io);
    Jv = shift(Jv, io);
    extern __shared__ __align__(16) float jz_smem[];
    float *sv = jz_smem;                            // [JZ_NV][NF][JZ_VP]
    float *sg = jz_smem + JZ_NV * NF * JZ_VP;       // [3][1 + NS][JZ_SP]
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], bc = g.bc;
    const int N = (int)g.N, nxy = nx * ny;
    const int tx_n = (nx + JZ_TX - 1) / JZ_TX, ty_n = (ny + JZ_TY - 1) / JZ_TY;
    int b = blockIdx.x;
    const int x0 = (b % tx_n) * JZ_TX;
    b /= tx_n;
    const int y0 = (b % ty_n) * JZ_TY;
    const int z0 = (b / ty_n) * zc;
    const int z1 = min(z0 + zc, nz);
    const int tid = threadIdx.x;
    __shared__ float sidt, sm;
    if (tid == 0) {
        sidt = (float)shift(isc, io)[I_IDT];
        sm = zsum ? (float)(shift(zsum, io)[0] * (double)c.invN) : 0.f;
    }
    // in-plane source offsets of this thread's v-tile cells (at most two); -1: unused cell
    int voff[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int q = tid + r * JZ_THREADS;
        voff[r] = -1;
        if (q < JZ_VP) {
            const int gx = x0 - 2 + q % JZ_VX, gy = y0 - 2 + q / JZ_VX;
            if (gx <= nx + 1 && gy <= ny + 1) voff[r] = halo_coord(gx, nx, bc) + nx * halo_coord(gy, ny, bc);
        }
    }
    // ring slots: planes are visited in increasing order from z0 - 2, so the slot of a
    // plane is its distance from z0 - 2 modulo the ring size (no negative operands)
    auto vplane = [&](int plane) -> float * { return sv + (size_t)((plane - z0 + 2) % JZ_NV) * NF * JZ_VP; };
    auto splane = [&](int plane) -> float * { return sg + (size_t)((plane - z0 + 3) % 3) * (1 + NS) * JZ_SP; };
    auto load_plane = [&](int plane) {
        const float *src = v + (size_t)halo_coord(plane, nz, bc) * nxy;
        float *dst = vplane(plane);
#pragma unroll
        for (int r = 0; r < 2; r++)
            if (voff[r] >= 0) {
                const int q = tid + r * JZ_THREADS;
#pragma unroll
                for (int f = 0; f < NF; f++) cp_async4(dst + f * JZ_VP + q, src + (size_t)f * N + voff[r]);
            }
        cp_async_commit();
    };

    // stage 1: dG_c and sigma of plane zs on the 1-cell-halo tile
    auto stage1 = [&](int zs, float m) {
        const int zsrc = bc ? (zs < 0 ? 0 : (zs >= nz ? nz - 1 : zs)) : zs;  // plane whose values zs holds
        const int zg = halo_coord(zsrc, nz, 0);                                // its index in the grid
        const float *__restrict__ Vm = vplane(zsrc - 1), *__restrict__ V0 = vplane(zsrc),
                    *__restrict__ Vp = vplane(zsrc + 1);
        float *__restrict__ Sz = splane(zs);
        for (int q = tid; q < JZ_SP; q += JZ_THREADS) {
            const int gx = x0 - 1 + q % JZ_SX, gy = y0 - 1 + q / JZ_SX;
            if (gx > nx || gy > ny) continue;  // beyond a ragged tile: never read
            const int sx = bc ? (gx < 0 ? 0 : (gx >= nx ? nx - 1 : gx)) : gx;
            const int sy = bc ? (gy < 0 ? 0 : (gy >= ny ? ny - 1 : gy)) : gy;
            const int o = (sx - x0 + 2) + JZ_VX * (sy - y0 + 2);  // the source cell in the v tile
            const float v0 = V0[o], vc = v0 - m;
            float trd = 0.f;
            if constexpr (EL) {
                float Dd[3][3];
#pragma unroll
                for (int I = 0; I < 3; I++) {
                    const int fo = (KU + I) * JZ_VP + o;
                    Dd[I][0] = V0[fo + 1] - V0[fo - 1];
                    Dd[I][1] = V0[fo + JZ_VX] - V0[fo - JZ_VX];
                    Dd[I][2] = Vp[fo] - Vm[fo];
                }
                trd = Dd[0][0] + Dd[1][1] + Dd[2][2];
                const float common = c.b * trd - c.ls * vc;
#pragma unroll
                for (int I = 0; I < 3; I++) {
                    Sz[(1 + I) * JZ_SP + q] = c.ab * Dd[I][I] + common;
#pragma unroll
                    for (int J = I + 1; J < 3; J++) Sz[(1 + scomp(3, I, J)) * JZ_SP + q] = c.c4 * (Dd[I][J] + Dd[J][I]);
                }
            }
            if (c.mode == 0) {
                const int p = halo_coord(sx, nx, 0) + nx * (halo_coord(sy, ny, 0) + ny * zg);
                const float sn = V0[o + 1] + V0[o - 1] + V0[o + JZ_VX] + V0[o - JZ_VX] + Vp[o] + Vm[o];
                const float lc = sn - 6.f * v0;
                float dg = part[p] * vc;
#pragma unroll
                for (int j = 1; j <= NE; j++) dg += part[(size_t)j * N + p] * V0[j * JZ_VP + o];
                dg -= c.gc * lc;
                if constexpr (EL) dg += c.el_c * vc - c.el_t * trd;
                Sz[q] = dg;
            }
        }
    };

    // prologue: v planes z0-2 .. z0+2, stage 1 of planes z0-1 and z0
    for (int pl = z0 - 2; pl <= z0 + 2; pl++) load_plane(pl);
    cp_async_wait_all();
    __syncthreads();
    const float m = sm, idt = sidt;
    stage1(z0 - 1, m);
    stage1(z0, m);
    const float ih2 = c.ih2, ge = c.ge, i2h = c.i2h;
    const int txl = tid % JZ_TX, tyl = tid / JZ_TX;
    const int hq = (txl + 1) + JZ_SX * (tyl + 1), o = (txl + 2) + JZ_VX * (tyl + 2);
    const bool inxy = tid < JZ_TX * JZ_TY && x0 + txl < nx && y0 + tyl < ny;
    for (int z = z0; z < z1; z++) {
        cp_async_wait_all();  // v plane z + 2 (issued one iteration ago)
        __syncthreads();      // ... visible to all; stage 2 of plane z - 1 finished
        load_plane(z + 3);    // into the slot of plane z - 2, no longer read
        stage1(z + 1, m);     // into the ring slot of plane z - 2
        __syncthreads();
        // stage 2: J v on plane z
        if (inxy) {
            const float *__restrict__ Vm = vplane(z - 1), *__restrict__ V0 = vplane(z), *__restrict__ Vp = vplane(z + 1);
            const float *__restrict__ Sm = splane(z - 1), *__restrict__ S0 = splane(z), *__restrict__ Sp = splane(z + 1);
            const int c3[3] = {x0 + txl, y0 + tyl, z};
            const int nn[3] = {nx, ny, nz};
            const int p = c3[0] + nx * (c3[1] + ny * z);
            int im[3], ip[3];
            nbr_offsets<3>(c3, nn, p, im, ip, bc);
            const float vc = V0[o] - m;
            float ve[NE], je[NE], jc;
#pragma unroll
            for (int j = 0; j < NE; j++) ve[j] = V0[(1 + j) * JZ_VP + o];
            if (c.mode == 0) {
                const float G0 = S0[hq];
                const float gp[3] = {S0[hq + 1], S0[hq + JZ_SX], Sp[hq]};
                const float gm[3] = {S0[hq - 1], S0[hq - JZ_SX], Sm[hq]};
                float flux = 0.f;
#pragma unroll
                for (int J = 0; J < 3; J++) flux += mob[J * N + p] * (gp[J] - G0) - mob[J * N + im[J]] * (G0 - gm[J]);
                jc = vc * idt - flux * ih2;
#pragma unroll
                for (int j = 0; j < NE; j++) {
                    const int fo = (1 + j) * JZ_VP + o;
                    const float sn = V0[fo + 1] + V0[fo - 1] + V0[fo + JZ_VX] + V0[fo - JZ_VX] + Vp[fo] + Vm[fo];
                    const float *pr = part + (size_t)(1 + j) * KU * N + p;
                    if constexpr (NE == 1) {
                        je[j] = ve[j] * idt + pr[0] * vc + pr[N] * ve[j] - ge * (sn - 6.f * ve[j]);
                    } else {
                        float pw = pr[0] * vc;
#pragma unroll
                        for (int i = 0; i < NE; i++) pw += pr[(size_t)(1 + i) * N] * ve[i];
                        je[j] = ve[j] * idt + c.keta * pw - ge * (sn - 6.f * ve[j]);
                    }
                }
            } else {
                jc = vc;
#pragma unroll
                for (int j = 0; j < NE; j++) je[j] = ve[j];
            }
            Jv[p] = jc;
#pragma unroll
            for (int j = 0; j < NE; j++) Jv[(size_t)(1 + j) * N + p] = je[j];
            if constexpr (EL) {
                // the mirrored neighbour's stress enters with the opposite sign (Neumann)
#pragma unroll
                for (int I = 0; I < 3; I++) {
                    float div = 0.f;
#pragma unroll
                    for (int J = 0; J < 3; J++) {
                        const int k = (1 + scomp(3, I, J)) * JZ_SP + hq;
                        const float a = J == 0 ? S0[k + 1] : (J == 1 ? S0[k + JZ_SX] : Sp[k]);
                        const float bb = J == 0 ? S0[k - 1] : (J == 1 ? S0[k - JZ_SX] : Sm[k]);
                        div += (ip[J] == p ? -a : a) - (im[J] == p ? -bb : bb);
                    }
                    Jv[(size_t)(KU + I) * N + p] = div * i2h;
                }
            }
        }
    }
    cp_async_wait_all();  // no copy outlives the block
}

__device__ inline double Psi(double z) { return z * log(z) + (1.0 - z) * log1p(-z); }

// E_1 and E_2 densities of the model with three order parameters (App. A):
//   E_1 = dis(c) + a(c) S(eta) + b(c) T(eta), dis(c) = dE0 c + c(1-c) sum_i L_i (2c-1)^i,
//   a(c) = (4 U1 + 12 U4) c^2 - 24 U4 c^3, b(c) = -48 U4 c^3,
//   S = phi_1^2 + phi_2^2 + phi_3^2, T = phi_1 phi_2 phi_3 (phi of nks_model3.cuh);
//   E_2 = theta (w Psi(c) + 1/4 sum_{i=1..4} Psi(c eta_i)), eta_4 = 4 - sum
__device__ inline void energy12_3(const DCoef &k, double c, const double (&e)[3], double &e1, double &e2)
{
    const double s = 2.0 * c - 1.0;
    const double dis = k.dE0 * c + c * (1.0 - c) * (k.L[0] + s * (k.L[1] + s * (k.L[2] + s * k.L[3])));
    const double f0 = 1.0 - 0.5 * (e[0] + e[1]), f1 = 1.0 - 0.5 * (e[0] + e[2]), f2 = 1.0 - 0.5 * (e[1] + e[2]);
    const double c2 = c * c, c3 = c2 * c;
    const double a = (4.0 * k.U1 + 12.0 * k.U4) * c2 - 24.0 * k.U4 * c3, b = -48.0 * k.U4 * c3;
    e1 = dis + a * (f0 * f0 + f1 * f1 + f2 * f2) + b * (f0 * f1 * f2);
    const double e4 = 4.0 - e[0] - e[1] - e[2];
    e2 = k.theta * (k.w_psi * Psi(c) + 0.25 * (Psi(c * e[0]) + Psi(c * e[1]) + Psi(c * e[2]) + Psi(c * e4)));
}

// energy parts e1..e4 (Eq. relations) and mass, per-block partial sums
__global__ void __launch_bounds__(kRedThreads) k_energy(DGrid g, DCoef k, Bat bt, const double *__restrict__ isc,
                                                        const double *__restrict__ X, double *__restrict__ partials)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    X = shift(X, io);
    partials = shift(partials, io);
    const double cbar0 = shift(isc, io)[I_CBAR0];
    const long long N = g.N;
    const double ih = g.ih;
    double acc[5] = {0, 0, 0, 0, 0};
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
         p += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        coords_of(g, p, x, y, z);
        const double c = X[p];
        double e1, e2;
        if (k.ne == 3) {
            const double ee[3] = {X[N + p], X[2 * N + p], X[3 * N + p]};
            energy12_3(k, c, ee, e1, e2);
        } else {
            const double e = X[N + p], f = 1.0 - e;
            // E1 = Phi(c, phi): App. A with one order parameter
            const double s = 2.0 * c - 1.0;
            const double ex = c * (1.0 - c) * (k.L[0] + s * (k.L[1] + s * (k.L[2] + s * k.L[3])));
            e1 = k.dE0 * c + ex + 12.0 * k.U1 * c * c * f * f + 36.0 * k.U4 * (1.0 - 2.0 * c) * c * c * f * f -
                 48.0 * k.U4 * c * c * c * f * f * f;
            e2 = k.theta * (k.w_psi * Psi(c) + 0.75 * Psi(c * e) + 0.25 * Psi(c * (4.0 - 3.0 * e)));
        }
        double e3 = 0.0;
        if (k.elastic) {
            double Du[3][3];
            grad_u(g, X + (1 + k.ne) * N, x, y, z, Du);
            const double s0 = k.eps0 * (c - cbar0);
            double tr = 0.0, sq = 0.0, off = 0.0;
            for (int I = 0; I < g.dim; I++) {
                const double eII = Du[I][I] - s0;
                tr += eII;
                sq += eII * eII;
                for (int J = I + 1; J < g.dim; J++) {
                    const double eIJ = 0.5 * (Du[I][J] + Du[J][I]);
                    off += eIJ * eIJ;
                }
            }
            e3 = 0.5 * (k.C12 * tr * tr + (k.C11 - k.C12) * sq + 4.0 * k.C44 * off);
        }
        // E4: gamma_c/2 |D c|^2 + 3 gamma_eta/2 |D eta|^2, or gamma_eta/2 per eta_j (App. A)
        double gc = 0.0, ge = 0.0;
        for (int J = 0; J < g.dim; J++) {
            const long long pp = nbrJ(g, x, y, z, J, +1), pm = nbrJ(g, x, y, z, J, -1);
            const double dpc = (X[pp] - c) * ih, dmc = (c - X[pm]) * ih;
            gc += 0.5 * (dpc * dpc + dmc * dmc);
            for (int j = 0; j < k.ne; j++) {
                const long long o = (1 + j) * N;
                const double e = X[o + p];
                const double dpe = (X[o + pp] - e) * ih, dme = (e - X[o + pm]) * ih;
                ge += 0.5 * (dpe * dpe + dme * dme);
            }
        }
        acc[0] += e1;
        acc[1] += e2;
        acc[2] += e3;
        acc[3] += 0.5 * k.gamma_c * gc + (k.ne == 3 ? 0.5 : 1.5) * k.gamma_eta * ge;
        acc[4] += c;
    }
    block_reduce_store<5>(acc, partials);
}

// sums K columns of nblocks partial rows in a fixed order (one block)
__global__ void k_finalize(Bat bt, const double *__restrict__ partials, int nblocks, int K, double *__restrict__ out)
{
    long long io;
    if (!inst_off(bt, blockIdx.x, io)) return;
    partials = shift(partials, io);
    out = shift(out, io);
    __shared__ double red[kRedThreads];
    for (int kk = 0; kk < K; kk++) {
        double a = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += partials[(size_t)b * K + kk];
        red[threadIdx.x] = a;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[kk] = red[0];
        __syncthreads();
    }
}

}  // namespace

int launch_mobility(const DGrid &g, const DCoef &k, const double *c0, double *mob, cudaStream_t st, const Bat &bt)
{
    k_mobility<<<dim3(blocks_for(g.N), bt.nb), kThreads, 0, st>>>(g, k, bt, c0, mob);
    return 1;
}

int launch_trace0(const DGrid &g, const DCoef &k, const double *isc, const double *X0, double *tr0, cudaStream_t st,
                  const Bat &bt)
{
    k_trace0<<<dim3(blocks_for(g.N), bt.nb), kThreads, 0, st>>>(g, k, bt, isc, X0, tr0);
    return 1;
}

int launch_residual(const DGrid &g, const DCoef &k, const double *isc, int mode, const double *X1, const double *X0,
                    const double *tr0, const double *mob, double *Gc, double *sig, double *part, double *F, int *flag,
                    double *partials, int rb, cudaStream_t st, const Bat &bt)
{
    if (k.ne == 3)
        k_res_a<3><<<dim3(blocks_for(g.N), bt.nb), kThreads, 0, st>>>(g, k, bt, isc, mode, X1, X0, tr0, Gc, sig, part,
                                                                       F, flag);
    else
        k_res_a<1><<<dim3(blocks_for(g.N), bt.nb), kThreads, 0, st>>>(g, k, bt, isc, mode, X1, X0, tr0, Gc, sig, part,
                                                                       F, flag);
    k_res_b<<<dim3(rb, bt.nb), kRedThreads, 0, st>>>(g, k, bt, isc, mode, X1, X0, Gc, mob, sig, F, partials);
    return 2;
}

template <int D, bool EL, int NE>
static void launch_jv64_d(const DGrid &g, const JvConst<double> &c, const Bat &bt, const double *isc, const double *part,
                          const double *mob, const double *v, double *dG, double *sig, double *Jv, cudaStream_t st,
                          const double *zsum)
{
    const dim3 blk(D == 1 ? 256 : 32, D == 1 ? 1 : 8);
    const dim3 grd((g.n[0] + blk.x - 1) / blk.x, (g.n[1] + blk.y - 1) / blk.y, g.n[2] * bt.nb);
    k_jv64_a<D, EL, NE><<<grd, blk, 0, st>>>(g, c, bt, part, v, dG, sig, zsum);
    k_jv64_b<D, EL, NE><<<grd, blk, 0, st>>>(g, c, bt, isc, part, mob, v, dG, sig, Jv, zsum);
}

template <int D, bool EL, int NE>
static void launch_jv32_d(const DGrid &g, const JvConst<float> &c, const Bat &bt, const double *isc, const float *part,
                          const float *mob, const float *v, float *Jv, cudaStream_t st, const double *zsum)
{
    if constexpr (D == 3) {
        constexpr int NF = 1 + NE + (EL ? 3 : 0);
        const size_t smem = jv32z_smem<NF>(EL ? 6 : 1);  // limit set by prepare_jv32
        // planes per block: split each column into as many chunks as one wave of resident
        // blocks holds (each chunk forms two extra planes of dG and sigma)
        const long long cols = (long long)((g.n[0] + JZ_TX - 1) / JZ_TX) * ((g.n[1] + JZ_TY - 1) / JZ_TY) * bt.nb;
        const long long cap = (long long)std::max(1, JzOcc<EL, NE>::resident);
        const long long want = std::max(1LL, (cap + cols / 2) / cols);
        const int zc = std::max(4, (int)((g.n[2] + want - 1) / want));
        const long long tiles = cols / bt.nb * ((g.n[2] + zc - 1) / zc);
        k_jv32_z<EL, NE><<<dim3((unsigned)tiles, bt.nb), JZ_THREADS, smem, st>>>(g, c, bt, isc, part, mob, v, Jv, zsum,
                                                                                zc);
        return;
    }
    constexpr int TX = JvTile<D>::TX, TY = JvTile<D>::TY, TZ = JvTile<D>::TZ;
    const long long tiles = (long long)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY) * ((g.n[2] + TZ - 1) / TZ);
    k_jv32<D, EL, NE><<<dim3((unsigned)tiles, bt.nb), 256, 0, st>>>(g, c, bt, isc, part, mob, v, Jv, zsum);
}

// dimension, elasticity and order parameters (1 or 3)
#define NKS_JV_DISPATCH(FN, ...)                                      \
    switch ((k.ne == 3 ? 8 : 0) + g.dim * 2 + (k.elastic ? 1 : 0)) { \
    case 2: FN<1, false, 1>(__VA_ARGS__); break;                      \
    case 3: FN<1, true, 1>(__VA_ARGS__); break;                       \
    case 4: FN<2, false, 1>(__VA_ARGS__); break;                      \
    case 5: FN<2, true, 1>(__VA_ARGS__); break;                       \
    case 6: FN<3, false, 1>(__VA_ARGS__); break;                      \
    case 7: FN<3, true, 1>(__VA_ARGS__); break;                       \
    case 10: FN<1, false, 3>(__VA_ARGS__); break;                     \
    case 11: FN<1, true, 3>(__VA_ARGS__); break;                      \
    case 12: FN<2, false, 3>(__VA_ARGS__); break;                     \
    case 13: FN<2, true, 3>(__VA_ARGS__); break;                      \
    case 14: FN<3, false, 3>(__VA_ARGS__); break;                     \
    default: FN<3, true, 3>(__VA_ARGS__); break;                      \
    }

template <int D, bool EL, int NE>
static void prepare_jv32_d()
{
    if constexpr (D == 3) {
        constexpr int NF = 1 + NE + (EL ? 3 : 0);
        const int smem = (int)jv32z_smem<NF>(EL ? 6 : 1);
        cudaFuncSetAttribute(k_jv32_z<EL, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int per_sm = 0, nsm = 0, dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jv32_z<EL, NE>, JZ_THREADS, smem) == cudaSuccess)
            JzOcc<EL, NE>::resident = per_sm * nsm;  // otherwise one block: one chunk per column
    }
}

void prepare_jv32(const DGrid &g, const DCoef &k) { NKS_JV_DISPATCH(prepare_jv32_d); }

int launch_jv64(const DGrid &g, const DCoef &k, const double *isc, int mode, const double *part, const double *mob,
                const double *v, double *dG, double *sig, double *Jv, cudaStream_t st, const Bat &bt,
                const double *zsum)
{
    const JvConst<double> c = jv_const<double>(g, k, mode);
    NKS_JV_DISPATCH(launch_jv64_d, g, c, bt, isc, part, mob, v, dG, sig, Jv, st, zsum);
    return 2;
}

int launch_jv32(const DGrid &g, const DCoef &k, const double *isc, int mode, const float *part, const float *mob,
                const float *v, float *Jv, cudaStream_t st, const Bat &bt, const double *zsum)
{
    const JvConst<float> c = jv_const<float>(g, k, mode);
    NKS_JV_DISPATCH(launch_jv32_d, g, c, bt, isc, part, mob, v, Jv, st, zsum);
    return 1;
}

int launch_energy(const DGrid &g, const DCoef &k, const double *isc, const double *X, double *partials, int rb,
                  cudaStream_t st, const Bat &bt)
{
    k_energy<<<dim3(rb, bt.nb), kRedThreads, 0, st>>>(g, k, bt, isc, X, partials);
    return 1;
}

int launch_finalize(const double *partials, int nblocks, int K, double *out, cudaStream_t st, const Bat &bt)
{
    k_finalize<<<bt.nb, kRedThreads, 0, st>>>(bt, partials, nblocks, K, out);
    return 1;
}

}  // namespace nks
