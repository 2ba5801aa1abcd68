/*
 * nks_oracle.c -- plain, slow FP64 CPU oracle for the per-time-step
 * Newton-Krylov-Schwarz (NKS) solve of the semi-implicit discrete variational
 * derivative (DVD) scheme NSOA-1 of Huang & Yang, "Parallel energy stable
 * phase field simulations of Ni-based alloys system" (arXiv 2209.08001).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline / reference legs of the benchmark may load this library.  It
 * shares no source, header, table or helper with the CUDA path; the product
 * never calls it.
 *
 * Conventions (Sec. 3 and Sec. 4 of the paper):
 *   - cell-centred grid, periodic (or homogeneous Neumann: mirror ghost cells),
 *     points numbered x-fastest, p = x + nx*(y + ny*z);
 *   - unknowns point-interleaved, X = (c_1, eta_1, u_1.., c_2, eta_2, u_2.., ...)
 *     (Sec. 4: "the unknown X is organized by points");
 *   - fields per point: c, eta and, when elasticity is on, the d displacement
 *     components u_1..u_d; with three order parameters (App. A, n_eta = 3)
 *     c, eta_1, eta_2, eta_3, then u_1..u_d;
 *   - loops over independent points, rows, subdomains or vector entries are
 *     shared among the host's threads (OpenMP); each thread computes whole
 *     points or rows exactly as the serial loop would;
 *   - every sum over points or vector entries is taken in fixed blocks of
 *     ORC_SUM_BLOCK consecutive terms, each block added in index order, then the
 *     block sums added in block order, so every result is the same for any
 *     number of threads; nothing else is blocked or fused.
 *
 * The readings of passages the paper leaves open (tolerances, line search,
 * projection of the Krylov corrections, the elastic gauge, ...) are stated at
 * each function.
 */
#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#undef I /* complex.h's imaginary unit: _Complex_I is used by name, I stays an axis index */

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by ctypes in oracle/__init__.py)              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int dim;      /* d = 1, 2 or 3                                           */
    int n[3];     /* cells per axis; n[J] = 1 for J >= dim                   */
    double h;     /* mesh size, equal on every axis                          */
    int neumann;  /* 0: periodic; 1: homogeneous Neumann (Eq. boundaryequ) on the
                     cell-centred grid of Sec. 3: the ghost cell beyond a boundary
                     cell mirrors it, so D^+ / D^- across the boundary face vanish
                     and the flux form has no boundary flux; the displacement rows
                     are the exact variation of the discrete elastic energy (its
                     natural boundary condition is the traction-free one)        */
} orc_grid;

typedef struct {
    double kappa;     /* mobility parameter: M = kappa c (1 - c)    (Eq. CHGL) */
    double gamma_c;   /* gradient coefficient of c        (Eq. simple free energy-1) */
    double gamma_eta; /* gradient coefficient of eta (enters as 3 gamma_eta)  */
    double theta;     /* RT / (V_m dE), weight of the logarithmic terms        */
    double w_psi;     /* weight of theta Psi(c) in E_2 (main text: 1)          */
    double dE0;       /* (E0_Al - E0_Ni) / (V_m dE), App. A                    */
    double L[4];      /* L_0..L_3 / (V_m dE), App. A excess energy             */
    double U1, U4;    /* U_1, U_4 / (V_m dE), App. A ordering energy           */
    double eps0;      /* composition expansion coefficient of the lattice      */
    double C11, C12, C44; /* dimensionless cubic Hooke constants (x Lscale)    */
    int S;            /* Taylor order of Psi_S (Sec. 3); S <= 0: exact quotient */
    int n_eta;        /* order parameters: 1 (the reduced model of the main text) or
                         3 (App. A: eta_1..eta_3, eta_4 = 4 - sum); 0 reads as 1      */
} orc_coeffs;

typedef struct {
    double newton_rtol, newton_atol;   /* eps_r, eps_a (Sec. 4)            */
    int newton_maxit;
    double ls_alpha, ls_lambda_min;    /* backtracking line search          */
    int gmres_restart, gmres_maxit;
    double gmres_rtol, gmres_atol;     /* xi_r, xi_a (Sec. 4)               */
    int sub[3];                        /* subdomains per axis               */
    int overlap;                       /* delta, layers per side            */
    int subsolver;                     /* 0 ILU(0), 1 dense LU              */
    int reuse;                         /* 1: factor once per time step      */
    int project;                       /* 1: apply the projection P         */
    double dt_init, dt_min, dt_max, zeta;
    int dt_mode;                       /* 0 fixed, 1 solution change, 2 energy change */
    int zeta_persist;                  /* 1: zeta doublings persist         */
    int max_retries;
    double u0_rtol, u0_atol;
    int u0_maxit;
    int variant;                       /* Schwarz type (Sec. 4, Table 2): 0 left-RAS,
                                          1 classical AS, 2 right-RAS                */
} orc_opts;

typedef struct {
    double dt, t, energy, mass, fnorm0, fnorm;
    int retries, newton_its, gmres_its, status;
} orc_step_info;

enum { ORC_OK = 0, ORC_EDOMAIN = 2, ORC_EDIVERGED = 4, ORC_EPIVOT = 7, ORC_EINVAL = 1 };

/* ------------------------------------------------------------------------ */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static long grid_N(const orc_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static double cell_volume(const orc_grid *g)
{
    double v = 1.0;
    for (int J = 0; J < g->dim; J++) v *= g->h;
    return v;
}

/* periodic neighbour of point p shifted by s cells along axis J */
static long nbr(const orc_grid *g, long p, int J, int s)
{
    long n0 = g->n[0], n1 = g->n[1];
    long x[3];
    x[0] = p % n0;
    x[1] = (p / n0) % n1;
    x[2] = p / (n0 * n1);
    long nJ = g->n[J];
    if (g->neumann) {
        /* mirror ghost: beyond the boundary the neighbour is the cell itself */
        long y = x[J] + s;
        if (y < 0 || y >= nJ) return p;
        x[J] = y;
        return x[0] + n0 * (x[1] + n1 * x[2]);
    }
    x[J] = ((x[J] + s) % nJ + nJ) % nJ;
    return x[0] + n0 * (x[1] + n1 * x[2]);
}

static void coords(const orc_grid *g, long p, long x[3])
{
    x[0] = p % g->n[0];
    x[1] = (p / g->n[0]) % g->n[1];
    x[2] = p / ((long)g->n[0] * g->n[1]);
}

/* host threads the parallel loops use (1 without OpenMP) */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following parallel loops: n >= 1, or n <= 0 for all processors */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Sums in a fixed order (independent of the thread count)                   */
/* ------------------------------------------------------------------------ */

#define ORC_SUM_BLOCK 4096

static long n_blocks(long n) { return (n + ORC_SUM_BLOCK - 1) / ORC_SUM_BLOCK; }

/* sum of the block sums part[0..nb-1], in block order */
static double sum_parts(const double *part, long nb)
{
    double s = 0.0;
    for (long q = 0; q < nb; q++) s += part[q];
    return s;
}

/* sum_i a[i * stride] */
static double strided_sum(long n, const double *a, long stride)
{
    long nb = n_blocks(n);
    double *part = (double *)malloc(sizeof(double) * (nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
    for (long q = 0; q < nb; q++) {
        long i1 = (q + 1) * ORC_SUM_BLOCK < n ? (q + 1) * ORC_SUM_BLOCK : n;
        double s = 0.0;
        for (long i = q * ORC_SUM_BLOCK; i < i1; i++) s += a[i * stride];
        part[q] = s;
    }
    double s = sum_parts(part, nb);
    free(part);
    return s;
}

static int is_elastic(const orc_coeffs *k) { return k->C11 != 0.0 || k->C12 != 0.0 || k->C44 != 0.0; }
static int n_eta(const orc_coeffs *k) { return k->n_eta == 3 ? 3 : 1; }
/* per point: c, the order parameters, then (with elasticity) u_1..u_d from field ufield(k) */
static int ufield(const orc_coeffs *k) { return 1 + n_eta(k); }

int orc_nfields(const orc_grid *g, const orc_coeffs *k) { return ufield(k) + (is_elastic(k) ? g->dim : 0); }

/* ------------------------------------------------------------------------ */
/* Free energy (Sec. 2, App. A) and its discrete form (Sec. 3, Eq. relations) */
/* ------------------------------------------------------------------------ */

/* Psi(z) = z ln z + (1 - z) ln(1 - z)  (Sec. 2, after the E_G definition) */
static double Psi(double z) { return z * log(z) + (1.0 - z) * log(1.0 - z); }

/* Psi'(z) = ln z - ln(1 - z) */
static double dPsi(double z) { return log(z) - log(1.0 - z); }

/*
 * Polynomial part Phi(c, phi) of the Gibbs energy, phi = 1 - eta, obtained from
 * App. A with eta_1 = eta_2 = eta_3 = eta (so phi_1 = phi_2 = phi_3 = phi and
 * sum_i phi_i^2 = 3 phi^2), scaled by 1/(V_m dE):
 *   E^dis_0 + excess:  dE0 c + c(1-c) sum_i L_i (2c-1)^i     (constant E0_Ni dropped)
 *   E^ord_0:           6 U1 c^2 sum phi_i^2
 *   excess of E^ord:  -2 U1 c^2 sum phi_i^2 + 12 U4 (1-2c) c^2 sum phi_i^2
 *                     - 48 U4 c^3 phi_1 phi_2 phi_3
 *   minus E^ord(c,1,1,1), whose polynomial part is zero (phi_i = 0 there).
 */
static double Phi_poly(const orc_coeffs *k, double c, double phi)
{
    double s = 2.0 * c - 1.0;
    double dis = k->dE0 * c + c * (1.0 - c) * (k->L[0] + k->L[1] * s + k->L[2] * s * s + k->L[3] * s * s * s);
    double sum_phi2 = 3.0 * phi * phi;
    double ord = 6.0 * k->U1 * c * c * sum_phi2
               - 2.0 * k->U1 * c * c * sum_phi2
               + 12.0 * k->U4 * (1.0 - 2.0 * c) * c * c * sum_phi2
               - 48.0 * k->U4 * c * c * c * phi * phi * phi;
    return dis + ord;
}

/* E_2 = theta { w Psi(c) + 3/4 Psi(c eta) + 1/4 Psi(c (4 - 3 eta)) }  (Eq. neq:01) */
static double E2_density(const orc_coeffs *k, double c, double eta)
{
    return k->theta * (k->w_psi * Psi(c) + 0.75 * Psi(c * eta) + 0.25 * Psi(c * (4.0 - 3.0 * eta)));
}

/* discrete elastic strain at point p (Sec. 3):
 *   eps_IJ = (Dhat_J u_I + Dhat_I u_J)/2,  eps^el = eps - eps0 (c - cbar0) I,
 * with the centred difference Dhat (neighbours i-1, i+1). */
static void el_strain(const orc_grid *g, const orc_coeffs *k, int nf, double cbar0,
                      const double *X, long p, double e[3][3])
{
    int d = g->dim;
    double h = g->h;
    double Du[3][3] = {{0}};
    for (int I = 0; I < d; I++)
        for (int J = 0; J < d; J++)
            Du[I][J] = (X[nbr(g, p, J, +1) * nf + ufield(k) + I] - X[nbr(g, p, J, -1) * nf + ufield(k) + I]) / (2.0 * h);
    double c = X[p * nf + 0];
    for (int I = 0; I < 3; I++)
        for (int J = 0; J < 3; J++) e[I][J] = 0.0;
    for (int I = 0; I < d; I++)
        for (int J = 0; J < d; J++)
            e[I][J] = 0.5 * (Du[I][J] + Du[J][I]) - (I == J ? k->eps0 * (c - cbar0) : 0.0);
}

/* cubic Hooke law: sigma_II = C11 e_II + C12 sum_{K != I} e_KK, sigma_IJ = 2 C44 e_IJ */
static void hooke(const orc_coeffs *k, int d, double e[3][3], double s[3][3])
{
    double tr = 0.0;
    for (int I = 0; I < d; I++) tr += e[I][I];
    for (int I = 0; I < 3; I++)
        for (int J = 0; J < 3; J++) s[I][J] = 0.0;
    for (int I = 0; I < d; I++) {
        s[I][I] = k->C11 * e[I][I] + k->C12 * (tr - e[I][I]);
        for (int J = 0; J < d; J++)
            if (J != I) s[I][J] = 2.0 * k->C44 * e[I][J];
    }
}

/* elastic energy density, App. A (Eq. elastic-energy):
 *   1/2 ( C12 (sum e_II)^2 + (C11 - C12) sum e_II^2 + 4 C44 sum_{I<J} e_IJ^2 ) */
static double E3_density(const orc_coeffs *k, int d, double e[3][3])
{
    double tr = 0.0, sq = 0.0, off = 0.0;
    for (int I = 0; I < d; I++) {
        tr += e[I][I];
        sq += e[I][I] * e[I][I];
        for (int J = I + 1; J < d; J++) off += e[I][J] * e[I][J];
    }
    return 0.5 * (k->C12 * tr * tr + (k->C11 - k->C12) * sq + 4.0 * k->C44 * off);
}

/* discrete energy Ẽ = sum_i (E1 + E2 + E3 + E4) h^d  (Eq. relations, Eq. freeenergy);
 * E4 = gamma_c/2 [(D^pm c)^2] + 3 gamma_eta/2 [(D^pm eta)^2] with
 * [(D^pm f)^2] = ((D^+ f)^2 + (D^- f)^2)/2 summed over the d axes.
 * parts (optional) receives the four sums times h^d. */
static void E12_density3(const orc_coeffs *k, double c, const double e[3], double *e1, double *e2);

/* the four energy densities e1..e4 of point p */
static void energy_point(const orc_grid *g, const orc_coeffs *k, double cbar0, const double *X, long p, double e4[4])
{
    int nf = orc_nfields(g, k), d = g->dim;
    double h = g->h;
    e4[0] = e4[1] = e4[2] = e4[3] = 0.0;
    if (n_eta(k) == 3) {
        /* three order parameters: E_1, E_2 of App. A, E_4 with gamma_eta/2 per eta_j */
        double c = X[p * nf], e[3] = {X[p * nf + 1], X[p * nf + 2], X[p * nf + 3]}, a, b;
        E12_density3(k, c, e, &a, &b);
        e4[0] = a;
        e4[1] = b;
        if (is_elastic(k)) {
            double ee[3][3];
            el_strain(g, k, nf, cbar0, X, p, ee);
            e4[2] = E3_density(k, d, ee);
        }
        for (int f = 0; f < 4; f++) {
            double gs = 0.0, v0 = X[p * nf + f];
            for (int J = 0; J < d; J++) {
                double dp = (X[nbr(g, p, J, +1) * nf + f] - v0) / h, dm = (v0 - X[nbr(g, p, J, -1) * nf + f]) / h;
                gs += 0.5 * (dp * dp + dm * dm);
            }
            e4[3] += 0.5 * (f == 0 ? k->gamma_c : k->gamma_eta) * gs;
        }
        return;
    }
    double c = X[p * nf], eta = X[p * nf + 1];
    e4[0] = Phi_poly(k, c, 1.0 - eta);
    e4[1] = E2_density(k, c, eta);
    if (is_elastic(k)) {
        double e[3][3];
        el_strain(g, k, nf, cbar0, X, p, e);
        e4[2] = E3_density(k, d, e);
    }
    double gc = 0.0, ge = 0.0;
    for (int J = 0; J < d; J++) {
        long pp = nbr(g, p, J, +1), pm = nbr(g, p, J, -1);
        double dpc = (X[pp * nf] - c) / h, dmc = (c - X[pm * nf]) / h;
        double dpe = (X[pp * nf + 1] - eta) / h, dme = (eta - X[pm * nf + 1]) / h;
        gc += 0.5 * (dpc * dpc + dmc * dmc);
        ge += 0.5 * (dpe * dpe + dme * dme);
    }
    e4[3] = 0.5 * k->gamma_c * gc + 1.5 * k->gamma_eta * ge;
}

double orc_energy(const orc_grid *g, const orc_coeffs *k, double cbar0, const double *X, double *parts)
{
    long N = grid_N(g), nb = n_blocks(N);
    double *part = (double *)malloc(sizeof(double) * 4 * (nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
    for (long q = 0; q < nb; q++) {
        long p1 = (q + 1) * ORC_SUM_BLOCK < N ? (q + 1) * ORC_SUM_BLOCK : N;
        double a[4] = {0.0, 0.0, 0.0, 0.0}, e4[4];
        for (long p = q * ORC_SUM_BLOCK; p < p1; p++) {
            energy_point(g, k, cbar0, X, p, e4);
            for (int t = 0; t < 4; t++) a[t] += e4[t];
        }
        for (int t = 0; t < 4; t++) part[t * nb + q] = a[t];
    }
    double s1 = sum_parts(part, nb), s2 = sum_parts(part + nb, nb), s3 = sum_parts(part + 2 * nb, nb),
           s4 = sum_parts(part + 3 * nb, nb);
    free(part);
    double v = cell_volume(g);
    if (parts) {
        parts[0] = s1 * v;
        parts[1] = s2 * v;
        parts[2] = s3 * v;
        parts[3] = s4 * v;
    }
    return (s1 + s2 + s3 + s4) * v;
}

/* mass <c> = sum_i c_i h^d  (Theorem 3.1) */
double orc_mass(const orc_grid *g, const orc_coeffs *k, const double *X)
{
    int nf = orc_nfields(g, k);
    return strided_sum(grid_N(g), X, nf) * cell_volume(g);
}

/* ------------------------------------------------------------------------ */
/* Discrete variational derivative G (Sec. 3, App. B)                        */
/* ------------------------------------------------------------------------ */

/*
 * Taylor-truncated first-order quotient Psi_S[y1, y2] (Sec. 3, before Eq. D2-1):
 *   Psi_S(y, delta) = Psi(y) + sum_{s=1}^{2S} delta^s Psi^(s)(y)/s!,
 *   Psi_S[y1, y2]   = (Psi_S(ybar, delta) - Psi_S(ybar, -delta)) / (2 delta),
 * ybar = (y1 + y2)/2, delta = (y2 - y1)/2.  Only odd s survive; with
 * Psi^(2k+1)(z) = (2k-1)! ( (1-z)^(-2k) - z^(-2k) ) for k >= 1 this is
 *   Psi'(ybar) + sum_{k=1}^{S-1} [ (delta/(1-ybar))^(2k) - (delta/ybar)^(2k) ] / (2k (2k+1)).
 * S <= 0 selects the exact quotient (Psi(y1) - Psi(y2))/(y1 - y2) of Eq. D2.
 */
double orc_psi_quot(double y1, double y2, int S)
{
    if (S <= 0) {
        if (y1 == y2) return dPsi(y1);
        return (Psi(y1) - Psi(y2)) / (y1 - y2);
    }
    double yb = 0.5 * (y1 + y2), de = 0.5 * (y2 - y1);
    double a2 = (de / (1.0 - yb)) * (de / (1.0 - yb));
    double b2 = (de / yb) * (de / yb);
    double q = dPsi(yb);
    double ak = 1.0, bk = 1.0;
    for (int kk = 1; kk <= S - 1; kk++) {
        ak *= a2;
        bk *= b2;
        q += (ak - bk) / (2.0 * kk * (2.0 * kk + 1.0));
    }
    return q;
}

/* partial derivative of Psi_S[y1, y2] with respect to its first argument:
 * d/dy1 = 1/2 dg/dybar - 1/2 dg/ddelta with
 *   dg/dybar  = Psi''(ybar) + sum_k [ a^(2k)/(1-ybar) + b^(2k)/ybar ] / (2k+1),
 *   dg/ddelta = sum_k [ a^(2k-1)/(1-ybar) - b^(2k-1)/ybar ] / (2k+1),
 * a = delta/(1-ybar), b = delta/ybar. */
double orc_psi_quot_d1(double y1, double y2, int S)
{
    double yb = 0.5 * (y1 + y2), de = 0.5 * (y2 - y1);
    double a = de / (1.0 - yb), b = de / yb;
    double gy = 1.0 / yb + 1.0 / (1.0 - yb);
    double gd = 0.0;
    double apow = 1.0, bpow = 1.0; /* a^(2k-2), b^(2k-2) */
    for (int kk = 1; kk <= S - 1; kk++) {
        double aodd = apow * a, bodd = bpow * b;
        double aev = aodd * a, bev = bodd * b;
        gy += (aev / (1.0 - yb) + bev / yb) / (2.0 * kk + 1.0);
        gd += (aodd / (1.0 - yb) - bodd / yb) / (2.0 * kk + 1.0);
        apow = aev;
        bpow = bev;
    }
    return 0.5 * gy - 0.5 * gd;
}

/* App. B coefficient functions, all already divided by V_m dE */
static double M0c(const orc_coeffs *k) { return k->dE0 + (k->L[0] - k->L[1] + k->L[2] - k->L[3]); }
static double M1f(const orc_coeffs *k, double phi)
{
    return -(2.0 * k->L[0] - 6.0 * k->L[1] + 10.0 * k->L[2] - 14.0 * k->L[3]) + 24.0 * k->U1 * phi * phi + 72.0 * k->U4 * phi * phi;
}
static double M2f(const orc_coeffs *k, double phi)
{
    return -(6.0 * k->L[1] - 24.0 * k->L[2] + 54.0 * k->L[3]) - 216.0 * k->U4 * phi * phi - 144.0 * k->U4 * phi * phi * phi;
}
static double M3c(const orc_coeffs *k) { return -(16.0 * k->L[2] - 80.0 * k->L[3]); }
static double M4c(const orc_coeffs *k) { return -40.0 * k->L[3]; }
static double M5f(const orc_coeffs *k, double c) { return -(24.0 * k->U1 * c * c + 72.0 * k->U4 * (1.0 - 2.0 * c) * c * c); }
static double M6f(const orc_coeffs *k, double c) { return 144.0 * k->U4 * c * c * c; }

/* (a^n - b^n)/(a - b) written as its polynomial expansion sum_j a^j b^(n-1-j) */
static double quotpow(double a, double b, int n)
{
    double s = 0.0;
    for (int j = 0; j < n; j++) s += pow(a, j) * pow(b, n - 1 - j);
    return s;
}

/* G^1 (App. B), the polynomial part: returns (G1_c, G1_eta) at one point. */
static void G1_point(const orc_coeffs *k, double c1, double e1, double c0, double e0, double *gc, double *ge)
{
    double f1 = 1.0 - e1, f0 = 1.0 - e0;
    double ch = 0.5 * (c1 + c0), fh = 0.5 * (f1 + f0);
    *gc = (M1f(k, f0) + M1f(k, f1)) / 2.0 * ch
        + (M2f(k, f0) + M2f(k, f1)) / 6.0 * quotpow(c1, c0, 3)
        + M3c(k) / 4.0 * quotpow(c1, c0, 4)
        + M4c(k) / 5.0 * quotpow(c1, c0, 5)
        + M0c(k);
    *ge = (M5f(k, c0) + M5f(k, c1)) / 2.0 * fh
        + (M6f(k, c0) + M6f(k, c1)) / 6.0 * quotpow(f1, f0, 3);
}

/* G^{2,S} (Eq. D2-1), or G^2 (Eq. D2) when S <= 0, at one point:
 *   p = c eta, q = c (4 - 3 eta),
 *   G_c   = theta/4 [ 4 w Psi[c] + 3 eta_h Psi[p] + (4 - 3 eta)_h Psi[q] ],
 *   G_eta = theta/4 * 3 c_h ( Psi[p] - Psi[q] ). */
static void G2_point(const orc_coeffs *k, double c1, double e1, double c0, double e0, double *gc, double *ge)
{
    double p1 = c1 * e1, p0 = c0 * e0, q1 = c1 * (4.0 - 3.0 * e1), q0 = c0 * (4.0 - 3.0 * e0);
    double Qc = orc_psi_quot(c1, c0, k->S), Qp = orc_psi_quot(p1, p0, k->S), Qq = orc_psi_quot(q1, q0, k->S);
    double eh = 0.5 * (e1 + e0), ch = 0.5 * (c1 + c0);
    *gc = k->theta / 4.0 * (4.0 * k->w_psi * Qc + 3.0 * eh * Qp + (4.0 - 3.0 * eh) * Qq);
    *ge = k->theta / 4.0 * 3.0 * ch * (Qp - Qq);
}

/* ------------------------------------------------------------------------ */
/* Three order parameters (App. A): eta_1, eta_2, eta_3 and eta_4 = 4 - sum  */
/* ------------------------------------------------------------------------ */

/*
 * Gibbs energy of App. A with the four sublattice site fractions c eta_i
 * (scaled by 1/(V_m dE) as the reduced model):
 *   E_1 = dis(c) + a(c) S(eta) + b(c) T(eta),
 *     dis(c) = dE0 c + c(1-c) sum_i L_i (2c-1)^i,
 *     a(c)   = 6 U1 c^2 - 2 U1 c^2 + 12 U4 (1-2c) c^2,   b(c) = -48 U4 c^3,
 *     S = phi_1^2 + phi_2^2 + phi_3^2,  T = phi_1 phi_2 phi_3,
 *     phi_1 = 1 - (eta_1+eta_2)/2, phi_2 = 1 - (eta_1+eta_3)/2, phi_3 = 1 - (eta_2+eta_3)/2;
 *   E_2 = theta { w Psi(c) + 1/4 sum_{i=1..4} Psi(c eta_i) };
 *   E_4 = gamma_c/2 |grad c|^2 + gamma_eta/2 sum_{i=1..3} |grad eta_i|^2.
 * With eta_1 = eta_2 = eta_3 = eta these are the reduced model's E_1, E_2, E_4.
 *
 * Discrete variational derivative (reading: the reduced scheme of Sec. 3 /
 * App. B extended so that the discrete chain rule holds term by term):
 *   a product f(c) g(eta) splits symmetrically,
 *     G_c      += f[c1, c0] (g(eta^0) + g(eta^1))/2,
 *     G_eta_j  += (f(c0) + f(c1))/2 g_j[eta^0, eta^1],
 *   with f[c1, c0] = int_0^1 f'(c0 + s (c1 - c0)) ds (the polynomial quotient) and
 *   g_j the average-vector-field discrete gradient int_0^1 dg/deta_j(eta^0 + s (eta^1 - eta^0)) ds,
 *   both exact here with 3-point Gauss-Legendre (integrands of degree <= 4);
 *   the logarithms use the Psi_S quotients of Sec. 3 with p_i = c eta_i:
 *     G_c     += theta/4 [ 4 w Psi_S[c] + sum_{i=1..4} (eta_i)_h Psi_S[p_i] ],
 *     G_eta_j += theta/4 c_h ( Psi_S[p_j] - Psi_S[p_4] );
 *   G^4: G_c = -gamma_c D^2 c_h, G_eta_j = -gamma_eta D^2 (eta_j)_h; G^3 as before.
 * For eta_1 = eta_2 = eta_3 this gives the reduced G_c and sum_j G_eta_j = G_eta.
 * The Allen-Cahn rows take the kinetic factor 3, F_eta_j = (eta_j^1 - eta_j^0)/dt
 * + 3 G_eta_j (reading: the reduced model's eta equation is then the symmetric
 * solution of this one, whose order parameters stay equal).
 *
 * The pointwise functions are written in complex arithmetic so that the
 * Jacobian's pointwise block is their complex-step derivative (Im f(x + i t)/t,
 * exact to rounding, no difference quotient); that needs the Taylor form of
 * Psi_S (S > 0).
 */
typedef double complex cplx;

static const double kEtaKinetic3 = 3.0;

static void gauss3(double t[3], double w[3])
{
    const double r = sqrt(0.6);
    t[0] = 0.5 - 0.5 * r;
    t[1] = 0.5;
    t[2] = 0.5 + 0.5 * r;
    w[0] = 5.0 / 18.0;
    w[1] = 8.0 / 18.0;
    w[2] = 5.0 / 18.0;
}

static cplx dis3(const orc_coeffs *k, cplx c)
{
    cplx s = 2.0 * c - 1.0;
    return k->dE0 * c + c * (1.0 - c) * (k->L[0] + k->L[1] * s + k->L[2] * s * s + k->L[3] * s * s * s);
}
static cplx dis3_d(const orc_coeffs *k, cplx c)
{
    cplx s = 2.0 * c - 1.0;
    cplx P = k->L[0] + k->L[1] * s + k->L[2] * s * s + k->L[3] * s * s * s;
    cplx dP = k->L[1] + 2.0 * k->L[2] * s + 3.0 * k->L[3] * s * s;
    return k->dE0 + (1.0 - 2.0 * c) * P + c * (1.0 - c) * 2.0 * dP;
}
static cplx a3(const orc_coeffs *k, cplx c) { return 6.0 * k->U1 * c * c - 2.0 * k->U1 * c * c + 12.0 * k->U4 * (1.0 - 2.0 * c) * c * c; }
static cplx a3_d(const orc_coeffs *k, cplx c) { return 8.0 * k->U1 * c + 12.0 * k->U4 * (2.0 * c - 6.0 * c * c); }
static cplx b3(const orc_coeffs *k, cplx c) { return -48.0 * k->U4 * c * c * c; }
static cplx b3_d(const orc_coeffs *k, cplx c) { return -144.0 * k->U4 * c * c; }

static void phi3(const cplx e[3], cplx f[3])
{
    f[0] = 1.0 - 0.5 * (e[0] + e[1]);
    f[1] = 1.0 - 0.5 * (e[0] + e[2]);
    f[2] = 1.0 - 0.5 * (e[1] + e[2]);
}
static cplx S3(const cplx e[3])
{
    cplx f[3];
    phi3(e, f);
    return f[0] * f[0] + f[1] * f[1] + f[2] * f[2];
}
static cplx T3(const cplx e[3])
{
    cplx f[3];
    phi3(e, f);
    return f[0] * f[1] * f[2];
}
/* dS/deta_j and dT/deta_j */
static void dST3(const cplx e[3], cplx dS[3], cplx dT[3])
{
    cplx f[3];
    phi3(e, f);
    dS[0] = -(f[0] + f[1]);
    dS[1] = -(f[0] + f[2]);
    dS[2] = -(f[1] + f[2]);
    dT[0] = -0.5 * f[2] * (f[0] + f[1]);
    dT[1] = -0.5 * f[1] * (f[0] + f[2]);
    dT[2] = -0.5 * f[0] * (f[1] + f[2]);
}

static cplx Psi_cx(cplx z) { return z * clog(z) + (1.0 - z) * clog(1.0 - z); }
static cplx dPsi_cx(cplx z) { return clog(z) - clog(1.0 - z); }

/* Psi_S[y1, y2] of Sec. 3 (as orc_psi_quot) in complex arithmetic */
static cplx psi_quot_cx(cplx y1, cplx y2, int S)
{
    if (S <= 0) {
        if (creal(y1) == creal(y2) && cimag(y1) == cimag(y2)) return dPsi_cx(y1);
        return (Psi_cx(y1) - Psi_cx(y2)) / (y1 - y2);
    }
    cplx yb = 0.5 * (y1 + y2), de = 0.5 * (y2 - y1);
    cplx a2 = (de / (1.0 - yb)) * (de / (1.0 - yb));
    cplx b2 = (de / yb) * (de / yb);
    cplx q = dPsi_cx(yb);
    cplx ak = 1.0, bk = 1.0;
    for (int kk = 1; kk <= S - 1; kk++) {
        ak *= a2;
        bk *= b2;
        q += (ak - bk) / (2.0 * kk * (2.0 * kk + 1.0));
    }
    return q;
}

/* pointwise G^1 (which & 1) + G^{2,S} (which & 2): out = (G_c, G_eta_1, G_eta_2, G_eta_3) */
static void G3_point(const orc_coeffs *k, int which, cplx c1, const cplx e1[3], cplx c0, const cplx e0[3], cplx out[4])
{
    for (int a = 0; a < 4; a++) out[a] = 0.0;
    if (which & 1) {
        double t[3], w[3];
        gauss3(t, w);
        cplx qd = 0.0, qa = 0.0, qb = 0.0, Sj[3] = {0, 0, 0}, Tj[3] = {0, 0, 0};
        for (int i = 0; i < 3; i++) {
            cplx c = c0 + t[i] * (c1 - c0), e[3], dS[3], dT[3];
            for (int j = 0; j < 3; j++) e[j] = e0[j] + t[i] * (e1[j] - e0[j]);
            qd += w[i] * dis3_d(k, c);
            qa += w[i] * a3_d(k, c);
            qb += w[i] * b3_d(k, c);
            dST3(e, dS, dT);
            for (int j = 0; j < 3; j++) {
                Sj[j] += w[i] * dS[j];
                Tj[j] += w[i] * dT[j];
            }
        }
        out[0] += qd + qa * 0.5 * (S3(e0) + S3(e1)) + qb * 0.5 * (T3(e0) + T3(e1));
        cplx am = 0.5 * (a3(k, c0) + a3(k, c1)), bm = 0.5 * (b3(k, c0) + b3(k, c1));
        for (int j = 0; j < 3; j++) out[1 + j] += am * Sj[j] + bm * Tj[j];
    }
    if (which & 2) {
        cplx e14 = 4.0 - e1[0] - e1[1] - e1[2], e04 = 4.0 - e0[0] - e0[1] - e0[2];
        cplx E1[4] = {e1[0], e1[1], e1[2], e14}, E0[4] = {e0[0], e0[1], e0[2], e04};
        cplx Q[4];
        for (int i = 0; i < 4; i++) Q[i] = psi_quot_cx(c1 * E1[i], c0 * E0[i], k->S);
        cplx ch = 0.5 * (c1 + c0), t4 = k->theta / 4.0;
        cplx gc = 4.0 * k->w_psi * psi_quot_cx(c1, c0, k->S);
        for (int i = 0; i < 4; i++) gc += 0.5 * (E1[i] + E0[i]) * Q[i];
        out[0] += t4 * gc;
        for (int j = 0; j < 3; j++) out[1 + j] += t4 * ch * (Q[j] - Q[3]);
    }
}

/* E_1 + E_2 densities of the three-parameter model at one point */
static void E12_density3(const orc_coeffs *k, double c, const double e[3], double *e1, double *e2)
{
    cplx ec[3] = {e[0], e[1], e[2]};
    *e1 = creal(dis3(k, c) + a3(k, c) * S3(ec) + b3(k, c) * T3(ec));
    double s = k->w_psi * creal(Psi_cx(c));
    double e4 = 4.0 - e[0] - e[1] - e[2];
    for (int i = 0; i < 3; i++) s += 0.25 * creal(Psi_cx(c * e[i]));
    s += 0.25 * creal(Psi_cx(c * e4));
    *e2 = k->theta * s;
}

/* pointwise derivatives d(G_c, G_eta_j)/d(c1, eta_1..3) (row-major 4 x 4) by complex step */
static void G3_partials(const orc_coeffs *k, double c1, const double e1[3], double c0, const double e0[3], double out[16])
{
    const double t = 1e-40;
    cplx C0 = c0, E0[3] = {e0[0], e0[1], e0[2]};
    for (int b = 0; b < 4; b++) {
        cplx C1 = c1, E1[3] = {e1[0], e1[1], e1[2]}, G[4];
        if (b == 0) C1 += _Complex_I * t;
        else E1[b - 1] += _Complex_I * t;
        G3_point(k, 3, C1, E1, C0, E0, G);
        for (int a = 0; a < 4; a++) out[a * 4 + b] = cimag(G[a]) / t;
    }
}

/*
 * Grid functions G_c, G_eta of the DVD derivative, term by term
 * (which: bit 0 = G^1, bit 1 = G^2, bit 2 = G^3, bit 3 = G^4):
 *   G^3 = ( -eps0 sum_I sigma_II(eps^el_{n+1/2}), 0 )          (Sec. 3, generalised from 1-D)
 *   G^4 = ( -gamma_c D^2 c_{n+1/2}, -3 gamma_eta D^2 eta_{n+1/2} ), D^2 = sum_J D^+_J D^-_J.
 */
void orc_dvd_G(const orc_grid *g, const orc_coeffs *k, double cbar0, const double *X1, const double *X0,
               int which, double *Gc, double *Ge)
{
    int nf = orc_nfields(g, k), d = g->dim;
    long N = grid_N(g);
    double h = g->h;
    if (n_eta(k) == 3) {
        /* Ge holds G_eta_j at Ge[j N + p] */
#pragma omp parallel for schedule(static)
        for (long p = 0; p < N; p++) {
            cplx c1 = X1[p * nf], c0 = X0[p * nf], e1[3], e0[3], G[4];
            for (int j = 0; j < 3; j++) {
                e1[j] = X1[p * nf + 1 + j];
                e0[j] = X0[p * nf + 1 + j];
            }
            G3_point(k, which & 3, c1, e1, c0, e0, G);
            double gc = creal(G[0]), ge[3] = {creal(G[1]), creal(G[2]), creal(G[3])};
            if ((which & 4) && is_elastic(k)) {
                double eps1[3][3], eps0m[3][3], s1[3][3], s0[3][3];
                el_strain(g, k, nf, cbar0, X1, p, eps1);
                el_strain(g, k, nf, cbar0, X0, p, eps0m);
                hooke(k, d, eps1, s1);
                hooke(k, d, eps0m, s0);
                double tr = 0.0;
                for (int I = 0; I < d; I++) tr += 0.5 * (s1[I][I] + s0[I][I]);
                gc += -k->eps0 * tr;
            }
            if (which & 8) {
                for (int f = 0; f < 4; f++) {
                    double lap = 0.0, mid = 0.5 * (X1[p * nf + f] + X0[p * nf + f]);
                    for (int J = 0; J < d; J++) {
                        long pp = nbr(g, p, J, +1), pm = nbr(g, p, J, -1);
                        lap += (0.5 * (X1[pp * nf + f] + X0[pp * nf + f]) - 2.0 * mid +
                                0.5 * (X1[pm * nf + f] + X0[pm * nf + f])) / (h * h);
                    }
                    if (f == 0) gc += -k->gamma_c * lap;
                    else ge[f - 1] += -k->gamma_eta * lap;
                }
            }
            Gc[p] = gc;
            for (int j = 0; j < 3; j++) Ge[j * N + p] = ge[j];
        }
        return;
    }
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) {
        double c1 = X1[p * nf], e1 = X1[p * nf + 1], c0 = X0[p * nf], e0 = X0[p * nf + 1];
        double gc = 0.0, ge = 0.0, a, b;
        if (which & 1) {
            G1_point(k, c1, e1, c0, e0, &a, &b);
            gc += a;
            ge += b;
        }
        if (which & 2) {
            G2_point(k, c1, e1, c0, e0, &a, &b);
            gc += a;
            ge += b;
        }
        if ((which & 4) && is_elastic(k)) {
            double eps1[3][3], eps0m[3][3], s1[3][3], s0[3][3];
            el_strain(g, k, nf, cbar0, X1, p, eps1);
            el_strain(g, k, nf, cbar0, X0, p, eps0m);
            hooke(k, d, eps1, s1);
            hooke(k, d, eps0m, s0);
            double tr = 0.0;
            for (int I = 0; I < d; I++) tr += 0.5 * (s1[I][I] + s0[I][I]);
            gc += -k->eps0 * tr;
        }
        if (which & 8) {
            double lc = 0.0, le = 0.0;
            double chp = 0.5 * (c1 + c0), ehp = 0.5 * (e1 + e0);
            for (int J = 0; J < d; J++) {
                long pp = nbr(g, p, J, +1), pm = nbr(g, p, J, -1);
                double chpp = 0.5 * (X1[pp * nf] + X0[pp * nf]), chpm = 0.5 * (X1[pm * nf] + X0[pm * nf]);
                double ehpp = 0.5 * (X1[pp * nf + 1] + X0[pp * nf + 1]), ehpm = 0.5 * (X1[pm * nf + 1] + X0[pm * nf + 1]);
                lc += (chpp - 2.0 * chp + chpm) / (h * h);
                le += (ehpp - 2.0 * ehp + ehpm) / (h * h);
            }
            gc += -k->gamma_c * lc;
            ge += -3.0 * k->gamma_eta * le;
        }
        Gc[p] = gc;
        Ge[p] = ge;
    }
}

/* edge mobility at level n, M_{p+1/2 e_J} = kappa (c_p(1-c_p) + c_{p+e_J}(1-c_{p+e_J}))/2  (Sec. 3) */
static double edge_mob(const orc_grid *g, const orc_coeffs *k, int nf, const double *X0, long p, int J)
{
    double ca = X0[p * nf], cb = X0[nbr(g, p, J, +1) * nf];
    return k->kappa * (ca * (1.0 - ca) + cb * (1.0 - cb)) / 2.0;
}

/* ------------------------------------------------------------------------ */
/* Residual of NSOA-1 (Sec. 3, Eq. NSOA-1)                                   */
/* ------------------------------------------------------------------------ */

/*
 * mode 0: full system
 *   F_c   = (c1 - c0)/dt - [D M D G_c]          (V_t = -A G, A = diag(-D M D, 1))
 *   F_eta = (eta1 - eta0)/dt + G_eta
 *   F_uI  = sum_J Dhat_J sigma_IJ(eps^el(u1, c1))  (discrete equilibrium at n+1)
 * mode 1: displacement-only system used for the initial equilibrium
 *   F_c = F_eta = 0, F_uI as above.
 */
void orc_residual(const orc_grid *g, const orc_coeffs *k, double cbar0, double dt, const double *X1,
                  const double *X0, int mode, double *F)
{
    int nf = orc_nfields(g, k), d = g->dim, ne = n_eta(k), ku = ufield(k);
    long N = grid_N(g);
    double h = g->h;
    /* kinetic factor of the Allen-Cahn rows: 1 (reduced model), 3 (three order parameters) */
    double keta = ne == 3 ? kEtaKinetic3 : 1.0;
    double *Gc = (double *)malloc(sizeof(double) * N), *Ge = (double *)malloc(sizeof(double) * N * ne);
    if (mode == 0) orc_dvd_G(g, k, cbar0, X1, X0, 15, Gc, Ge);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) {
        if (mode == 0) {
            double flux = 0.0;
            for (int J = 0; J < d; J++) {
                long pp = nbr(g, p, J, +1), pm = nbr(g, p, J, -1);
                double Mp = edge_mob(g, k, nf, X0, p, J), Mm = edge_mob(g, k, nf, X0, pm, J);
                flux += (Mp * (Gc[pp] - Gc[p]) - Mm * (Gc[p] - Gc[pm])) / (h * h);
            }
            F[p * nf] = (X1[p * nf] - X0[p * nf]) / dt - flux;
            for (int j = 0; j < ne; j++)
                F[p * nf + 1 + j] = (X1[p * nf + 1 + j] - X0[p * nf + 1 + j]) / dt + keta * Ge[j * N + p];
        } else {
            for (int f = 0; f < ku; f++) F[p * nf + f] = 0.0;
        }
        if (is_elastic(k) && g->neumann) {
            /* traction-free boundaries: F_u = -dE_3/du of the discrete elastic energy,
             * the adjoint of the centred differences with mirror ghosts:
             *   F_uI(p) = -sum_q sum_J sigma_IJ(q) w_J(q, p),
             *   w_J(q, p) = ([p == nbr(q, J, +1)] - [p == nbr(q, J, -1)]) / (2h),
             * over the cells q whose strain reads u(p) (p and its axis neighbours);
             * on a periodic grid this is the divergence form below */
            for (int I = 0; I < d; I++) F[p * nf + ku + I] = 0.0;
            long qs[7];
            int nq = 0;
            qs[nq++] = p;
            for (int J = 0; J < d; J++) {
                long a = nbr(g, p, J, +1), b = nbr(g, p, J, -1);
                if (a != p) qs[nq++] = a;
                if (b != p) qs[nq++] = b;
            }
            for (int t = 0; t < nq; t++) {
                long q = qs[t];
                double e[3][3], sg[3][3];
                el_strain(g, k, nf, cbar0, X1, q, e);
                hooke(k, d, e, sg);
                for (int J = 0; J < d; J++) {
                    double w = ((p == nbr(g, q, J, +1)) - (p == nbr(g, q, J, -1))) / (2.0 * h);
                    if (w == 0.0) continue;
                    for (int I = 0; I < d; I++) F[p * nf + ku + I] -= sg[I][J] * w;
                }
            }
        } else if (is_elastic(k)) {
            for (int I = 0; I < d; I++) {
                double div = 0.0;
                for (int J = 0; J < d; J++) {
                    double ep[3][3], em[3][3], sp[3][3], sm[3][3];
                    el_strain(g, k, nf, cbar0, X1, nbr(g, p, J, +1), ep);
                    el_strain(g, k, nf, cbar0, X1, nbr(g, p, J, -1), em);
                    hooke(k, d, ep, sp);
                    hooke(k, d, em, sm);
                    div += (sp[I][J] - sm[I][J]) / (2.0 * h);
                }
                F[p * nf + ku + I] = div;
            }
        }
    }
    free(Gc);
    free(Ge);
}

/* ------------------------------------------------------------------------ */
/* Analytic Jacobian dF/dX1 (Sec. 4, J_m = grad F(X_m)) assembled in CSR     */
/* ------------------------------------------------------------------------ */

#define ROWCAP 192

typedef struct {
    int n;
    long col[ROWCAP];
    double val[ROWCAP];
} rowacc;

static void ra_clear(rowacc *r) { r->n = 0; }

static void ra_add(rowacc *r, long col, double v)
{
    for (int i = 0; i < r->n; i++)
        if (r->col[i] == col) {
            r->val[i] += v;
            return;
        }
    if (r->n >= ROWCAP) {
        fprintf(stderr, "oracle: row accumulator overflow\n");
        abort();
    }
    r->col[r->n] = col;
    r->val[r->n] = v;
    r->n++;
}

static void ra_axpy(rowacc *dst, double a, const rowacc *src)
{
    for (int i = 0; i < src->n; i++) ra_add(dst, src->col[i], a * src->val[i]);
}

static void ra_sort(rowacc *r)
{
    for (int i = 1; i < r->n; i++) {
        long c = r->col[i];
        double v = r->val[i];
        int j = i - 1;
        while (j >= 0 && r->col[j] > c) {
            r->col[j + 1] = r->col[j];
            r->val[j + 1] = r->val[j];
            j--;
        }
        r->col[j + 1] = c;
        r->val[j + 1] = v;
    }
}

typedef struct {
    long n;
    long *rp;
    long *ci;
    double *v;
} csr;

static void csr_free(csr *A)
{
    free(A->rp);
    free(A->ci);
    free(A->v);
    A->rp = A->ci = NULL;
    A->v = NULL;
}

/*
 * Pointwise derivatives of G^1 + G^{2,S} with respect to (c1, eta1):
 * out[0] = dGc/dc1, out[1] = dGc/deta1, out[2] = dGeta/dc1, out[3] = dGeta/deta1.
 */
static void G12_partials(const orc_coeffs *k, double c1, double e1, double c0, double e0, double out[4])
{
    double f1 = 1.0 - e1, f0 = 1.0 - e0;
    double ch = 0.5 * (c1 + c0), fh = 0.5 * (f1 + f0), eh = 0.5 * (e1 + e0);
    int S = k->S;
    /* G^1_c = avgM1 ch + avgM2/3 Q3(c) + M3/4 Q4(c) + M4/5 Q5(c) + M0 */
    double avgM1 = (M1f(k, f0) + M1f(k, f1)) / 2.0;
    double avgM2 = (M2f(k, f0) + M2f(k, f1)) / 2.0;
    double dQ3 = 2.0 * c1 + c0;
    double dQ4 = 3.0 * c1 * c1 + 2.0 * c1 * c0 + c0 * c0;
    double dQ5 = 4.0 * c1 * c1 * c1 + 3.0 * c1 * c1 * c0 + 2.0 * c1 * c0 * c0 + c0 * c0 * c0;
    double g1c_c = avgM1 * 0.5 + avgM2 / 3.0 * dQ3 + M3c(k) / 4.0 * dQ4 + M4c(k) / 5.0 * dQ5;
    /* d/dphi1 of the averages: dM1/dphi = 2 (24U1 + 72U4) phi, dM2/dphi = -432 U4 phi - 432 U4 phi^2 */
    double dM1 = 2.0 * (24.0 * k->U1 + 72.0 * k->U4) * f1;
    double dM2 = -432.0 * k->U4 * f1 - 432.0 * k->U4 * f1 * f1;
    double g1c_e = -(0.5 * dM1 * ch + 0.5 * dM2 / 3.0 * quotpow(c1, c0, 3));
    /* G^1_eta = avgM5 phi_h + avgM6/3 Q3(phi) */
    double dM5 = -(48.0 * k->U1 * c1 + 72.0 * k->U4 * (2.0 * c1 - 6.0 * c1 * c1));
    double dM6 = 432.0 * k->U4 * c1 * c1;
    double g1e_c = 0.5 * dM5 * fh + 0.5 * dM6 / 3.0 * quotpow(f1, f0, 3);
    double avgM5 = (M5f(k, c0) + M5f(k, c1)) / 2.0, avgM6 = (M6f(k, c0) + M6f(k, c1)) / 2.0;
    double g1e_e = -(avgM5 * 0.5 + avgM6 / 3.0 * (2.0 * f1 + f0));

    /* G^{2,S} */
    double p1 = c1 * e1, p0 = c0 * e0, q1 = c1 * (4.0 - 3.0 * e1), q0 = c0 * (4.0 - 3.0 * e0);
    double Qp = orc_psi_quot(p1, p0, S), Qq = orc_psi_quot(q1, q0, S);
    double Dc = orc_psi_quot_d1(c1, c0, S), Dp = orc_psi_quot_d1(p1, p0, S), Dq = orc_psi_quot_d1(q1, q0, S);
    double t4 = k->theta / 4.0;
    double g2c_c = t4 * (4.0 * k->w_psi * Dc + 3.0 * eh * Dp * e1 + (4.0 - 3.0 * eh) * Dq * (4.0 - 3.0 * e1));
    double g2c_e = t4 * (1.5 * Qp + 3.0 * eh * Dp * c1 - 1.5 * Qq + (4.0 - 3.0 * eh) * Dq * (-3.0 * c1));
    double g2e_c = t4 * 3.0 * (0.5 * (Qp - Qq) + ch * (Dp * e1 - Dq * (4.0 - 3.0 * e1)));
    double g2e_e = t4 * 3.0 * ch * (Dp * c1 + 3.0 * c1 * Dq);
    out[0] = g1c_c + g2c_c;
    out[1] = g1c_e + g2c_e;
    out[2] = g1e_c + g2e_c;
    out[3] = g1e_e + g2e_e;
}

typedef struct {
    const orc_grid *g;
    const orc_coeffs *k;
    int nf, d, ne, ku;
    double cbar0, dt;
    const double *X1, *X0;
    double *part; /* (1 + ne)^2 per point: d(G_c, G_eta_j)/d(c1, eta_j1), row-major */
} jac_ctx;

/* row of dG_c(q)/dX1 */
static void Gc_row(const jac_ctx *cx, long q, rowacc *r)
{
    const orc_grid *g = cx->g;
    const orc_coeffs *k = cx->k;
    int nf = cx->nf, d = cx->d;
    double h = g->h;
    const int P = (1 + cx->ne) * (1 + cx->ne), ku = cx->ku;
    ra_clear(r);
    double diag = cx->part[q * P + 0] + k->gamma_c * d / (h * h);
    if (is_elastic(k)) {
        double lam = k->C11 + (d - 1) * k->C12;
        diag += 0.5 * d * k->eps0 * k->eps0 * lam;
    }
    ra_add(r, q * nf + 0, diag);
    for (int J = 0; J < d; J++) {
        ra_add(r, nbr(g, q, J, +1) * nf + 0, -0.5 * k->gamma_c / (h * h));
        ra_add(r, nbr(g, q, J, -1) * nf + 0, -0.5 * k->gamma_c / (h * h));
    }
    for (int j = 0; j < cx->ne; j++) ra_add(r, q * nf + 1 + j, cx->part[q * P + 1 + j]);
    if (is_elastic(k)) {
        /* G^3_c = -eps0 (C11 + (d-1) C12) tr eps^el_h, tr eps^el = sum_K Dhat_K u_K - d eps0 (c - cbar0) */
        double lam = k->C11 + (d - 1) * k->C12;
        for (int K = 0; K < d; K++) {
            ra_add(r, nbr(g, q, K, +1) * nf + ku + K, -k->eps0 * lam * 0.5 / (2.0 * h));
            ra_add(r, nbr(g, q, K, -1) * nf + ku + K, +k->eps0 * lam * 0.5 / (2.0 * h));
        }
    }
}

/* row of dsigma_IJ(q)/dX1 for eps^el(u1, c1) */
static void sig_row(const jac_ctx *cx, long q, int I, int J, rowacc *r)
{
    const orc_grid *g = cx->g;
    const orc_coeffs *k = cx->k;
    int nf = cx->nf, d = cx->d, ku = cx->ku;
    double h = g->h;
    ra_clear(r);
    if (I == J) {
        for (int K = 0; K < d; K++) {
            double cf = (K == I) ? k->C11 : k->C12;
            ra_add(r, nbr(g, q, K, +1) * nf + ku + K, cf / (2.0 * h));
            ra_add(r, nbr(g, q, K, -1) * nf + ku + K, -cf / (2.0 * h));
        }
        ra_add(r, q * nf + 0, -k->eps0 * (k->C11 + (d - 1) * k->C12));
    } else {
        ra_add(r, nbr(g, q, J, +1) * nf + ku + I, k->C44 / (2.0 * h));
        ra_add(r, nbr(g, q, J, -1) * nf + ku + I, -k->C44 / (2.0 * h));
        ra_add(r, nbr(g, q, I, +1) * nf + ku + J, k->C44 / (2.0 * h));
        ra_add(r, nbr(g, q, I, -1) * nf + ku + J, -k->C44 / (2.0 * h));
    }
}

/* assemble dF/dX1 at (X1, X0); mode as in orc_residual (mode 1: c and eta rows are identity rows) */
static void assemble_jacobian(const orc_grid *g, const orc_coeffs *k, double cbar0, double dt, const double *X1,
                              const double *X0, int mode, csr *A)
{
    int nf = orc_nfields(g, k), d = g->dim, ne = n_eta(k), ku = ufield(k);
    long N = grid_N(g);
    double h = g->h;
    const int P = (1 + ne) * (1 + ne);
    double keta = ne == 3 ? kEtaKinetic3 : 1.0;
    jac_ctx cx = {g, k, nf, d, ne, ku, cbar0, dt, X1, X0, NULL};
    cx.part = (double *)malloc(sizeof(double) * P * N);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) {
        if (ne == 3) {
            double e1[3] = {X1[p * nf + 1], X1[p * nf + 2], X1[p * nf + 3]};
            double e0[3] = {X0[p * nf + 1], X0[p * nf + 2], X0[p * nf + 3]};
            G3_partials(k, X1[p * nf], e1, X0[p * nf], e0, cx.part + P * p);
        } else {
            G12_partials(k, X1[p * nf], X1[p * nf + 1], X0[p * nf], X0[p * nf + 1], cx.part + P * p);
        }
    }

    /* rows of consecutive chunks of points are assembled independently (one
     * thread per chunk) into chunk buffers, then laid out in row order */
    const long CH = 1024;
    long nch = (N + CH - 1) / CH;
    long **cci = (long **)calloc(nch, sizeof(long *));
    double **cv = (double **)calloc(nch, sizeof(double *));
    long *cnnz = (long *)calloc(nch, sizeof(long));
    A->n = N * nf;
    A->rp = (long *)malloc(sizeof(long) * (A->n + 1));
#pragma omp parallel
    {
        rowacc *row = (rowacc *)malloc(sizeof(rowacc)), *t = (rowacc *)malloc(sizeof(rowacc));
#pragma omp for schedule(dynamic, 1)
        for (long ch = 0; ch < nch; ch++) {
            long pa = ch * CH, pb = pa + CH < N ? pa + CH : N;
            long cap = (pb - pa) * nf * 40 + 16, nnz = 0;
            long *ci = (long *)malloc(sizeof(long) * cap);
            double *v = (double *)malloc(sizeof(double) * cap);
            for (long p = pa; p < pb; p++) {
                for (int f = 0; f < nf; f++) {
                    ra_clear(row);
                    if (f == 0) {
                        if (mode == 0) {
                            ra_add(row, p * nf + 0, 1.0 / dt);
                            /* - (1/h^2) sum_J [ Mp G(p+J) + Mm G(p-J) - (Mp + Mm) G(p) ] */
                            for (int J = 0; J < d; J++) {
                                long pp = nbr(g, p, J, +1), pm = nbr(g, p, J, -1);
                                double Mp = edge_mob(g, k, nf, X0, p, J), Mm = edge_mob(g, k, nf, X0, pm, J);
                                Gc_row(&cx, pp, t);
                                ra_axpy(row, -Mp / (h * h), t);
                                Gc_row(&cx, pm, t);
                                ra_axpy(row, -Mm / (h * h), t);
                                Gc_row(&cx, p, t);
                                ra_axpy(row, (Mp + Mm) / (h * h), t);
                            }
                        } else {
                            ra_add(row, p * nf + 0, 1.0);
                        }
                    } else if (f < ku) {
                        /* eta_j row, j = f - 1: (eta_j1 - eta_j0)/dt + keta G_eta_j; the gradient
                         * part of keta G_eta_j is -3/2 gamma_eta D^2 eta_j1 + ... in both models */
                        const int j = f - 1;
                        if (mode == 0) {
                            const double *pr = cx.part + (long)P * p + (1 + j) * (1 + ne);
                            ra_add(row, p * nf + f, 1.0 / dt + keta * pr[1 + j] + 3.0 * k->gamma_eta * d / (h * h));
                            ra_add(row, p * nf + 0, keta * pr[0]);
                            for (int jj = 0; jj < ne; jj++)
                                if (jj != j) ra_add(row, p * nf + 1 + jj, keta * pr[1 + jj]);
                            for (int J = 0; J < d; J++) {
                                ra_add(row, nbr(g, p, J, +1) * nf + f, -1.5 * k->gamma_eta / (h * h));
                                ra_add(row, nbr(g, p, J, -1) * nf + f, -1.5 * k->gamma_eta / (h * h));
                            }
                        } else {
                            ra_add(row, p * nf + f, 1.0);
                        }
                    } else if (g->neumann) {
                        /* traction-free: the adjoint form of orc_residual */
                        int I = f - ku;
                        long qs[7];
                        int nq = 0;
                        qs[nq++] = p;
                        for (int J = 0; J < d; J++) {
                            long a = nbr(g, p, J, +1), b = nbr(g, p, J, -1);
                            if (a != p) qs[nq++] = a;
                            if (b != p) qs[nq++] = b;
                        }
                        for (int q = 0; q < nq; q++)
                            for (int J = 0; J < d; J++) {
                                double w = ((p == nbr(g, qs[q], J, +1)) - (p == nbr(g, qs[q], J, -1))) / (2.0 * h);
                                if (w == 0.0) continue;
                                sig_row(&cx, qs[q], I, J, t);
                                ra_axpy(row, -w, t);
                            }
                    } else {
                        int I = f - ku;
                        for (int J = 0; J < d; J++) {
                            sig_row(&cx, nbr(g, p, J, +1), I, J, t);
                            ra_axpy(row, 1.0 / (2.0 * h), t);
                            sig_row(&cx, nbr(g, p, J, -1), I, J, t);
                            ra_axpy(row, -1.0 / (2.0 * h), t);
                        }
                    }
                    ra_sort(row);
                    if (nnz + row->n > cap) {
                        cap = cap * 2 + row->n;
                        ci = (long *)realloc(ci, sizeof(long) * cap);
                        v = (double *)realloc(v, sizeof(double) * cap);
                    }
                    for (int i = 0; i < row->n; i++) {
                        ci[nnz] = row->col[i];
                        v[nnz] = row->val[i];
                        nnz++;
                    }
                    A->rp[p * nf + f + 1] = row->n; /* row length; offsets below */
                }
            }
            cci[ch] = (long *)realloc(ci, sizeof(long) * (nnz > 0 ? nnz : 1));
            cv[ch] = (double *)realloc(v, sizeof(double) * (nnz > 0 ? nnz : 1));
            cnnz[ch] = nnz;
        }
        free(row);
        free(t);
    }
    A->rp[0] = 0;
    for (long r = 0; r < A->n; r++) A->rp[r + 1] += A->rp[r];
    long total = A->rp[A->n];
    A->ci = (long *)malloc(sizeof(long) * (total > 0 ? total : 1));
    A->v = (double *)malloc(sizeof(double) * (total > 0 ? total : 1));
#pragma omp parallel for schedule(static)
    for (long ch = 0; ch < nch; ch++) {
        long off = A->rp[ch * CH * nf];
        memcpy(A->ci + off, cci[ch], sizeof(long) * cnnz[ch]);
        memcpy(A->v + off, cv[ch], sizeof(double) * cnnz[ch]);
        free(cci[ch]);
        free(cv[ch]);
    }
    free(cci);
    free(cv);
    free(cnnz);
    free(cx.part);
}

static void csr_matvec(const csr *A, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < A->n; i++) {
        double s = 0.0;
        for (long jj = A->rp[i]; jj < A->rp[i + 1]; jj++) s += A->v[jj] * x[A->ci[jj]];
        y[i] = s;
    }
}

/* exported: assemble the Jacobian and hand it out (opaque handle) */
void *orc_jacobian_new(const orc_grid *g, const orc_coeffs *k, double cbar0, double dt, const double *X1,
                       const double *X0, int mode)
{
    csr *A = (csr *)calloc(1, sizeof(csr));
    assemble_jacobian(g, k, cbar0, dt, X1, X0, mode, A);
    return A;
}
long orc_csr_n(void *h) { return ((csr *)h)->n; }
long orc_csr_nnz(void *h) { return ((csr *)h)->rp[((csr *)h)->n]; }
void orc_csr_copy(void *h, long *rp, long *ci, double *v)
{
    csr *A = (csr *)h;
    memcpy(rp, A->rp, sizeof(long) * (A->n + 1));
    memcpy(ci, A->ci, sizeof(long) * A->rp[A->n]);
    memcpy(v, A->v, sizeof(double) * A->rp[A->n]);
}
void orc_csr_free(void *h)
{
    csr_free((csr *)h);
    free(h);
}

/* ------------------------------------------------------------------------ */
/* ILU(0) and dense LU subdomain solvers (Sec. 4, Sec. 5.4)                  */
/* ------------------------------------------------------------------------ */

/*
 * ILU(0): incomplete LU with the sparsity pattern of A and no fill
 * (textbook IKJ form).  In place: the strict lower part receives L (unit
 * diagonal implied), the rest U.  Columns in each row must be sorted.
 * Returns 0, or ORC_EPIVOT on a zero pivot.
 */
int orc_ilu0(long n, const long *rp, const long *ci, double *v)
{
    long *diag = (long *)malloc(sizeof(long) * n);
    long *pos = (long *)malloc(sizeof(long) * n);
    for (long i = 0; i < n; i++) pos[i] = -1;
    for (long i = 0; i < n; i++) {
        diag[i] = -1;
        for (long jj = rp[i]; jj < rp[i + 1]; jj++)
            if (ci[jj] == i) diag[i] = jj;
        if (diag[i] < 0) {
            free(diag);
            free(pos);
            return ORC_EPIVOT;
        }
    }
    int rc = 0;
    for (long i = 0; i < n && rc == 0; i++) {
        for (long jj = rp[i]; jj < rp[i + 1]; jj++) pos[ci[jj]] = jj;
        for (long kk = rp[i]; kk < rp[i + 1] && ci[kk] < i; kk++) {
            long kr = ci[kk];
            v[kk] = v[kk] / v[diag[kr]];
            for (long jj = diag[kr] + 1; jj < rp[kr + 1]; jj++) {
                long j = ci[jj];
                if (pos[j] >= 0) v[pos[j]] -= v[kk] * v[jj];
            }
        }
        for (long jj = rp[i]; jj < rp[i + 1]; jj++) pos[ci[jj]] = -1;
        if (v[diag[i]] == 0.0 || !isfinite(v[diag[i]])) rc = ORC_EPIVOT;
    }
    free(diag);
    free(pos);
    return rc;
}

/* solve (L U) x = b with the factors produced by orc_ilu0 */
static void ilu0_solve(const csr *A, const double *b, double *x)
{
    long n = A->n;
    for (long i = 0; i < n; i++) {
        double s = b[i];
        for (long jj = A->rp[i]; jj < A->rp[i + 1] && A->ci[jj] < i; jj++) s -= A->v[jj] * x[A->ci[jj]];
        x[i] = s;
    }
    for (long i = n - 1; i >= 0; i--) {
        double s = x[i], dg = 0.0;
        for (long jj = A->rp[i]; jj < A->rp[i + 1]; jj++) {
            long j = A->ci[jj];
            if (j > i) s -= A->v[jj] * x[j];
            else if (j == i) dg = A->v[jj];
        }
        x[i] = s / dg;
    }
}

void orc_ilu0_solve(long n, const long *rp, const long *ci, const double *v, const double *b, double *x)
{
    csr A = {n, (long *)rp, (long *)ci, (double *)v};
    ilu0_solve(&A, b, x);
}

/* dense LU with partial pivoting (textbook Doolittle), column-major free */
static int dense_lu(long n, double *a, long *piv)
{
    for (long kk = 0; kk < n; kk++) {
        long pr = kk;
        double best = fabs(a[kk * n + kk]);
        for (long i = kk + 1; i < n; i++)
            if (fabs(a[i * n + kk]) > best) {
                best = fabs(a[i * n + kk]);
                pr = i;
            }
        piv[kk] = pr;
        if (best == 0.0) return ORC_EPIVOT;
        if (pr != kk)
            for (long j = 0; j < n; j++) {
                double t = a[kk * n + j];
                a[kk * n + j] = a[pr * n + j];
                a[pr * n + j] = t;
            }
        for (long i = kk + 1; i < n; i++) {
            a[i * n + kk] /= a[kk * n + kk];
            double l = a[i * n + kk];
            for (long j = kk + 1; j < n; j++) a[i * n + j] -= l * a[kk * n + j];
        }
    }
    return 0;
}

static void dense_lu_solve(long n, const double *a, const long *piv, const double *b, double *x)
{
    for (long i = 0; i < n; i++) x[i] = b[i];
    for (long kk = 0; kk < n; kk++) {
        long pr = piv[kk];
        if (pr != kk) {
            double t = x[kk];
            x[kk] = x[pr];
            x[pr] = t;
        }
    }
    for (long i = 0; i < n; i++)
        for (long j = 0; j < i; j++) x[i] -= a[i * n + j] * x[j];
    for (long i = n - 1; i >= 0; i--) {
        for (long j = i + 1; j < n; j++) x[i] -= a[i * n + j] * x[j];
        x[i] /= a[i * n + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Restricted additive Schwarz (Sec. 4: left-RAS of Cai & Sarkis) + P        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nsub, nf;
    int ku;              /* first displacement field (nf: none)            */
    long *next;          /* overlapped (extended) points per subdomain     */
    long **pts;          /* global point of each local point (x-fastest)   */
    unsigned char **own; /* 1 if the local point is owned (restricted)     */
    csr *A;              /* local matrices, factored in place              */
    double **dense;
    long **piv;
    int subsolver;
    int variant;         /* 0 left-RAS, 1 classical AS, 2 right-RAS         */
} ras_t;

/* owned cells [o0, o1) of subdomain s along an axis of n cells split in nsub
 * pieces; the extended range adds delta layers per side (periodic), or is the
 * whole axis when that would cover it. */
static void axis_range(int n, int nsub, int s, int delta, int clip, long *start, long *len, long *o0, long *o1)
{
    *o0 = (long)s * n / nsub;
    *o1 = (long)(s + 1) * n / nsub;
    if (clip) {
        /* Neumann: boxes stop at the boundary (no wrap) */
        long a = *o0 - delta, b = *o1 + delta;
        if (a < 0) a = 0;
        if (b > n) b = n;
        *start = a;
        *len = b - a;
        return;
    }
    if (*o1 - *o0 + 2 * delta >= n) {
        *start = 0;
        *len = n;
    } else {
        *start = *o0 - delta;
        *len = *o1 - *o0 + 2 * delta;
    }
}

static void ras_free(ras_t *R)
{
    for (int s = 0; s < R->nsub; s++) {
        free(R->pts[s]);
        free(R->own[s]);
        if (R->subsolver == 0) csr_free(&R->A[s]);
        else {
            free(R->dense[s]);
            free(R->piv[s]);
        }
    }
    free(R->next);
    free(R->pts);
    free(R->own);
    free(R->A);
    free(R->dense);
    free(R->piv);
    memset(R, 0, sizeof(*R));
}

/* build the subdomains of the box decomposition and factor J restricted to each overlapped box */
static int ras_setup(const orc_grid *g, int nf, int ku, const orc_opts *o, const csr *J, ras_t *R)
{
    int d = g->dim;
    int sub[3] = {1, 1, 1};
    for (int a = 0; a < d; a++) sub[a] = o->sub[a] > 0 ? o->sub[a] : 1;
    R->nsub = sub[0] * sub[1] * sub[2];
    R->nf = nf;
    R->ku = ku;
    R->subsolver = o->subsolver;
    R->variant = o->variant;
    R->next = (long *)calloc(R->nsub, sizeof(long));
    R->pts = (long **)calloc(R->nsub, sizeof(long *));
    R->own = (unsigned char **)calloc(R->nsub, sizeof(unsigned char *));
    R->A = (csr *)calloc(R->nsub, sizeof(csr));
    R->dense = (double **)calloc(R->nsub, sizeof(double *));
    R->piv = (long **)calloc(R->nsub, sizeof(long *));
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (int s = 0; s < R->nsub; s++) {
        int sidx[3] = {s % sub[0], (s / sub[0]) % sub[1], s / (sub[0] * sub[1])};
        long st[3], ln[3], o0[3], o1[3];
        for (int a = 0; a < 3; a++) {
            if (a < d)
                axis_range(g->n[a], sub[a], sidx[a], o->overlap, g->neumann, &st[a], &ln[a], &o0[a], &o1[a]);
            else {
                st[a] = 0;
                ln[a] = 1;
                o0[a] = 0;
                o1[a] = 1;
            }
        }
        long np = ln[0] * ln[1] * ln[2];
        R->next[s] = np;
        R->pts[s] = (long *)malloc(sizeof(long) * np);
        R->own[s] = (unsigned char *)malloc(np);
        long lp = 0;
        for (long z = 0; z < ln[2]; z++)
            for (long y = 0; y < ln[1]; y++)
                for (long x = 0; x < ln[0]; x++) {
                    long gx[3] = {x, y, z}, gc[3];
                    int owned = 1;
                    for (int a = 0; a < 3; a++) {
                        long n = g->n[a];
                        gc[a] = ((st[a] + gx[a]) % n + n) % n;
                        if (gc[a] < o0[a] || gc[a] >= o1[a]) owned = 0;
                    }
                    long gp = gc[0] + (long)g->n[0] * (gc[1] + (long)g->n[1] * gc[2]);
                    R->pts[s][lp] = gp;
                    R->own[s][lp] = (unsigned char)owned;
                    lp++;
                }
        /* local matrix: rows and columns of J restricted to the extended box; a
         * global point is in the box when its offset from the box start (modulo
         * the axis length) is below the box length on every axis, and its local
         * index is then the x-fastest number of those offsets */
        csr *L = &R->A[s];
        L->n = np * nf;
        L->rp = (long *)malloc(sizeof(long) * (L->n + 1));
        long cap = 0;
        for (long q = 0; q < np; q++)
            for (int f = 0; f < nf; f++) {
                long r = R->pts[s][q] * nf + f;
                cap += J->rp[r + 1] - J->rp[r];
            }
        L->ci = (long *)malloc(sizeof(long) * (cap + 1));
        L->v = (double *)malloc(sizeof(double) * (cap + 1));
        long nnz = 0;
        L->rp[0] = 0;
        rowacc *ra = (rowacc *)malloc(sizeof(rowacc));
        for (long q = 0; q < np; q++)
            for (int f = 0; f < nf; f++) {
                long r = R->pts[s][q] * nf + f;
                ra_clear(ra);
                for (long jj = J->rp[r]; jj < J->rp[r + 1]; jj++) {
                    long cp = J->ci[jj] / nf, cf = J->ci[jj] % nf;
                    long cc[3];
                    coords(g, cp, cc);
                    long loc = 0, mul = 1;
                    int inside = 1;
                    for (int a = 0; a < 3; a++) {
                        long n = g->n[a], off = ((cc[a] - st[a]) % n + n) % n;
                        if (off >= ln[a]) inside = 0;
                        loc += off * mul;
                        mul *= ln[a];
                    }
                    if (inside) ra_add(ra, loc * nf + cf, J->v[jj]);
                }
                ra_sort(ra);
                for (int i = 0; i < ra->n; i++) {
                    L->ci[nnz] = ra->col[i];
                    L->v[nnz] = ra->val[i];
                    nnz++;
                }
                L->rp[q * nf + f + 1] = nnz;
            }
        free(ra);
        if (o->subsolver == 0) {
            if (orc_ilu0(L->n, L->rp, L->ci, L->v) != 0) rc |= ORC_EPIVOT;
        } else {
            long n = L->n;
            R->dense[s] = (double *)calloc((size_t)n * n, sizeof(double));
            R->piv[s] = (long *)malloc(sizeof(long) * n);
            for (long i = 0; i < n; i++)
                for (long jj = L->rp[i]; jj < L->rp[i + 1]; jj++) R->dense[s][i * n + L->ci[jj]] = L->v[jj];
            if (dense_lu(n, R->dense[s], R->piv[s]) != 0) rc |= ORC_EPIVOT;
            csr_free(L);
        }
    }
    return rc;
}

/* centred staircase along an axis of n cells (n even): S(x) = floor((x+1)/2) - n/4.
 * With mirror ghosts its centred difference is 1/h at every cell, boundary cells
 * included: (S(1) - S(0))/(2h) = (S(x+1) - S(x-1))/(2h) = (S(n-1) - S(n-2))/(2h). */
static double staircase(long x, long n) { return (double)((x + 1) / 2) - 0.25 * (double)n; }

/*
 * Projection P applied after the Schwarz sweep (reading of the paper, which
 * only states that mass is conserved):
 *   - subtract the mean of z_c, so every Newton correction has sum s_c = 0;
 *   - remove from each z_uI its components along the null modes of the
 *     centred-difference strain: tensor products over the axes of 1 and, on
 *     axes with an even number of cells, (-1)^x (periodic grids);
 *   - with Neumann boundaries (mirror ghosts) the translations, and for every
 *     pair of axes I < J that both have an even number of cells the discrete
 *     rotation u_I = -S(x_J), u_J = S(x_I) (S the staircase above): its strain
 *     sym(Dhat u) vanishes at every cell, so it is an exact null mode of the
 *     displacement block, and every residual is orthogonal to it.
 */
static void project(const orc_grid *g, int nf, int ku, double *z)
{
    long N = grid_N(g);
    double mean = strided_sum(N, z, nf) / (double)N;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < N; p++) z[p * nf] -= mean;
    if (ku >= nf) return;
    int d = g->dim;
    int even_mask = 0; /* Neumann (mirror ghosts): translations only */
    for (int J = 0; J < d; J++)
        if (g->n[J] % 2 == 0 && !g->neumann) even_mask |= 1 << J;
    double *sv = (double *)malloc(sizeof(double) * N);
    for (int I = 0; I < d; I++) {
        for (int m = 0; m < (1 << d); m++) {
            if ((m & ~even_mask) != 0) continue;
            /* sv_p = mode(p) z_uI(p), mode(p) = (-1)^(sum of the coordinates selected by m) */
#pragma omp parallel for schedule(static)
            for (long p = 0; p < N; p++) {
                long x[3];
                coords(g, p, x);
                int par = 0;
                for (int J = 0; J < d; J++)
                    if (m & (1 << J)) par += (int)(x[J] & 1);
                double sg = (par & 1) ? -1.0 : 1.0;
                sv[p] = sg * z[p * nf + ku + I];
            }
            double a = strided_sum(N, sv, 1) / (double)N;
#pragma omp parallel for schedule(static)
            for (long p = 0; p < N; p++) {
                long x[3];
                coords(g, p, x);
                int par = 0;
                for (int J = 0; J < d; J++)
                    if (m & (1 << J)) par += (int)(x[J] & 1);
                double sg = (par & 1) ? -1.0 : 1.0;
                z[p * nf + ku + I] -= a * sg;
            }
        }
    }
    if (g->neumann) {
        double *nv = (double *)malloc(sizeof(double) * N);
        for (int I = 0; I < d; I++)
            for (int J = I + 1; J < d; J++) {
                if (g->n[I] % 2 != 0 || g->n[J] % 2 != 0) continue;
#pragma omp parallel for schedule(static)
                for (long p = 0; p < N; p++) {
                    long x[3];
                    coords(g, p, x);
                    double mi = -staircase(x[J], g->n[J]), mj = staircase(x[I], g->n[I]);
                    sv[p] = mi * z[p * nf + ku + I] + mj * z[p * nf + ku + J];
                    nv[p] = mi * mi + mj * mj;
                }
                double a = strided_sum(N, sv, 1) / strided_sum(N, nv, 1);
#pragma omp parallel for schedule(static)
                for (long p = 0; p < N; p++) {
                    long x[3];
                    coords(g, p, x);
                    z[p * nf + ku + I] -= a * -staircase(x[J], g->n[J]);
                    z[p * nf + ku + J] -= a * staircase(x[I], g->n[I]);
                }
            }
        free(nv);
    }
    free(sv);
}

/*
 * z = P M^-1 r for the three one-level Schwarz preconditioners of Sec. 4
 * (A_i: J restricted to the overlapped box i, R_i^delta: restriction to the
 * overlapped box, R_i^0: restriction to its owned points, zero elsewhere):
 *   left-RAS     M^-1 = sum_i R_i^0T     A_i^-1 R_i^delta  (owned points written)
 *   classical AS M^-1 = sum_i R_i^deltaT A_i^-1 R_i^delta  (overlaps summed)
 *   right-RAS    M^-1 = sum_i R_i^deltaT A_i^-1 R_i^0      (owned input, overlaps summed)
 * Sums run over the subdomains in index order.
 */
static void ras_apply(const orc_grid *g, const ras_t *R, int do_project, const double *r, double *z)
{
    int nf = R->nf;
    long N = grid_N(g);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N * nf; i++) z[i] = 0.0;
    /* the subdomain solves are independent; left-RAS writes disjoint owned
     * points, the other types keep each solution and add them in box order */
    double **xs = (double **)calloc(R->nsub, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < R->nsub; s++) {
        long np = R->next[s], n = np * nf;
        double *b = (double *)malloc(sizeof(double) * n), *x = (double *)malloc(sizeof(double) * n);
        for (long q = 0; q < np; q++)
            for (int f = 0; f < nf; f++)
                b[q * nf + f] = (R->variant == 2 && !R->own[s][q]) ? 0.0 : r[R->pts[s][q] * nf + f];
        if (R->subsolver == 0) ilu0_solve(&R->A[s], b, x);
        else dense_lu_solve(n, R->dense[s], R->piv[s], b, x);
        free(b);
        if (R->variant == 0) {
            for (long q = 0; q < np; q++)
                if (R->own[s][q])
                    for (int f = 0; f < nf; f++) z[R->pts[s][q] * nf + f] = x[q * nf + f];
            free(x);
        } else {
            xs[s] = x;
        }
    }
    if (R->variant != 0) {
        for (int s = 0; s < R->nsub; s++) {
            long np = R->next[s];
            for (long q = 0; q < np; q++)
                for (int f = 0; f < nf; f++) z[R->pts[s][q] * nf + f] += xs[s][q * nf + f];
            free(xs[s]);
        }
    }
    free(xs);
    if (do_project) project(g, nf, R->ku, z);
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES, right preconditioned, classical Gram-Schmidt (Sec. 4)    */
/* ------------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b)
{
    long nb = n_blocks(n);
    double *part = (double *)malloc(sizeof(double) * (nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
    for (long q = 0; q < nb; q++) {
        long i1 = (q + 1) * ORC_SUM_BLOCK < n ? (q + 1) * ORC_SUM_BLOCK : n;
        double s = 0.0;
        for (long i = q * ORC_SUM_BLOCK; i < i1; i++) s += a[i] * b[i];
        part[q] = s;
    }
    double s = sum_parts(part, nb);
    free(part);
    return s;
}

/*
 * Solves A x = b from x = 0 by GMRES(m) with right preconditioner M^-1 = P RAS^-1:
 * Arnoldi on A M^-1 with classical Gram-Schmidt (all projections taken from
 * the same w), one re-orthogonalisation pass when the norm drops below 0.7 of
 * its value before orthogonalisation, Givens rotations for the least squares
 * problem.  A cycle ends when the estimated residual reaches tol; the true
 * residual b - A x is then formed, and the solve ends when it is <= tol.
 */
static int gmres(const orc_grid *g, const csr *A, const ras_t *R, int do_project, const double *b, double *x,
                 int m, int maxit, double tol, int *its_out, double *res_out)
{
    long n = A->n;
    double **V = (double **)malloc(sizeof(double *) * (m + 1));
    for (int i = 0; i <= m; i++) V[i] = (double *)malloc(sizeof(double) * n);
    double *H = (double *)calloc((size_t)(m + 1) * m, sizeof(double)); /* H[i*m + j] */
    double *cs = (double *)malloc(sizeof(double) * m), *sn = (double *)malloc(sizeof(double) * m);
    double *gv = (double *)malloc(sizeof(double) * (m + 1)), *y = (double *)malloc(sizeof(double) * m);
    double *w = (double *)malloc(sizeof(double) * n), *z = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * n), *hv = (double *)malloc(sizeof(double) * (m + 1));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) {
        x[i] = 0.0;
        r[i] = b[i];
    }
    double beta = sqrt(dot(n, r, r));
    int its = 0;
    while (beta > tol && its < maxit) {
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) V[0][i] = r[i] / beta;
        for (int i = 0; i <= m; i++) gv[i] = 0.0;
        gv[0] = beta;
        int kdim = 0;
        for (int j = 0; j < m; j++) {
            ras_apply(g, R, do_project, V[j], z);
            csr_matvec(A, z, w);
            double wn0 = sqrt(dot(n, w, w));
            for (int i = 0; i <= j; i++) hv[i] = dot(n, V[i], w);
            /* per entry, the j + 1 updates in order i = 0..j */
#pragma omp parallel for schedule(static)
            for (long l = 0; l < n; l++)
                for (int i = 0; i <= j; i++) w[l] -= hv[i] * V[i][l];
            double wn = sqrt(dot(n, w, w));
            if (wn < 0.7 * wn0) {
                for (int i = 0; i <= j; i++) {
                    double h2 = dot(n, V[i], w);
                    hv[i] += h2;
#pragma omp parallel for schedule(static)
                    for (long l = 0; l < n; l++) w[l] -= h2 * V[i][l];
                }
                wn = sqrt(dot(n, w, w));
            }
            for (int i = 0; i <= j; i++) H[i * m + j] = hv[i];
            H[(j + 1) * m + j] = wn;
            for (int i = 0; i < j; i++) {
                double a = H[i * m + j], bb = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * bb;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
            }
            double a = H[j * m + j], bb = H[(j + 1) * m + j];
            double rr = sqrt(a * a + bb * bb);
            cs[j] = (rr == 0.0) ? 1.0 : a / rr;
            sn[j] = (rr == 0.0) ? 0.0 : bb / rr;
            H[j * m + j] = rr;
            H[(j + 1) * m + j] = 0.0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            its++;
            kdim = j + 1;
            if (wn != 0.0) {
#pragma omp parallel for schedule(static)
                for (long l = 0; l < n; l++) V[j + 1][l] = w[l] / wn;
            }
            if (fabs(gv[j + 1]) <= tol || its >= maxit || wn == 0.0) break;
        }
        for (int i = kdim - 1; i >= 0; i--) {
            double s = gv[i];
            for (int l = i + 1; l < kdim; l++) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        /* per entry, w = sum_i y_i V_i in order i = 0..kdim-1 */
#pragma omp parallel for schedule(static)
        for (long l = 0; l < n; l++) {
            w[l] = 0.0;
            for (int i = 0; i < kdim; i++) w[l] += y[i] * V[i][l];
        }
        ras_apply(g, R, do_project, w, z);
#pragma omp parallel for schedule(static)
        for (long l = 0; l < n; l++) x[l] += z[l];
        csr_matvec(A, x, w);
#pragma omp parallel for schedule(static)
        for (long l = 0; l < n; l++) r[l] = b[l] - w[l];
        beta = sqrt(dot(n, r, r));
    }
    *its_out = its;
    *res_out = beta;
    for (int i = 0; i <= m; i++) free(V[i]);
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(gv);
    free(y);
    free(w);
    free(z);
    free(r);
    free(hv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Newton with line search (Sec. 4)                                          */
/* ------------------------------------------------------------------------ */

/* c, c eta and c (4 - 3 eta) must lie in (0, 1) for the logarithms; with three
 * order parameters c and the four site fractions c eta_i (eta_4 = 4 - sum) */
static int in_domain(const orc_coeffs *k, long N, int nf, const double *X)
{
    int ok = 1;
    if (n_eta(k) == 3) {
#pragma omp parallel for schedule(static) reduction(& : ok)
        for (long p = 0; p < N; p++) {
            double c = X[p * nf], e4 = 4.0 - X[p * nf + 1] - X[p * nf + 2] - X[p * nf + 3];
            if (!(c > 0.0 && c < 1.0 && c * e4 > 0.0 && c * e4 < 1.0)) ok = 0;
            for (int j = 1; j <= 3; j++) {
                double q = c * X[p * nf + j];
                if (!(q > 0.0 && q < 1.0)) ok = 0;
            }
        }
        return ok;
    }
#pragma omp parallel for schedule(static) reduction(& : ok)
    for (long p = 0; p < N; p++) {
        double c = X[p * nf], e = X[p * nf + 1];
        double pp = c * e, q = c * (4.0 - 3.0 * e);
        if (!(c > 0.0 && c < 1.0 && pp > 0.0 && pp < 1.0 && q > 0.0 && q < 1.0)) ok = 0;
    }
    return ok;
}

/*
 * One NKS solve of NSOA-1 for X^{n+1} given X^n = X0 and dt:
 *   X_0 = X^n; J_m S_m = -F(X_m) by GMRES until ||J S + F|| <= max(xi_r ||F||, xi_a);
 *   X_{m+1} = X_m + lambda S_m, lambda from backtracking (halve while
 *   ||F(X+lambda S)||^2 > (1 - 2 alpha lambda) ||F||^2 or the trial leaves the
 *   domain; fail below lambda_min); stop when ||F|| <= max(eps_r ||F(X_0)||, eps_a).
 * The Schwarz factors come from J(X_0) and are reused for the whole solve when
 * opts->reuse (ILU(0)-reuse, Sec. 5.4).  mode 1 solves the displacement-only system.
 * Returns 0, ORC_EDIVERGED or ORC_EPIVOT.
 */
static int newton(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double cbar0, double dt,
                  const double *X0, double *X, int mode, double rtol, double atol, int maxit, orc_step_info *info)
{
    int nf = orc_nfields(g, k);
    long N = grid_N(g), n = N * nf;
    double *F = (double *)malloc(sizeof(double) * n), *S = (double *)malloc(sizeof(double) * n);
    double *Xt = (double *)malloc(sizeof(double) * n), *Ft = (double *)malloc(sizeof(double) * n);
    double *b = (double *)malloc(sizeof(double) * n);
    orc_residual(g, k, cbar0, dt, X, X0, mode, F);
    double fn0 = sqrt(dot(n, F, F)), fn = fn0;
    double tol = fmax(rtol * fn0, atol);
    info->fnorm0 = fn0;
    info->newton_its = 0;
    info->gmres_its = 0;
    int rc = ORC_EDIVERGED;
    ras_t R;
    memset(&R, 0, sizeof(R));
    int have_R = 0;
    if (!isfinite(fn0)) goto done;
    if (fn0 <= tol) {
        rc = ORC_OK;
        goto done;
    }
    for (int it = 0; it < maxit; it++) {
        csr J;
        assemble_jacobian(g, k, cbar0, dt, X, X0, mode, &J);
        if (!have_R || !o->reuse) {
            if (have_R) ras_free(&R);
            if (ras_setup(g, nf, ufield(k), o, &J, &R) != 0) {
                have_R = 1;
                csr_free(&J);
                rc = ORC_EPIVOT;
                goto done;
            }
            have_R = 1;
        }
#pragma omp parallel for schedule(static)
        for (long i = 0; i < n; i++) b[i] = -F[i];
        int gits;
        double gres;
        gmres(g, &J, &R, o->project, b, S, o->gmres_restart, o->gmres_maxit, fmax(o->gmres_rtol * fn, o->gmres_atol),
              &gits, &gres);
        csr_free(&J);
        info->gmres_its += gits;
        double lam = 1.0, ftn = 0.0;
        int ok = 0;
        while (lam >= o->ls_lambda_min) {
#pragma omp parallel for schedule(static)
            for (long i = 0; i < n; i++) Xt[i] = X[i] + lam * S[i];
            if (in_domain(k, N, nf, Xt)) {
                orc_residual(g, k, cbar0, dt, Xt, X0, mode, Ft);
                ftn = sqrt(dot(n, Ft, Ft));
                if (isfinite(ftn) && ftn * ftn <= (1.0 - 2.0 * o->ls_alpha * lam) * fn * fn) {
                    ok = 1;
                    break;
                }
            }
            lam *= 0.5;
        }
        info->newton_its = it + 1;
        if (!ok) break;
        memcpy(X, Xt, sizeof(double) * n);
        memcpy(F, Ft, sizeof(double) * n);
        fn = ftn;
        if (fn <= tol) {
            rc = ORC_OK;
            break;
        }
    }
done:
    info->fnorm = fn;
    if (have_R) ras_free(&R);
    free(F);
    free(S);
    free(Xt);
    free(Ft);
    free(b);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Exported drivers                                                          */
/* ------------------------------------------------------------------------ */

/* initial mechanical equilibrium (reading: solve F_u(u; c) = 0 for u before the
 * first step, since the energy law assumes equilibrium at level n).  In place. */
int orc_equilibrate(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double cbar0, double *X,
                    orc_step_info *info)
{
    memset(info, 0, sizeof(*info));
    if (!is_elastic(k)) return ORC_OK;
    long n = grid_N(g) * orc_nfields(g, k);
    double *X0 = (double *)malloc(sizeof(double) * n);
    memcpy(X0, X, sizeof(double) * n);
    int rc = newton(g, k, o, cbar0, 1.0, X0, X, 1, o->u0_rtol, o->u0_atol, o->u0_maxit, info);
    free(X0);
    return rc;
}

/* one NKS time step from X0 with the given dt; X receives X^{n+1} (X0 on failure) */
int orc_newton_step(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double cbar0, double dt,
                    const double *X0, double *X, orc_step_info *info)
{
    memset(info, 0, sizeof(*info));
    long n = grid_N(g) * orc_nfields(g, k);
    memcpy(X, X0, sizeof(double) * n);
    int rc = newton(g, k, o, cbar0, dt, X0, X, 0, o->newton_rtol, o->newton_atol, o->newton_maxit, info);
    if (rc != ORC_OK) memcpy(X, X0, sizeof(double) * n);
    info->dt = dt;
    info->status = rc;
    return rc;
}

/* preconditioner action z = P RAS^-1 r with the Schwarz factors of J(X1, X0) */
int orc_precond_apply(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double cbar0, double dt,
                      const double *X1, const double *X0, const double *r, double *z)
{
    csr J;
    assemble_jacobian(g, k, cbar0, dt, X1, X0, 0, &J);
    ras_t R;
    memset(&R, 0, sizeof(R));
    int rc = ras_setup(g, orc_nfields(g, k), ufield(k), o, &J, &R);
    if (rc == 0) ras_apply(g, &R, o->project, r, z);
    ras_free(&R);
    csr_free(&J);
    return rc;
}

/* linear solve J(X1, X0) x = b by GMRES + RAS; its/res receive the iteration count and true residual */
int orc_linear_solve(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double cbar0, double dt,
                     const double *X1, const double *X0, int mode, const double *b, double *x, double tol,
                     int *its, double *res)
{
    csr J;
    assemble_jacobian(g, k, cbar0, dt, X1, X0, mode, &J);
    ras_t R;
    memset(&R, 0, sizeof(R));
    int rc = ras_setup(g, orc_nfields(g, k), ufield(k), o, &J, &R);
    if (rc == 0) gmres(g, &J, &R, o->project, b, x, o->gmres_restart, o->gmres_maxit, tol, its, res);
    ras_free(&R);
    csr_free(&J);
    return rc;
}

/* adaptive step size prediction (Sec. 4, Eq. sencondt):
 *   dt = max(dt_min, dt_max / sqrt(1 + zeta * Xd^2)) */
double orc_dt_predict(double dt_min, double dt_max, double zeta, double Xd)
{
    return fmax(dt_min, dt_max / sqrt(1.0 + zeta * Xd * Xd));
}

/*
 * Time integration (Sec. 4): X holds X^0 = (c, eta, u = 0) on entry and the
 * final state on exit.  Step 1 uses dt_init; later steps predict dt from the
 * change rate of the two previous levels (dt_mode 1: ||X^n - X^{n-1}||_2 /
 * dt_{n-1}; dt_mode 2: |E^n - E^{n-1}| / dt_{n-1}), or take dt_replay[n-1]
 * when dt_replay is given.  A failed NKS solve retries with dt/sqrt(2) and
 * zeta doubled; the doubled zeta is used for the next prediction and then
 * reset unless zeta_persist.  info[n-1] describes step n.
 */
int orc_simulate(const orc_grid *g, const orc_coeffs *k, const orc_opts *o, double *X, int nsteps,
                 const double *dt_replay, orc_step_info *info, double *energy0)
{
    int nf = orc_nfields(g, k);
    long N = grid_N(g), n = N * nf;
    double cbar0 = strided_sum(N, X, nf) / (double)N;
    orc_step_info ei;
    int rc = orc_equilibrate(g, k, o, cbar0, X, &ei);
    if (rc != ORC_OK) return rc;
    double *Xprev = (double *)malloc(sizeof(double) * n), *Xnew = (double *)malloc(sizeof(double) * n);
    memcpy(Xprev, X, sizeof(double) * n);
    double E = orc_energy(g, k, cbar0, X, NULL), Eprev = E;
    if (energy0) *energy0 = E;
    double t = 0.0, dt_prev = o->dt_init, zeta = o->zeta;
    for (int st = 0; st < nsteps; st++) {
        double dt;
        if (dt_replay) dt = dt_replay[st];
        else if (st == 0 || o->dt_mode == 0) dt = o->dt_init;
        else {
            double Xd;
            if (o->dt_mode == 1) {
                double *dx = (double *)malloc(sizeof(double) * n);
#pragma omp parallel for schedule(static)
                for (long i = 0; i < n; i++) dx[i] = X[i] - Xprev[i];
                Xd = sqrt(dot(n, dx, dx)) / dt_prev;
                free(dx);
            } else {
                Xd = fabs(E - Eprev) / dt_prev;
            }
            dt = orc_dt_predict(o->dt_min, o->dt_max, zeta, Xd);
        }
        if (!o->zeta_persist) zeta = o->zeta;
        int retries = 0;
        orc_step_info si;
        for (;;) {
            rc = orc_newton_step(g, k, o, cbar0, dt, X, Xnew, &si);
            if (rc == ORC_OK) break;
            if (dt_replay || retries >= o->max_retries) break;
            dt /= sqrt(2.0);
            zeta *= 2.0;
            retries++;
        }
        if (rc != ORC_OK) {
            info[st] = si;
            info[st].retries = retries;
            info[st].status = rc;
            free(Xprev);
            free(Xnew);
            return rc;
        }
        memcpy(Xprev, X, sizeof(double) * n);
        memcpy(X, Xnew, sizeof(double) * n);
        Eprev = E;
        E = orc_energy(g, k, cbar0, X, NULL);
        t += dt;
        dt_prev = dt;
        si.dt = dt;
        si.t = t;
        si.energy = E;
        si.mass = orc_mass(g, k, X);
        si.retries = retries;
        si.status = ORC_OK;
        info[st] = si;
    }
    free(Xprev);
    free(Xnew);
    return ORC_OK;
}
