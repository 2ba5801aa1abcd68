// nks_krylov.cu -- restarted GMRES (Sec. 4) with classical Gram-Schmidt.
//
// Right-preconditioned GMRES(m) on J M^-1 with M^-1 = P RAS^-1:
//   - classical Gram-Schmidt: all projections h_i = v_i . w of one Arnoldi step
//     come from a single fused pass over V and w (which also yields w . w),
//     followed by one fused pass w -= V h that also yields ||w||^2;
//   - one re-orthogonalisation pass when ||w|| drops below 0.7 of its value
//     before orthogonalisation (decided on the device, no host round trip);
//   - Givens rotations and the small least-squares solve run in one thread;
//   - a cycle ends when the estimated residual reaches tol; x is then formed
//     as x += M^-1 (V y) and the true residual b - J x decides termination.
// Every reduction uses a fixed grid and a fixed tree, so results do not
// depend on timing.
#include <math.h>

#include <array>
#include <utility>

#include "nks_internal.cuh"

namespace nks {

namespace {

constexpr int kT = 256;
constexpr int kMaxDots = 33;  // m + 1 basis vectors + w.w for m <= 31 per pass

inline int nb(long long n) { return (int)((n + kT - 1) / kT); }

// layout of the small device state (doubles)
struct GmLayout {
    int m;
    int H, cs, sn, g, y, hcol, h2, scal;
    int total;
    explicit GmLayout(int m_) : m(m_)
    {
        H = 0;
        cs = H + (m + 1) * m;
        sn = cs + m;
        g = sn + m;
        y = g + m + 1;
        hcol = y + m;
        h2 = hcol + kMaxDots + 1;
        scal = h2 + kMaxDots + 1;
        total = scal + 16;
    }
};
// scal slots
enum { S_WN0 = 0, S_WN = 1, S_RES = 2, S_INV = 3, S_FLAG = 4, S_BETA = 5 };

__global__ void k_axpby(long long n, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_waxpy(long long n, const double *__restrict__ x, double a, const double *__restrict__ y,
                        double *__restrict__ w)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) w[i] = x[i] + a * y[i];
}

__global__ void k_scale_dev(long long n, const double *__restrict__ src, const double *__restrict__ s,
                            double *__restrict__ dst)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] * (*s);
}

__global__ void __launch_bounds__(kRedThreads) k_dot2(long long n, const double *__restrict__ x,
                                                      const double *__restrict__ y, double *__restrict__ partials)
{
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = x[i], b = y[i];
        acc[0] += a * b;
        acc[1] += b * b;
    }
    block_reduce_store<2>(acc, partials);
}

// CGS pass 1: h_i = v_i . w (i < NV) and w . w, one read of V and w.
// gate (optional): skip unless gate[0] != 0.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_multidot(long long n, const double *__restrict__ V, long long ldv,
                                                          const double *__restrict__ w, double *__restrict__ partials,
                                                          const double *gate)
{
    if (gate && gate[0] == 0.0) return;
    double acc[NV + 1];
#pragma unroll
    for (int k = 0; k <= NV; k++) acc[k] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] += V[k * ldv + i] * wi;
        acc[NV] += wi * wi;
    }
    block_reduce_store<NV + 1>(acc, partials);
}

// CGS pass 2: w -= sum_i h_i v_i, accumulating ||w||^2.
template <int NV>
__global__ void __launch_bounds__(kRedThreads) k_cgs_update(long long n, const double *__restrict__ V, long long ldv,
                                                            const double *__restrict__ h, double *__restrict__ w,
                                                            double *__restrict__ partials, const double *gate)
{
    if (gate && gate[0] == 0.0) return;
    double hk[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) hk[k] = h[k];
    double acc[1] = {0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = w[i];
#pragma unroll
        for (int k = 0; k < NV; k++) s -= hk[k] * V[k * ldv + i];
        w[i] = s;
        acc[0] += s * s;
    }
    block_reduce_store<1>(acc, partials);
}

using MultidotFn = void (*)(long long, const double *, long long, const double *, double *, const double *);
using UpdateFn = void (*)(long long, const double *, long long, const double *, double *, double *, const double *);

template <int... I>
constexpr auto multidot_table(std::integer_sequence<int, I...>)
{
    return std::array<MultidotFn, sizeof...(I)>{{&k_multidot<I + 1>...}};
}
template <int... I>
constexpr auto update_table(std::integer_sequence<int, I...>)
{
    return std::array<UpdateFn, sizeof...(I)>{{&k_cgs_update<I + 1>...}};
}
constexpr int kMaxNv = 31;
const auto g_multidot = multidot_table(std::make_integer_sequence<int, kMaxNv>{});
const auto g_update = update_table(std::make_integer_sequence<int, kMaxNv>{});

void launch_multidot(int nv, long long n, const double *V, const double *w, double *partials, const double *gate,
                     cudaStream_t st)
{
    g_multidot[nv - 1]<<<kRedBlocks, kRedThreads, 0, st>>>(n, V, n, w, partials, gate);
}

void launch_update(int nv, long long n, const double *V, const double *h, double *w, double *partials,
                   const double *gate, cudaStream_t st)
{
    g_update[nv - 1]<<<kRedBlocks, kRedThreads, 0, st>>>(n, V, n, h, w, partials, gate);
}

__global__ void k_finalize_g(const double *__restrict__ partials, int nblocks, int K, double *__restrict__ out,
                             const double *gate)
{
    if (gate && gate[0] == 0.0) return;
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

// after pass 2: remember ||w||^2 before orthogonalisation, decide on a second pass
__global__ void k_cgs_decide(double *gm, GmLayout L, int j)
{
    double *sc = gm + L.scal;
    sc[S_WN0] = gm[L.hcol + j + 1];  // w . w from pass 1
    const double wn = sqrt(sc[S_WN]), wn0 = sqrt(sc[S_WN0]);
    sc[S_FLAG] = (wn < 0.7 * wn0) ? 1.0 : 0.0;
}

// second pass accumulated into the projection coefficients
__global__ void k_cgs_accum(double *gm, GmLayout L, int j)
{
    if (gm[L.scal + S_FLAG] == 0.0) return;
    for (int i = 0; i <= j; i++) gm[L.hcol + i] += gm[L.h2 + i];
}

// Arnoldi column j: Hessenberg entries, Givens rotations, residual estimate
__global__ void k_arnoldi(double *gm, GmLayout L, int j)
{
    const int m = L.m;
    double *H = gm + L.H, *cs = gm + L.cs, *sn = gm + L.sn, *g = gm + L.g, *sc = gm + L.scal;
    const double wn = sqrt(sc[S_WN]);
    for (int i = 0; i <= j; i++) H[i * m + j] = gm[L.hcol + i];
    H[(j + 1) * m + j] = wn;
    for (int i = 0; i < j; i++) {
        const double a = H[i * m + j], b = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
    }
    const double a = H[j * m + j], b = H[(j + 1) * m + j];
    const double r = sqrt(a * a + b * b);
    cs[j] = (r == 0.0) ? 1.0 : a / r;
    sn[j] = (r == 0.0) ? 0.0 : b / r;
    H[j * m + j] = r;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    sc[S_RES] = fabs(g[j + 1]);
    sc[S_INV] = (wn != 0.0) ? 1.0 / wn : 0.0;
}

__global__ void k_gm_start(double *gm, GmLayout L, double beta)
{
    for (int i = 0; i <= L.m; i++) gm[L.g + i] = 0.0;
    gm[L.g] = beta;
    gm[L.scal + S_INV] = 1.0 / beta;
}

// upper-triangular solve H y = g for the first kdim columns
__global__ void k_hsolve(double *gm, GmLayout L, int kdim)
{
    const int m = L.m;
    double *H = gm + L.H, *g = gm + L.g, *y = gm + L.y;
    for (int i = kdim - 1; i >= 0; i--) {
        double s = g[i];
        for (int l = i + 1; l < kdim; l++) s -= H[i * m + l] * y[l];
        y[i] = s / H[i * m + i];
    }
}

// out = sum_{i < kdim} y_i v_i
__global__ void k_lincomb(long long n, const double *__restrict__ V, long long ldv, int kdim,
                          const double *__restrict__ y, double *__restrict__ out)
{
    __shared__ double ys[kMaxDots];
    if ((int)threadIdx.x < kdim) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxDots; k++)
        if (k < kdim) s += ys[k] * V[k * ldv + i];
    out[i] = s;
}

}  // namespace

int launch_axpby(long long n, double a, const double *x, double b, double *y, cudaStream_t st)
{
    k_axpby<<<nb(n), kT, 0, st>>>(n, a, x, b, y);
    return 1;
}

int launch_waxpy(long long n, const double *x, double a, const double *y, double *w, cudaStream_t st)
{
    k_waxpy<<<nb(n), kT, 0, st>>>(n, x, a, y, w);
    return 1;
}

int launch_scale_dev(long long n, const double *src, const double *inv, double *dst, cudaStream_t st)
{
    k_scale_dev<<<nb(n), kT, 0, st>>>(n, src, inv, dst);
    return 1;
}

int launch_dot2(long long n, const double *x, const double *y, double *partials, cudaStream_t st)
{
    k_dot2<<<kRedBlocks, kRedThreads, 0, st>>>(n, x, y, partials);
    return 1;
}

size_t gmres_state_doubles(int m) { return (size_t)GmLayout(m).total; }

// ||x||^2 of a device vector into P->hscal[0] (synchronises)
static double norm2_host(Problem *P, const double *x)
{
    P->tick(8);
    P->count(launch_dot2(P->nvec, x, x, P->partials, P->stream));
    P->count(launch_finalize(P->partials, kRedBlocks, 2, P->dscal, P->stream));
    P->tock(8);
    cudaMemcpyAsync(P->hscal, P->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, P->stream);
    cudaStreamSynchronize(P->stream);
    return P->hscal[0];
}

static void apply_J(Problem *P, int mode, const double *v, double *out)
{
    P->tick(1);
    P->count(launch_jv(P->g, P->k, P->cur_dt, mode, P->part, P->mob, v, P->Gc, P->sig, out, P->stream));
    P->tock(1);
}

int gmres_solve(Problem *P, int mode, const double *b, double *x, double tol, int *its_out, double *res_out)
{
    const int m = P->opts.gmres_restart;
    const GmLayout L(m);
    const long long n = P->nvec;
    cudaStream_t st = P->stream;
    double *V = P->V, *W = P->W, *Z = P->Z, *R = P->R, *gm = P->gm;
    cudaMemsetAsync(x, 0, sizeof(double) * n, st);
    cudaMemcpyAsync(R, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    double beta = sqrt(norm2_host(P, R));
    int its = 0;
    const int maxit = P->opts.gmres_maxit;
    while (beta > tol && its < maxit) {
        k_gm_start<<<1, 1, 0, st>>>(gm, L, beta);
        P->count(1 + launch_scale_dev(n, R, gm + L.scal + S_INV, V, st));
        int kdim = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            ras_apply(P, vj, Z);
            apply_J(P, mode, Z, W);
            // CGS pass 1 and 2
            P->tick(4);
            launch_multidot(j + 1, n, V, W, P->partials, nullptr, st);
            k_finalize_g<<<1, kRedThreads, 0, st>>>(P->partials, kRedBlocks, j + 2, gm + L.hcol, nullptr);
            P->tock(4);
            P->tick(5);
            launch_update(j + 1, n, V, gm + L.hcol, W, P->partials, nullptr, st);
            k_finalize_g<<<1, kRedThreads, 0, st>>>(P->partials, kRedBlocks, 1, gm + L.scal + S_WN, nullptr);
            P->tock(5);
            // optional second pass (CGS2), gated on the device
            k_cgs_decide<<<1, 1, 0, st>>>(gm, L, j);
            const double *gate = gm + L.scal + S_FLAG;
            P->tick(4);
            launch_multidot(j + 1, n, V, W, P->partials, gate, st);
            k_finalize_g<<<1, kRedThreads, 0, st>>>(P->partials, kRedBlocks, j + 2, gm + L.h2, gate);
            P->tock(4);
            P->tick(5);
            launch_update(j + 1, n, V, gm + L.h2, W, P->partials, gate, st);
            k_finalize_g<<<1, kRedThreads, 0, st>>>(P->partials, kRedBlocks, 1, gm + L.scal + S_WN, gate);
            P->tock(5);
            k_cgs_accum<<<1, 1, 0, st>>>(gm, L, j);
            P->tick(9);
            k_arnoldi<<<1, 1, 0, st>>>(gm, L, j);
            P->tock(9);
            launch_scale_dev(n, W, gm + L.scal + S_INV, vn, st);
            P->count(12);  // 2 multidot + 4 finalize + 2 update + decide + accum + arnoldi + scale
            its++;
            kdim = j + 1;
            cudaMemcpyAsync(P->hscal, gm + L.scal, 8 * sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(P, e, "gmres");
            const double res = P->hscal[S_RES], wn = sqrt(P->hscal[S_WN]);
            if (!(res == res)) break;  // NaN: leave the cycle, the true residual decides
            if (res <= tol || its >= maxit || wn == 0.0) break;
        }
        k_hsolve<<<1, 1, 0, st>>>(gm, L, kdim);
        k_lincomb<<<nb(n), kT, 0, st>>>(n, V, n, kdim, gm + L.y, W);
        P->count(2);
        ras_apply(P, W, Z);
        P->count(launch_axpby(n, 1.0, Z, 1.0, x, st));
        apply_J(P, mode, x, W);
        P->count(launch_waxpy(n, b, -1.0, W, R, st));
        beta = sqrt(norm2_host(P, R));
        if (!(beta == beta)) break;
    }
    *its_out = its;
    *res_out = beta;
    return NKS_OK;
}

}  // namespace nks
