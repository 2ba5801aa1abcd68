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
//
// The basis type TV is FP64, or FP32 in the mixed-precision mode: there the
// basis, the Arnoldi vectors, the Schwarz sweeps and the Jacobian action's
// inputs/outputs are FP32 (per-thread dot products accumulate in FP32, block
// and grid sums in FP64), while the Hessenberg/Givens state, the solution x,
// the true residual b - J x and the Jacobian arithmetic stay FP64.
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
// scal slots; S_GTOL .. S_CGSV: the device-side control of a cycle (its tolerance,
// iterations left in the solve, 1 while iterating, iterations, second passes and
// Gram-Schmidt vector transfers so far in the cycle)
enum { S_WN0 = 0, S_WN = 1, S_RES = 2, S_INV = 3, S_FLAG = 4, S_BETA = 5, S_KDIM = 6, S_GTOL = 7, S_LEFT = 8,
       S_ACTV = 9, S_NIT = 10, S_NREO = 11, S_CGSV = 12 };
constexpr int kCycleRow = 6;  // S_GTOL .. S_CGSV, written by the host at the start of a cycle

// Element-wise kernels run instance blockIdx.y of the batch.
#define NKS_INST(...)                         \
    long long io;                             \
    if (!inst_off(bt, blockIdx.y, io)) return; \
    __VA_ARGS__

__global__ void k_axpby(Bat bt, long long n, double a, const double *__restrict__ x, double b, double *__restrict__ y)
{
    NKS_INST(x = shift(x, io); y = shift(y, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + b * y[i];
}

__global__ void k_waxpy(Bat bt, long long n, const double *__restrict__ x, double a, const double *__restrict__ y,
                        double *__restrict__ w)
{
    NKS_INST(x = shift(x, io); y = shift(y, io); w = shift(w, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) w[i] = x[i] + a * y[i];
}

// w = x + lam y, lam = isc[I_LAM] of the instance
__global__ void k_waxpy_lam(Bat bt, long long n, const double *__restrict__ x, const double *__restrict__ isc,
                            const double *__restrict__ y, double *__restrict__ w)
{
    NKS_INST(x = shift(x, io); y = shift(y, io); w = shift(w, io); isc = shift(isc, io);)
    const double a = isc[I_LAM];
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) w[i] = x[i] + a * y[i];
}

__global__ void k_copy(Bat bt, long long n, const double *__restrict__ x, double *__restrict__ y)
{
    NKS_INST(x = shift(x, io); y = shift(y, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = x[i];
}

__global__ void k_zero(Bat bt, long long n, double *__restrict__ y)
{
    NKS_INST(y = shift(y, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = 0.0;
}

template <typename TS, typename TD>
__global__ void k_scale_dev(Bat bt, long long n, const TS *__restrict__ src, const double *__restrict__ s,
                            TD *__restrict__ dst)
{
    NKS_INST(src = shift(src, io); s = shift(s, io); dst = shift(dst, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if constexpr (sizeof(TS) == sizeof(float) && sizeof(TD) == sizeof(float)) {
        // FP32 basis: FP32 arithmetic, the factor converted once per block (a
        // double-to-float conversion per element would occupy the FP64 pipe);
        // 16-byte accesses (basis vectors start 16-byte aligned), thread i takes
        // elements 4i..4i+3, the last thread also the n % 4 tail
        __shared__ float sf;
        if (threadIdx.x == 0) sf = (float)(*s);
        __syncthreads();
        const long long n4 = n / 4;
        if (i < n4) {
            float4 v = reinterpret_cast<const float4 *>(src)[i];
            v.x *= sf;
            v.y *= sf;
            v.z *= sf;
            v.w *= sf;
            reinterpret_cast<float4 *>(dst)[i] = v;
        }
        if (i == n4)
            for (long long t = 4 * n4; t < n; t++) dst[t] = src[t] * sf;
    } else {
        if (i >= n) return;
        dst[i] = (TD)((double)src[i] * (*s));
    }
}

// y += x (x stored as TV)
template <typename TV>
__global__ void k_add(Bat bt, long long n, const TV *__restrict__ x, double *__restrict__ y)
{
    NKS_INST(x = shift(x, io); y = shift(y, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] += (double)x[i];
}

__global__ void __launch_bounds__(kRedThreads) k_dot2(Bat bt, long long n, const double *__restrict__ x,
                                                      const double *__restrict__ y, double *__restrict__ partials)
{
    NKS_INST(x = shift(x, io); y = shift(y, io); partials = shift(partials, io);)
    double acc[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = x[i], b = y[i];
        acc[0] += a * b;
        acc[1] += b * b;
    }
    block_reduce_store<2>(acc, partials);
}

template <typename TV>
struct Vec;
template <>
struct Vec<double> {
    using type = double2;
    static constexpr int W = 2;
};
template <>
struct Vec<float> {
    using type = float4;
    static constexpr int W = 4;
};

template <typename TV>
__device__ __forceinline__ void unpack(const typename Vec<TV>::type &t, TV (&a)[Vec<TV>::W])
{
    a[0] = t.x;
    a[1] = t.y;
    if constexpr (Vec<TV>::W == 4) {
        a[2] = t.z;
        a[3] = t.w;
    }
}

template <typename TV>
__device__ __forceinline__ typename Vec<TV>::type pack(const TV (&a)[Vec<TV>::W])
{
    typename Vec<TV>::type t;
    t.x = a[0];
    t.y = a[1];
    if constexpr (Vec<TV>::W == 4) {
        t.z = a[2];
        t.w = a[3];
    }
    return t;
}

// Per-thread sums of the basis type: each warp adds its lanes in that type (a
// fixed shuffle tree), the warps' sums are added in FP64 (fixed order) and
// stored as row blockIdx.x of partials.  For FP32 sums this keeps FP64
// arithmetic to one add per warp: GB300 runs FP64 at 1/64 of the FP32 rate.
template <int K, typename TV>
__device__ __forceinline__ void warp_then_block_store(TV (&v)[K], double *partials)
{
    if constexpr (sizeof(TV) == sizeof(double)) {
        block_reduce_store<K>(v, partials);
    } else {
        __shared__ double red[K][32];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < K; k++) {
            TV a = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) red[k][warp] = (double)a;
        }
        __syncthreads();
        if (threadIdx.x < K) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) a += red[threadIdx.x][w];
            partials[(size_t)blockIdx.x * K + threadIdx.x] = a;
        }
    }
}

// CGS pass 1: h_i = v_i . w (i < NV) and w . w, one read of V and w.
// Vectors are read as 16-byte packs (nq packs each): ldv is a multiple of the
// pack and entries past the vector length are zero.  gate (optional): skip
// unless gate[0] != 0.
template <int NV, typename TV>
__global__ void __launch_bounds__(kRedThreads, 4) k_multidot(Bat bt, long long nq, const TV *__restrict__ V,
                                                             long long ldv, const TV *__restrict__ w,
                                                             double *__restrict__ partials, const double *gate,
                                                             double *out, unsigned int *ticket)
{
    NKS_INST(V = shift(V, io); w = shift(w, io); partials = shift(partials, io); gate = shift(gate, io);
             out = shift(out, io); ticket = shift(ticket, io);)
    if (gate && gate[0] == 0.0) return;
    using VT = typename Vec<TV>::type;
    constexpr int WD = Vec<TV>::W;
    TV acc[NV + 1];
#pragma unroll
    for (int k = 0; k <= NV; k++) acc[k] = (TV)0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nq; i += (long long)gridDim.x * blockDim.x) {
        TV wa[WD];
        unpack<TV>(reinterpret_cast<const VT *>(w)[i], wa);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            TV va[WD];
            unpack<TV>(reinterpret_cast<const VT *>(V + k * ldv)[i], va);
#pragma unroll
            for (int e = 0; e < WD; e++) acc[k] += va[e] * wa[e];
        }
#pragma unroll
        for (int e = 0; e < WD; e++) acc[NV] += wa[e] * wa[e];
    }
    warp_then_block_store<NV + 1, TV>(acc, partials);
    grid_finalize(partials, NV + 1, out, ticket);
}

// CGS pass 2: w -= sum_i h_i v_i, accumulating ||w||^2.
template <int NV, typename TV>
__global__ void __launch_bounds__(kRedThreads, 4) k_cgs_update(Bat bt, long long nq, const TV *__restrict__ V,
                                                               long long ldv, const double *__restrict__ h,
                                                               TV *__restrict__ w, double *__restrict__ partials,
                                                               const double *gate, double *out, unsigned int *ticket)
{
    NKS_INST(V = shift(V, io); h = shift(h, io); w = shift(w, io); partials = shift(partials, io);
             gate = shift(gate, io); out = shift(out, io); ticket = shift(ticket, io);)
    if (gate && gate[0] == 0.0) return;
    using VT = typename Vec<TV>::type;
    constexpr int WD = Vec<TV>::W;
    // the coefficients in the basis type, converted once per block
    __shared__ TV hs[NV];
    if ((int)threadIdx.x < NV) hs[threadIdx.x] = (TV)h[threadIdx.x];
    __syncthreads();
    TV hk[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) hk[k] = hs[k];
    TV acc = (TV)0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nq; i += (long long)gridDim.x * blockDim.x) {
        TV sa[WD];
        unpack<TV>(reinterpret_cast<const VT *>(w)[i], sa);
#pragma unroll
        for (int k = 0; k < NV; k++) {
            TV va[WD];
            unpack<TV>(reinterpret_cast<const VT *>(V + k * ldv)[i], va);
#pragma unroll
            for (int e = 0; e < WD; e++) sa[e] -= hk[k] * va[e];
        }
        reinterpret_cast<VT *>(w)[i] = pack<TV>(sa);
#pragma unroll
        for (int e = 0; e < WD; e++) acc += sa[e] * sa[e];
    }
    TV acc1[1] = {acc};
    warp_then_block_store<1, TV>(acc1, partials);
    grid_finalize(partials, 1, out, ticket);
}

// CGS pass 2 fused with the dot products of the second pass (FP32 basis):
// w -= sum_i h_i v_i, and with each updated element still in registers,
// h2_i = v_i . w (i < NV) and w . w, written to out[0..NV].  One read of V
// and w instead of two.  Two elements per thread and iteration (8-byte loads:
// the NV basis pairs of those elements stay in registers; with one element
// per load the load instructions, not the bytes, bounded the kernel); the
// coefficients are read from shared memory.  n is even (the basis stride is a
// multiple of 4 elements).  Above 27 basis vectors the pairs need more than the
// 128 registers of two blocks per SM: one block per SM, no spills.
template <int NV, typename TV>
__global__ void __launch_bounds__(kRedThreads, NV > 27 ? 1 : 2) k_cgs_update_dots(Bat bt, long long n, const TV *__restrict__ V,
                                                                    long long ldv, const double *__restrict__ h,
                                                                    TV *__restrict__ w, double *__restrict__ partials,
                                                                    double *out, unsigned int *ticket)
{
    static_assert(sizeof(TV) == sizeof(float), "the fused pass serves the FP32 basis");
    NKS_INST(V = shift(V, io); h = shift(h, io); w = shift(w, io); partials = shift(partials, io);
             out = shift(out, io); ticket = shift(ticket, io);)
    __shared__ TV hs[NV];
    if ((int)threadIdx.x < NV) hs[threadIdx.x] = (TV)h[threadIdx.x];
    __syncthreads();
    TV acc[NV + 1];
#pragma unroll
    for (int k = 0; k <= NV; k++) acc[k] = (TV)0;
    const long long n2 = n / 2;
    float2 *w2 = reinterpret_cast<float2 *>(w);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n2; i += (long long)gridDim.x * blockDim.x) {
        float2 va[NV];
        float2 sa = w2[i];
#pragma unroll
        for (int k = 0; k < NV; k++) {
            va[k] = reinterpret_cast<const float2 *>(V + k * ldv)[i];
            sa.x -= hs[k] * va[k].x;
            sa.y -= hs[k] * va[k].y;
        }
        w2[i] = sa;
#pragma unroll
        for (int k = 0; k < NV; k++) acc[k] += va[k].x * sa.x + va[k].y * sa.y;
        acc[NV] += sa.x * sa.x + sa.y * sa.y;
    }
    warp_then_block_store<NV + 1, TV>(acc, partials);
    grid_finalize(partials, NV + 1, out, ticket);
}

template <typename TV>
using MultidotFn = void (*)(Bat, long long, const TV *, long long, const TV *, double *, const double *, double *,
                            unsigned int *);
template <typename TV>
using UpdateFn = void (*)(Bat, long long, const TV *, long long, const double *, TV *, double *, const double *,
                          double *, unsigned int *);

template <typename TV, int... I>
constexpr auto multidot_table(std::integer_sequence<int, I...>)
{
    return std::array<MultidotFn<TV>, sizeof...(I)>{{&k_multidot<I + 1, TV>...}};
}
template <typename TV, int... I>
constexpr auto update_table(std::integer_sequence<int, I...>)
{
    return std::array<UpdateFn<TV>, sizeof...(I)>{{&k_cgs_update<I + 1, TV>...}};
}
using UpdDotsFn = void (*)(Bat, long long, const float *, long long, const double *, float *, double *, double *,
                           unsigned int *);
template <int... I>
constexpr auto update_dots_table(std::integer_sequence<int, I...>)
{
    return std::array<UpdDotsFn, sizeof...(I)>{{&k_cgs_update_dots<I + 1, float>...}};
}
constexpr int kMaxNv = 31;
const auto g_multidot64 = multidot_table<double>(std::make_integer_sequence<int, kMaxNv>{});
const auto g_update64 = update_table<double>(std::make_integer_sequence<int, kMaxNv>{});
const auto g_multidot32 = multidot_table<float>(std::make_integer_sequence<int, kMaxNv>{});
const auto g_update32 = update_table<float>(std::make_integer_sequence<int, kMaxNv>{});
const auto g_update_dots32 = update_dots_table(std::make_integer_sequence<int, kMaxNv>{});

// FP32 basis: w -= V h, then h2 = V^T w and w . w into out[0..nv]
void launch_update_dots(int nv, long long ldv, const float *V, const double *h, float *w, double *partials,
                        double *out, unsigned int *ticket, int rb, cudaStream_t st, const Bat &bt)
{
    g_update_dots32[nv - 1]<<<dim3(rb, bt.nb), kRedThreads, 0, st>>>(bt, ldv, V, ldv, h, w, partials, out, ticket);
}

// h_i = v_i . w (i < nv) and w . w into out[0..nv]; ldv a multiple of the 16-byte pack
template <typename TV>
void launch_multidot(int nv, long long ldv, const TV *V, const TV *w, double *partials, const double *gate,
                     double *out, unsigned int *ticket, int rb, cudaStream_t st, const Bat &bt)
{
    constexpr int WD = Vec<TV>::W;
    const dim3 grd(rb, bt.nb);
    if constexpr (sizeof(TV) == 8)
        g_multidot64[nv - 1]<<<grd, kRedThreads, 0, st>>>(bt, ldv / WD, V, ldv, w, partials, gate, out, ticket);
    else
        g_multidot32[nv - 1]<<<grd, kRedThreads, 0, st>>>(bt, ldv / WD, V, ldv, w, partials, gate, out, ticket);
}

// w -= V h, ||w||^2 into out[0]
template <typename TV>
void launch_update(int nv, long long ldv, const TV *V, const double *h, TV *w, double *partials, const double *gate,
                   double *out, unsigned int *ticket, int rb, cudaStream_t st, const Bat &bt)
{
    constexpr int WD = Vec<TV>::W;
    const dim3 grd(rb, bt.nb);
    if constexpr (sizeof(TV) == 8)
        g_update64[nv - 1]<<<grd, kRedThreads, 0, st>>>(bt, ldv / WD, V, ldv, h, w, partials, gate, out, ticket);
    else
        g_update32[nv - 1]<<<grd, kRedThreads, 0, st>>>(bt, ldv / WD, V, ldv, h, w, partials, gate, out, ticket);
}

// Small GMRES kernels: one thread per instance, instance = blockIdx.x.
#define NKS_GM_INST()                          \
    long long io;                              \
    if (!inst_off(bt, blockIdx.x, io)) return; \
    gm = shift(gm, io);

// after pass 2: remember ||w||^2 before orthogonalisation, decide on a second pass
__global__ void k_cgs_decide(Bat bt, double *gm, GmLayout L, int j)
{
    NKS_GM_INST()
    double *sc = gm + L.scal;
    sc[S_WN0] = gm[L.hcol + j + 1];  // w . w from pass 1
    const double wn = sqrt(sc[S_WN]), wn0 = sqrt(sc[S_WN0]);
    sc[S_FLAG] = (wn < 0.7 * wn0) ? 1.0 : 0.0;
}

// the fused form: w . w before the update is hcol[j + 1], after it h2[j + 1]
__global__ void k_cgs_decide_fused(Bat bt, double *gm, GmLayout L, int j)
{
    NKS_GM_INST()
    double *sc = gm + L.scal;
    sc[S_WN0] = gm[L.hcol + j + 1];
    sc[S_WN] = gm[L.h2 + j + 1];
    const double wn = sqrt(sc[S_WN]), wn0 = sqrt(sc[S_WN0]);
    sc[S_FLAG] = (wn < 0.7 * wn0) ? 1.0 : 0.0;
}

// second pass accumulated into the projection coefficients
__global__ void k_cgs_accum(Bat bt, double *gm, GmLayout L, int j)
{
    NKS_GM_INST()
    if (gm[L.scal + S_FLAG] == 0.0) return;
    for (int i = 0; i <= j; i++) gm[L.hcol + i] += gm[L.h2 + i];
}

// Arnoldi column j: Hessenberg entries, Givens rotations, residual estimate
__global__ void k_arnoldi(Bat bt, double *gm, GmLayout L, int j)
{
    NKS_GM_INST()
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
    sc[S_KDIM] = j + 1;
}

// End of Arnoldi step j of every instance still iterating: count the step, its
// second pass and its Gram-Schmidt vector transfers (pass 1 reads j + 2 vectors, the
// update reads j + 2 and writes 1; a second pass repeats both, or with the FP32 basis,
// whose second-pass products ride on the first update, adds only its update, j + 3),
// and take the instance out of the cycle (act[i] = 0) when its residual estimate met
// the tolerance, its iterations are spent, the Krylov space broke down, or the estimate
// is not a number (the true residual decides then).  The host reads the counters once
// per few steps instead of after every step.
__global__ void k_gm_continue(Bat bt, double *gm, GmLayout L, int j, int *act, int fp32_basis)
{
    NKS_GM_INST()
    double *sc = gm + L.scal;
    const bool second = sc[S_FLAG] != 0.0;
    sc[S_NIT] = j + 1;
    sc[S_NREO] += second ? 1.0 : 0.0;
    const double extra = fp32_basis ? (j + 3.0) : (2.0 * j + 5.0);
    sc[S_CGSV] += (2.0 * j + 5.0) + (second ? extra : 0.0);
    const double res = sc[S_RES], wn = sqrt(sc[S_WN]);
    if (!(res == res) || res <= sc[S_GTOL] || (double)(j + 1) >= sc[S_LEFT] || wn == 0.0) {
        act[blockIdx.x] = 0;
        sc[S_ACTV] = 0.0;
    }
}

// beta = sqrt(beta2[0]): the norm of the starting residual
__global__ void k_gm_start(Bat bt, double *gm, GmLayout L, const double *beta2)
{
    NKS_GM_INST()
    const double beta = sqrt(shift(beta2, io)[0]);
    for (int i = 0; i <= L.m; i++) gm[L.g + i] = 0.0;
    gm[L.scal + S_KDIM] = 0.0;
    gm[L.g] = beta;
    gm[L.scal + S_INV] = 1.0 / beta;
}

// upper-triangular solve H y = g for the first kdim columns
__global__ void k_hsolve(Bat bt, double *gm, GmLayout L)
{
    NKS_GM_INST()
    const int kdim = (int)gm[L.scal + S_KDIM];
    const int m = L.m;
    double *H = gm + L.H, *g = gm + L.g, *y = gm + L.y;
    for (int i = kdim - 1; i >= 0; i--) {
        double s = g[i];
        for (int l = i + 1; l < kdim; l++) s -= H[i * m + l] * y[l];
        y[i] = s / H[i * m + i];
    }
}

// out = sum_{i < kdim} y_i v_i, kdim = the instance's Krylov dimension (gm scalar).
// FP64 basis: FP64 sums.  FP32 basis: FP32 coefficients (converted once per block)
// and FP32 sums, k ascending: the result is rounded to FP32 and enters the FP32
// sweep, and FP64 sums of FP32 values would run on the 1/64-rate FP64 pipe.
template <typename TV>
__global__ void k_lincomb(Bat bt, long long n, const TV *__restrict__ V, long long ldv, const double *__restrict__ gm,
                          GmLayout L, TV *__restrict__ out)
{
    NKS_INST(V = shift(V, io); gm = shift(gm, io); out = shift(out, io);)
    const int kdim = (int)gm[L.scal + S_KDIM];
    const double *y = gm + L.y;
    __shared__ TV ys[kMaxDots];
    if ((int)threadIdx.x < kdim) ys[threadIdx.x] = (TV)y[threadIdx.x];
    __syncthreads();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    TV s = (TV)0;
#pragma unroll
    for (int k = 0; k < kMaxDots; k++)
        if (k < kdim) s += ys[k] * V[k * ldv + i];
    out[i] = s;
}

}  // namespace

int launch_axpby(long long n, double a, const double *x, double b, double *y, cudaStream_t st, const Bat &bt)
{
    k_axpby<<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, a, x, b, y);
    return 1;
}

int launch_waxpy(long long n, const double *x, double a, const double *y, double *w, cudaStream_t st, const Bat &bt)
{
    k_waxpy<<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, x, a, y, w);
    return 1;
}

int launch_waxpy_lam(long long n, const double *x, const double *isc, const double *y, double *w, cudaStream_t st,
                     const Bat &bt)
{
    k_waxpy_lam<<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, x, isc, y, w);
    return 1;
}

int launch_copy(long long n, const double *x, double *y, cudaStream_t st, const Bat &bt)
{
    k_copy<<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, x, y);
    return 1;
}

static int launch_zero(long long n, double *y, cudaStream_t st, const Bat &bt)
{
    k_zero<<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, y);
    return 1;
}

template <typename TS, typename TD>
__global__ void k_convert(Bat bt, long long n, const TS *__restrict__ a, TD *__restrict__ b)
{
    NKS_INST(a = shift(a, io); b = shift(b, io);)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (TD)a[i];
}

int launch_convert(long long n, const double *a, float *b, cudaStream_t st, const Bat &bt)
{
    k_convert<double, float><<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, a, b);
    return 1;
}

int launch_convert(long long n, const float *a, double *b, cudaStream_t st, const Bat &bt)
{
    k_convert<float, double><<<dim3(nb(n), bt.nb), kT, 0, st>>>(bt, n, a, b);
    return 1;
}

int launch_dot2(long long n, const double *x, const double *y, double *partials, int rb, cudaStream_t st,
                const Bat &bt)
{
    k_dot2<<<dim3(rb, bt.nb), kRedThreads, 0, st>>>(bt, n, x, y, partials);
    return 1;
}

size_t gmres_state_doubles(int m) { return (size_t)GmLayout(m).total; }

// ||x||^2 of each instance's vector (bt's instances) into beta2[i] (synchronises);
// the squared norm stays in dscal[1] of each instance
static int norm2_batch(Problem *P, const double *x, const Bat &bt, std::vector<double> &beta2)
{
    P->tick(8);
    P->count(launch_dot2(P->nvec, x, x, P->partials, P->rb, P->stream, bt));
    P->count(launch_finalize(P->partials, P->rb, 2, P->dscal, P->stream, bt));
    P->tock(8);
    int rc = P->read_scalars(P->dscal + 1, 1, "gmres norm");
    if (rc) return rc;
    beta2.resize(P->nb);
    for (int i = 0; i < P->nb; i++) beta2[i] = P->hread[(size_t)i * 64];
    return NKS_OK;
}

// cls: the timer class (1: the Arnoldi steps' action, 10: the true residual's)
template <typename TV>
static void apply_J(Problem *P, int mode, const TV *v, TV *out, bool project_input, const Bat &bt, int cls = 1)
{
    P->tick(cls);
    if constexpr (sizeof(TV) == sizeof(float))
        P->count(launch_jv32(P->g, P->k, P->isc, mode, P->partf, P->mobf, v, out, P->stream, bt,
                             project_input ? P->zsum : nullptr));
    else
        P->count(launch_jv64(P->g, P->k, P->isc, mode, P->part, P->mob, v, P->Gc, P->sig, out, P->stream, bt,
                             project_input ? P->zsum : nullptr));
    P->tock(cls);
}

// Start of a solve: in mixed precision the FP32 copies of the operator's
// coefficients at the current iterate.  (The projection needs no set-up: the
// Arnoldi step applies J to z with the mean of z_c taken off, see the Jacobian
// action.)
static void prepare_operator(Problem *P, int mode, const Bat &bt)
{
    if (!P->inner_f32(mode)) return;
    P->tick(1);
    refresh_f32_coefficients(P, bt);
    P->tock(1);
}

// FP32 copies of the Jacobian action's coefficients at the current iterate
void refresh_f32_coefficients(Problem *P, const Bat &bt)
{
    P->count(launch_convert((1 + P->k.ne) * (1 + P->k.ne) * P->N, P->part, P->partf, P->stream, bt));
    P->count(launch_convert(P->g.dim * P->N, P->mob, P->mobf, P->stream, bt));
}

// Krylov work vectors of the basis type
template <typename TV>
struct Basis {
    TV *V, *W, *Z;
    long long ldv;
};
static Basis<double> basis64(Problem *P) { return {P->V, P->W, P->Z, P->ldv}; }
static Basis<float> basis32(Problem *P) { return {P->Vf, P->Wf, P->Zf, P->ldvf}; }

// Replay the captured graph of GMRES iteration j (capturing it on first use).
// Returns false when graphs are unavailable (the caller launches directly).
template <class Fn>
static bool run_graph(Problem *P, int mode, int j, Fn &&enqueue)
{
    Problem::IterGraph &G = P->graphs[mode & 1][j];
    if (!G.exec) {
        const nks_stats before = P->stats;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue();
            e = cudaStreamEndCapture(P->stream, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        // the capture counted one replay's launches: keep them per graph instead
        G.kernels = P->stats.kernel_launches - before.kernel_launches;
        for (int c = 0; c < NKS_NCLASS; c++) G.launches[c] = P->stats.launches[c] - before.launches[c];
        P->stats = before;
        if (e != cudaSuccess) {
            cudaGetLastError();
            G.exec = nullptr;
            P->graphs_off = true;
            return false;
        }
    }
    if (cudaGraphLaunch(G.exec, P->stream) != cudaSuccess) {
        cudaGetLastError();
        P->graphs_off = true;
        return false;
    }
    P->stats.kernel_launches += G.kernels;
    for (int c = 0; c < NKS_NCLASS; c++) P->stats.launches[c] += G.launches[c];
    return true;
}

// Batched GMRES(m): every instance with is[i].gin runs its own Arnoldi process
// (own Hessenberg matrix, own stopping test) in lockstep with the others; an
// instance that has met its test is masked out of the remaining launches, so
// each instance performs exactly the operations it performs alone.
template <typename TV>
static int gmres_t(Problem *P, Basis<TV> K, int mode, const double *b, double *x)
{
    const int m = P->opts.gmres_restart;
    const GmLayout L(m);
    const long long n = P->nvec, ldv = K.ldv;
    const int nbt = P->nb;
    cudaStream_t st = P->stream;
    TV *V = K.V, *W = K.W, *Z = K.Z;
    double *R = P->R, *gm = P->gm, *Jx = P->T64;
    const int maxit = P->opts.gmres_maxit;
    const bool use_graphs = P->opts.graphs && !P->opts.timing && !P->graphs_off;
    std::vector<char> in(nbt), cyc(nbt), act(nbt);
    for (int i = 0; i < nbt; i++) {
        in[i] = P->is[i].gin ? 1 : 0;
        P->is[i].gits = 0;
    }
    const Bat bin = P->set_mask(M_GIN, in);
    // the sweeps' failure word starts clear for this solve
    cudaMemset2DAsync(P->dflag + 1, (size_t)P->stride, 0, sizeof(int), (size_t)P->nb, st);
    P->count(launch_zero(n, x, st, bin));
    P->count(launch_copy(n, b, R, st, bin));
    prepare_operator(P, mode, bin);
    std::vector<double> b2;
    int rc = norm2_batch(P, R, bin, b2);
    if (rc) return rc;
    for (int i = 0; i < nbt; i++)
        if (in[i]) P->is[i].beta = sqrt(b2[i]);
    for (;;) {
        bool any = false;
        for (int i = 0; i < nbt; i++) {
            const IState &s = P->is[i];
            cyc[i] = in[i] && s.beta == s.beta && s.beta > s.gtol && s.gits < maxit;
            any = any || cyc[i];
        }
        if (!any) break;
        const Bat bc = P->set_mask(M_CYC, cyc);
        act = cyc;
        const Bat ba = P->set_mask(M_ACT, act);
        {
            // the cycle's control rows: tolerance, iterations left, active, counters
            std::vector<double> rows((size_t)nbt * kCycleRow, 0.0);
            for (int i = 0; i < nbt; i++) {
                rows[(size_t)i * kCycleRow + 0] = P->is[i].gtol;
                rows[(size_t)i * kCycleRow + 1] = (double)(maxit - P->is[i].gits);
                rows[(size_t)i * kCycleRow + 2] = cyc[i] ? 1.0 : 0.0;
            }
            P->upload_rows(gm + L.scal + S_GTOL, rows.data(), kCycleRow);
        }
        k_gm_start<<<nbt, 1, 0, st>>>(bc, gm, L, P->dscal + 1);
        k_scale_dev<double, TV><<<dim3(nb(n), nbt), kT, 0, st>>>(bc, n, R, gm + L.scal + S_INV, V);
        P->count(2);
        // Arnoldi steps in groups of kGroup between host read-backs: each step ends with
        // the device-side test of every instance (k_gm_continue), which masks finished
        // instances out of the steps that follow; the host learns of them at the group's end
        constexpr int kGroup = 4;
        for (int j = 0; j < m; j++) {
            // one Arnoldi step of every instance still iterating (one graph when graphs are on)
            auto iteration = [&]() {
                TV *vj = V + (size_t)j * ldv, *vn = V + (size_t)(j + 1) * ldv;
                ras_apply_t<TV>(P, vj, Z, ba);         // z = RAS^-1 v_j (sum of z_c to zsum)
                apply_J<TV>(P, mode, Z, W, true, ba);  // w = J P z
                // CGS pass 1 and 2
                P->tick(4);
                launch_multidot<TV>(j + 1, ldv, V, W, P->partials, nullptr, gm + L.hcol, P->tickets, P->rb, st, ba);
                P->tock(4);
                const double *gate = gm + L.scal + S_FLAG;
                if constexpr (sizeof(TV) == sizeof(float)) {
                    // FP32 basis: the update also forms the second pass's dot products
                    P->tick(5);
                    launch_update_dots(j + 1, ldv, V, gm + L.hcol, W, P->partials, gm + L.h2, P->tickets + 1,
                                       P->rb, st, ba);
                    P->tock(5);
                    k_cgs_decide_fused<<<nbt, 1, 0, st>>>(ba, gm, L, j);
                } else {
                    P->tick(5);
                    launch_update<TV>(j + 1, ldv, V, gm + L.hcol, W, P->partials, nullptr, gm + L.scal + S_WN,
                                      P->tickets + 1, P->rb, st, ba);
                    P->tock(5);
                    // optional second pass (CGS2), gated on the device
                    k_cgs_decide<<<nbt, 1, 0, st>>>(ba, gm, L, j);
                    P->tick(4);
                    launch_multidot<TV>(j + 1, ldv, V, W, P->partials, gate, gm + L.h2, P->tickets, P->rb, st, ba);
                    P->tock(4);
                    P->count(1);
                }
                P->tick(5);
                launch_update<TV>(j + 1, ldv, V, gm + L.h2, W, P->partials, gate, gm + L.scal + S_WN,
                                  P->tickets + 1, P->rb, st, ba);
                P->tock(5);
                k_cgs_accum<<<nbt, 1, 0, st>>>(ba, gm, L, j);
                P->tick(9);
                k_arnoldi<<<nbt, 1, 0, st>>>(ba, gm, L, j);
                P->tock(9);
                k_scale_dev<TV, TV><<<dim3(nb(sizeof(TV) == sizeof(float) ? n / 4 + 1 : n), nbt), kT, 0, st>>>(
                    ba, n, W, gm + L.scal + S_INV, vn);
                P->count(7);  // multidot + update (+ dots) + decide + update + accum + arnoldi + scale
                k_gm_continue<<<nbt, 1, 0, st>>>(ba, gm, L, j, P->dmask + (size_t)M_ACT * nbt,
                                                   sizeof(TV) == sizeof(float) ? 1 : 0);
                P->count(1);
            };
            if (!(use_graphs && run_graph(P, mode, j, iteration))) iteration();
            if ((j + 1) % kGroup != 0 && j + 1 < m) continue;
            rc = P->read_scalars(gm + L.scal, S_CGSV + 1, "gmres");
            if (rc) return rc;
            for (int i = 0; i < nbt; i++)
                if (cyc[i] && (P->hflags[2 * i + 1] & 4)) {
                    P->err = "Schwarz sweep: a bulk copy of the factors did not complete";
                    return NKS_ETIMEOUT;
                }
            bool left = false;
            for (int i = 0; i < nbt; i++) left = left || (cyc[i] && P->hread[(size_t)i * 64 + S_ACTV] != 0.0);
            if (!left) break;
        }
        // the cycle's iterations and Gram-Schmidt work of every instance (read back above)
        for (int i = 0; i < nbt; i++) {
            if (!cyc[i]) continue;
            const double *h = P->hread + (size_t)i * 64;
            P->is[i].gits += (int)h[S_NIT];
            P->stats.reorth += (long long)h[S_NREO];
            P->stats.cgs_bytes += h[S_CGSV] * (double)n * sizeof(TV);
        }
        // x += M^-1 (V y), then the true residual in FP64
        k_hsolve<<<nbt, 1, 0, st>>>(bc, gm, L);
        k_lincomb<TV><<<dim3(nb(n), nbt), kT, 0, st>>>(bc, n, V, ldv, gm, L, W);
        P->count(2);
        ras_apply_t<TV>(P, W, Z, bc);
        k_add<TV><<<dim3(nb(n), nbt), kT, 0, st>>>(bc, n, Z, x);
        P->count(1);
        // x = x + P z: x is already in the range of P and P is linear and idempotent,
        // so P is applied once to the FP64 sum; every Newton correction keeps
        // sum s_c = 0 and the gauge of u to FP64 rounding
        project(P, x, bc);
        apply_J<double>(P, mode, x, Jx, false, bc, 10);
        P->count(launch_waxpy(n, b, -1.0, Jx, R, st, bc));
        rc = norm2_batch(P, R, bc, b2);
        if (rc) return rc;
        for (int i = 0; i < nbt; i++)
            if (cyc[i]) P->is[i].beta = sqrt(b2[i]);
    }
    for (int i = 0; i < nbt; i++)
        if (in[i]) P->is[i].res = P->is[i].beta;
    // a Schwarz sweep whose factor copy never completed flags its instance (bounded wait)
    rc = P->read_flags("gmres");
    if (rc) return rc;
    for (int i = 0; i < nbt; i++)
        if (in[i] && (P->hflags[2 * i + 1] & 4)) {
            P->err = "Schwarz sweep: a bulk copy of the factors did not complete";
            return NKS_ETIMEOUT;
        }
    return NKS_OK;
}

void destroy_graphs(Problem *P)
{
    for (auto &row : P->graphs)
        for (auto &G : row)
            if (G.exec) {
                cudaGraphExecDestroy(G.exec);
                G.exec = nullptr;
            }
}

int gmres_solve(Problem *P, int mode, const double *b, double *x)
{
    if (P->inner_f32(mode)) return gmres_t<float>(P, basis32(P), mode, b, x);
    return gmres_t<double>(P, basis64(P), mode, b, x);
}

}  // namespace nks
