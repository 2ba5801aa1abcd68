// nks_internal.cuh -- shared declarations of the GB300 NKS solver.
//
// Layout in HBM: every state vector is structure-of-arrays, field-major:
//   X[f * N + p],  f = 0 (c), 1..ne (eta_1..eta_ne), 1 + ne.. (u_1..u_d),
//   p = x + nx (y + ny z), with ne = 1 (reduced model) or 3 (App. A).
// One Newton iterate therefore streams nf contiguous, coalesced planes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nks.h"

namespace nks {

constexpr int kRedBlocks = 608;    // 4 x 152 SMs: fixed reduction grid (deterministic sums)
constexpr int kRedThreads = 256;
constexpr int kMaxNf = 7;          // c, eta_1..eta_3, u_1..u_3
constexpr int kMaxRow = 128;       // longest Jacobian row (3-D c-row): 71 entries, 83 with Neumann
                                   // boundaries; 85 / 97 with three order parameters (at most 128:
                                   // the factor kernel marks present slots in two 64-bit words)
constexpr int kMaxRestart = 64;

// Grid as seen by the kernels.
struct DGrid {
    int dim;
    int n[3];
    long long N;
    double h;
    double ih, ih2, i2h;  // 1/h, 1/h^2, 1/(2h), formed on the host
    int bc;               // NKS_PERIODIC or NKS_NEUMANN (mirror ghost cells)
};

inline void set_spacing(DGrid &g, double h)
{
    g.h = h;
    g.ih = 1.0 / h;
    g.ih2 = 1.0 / (h * h);
    g.i2h = 0.5 / h;
}

// Coefficients after the App. B reduction to the polynomial coefficients M_k.
struct DCoef {
    double kappa, gamma_c, gamma_eta, theta, w_psi;
    double M0, m1a, m1b, m2a, m2b, m2c, M3, M4;  // M1 = m1a + m1b phi^2, M2 = m2a + m2b phi^2 + m2c phi^3
    double U1, U4;                               // M5(c), M6(c)
    double eps0, C11, C12, C44, lam;             // lam = C11 + (d - 1) C12
    double L[4], dE0;                            // App. A, for the energy E1
    double cbar0;                                // initial mean composition (Sec. 3)
    double ser_c[16];                            // 1/(2k(2k+1)), k = 1..S-1  (Psi_S series)
    double ser_e[16];                            // 1/(2k+1)
    int S;
    int elastic;
    int nf;
    int ne;                                      // order parameters: 1 or 3 (App. A)
    double keta;                                 // kinetic factor of the eta rows: 1, or 3 with ne = 3
};

// Batches.  A problem holds nb instances of the same grid, coefficients and
// options (a single problem is a batch of one).  Every per-instance buffer is
// carved from the instance's slab at the same offset, so instance b's copy of
// any per-instance buffer lies b * stride bytes after instance 0's.  One launch
// runs all instances of a phase: the instance is blockIdx.y (or the dimension
// a kernel states), and an instance whose mask entry is 0 is skipped.
struct Bat {
    long long stride = 0;        // bytes between the slabs of consecutive instances
    const int *mask = nullptr;   // [nb] (device): run instance b when mask[b] != 0; nullptr: all
    int nb = 1;
};

template <class T>
__host__ __device__ __forceinline__ T *shift(T *p, long long off)
{
    return p ? (T *)((const char *)p + off) : p;
}

__device__ __forceinline__ bool inst_off(const Bat &bt, int b, long long &off)
{
    off = (long long)b * bt.stride;
    return !bt.mask || bt.mask[b] != 0;
}

// per-instance device scalars (isc, 8 doubles in each slab)
// I_IDT = 1/dt, formed on the host: a division per thread costs a dozen FP64-pipe operations
enum { I_DT = 0, I_CBAR0 = 1, I_LAM = 2, I_IDT = 3, I_NSC = 8 };

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------

__host__ __device__ inline int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// coordinate of a one-cell step s (|s| <= 1) from a on an axis of n cells: periodic
// wrap, or (Neumann) the cell itself when the step leaves the grid (mirror ghost)
__host__ __device__ inline int stepi(int a, int s, int n, int bc)
{
    const int b = a + s;
    if (bc) return (b < 0 || b >= n) ? a : b;
    return wrapi(b, n);
}

__host__ __device__ inline void coords_of(const DGrid &g, long long p, int &x, int &y, int &z)
{
    x = (int)(p % g.n[0]);
    long long q = p / g.n[0];
    y = (int)(q % g.n[1]);
    z = (int)(q / g.n[1]);
}

__host__ __device__ inline long long index_of(const DGrid &g, int x, int y, int z)
{
    return (long long)x + (long long)g.n[0] * ((long long)y + (long long)g.n[1] * z);
}

// neighbour of (x, y, z) shifted by (dx, dy, dz), each |d| <= 1: periodic, or the
// mirror ghost's cell with Neumann boundaries
__host__ __device__ inline long long nbr_of(const DGrid &g, int x, int y, int z, int dx, int dy, int dz)
{
    return index_of(g, stepi(x, dx, g.n[0], g.bc), stepi(y, dy, g.n[1], g.bc), stepi(z, dz, g.n[2], g.bc));
}

__device__ inline long long nbrJ(const DGrid &g, int x, int y, int z, int J, int s)
{
    return nbr_of(g, x, y, z, J == 0 ? s : 0, J == 1 ? s : 0, J == 2 ? s : 0);
}

// ---------------------------------------------------------------------------
// deterministic block reduction of K values (fixed tree, fixed grid)
// ---------------------------------------------------------------------------

// reduce K values over a block of any multiple of 32 threads (up to 1024) and
// store them as row blockIdx.x of partials
template <int K>
__device__ inline void block_reduce_store_n(double (&v)[K], double *partials /* [gridDim.x][K] */)
{
    __shared__ double red[K][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) {
        double a = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[k][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) a += red[threadIdx.x][w];
        partials[(size_t)blockIdx.x * K + threadIdx.x] = a;
    }
}

template <int K>
__device__ inline void block_reduce_store(double (&v)[K], double *partials /* [gridDim.x][K] */)
{
    block_reduce_store_n<K>(v, partials);
}

// Last-block finalisation: after every block stored its K partial sums, the
// block that finishes last adds the columns of all blocks' partials in a fixed
// order (lanes stride over blocks, then a fixed shuffle tree) and writes out[K];
// counter returns to zero.  The result does not depend on which block is last.
__device__ inline void grid_finalize(const double *partials, int K, double *out, unsigned int *counter)
{
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const volatile double *vp = partials;
    for (int k = warp; k < K; k += nw) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a += vp[(size_t)b * K + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) out[k] = a;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ---------------------------------------------------------------------------
// stencil / reduction kernels (nks_stencil.cu)
// ---------------------------------------------------------------------------

// isc: the instance's scalars (I_DT, I_CBAR0, I_LAM); rb: reduction blocks per instance
int launch_mobility(const DGrid &g, const DCoef &k, const double *c0, double *mob, cudaStream_t st, const Bat &bt);
int launch_trace0(const DGrid &g, const DCoef &k, const double *isc, const double *X0, double *tr0, cudaStream_t st,
                  const Bat &bt);
int launch_residual(const DGrid &g, const DCoef &k, const double *isc, int mode, const double *X1, const double *X0,
                    const double *tr0, const double *mob, double *Gc, double *sig, double *part, double *F, int *flag,
                    double *partials, int rb, cudaStream_t st, const Bat &bt);
// J v, or J P v with zsum[0] = sum of v_c (P: mean of v_c removed).
// FP64: two passes through the dG / sig temporaries (N and d(d+1)/2 N doubles).
int launch_jv64(const DGrid &g, const DCoef &k, const double *isc, int mode, const double *part, const double *mob,
                const double *v, double *dG, double *sig, double *Jv, cudaStream_t st, const Bat &bt,
                const double *zsum = nullptr);
// FP32 arithmetic and storage (FP32 copies of part and mob); prepare_jv32 sets the
// kernel attributes it needs (once per problem, before any graph capture)
void prepare_jv32(const DGrid &g, const DCoef &k);
int launch_jv32(const DGrid &g, const DCoef &k, const double *isc, int mode, const float *part, const float *mob,
                const float *v, float *Jv, cudaStream_t st, const Bat &bt, const double *zsum);
int launch_energy(const DGrid &g, const DCoef &k, const double *isc, const double *X, double *partials, int rb,
                  cudaStream_t st, const Bat &bt);
int launch_finalize(const double *partials, int nblocks, int K, double *out, cudaStream_t st, const Bat &bt);

// ---------------------------------------------------------------------------
// vector kernels (nks_krylov.cu); n entries per instance
// ---------------------------------------------------------------------------

int launch_axpby(long long n, double a, const double *x, double b, double *y, cudaStream_t st, const Bat &bt);
int launch_waxpy(long long n, const double *x, double a, const double *y, double *w, cudaStream_t st,
                 const Bat &bt);  // w = x + a y
// w = x + lam y with lam = isc[I_LAM] of the instance
int launch_waxpy_lam(long long n, const double *x, const double *isc, const double *y, double *w, cudaStream_t st,
                     const Bat &bt);
int launch_copy(long long n, const double *x, double *y, cudaStream_t st, const Bat &bt);
int launch_dot2(long long n, const double *x, const double *y, double *partials, int rb, cudaStream_t st,
                const Bat &bt);  // x.y, y.y
int launch_convert(long long n, const double *a, float *b, cudaStream_t st, const Bat &bt);
int launch_convert(long long n, const float *a, double *b, cudaStream_t st, const Bat &bt);

// GMRES(m) with right preconditioning; see nks_krylov.cu.  Solves J x = b for
// every instance with is[i].gin set, to is[i].gtol; leaves is[i].gits, is[i].res.
struct Problem;
int gmres_solve(Problem *P, int mode, const double *b, double *x);

// ---------------------------------------------------------------------------
// restricted additive Schwarz (nks_ras.cu)
// ---------------------------------------------------------------------------

struct RasPlan;
int ras_plan_create(Problem *P, std::string &err);     // shared tables; per-instance sizes
struct SlabItem {
    void **ptr;
    size_t bytes;
};
void ras_slab_items(Problem *P, std::vector<SlabItem> &items);  // per-instance Schwarz buffers
void ras_prepare_launch(Problem *P);                             // kernel attributes (before any capture)
void ras_plan_destroy(Problem *P);
// assemble J restricted + ILU(0) for the instances of bt (on: the same set on the host);
// a zero pivot marks the instance failed in is[]
int ras_factor(Problem *P, int mode, const Bat &bt, const std::vector<char> &on);
void ras_apply(Problem *P, const double *r, double *z, const Bat &bt);  // z = P RAS^-1 r
// z = RAS^-1 r without P (FP64 or FP32 vectors); the sum of z_c goes to zsum[0]
template <typename TV>
void ras_apply_t(Problem *P, const TV *r, TV *z, const Bat &bt);
template <typename TV>
void ras_apply_projected(Problem *P, const TV *r, TV *z, const Bat &bt);
// mixed precision: FP32 copies of part and mob for the FP32 Jacobian action
void refresh_f32_coefficients(Problem *P, const Bat &bt);
void project(Problem *P, double *z, const Bat &bt);   // with P
void ras_work(const Problem *P, double *bytes, double *flops);  // algorithmic work of one sweep

// ---------------------------------------------------------------------------
// problem object (nks_api.cu)
// ---------------------------------------------------------------------------

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
};

// per-class pool of event pairs, reused across steps
struct TimerPool {
    std::vector<Timer> ev;
    size_t used = 0;
};

// host state of one instance
struct IState {
    bool loaded = false;                        // holds a state (serving slots may be empty)
    // time stepping
    double t = 0.0, dt_prev = 0.0, zeta = 0.0, E = 0.0, Eprev = 0.0;
    long long nstep = 0;
    double cbar0 = 0.0;
    double dt = 0.0;                            // dt of the system being solved
    // Newton
    int nst = 0;                                // 1 running, 0 converged, < 0: -status
    double fn0 = 0.0, fn = 0.0, tol = 0.0, lam = 1.0, ftn = 0.0;
    int newton_its = 0, gmres_its = 0;
    bool searching = false, accepted = false, dom_ok = true;
    std::string err;
    // GMRES
    double beta = 0.0, gtol = 0.0, res = 0.0;
    int gits = 0;
    bool gin = false, cyc = false;
};

// device masks: Newton running set, GMRES (solving, in the current cycle, still
// iterating), line search, accepted, spare
enum { M_RUN = 0, M_GIN, M_CYC, M_ACT, M_LS, M_ACC, M_X1, M_X2, kMasks };

struct Problem {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    nks_allocator alloc{};
    bool have_alloc = false;
    std::vector<void *> allocations;

    nks_grid grid{};
    nks_coeffs coeffs{};
    nks_opts opts{};
    DGrid g{};
    DCoef k{};
    int nf = 2;
    long long N = 0, nvec = 0;
    long long ldv = 0;                          // stride of the Krylov basis: nvec rounded up to even
    int rb = kRedBlocks;                        // reduction blocks per instance (from the vector length)

    // batch: nb instances; per-instance buffers in slabs of stride bytes
    int nb = 1;
    long long stride = 0;
    char *slab = nullptr;
    int *dmask = nullptr;                       // kMasks x nb device masks
    int *hmask_ring = nullptr;                  // pinned staging ring for mask and scalar uploads
    double *hsc_ring = nullptr;
    int ring_pos = 0;
    double *isc = nullptr;                      // per-instance device scalars (I_DT, ...)
    double *hread = nullptr;                    // pinned: per-instance scalars read back (nb x 64)
    int *hflags = nullptr;                      // pinned: both flag words of every instance (nb x 2)

    // state
    double *Xn = nullptr, *Xprev = nullptr, *X = nullptr, *Xt = nullptr;
    double *F = nullptr, *Ft = nullptr, *S = nullptr, *B = nullptr;
    double *part = nullptr, *part_t = nullptr;  // 4 N: pointwise derivatives of G^1 + G^2 at X / Xt
    double *mob = nullptr;                      // d N edge mobilities at level n
    double *tr0 = nullptr;                      // N: trace of eps^el at level n
    double *Gc = nullptr, *sig = nullptr;       // residual / Jv temporaries
    double *partials = nullptr;                 // kRedBlocks * 64
    double *dscal = nullptr;                    // small device scalars
    int *dflag = nullptr;
    double *zsum = nullptr;                     // sum of z_c of the last Schwarz sweep (device)
    float *partf = nullptr, *mobf = nullptr;    // mixed precision: FP32 copies of part and mob for J v
    unsigned int *tickets = nullptr;            // last-block counters of the fused reductions (start at 0)

    // Krylov workspace
    double *V = nullptr;                        // (m + 1) ldv, FP64 basis
    double *W = nullptr, *Z = nullptr, *R = nullptr;
    double *T64 = nullptr;                      // FP64 J x of the true residual
    float *Vf = nullptr, *Wf = nullptr, *Zf = nullptr;  // FP32 basis and Arnoldi vectors (mixed precision)
    long long ldvf = 0;                         // FP32 basis stride: nvec rounded up to a multiple of 4
    double *gm = nullptr;                       // device GMRES small state

    RasPlan *ras = nullptr;

    int cur_mode = 0;                           // 0 full system, 1 displacement only

    // per-instance host state
    std::vector<IState> is;

    nks_stats stats{};
    TimerPool timers[NKS_NCLASS];
    // captured GMRES iterations: [mode][j], with the counters one replay adds
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        long long launches[NKS_NCLASS] = {};
    };
    IterGraph graphs[2][kMaxRestart];
    bool graphs_off = false;                    // a capture failed: launch directly
    bool f32 = false;                           // the FP32 buffers of the mixed form exist
    // does a linear solve of this mode run in the mixed form (FP32 factors, sweeps, basis)?
    bool inner_f32(int mode) const { return opts.precision == NKS_MIXED || (mode == 1 && opts.u0_mixed); }
    int withhold_copy = 0;                      // test hook: sweeps withhold their first factor copy
    std::string err;

    void *dalloc(size_t bytes);
    void dfree_all();
    // batch helpers (nks_api.cu)
    Bat all() const { return Bat{stride, nullptr, nb}; }
    Bat masked(int m) const { return Bat{stride, dmask + (size_t)m * nb, nb}; }
    Bat set_mask(int m, const std::vector<char> &on);   // upload mask m, return its Bat
    void upload_isc();                                  // isc of every instance from is[]
    // count (<= I_NSC) doubles per instance, host rows[i * count + q], to dev0 (instance 0's
    // address) + the slab stride; staged through the pinned ring, no synchronisation
    void upload_rows(double *dev0, const double *rows, int count);
    int read_scalars(const double *dev0, int count, const char *where);  // -> hread[b * 64 + i], hflags
    int read_flags(const char *where);                                   // -> hflags[2 b + q]
    void enqueue_readback(const double *dev0, int count);                // the copies of read_scalars
    void count(int n) { stats.kernel_launches += n; }  // kernels launched on this problem
    void tick(int cls);                         // count a launch of class cls (and start a timer)
    void tock(int cls);                         // stop its timer
    int sync_check(const char *where);
};

int cuda_fail(Problem *P, cudaError_t e, const char *where);
void destroy_graphs(Problem *P);
DCoef derive_coefficients(const nks_coeffs &c, int dim, double cbar0);  // App. B reduction
void set_thread_error(const char *msg);                                 // for nks_last_error(NULL)

}  // namespace nks
