// nks_ras.cu -- restricted additive Schwarz with ILU(0) subdomain solves.
//
// Sec. 4 preconditions GMRES with a Schwarz method over a box decomposition
// (one subdomain per core in the paper); Sec. 5.4 selects ILU(0) reused for
// the whole time step.  Here one overlapping subdomain is one thread block:
//
//   * plan (host, once): per subdomain the overlapped box, its owned part and
//     its wavefront levels lv = x + 2y + 3z, which order every lower
//     neighbour of a point (every column left of the diagonal in the exact
//     Jacobian pattern, x-fastest point-interleaved numbering) before the
//     point itself;
//   * factor (device, once per time step): assemble J restricted to the box
//     (columns outside it dropped) and run ILU(0) row by row, all points of a
//     level in parallel, level after level;
//   * apply (device, every GMRES iteration): gather r on the box into shared
//     memory, forward and backward sweeps level by level, write the owned
//     points (restricted prolongation, no atomics), then the projection P.
//
// Factor layout (level-major).  For each level the factors of its points form
// one block: a forward part with the strictly lower entries (rows of the
// pattern's lower slots, points contiguous within a row) and a backward part
// with the strictly upper entries and the inverse pivots.  Each part of a
// level is one contiguous, 16-byte aligned run, so one TMA bulk copy
// (cp.async.bulk + mbarrier) brings it into shared memory while the previous
// level is being computed; the dependent path touches shared memory only.
#include <math.h>
#include <type_traits>

#include <algorithm>
#include <set>
#include <tuple>
#include <utility>

#include "nks_internal.cuh"
#include "nks_pattern.cuh"

namespace nks {

struct SubInfo {
    int org[3];               // global coordinates of local (0,0,0) (may be negative: periodic)
    int L[3];                 // box extent
    int own0[3], own1[3];     // owned local range [own0, own1)
    int np, nlev;
    int px, py, npx;          // odd row pitches of the box vector and its padded size (bank-conflict free levels)
    int qx, qy, nqx;          // pitches and plane size of the FP32 sweep's branch-free layout: 1-D and 2-D
                              // boxes with kHalo zero cells around them, 3-D boxes the pitches above
    long long lvl_off;        // into lvl_ptr / lvl_blk (nlev + 1 entries)
    long long pos_off;        // into lvl_lp (np entries): packed coordinates x | y << 10 | z << 20
    long long fac_off;        // into the factor array (elements)
    long long scr_off;        // into the global scratch vector (nf * np), when not in shared memory
};

struct RasPlan {
    int nsub = 0, nslot = 0, nlow = 0, nup = 0;
    int threads = 64;
    int maxnp = 0;
    int maxnpx = 0;                 // largest padded box vector
    int maxcnt = 0;                 // most points in one wavefront level
    int maxnlev = 0;                // most wavefront levels of one box
    int npart = 0;                  // stage-A partial sums per point (largest of the two sweeps)
    long long maxblk = 0;           // largest forward or backward part of a level (elements)
    long long fac_elems = 0;
    // FP32 factors, point-major inside each level part: point k's forward values at
    // k * sf32, its backward values (strict upper, then inverse pivots) at k * sb32
    int sf32 = 0, sb32 = 0;
    long long maxblk32 = 0;         // largest FP32 level part (elements)
    long long fac32_elems = 0;
    long long nlev_all = 0;         // levels of all boxes
    long long *lvl_src = nullptr;   // FP64 factor offset of every level's block (nlev_all + 1 entries)
    int maxnqx = 0;                 // largest box plane with the halo
    int guard32 = 0;                // zero cells before and after the 3-D box planes (the stencil reach)
    int shape32 = 0;                // 1: every box has the compiled-in shape of its dimension
    bool halo32 = false;            // FP32 sweep on the branch-free layout (no neighbour bounds checks)
    long long scr_elems = 0;        // global scratch vector of the sweeps (when x is not in shared memory)
    long long total_np = 0;         // overlapped points of all subdomains
    bool x_smem = true;
    size_t smem_bytes = 0;          // dynamic shared memory of the apply kernel (FP64 factors)
    bool x_smem32 = true;
    int lane_bufs = 2;              // factor buffers of the FP32 sweep
    int blocks_per_sm32 = 1;        // resident FP32 sweep blocks per SM (plan estimate)
    size_t smem_bytes32 = 0;        // same for the FP32 factors of the mixed-precision mode
    SubInfo *sub = nullptr;
    // runtime copies of the pattern for the assembly kernel
    char4 *tmpl = nullptr;          // (dx, dy, dz, field) per slot
    short *st = nullptr;            // storage row per slot
    short *slotmap = nullptr;       // [f][(dz+2)*25 + (dy+2)*5 + (dx+2)][field] -> slot in row f, or -1
    int *upd_ptr = nullptr;         // ILU(0) update pairs of each lower slot
    short2 *upd = nullptr;          // (later slot b of row i, slot c of the same column in row k)
    int *lvl_ptr = nullptr, *lvl_lp = nullptr;
    long long *lvl_blk = nullptr;
    double *fac = nullptr;
    float *fac32 = nullptr;         // FP32 copy of the factors (mixed precision)
    double *scratch = nullptr;
    float *scratch32 = nullptr;
    double *proj = nullptr;         // projection sums
    int nmodes = 1;                 // null modes per displacement component
    int evenmask = 0;
    double rot_inorm[3] = {0.0, 0.0, 0.0};  // Neumann: 1/|rotation mode|^2 per plane (0: no mode)
    bool attr_set = false, attr_set32 = false;
};

// V: the pattern variant (bit 0: elasticity under Neumann boundaries, bit 1:
// three order parameters; see make_pattern)
template <int D, int NF, int V = 0>
struct Pat {
    static constexpr Pattern v = make_pattern<D, NF, V>();
};

template <int D, int NF, bool FWD, int V = 0>
struct SPlan {
    static constexpr SweepPlan v = make_sweep_plan<D, NF, FWD, V>();
};

template <int D, int NF, int V = 0>
struct Sched {
    static constexpr SweepPlan fwd = SPlan<D, NF, true, V>::v;
    static constexpr SweepPlan bwd = SPlan<D, NF, false, V>::v;
    static constexpr int ntask = fwd.ntask > bwd.ntask ? fwd.ntask : bwd.ntask;
    static constexpr int npart = fwd.npart > bwd.npart ? fwd.npart : bwd.npart;
};


// every (dimension, fields, pattern variant) the solver instantiates: the reduced
// model (variants 0, 1) and three order parameters (2, 3), without and with
// elasticity
#define NKS_PAT_CASES(X)                                                                                      \
    X(1, 2, 0) X(1, 3, 0) X(2, 2, 0) X(2, 4, 0) X(3, 2, 0) X(3, 5, 0) X(1, 3, 1) X(2, 4, 1) X(3, 5, 1)       \
    X(1, 4, 2) X(1, 5, 2) X(2, 4, 2) X(2, 6, 2) X(3, 4, 2) X(3, 7, 2) X(1, 5, 3) X(2, 6, 3) X(3, 7, 3)

static Pattern compile_time_pattern(int d, int nf, int var)
{
    switch (d * 100 + nf * 10 + var) {
#define NKS_PAT_CASE(D, NF, V) \
    case D * 100 + NF * 10 + V: return Pat<D, NF, V>::v;
        NKS_PAT_CASES(NKS_PAT_CASE)
#undef NKS_PAT_CASE
    }
    return Pattern{};
}

// the pattern variant of a problem: bit 0 for elasticity under Neumann boundaries,
// bit 1 for three order parameters
static int pat_var(const Problem *P)
{
    return (P->g.bc == NKS_NEUMANN && P->k.elastic ? 1 : 0) + (P->k.ne == 3 ? 2 : 0);
}

__host__ __device__ static inline long long pad4(long long n) { return (n + 3) & ~3LL; }

// centred staircase on an axis of n cells (n even) and the axes of rotation plane q
// (0: (0, 1), 1: (0, 2), 2: (1, 2)); see ModeMasks
__host__ __device__ inline double staircase(int x, int n) { return (double)((x + 1) / 2) - 0.25 * (double)n; }

__host__ __device__ constexpr int plane_axis(int q, int which)
{
    return which == 0 ? (q == 2 ? 1 : 0) : (q == 0 ? 1 : 2);
}

// Row stride of the FP32 point-major factor layout for n values per point: a
// multiple of 4 (16-byte loads) whose quotient by 4 is odd, so the 16-byte loads
// of 8 consecutive points fall in 8 distinct bank groups.
__host__ __device__ constexpr int pm_stride(int n)
{
    const int s = (n + 3) & ~3;
    return (s / 4) % 2 == 1 ? s : s + 4;
}

template <int D, int NF, int V = 0>
struct PM {
    static constexpr Pattern P = make_pattern<D, NF, V>();
    static constexpr int SF = pm_stride(P.nlow), SB = pm_stride(P.nup + NF), PP = P.nlow + P.nup + NF;
};

// zero cells on each side of the box in the halo layout: the stencil reach
constexpr int kHalo = 2;

// cells a thread gathers per pass in the FP32 sweep
constexpr int kGatherIlp = 4;

// box plane pitches compiled into the FP32 sweep for the common box shapes (every
// neighbour offset then an immediate): 3-D 18^3 boxes (16^3 owned, overlap 1) and
// 2-D 68^2 boxes (64^2 owned, overlap 2) on the branch-free layout
struct LaneShape {
    int qx, qy, l2;
};
constexpr LaneShape kShape3 = {19, 19, 18};
constexpr LaneShape kShape2 = {73, 72, 1};

// L2 prefetch distance (levels) of the FP32 sweep on 3-D boxes (measured on the
// 18^3 boxes of the 128^3 workload: 8 levels ahead 6% faster than none; on the
// 2-D boxes of the 1024^2 workload the copies land in time without it)
constexpr int kPrefetch3 = 8;

// Wavefront level of a box point.  Every lower neighbour of the stencil
// (offsets (1,-1,0), (1,0,-1), (0,1,-1) and the axis offsets) must lie on an
// earlier level, which the weights 1 < 2 < 3 give with the fewest levels; the
// plan checks it against the pattern.
__host__ __device__ static inline int wave(int x, int y, int z) { return x + 2 * y + 3 * z; }
__host__ __device__ static inline size_t pad16(size_t n) { return (n + 15) & ~(size_t)15; }

// dynamic shared memory of the apply kernel: barriers, point table, two level
// buffers, stage-A partial sums and (when it fits) the sub-vector
// the same for the one-thread-per-point sweep (FP32): no partial sums, kLaneBufs buffers
static size_t apply_smem_lane(const RasPlan *R, int nf, bool halo, bool with_x, int nbuf)
{
    size_t b = 32 + pad16((size_t)R->maxnp * (halo ? sizeof(unsigned short) : sizeof(int))) +
               pad16(2 * sizeof(int) * (size_t)(R->maxnlev + 1)) + nbuf * pad16((size_t)R->maxblk32 * sizeof(float));
    if (with_x)
        b += pad16(((size_t)(halo ? R->maxnqx : R->maxnpx) * nf + (halo ? 2 * (size_t)R->guard32 : 0)) *
                   sizeof(float));
    return b;
}

static size_t apply_smem(const RasPlan *R, int nf, size_t tsize, bool with_x)
{
    const int pstride = (R->maxcnt + 31) / 32 * 32;
    size_t b = 16 + pad16((size_t)R->maxnp * sizeof(int)) + pad16(2 * sizeof(int) * (size_t)(R->maxnlev + 1)) +
               2 * pad16((size_t)R->maxblk * tsize) + pad16((size_t)R->npart * pstride * tsize);
    if (with_x) b += pad16((size_t)R->maxnpx * nf * tsize);
    return b;
}

static int sweep_partials(int d, int nf, int bc)
{
    switch (d * 100 + nf * 10 + bc) {
#define NKS_NPART(D, NF, V) \
    case D * 100 + NF * 10 + V: return Sched<D, NF, V>::npart;
        NKS_PAT_CASES(NKS_NPART)
#undef NKS_NPART
    }
    return 0;
}

static int sweep_tasks(int d, int nf, int bc)
{
    switch (d * 100 + nf * 10 + bc) {
#define NKS_NTASK(D, NF, V) \
    case D * 100 + NF * 10 + V: return Sched<D, NF, V>::ntask;
        NKS_PAT_CASES(NKS_NTASK)
#undef NKS_NTASK
    }
    return 1;
}

static int fp64_sweep_regs(int d, int nf, int bc, bool xs);  // registers per thread of the FP64 sweep

static void sm_limits(int &nsm, int &smem_sm)
{
    int dev = 0;
    nsm = 152;
    smem_sm = 228 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    }
}

// Placement of the box vector of the FP64 sweep: in shared memory unless keeping
// it there costs a wave of blocks (FP64 boxes of 2-D workloads fill an SM's shared
// memory alone; resident boxes add throughput, the sweep being a latency-bound
// chain of levels per box, and measured on the 16x16-box 1024^2 workload the
// global-memory placement with every box resident is the faster one).
static void choose_x64(const Problem *P, RasPlan *R, int nf)
{
    int nsm, smem_sm;
    sm_limits(nsm, smem_sm);
    const int d = P->g.dim, ntask = sweep_tasks(d, nf, pat_var(P));
    const int wpt = std::max(1, std::min((R->maxcnt + 31) / 32, 32 / ntask));
    const int threads = ntask * wpt * 32;
    const long long blocks = (long long)R->nsub * std::max(1, P->nb);
    auto waves = [&](bool xs) -> long long {
        const size_t b = apply_smem(R, nf, sizeof(double), xs);
        const int regs = std::max(1, fp64_sweep_regs(d, nf, pat_var(P), xs));
        int per_sm = (int)((size_t)smem_sm / (b + 1024));
        per_sm = std::min(per_sm, 2048 / threads);
        per_sm = std::min(per_sm, 65536 / (threads * ((regs + 7) & ~7)));
        per_sm = std::max(1, per_sm);
        return (blocks + (long long)nsm * per_sm - 1) / ((long long)nsm * per_sm);
    };
    R->x_smem = apply_smem(R, nf, sizeof(double), true) <= 227 * 1024;
    if (R->x_smem && waves(false) < waves(true)) R->x_smem = false;
    R->smem_bytes = apply_smem(R, nf, sizeof(double), R->x_smem);
}

// Shared-memory layout of the FP32 sweep.  The box vector stays in shared memory
// (from global memory its level-to-level reads run several times slower); among
// the layouts that fit, the one with the fewest waves of blocks wins (each box
// is a latency-bound chain of levels, so resident boxes add throughput), then
// the halo layout (no neighbour bounds checks), then the third factor buffer.
static void choose_lane_config(const Problem *P, RasPlan *R, int nf)
{
    int nsm, smem_sm;
    sm_limits(nsm, smem_sm);
    const long long blocks = (long long)R->nsub * std::max(1, P->nb);
    // the branch-free layout needs 16-bit cell indices
    const bool halo_ok = R->maxnqx < 65536;
    struct Cand {
        bool halo;
        int nbuf;
    };
    const Cand cands[] = {{true, 3}, {true, 2}, {false, 3}, {false, 2}};
    long long best_waves = -1;
    for (const Cand &c : cands) {
        if (c.halo && !halo_ok) continue;
        const size_t b = apply_smem_lane(R, nf, c.halo, true, c.nbuf);
        if (b > 227 * 1024) continue;
        const int per_sm = std::max(1, std::min(32, (int)((size_t)smem_sm / (b + 1024))));
        const long long waves = (blocks + (long long)nsm * per_sm - 1) / ((long long)nsm * per_sm);
        if (best_waves < 0 || waves < best_waves) {
            best_waves = waves;
            R->halo32 = c.halo;
            R->lane_bufs = c.nbuf;
            R->blocks_per_sm32 = per_sm;
        }
    }
    R->x_smem32 = best_waves >= 0;
    if (!R->x_smem32) {
        R->halo32 = false;
        R->lane_bufs = 2;
    }
    R->smem_bytes32 = apply_smem_lane(R, nf, R->halo32, R->x_smem32, R->lane_bufs);
}

int ras_plan_create(Problem *P, std::string &err)
{
    RasPlan *R = new RasPlan();
    P->ras = R;
    const int d = P->g.dim, nf = P->nf;
    const Pattern CP = compile_time_pattern(d, nf, pat_var(P));
    if (CP.nf != nf) {
        err = "internal: no Jacobian pattern for this dimension";
        return NKS_EINVAL;
    }
    // the factor kernel's row capacity (k_ras_factor<CAP, ...>)
    for (int f = 0; f < nf; f++)
        if (CP.len[f] > (P->k.ne == 3 ? 100 : 84)) {
            err = "internal: a Jacobian row exceeds the factor kernel's row capacity";
            return NKS_EINVAL;
        }
    // every column left of the diagonal lies on an earlier wavefront level or at the same point
    for (int f = 0; f < nf; f++)
        for (int a = 0; a < CP.diag[f]; a++) {
            const int i = CP.rowoff[f] + a;
            const int lv = wave(CP.dx[i], CP.dy[i], CP.dz[i]);
            if (!((CP.dx[i] == 0 && CP.dy[i] == 0 && CP.dz[i] == 0) || lv < 0)) {
                err = "internal: wavefront ordering";
                return NKS_EINVAL;
            }
        }
    R->nslot = CP.rowoff[nf];
    R->nlow = CP.nlow;
    R->nup = CP.nup;
    const int per_pt = CP.nlow + CP.nup + nf;
    // runtime tables for the assembly kernel
    std::vector<char4> tmpl(R->nslot);
    std::vector<short> st(R->nslot), slotmap((size_t)nf * 125 * nf, -1);
    for (int f = 0; f < nf; f++)
        for (int a = 0; a < CP.len[f]; a++) {
            const int i = CP.rowoff[f] + a;
            tmpl[i] = make_char4(CP.dx[i], CP.dy[i], CP.dz[i], CP.fc[i]);
            st[i] = CP.st[i];
            slotmap[((size_t)f * 125 + (CP.dz[i] + 2) * 25 + (CP.dy[i] + 2) * 5 + (CP.dx[i] + 2)) * nf + CP.fc[i]] =
                (short)a;
        }
    // ILU(0) update lists: for row f and lower slot a (row k = p + o_a, field f_a), every
    // later slot b of row f whose column also appears among the upper entries of row k
    std::vector<int> upd_ptr(R->nslot + 1, 0);
    std::vector<short2> upd;
    for (int f = 0; f < nf; f++)
        for (int a = 0; a < CP.len[f]; a++) {
            const int ia = CP.rowoff[f] + a;
            upd_ptr[ia] = (int)upd.size();
            if (a >= CP.diag[f]) continue;
            const int fk = CP.fc[ia];
            for (int b = a + 1; b < CP.len[f]; b++) {
                const int ib = CP.rowoff[f] + b;
                const int rx = CP.dx[ib] - CP.dx[ia], ry = CP.dy[ib] - CP.dy[ia], rz = CP.dz[ib] - CP.dz[ia];
                for (int c = CP.diag[fk] + 1; c < CP.len[fk]; c++) {
                    const int ic = CP.rowoff[fk] + c;
                    if (CP.dx[ic] == rx && CP.dy[ic] == ry && CP.dz[ic] == rz && CP.fc[ic] == CP.fc[ib]) {
                        upd.push_back(make_short2((short)b, (short)c));
                        break;
                    }
                }
            }
        }
    upd_ptr[R->nslot] = (int)upd.size();

    int sub[3] = {1, 1, 1};
    for (int J = 0; J < d; J++) sub[J] = std::max(1, P->opts.sub[J]);
    const int delta = P->opts.overlap;
    R->nsub = sub[0] * sub[1] * sub[2];
    if ((long long)sub[0] * sub[1] * sub[2] > (long long)kRedBlocks * 64) {
        // one reduction partial per subdomain sweep
        err = "decomposition: too many subdomains";
        return NKS_EINVAL;
    }
    std::vector<SubInfo> infos(R->nsub);
    std::vector<int> lvl_ptr, lvl_lp;
    std::vector<long long> lvl_blk, lvl_src;
    R->sf32 = pm_stride(CP.nlow);
    R->sb32 = pm_stride(CP.nup + nf);
    long long fac_off = 0, scr_off = 0;
    for (int s2 = 0; s2 < sub[2]; s2++)
        for (int s1 = 0; s1 < sub[1]; s1++)
            for (int s0 = 0; s0 < sub[0]; s0++) {
                const int s = s0 + sub[0] * (s1 + sub[1] * s2);
                const int sidx[3] = {s0, s1, s2};
                SubInfo &si = infos[s];
                for (int J = 0; J < 3; J++) {
                    if (J < d && P->g.bc == NKS_NEUMANN) {
                        // Neumann: the overlapped box stops at the boundary (no wrap)
                        const int n = P->g.n[J];
                        const int o0 = (int)((long long)sidx[J] * n / sub[J]);
                        const int o1 = (int)((long long)(sidx[J] + 1) * n / sub[J]);
                        si.org[J] = std::max(0, o0 - delta);
                        si.L[J] = std::min(n, o1 + delta) - si.org[J];
                        si.own0[J] = o0 - si.org[J];
                        si.own1[J] = o1 - si.org[J];
                        if (o1 - o0 < 1) {
                            err = "decomposition: more subdomains than cells along an axis";
                            return NKS_EINVAL;
                        }
                    } else if (J < d) {
                        const int n = P->g.n[J];
                        const int o0 = (int)((long long)sidx[J] * n / sub[J]);
                        const int o1 = (int)((long long)(sidx[J] + 1) * n / sub[J]);
                        si.org[J] = o0 - delta;
                        si.L[J] = o1 - o0 + 2 * delta;
                        si.own0[J] = delta;
                        si.own1[J] = delta + o1 - o0;
                        if (o1 - o0 < 1 || si.L[J] > n - 2) {
                            err = "decomposition: every overlapped box must be at least 2 cells shorter than the "
                                  "grid along each axis (sub and overlap too large for the grid)";
                            return NKS_EINVAL;
                        }
                    } else {
                        si.org[J] = 0;
                        si.L[J] = 1;
                        si.own0[J] = 0;
                        si.own1[J] = 1;
                    }
                }
                si.np = si.L[0] * si.L[1] * si.L[2];
                R->maxnp = std::max(R->maxnp, si.np);
                // odd pitches: points of one wavefront level are (pitch - 2), (pitch_xy - 4), ... apart,
                // all odd, so their 8-byte accesses spread over the shared-memory banks
                si.px = si.L[0] | 1;
                si.py = d >= 2 ? (si.L[1] | 1) : 1;
                si.npx = si.px * si.py * si.L[2];
                R->maxnpx = std::max(R->maxnpx, si.npx);
                if (d <= 2) {
                    // kHalo zero cells around the box: every neighbour at a fixed offset
                    si.qx = (si.L[0] + 2 * kHalo) | 1;
                    si.qy = d >= 2 ? si.L[1] + 2 * kHalo : 1;
                } else {
                    // 3-D: the box's own (odd) pitches; a neighbour outside the box lands on
                    // another cell of the zero-filled planes or on the zero guard cells, and
                    // its factor entry is an exact zero
                    si.qx = si.px;
                    si.qy = si.py;
                    R->guard32 = std::max(R->guard32, 2 * si.qx * si.qy);  // |dx + qx dy + qx qy dz| <= 2 qx qy
                }
                si.nqx = si.qx * si.qy * si.L[2];
                R->maxnqx = std::max(R->maxnqx, si.nqx);
                R->total_np += si.np;
                const int nlev = wave(si.L[0] - 1, si.L[1] - 1, si.L[2] - 1) + 1;
                si.nlev = nlev;
                R->maxnlev = std::max(R->maxnlev, nlev);
                si.lvl_off = (long long)lvl_ptr.size();
                si.pos_off = (long long)lvl_lp.size();
                si.fac_off = fac_off;
                std::vector<std::vector<int>> bylev(nlev);
                for (int lz = 0; lz < si.L[2]; lz++)
                    for (int ly = 0; ly < si.L[1]; ly++)
                        for (int lx = 0; lx < si.L[0]; lx++)
                            bylev[wave(lx, ly, lz)].push_back(lx | (ly << 10) | (lz << 20));
                int cnt = 0;
                long long blk = 0;
                for (int l = 0; l < nlev; l++) {
                    lvl_ptr.push_back(cnt);
                    lvl_blk.push_back(blk);
                    for (int lp : bylev[l]) {
                        lvl_lp.push_back(lp);
                        cnt++;
                    }
                    const long long cp = pad4((long long)bylev[l].size());
                    R->maxblk = std::max(R->maxblk, std::max<long long>(CP.nlow, CP.nup + nf) * cp);
                    R->maxblk32 = std::max(R->maxblk32, (long long)std::max(R->sf32, R->sb32) * cp);
                    lvl_src.push_back(fac_off + blk);
                    R->maxcnt = std::max(R->maxcnt, (int)bylev[l].size());
                    blk += (long long)per_pt * cp;
                }
                lvl_ptr.push_back(cnt);
                lvl_blk.push_back(blk);
                fac_off += blk;
                si.scr_off = scr_off;
                scr_off += (long long)nf * si.npx;
            }
    R->npart = sweep_partials(d, nf, pat_var(P));
    {
        const LaneShape sh = d == 3 ? kShape3 : kShape2;
        bool uni = d >= 2;
        for (const SubInfo &si : infos) uni = uni && si.qx == sh.qx && si.qy == sh.qy && si.L[2] == sh.l2;
        R->shape32 = uni ? 1 : 0;
    }
    R->fac_elems = fac_off;
    R->nlev_all = (long long)lvl_src.size();
    lvl_src.push_back(fac_off);
    R->fac32_elems = fac_off / per_pt * (R->sf32 + R->sb32);
    choose_x64(P, R, nf);
    choose_lane_config(P, R, nf);
    const bool f32_sweeps = P->opts.precision == NKS_MIXED || (P->opts.u0_mixed && P->k.elastic);
    if (R->smem_bytes > 227 * 1024 || (f32_sweeps && R->smem_bytes32 > 227 * 1024)) {
        err = "decomposition: subdomain boxes too large for the Schwarz kernel (use more subdomains)";
        return NKS_EINVAL;
    }
    // null modes of the centred-difference strain: sign patterns over the even axes on a
    // periodic grid; with Neumann boundaries (mirror ghosts) the translations and the
    // discrete rotations of the planes whose two axes have an even number of cells
    R->evenmask = 0;
    for (int J = 0; J < d; J++)
        if (P->g.n[J] % 2 == 0 && P->g.bc == NKS_PERIODIC) R->evenmask |= 1 << J;
    R->nmodes = 1 << __builtin_popcount(R->evenmask);
    for (int q = 0; q < 3; q++) {
        const int A = plane_axis(q, 0), B = plane_axis(q, 1);
        R->rot_inorm[q] = 0.0;
        if (P->g.bc != NKS_NEUMANN || B >= d || P->g.n[A] % 2 || P->g.n[B] % 2) continue;
        // |m|^2 = sum over the grid of S_B(x_B)^2 + S_A(x_A)^2
        double sa = 0.0, sb = 0.0;
        for (int x = 0; x < P->g.n[A]; x++) sa += staircase(x, P->g.n[A]) * staircase(x, P->g.n[A]);
        for (int x = 0; x < P->g.n[B]; x++) sb += staircase(x, P->g.n[B]) * staircase(x, P->g.n[B]);
        R->rot_inorm[q] = 1.0 / ((double)P->N / P->g.n[B] * sb + (double)P->N / P->g.n[A] * sa);
    }

    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        *dst = P->dalloc(bytes);
        if (!*dst) return false;
        cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        return true;
    };
    bool ok = up((void **)&R->tmpl, tmpl.data(), tmpl.size() * sizeof(char4)) &&
              up((void **)&R->st, st.data(), st.size() * sizeof(short)) &&
              up((void **)&R->slotmap, slotmap.data(), slotmap.size() * sizeof(short)) &&
              up((void **)&R->upd_ptr, upd_ptr.data(), upd_ptr.size() * sizeof(int)) &&
              up((void **)&R->upd, upd.data(), std::max<size_t>(1, upd.size()) * sizeof(short2)) &&
              up((void **)&R->sub, infos.data(), infos.size() * sizeof(SubInfo)) &&
              up((void **)&R->lvl_ptr, lvl_ptr.data(), lvl_ptr.size() * sizeof(int)) &&
              up((void **)&R->lvl_blk, lvl_blk.data(), lvl_blk.size() * sizeof(long long)) &&
              up((void **)&R->lvl_lp, lvl_lp.data(), lvl_lp.size() * sizeof(int)) &&
              up((void **)&R->lvl_src, lvl_src.data(), lvl_src.size() * sizeof(long long));
    if (!ok) {
        err = "out of device memory (Schwarz tables)";
        return NKS_ENOMEM;
    }
    R->scr_elems = scr_off;
    P->stats.factor_bytes = (long long)(sizeof(double) * (size_t)fac_off);
    P->stats.schwarz_points = (double)R->total_np;
    ras_work(P, &P->stats.schwarz_bytes, &P->stats.schwarz_flops);
    return NKS_OK;
}

void ras_plan_destroy(Problem *P)
{
    delete P->ras;
    P->ras = nullptr;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

namespace {

template <int B, int E, class Fn>
__device__ __forceinline__ void static_for(Fn &&fn)
{
    if constexpr (B < E) {
        fn(std::integral_constant<int, B>{});
        static_for<B + 1, E>(fn);
    }
}

__host__ __device__ inline bool inbox(const SubInfo &si, int lx, int ly, int lz)
{
    return lx >= 0 && lx < si.L[0] && ly >= 0 && ly < si.L[1] && lz >= 0 && lz < si.L[2];
}

struct FacTables {
    int rowoff[kMaxNf + 1], len[kMaxNf], diag[kMaxNf];
    int nlow, nup, nf;
};

// adds the contributions of one Jacobian row into a slot-indexed row (columns
// outside the box dropped); MASK: also mark the slots the row's paths reach
template <bool MASK>
struct DevAcc {
    double *vals;
    unsigned long long *pres;  // bit s: a path of the row ends in slot s (the row's own pattern)
    const short *slotmap;  // block of row f
    int nf, lx, ly, lz;
    const SubInfo *si;
    int gx, gy, gz;        // the row's point in the grid
    int n0, n1, n2, bc;    // grid extents, boundary kind
    // end of the path o then e from the row's point, as an offset: the sum on a
    // periodic grid; with Neumann boundaries each step stays on the cell where it
    // would leave the grid (mirror ghost)
    __host__ __device__ void end(int o, int e, int g, int n, int &d) const
    {
        const int a = stepi(g, o, n, bc);
        d = bc ? stepi(a, e, n, bc) - g : o + e;
    }
    __host__ __device__ void operator()(int ox, int oy, int oz, int ex, int ey, int ez, int fc, double v)
    {
        int dx, dy, dz;
        end(ox, ex, gx, n0, dx);
        end(oy, ey, gy, n1, dy);
        end(oz, ez, gz, n2, dz);
        if (!inbox(*si, lx + dx, ly + dy, lz + dz)) return;
        const int s = slotmap[((dz + 2) * 25 + (dy + 2) * 5 + (dx + 2)) * nf + fc];
        if (s >= 0) {
            vals[s] += v;
            if constexpr (MASK) pres[s >> 6] |= 1ull << (s & 63);
        }
    }
    // -1 when the one-cell step o stays on the cell (Neumann boundary), else 1
    __host__ __device__ double flip(int ox, int oy, int oz) const
    {
        if (!bc) return 1.0;
        const bool out = gx + ox < 0 || gx + ox >= n0 || gy + oy < 0 || gy + oy >= n1 || gz + oz < 0 || gz + oz >= n2;
        return out ? -1.0 : 1.0;
    }
};

// Fused assembly + ILU(0) (textbook IKJ order within a row) of J restricted to
// each overlapped box.  Rows of earlier points are final when a level starts.
// NE: the order parameters (1 or 3); the row is accumulated in per-thread memory of
// the pattern's longest row (83 entries with one order parameter, 97 with three).
// MASK: the pattern is a union over boundary situations (elasticity under Neumann
// boundaries), so each point's fill is kept to its own slots.
template <int NE, bool MASK>
__global__ void k_ras_factor(DGrid g, DCoef k, Bat bt, const double *__restrict__ isc, int mode, FacTables T,
                             const SubInfo *__restrict__ subs,
                             const int *__restrict__ lvl_ptr, const long long *__restrict__ lvl_blk,
                             const int *__restrict__ lvl_lp, const char4 *__restrict__ tmpl,
                             const short *__restrict__ st, const short *__restrict__ slotmap,
                             const int *__restrict__ upd_ptr, const short2 *__restrict__ upd,
                             const double *__restrict__ part, const double *__restrict__ mob,
                             double *__restrict__ fac, int *__restrict__ flag)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    part = shift(part, io);
    mob = shift(mob, io);
    fac = shift(fac, io);
    flag = shift(flag, io);
    const double dt = shift(isc, io)[I_DT];
    const SubInfo si = subs[blockIdx.x];
    const int nf = T.nf, D = g.dim;
    const int *lptr = lvl_ptr + si.lvl_off;
    const long long *lblk = lvl_blk + si.lvl_off;
    const int *lp_of = lvl_lp + si.pos_off;
    double *F = fac + si.fac_off;
    const long long N = g.N;
    constexpr int CAP = NE == 3 ? 100 : 84;
    double vals[CAP];
    for (int lev = 0; lev < si.nlev; lev++) {
        const long long cp = pad4((long long)(lptr[lev + 1] - lptr[lev]));
        double *blk = F + lblk[lev];
        for (int i = lptr[lev] + threadIdx.x; i < lptr[lev + 1]; i += blockDim.x) {
            const int kk = i - lptr[lev];
            const int pk = lp_of[i];
            const int lx = pk & 1023, ly = (pk >> 10) & 1023, lz = pk >> 20;
            const int gx = wrapi(si.org[0] + lx, g.n[0]), gy = wrapi(si.org[1] + ly, g.n[1]),
                      gz = wrapi(si.org[2] + lz, g.n[2]);
            const long long gp = index_of(g, gx, gy, gz);
            RowCtx rc;  // mode 0 fills every entry the rows read; mode 1 reads none
            if (mode == 0) {
                // pointwise block part[(a * (1 + ne) + b) N + p] = dG_a / dx_b, x = (c, eta_1..eta_ne)
                constexpr int ne = NE, w = 1 + NE;
                rc.a0[0] = part[gp];
                for (int j = 0; j < ne; j++) {
                    rc.a1[0][j] = part[(1 + j) * N + gp];
                    rc.a2[j] = part[(long long)(1 + j) * w * N + gp];
                    for (int i = 0; i < ne; i++) rc.a3[j][i] = part[((long long)(1 + j) * w + 1 + i) * N + gp];
                }
                for (int J = 0; J < D; J++) {
                    const long long pp = nbrJ(g, gx, gy, gz, J, +1), pm = nbrJ(g, gx, gy, gz, J, -1);
                    rc.a0[1 + 2 * J] = part[pp];
                    rc.a0[2 + 2 * J] = part[pm];
                    for (int j = 0; j < ne; j++) {
                        rc.a1[1 + 2 * J][j] = part[(1 + j) * N + pp];
                        rc.a1[2 + 2 * J][j] = part[(1 + j) * N + pm];
                    }
                    rc.Mp[J] = mob[J * N + gp];
                    rc.Mm[J] = mob[J * N + pm];
                }
            }
            for (int f = 0; f < nf; f++) {
                const int len = T.len[f], r0 = T.rowoff[f];
                for (int a = 0; a < len; a++) vals[a] = 0.0;
                // the slots this row's point has: with Neumann boundaries the compile-time
                // pattern is the union over all places in the grid, and ILU(0) fills only
                // the point's own pattern (as on a periodic grid, where they coincide)
                unsigned long long pres[2] = {0ull, 0ull};
                DevAcc<MASK> acc{vals, pres, slotmap + (size_t)f * 125 * nf, nf, lx, ly, lz, &si, gx, gy, gz, g.n[0],
                                 g.n[1], g.n[2], g.bc};
                jac_row<NE>(acc, f, k, D, g.h, dt, mode, rc);
                for (int a = 0; a < T.diag[f]; a++) {
                    const char4 o = tmpl[r0 + a];
                    const int nx = lx + o.x, ny = ly + o.y, nz = lz + o.z;
                    if (!inbox(si, nx, ny, nz)) continue;  // stays exactly 0
                    const int fk = o.w;
                    // level-major position of the earlier point (points of a level are stored in lp order)
                    const int lv = wave(nx, ny, nz);
                    const int lpk = nx | (ny << 10) | (nz << 20);  // points of a level are stored in this key's order
                    int lo = lptr[lv], hi = lptr[lv + 1] - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (lp_of[mid] < lpk) lo = mid + 1;
                        else hi = mid;
                    }
                    const int qk = lo - lptr[lv];
                    const long long qcp = pad4((long long)(lptr[lv + 1] - lptr[lv]));
                    const double *U = F + lblk[lv] + (long long)T.nlow * qcp;  // backward part of that level
                    const int rk = T.rowoff[fk];
                    const double l = vals[a] * U[(long long)st[rk + T.diag[fk]] * qcp + qk];  // times 1/u_kk
                    vals[a] = l;
                    // a_ib -= l * u_kb for every later column b of row i present in row k
                    for (int u = upd_ptr[r0 + a]; u < upd_ptr[r0 + a + 1]; u++) {
                        const short2 bc = upd[u];
                        if (!MASK || ((pres[bc.x >> 6] >> (bc.x & 63)) & 1ull))
                            vals[bc.x] -= l * U[(long long)st[rk + bc.y] * qcp + qk];
                    }
                }
                const double piv = vals[T.diag[f]];
                if (piv == 0.0 || !isfinite(piv)) atomicOr(flag, 2);
                for (int a = 0; a < len; a++) {
                    const int ia = r0 + a;
                    if (a < T.diag[f]) blk[(long long)st[ia] * cp + kk] = vals[a];
                    else if (a > T.diag[f]) blk[((long long)T.nlow + st[ia]) * cp + kk] = vals[a];
                    else blk[((long long)T.nlow + st[ia]) * cp + kk] = 1.0 / piv;
                }
            }
        }
        __syncthreads();
    }
}

// ---- TMA bulk copies and mbarriers (inline PTX) ---------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: gives up after ~2^31 clocks (about a second) and reports it
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}

// is the neighbour at the compile-time offset (DX, DY, DZ) inside the box?
template <int DX, int DY, int DZ>
__device__ __forceinline__ bool nb_inbox(int lx, int ly, int lz, const SubInfo &si)
{
    bool ok = true;
    if constexpr (DX < 0) ok = ok && lx >= -DX;
    if constexpr (DX > 0) ok = ok && lx < si.L[0] - DX;
    if constexpr (DY < 0) ok = ok && ly >= -DY;
    if constexpr (DY > 0) ok = ok && ly < si.L[1] - DY;
    if constexpr (DZ < 0) ok = ok && lz >= -DZ;
    if constexpr (DZ > 0) ok = ok && lz < si.L[2] - DZ;
    return ok;
}

// sum over pattern slots [B, E) of stored entries times x at their columns (see row_dot)
template <int D, int NF, int B, int E, typename T, int V>
__device__ __forceinline__ T slot_sum(const T *__restrict__ part, long long cp, int k, const T *x, int np, int lp,
                                      int lx, int ly, int lz, const SubInfo &si, int sy, int sz)
{
    T s = (T)0;
    static_for<B, E>([&](auto ic) {
        constexpr int a = decltype(ic)::value;
        constexpr int dx = Pat<D, NF, V>::v.dx[a], dy = Pat<D, NF, V>::v.dy[a], dz = Pat<D, NF, V>::v.dz[a];
        constexpr int fc = Pat<D, NF, V>::v.fc[a];
        constexpr int row = Pat<D, NF, V>::v.st[a];
        const bool ok = nb_inbox<dx, dy, dz>(lx, ly, lz, si);
        const int idx = ok ? lp + dx + sy * dy + sz * dz : lp;
        s += part[row * cp + k] * x[fc * np + idx];
    });
    return s;
}

// Stage A of one sweep over a level: task t of the compile-time schedule for point k.
template <int D, int NF, bool FWD, typename T, int V>
__device__ __forceinline__ void stage_a(int task, int kk, int lp, int lx, int ly, int lz, const T *B, long long cp,
                                        T *x, int np, T *pt, int pstride, const SubInfo &si, int sy, int sz)
{
    using SP = SPlan<D, NF, FWD, V>;
    static_for<0, SP::v.ntask>([&](auto ti) {
        constexpr int t = decltype(ti)::value;
        if (task != t) return;
        constexpr int f = SP::v.t_row[t];
        constexpr int tb = SP::v.t_b[t], te = SP::v.t_e[t], tp = SP::v.t_part[t];
        constexpr int drow = Pat<D, NF, V>::v.nup + f;  // inverse pivot row in the backward part
        const T s = slot_sum<D, NF, tb, te, T, V>(B, cp, kk, x, np, lp, lx, ly, lz, si, sy, sz);
        if constexpr (tp >= 0) {
            pt[tp * pstride + kk] = s;
        } else if constexpr (FWD) {
            x[f * np + lp] -= s;
        } else {
            x[f * np + lp] = (x[f * np + lp] - s) * B[(long long)drow * cp + kk];
        }
    });
}

// Stage B: rows of one point finished from their partials and same-point entries, in sweep order.
template <int D, int NF, bool FWD, typename T, int V>
__device__ __forceinline__ void stage_b(int kk, int lp, int lx, int ly, int lz, const T *B, long long cp, T *x,
                                        int np, const T *pt, int pstride, const SubInfo &si, int sy, int sz)
{
    using SP = SPlan<D, NF, FWD, V>;
    static_for<0, NF>([&](auto fi) {
        constexpr int f = FWD ? decltype(fi)::value : NF - 1 - decltype(fi)::value;
        constexpr int stb = SP::v.row_stage_b[f];
        if constexpr (stb) {
            constexpr int sb = SP::v.same_b[f], se = SP::v.same_e[f], pb = SP::v.row_pb[f], pe = SP::v.row_pe[f];
            constexpr int drow = Pat<D, NF, V>::v.nup + f;
            T s = slot_sum<D, NF, sb, se, T, V>(B, cp, kk, x, np, lp, lx, ly, lz, si, sy, sz);
            static_for<pb, pe>([&](auto pi) {
                constexpr int q = decltype(pi)::value;
                s += pt[q * pstride + kk];
            });
            if constexpr (FWD) x[f * np + lp] -= s;
            else x[f * np + lp] = (x[f * np + lp] - s) * B[(long long)drow * cp + kk];
        }
    });
}

// One Schwarz subdomain per block: gather, forward and backward ILU(0) sweeps
// level by level (factor parts streamed by TMA one level ahead, two-stage
// schedule inside a level), restricted prolongation.  Threads are grouped in
// warps per stage-A task: warp w serves task w / wpt, points (w % wpt) * 32 + lane.
// XS: the box vector x lives in shared memory (a compile-time choice, so that its
// loads are shared-memory loads rather than generic ones), else in global scratch.
// nwb_req: warps sharing stage B (each on its own SM sub-partition; a partial warp
// occupies the FP64 pipe for less time than a full one, so spreading shortens the
// row chains but adds pipe time: 2 warps measured fastest on the 2-D 68^2 boxes at
// two boxes per SM, 4 on the 3-D 18^3 boxes).
template <int D, int NF, typename T, typename TV, bool XS, int V>
__global__ void __launch_bounds__(1024) k_ras_apply(DGrid g, Bat bt, const SubInfo *__restrict__ subs, const int *__restrict__ lvl_ptr,
                            const long long *__restrict__ lvl_blk, const int *__restrict__ lvl_lp,
                            const T *__restrict__ fac, const TV *__restrict__ r, TV *__restrict__ z,
                            T *__restrict__ scratch, int maxnp, int maxnlev, long long maxblk, int wpt, int nwb_req,
                            int pstride, int *flag, double *__restrict__ cpart, double *__restrict__ csum,
                            unsigned int *ticket, int withhold, int variant)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    fac = shift(fac, io);
    r = shift(r, io);
    z = shift(z, io);
    scratch = shift(scratch, io);
    flag = shift(flag, io);
    cpart = shift(cpart, io);
    csum = shift(csum, io);
    ticket = shift(ticket, io);
    constexpr Pattern PT = Pat<D, NF, V>::v;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int *lps = reinterpret_cast<int *>(smem + 16);
    // level tables: first point of each level, factor offset of each level block
    int *const slp = reinterpret_cast<int *>(smem + 16 + pad16((size_t)maxnp * sizeof(int)));
    int *const slo = slp + (maxnlev + 1);
    T *buf0 = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(slp) +
                                    pad16(2 * sizeof(int) * (size_t)(maxnlev + 1)));
    T *buf1 = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(buf0) + pad16((size_t)maxblk * sizeof(T)));
    T *pt = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(buf1) + pad16((size_t)maxblk * sizeof(T)));
    const SubInfo si = subs[blockIdx.x];
    T *x;
    if constexpr (XS)
        x = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(pt) +
                                  pad16((size_t)Sched<D, NF, V>::npart * pstride * sizeof(T)));
    else
        x = scratch + si.scr_off;
    const int np = si.np, nlev = si.nlev;  // x holds NF planes of si.npx (padded) entries
    const int *lptr = lvl_ptr + si.lvl_off;
    const long long *lblk = lvl_blk + si.lvl_off;
    const T *F = fac + si.fac_off;
    const long long N = g.N;
    const int sy = si.px, sz = si.px * si.py;
    const int npx = si.npx;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int task = warp / wpt, kq0 = (warp % wpt) * 32 + lane;
    const int nwb = min(nwb_req, (int)(blockDim.x >> 5));
    const int prod = blockDim.x - 1;  // the copy-issuing thread (its warp has the fewest stage-A points)
    const int nuse = 2 * nlev;  // forward parts of levels 0..nlev-1, then backward parts of nlev-1..0

    // the copy of use `it` into buffer it & 1
    auto issue = [&](int it) {
        if (withhold && it == 0) return;  // test hook: this copy never lands, the bounded wait expires
        const int lev = it < nlev ? it : 2 * nlev - 1 - it;
        const int cp = (slp[lev + 1] - slp[lev] + 3) & ~3;
        const T *src = F + slo[lev] + (it < nlev ? 0 : PT.nlow * cp);
        const uint32_t bytes = (uint32_t)((it < nlev ? PT.nlow : PT.nup + NF) * cp * (long long)sizeof(T));
        uint64_t *b = &bar[it & 1];
        fence_proxy_async();
        mbar_expect_tx(b, bytes);
        bulk_g2s((it & 1) ? buf1 : buf0, src, bytes, b);
    };

    if (tid == prod) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    for (int i = tid; i <= nlev; i += blockDim.x) {
        slp[i] = lptr[i];
        slo[i] = (int)lblk[i];
    }
    __syncthreads();
    if (tid == prod) issue(0);
    for (int i = tid; i < np; i += blockDim.x) lps[i] = lvl_lp[si.pos_off + i];
    // gather R_i^delta r (right-RAS: R_i^0 r, the owned points only), several points
    // per thread and pass with every load of the pass issued before the first store
    // (two for FP64 values: the 1024-thread bound leaves 64 registers)
    constexpr int G = sizeof(T) == 8 ? 2 : kGatherIlp;
    for (int q0 = tid; q0 < np; q0 += G * blockDim.x) {
        int lp[G];
        long long gp[G];
        bool take[G];
#pragma unroll
        for (int j = 0; j < G; j++) {
            const int q = q0 + j * blockDim.x;
            const int lx = q % si.L[0], ly = (q / si.L[0]) % si.L[1], lz = q / (si.L[0] * si.L[1]);
            lp[j] = lx + sy * ly + sz * lz;
            gp[j] = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                             wrapi(si.org[2] + lz, g.n[2]));
            take[j] = q < np && (variant != NKS_RIGHT_RAS ||
                                 (lx >= si.own0[0] && lx < si.own1[0] && ly >= si.own0[1] && ly < si.own1[1] &&
                                  lz >= si.own0[2] && lz < si.own1[2]));
        }
        T v[G][NF];
#pragma unroll
        for (int j = 0; j < G; j++)
#pragma unroll
            for (int f = 0; f < NF; f++) v[j][f] = take[j] ? (T)r[f * N + gp[j]] : (T)0;
#pragma unroll
        for (int j = 0; j < G; j++)
            if (q0 + j * blockDim.x < np)
#pragma unroll
                for (int f = 0; f < NF; f++) x[f * npx + lp[j]] = v[j][f];
    }
    __syncthreads();
    bool failed = false;
    for (int it = 0; it < nuse; it++) {
        if (tid == prod && it + 1 < nuse) issue(it + 1);
        const bool ok = mbar_wait_bounded(&bar[it & 1], (uint32_t)((it >> 1) & 1));
        const int lev = it < nlev ? it : 2 * nlev - 1 - it;
        const int base = slp[lev], cnt = slp[lev + 1] - base;
        const long long cp = pad4((long long)cnt);
        const T *B = (it & 1) ? buf1 : buf0;
        const bool fwd = it < nlev;
        // stage A: chunks of other-point entries, warp-uniform tasks
        if (ok)
            for (int kq = kq0; kq < cnt; kq += wpt * 32) {
                const int pk = lps[base + kq];
                const int lx = pk & 1023, ly = (pk >> 10) & 1023, lz = pk >> 20;
                const int lp = lx + sy * ly + sz * lz;
                if (fwd) stage_a<D, NF, true, T, V>(task, kq, lp, lx, ly, lz, B, cp, x, npx, pt, pstride, si, sy, sz);
                else stage_a<D, NF, false, T, V>(task, kq, lp, lx, ly, lz, B, cp, x, npx, pt, pstride, si, sy, sz);
            }
        __syncthreads();
        // stage B: one thread per point, the points spread over the first nwb warps
        // (one per SM sub-partition: their FP64 pipes run the row chains side by side)
        if (ok && warp < nwb)
            for (int k = lane * nwb + warp; k < cnt; k += 32 * nwb) {
                const int pk = lps[base + k];
                const int lx = pk & 1023, ly = (pk >> 10) & 1023, lz = pk >> 20;
                const int lp = lx + sy * ly + sz * lz;
                if (fwd) stage_b<D, NF, true, T, V>(k, lp, lx, ly, lz, B, cp, x, npx, pt, pstride, si, sy, sz);
                else stage_b<D, NF, false, T, V>(k, lp, lx, ly, lz, B, cp, x, npx, pt, pstride, si, sy, sz);
            }
        failed = __syncthreads_or(!ok);
        if (failed) break;
    }
    if (failed) {
        // a copy never completed: report it, let outstanding copies land (bounded), and
        // write nothing (the block still takes its turn in the sum below)
        if (tid == prod) {
            atomicOr(flag + 1, 4);
            mbar_wait_bounded(&bar[0], 0);
            mbar_wait_bounded(&bar[1], 0);
        }
    }
    if (variant != NKS_LEFT_RAS) {
        // overlapped prolongation (classical AS, right-RAS): the whole box solution goes
        // to the box's slot of the scratch vector; k_as_sum adds the boxes covering a point
        if (XS) {
            T *bo = scratch + si.scr_off;
            for (int i = failed ? NF * npx : tid; i < NF * npx; i += blockDim.x) bo[i] = x[i];
        }
        return;
    }
    // restricted prolongation: owned points only; the sum of the written z_c feeds the
    // projection's mean (FP64 per thread, fixed block tree, last block adds the blocks in order)
    double cs[1] = {0.0};
    for (int q = failed ? np : tid; q < np; q += blockDim.x) {
        const int lx = q % si.L[0], ly = (q / si.L[0]) % si.L[1], lz = q / (si.L[0] * si.L[1]);
        if (lx < si.own0[0] || lx >= si.own1[0] || ly < si.own0[1] || ly >= si.own1[1] || lz < si.own0[2] ||
            lz >= si.own1[2])
            continue;
        const int lp = lx + sy * ly + sz * lz;
        const long long gp = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                      wrapi(si.org[2] + lz, g.n[2]));
#pragma unroll
        for (int f = 0; f < NF; f++) z[f * N + gp] = (TV)x[f * npx + lp];
        cs[0] += (double)(TV)x[lp];
    }
    if (csum) {
        __syncthreads();
        block_reduce_store_n<1>(cs, cpart);
        grid_finalize(cpart, 1, csum, ticket);
    }
}

// All rows of one point in sweep order, from the point's own factor values Bk
// (point-major FP32 layout, 16-byte aligned): each row's full lower (forward) or
// upper (backward) part, including the same-point entries computed just before.
// HALO: every neighbour is read at a fixed offset from lp.  An entry whose
// column lies outside the box holds an exact 0 in the factors; in 1-D and 2-D
// it meets one of the kHalo zero cells around the box, in 3-D another finite
// cell of the zero-filled planes or a zero guard cell (0 times a finite value).
// Otherwise the neighbour is bounds-checked against the box and an outside
// column reads x at lp itself (times 0).
template <int D, int NF, bool FWD, bool HALO, int V>
__device__ __forceinline__ void point_rows_pm(const float *__restrict__ Bk, float *x, int npx, int lp, int lx, int ly,
                                              int lz, const SubInfo &si, int sy, int sz)
{
    constexpr Pattern PT = Pat<D, NF, V>::v;
    constexpr int NR = FWD ? PT.nlow : PT.nup + NF;
    constexpr int NV = (NR + 3) / 4;
    float4 bv[NV];
    static_for<0, NV>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        bv[j] = reinterpret_cast<const float4 *>(Bk)[j];
    });
    auto val = [&](auto rc) -> float {
        constexpr int r = decltype(rc)::value;
        if constexpr (r % 4 == 0) return bv[r / 4].x;
        else if constexpr (r % 4 == 1) return bv[r / 4].y;
        else if constexpr (r % 4 == 2) return bv[r / 4].z;
        else return bv[r / 4].w;
    };
    static_for<0, NF>([&](auto fi) {
        constexpr int f = FWD ? decltype(fi)::value : NF - 1 - decltype(fi)::value;
        constexpr int b = FWD ? PT.rowoff[f] : PT.rowoff[f] + PT.diag[f] + 1;
        constexpr int e = FWD ? PT.rowoff[f] + PT.diag[f] : PT.rowoff[f] + PT.len[f];
        float s = 0.f;
        static_for<b, e>([&](auto ic) {
            constexpr int a = decltype(ic)::value;
            constexpr int dx = PT.dx[a], dy = PT.dy[a], dz = PT.dz[a], fc = PT.fc[a];
            int idx;
            if constexpr (HALO) {
                static_assert(D == 3 || (dz == 0 && dx >= -kHalo && dx <= kHalo && dy >= -kHalo && dy <= kHalo),
                              "stencil reach beyond the halo");
                static_assert((dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz) <= 2,
                              "stencil reach beyond the guard cells");
                idx = lp + dx + sy * dy + sz * dz;
            } else {
                const bool ok = nb_inbox<dx, dy, dz>(lx, ly, lz, si);
                idx = ok ? lp + dx + sy * dy + sz * dz : lp;
            }
            s += val(std::integral_constant<int, PT.st[a]>{}) * x[fc * npx + idx];
        });
        if constexpr (FWD) x[f * npx + lp] -= s;
        else x[f * npx + lp] = (x[f * npx + lp] - s) * val(std::integral_constant<int, PT.nup + f>{});
    });
}

// The sweeps with one thread per point doing all its rows (every lower or upper
// entry, then the next row): one block barrier per level and no partial sums.
// Used for FP32 factors, where the per-point instruction stream is cheap and
// the latency of the two-stage schedule dominates; the FP64 pipe (1/64 rate)
// prefers the two-stage schedule's spread over warps.  Factor parts (point-major)
// are streamed by TMA NBUF - 1 levels ahead (and, for 3-D boxes, whose level parts
// are larger, prefetched into L2 kPrefetch3 levels ahead), issued by the block's last thread
// (its warp has the fewest points of a level, warp 0 the most); the level tables
// are copied to shared memory first (global loads on every level's critical path
// cost more than the arithmetic).  XS: x in shared memory; HALO: x on the
// branch-free layout (1-D and 2-D: kHalo zero cells around the box; 3-D: the
// box planes between `guard` zero cells on each side), the point table then
// holds 16-bit x indices.
template <int D, int NF, int NBUF, bool XS, bool HALO, bool SHAPE, int V>
__global__ void __launch_bounds__(256) k_ras_apply_lane(DGrid g, Bat bt, const SubInfo *__restrict__ subs, const int *__restrict__ lvl_ptr,
                            const long long *__restrict__ lvl_blk, const int *__restrict__ lvl_lp,
                            const float *__restrict__ fac, const float *__restrict__ r, float *__restrict__ z,
                            float *__restrict__ scratch, int maxnp, int maxnlev, long long maxblk, int *flag,
                            double *__restrict__ cpart, double *__restrict__ csum, unsigned int *ticket,
                            int withhold, int variant, int guard)
{
    static_assert(XS || !HALO, "the halo layout lives in shared memory");
    static_assert(HALO || !SHAPE, "compiled-in pitches are those of the branch-free layout");
    constexpr LaneShape SH = D == 3 ? kShape3 : kShape2;
    using T = float;
    using LT = typename std::conditional<HALO, unsigned short, int>::type;
    using L = PM<D, NF, V>;
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    fac = shift(fac, io);
    r = shift(r, io);
    z = shift(z, io);
    scratch = shift(scratch, io);
    flag = shift(flag, io);
    cpart = shift(cpart, io);
    csum = shift(csum, io);
    ticket = shift(ticket, io);
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    LT *lps = reinterpret_cast<LT *>(smem + 32);
    const size_t bstride = pad16((size_t)maxblk * sizeof(T)) / sizeof(T);
    // level tables: first point of each level, FP32 factor offset of each level block
    int *const slp = reinterpret_cast<int *>(smem + 32 + pad16((size_t)maxnp * sizeof(LT)));
    int *const slo = slp + (maxnlev + 1);
    T *const buf0 = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(slp) +
                                          pad16(2 * sizeof(int) * (size_t)(maxnlev + 1)));
    const SubInfo si = subs[blockIdx.x];
    T *x;
    if constexpr (XS) x = buf0 + NBUF * bstride + (HALO && D == 3 ? guard : 0);
    else x = scratch + si.scr_off;
    const int np = si.np, nlev = si.nlev;
    const int *lptr = lvl_ptr + si.lvl_off;
    const long long *lblk = lvl_blk + si.lvl_off;
    const T *F = fac + si.fac_off / L::PP * (L::SF + L::SB);
    const long long N = g.N;
    // x layout: NF planes of npx entries, local (lx, ly, lz) at l0 + lx + sy ly + sz lz
    const int sy = SHAPE ? SH.qx : (HALO ? si.qx : si.px);
    const int sz = SHAPE ? SH.qx * SH.qy : (HALO ? si.qx * si.qy : si.px * si.py);
    const int npx = SHAPE ? SH.qx * SH.qy * SH.l2 : (HALO ? si.nqx : si.npx);
    const int l0 = HALO && D <= 2 ? kHalo * (1 + (D >= 2 ? sy : 0)) : 0;
    const int tid = threadIdx.x;
    const int prod = blockDim.x - 1;  // the copy-issuing thread
    const int nuse = 2 * nlev;  // forward parts of levels 0..nlev-1, then backward parts of nlev-1..0

    // the copy of use `it` into buffer it % NBUF (NBUF - 1 levels ahead)
    auto issue = [&](int it) {
        if (withhold && it == 0) return;  // test hook: this copy never lands, the bounded wait expires
        const bool fw = it < nlev;
        const int lev = fw ? it : 2 * nlev - 1 - it;
        const int cp = (slp[lev + 1] - slp[lev] + 3) & ~3;
        const T *src = F + slo[lev] + (fw ? 0 : cp * L::SF);
        const uint32_t bytes = (uint32_t)((fw ? L::SF : L::SB) * cp * (long long)sizeof(T));
        if constexpr (D == 3) {
            const int iu = it + kPrefetch3;
            if (iu < nuse) {
                const bool fu = iu < nlev;
                const int lu = fu ? iu : 2 * nlev - 1 - iu;
                const int cu = (slp[lu + 1] - slp[lu] + 3) & ~3;
                bulk_prefetch_l2(F + slo[lu] + (fu ? 0 : cu * L::SF),
                                 (uint32_t)((fu ? L::SF : L::SB) * cu * sizeof(T)));
            }
        }
        uint64_t *b = &bar[it % NBUF];
        fence_proxy_async();
        mbar_expect_tx(b, bytes);
        bulk_g2s(buf0 + (it % NBUF) * bstride, src, bytes, b);
    };

    if (tid == prod) {
        for (int q = 0; q < NBUF; q++) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    for (int i = tid; i <= nlev; i += blockDim.x) {
        slp[i] = lptr[i];
        slo[i] = (int)(lblk[i] / L::PP * (L::SF + L::SB));
    }
    __syncthreads();
    if (tid == prod)
        for (int q = 0; q < NBUF - 1 && q < nuse; q++) issue(q);
    for (int i = tid; i < np; i += blockDim.x) {
        const int pk = lvl_lp[si.pos_off + i];
        if constexpr (HALO) lps[i] = (LT)(l0 + (pk & 1023) + sy * ((pk >> 10) & 1023) + sz * (pk >> 20));
        else lps[i] = pk;
    }
    auto owned = [&](int lx, int ly, int lz) {
        return lx >= si.own0[0] && lx < si.own1[0] && ly >= si.own0[1] && ly < si.own1[1] && lz >= si.own0[2] &&
               lz < si.own1[2];
    };
    // gather R_i^delta r (right-RAS: R_i^0 r, the owned points only); with the
    // branch-free layout every cell of the planes is written (zero outside the box),
    // and in 3-D the guard cells before and after the planes are zeroed
    if constexpr (HALO) {
        const int qy = D == 3 ? (SHAPE ? SH.qy : si.qy) : 1;
        // kGatherIlp cells per thread and pass: every load of the pass is issued before
        // the first value is stored (the gather is a latency-bound chain of global loads)
        constexpr int G = kGatherIlp;
        for (int q0 = tid; q0 < npx; q0 += G * blockDim.x) {
            int gp[G];
            bool take[G];
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int q = q0 + j * blockDim.x;
                int lx, ly, lz;
                if constexpr (D == 3) {
                    lx = q % sy;
                    ly = (q / sy) % qy;
                    lz = q / sz;
                } else {
                    lx = q % sy - kHalo;
                    ly = D >= 2 ? q / sy - kHalo : 0;
                    lz = 0;
                }
                const bool in = q < npx && lx >= 0 && lx < si.L[0] && ly >= 0 && ly < si.L[1] && lz < si.L[2];
                take[j] = in && (variant != NKS_RIGHT_RAS || owned(lx, ly, lz));
                gp[j] = take[j] ? (int)index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                                wrapi(si.org[2] + lz, g.n[2]))
                                : 0;
            }
            T v[G][NF];
#pragma unroll
            for (int j = 0; j < G; j++)
#pragma unroll
                for (int f = 0; f < NF; f++) v[j][f] = take[j] ? r[f * N + gp[j]] : (T)0;
#pragma unroll
            for (int j = 0; j < G; j++) {
                const int q = q0 + j * blockDim.x;
                if (q < npx)
#pragma unroll
                    for (int f = 0; f < NF; f++) x[f * npx + q] = v[j][f];
            }
        }
        if constexpr (D == 3)
            for (int q = tid; q < guard; q += blockDim.x) {
                x[q - guard] = (T)0;
                x[NF * npx + q] = (T)0;
            }
    } else {
        for (int q = tid; q < np; q += blockDim.x) {
            const int lx = q % si.L[0], ly = (q / si.L[0]) % si.L[1], lz = q / (si.L[0] * si.L[1]);
            const int lp = lx + sy * ly + sz * lz;
            const long long gp = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                          wrapi(si.org[2] + lz, g.n[2]));
            const bool take = variant != NKS_RIGHT_RAS || owned(lx, ly, lz);
#pragma unroll
            for (int f = 0; f < NF; f++) x[f * npx + lp] = take ? (T)r[f * N + gp] : (T)0;
        }
    }
    __syncthreads();
    bool failed = false;
    int failed_at = 0;
    for (int it = 0; it < nuse; it++) {
        // buffer (it + NBUF - 1) % NBUF last served use it - 1 (finished at the barrier)
        if (tid == prod && it + NBUF - 1 < nuse) issue(it + NBUF - 1);
        const bool ok = mbar_wait_bounded(&bar[it % NBUF], (uint32_t)((it / NBUF) & 1));
        const int lev = it < nlev ? it : 2 * nlev - 1 - it;
        const int base = slp[lev], cnt = slp[lev + 1] - base;
        const T *B = buf0 + (it % NBUF) * bstride;
        const bool fwd = it < nlev;
        if (ok)
            for (int k = tid; k < cnt; k += blockDim.x) {
                if constexpr (HALO) {
                    const int lp = lps[base + k];
                    if (fwd) point_rows_pm<D, NF, true, true, V>(B + k * L::SF, x, npx, lp, 0, 0, 0, si, sy, sz);
                    else point_rows_pm<D, NF, false, true, V>(B + k * L::SB, x, npx, lp, 0, 0, 0, si, sy, sz);
                } else {
                    const int pk = lps[base + k];
                    const int lx = pk & 1023, ly = (pk >> 10) & 1023, lz = pk >> 20;
                    const int lp = lx + sy * ly + sz * lz;
                    if (fwd) point_rows_pm<D, NF, true, false, V>(B + k * L::SF, x, npx, lp, lx, ly, lz, si, sy, sz);
                    else point_rows_pm<D, NF, false, false, V>(B + k * L::SB, x, npx, lp, lx, ly, lz, si, sy, sz);
                }
            }
        failed = __syncthreads_or(!ok);
        if (failed) {
            failed_at = it;
            break;
        }
    }
    if (failed) {
        // a copy never completed: report it, let outstanding copies land (bounded), and
        // write nothing (the block still takes its turn in the sum below)
        if (tid == prod) {
            atomicOr(flag + 1, 4);
            for (int u = failed_at; u < nuse && u < failed_at + NBUF; u++)
                mbar_wait_bounded(&bar[u % NBUF], (uint32_t)((u / NBUF) & 1));
        }
    }
    if (variant != NKS_LEFT_RAS) {
        // overlapped prolongation (classical AS, right-RAS): the box solution goes to the
        // box's slot of the scratch vector (unpadded box layout); k_as_sum adds the boxes
        // covering a point
        if (XS) {
            T *bo = scratch + si.scr_off;
            for (int q = failed ? np : tid; q < np; q += blockDim.x) {
                const int lx = q % si.L[0], ly = (q / si.L[0]) % si.L[1], lz = q / (si.L[0] * si.L[1]);
                const int lo = lx + si.px * ly + si.px * si.py * lz, lq = l0 + lx + sy * ly + sz * lz;
#pragma unroll
                for (int f = 0; f < NF; f++) bo[f * si.npx + lo] = x[f * npx + lq];
            }
        }
        return;
    }
    // restricted prolongation: owned points only; the sum of the written z_c feeds the
    // projection's mean (FP64 per thread, fixed block tree, last block adds the blocks in order)
    double cs[1] = {0.0};
    for (int q = failed ? np : tid; q < np; q += blockDim.x) {
        const int lx = q % si.L[0], ly = (q / si.L[0]) % si.L[1], lz = q / (si.L[0] * si.L[1]);
        if (!owned(lx, ly, lz)) continue;
        const int lp = l0 + lx + sy * ly + sz * lz;
        const long long gp = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                      wrapi(si.org[2] + lz, g.n[2]));
#pragma unroll
        for (int f = 0; f < NF; f++) z[f * N + gp] = x[f * npx + lp];
        cs[0] += (double)x[lp];
    }
    if (csum) {
        __syncthreads();
        block_reduce_store_n<1>(cs, cpart);
        grid_finalize(cpart, 1, csum, ticket);
    }
}

// Overlapped prolongation of classical AS and right-RAS: z at a grid point is
// the sum, over the boxes whose overlapped range covers it, of their solutions
// there, added in box-index order (a fixed order: deterministic sums).  Per
// axis the covering boxes are among the owner and its two neighbours; the sum
// of z_c feeds the projection's mean as in the restricted prolongation.
template <int NF, typename T, typename TV>
__global__ void __launch_bounds__(kRedThreads) k_as_sum(DGrid g, Bat bt, const SubInfo *__restrict__ subs, int sub0,
                                                        int sub1, int sub2, const T *__restrict__ bout,
                                                        TV *__restrict__ z, double *__restrict__ cpart,
                                                        double *__restrict__ csum, unsigned int *ticket)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    bout = shift(bout, io);
    z = shift(z, io);
    cpart = shift(cpart, io);
    csum = shift(csum, io);
    ticket = shift(ticket, io);
    const int sub[3] = {sub0, sub1, sub2};
    const int astride[3] = {1, sub0, sub0 * sub1};
    const int N = (int)g.N;
    double cs[1] = {0.0};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const int c3[3] = {p % g.n[0], (p / g.n[0]) % g.n[1], p / (g.n[0] * g.n[1])};
        int nb[3], bi[3][3], li[3][3];
#pragma unroll
        for (int J = 0; J < 3; J++) {
            nb[J] = 0;
            const int n = g.n[J], sb = sub[J], c = c3[J];
            if (J >= g.dim || sb == 1) {
                // one box along this axis (every box of a periodic single-box axis spans it)
                const SubInfo &b0 = subs[0];
                bi[J][0] = 0;
                li[J][0] = J >= g.dim ? 0 : ((c - b0.org[J]) % n + n) % n;
                nb[J] = 1;
                continue;
            }
            int s = (int)((long long)c * sb / n);
            while ((long long)s * n / sb > c) s--;
            while ((long long)(s + 1) * n / sb <= c) s++;
            // candidates in increasing box index
            int cand[3] = {(s + sb - 1) % sb, s, (s + 1) % sb};
            for (int a = 1; a < 3; a++)
                for (int q = a; q > 0 && cand[q - 1] > cand[q]; q--) {
                    const int t = cand[q];
                    cand[q] = cand[q - 1];
                    cand[q - 1] = t;
                }
            for (int a = 0; a < 3; a++) {
                if (a > 0 && cand[a] == cand[a - 1]) continue;
                const SubInfo &b = subs[cand[a] * astride[J]];
                const int l = ((c - b.org[J]) % n + n) % n;
                if (l < b.L[J]) {
                    bi[J][nb[J]] = cand[a];
                    li[J][nb[J]] = l;
                    nb[J]++;
                }
            }
        }
        T acc[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) acc[f] = (T)0;
        for (int i2 = 0; i2 < nb[2]; i2++)
            for (int i1 = 0; i1 < nb[1]; i1++)
                for (int i0 = 0; i0 < nb[0]; i0++) {
                    const int s = bi[0][i0] + sub0 * (bi[1][i1] + sub1 * bi[2][i2]);
                    const SubInfo &b = subs[s];
                    const int lp = li[0][i0] + b.px * (li[1][i1] + b.py * li[2][i2]);
                    const T *xb = bout + b.scr_off;
#pragma unroll
                    for (int f = 0; f < NF; f++) acc[f] += xb[f * b.npx + lp];
                }
#pragma unroll
        for (int f = 0; f < NF; f++) z[(long long)f * N + p] = (TV)acc[f];
        cs[0] += (double)(TV)acc[0];
    }
    block_reduce_store_n<1>(cs, cpart);
    grid_finalize(cpart, 1, csum, ticket);
}

// projection P: sums of z_c and of sign_m(p) z_uI for every null mode m.
// Mode mi is the sign pattern prod over the axes J in mask[mi] of (-1)^x_J.
// With Neumann boundaries (mirror ghosts) the null modes are the translations and,
// for every pair of axes I < J that both have an even number of cells, the discrete
// rotation u_I = -S_J(x_J), u_J = S_I(x_I), S(x) = floor((x + 1) / 2) - n / 4 (the
// centred staircase whose mirrored centred difference is 1/h at every cell, so the
// strain of the rotation vanishes).  Planes (0, 1), (0, 2), (1, 2); inorm[q] =
// 1 / |mode q|^2, or 0 for a plane without the mode.
struct ModeMasks {
    int m[8];
    double inorm[3];
};


// NU displacement components from field ku (NU = 0: the model without elasticity);
// NR rotation planes (Neumann boundaries: d(d-1)/2, else 0)
template <int NU, int NM, int NR, typename TV>
__global__ void __launch_bounds__(kRedThreads, 4) k_proj_dots(DGrid g, Bat bt, ModeMasks mm, int ku,
                                                              const TV *__restrict__ z, double *__restrict__ partials,
                                                              double *__restrict__ out, unsigned int *ticket)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    z = shift(z, io);
    partials = shift(partials, io);
    out = shift(out, io);
    ticket = shift(ticket, io);
    constexpr int K = 1 + NU * NM + NR;
    const long long N = g.N;
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; i++) acc[i] = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        acc[0] += (double)z[p];
        if constexpr (NU > 0) {
            int x, y, zz;
            coords_of(g, p, x, y, zz);
            const int par = (x & 1) | ((y & 1) << 1) | ((zz & 1) << 2);
#pragma unroll
            for (int mi = 0; mi < NM; mi++) {
                const double sg = (__popc(mm.m[mi] & par) & 1) ? -1.0 : 1.0;
#pragma unroll
                for (int I = 0; I < NU; I++) acc[1 + I * NM + mi] += sg * (double)z[(ku + I) * N + p];
            }
            if constexpr (NR > 0) {
                const int c3[3] = {x, y, zz};
#pragma unroll
                for (int q = 0; q < NR; q++) {
                    const int I = plane_axis(q, 0), J = plane_axis(q, 1);
                    acc[1 + NU * NM + q] += -staircase(c3[J], g.n[J]) * (double)z[(ku + I) * N + p] +
                                            staircase(c3[I], g.n[I]) * (double)z[(ku + J) * N + p];
                }
            }
        }
    }
    block_reduce_store<K>(acc, partials);
    grid_finalize(partials, K, out, ticket);
}

template <int NU, int NM, int NR, typename TV>
__global__ void k_proj_sub(DGrid g, Bat bt, ModeMasks mm, int ku, const double *__restrict__ sums,
                           TV *__restrict__ z)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    sums = shift(sums, io);
    z = shift(z, io);
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long N = g.N;
    if (p >= N) return;
    const double invN = 1.0 / (double)N;
    z[p] = (TV)((double)z[p] - sums[0] * invN);
    if constexpr (NU > 0) {
        int x, y, zz;
        coords_of(g, p, x, y, zz);
        const int par = (x & 1) | ((y & 1) << 1) | ((zz & 1) << 2);
        const int c3[3] = {x, y, zz};
#pragma unroll
        for (int I = 0; I < NU; I++) {
            double s = 0.0;
#pragma unroll
            for (int mi = 0; mi < NM; mi++) {
                const double sg = (__popc(mm.m[mi] & par) & 1) ? -1.0 : 1.0;
                s += sums[1 + I * NM + mi] * sg;
            }
            double r = 0.0;  // the rotation modes' values at p for component I, times their coefficients
#pragma unroll
            for (int q = 0; q < NR; q++) {
                const int A = plane_axis(q, 0), B = plane_axis(q, 1);
                const double a = sums[1 + NU * NM + q] * mm.inorm[q];
                if (I == A) r += a * -staircase(c3[B], g.n[B]);
                if (I == B) r += a * staircase(c3[A], g.n[A]);
            }
            z[(ku + I) * N + p] = (TV)((double)z[(ku + I) * N + p] - s * invN - r);
        }
    }
}

template <int NU, int NM, int NR, typename TV>
void launch_project_t(Problem *P, TV *z, const Bat &bt)
{
    const int ku = 1 + P->k.ne;
    RasPlan *R = P->ras;
    ModeMasks mm{};
    int mi = 0;
    for (int m = 0; m < (1 << P->g.dim); m++)
        if ((m & ~R->evenmask) == 0) mm.m[mi++] = m;
    for (int q = 0; q < 3; q++) mm.inorm[q] = R->rot_inorm[q];
    k_proj_dots<NU, NM, NR, TV><<<dim3(P->rb, bt.nb), kRedThreads, 0, P->stream>>>(P->g, bt, mm, ku, z, P->partials,
                                                                                    R->proj, P->tickets + 2);
    k_proj_sub<NU, NM, NR, TV><<<dim3((unsigned)((P->N + 255) / 256), bt.nb), 256, 0, P->stream>>>(
        P->g, bt, mm, ku, R->proj, z);
}

// FP32 copy of the factors in the point-major layout: level block i (FP64 offset
// lvl_src[i], cp padded points, rows of cp values) becomes cp rows of SF forward
// values then cp rows of SB backward values; the padding values are zero.
template <int D, int NF, int V>
__global__ void __launch_bounds__(256) k_fac_to_f32(Bat bt, long long nlev_all, const long long *__restrict__ lvl_src,
                                                    const double *__restrict__ a, float *__restrict__ b)
{
    long long io;
    if (!inst_off(bt, blockIdx.y, io)) return;
    a = shift(a, io);
    b = shift(b, io);
    using L = PM<D, NF, V>;
    constexpr int NL = L::P.nlow, NU = L::P.nup + NF;
    for (long long i = blockIdx.x; i < nlev_all; i += gridDim.x) {
        const long long s0 = lvl_src[i];
        const int cp = (int)((lvl_src[i + 1] - s0) / L::PP);
        const long long d0 = s0 / L::PP * (L::SF + L::SB);
        const int nfw = cp * L::SF, tot = cp * (L::SF + L::SB);
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            float v = 0.f;
            if (e < nfw) {
                const int k = e / L::SF, r = e - k * L::SF;
                if (r < NL) v = (float)a[s0 + (long long)r * cp + k];
            } else {
                const int e2 = e - nfw, k = e2 / L::SB, r = e2 - k * L::SB;
                if (r < NU) v = (float)a[s0 + (long long)(NL + r) * cp + k];
            }
            b[d0 + e] = v;
        }
    }
}

template <int D, int NF, int V>
void launch_fac_to_f32(Problem *P, const Bat &bt)
{
    RasPlan *R = P->ras;
    const unsigned nblk = (unsigned)std::min<long long>(R->nlev_all, 8 * 152);
    k_fac_to_f32<D, NF, V><<<dim3(nblk, bt.nb), 256, 0, P->stream>>>(bt, R->nlev_all, R->lvl_src, R->fac, R->fac32);
}

void launch_factor(Problem *P, int mode, const Bat &bt)
{
    RasPlan *R = P->ras;
    const Pattern CP = compile_time_pattern(P->g.dim, P->nf, pat_var(P));
    FacTables T{};
    for (int f = 0; f <= P->nf; f++) T.rowoff[f] = CP.rowoff[f];
    for (int f = 0; f < P->nf; f++) {
        T.len[f] = CP.len[f];
        T.diag[f] = CP.diag[f];
    }
    T.nlow = CP.nlow;
    T.nup = CP.nup;
    T.nf = P->nf;
    auto kern = P->k.ne == 3 ? (pat_var(P) & 1 ? k_ras_factor<3, true> : k_ras_factor<3, false>)
                             : (pat_var(P) & 1 ? k_ras_factor<1, true> : k_ras_factor<1, false>);
    // one thread per point of the largest level (a level's points are independent),
    // so every level is one round of row eliminations
    const int threads = std::min(256, std::max(64, (R->maxcnt + 31) / 32 * 32));
    kern<<<dim3(R->nsub, bt.nb), threads, 0, P->stream>>>(P->g, P->k, bt, P->isc, mode, T, R->sub, R->lvl_ptr, R->lvl_blk,
                                                     R->lvl_lp, R->tmpl, R->st, R->slotmap, R->upd_ptr, R->upd, P->part,
                                                     P->mob, R->fac, P->dflag);
}

using LaneKernel = void (*)(DGrid, Bat, const SubInfo *, const int *, const long long *, const int *, const float *,
                           const float *, float *, float *, int, int, long long, int *, double *, double *,
                           unsigned int *, int, int, int);

// the FP32 sweep instantiation of the plan's layout (three buffers and the
// branch-free layout only with x in shared memory)
template <int D, int NF, int V>
LaneKernel lane_kernel(const RasPlan *R)
{
    // the compiled-in box shapes are those of the periodic workloads (Neumann boxes
    // are clipped at the boundary)
    if constexpr (D >= 2 && V == 0)
        if (R->halo32 && R->shape32)
            return R->lane_bufs == 3 ? k_ras_apply_lane<D, NF, 3, true, true, true, V>
                                     : k_ras_apply_lane<D, NF, 2, true, true, true, V>;
    if (R->halo32) return R->lane_bufs == 3 ? k_ras_apply_lane<D, NF, 3, true, true, false, V>
                                            : k_ras_apply_lane<D, NF, 2, true, true, false, V>;
    if (!R->x_smem32) return k_ras_apply_lane<D, NF, 2, false, false, false, V>;
    return R->lane_bufs == 3 ? k_ras_apply_lane<D, NF, 3, true, false, false, V>
                             : k_ras_apply_lane<D, NF, 2, true, false, false, V>;
}

// the sweep kernel's dynamic shared memory limit (set once, before any graph capture)
template <int D, int NF, int V, typename TV>
void apply_attr(Problem *P)
{
    RasPlan *R = P->ras;
    constexpr bool f32 = sizeof(TV) == sizeof(float);
    const size_t smem = f32 ? R->smem_bytes32 : R->smem_bytes;
    bool &attr = f32 ? R->attr_set32 : R->attr_set;
    if (smem > 48 * 1024 && !attr) {
        if constexpr (f32) {
            cudaFuncSetAttribute(lane_kernel<D, NF, V>(R), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        } else {
            cudaFuncSetAttribute(k_ras_apply<D, NF, TV, TV, false, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            cudaFuncSetAttribute(k_ras_apply<D, NF, TV, TV, true, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        }
        attr = true;
    }
}

template <int D, int NF, int V>
void apply_attrs(Problem *P)
{
    apply_attr<D, NF, V, double>(P);
    if (P->f32) apply_attr<D, NF, V, float>(P);
}

// FP64 vectors use the FP64 factors; FP32 vectors (mixed precision) the FP32 copy
template <int D, int NF, int V, typename TV>
void launch_apply_t(Problem *P, const TV *r, TV *z, const Bat &bt)
{
    RasPlan *R = P->ras;
    const int ntask = Sched<D, NF, V>::ntask;
    const int wpt = std::max(1, std::min((R->maxcnt + 31) / 32, 32 / ntask));  // warps per stage-A task
    const int threads = ntask * wpt * 32;
    const int pstride = (R->maxcnt + 31) / 32 * 32;
    constexpr bool f32 = sizeof(TV) == sizeof(float);
    using T = TV;
    const size_t smem = f32 ? R->smem_bytes32 : R->smem_bytes;
    apply_attr<D, NF, V, TV>(P);
    const T *fac = f32 ? reinterpret_cast<const T *>(R->fac32) : reinterpret_cast<const T *>(R->fac);
    T *scr = f32 ? reinterpret_cast<T *>(R->scratch32) : reinterpret_cast<T *>(R->scratch);
    const int xs = f32 ? R->x_smem32 : R->x_smem;
    if constexpr (f32) {
        // one thread per point of the widest level
        const int tl = std::min(256, std::max(32, (R->maxcnt + 31) / 32 * 32));
        lane_kernel<D, NF, V>(R)<<<dim3(R->nsub, bt.nb), tl, smem, P->stream>>>(
            P->g, bt, R->sub, R->lvl_ptr, R->lvl_blk, R->lvl_lp, reinterpret_cast<const float *>(fac),
            reinterpret_cast<const float *>(r), reinterpret_cast<float *>(z), reinterpret_cast<float *>(scr), R->maxnp,
            R->maxnlev, R->maxblk32, P->dflag, P->partials, P->zsum, P->tickets + 3, P->withhold_copy, P->opts.ras_variant,
            R->guard32);
    } else {
        auto kern = xs ? k_ras_apply<D, NF, T, TV, true, V> : k_ras_apply<D, NF, T, TV, false, V>;
        kern<<<dim3(R->nsub, bt.nb), threads, smem, P->stream>>>(
            P->g, bt, R->sub, R->lvl_ptr, R->lvl_blk, R->lvl_lp, fac, r, z, scr, R->maxnp, R->maxnlev, R->maxblk, wpt,
            P->g.dim == 3 ? 4 : 2,
            pstride, P->dflag, P->partials, P->zsum, P->tickets + 3, P->withhold_copy, P->opts.ras_variant);
    }
    if (P->opts.ras_variant != NKS_LEFT_RAS) {
        int sub[3] = {1, 1, 1};
        for (int J = 0; J < P->g.dim; J++) sub[J] = std::max(1, P->opts.sub[J]);
        k_as_sum<NF, T, TV><<<dim3(P->rb, bt.nb), kRedThreads, 0, P->stream>>>(
            P->g, bt, R->sub, sub[0], sub[1], sub[2], scr, z, P->partials, P->zsum, P->tickets + 3);
    }
}

}  // namespace

static int fp64_sweep_regs(int d, int nf, int bc, bool xs)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaErrorInvalidValue;
    switch (d * 100 + nf * 10 + bc) {
#define NKS_REGS_CASE(D, NF, V)                                                                              \
    case D * 100 + NF * 10 + V:                                                                              \
        e = xs ? cudaFuncGetAttributes(&fa, k_ras_apply<D, NF, double, double, true, V>)                     \
               : cudaFuncGetAttributes(&fa, k_ras_apply<D, NF, double, double, false, V>);                   \
        break;
        NKS_PAT_CASES(NKS_REGS_CASE)
#undef NKS_REGS_CASE
    }
    return e == cudaSuccess ? fa.numRegs : 64;
}

// calls fn(D, NF, V) (integral constants) for the problem's instantiation
template <class Fn>
static void dispatch(const Problem *P, Fn &&fn)
{
    switch (P->g.dim * 100 + P->nf * 10 + pat_var(P)) {
#define NKS_DISPATCH_CASE(D, NF, V)                                                                          \
    case D * 100 + NF * 10 + V:                                                                              \
        fn(std::integral_constant<int, D>{}, std::integral_constant<int, NF>{}, std::integral_constant<int, V>{}); \
        break;
        NKS_PAT_CASES(NKS_DISPATCH_CASE)
#undef NKS_DISPATCH_CASE
    }
}
#define NKS_DISPATCH(FN, ...)                                                                                  \
    dispatch(P, [&](auto d_, auto nf_, auto v_) {                                                             \
        FN<decltype(d_)::value, decltype(nf_)::value, decltype(v_)::value>(__VA_ARGS__);                      \
    })

// factors of the instances of bt; an instance whose factorisation meets a zero
// pivot is marked failed (is[i].nst = -NKS_EPIVOT); on[i] mirrors bt's mask
int ras_factor(Problem *P, int mode, const Bat &bt, const std::vector<char> &on)
{
    cudaMemset2DAsync(P->dflag, (size_t)P->stride, 0, sizeof(int), (size_t)P->nb, P->stream);
    P->tick(3);
    launch_factor(P, mode, bt);
    P->count(1);
    P->tock(3);
    int rc = P->read_flags("ras_factor");
    if (rc) return rc;
    for (int i = 0; i < P->nb; i++) {
        if (!on[i]) continue;
        if (P->hflags[2 * i] & 2) {
            P->is[i].nst = -NKS_EPIVOT;
            P->is[i].err = "zero pivot in an ILU(0) subdomain factorisation";
        }
    }
    if (P->inner_f32(mode)) {
        NKS_DISPATCH(launch_fac_to_f32, P, bt);
        P->count(1);
    }
    return NKS_OK;
}

template <typename TV>
void project_t(Problem *P, TV *z, const Bat &bt)
{
    RasPlan *R = P->ras;
    P->tick(6);
    if (!P->k.elastic) launch_project_t<0, 1, 0, TV>(P, z, bt);
    else if (P->g.bc == NKS_NEUMANN) {
        // translations and the discrete rotations (planes without the mode weigh 0)
        switch (P->g.dim) {
        case 1: launch_project_t<1, 1, 0, TV>(P, z, bt); break;
        case 2: launch_project_t<2, 1, 1, TV>(P, z, bt); break;
        default: launch_project_t<3, 1, 3, TV>(P, z, bt); break;
        }
    } else {
        // displacement components (the dimension) and null modes per component
        const int code = P->g.dim * 10 + R->nmodes;
        switch (code) {
        case 11: launch_project_t<1, 1, 0, TV>(P, z, bt); break;
        case 12: launch_project_t<1, 2, 0, TV>(P, z, bt); break;
        case 21: launch_project_t<2, 1, 0, TV>(P, z, bt); break;
        case 22: launch_project_t<2, 2, 0, TV>(P, z, bt); break;
        case 24: launch_project_t<2, 4, 0, TV>(P, z, bt); break;
        case 31: launch_project_t<3, 1, 0, TV>(P, z, bt); break;
        case 32: launch_project_t<3, 2, 0, TV>(P, z, bt); break;
        case 34: launch_project_t<3, 4, 0, TV>(P, z, bt); break;
        case 38: launch_project_t<3, 8, 0, TV>(P, z, bt); break;
        }
    }
    P->count(2);
    P->tock(6);
}

void project(Problem *P, double *z, const Bat &bt) { project_t<double>(P, z, bt); }

template <typename TV>
void ras_apply_t(Problem *P, const TV *r, TV *z, const Bat &bt)
{
    P->tick(2);
    dispatch(P, [&](auto d_, auto nf_, auto v_) {
        launch_apply_t<decltype(d_)::value, decltype(nf_)::value, decltype(v_)::value, TV>(P, r, z, bt);
    });
    P->count(P->opts.ras_variant != NKS_LEFT_RAS ? 2 : 1);
    P->tock(2);
}
template void ras_apply_t<double>(Problem *, const double *, double *, const Bat &);
template void ras_apply_t<float>(Problem *, const float *, float *, const Bat &);

void ras_apply(Problem *P, const double *r, double *z, const Bat &bt)
{
    ras_apply_t<double>(P, r, z, bt);
    project(P, z, bt);
}

template <typename TV>
void ras_apply_projected(Problem *P, const TV *r, TV *z, const Bat &bt)
{
    ras_apply_t<TV>(P, r, z, bt);
    project_t<TV>(P, z, bt);
}
template void ras_apply_projected<float>(Problem *, const float *, float *, const Bat &);

void ras_prepare_launch(Problem *P) { NKS_DISPATCH(apply_attrs, P); }

// per-instance buffers of the Schwarz preconditioner (carved from each instance's slab)
void ras_slab_items(Problem *P, std::vector<SlabItem> &items)
{
    RasPlan *R = P->ras;
    const bool mixed = P->opts.precision == NKS_MIXED;
    items.push_back({(void **)&R->fac, sizeof(double) * (size_t)R->fac_elems});
    items.push_back({(void **)&R->proj, sizeof(double) * 64});
    // the scratch vector holds the sub-vectors when they miss shared memory, and the box
    // solutions of the overlapped prolongation (classical AS, right-RAS)
    const bool summed = P->opts.ras_variant != NKS_LEFT_RAS;
    if ((!R->x_smem || summed) && !mixed)
        items.push_back({(void **)&R->scratch, sizeof(double) * (size_t)R->scr_elems});
    if (P->f32) {
        items.push_back({(void **)&R->fac32, sizeof(float) * (size_t)R->fac32_elems});
        if (!R->x_smem32 || summed) items.push_back({(void **)&R->scratch32, sizeof(float) * (size_t)R->scr_elems});
    }
}

// algorithmic work of one Schwarz sweep (both triangular solves over every
// overlapped point): bytes of factors + gathered and written vectors, FLOPs
void ras_work(const Problem *P, double *bytes, double *flops)
{
    const RasPlan *R = P->ras;
    const double pts = (double)R->total_np, owned = (double)P->N;
    const double b = P->opts.precision == NKS_MIXED ? 4.0 : 8.0;  // FP32 factors and vectors in mixed mode
    // factors (lower + upper entries + inverse pivots) of every overlapped point, the
    // gathered sub-vectors and the owned output, each moved once
    *bytes = pts * (R->nlow + R->nup + P->nf) * b + pts * P->nf * b + owned * P->nf * b;
    *flops = pts * (2.0 * (R->nlow + R->nup) + P->nf);
}

}  // namespace nks
