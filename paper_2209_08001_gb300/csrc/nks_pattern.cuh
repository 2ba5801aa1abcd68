// nks_pattern.cuh -- one row of the Jacobian dF/dX1 of NSOA-1 and its
// compile-time sparsity pattern.
//
// jac_row() lists the entries of row f at a point as (path, field, value)
// contributions, the path being one or two one-cell steps from the point (o,
// then e): with Neumann boundaries a step that leaves the grid stays on the
// cell (mirror ghost), so only the accumulator, which knows the point's place
// in the grid, can tell where a path ends.  The assembly kernel evaluates the
// rows numerically; the same function, run at compile time with a structural
// accumulator, yields the exact pattern (and its column order) that the
// Schwarz sweeps unroll over: every end a path can have at some place in the
// grid.
#pragma once

#include "nks_internal.cuh"

namespace nks {

// ---------------------------------------------------------------------------
// one row of the Jacobian dF/dX1 as a list of (offset, field, value)
// ---------------------------------------------------------------------------

// Fields of a point: c (0), the k.ne order parameters (1..k.ne), then the
// displacement components (from 1 + k.ne).  The row functions take the count as
// a template argument NE when the caller knows it (NE = 0: k.ne at run time).
struct RowCtx {
    double a0[7];         // dGc/dc1 at p (0) and p + e_J (1 + 2J), p - e_J (2 + 2J)
    double a1[7][3];      // dGc/deta_j1 at the same points
    double a2[3];         // dGeta_j/dc1 at p
    double a3[3][3];      // dGeta_j/deta_i1 at p
    double Mp[3], Mm[3];  // edge mobilities M_{p + e_J/2}, M_{p - e_J/2}
};

// contributions of the linearised G_c at q = the end of step o from p (o = 0 or
// +-e_J) with weight w
template <int NE = 0, class Acc>
__host__ __device__ constexpr void add_grow(Acc &acc, const DCoef &k, int d, double h, int ox, int oy, int oz, double w,
                                         double a0, const double (&a1)[3])
{
    const double ih2 = 1.0 / (h * h);
    double diag = a0 + k.gamma_c * d * ih2;
    if (k.elastic) diag += 0.5 * d * k.eps0 * k.eps0 * k.lam;
    acc(ox, oy, oz, 0, 0, 0, 0, w * diag);
    for (int J = 0; J < d; J++) {
        const int ex = J == 0, ey = J == 1, ez = J == 2;
        acc(ox, oy, oz, ex, ey, ez, 0, -w * 0.5 * k.gamma_c * ih2);
        acc(ox, oy, oz, -ex, -ey, -ez, 0, -w * 0.5 * k.gamma_c * ih2);
    }
    const int ne = NE ? NE : k.ne;
    for (int j = 0; j < ne; j++) acc(ox, oy, oz, 0, 0, 0, 1 + j, w * a1[j]);
    if (k.elastic) {
        const double t = w * k.eps0 * k.lam * 0.25 / h;  // G^3_c = -eps0 lam (sum_K Dhat_K u_K - d eps0 c ...)/2
        const int ku = 1 + ne;
        for (int K = 0; K < d; K++) {
            const int ex = K == 0, ey = K == 1, ez = K == 2;
            acc(ox, oy, oz, ex, ey, ez, ku + K, -t);
            acc(ox, oy, oz, -ex, -ey, -ez, ku + K, +t);
        }
    }
}

// sigma_IJ(q) row, q = the end of step o from p, weight w (stress of eps(u) -
// eps0 (c - cbar) I)
template <int NE = 0, class Acc>
__host__ __device__ constexpr void add_sigrow(Acc &acc, const DCoef &k, int d, double h, int ox, int oy, int oz, int I,
                                           int J, double w)
{
    const double i2h = 0.5 / h;
    const int ku = 1 + (NE ? NE : k.ne);
    if (I == J) {
        for (int K = 0; K < d; K++) {
            const int ex = K == 0, ey = K == 1, ez = K == 2;
            const double cf = (K == I) ? k.C11 : k.C12;
            acc(ox, oy, oz, ex, ey, ez, ku + K, w * cf * i2h);
            acc(ox, oy, oz, -ex, -ey, -ez, ku + K, -w * cf * i2h);
        }
        acc(ox, oy, oz, 0, 0, 0, 0, -w * k.eps0 * k.lam);
    } else {
        const int jx = J == 0, jy = J == 1, jz = J == 2;
        const int ix = I == 0, iy = I == 1, iz = I == 2;
        acc(ox, oy, oz, jx, jy, jz, ku + I, w * k.C44 * i2h);
        acc(ox, oy, oz, -jx, -jy, -jz, ku + I, -w * k.C44 * i2h);
        acc(ox, oy, oz, ix, iy, iz, ku + J, w * k.C44 * i2h);
        acc(ox, oy, oz, -ix, -iy, -iz, ku + J, -w * k.C44 * i2h);
    }
}

// Row f of J at a point: c-row from F_c = (c1-c0)/dt - D M D G_c, eta_j-row from
// F_eta_j = (eta_j1-eta_j0)/dt + k.keta G_eta_j (the kinetic factor: 1 in the
// reduced model, whose G^4_eta carries 3 gamma_eta; 3 with three order parameters,
// whose G^4_eta_j carries gamma_eta), u_I-row from F_uI = sum_J Dhat_J sigma_IJ
// (with Neumann boundaries its traction-free form: a step that stays on the cell
// enters with the opposite sign, acc.flip).
// mode 1 (displacement-only system): c and eta rows are identity rows.
template <int NE = 0, class Acc>
__host__ __device__ constexpr void jac_row(Acc &acc, int f, const DCoef &k, int d, double h, double dt, int mode,
                                        const RowCtx &r)
{
    const double ih2 = 1.0 / (h * h);
    if (f == 0) {
        if (mode != 0) {
            acc(0, 0, 0, 0, 0, 0, 0, 1.0);
            return;
        }
        acc(0, 0, 0, 0, 0, 0, 0, 1.0 / dt);
        double wc = 0.0;
        for (int J = 0; J < d; J++) wc += (r.Mp[J] + r.Mm[J]) * ih2;
        add_grow<NE>(acc, k, d, h, 0, 0, 0, wc, r.a0[0], r.a1[0]);
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            add_grow<NE>(acc, k, d, h, ex, ey, ez, -r.Mp[J] * ih2, r.a0[1 + 2 * J], r.a1[1 + 2 * J]);
            add_grow<NE>(acc, k, d, h, -ex, -ey, -ez, -r.Mm[J] * ih2, r.a0[2 + 2 * J], r.a1[2 + 2 * J]);
        }
    } else if (f <= (NE ? NE : k.ne)) {
        if (mode != 0) {
            acc(0, 0, 0, 0, 0, 0, f, 1.0);
            return;
        }
        // (gamma_eta/2 per |grad eta_j|^2) x 3 = 3 gamma_eta/2 for |grad eta|^2: the same
        // Laplacian weights in both models
        const int j = f - 1;
        acc(0, 0, 0, 0, 0, 0, f, 1.0 / dt + k.keta * r.a3[j][j] + 3.0 * k.gamma_eta * d * ih2);
        acc(0, 0, 0, 0, 0, 0, 0, k.keta * r.a2[j]);
        for (int i = 0; i < (NE ? NE : k.ne); i++)
            if (i != j) acc(0, 0, 0, 0, 0, 0, 1 + i, k.keta * r.a3[j][i]);
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            acc(0, 0, 0, ex, ey, ez, f, -1.5 * k.gamma_eta * ih2);
            acc(0, 0, 0, -ex, -ey, -ez, f, -1.5 * k.gamma_eta * ih2);
        }
    } else {
        const int I = f - 1 - (NE ? NE : k.ne);
        const double i2h = 0.5 / h;
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            add_sigrow<NE>(acc, k, d, h, ex, ey, ez, I, J, i2h * acc.flip(ex, ey, ez));
            add_sigrow<NE>(acc, k, d, h, -ex, -ey, -ez, I, J, -i2h * acc.flip(-ex, -ey, -ez));
        }
    }
}

// ---------------------------------------------------------------------------
// compile-time pattern
// ---------------------------------------------------------------------------

constexpr int kMaxSlots = 232;  // 229 in 3-D with three order parameters and Neumann boundaries

struct Pattern {
    int nf;
    int len[kMaxNf];
    int diag[kMaxNf];
    int rowoff[kMaxNf + 1];
    signed char dx[kMaxSlots], dy[kMaxSlots], dz[kMaxSlots], fc[kMaxSlots];
    // storage of a point's factors: the strictly lower entries of all rows form
    // the forward part (nlow rows), the strictly upper entries then the inverse
    // pivots form the backward part (nup + nf rows); st[a] is the row of slot a
    // inside its part (the pivot slot itself is stored as its inverse, st = nup + f)
    int nlow, nup;
    short st[kMaxSlots];
};

// ends along one axis of the two-step path (a, b) over every place in the grid:
// periodic, the sum; Neumann, each step stays on the cell where it would leave the
// grid (positions 0..6 of an axis of 7 cells cover every boundary situation)
struct AxisEnds {
    int n = 0;
    int v[3] = {};
};
__host__ __device__ constexpr AxisEnds axis_ends(int a, int b, int bc)
{
    AxisEnds r{};
    for (int x = 0; x < (bc ? 7 : 1); x++) {
        int y = x + a, e = 0;
        if (bc && (y < 0 || y >= 7)) y = x;
        int z = y + b;
        if (bc && (z < 0 || z >= 7)) z = y;
        e = bc ? z - x : a + b;
        bool seen = false;
        for (int i = 0; i < r.n; i++) seen = seen || r.v[i] == e;
        if (!seen) r.v[r.n++] = e;
    }
    return r;
}

// structural accumulator: records each (offset, field) once, for every end the path
// can have (BC 1: Neumann boundaries)
template <int BC>
struct CxAcc {
    int n = 0;
    signed char dx[kMaxRow] = {}, dy[kMaxRow] = {}, dz[kMaxRow] = {}, fc[kMaxRow] = {};
    __host__ __device__ constexpr void add(int x, int y, int z, int f)
    {
        for (int i = 0; i < n; i++)
            if (dx[i] == x && dy[i] == y && dz[i] == z && fc[i] == f) return;
        dx[n] = (signed char)x;
        dy[n] = (signed char)y;
        dz[n] = (signed char)z;
        fc[n] = (signed char)f;
        n++;
    }
    __host__ __device__ constexpr void operator()(int ox, int oy, int oz, int ex, int ey, int ez, int f, double)
    {
        const AxisEnds X = axis_ends(ox, ex, BC), Y = axis_ends(oy, ey, BC), Z = axis_ends(oz, ez, BC);
        for (int a = 0; a < X.n; a++)
            for (int b = 0; b < Y.n; b++)
                for (int c = 0; c < Z.n; c++) add(X.v[a], Y.v[b], Z.v[c], f);
    }
    __host__ __device__ constexpr double flip(int, int, int) const { return 1.0; }
};

// column order of a box-local row: lexicographic in (dz, dy, dx, field)
__host__ __device__ constexpr bool col_less(int z1, int y1, int x1, int f1, int z2, int y2, int x2, int f2)
{
    if (z1 != z2) return z1 < z2;
    if (y1 != y2) return y1 < y2;
    if (x1 != x2) return x1 < x2;
    return f1 < f2;
}

// Pattern variant V: bit 0, the model with elasticity under Neumann boundaries
// (the mirrored paths add columns; without elasticity both boundary kinds share
// one pattern); bit 1, three order parameters (App. A)
template <int DIM, int NF, int V = 0>
__host__ __device__ constexpr Pattern make_pattern()
{
    Pattern P{};
    P.nf = NF;
    DCoef k{};
    k.gamma_c = k.gamma_eta = k.eps0 = k.lam = k.C11 = k.C12 = k.C44 = k.keta = 1.0;
    k.ne = (V & 2) ? 3 : 1;
    k.elastic = NF > 1 + k.ne ? 1 : 0;
    RowCtx r{};
    for (int i = 0; i < 7; i++) {
        r.a0[i] = 1.0;
        for (int j = 0; j < 3; j++) r.a1[i][j] = 1.0;
    }
    for (int j = 0; j < 3; j++) {
        r.a2[j] = 1.0;
        for (int i = 0; i < 3; i++) r.a3[j][i] = 1.0;
    }
    for (int J = 0; J < 3; J++) r.Mp[J] = r.Mm[J] = 1.0;
    int off = 0;
    for (int f = 0; f < NF; f++) {
        CxAcc<(V & 1)> a{};
        jac_row(a, f, k, DIM, 1.0, 1.0, 0, r);
        for (int i = 1; i < a.n; i++) {  // insertion sort into column order
            int j = i;
            while (j > 0 && col_less(a.dz[j], a.dy[j], a.dx[j], a.fc[j], a.dz[j - 1], a.dy[j - 1], a.dx[j - 1],
                                     a.fc[j - 1])) {
                signed char t = 0;
                t = a.dx[j]; a.dx[j] = a.dx[j - 1]; a.dx[j - 1] = t;
                t = a.dy[j]; a.dy[j] = a.dy[j - 1]; a.dy[j - 1] = t;
                t = a.dz[j]; a.dz[j] = a.dz[j - 1]; a.dz[j - 1] = t;
                t = a.fc[j]; a.fc[j] = a.fc[j - 1]; a.fc[j - 1] = t;
                j--;
            }
        }
        P.rowoff[f] = off;
        P.len[f] = a.n;
        P.diag[f] = -1;
        for (int i = 0; i < a.n; i++) {
            P.dx[off + i] = a.dx[i];
            P.dy[off + i] = a.dy[i];
            P.dz[off + i] = a.dz[i];
            P.fc[off + i] = a.fc[i];
            if (a.dx[i] == 0 && a.dy[i] == 0 && a.dz[i] == 0 && a.fc[i] == f) P.diag[f] = i;
        }
        off += a.n;
    }
    P.rowoff[NF] = off;
    int lo = 0, up = 0;
    for (int f = 0; f < NF; f++)
        for (int i = 0; i < P.len[f]; i++) {
            const int a = P.rowoff[f] + i;
            if (i < P.diag[f]) P.st[a] = (short)lo++;
            else if (i > P.diag[f]) P.st[a] = (short)up++;
        }
    P.nlow = lo;
    P.nup = up;
    for (int f = 0; f < NF; f++) P.st[P.rowoff[f] + P.diag[f]] = (short)(up + f);
    return P;
}

}  // namespace nks

namespace nks {

// ---------------------------------------------------------------------------
// two-stage schedule of one triangular sweep over a wavefront level
// ---------------------------------------------------------------------------
//
// Forward sweep (L y = b) row f of a point uses its strictly lower entries;
// backward sweep (U x = y) its strictly upper entries.  Entries at other
// points refer to earlier (forward) or later (backward) levels, which are
// final when the level starts; entries at the same point refer to rows of
// the same point.  Stage A runs, for every point of the level in parallel,
// warp-uniform tasks over chunks of the other-point entries (at most
// chunk_size(D) entries each): a row with one chunk and no same-point entry is finished in
// stage A, otherwise the chunk sum goes to a partial.  Stage B, one thread
// per point, finishes the remaining rows in sweep order from their partials
// and same-point entries.

// Entries per stage-A chunk: a shorter FP64 chain per task against more tasks,
// partial sums and FP64 instructions.  Measured per Schwarz application on the
// bench workloads' boxes: 2-D 68^2 boxes 5: 0.98 ms (4: 1.02, 6: 1.21, 7: 1.22,
// 10: 1.16); 3-D 18^3 boxes 13: 2.41 ms (16: 2.41, 10: 2.68, 24: 2.76, 7: 3.25,
// 5: 3.31).
constexpr int kChunk2 = 5;
constexpr int kChunk3 = 13;
__host__ __device__ constexpr int chunk_size(int D) { return D == 3 ? kChunk3 : kChunk2; }
constexpr int kMaxTasks = 24;
constexpr int kMaxPartials = 24;

struct SweepPlan {
    int ntask;
    int t_row[kMaxTasks], t_b[kMaxTasks], t_e[kMaxTasks], t_part[kMaxTasks];  // t_part < 0: finishes the row
    int npart;
    int row_stage_b[kMaxNf];           // 1: the row is finished in stage B
    int row_pb[kMaxNf], row_pe[kMaxNf];  // its partials [pb, pe)
    int same_b[kMaxNf], same_e[kMaxNf];  // its same-point slot range (contiguous in column order)
};

template <int D, int NF, bool FWD, int V = 0>
__host__ __device__ constexpr SweepPlan make_sweep_plan()
{
    constexpr Pattern P = make_pattern<D, NF, V>();
    SweepPlan S{};
    for (int f = 0; f < NF; f++) {
        const int b = FWD ? P.rowoff[f] : P.rowoff[f] + P.diag[f] + 1;
        const int e = FWD ? P.rowoff[f] + P.diag[f] : P.rowoff[f] + P.len[f];
        // same-point entries form a contiguous run at offset (0,0,0) in column order
        int sb = e, se = e;
        for (int a = b; a < e; a++)
            if (P.dx[a] == 0 && P.dy[a] == 0 && P.dz[a] == 0) {
                if (sb == e) sb = a;
                se = a + 1;
            }
        S.same_b[f] = sb;
        S.same_e[f] = se;
        // other-point entries: [b, sb) and [se, e)
        const int n_other = (sb - b) + (e - se);
        const int nch = (n_other + chunk_size(D) - 1) / chunk_size(D);
        const bool finish_in_a = (nch <= 1) && (se == sb);
        S.row_stage_b[f] = finish_in_a ? 0 : 1;
        S.row_pb[f] = S.npart;
        // split [b, sb) then [se, e) into nch balanced chunks
        int taken = 0;
        for (int c = 0; c < nch; c++) {
            const int want = (n_other * (c + 1)) / nch - (n_other * c) / nch;
            // a chunk never straddles the same-point run: take from the first range, then the second
            const int lo_idx = taken, hi_idx = taken + want;
            const int first_len = sb - b;
            int cb = 0, ce = 0;
            if (hi_idx <= first_len) {
                cb = b + lo_idx;
                ce = b + hi_idx;
            } else if (lo_idx >= first_len) {
                cb = se + (lo_idx - first_len);
                ce = se + (hi_idx - first_len);
            } else {  // split at the run: two tasks
                S.t_row[S.ntask] = f;
                S.t_b[S.ntask] = b + lo_idx;
                S.t_e[S.ntask] = sb;
                S.t_part[S.ntask] = finish_in_a ? -1 : S.npart++;
                S.ntask++;
                cb = se;
                ce = se + (hi_idx - first_len);
            }
            S.t_row[S.ntask] = f;
            S.t_b[S.ntask] = cb;
            S.t_e[S.ntask] = ce;
            S.t_part[S.ntask] = finish_in_a ? -1 : S.npart++;
            S.ntask++;
            taken = hi_idx;
        }
        S.row_pe[f] = S.npart;
    }
    return S;
}

}  // namespace nks
