// nks_ras.cu -- restricted additive Schwarz with ILU(0) subdomain solves.
//
// Sec. 4 preconditions GMRES with a Schwarz method over a box decomposition
// (one subdomain per core in the paper); Sec. 5.4 selects ILU(0) reused for
// the whole time step.  Here one overlapping subdomain is one thread block:
//
//   * plan (host, once): the exact nonzero pattern of a Jacobian row per
//     field, derived structurally from the same row function the assembly
//     kernel evaluates; the ILU(0) update lists (which entries of row k
//     update which entries of row i); per subdomain the overlapped box,
//     its owned part and its wavefront levels lv = x + 2y + 4z, which order
//     every lower neighbour of a point before the point itself;
//   * factor (device, once per time step): assemble J restricted to the box
//     (columns outside the box dropped) and run ILU(0) row by row, level by
//     level, all rows of one level in parallel.  Factors are stored
//     slot-major and level-ordered, so one level's threads read
//     consecutive addresses;
//   * apply (device, every GMRES iteration): gather r on the box into shared
//     memory, forward and backward sweeps level by level, write the owned
//     points (restricted prolongation, no atomics), then the projection P.
#include <math.h>

#include <algorithm>
#include <map>
#include <set>
#include <tuple>

#include "nks_internal.cuh"

namespace nks {

// ---------------------------------------------------------------------------
// one row of the Jacobian dF/dX1 as a list of (offset, field, value)
// ---------------------------------------------------------------------------

struct RowCtx {
    double a0[7], a1[7];  // dGc/dc1, dGc/deta1 at p (0) and p + e_J (1 + 2J), p - e_J (2 + 2J)
    double a2, a3;        // dGeta/dc1, dGeta/deta1 at p
    double Mp[3], Mm[3];  // edge mobilities M_{p + e_J/2}, M_{p - e_J/2}
};

// contributions of the linearised G_c at q = p + o (o = 0 or +-e_J) with weight w
template <class Acc>
__host__ __device__ inline void add_grow(Acc &acc, const DCoef &k, int d, double h, int ox, int oy, int oz, double w,
                                         double a0, double a1)
{
    const double ih2 = 1.0 / (h * h);
    double diag = a0 + k.gamma_c * d * ih2;
    if (k.elastic) diag += 0.5 * d * k.eps0 * k.eps0 * k.lam;
    acc(ox, oy, oz, 0, w * diag);
    for (int J = 0; J < d; J++) {
        const int ex = J == 0, ey = J == 1, ez = J == 2;
        acc(ox + ex, oy + ey, oz + ez, 0, -w * 0.5 * k.gamma_c * ih2);
        acc(ox - ex, oy - ey, oz - ez, 0, -w * 0.5 * k.gamma_c * ih2);
    }
    acc(ox, oy, oz, 1, w * a1);
    if (k.elastic) {
        const double t = w * k.eps0 * k.lam * 0.25 / h;  // G^3_c = -eps0 lam (sum_K Dhat_K u_K - d eps0 c ...)/2
        for (int K = 0; K < d; K++) {
            const int ex = K == 0, ey = K == 1, ez = K == 2;
            acc(ox + ex, oy + ey, oz + ez, 2 + K, -t);
            acc(ox - ex, oy - ey, oz - ez, 2 + K, +t);
        }
    }
}

// sigma_IJ(q) row, q = p + o, weight w (stress of eps(u) - eps0 (c - cbar) I)
template <class Acc>
__host__ __device__ inline void add_sigrow(Acc &acc, const DCoef &k, int d, double h, int ox, int oy, int oz, int I,
                                           int J, double w)
{
    const double i2h = 0.5 / h;
    if (I == J) {
        for (int K = 0; K < d; K++) {
            const int ex = K == 0, ey = K == 1, ez = K == 2;
            const double cf = (K == I) ? k.C11 : k.C12;
            acc(ox + ex, oy + ey, oz + ez, 2 + K, w * cf * i2h);
            acc(ox - ex, oy - ey, oz - ez, 2 + K, -w * cf * i2h);
        }
        acc(ox, oy, oz, 0, -w * k.eps0 * k.lam);
    } else {
        const int jx = J == 0, jy = J == 1, jz = J == 2;
        const int ix = I == 0, iy = I == 1, iz = I == 2;
        acc(ox + jx, oy + jy, oz + jz, 2 + I, w * k.C44 * i2h);
        acc(ox - jx, oy - jy, oz - jz, 2 + I, -w * k.C44 * i2h);
        acc(ox + ix, oy + iy, oz + iz, 2 + J, w * k.C44 * i2h);
        acc(ox - ix, oy - iy, oz - iz, 2 + J, -w * k.C44 * i2h);
    }
}

// Row f of J at a point: c-row from F_c = (c1-c0)/dt - D M D G_c, eta-row from
// F_eta = (eta1-eta0)/dt + G_eta, u_I-row from F_uI = sum_J Dhat_J sigma_IJ.
// mode 1 (displacement-only system): c and eta rows are identity rows.
template <class Acc>
__host__ __device__ inline void jac_row(Acc &acc, int f, const DCoef &k, int d, double h, double dt, int mode,
                                        const RowCtx &r)
{
    const double ih2 = 1.0 / (h * h);
    if (f == 0) {
        if (mode != 0) {
            acc(0, 0, 0, 0, 1.0);
            return;
        }
        acc(0, 0, 0, 0, 1.0 / dt);
        double wc = 0.0;
        for (int J = 0; J < d; J++) wc += (r.Mp[J] + r.Mm[J]) * ih2;
        add_grow(acc, k, d, h, 0, 0, 0, wc, r.a0[0], r.a1[0]);
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            add_grow(acc, k, d, h, ex, ey, ez, -r.Mp[J] * ih2, r.a0[1 + 2 * J], r.a1[1 + 2 * J]);
            add_grow(acc, k, d, h, -ex, -ey, -ez, -r.Mm[J] * ih2, r.a0[2 + 2 * J], r.a1[2 + 2 * J]);
        }
    } else if (f == 1) {
        if (mode != 0) {
            acc(0, 0, 0, 1, 1.0);
            return;
        }
        acc(0, 0, 0, 1, 1.0 / dt + r.a3 + 3.0 * k.gamma_eta * d * ih2);
        acc(0, 0, 0, 0, r.a2);
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            acc(ex, ey, ez, 1, -1.5 * k.gamma_eta * ih2);
            acc(-ex, -ey, -ez, 1, -1.5 * k.gamma_eta * ih2);
        }
    } else {
        const int I = f - 2;
        const double i2h = 0.5 / h;
        for (int J = 0; J < d; J++) {
            const int ex = J == 0, ey = J == 1, ez = J == 2;
            add_sigrow(acc, k, d, h, ex, ey, ez, I, J, i2h);
            add_sigrow(acc, k, d, h, -ex, -ey, -ez, I, J, -i2h);
        }
    }
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------

struct SubInfo {
    int org[3];               // global coordinates of local (0,0,0) (may be negative: periodic)
    int L[3];                 // box extent
    int own0[3], own1[3];     // owned local range [own0, own1)
    int np, nlev;
    long long lvl_off;        // into lvl_ptr (nlev + 1 entries)
    long long pos_off;        // into lvl_lp / pos_of_lp (np entries)
    long long fac_off;        // into the factor array (nslot * np)
    long long scr_off;        // into the global scratch vector (nf * np), when not in shared memory
};

struct RasPlan {
    int nsub = 0, nslot = 0, threads = 128;
    int maxnp = 0;
    bool smem = true;
    size_t smem_bytes = 0;
    // device tables
    char4 *tmpl = nullptr;          // (dx, dy, dz, fc) per slot, rows concatenated
    short *slotmap = nullptr;       // [f][(dz+2)*25 + (dy+2)*5 + (dx+2)][fc]
    int *upd_ptr = nullptr;         // [rowoff[f] + a] -> start in upd (size nslot + 1)
    short2 *upd = nullptr;          // (b, c) pairs
    SubInfo *sub = nullptr;
    int *lvl_ptr = nullptr, *lvl_lp = nullptr, *pos_of_lp = nullptr;
    double *fac = nullptr;
    double *scratch = nullptr;
    double *proj = nullptr;         // projection coefficients
    int rowoff[kMaxNf + 1];
    int diag[kMaxNf];
    int nmodes = 1;                 // null modes per displacement component
    int evenmask = 0;
    bool attr_set = false;
};

namespace {

struct StructAcc {
    std::set<std::tuple<int, int, int, int>> *s;
    void operator()(int dx, int dy, int dz, int fc, double) { s->insert(std::make_tuple(dz, dy, dx, fc)); }
};

}  // namespace

int ras_plan_create(Problem *P, std::string &err)
{
    RasPlan *R = new RasPlan();
    P->ras = R;
    const int d = P->g.dim, nf = P->nf;
    // ---- templates (structural pattern of each row field)
    DCoef kk = P->k;
    kk.C11 = kk.C12 = kk.C44 = kk.lam = 1.0;  // structural pass: every coefficient non-zero
    kk.gamma_c = kk.gamma_eta = kk.eps0 = 1.0;
    RowCtx rc;
    for (int i = 0; i < 7; i++) rc.a0[i] = rc.a1[i] = 1.0;
    rc.a2 = rc.a3 = 1.0;
    for (int J = 0; J < 3; J++) rc.Mp[J] = rc.Mm[J] = 1.0;
    std::vector<std::vector<std::tuple<int, int, int, int>>> rows(nf);
    int total = 0;
    for (int f = 0; f < nf; f++) {
        std::set<std::tuple<int, int, int, int>> s;
        StructAcc acc{&s};
        jac_row(acc, f, kk, d, 1.0, 1.0, 0, rc);
        rows[f].assign(s.begin(), s.end());  // lexicographic (dz, dy, dx, fc) = column order
        R->rowoff[f] = total;
        total += (int)rows[f].size();
        R->diag[f] = -1;
        for (size_t a = 0; a < rows[f].size(); a++) {
            auto [dz, dy, dx, fc] = rows[f][a];
            if (dz == 0 && dy == 0 && dx == 0 && fc == f) R->diag[f] = (int)a;
        }
        if (R->diag[f] < 0 || rows[f].size() > (size_t)kMaxRow) {
            err = "internal: Jacobian row template";
            return NKS_EINVAL;
        }
        // every column before the diagonal must lie on an earlier wavefront level (or the same point)
        for (int a = 0; a < R->diag[f]; a++) {
            auto [dz, dy, dx, fc] = rows[f][a];
            const int lv = dx + 2 * dy + 4 * dz;
            if (!((dx == 0 && dy == 0 && dz == 0) || lv < 0)) {
                err = "internal: wavefront ordering";
                return NKS_EINVAL;
            }
        }
    }
    R->rowoff[nf] = total;
    R->nslot = total;
    std::vector<char4> tmpl(total);
    std::vector<short> slotmap((size_t)nf * 125 * nf, -1);
    for (int f = 0; f < nf; f++)
        for (size_t a = 0; a < rows[f].size(); a++) {
            auto [dz, dy, dx, fc] = rows[f][a];
            tmpl[R->rowoff[f] + a] = make_char4((signed char)dx, (signed char)dy, (signed char)dz, (signed char)fc);
            slotmap[((size_t)f * 125 + (dz + 2) * 25 + (dy + 2) * 5 + (dx + 2)) * nf + fc] = (short)a;
        }
    // ---- ILU(0) update lists: for row f, lower slot a (row k = p + o_a, field f_a), every later
    // slot b of row f whose column also appears in row k gives (b, slot c of that column in row k)
    std::vector<int> upd_ptr(total + 1, 0);
    std::vector<short2> upd;
    for (int f = 0; f < nf; f++)
        for (int a = 0; a < (int)rows[f].size(); a++) {
            upd_ptr[R->rowoff[f] + a] = (int)upd.size();
            if (a >= R->diag[f]) continue;
            auto [az, ay, ax, afc] = rows[f][a];
            for (int b = a + 1; b < (int)rows[f].size(); b++) {
                auto [bz, by, bx, bfc] = rows[f][b];
                const int rx = bx - ax, ry = by - ay, rz = bz - az;
                if (abs(rx) > 2 || abs(ry) > 2 || abs(rz) > 2) continue;
                const short c = slotmap[((size_t)afc * 125 + (rz + 2) * 25 + (ry + 2) * 5 + (rx + 2)) * nf + bfc];
                if (c >= 0) upd.push_back(make_short2((short)b, c));
            }
        }
    upd_ptr[total] = (int)upd.size();

    // ---- subdomains
    int sub[3] = {1, 1, 1};
    for (int J = 0; J < d; J++) sub[J] = std::max(1, P->opts.sub[J]);
    const int delta = P->opts.overlap;
    R->nsub = sub[0] * sub[1] * sub[2];
    std::vector<SubInfo> infos(R->nsub);
    std::vector<int> lvl_ptr, lvl_lp, pos_of_lp;
    long long fac_off = 0, scr_off = 0;
    for (int s2 = 0; s2 < sub[2]; s2++)
        for (int s1 = 0; s1 < sub[1]; s1++)
            for (int s0 = 0; s0 < sub[0]; s0++) {
                const int s = s0 + sub[0] * (s1 + sub[1] * s2);
                const int sidx[3] = {s0, s1, s2};
                SubInfo &si = infos[s];
                for (int J = 0; J < 3; J++) {
                    if (J < d) {
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
                // wavefront levels
                const int nlev = (si.L[0] - 1) + 2 * (si.L[1] - 1) + 4 * (si.L[2] - 1) + 1;
                si.nlev = nlev;
                si.lvl_off = (long long)lvl_ptr.size();
                si.pos_off = (long long)lvl_lp.size();
                std::vector<std::vector<int>> bylev(nlev);
                for (int lz = 0; lz < si.L[2]; lz++)
                    for (int ly = 0; ly < si.L[1]; ly++)
                        for (int lx = 0; lx < si.L[0]; lx++)
                            bylev[lx + 2 * ly + 4 * lz].push_back(lx + si.L[0] * (ly + si.L[1] * lz));
                std::vector<int> pos(si.np);
                int cnt = 0;
                for (int l = 0; l < nlev; l++) {
                    lvl_ptr.push_back(cnt);
                    for (int lp : bylev[l]) {
                        pos[lp] = cnt;
                        lvl_lp.push_back(lp);
                        cnt++;
                    }
                }
                lvl_ptr.push_back(cnt);
                for (int lp = 0; lp < si.np; lp++) pos_of_lp.push_back(pos[lp]);
                si.fac_off = fac_off;
                fac_off += (long long)R->nslot * si.np;
                si.scr_off = scr_off;
                scr_off += (long long)nf * si.np;
            }
    // shared memory for the sub-vector when it fits
    R->smem_bytes = (size_t)R->maxnp * nf * sizeof(double);
    R->smem = R->smem_bytes <= 200 * 1024;
    // null modes of the centred-difference strain: sign patterns over the even axes
    R->evenmask = 0;
    for (int J = 0; J < d; J++)
        if (P->g.n[J] % 2 == 0) R->evenmask |= 1 << J;
    R->nmodes = 1 << __builtin_popcount(R->evenmask);

    // ---- upload
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        *dst = P->dalloc(bytes);
        if (!*dst) return false;
        cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        return true;
    };
    bool ok = up((void **)&R->tmpl, tmpl.data(), tmpl.size() * sizeof(char4)) &&
              up((void **)&R->slotmap, slotmap.data(), slotmap.size() * sizeof(short)) &&
              up((void **)&R->upd_ptr, upd_ptr.data(), upd_ptr.size() * sizeof(int)) &&
              up((void **)&R->upd, upd.data(), std::max<size_t>(1, upd.size()) * sizeof(short2)) &&
              up((void **)&R->sub, infos.data(), infos.size() * sizeof(SubInfo)) &&
              up((void **)&R->lvl_ptr, lvl_ptr.data(), lvl_ptr.size() * sizeof(int)) &&
              up((void **)&R->lvl_lp, lvl_lp.data(), lvl_lp.size() * sizeof(int)) &&
              up((void **)&R->pos_of_lp, pos_of_lp.data(), pos_of_lp.size() * sizeof(int));
    if (!ok) {
        err = "out of device memory (Schwarz tables)";
        return NKS_ENOMEM;
    }
    R->fac = (double *)P->dalloc(sizeof(double) * (size_t)fac_off);
    R->proj = (double *)P->dalloc(sizeof(double) * 64);
    if (!R->smem) R->scratch = (double *)P->dalloc(sizeof(double) * (size_t)scr_off);
    if (!R->fac || !R->proj || (!R->smem && !R->scratch)) {
        err = "out of device memory (Schwarz factors)";
        return NKS_ENOMEM;
    }
    P->stats.factor_bytes = (long long)(sizeof(double) * (size_t)fac_off);
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

struct Tables {
    int rowoff[kMaxNf + 1];
    int diag[kMaxNf];
    int nf;
};

__device__ inline bool inbox(const SubInfo &si, int lx, int ly, int lz)
{
    return lx >= 0 && lx < si.L[0] && ly >= 0 && ly < si.L[1] && lz >= 0 && lz < si.L[2];
}

struct DevAcc {
    double *vals;
    const short *slotmap;  // row f block
    int nf, lx, ly, lz;
    const SubInfo *si;
    __device__ void operator()(int dx, int dy, int dz, int fc, double v)
    {
        if (!inbox(*si, lx + dx, ly + dy, lz + dz)) return;  // column outside the overlapped box: dropped
        const int s = slotmap[((dz + 2) * 25 + (dy + 2) * 5 + (dx + 2)) * nf + fc];
        if (s >= 0) vals[s] += v;
    }
};

__global__ void k_ras_factor(DGrid g, DCoef k, double dt, int mode, Tables T, const SubInfo *__restrict__ subs,
                             const int *__restrict__ lvl_ptr, const int *__restrict__ lvl_lp,
                             const int *__restrict__ pos_of_lp, const char4 *__restrict__ tmpl,
                             const short *__restrict__ slotmap, const int *__restrict__ upd_ptr,
                             const short2 *__restrict__ upd, const double *__restrict__ part,
                             const double *__restrict__ mob, double *__restrict__ fac, int *__restrict__ flag)
{
    const SubInfo si = subs[blockIdx.x];
    const int nf = T.nf, d = g.dim;
    const int np = si.np;
    double *F = fac + si.fac_off;
    const int *lp_of = lvl_lp + si.pos_off;
    const int *posof = pos_of_lp + si.pos_off;
    const int *lptr = lvl_ptr + si.lvl_off;
    const long long N = g.N;
    double vals[kMaxRow];
    for (int lev = 0; lev < si.nlev; lev++) {
        for (int i = lptr[lev] + threadIdx.x; i < lptr[lev + 1]; i += blockDim.x) {
            const int lp = lp_of[i];
            const int lx = lp % si.L[0], ly = (lp / si.L[0]) % si.L[1], lz = lp / (si.L[0] * si.L[1]);
            const int gx = wrapi(si.org[0] + lx, g.n[0]), gy = wrapi(si.org[1] + ly, g.n[1]),
                      gz = wrapi(si.org[2] + lz, g.n[2]);
            const long long gp = index_of(g, gx, gy, gz);
            RowCtx rc;
            if (mode == 0) {
                rc.a0[0] = part[gp];
                rc.a1[0] = part[N + gp];
                rc.a2 = part[2 * N + gp];
                rc.a3 = part[3 * N + gp];
                for (int J = 0; J < d; J++) {
                    const long long pp = nbrJ(g, gx, gy, gz, J, +1), pm = nbrJ(g, gx, gy, gz, J, -1);
                    rc.a0[1 + 2 * J] = part[pp];
                    rc.a1[1 + 2 * J] = part[N + pp];
                    rc.a0[2 + 2 * J] = part[pm];
                    rc.a1[2 + 2 * J] = part[N + pm];
                    rc.Mp[J] = mob[J * N + gp];
                    rc.Mm[J] = mob[J * N + pm];
                }
            }
            for (int f = 0; f < nf; f++) {
                const int len = T.rowoff[f + 1] - T.rowoff[f];
                for (int a = 0; a < len; a++) vals[a] = 0.0;
                DevAcc acc{vals, slotmap + (size_t)f * 125 * nf, nf, lx, ly, lz, &si};
                jac_row(acc, f, k, d, g.h, dt, mode, rc);
                // ILU(0) elimination of row (p, f) with the finished rows of earlier points / fields
                for (int a = 0; a < T.diag[f]; a++) {
                    const char4 o = tmpl[T.rowoff[f] + a];
                    if (!inbox(si, lx + o.x, ly + o.y, lz + o.z)) continue;
                    const int lpk = lp + o.x + si.L[0] * (o.y + si.L[1] * o.z);
                    const int posk = posof[lpk];
                    const int fk = o.w;
                    const double dk = F[(size_t)(T.rowoff[fk] + T.diag[fk]) * np + posk];
                    const double l = vals[a] / dk;
                    vals[a] = l;
                    for (int u = upd_ptr[T.rowoff[f] + a]; u < upd_ptr[T.rowoff[f] + a + 1]; u++) {
                        const short2 bc = upd[u];
                        vals[bc.x] -= l * F[(size_t)(T.rowoff[fk] + bc.y) * np + posk];
                    }
                }
                if (vals[T.diag[f]] == 0.0 || !isfinite(vals[T.diag[f]])) atomicOr(flag, 2);
                for (int a = 0; a < len; a++) F[(size_t)(T.rowoff[f] + a) * np + i] = vals[a];
            }
        }
        __syncthreads();
    }
}

__global__ void k_ras_apply(DGrid g, Tables T, const SubInfo *__restrict__ subs, const int *__restrict__ lvl_ptr,
                            const int *__restrict__ lvl_lp, const char4 *__restrict__ tmpl,
                            const double *__restrict__ fac, const double *__restrict__ r, double *__restrict__ z,
                            double *__restrict__ scratch, int use_smem)
{
    extern __shared__ double xs[];
    const SubInfo si = subs[blockIdx.x];
    const int nf = T.nf;
    const int np = si.np;
    const double *F = fac + si.fac_off;
    const int *lp_of = lvl_lp + si.pos_off;
    const int *lptr = lvl_ptr + si.lvl_off;
    double *x = use_smem ? xs : scratch + si.scr_off;
    const long long N = g.N;
    // gather R_i^delta r
    for (int lp = threadIdx.x; lp < np; lp += blockDim.x) {
        const int lx = lp % si.L[0], ly = (lp / si.L[0]) % si.L[1], lz = lp / (si.L[0] * si.L[1]);
        const long long gp = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                      wrapi(si.org[2] + lz, g.n[2]));
        for (int f = 0; f < nf; f++) x[f * np + lp] = r[f * N + gp];
    }
    __syncthreads();
    // forward sweep: L y = b (unit lower)
    for (int lev = 0; lev < si.nlev; lev++) {
        for (int i = lptr[lev] + threadIdx.x; i < lptr[lev + 1]; i += blockDim.x) {
            const int lp = lp_of[i];
            const int lx = lp % si.L[0], ly = (lp / si.L[0]) % si.L[1], lz = lp / (si.L[0] * si.L[1]);
            for (int f = 0; f < nf; f++) {
                double s = x[f * np + lp];
                for (int a = 0; a < T.diag[f]; a++) {
                    const char4 o = tmpl[T.rowoff[f] + a];
                    if (!inbox(si, lx + o.x, ly + o.y, lz + o.z)) continue;
                    const int lpk = lp + o.x + si.L[0] * (o.y + si.L[1] * o.z);
                    s -= F[(size_t)(T.rowoff[f] + a) * np + i] * x[o.w * np + lpk];
                }
                x[f * np + lp] = s;
            }
        }
        __syncthreads();
    }
    // backward sweep: U x = y
    for (int lev = si.nlev - 1; lev >= 0; lev--) {
        for (int i = lptr[lev] + threadIdx.x; i < lptr[lev + 1]; i += blockDim.x) {
            const int lp = lp_of[i];
            const int lx = lp % si.L[0], ly = (lp / si.L[0]) % si.L[1], lz = lp / (si.L[0] * si.L[1]);
            for (int f = nf - 1; f >= 0; f--) {
                const int len = T.rowoff[f + 1] - T.rowoff[f];
                double s = x[f * np + lp];
                for (int a = T.diag[f] + 1; a < len; a++) {
                    const char4 o = tmpl[T.rowoff[f] + a];
                    if (!inbox(si, lx + o.x, ly + o.y, lz + o.z)) continue;
                    const int lpk = lp + o.x + si.L[0] * (o.y + si.L[1] * o.z);
                    s -= F[(size_t)(T.rowoff[f] + a) * np + i] * x[o.w * np + lpk];
                }
                x[f * np + lp] = s / F[(size_t)(T.rowoff[f] + T.diag[f]) * np + i];
            }
        }
        __syncthreads();
    }
    // restricted prolongation: owned points only
    for (int lp = threadIdx.x; lp < np; lp += blockDim.x) {
        const int lx = lp % si.L[0], ly = (lp / si.L[0]) % si.L[1], lz = lp / (si.L[0] * si.L[1]);
        if (lx < si.own0[0] || lx >= si.own1[0] || ly < si.own0[1] || ly >= si.own1[1] || lz < si.own0[2] ||
            lz >= si.own1[2])
            continue;
        const long long gp = index_of(g, wrapi(si.org[0] + lx, g.n[0]), wrapi(si.org[1] + ly, g.n[1]),
                                      wrapi(si.org[2] + lz, g.n[2]));
        for (int f = 0; f < nf; f++) z[f * N + gp] = x[f * np + lp];
    }
}

// projection P: sums of z_c and of sign_m(p) z_uI for every null mode m
__global__ void __launch_bounds__(kRedThreads) k_proj_dots(DGrid g, int nf, int evenmask, int nmodes,
                                                           const double *__restrict__ z, double *__restrict__ partials)
{
    const long long N = g.N;
    const int K = 1 + (nf - 2) * nmodes;
    double acc[25];
    for (int i = 0; i < 25; i++) acc[i] = 0.0;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        acc[0] += z[p];
        if (nf > 2) {
            int x, y, zz;
            coords_of(g, p, x, y, zz);
            const int par[3] = {x & 1, y & 1, zz & 1};
            int mi = 0;
            for (int m = 0; m < 8; m++) {
                if ((m & ~evenmask) != 0 || m >= (1 << g.dim)) continue;
                int s = 0;
                for (int J = 0; J < g.dim; J++)
                    if (m & (1 << J)) s += par[J];
                const double sg = (s & 1) ? -1.0 : 1.0;
                for (int I = 0; I < nf - 2; I++) acc[1 + I * nmodes + mi] += sg * z[(2 + I) * N + p];
                mi++;
            }
        }
    }
    __shared__ double red[25][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < K; k++) {
        double a = acc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) red[k][warp] = a;
    }
    __syncthreads();
    if ((int)threadIdx.x < K) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) a += red[threadIdx.x][w];
        partials[(size_t)blockIdx.x * K + threadIdx.x] = a;
    }
}

__global__ void k_proj_sub(DGrid g, int nf, int evenmask, int nmodes, const double *__restrict__ sums,
                           double *__restrict__ z)
{
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long N = g.N;
    if (p >= N) return;
    const double invN = 1.0 / (double)N;
    z[p] -= sums[0] * invN;
    if (nf > 2) {
        int x, y, zz;
        coords_of(g, p, x, y, zz);
        const int par[3] = {x & 1, y & 1, zz & 1};
        int mi = 0;
        for (int m = 0; m < 8; m++) {
            if ((m & ~evenmask) != 0 || m >= (1 << g.dim)) continue;
            int s = 0;
            for (int J = 0; J < g.dim; J++)
                if (m & (1 << J)) s += par[J];
            const double sg = (s & 1) ? -1.0 : 1.0;
            for (int I = 0; I < nf - 2; I++) z[(2 + I) * N + p] -= sums[1 + I * nmodes + mi] * invN * sg;
            mi++;
        }
    }
}

Tables tables_of(const Problem *P)
{
    Tables T;
    for (int f = 0; f <= P->nf; f++) T.rowoff[f] = P->ras->rowoff[f];
    for (int f = 0; f < P->nf; f++) T.diag[f] = P->ras->diag[f];
    T.nf = P->nf;
    return T;
}

}  // namespace

int ras_factor(Problem *P, int mode)
{
    RasPlan *R = P->ras;
    cudaMemsetAsync(P->dflag, 0, sizeof(int), P->stream);
    P->tick(3);
    k_ras_factor<<<R->nsub, R->threads, 0, P->stream>>>(P->g, P->k, P->cur_dt, mode, tables_of(P), R->sub, R->lvl_ptr,
                                                        R->lvl_lp, R->pos_of_lp, R->tmpl, R->slotmap, R->upd_ptr,
                                                        R->upd, P->part, P->mob, R->fac, P->dflag);
    P->tock(3);
    int hflag = 0;
    cudaMemcpyAsync(&hflag, P->dflag, sizeof(int), cudaMemcpyDeviceToHost, P->stream);
    cudaError_t e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) return cuda_fail(P, e, "ras_factor");
    if (hflag & 2) {
        P->err = "zero pivot in an ILU(0) subdomain factorisation";
        return NKS_EPIVOT;
    }
    P->factored = true;
    return NKS_OK;
}

void project(Problem *P, double *z)
{
    RasPlan *R = P->ras;
    const int K = 1 + (P->nf - 2) * R->nmodes;
    P->tick(6);
    k_proj_dots<<<kRedBlocks, kRedThreads, 0, P->stream>>>(P->g, P->nf, R->evenmask, R->nmodes, z, P->partials);
    launch_finalize(P->partials, kRedBlocks, K, R->proj, P->stream);
    k_proj_sub<<<(int)((P->N + 255) / 256), 256, 0, P->stream>>>(P->g, P->nf, R->evenmask, R->nmodes, R->proj, z);
    P->tock(6);
}

void ras_apply(Problem *P, const double *r, double *z)
{
    RasPlan *R = P->ras;
    if (R->smem && R->smem_bytes > 48 * 1024 && !R->attr_set) {
        cudaFuncSetAttribute(k_ras_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R->smem_bytes);
        R->attr_set = true;
    }
    k_ras_apply<<<R->nsub, R->threads, R->smem ? R->smem_bytes : 0, P->stream>>>(
        P->g, tables_of(P), R->sub, R->lvl_ptr, R->lvl_lp, R->tmpl, R->fac, r, z, R->scratch, R->smem ? 1 : 0);
    project(P, z);
}

}  // namespace nks
