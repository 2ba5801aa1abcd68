// nks_api.cu -- C ABI, Newton iteration (Sec. 4) and adaptive time stepping,
// for batches of same-shape instances (a single problem is a batch of one).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>

#include "nks_internal.cuh"
#include "nks_model3.cuh"

namespace nks {

size_t gmres_state_doubles(int m);

static thread_local std::string g_create_error;

// message returned by nks_last_error(NULL) on this thread
void set_thread_error(const char *msg) { g_create_error = msg ? msg : ""; }

int cuda_fail(Problem *P, cudaError_t e, const char *where)
{
    P->err = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    return NKS_ECUDA;
}

void *Problem::dalloc(size_t bytes)
{
    if (bytes == 0) bytes = 8;
    void *p = nullptr;
    if (have_alloc) {
        p = alloc.alloc(bytes, alloc.ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) allocations.push_back(p);
    return p;
}

void Problem::dfree_all()
{
    for (void *p : allocations) {
        if (have_alloc) alloc.free(p, alloc.ctx);
        else cudaFree(p);
    }
    allocations.clear();
}

// kernel-class bookkeeping: launch counts always, CUDA-event intervals with opts.timing
void Problem::tick(int cls)
{
    stats.launches[cls]++;
    if (!opts.timing) return;
    TimerPool &tp = timers[cls];
    if (tp.used == tp.ev.size()) {
        Timer t;
        cudaEventCreate(&t.a);
        cudaEventCreate(&t.b);
        tp.ev.push_back(t);
    }
    cudaEventRecord(tp.ev[tp.used].a, stream);
}

void Problem::tock(int cls)
{
    if (!opts.timing) return;
    TimerPool &tp = timers[cls];
    if (tp.used < tp.ev.size()) cudaEventRecord(tp.ev[tp.used++].b, stream);
}

// accumulate the recorded intervals (synchronises) and recycle the events
static void harvest_timers(Problem *P)
{
    if (!P->opts.timing) return;
    cudaStreamSynchronize(P->stream);
    for (int c = 0; c < NKS_NCLASS; c++) {
        TimerPool &tp = P->timers[c];
        for (size_t i = 0; i < tp.used; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, tp.ev[i].a, tp.ev[i].b) == cudaSuccess) P->stats.ms[c] += ms;
        }
        tp.used = 0;
    }
    cudaGetLastError();
}

static void destroy_timers(Problem *P)
{
    for (int c = 0; c < NKS_NCLASS; c++) {
        for (Timer &t : P->timers[c].ev) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        P->timers[c].ev.clear();
        P->timers[c].used = 0;
    }
}

int Problem::sync_check(const char *where)
{
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(this, e, where);
    return NKS_OK;
}

// ---------------------------------------------------------------------------
// batch helpers.  Uploads go through a ring of pinned staging slots: an
// asynchronous copy reads its slot when the stream reaches it, and the driver
// synchronises far more often than the ring wraps.
// ---------------------------------------------------------------------------

constexpr int kRing = 256;

Bat Problem::set_mask(int m, const std::vector<char> &on)
{
    int *h = hmask_ring + (size_t)(ring_pos++ % kRing) * nb;
    for (int i = 0; i < nb; i++) h[i] = on[i] ? 1 : 0;
    cudaMemcpyAsync(dmask + (size_t)m * nb, h, sizeof(int) * nb, cudaMemcpyHostToDevice, stream);
    return masked(m);
}

void Problem::upload_isc()
{
    double *h = hsc_ring + (size_t)(ring_pos++ % kRing) * nb * I_NSC;
    for (int i = 0; i < nb; i++) {
        double *r = h + (size_t)i * I_NSC;
        for (int q = 0; q < I_NSC; q++) r[q] = 0.0;
        r[I_DT] = is[i].dt > 0.0 ? is[i].dt : 1.0;
        r[I_IDT] = 1.0 / r[I_DT];
        r[I_CBAR0] = is[i].cbar0;
        r[I_LAM] = is[i].lam;
    }
    cudaMemcpy2DAsync(isc, (size_t)stride, h, sizeof(double) * I_NSC, sizeof(double) * I_NSC, (size_t)nb,
                      cudaMemcpyHostToDevice, stream);
}

void Problem::upload_rows(double *dev0, const double *rows, int count)
{
    double *h = hsc_ring + (size_t)(ring_pos++ % kRing) * nb * I_NSC;
    for (int i = 0; i < nb; i++)
        for (int q = 0; q < count; q++) h[(size_t)i * count + q] = rows[(size_t)i * count + q];
    cudaMemcpy2DAsync(dev0, (size_t)stride, h, sizeof(double) * count, sizeof(double) * count, (size_t)nb,
                      cudaMemcpyHostToDevice, stream);
}

// count doubles at dev0 (instance 0's address) of every instance -> hread[i * 64 + q],
// and both flag words of every instance -> hflags[2 i + q]; synchronises
void Problem::enqueue_readback(const double *dev0, int count)
{
    if (dev0 && count > 0)
        cudaMemcpy2DAsync(hread, sizeof(double) * 64, dev0, (size_t)stride, sizeof(double) * count, (size_t)nb,
                          cudaMemcpyDeviceToHost, stream);
    cudaMemcpy2DAsync(hflags, sizeof(int) * 2, dflag, (size_t)stride, sizeof(int) * 2, (size_t)nb,
                      cudaMemcpyDeviceToHost, stream);
}

int Problem::read_scalars(const double *dev0, int count, const char *where)
{
    enqueue_readback(dev0, count);
    return sync_check(where);
}

int Problem::read_flags(const char *where) { return read_scalars(nullptr, 0, where); }

static std::vector<char> only(int nb, int i)
{
    std::vector<char> v(nb, 0);
    v[i] = 1;
    return v;
}

static bool any_of(const std::vector<char> &v)
{
    for (char c : v)
        if (c) return true;
    return false;
}

// App. B: dE_G/dc = M0 + M1(phi) c + M2(phi) c^2 + M3 c^3 + M4 c^4 + ..., with the
// coefficients expressed through the App. A parameters (all divided by V_m dE).
DCoef derive_coefficients(const nks_coeffs &c, int dim, double cbar0)
{
    DCoef k;
    memset(&k, 0, sizeof(k));
    k.kappa = c.kappa;
    k.gamma_c = c.gamma_c;
    k.gamma_eta = c.gamma_eta;
    k.theta = c.theta;
    k.w_psi = c.w_psi;
    const double *L = c.L;
    k.M0 = c.dE0 + (L[0] - L[1] + L[2] - L[3]);
    k.m1a = -(2.0 * L[0] - 6.0 * L[1] + 10.0 * L[2] - 14.0 * L[3]);
    k.m1b = 24.0 * c.U1 + 72.0 * c.U4;
    k.m2a = -(6.0 * L[1] - 24.0 * L[2] + 54.0 * L[3]);
    k.m2b = -216.0 * c.U4;
    k.m2c = -144.0 * c.U4;
    k.M3 = -(16.0 * L[2] - 80.0 * L[3]);
    k.M4 = -40.0 * L[3];
    k.U1 = c.U1;
    k.U4 = c.U4;
    for (int i = 0; i < 4; i++) k.L[i] = L[i];
    k.dE0 = c.dE0;
    k.eps0 = c.eps0;
    k.C11 = c.C11 * c.Lscale;
    k.C12 = c.C12 * c.Lscale;
    k.C44 = c.C44 * c.Lscale;
    k.lam = k.C11 + (dim - 1) * k.C12;
    k.elastic = (k.C11 != 0.0 || k.C12 != 0.0 || k.C44 != 0.0) ? 1 : 0;
    k.ne = c.n_eta == 3 ? 3 : 1;
    k.keta = k.ne == 3 ? 3.0 : 1.0;
    k.nf = 1 + k.ne + (k.elastic ? dim : 0);
    k.S = c.S;
    for (int i = 1; i < 16; i++) {
        k.ser_c[i] = 1.0 / ((2.0 * i) * (2.0 * i + 1.0));
        k.ser_e[i] = 1.0 / (2.0 * i + 1.0);
    }
    k.cbar0 = cbar0;
    return k;
}

// ||F||^2 and the domain flag of every instance in `on` (one launch each)
static int residual(Problem *P, int mode, const double *X1, const double *X0, double *F, double *part,
                    const std::vector<char> &on, std::vector<double> &fn, std::vector<char> &dok)
{
    const Bat bt = P->set_mask(M_X1, on);
    cudaMemset2DAsync(P->dflag, (size_t)P->stride, 0, sizeof(int), (size_t)P->nb, P->stream);
    P->tick(0);
    P->count(launch_residual(P->g, P->k, P->isc, mode, X1, X0, P->tr0, P->mob, P->Gc, P->sig, part, F, P->dflag,
                             P->partials, P->rb, P->stream, bt));
    P->count(launch_finalize(P->partials, P->rb, 1, P->dscal, P->stream, bt));
    P->tock(0);
    int rc = P->read_scalars(P->dscal, 1, "residual");
    if (rc) return rc;
    fn.assign(P->nb, 0.0);
    dok.assign(P->nb, 1);
    for (int i = 0; i < P->nb; i++) {
        if (!on[i]) continue;
        fn[i] = sqrt(P->hread[(size_t)i * 64]);
        dok[i] = (P->hflags[2 * i] & 1) == 0;
    }
    return NKS_OK;
}

// level-n quantities used by every residual of the step
static void prepare_level(Problem *P, const double *X0, const Bat &bt)
{
    P->tick(8);
    P->count(launch_mobility(P->g, P->k, X0, P->mob, P->stream, bt));
    if (P->k.elastic) P->count(launch_trace0(P->g, P->k, P->isc, X0, P->tr0, P->stream, bt));
    P->tock(8);
}

// One NKS solve (Sec. 4) for X^{n+1} of every instance in `on`: X holds the
// starting iterate (X^n), Xn holds X^n, is[i].dt the step (uploaded to isc).
// mode 1 solves the displacement-only system (initial equilibrium).  Outcome
// per instance in is[i]: nst = 0 converged, -status when it failed.  The
// instances run in lockstep; each one does exactly the work it does alone.
static int newton(Problem *P, int mode, double rtol, double atol, int maxit, const std::vector<char> &on)
{
    const long long n = P->nvec;
    const int nbt = P->nb;
    P->cur_mode = mode;
    std::vector<double> fn;
    std::vector<char> dok;
    int rc = residual(P, mode, P->X, P->Xn, P->F, P->part, on, fn, dok);
    if (rc) return rc;
    std::vector<char> run(nbt, 0);
    for (int i = 0; i < nbt; i++) {
        if (!on[i]) continue;
        IState &s = P->is[i];
        s.fn0 = s.fn = fn[i];
        s.newton_its = s.gmres_its = 0;
        s.err.clear();
        s.nst = 0;
        if (!dok[i]) {
            s.nst = -NKS_EDOMAIN;
            s.err = "state outside the domain of the logarithms";
        } else if (!(fn[i] == fn[i]) || isinf(fn[i])) {
            s.nst = -NKS_EDIVERGED;
            s.err = "non-finite residual";
        } else {
            s.tol = std::max(rtol * s.fn0, atol);
            if (s.fn0 > s.tol) {
                s.nst = 1;
                run[i] = 1;
            }
        }
    }
    for (int it = 0; it < maxit && any_of(run); it++) {
        Bat br = P->set_mask(M_RUN, run);
        if (it == 0 || !P->opts.ilu_reuse) {
            rc = ras_factor(P, mode, br, run);
            if (rc) return rc;
            bool changed = false;
            for (int i = 0; i < nbt; i++)
                if (run[i] && P->is[i].nst < 0) {
                    run[i] = 0;
                    changed = true;
                }
            if (!any_of(run)) break;
            if (changed) br = P->set_mask(M_RUN, run);
        }
        P->tick(8);
        P->count(launch_axpby(n, -1.0, P->F, 0.0, P->B, P->stream, br));
        P->tock(8);
        for (int i = 0; i < nbt; i++) {
            IState &s = P->is[i];
            s.gin = run[i] != 0;
            if (s.gin) s.gtol = std::max(P->opts.gmres_rtol * s.fn, P->opts.gmres_atol);
        }
        rc = gmres_solve(P, mode, P->B, P->S);
        if (rc) return rc;
        for (int i = 0; i < nbt; i++)
            if (run[i]) {
                P->is[i].gmres_its += P->is[i].gits;
                P->stats.gmres_its += P->is[i].gits;
            }
        // backtracking line search, each instance with its own lambda
        std::vector<char> ls = run;
        for (int i = 0; i < nbt; i++)
            if (run[i]) {
                P->is[i].lam = 1.0;
                P->is[i].accepted = false;
            }
        while (any_of(ls)) {
            P->upload_isc();
            const Bat bl = P->set_mask(M_LS, ls);
            P->tick(8);
            P->count(launch_waxpy_lam(n, P->X, P->isc, P->S, P->Xt, P->stream, bl));
            P->tock(8);
            rc = residual(P, mode, P->Xt, P->Xn, P->Ft, P->part_t, ls, fn, dok);
            if (rc) return rc;
            for (int i = 0; i < nbt; i++) {
                if (!ls[i]) continue;
                IState &s = P->is[i];
                const double f = fn[i];
                if (dok[i] && f == f && !isinf(f) && f * f <= (1.0 - 2.0 * P->opts.ls_alpha * s.lam) * s.fn * s.fn) {
                    s.accepted = true;
                    s.ftn = f;
                    ls[i] = 0;
                } else {
                    s.lam *= 0.5;
                    if (s.lam < P->opts.ls_lambda_min) ls[i] = 0;
                }
            }
        }
        std::vector<char> acc(nbt, 0);
        for (int i = 0; i < nbt; i++) {
            if (!run[i]) continue;
            IState &s = P->is[i];
            s.newton_its = it + 1;
            P->stats.newton_its++;
            if (!s.accepted) {
                s.nst = -NKS_EDIVERGED;
                s.err = "line search failed";
                run[i] = 0;
            } else {
                acc[i] = 1;
            }
        }
        if (any_of(acc)) {
            const Bat ba = P->set_mask(M_ACC, acc);
            P->tick(8);
            P->count(launch_copy(n, P->Xt, P->X, P->stream, ba));
            P->count(launch_copy(n, P->Ft, P->F, P->stream, ba));
            P->count(launch_copy((1 + P->k.ne) * (1 + P->k.ne) * P->N, P->part_t, P->part, P->stream, ba));
            P->tock(8);
        }
        for (int i = 0; i < nbt; i++) {
            if (!acc[i]) continue;
            IState &s = P->is[i];
            s.fn = s.ftn;
            if (s.fn <= s.tol) {
                s.nst = 0;
                run[i] = 0;
            }
        }
    }
    for (int i = 0; i < nbt; i++)
        if (run[i]) {
            P->is[i].nst = -NKS_EDIVERGED;
            P->is[i].err = "Newton iteration limit reached";
        }
    return NKS_OK;
}

// energy parts (e1..e4, total) and mass of every instance in `on`: parts[5 i + q], mass[i]
static int energy_mass(Problem *P, const double *X, const std::vector<char> &on, std::vector<double> &parts,
                       std::vector<double> &mass)
{
    const Bat bt = P->set_mask(M_X1, on);
    P->tick(7);
    P->count(launch_energy(P->g, P->k, P->isc, X, P->partials, P->rb, P->stream, bt));
    P->count(launch_finalize(P->partials, P->rb, 5, P->dscal, P->stream, bt));
    P->tock(7);
    int rc = P->read_scalars(P->dscal, 5, "energy");
    if (rc) return rc;
    double v = 1.0;
    for (int J = 0; J < P->g.dim; J++) v *= P->g.h;
    parts.assign((size_t)P->nb * 5, 0.0);
    mass.assign(P->nb, 0.0);
    for (int i = 0; i < P->nb; i++) {
        if (!on[i]) continue;
        const double *s = P->hread + (size_t)i * 64;
        for (int q = 0; q < 4; q++) parts[5 * i + q] = s[q] * v;
        parts[5 * i + 4] = (s[0] + s[1] + s[2] + s[3]) * v;
        mass[i] = s[4] * v;
    }
    return NKS_OK;
}

// initial mechanical equilibrium of the instances in `on` (u solved with c, eta fixed)
static int equilibrate(Problem *P, const std::vector<char> &on)
{
    if (!P->k.elastic) return NKS_OK;
    const Bat bt = P->set_mask(M_X2, on);
    P->count(launch_copy(P->nvec, P->Xn, P->X, P->stream, bt));
    for (int i = 0; i < P->nb; i++)
        if (on[i]) P->is[i].dt = 1.0;
    P->upload_isc();
    prepare_level(P, P->Xn, bt);
    int rc = newton(P, 1, P->opts.u0_rtol, P->opts.u0_atol, P->opts.u0_maxit, on);
    if (rc) return rc;
    for (int i = 0; i < P->nb; i++)
        if (on[i] && P->is[i].nst != 0) {
            P->err = P->is[i].err;
            return -P->is[i].nst;
        }
    const Bat b2 = P->set_mask(M_X2, on);
    P->count(launch_copy(P->nvec, P->X, P->Xn, P->stream, b2));
    return NKS_OK;
}

// one accepted time step of every instance in `on` (dt[i] > 0 fixed, else the
// adaptive rule of Sec. 4); per-instance results in info[i]
static int step_batch(Problem *P, const std::vector<char> &on, const double *dt_arg, nks_step_info *info)
{
    const int nbt = P->nb;
    const long long n = P->nvec;
    std::vector<double> dt(nbt, 0.0);
    std::vector<char> fixed(nbt, 0), need(nbt, 0);
    for (int i = 0; i < nbt; i++) {
        if (!on[i]) continue;
        IState &s = P->is[i];
        if (dt_arg && dt_arg[i] > 0.0) {
            dt[i] = dt_arg[i];
            fixed[i] = 1;
        } else if (s.nstep == 0 || P->opts.dt_mode == NKS_DT_FIXED) {
            dt[i] = P->opts.dt_init;
        } else if (P->opts.dt_mode == NKS_DT_SOLUTION) {
            need[i] = 1;
        } else {
            const double Xd = fabs(s.E - s.Eprev) / s.dt_prev;
            dt[i] = std::max(P->opts.dt_min, P->opts.dt_max / sqrt(1.0 + s.zeta * Xd * Xd));  // Eq. sencondt
        }
    }
    if (any_of(need)) {
        const Bat bn = P->set_mask(M_X2, need);
        P->count(launch_waxpy(n, P->Xn, -1.0, P->Xprev, P->W, P->stream, bn));
        P->count(launch_dot2(n, P->W, P->W, P->partials, P->rb, P->stream, bn));
        P->count(launch_finalize(P->partials, P->rb, 2, P->dscal, P->stream, bn));
        int rc = P->read_scalars(P->dscal + 1, 1, "dt");
        if (rc) return rc;
        for (int i = 0; i < nbt; i++)
            if (need[i]) {
                const IState &s = P->is[i];
                const double Xd = sqrt(P->hread[(size_t)i * 64]) / s.dt_prev;
                dt[i] = std::max(P->opts.dt_min, P->opts.dt_max / sqrt(1.0 + s.zeta * Xd * Xd));
            }
    }
    std::vector<int> retries(nbt, 0), status(nbt, NKS_OK);
    for (int i = 0; i < nbt; i++)
        if (on[i] && !P->opts.zeta_persist) P->is[i].zeta = P->opts.zeta;
    std::vector<char> pend = on;
    while (any_of(pend)) {
        const Bat bp = P->set_mask(M_X2, pend);
        P->count(launch_copy(n, P->Xn, P->X, P->stream, bp));
        for (int i = 0; i < nbt; i++)
            if (pend[i]) P->is[i].dt = dt[i];
        P->upload_isc();
        prepare_level(P, P->Xn, bp);
        int rc = newton(P, 0, P->opts.newton_rtol, P->opts.newton_atol, P->opts.newton_maxit, pend);
        if (rc) return rc;
        for (int i = 0; i < nbt; i++) {
            if (!pend[i]) continue;
            IState &s = P->is[i];
            if (s.nst == 0) {
                pend[i] = 0;
                continue;
            }
            const int st = -s.nst;
            if (st == NKS_ECUDA || fixed[i] || retries[i] >= P->opts.max_retries) {
                status[i] = st;
                pend[i] = 0;
                continue;
            }
            // Sec. 4: a diverged NKS solve restarts with dt / sqrt(2) and zeta doubled
            dt[i] /= sqrt(2.0);
            s.zeta *= 2.0;
            retries[i]++;
            P->stats.retries++;
        }
    }
    std::vector<char> ok(nbt, 0);
    for (int i = 0; i < nbt; i++) ok[i] = on[i] && status[i] == NKS_OK;
    std::vector<double> parts, mass;
    if (any_of(ok)) {
        const Bat bs = P->set_mask(M_X2, ok);
        P->count(launch_copy(n, P->Xn, P->Xprev, P->stream, bs));  // X^{n-1} <- X^n
        P->count(launch_copy(n, P->X, P->Xn, P->stream, bs));      // X^n <- X^{n+1}
        int rc = energy_mass(P, P->Xn, ok, parts, mass);
        if (rc) return rc;
    }
    for (int i = 0; i < nbt; i++) {
        if (!on[i]) continue;
        IState &s = P->is[i];
        nks_step_info f{};
        f.dt = dt[i];
        f.retries = retries[i];
        f.newton_its = s.newton_its;
        f.gmres_its = s.gmres_its;
        f.fnorm0 = s.fn0;
        f.fnorm = s.fn;
        if (ok[i]) {
            s.Eprev = s.E;
            s.E = parts[5 * i + 4];
            s.t += dt[i];
            s.dt_prev = dt[i];
            s.nstep++;
            P->stats.steps++;
            f.mass = mass[i];
        }
        f.t = s.t;
        f.energy = s.E;
        f.status = status[i];
        if (info) info[i] = f;
    }
    return NKS_OK;
}

// c and the site fractions in (0, 1): c eta and c (4 - 3 eta), or with three order
// parameters (eta: ne planes of N) c eta_i for i = 1..4, eta_4 = 4 - sum
static bool host_in_domain(long long N, int ne, const double *c, const double *e)
{
    for (long long p = 0; p < N; p++) {
        bool ok = c[p] > 0.0 && c[p] < 1.0;
        if (ne == 3) {
            const double e4 = 4.0 - e[p] - e[N + p] - e[2 * N + p];
            for (int i = 0; i < 4; i++) {
                const double q = c[p] * (i < 3 ? e[i * N + p] : e4);
                ok = ok && q > 0.0 && q < 1.0;
            }
        } else {
            const double pp = c[p] * e[p], q = c[p] * (4.0 - 3.0 * e[p]);
            ok = ok && pp > 0.0 && pp < 1.0 && q > 0.0 && q < 1.0;
        }
        if (!ok) return false;
    }
    return true;
}

static const char *domain_message(int ne)
{
    return ne == 3 ? "initial state outside the domain: c and c*eta_i (i = 1..4, eta_4 = 4 - sum) must lie in (0, 1)"
                   : "initial state outside the domain: c, c*eta and c*(4-3*eta) must lie in (0, 1)";
}

// fields of one instance into its X^n (c, eta_1..eta_ne; u = 0) and its level-0 scalars
static void load_fields(Problem *P, int i, const double *c, const double *eta)
{
    const size_t fb = sizeof(double) * (size_t)P->N;
    double *Xn = shift(P->Xn, (long long)i * P->stride);
    cudaMemsetAsync(Xn, 0, sizeof(double) * (size_t)P->ldv, P->stream);
    cudaMemcpyAsync(Xn, c, fb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(Xn + P->N, eta, fb * P->k.ne, cudaMemcpyHostToDevice, P->stream);
    double s = 0.0;
    for (long long p = 0; p < P->N; p++) s += c[p];
    IState &st = P->is[i];
    st = IState{};
    st.cbar0 = s / (double)P->N;
    st.zeta = P->opts.zeta;
    st.dt_prev = P->opts.dt_init;
    st.lam = 1.0;
}

// after load_fields: equilibrium, X^{n-1} = X^n, energy
static int init_instances(Problem *P, const std::vector<char> &on)
{
    P->upload_isc();
    int rc = P->sync_check("load");
    if (!rc) rc = equilibrate(P, on);
    if (rc) return rc;
    const Bat bt = P->set_mask(M_X2, on);
    P->count(launch_copy(P->nvec, P->Xn, P->Xprev, P->stream, bt));
    std::vector<double> parts, mass;
    rc = energy_mass(P, P->Xn, on, parts, mass);
    if (rc) return rc;
    for (int i = 0; i < P->nb; i++)
        if (on[i]) {
            P->is[i].E = P->is[i].Eprev = parts[5 * i + 4];
            P->is[i].loaded = true;
        }
    return NKS_OK;
}

}  // namespace nks

using namespace nks;

struct nks_problem {
    Problem P;
};


extern "C" {

void nks_default_opts(nks_opts *o)
{
    memset(o, 0, sizeof(*o));
    o->newton_rtol = 1e-10;
    o->newton_atol = 1e-12;
    o->newton_maxit = 20;
    o->ls_alpha = 1e-4;
    o->ls_lambda_min = 1.0 / 1024.0;
    o->gmres_restart = 30;
    o->gmres_maxit = 300;
    o->gmres_rtol = 1e-6;
    o->gmres_atol = 1e-14;
    o->sub[0] = o->sub[1] = 4;
    o->sub[2] = 1;
    o->overlap = 1;
    o->ilu_reuse = 1;
    o->precision = NKS_FP64;
    o->dt_init = 0.01;
    o->dt_min = 0.01;
    o->dt_max = 2.0;
    o->zeta = 100.0;
    o->dt_mode = NKS_DT_FIXED;
    o->zeta_persist = 0;
    o->max_retries = 8;
    o->u0_rtol = 1e-12;
    o->u0_atol = 1e-13;
    o->u0_maxit = 10;
    o->timing = 0;
    o->graphs = 1;
}

static int validate(const nks_grid *grid, const nks_coeffs *coeffs, const nks_opts *opts, int nb)
{
    if (!grid || !coeffs || !opts) {
        g_create_error = "null argument";
        return NKS_EINVAL;
    }
    if (grid->dim < 1 || grid->dim > 3 || !(grid->h > 0.0)) {
        g_create_error = "grid: dim must be 1..3 and h > 0";
        return NKS_EINVAL;
    }
    if (grid->bc != NKS_PERIODIC && grid->bc != NKS_NEUMANN) {
        g_create_error = "grid: bc must be NKS_PERIODIC or NKS_NEUMANN";
        return NKS_EINVAL;
    }
    long long npts = 1;
    for (int J = 0; J < grid->dim; J++) {
        if (grid->n[J] < 3) {
            g_create_error = "grid: at least 3 cells per axis";
            return NKS_EINVAL;
        }
        npts *= grid->n[J];
    }
    if (coeffs->n_eta != 0 && coeffs->n_eta != 1 && coeffs->n_eta != 3) {
        g_create_error = "coeffs: n_eta must be 1 (0 reads as 1) or 3";
        return NKS_EINVAL;
    }
    // the pointwise derivative block: (1 + n_eta)^2 planes
    const int ne = coeffs->n_eta == 3 ? 3 : 1, planes = std::max(1 + ne + grid->dim, (1 + ne) * (1 + ne));
    if (npts * planes >= (1LL << 31)) {
        // stencil kernels index the field planes with 32-bit offsets
        g_create_error = "grid: (1 + n_eta + dim) * points and (1 + n_eta)^2 * points must be below 2^31";
        return NKS_EINVAL;
    }
    if (nb < 1 || nb > 65535 || (grid->dim == 3 && (long long)grid->n[2] * nb > 65535)) {
        g_create_error = "batch: 1 <= nb <= 65535 (and n_z * nb <= 65535 in 3-D)";
        return NKS_EINVAL;
    }
    if (coeffs->S < 1 || coeffs->S > 16) {
        g_create_error = "coeffs: S must be in 1..16";
        return NKS_EINVAL;
    }
    if (opts->gmres_restart < 1 || opts->gmres_restart > 31) {
        g_create_error = "opts: gmres_restart must be in 1..31";
        return NKS_EINVAL;
    }
    if (opts->precision != NKS_FP64 && opts->precision != NKS_MIXED) {
        g_create_error = "opts: precision must be NKS_FP64 or NKS_MIXED";
        return NKS_EINVAL;
    }
    if (opts->u0_mixed != 0 && opts->u0_mixed != 1) {
        g_create_error = "opts: u0_mixed must be 0 or 1";
        return NKS_EINVAL;
    }
    if (opts->ras_variant < NKS_LEFT_RAS || opts->ras_variant > NKS_RIGHT_RAS) {
        g_create_error = "opts: ras_variant must be NKS_LEFT_RAS, NKS_AS or NKS_RIGHT_RAS";
        return NKS_EINVAL;
    }
    return NKS_OK;
}

int nks_create_batch(const nks_grid *grid, int nb, const double *c, const double *eta, const nks_coeffs *coeffs,
                     const nks_opts *opts, const nks_allocator *alloc, void *stream, nks_problem **out)
{
    if (!out) {
        g_create_error = "null argument";
        return NKS_EINVAL;
    }
    *out = nullptr;
    g_create_error.clear();
    int rc = validate(grid, coeffs, opts, nb);
    if (rc) return rc;
    if ((c == nullptr) != (eta == nullptr)) {
        g_create_error = "c and eta must both be given or both be NULL";
        return NKS_EINVAL;
    }
    long long N = 1;
    for (int J = 0; J < grid->dim; J++) N *= grid->n[J];
    const int ne = coeffs->n_eta == 3 ? 3 : 1;
    if (c)
        for (int i = 0; i < nb; i++)
            if (!host_in_domain(N, ne, c + (size_t)i * N, eta + (size_t)i * ne * N)) {
                g_create_error = domain_message(ne);
                return NKS_EDOMAIN;
            }
    nks_problem *H = new nks_problem();
    Problem *P = &H->P;
    cudaGetDevice(&P->device);
    P->grid = *grid;
    P->coeffs = *coeffs;
    P->opts = *opts;
    P->nb = nb;
    P->is.assign(nb, IState{});
    if (alloc && alloc->alloc && alloc->free) {
        P->alloc = *alloc;
        P->have_alloc = true;
    }
    if (stream) {
        P->stream = (cudaStream_t)stream;
    } else {
        cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
        P->own_stream = true;
    }
    DGrid &g = P->g;
    g.dim = grid->dim;
    for (int J = 0; J < 3; J++) g.n[J] = J < grid->dim ? grid->n[J] : 1;
    g.N = N;
    g.bc = grid->bc;
    set_spacing(g, grid->h);
    P->N = N;
    P->k = derive_coefficients(*coeffs, g.dim, 0.0);  // the mean composition of each instance lives in isc
    P->nf = P->k.nf;
    P->nvec = P->nf * g.N;
    P->ldv = (P->nvec + 1) & ~1LL;
    P->ldvf = (P->nvec + 3) & ~3LL;
    P->rb = (int)std::min<long long>(kRedBlocks, std::max<long long>(1, (P->ldv / 2 + 4 * kRedThreads - 1) /
                                                                           (4 * kRedThreads)));
    std::string err;
    rc = ras_plan_create(P, err);
    if (rc) {
        g_create_error = err;
        nks_destroy(H);
        return rc;
    }

    // per-instance slab: every buffer an instance owns, 256-byte aligned
    const size_t vb = sizeof(double) * (size_t)P->ldv, fb = sizeof(double) * (size_t)g.N;
    const int m = opts->gmres_restart;
    const bool mixed = opts->precision == NKS_MIXED;
    P->f32 = mixed || (opts->u0_mixed && P->k.elastic);
    std::vector<SlabItem> items;
    auto add = [&](void *pp, size_t bytes) { items.push_back({(void **)pp, bytes}); };
    double **vecs[] = {&P->Xn, &P->Xprev, &P->X, &P->Xt, &P->F, &P->Ft, &P->S, &P->B, &P->W, &P->Z, &P->R,
                       &P->T64};
    for (double **v : vecs) add(v, vb);
    add(&P->V, vb * (mixed ? 1 : m + 1));
    const int npart = (1 + P->k.ne) * (1 + P->k.ne);  // pointwise derivative block per point
    add(&P->part, npart * fb);
    add(&P->part_t, npart * fb);
    add(&P->mob, (size_t)g.dim * fb);
    add(&P->tr0, fb);
    add(&P->Gc, fb);
    add(&P->sig, 6 * fb);
    add(&P->partials, sizeof(double) * kRedBlocks * 64);
    add(&P->dscal, sizeof(double) * 64);
    add(&P->dflag, sizeof(int) * 4);
    add(&P->tickets, sizeof(unsigned int) * 16);
    add(&P->zsum, sizeof(double) * 8);
    add(&P->gm, sizeof(double) * gmres_state_doubles(m));
    add(&P->isc, sizeof(double) * I_NSC);
    if (P->f32) {
        const size_t fvb = sizeof(float) * (size_t)P->ldvf;
        add(&P->Vf, fvb * (m + 1));
        add(&P->Wf, fvb);
        add(&P->Zf, fvb);
        add(&P->partf, sizeof(float) * npart * (size_t)g.N);
        add(&P->mobf, sizeof(float) * g.dim * (size_t)g.N);
    }
    ras_slab_items(P, items);
    std::vector<size_t> off(items.size());
    size_t total = 0;
    for (size_t q = 0; q < items.size(); q++) {
        total = (total + 255) & ~(size_t)255;
        off[q] = total;
        total += items[q].bytes;
    }
    P->stride = (long long)((total + 255) & ~(size_t)255);
    P->slab = (char *)P->dalloc((size_t)P->stride * nb);
    P->dmask = (int *)P->dalloc(sizeof(int) * kMasks * nb);
    bool ok = P->slab && P->dmask &&
              cudaMallocHost((void **)&P->hread, sizeof(double) * 64 * nb) == cudaSuccess &&
              cudaMallocHost((void **)&P->hflags, sizeof(int) * 2 * nb) == cudaSuccess &&
              cudaMallocHost((void **)&P->hmask_ring, sizeof(int) * kRing * nb) == cudaSuccess &&
              cudaMallocHost((void **)&P->hsc_ring, sizeof(double) * kRing * nb * I_NSC) == cudaSuccess;
    if (!ok) {
        g_create_error = "out of device memory";
        nks_destroy(H);
        return NKS_ENOMEM;
    }
    for (size_t q = 0; q < items.size(); q++) *items[q].ptr = P->slab + off[q];
    ras_prepare_launch(P);
    if (P->f32) prepare_jv32(P->g, P->k);
    cudaMemsetAsync(P->slab, 0, (size_t)P->stride * nb, P->stream);
    cudaMemsetAsync(P->dmask, 0, sizeof(int) * kMasks * nb, P->stream);
    rc = P->sync_check("create");
    if (!rc && c) {
        for (int i = 0; i < nb; i++) load_fields(P, i, c + (size_t)i * N, eta + (size_t)i * ne * N);
        rc = init_instances(P, std::vector<char>(nb, 1));
    }
    if (rc) {
        g_create_error = P->err.empty() ? "initial equilibrium failed" : P->err;
        nks_destroy(H);
        return rc;
    }
    harvest_timers(P);
    *out = H;
    return NKS_OK;
}

int nks_create_problem(const nks_grid *grid, const double *c, const double *eta, const nks_coeffs *coeffs,
                       const nks_opts *opts, const nks_allocator *alloc, void *stream, nks_problem **out)
{
    if (!c || !eta) {
        g_create_error = "null argument";
        if (out) *out = nullptr;
        return NKS_EINVAL;
    }
    return nks_create_batch(grid, 1, c, eta, coeffs, opts, alloc, stream, out);
}

int nks_batch_size(const nks_problem *H) { return H ? H->P.nb : 0; }

static int check_slot(Problem *P, int slot, bool loaded)
{
    if (slot < 0 || slot >= P->nb) {
        P->err = "slot out of range";
        return NKS_EINVAL;
    }
    if (loaded && !P->is[slot].loaded) {
        P->err = "slot holds no problem";
        return NKS_EINVAL;
    }
    return NKS_OK;
}

int nks_batch_load(nks_problem *H, int slot, const double *c, const double *eta)
{
    Problem *P = &H->P;
    P->err.clear();
    int rc = check_slot(P, slot, false);
    if (rc) return rc;
    if (!c || !eta) {
        P->err = "null argument";
        return NKS_EINVAL;
    }
    if (!host_in_domain(P->N, P->k.ne, c, eta)) {
        P->err = domain_message(P->k.ne);
        return NKS_EDOMAIN;
    }
    load_fields(P, slot, c, eta);
    rc = init_instances(P, only(P->nb, slot));
    if (rc) P->is[slot].loaded = false;
    harvest_timers(P);
    return rc;
}

int nks_batch_unload(nks_problem *H, int slot)
{
    Problem *P = &H->P;
    int rc = check_slot(P, slot, false);
    if (rc) return rc;
    P->is[slot].loaded = false;
    return NKS_OK;
}

int nks_batch_loaded(const nks_problem *H, int slot)
{
    const Problem *P = &H->P;
    return slot >= 0 && slot < P->nb && P->is[slot].loaded ? 1 : 0;
}

int nks_batch_step(nks_problem *H, const int *active, const double *dt, nks_step_info *infos)
{
    Problem *P = &H->P;
    P->err.clear();
    std::vector<char> on(P->nb, 0);
    for (int i = 0; i < P->nb; i++) on[i] = P->is[i].loaded && (!active || active[i]);
    int rc = step_batch(P, on, dt, infos);
    harvest_timers(P);
    if (rc) return rc;
    for (int i = 0; i < P->nb; i++)
        if (on[i] && infos && infos[i].status != NKS_OK && P->err.empty()) P->err = P->is[i].err;
    return NKS_OK;
}

int nks_step(nks_problem *H, double dt_arg, nks_step_info *info_out)
{
    Problem *P = &H->P;
    P->err.clear();
    int rc = check_slot(P, 0, true);
    if (rc) return rc;
    std::vector<double> dts(P->nb, 0.0);
    dts[0] = dt_arg;
    std::vector<nks_step_info> infos(P->nb);
    rc = step_batch(P, only(P->nb, 0), dts.data(), infos.data());
    harvest_timers(P);
    if (rc) return rc;
    if (info_out) *info_out = infos[0];
    if (infos[0].status != NKS_OK) {
        P->err = P->is[0].err;
        return infos[0].status;
    }
    return NKS_OK;
}

int nks_batch_energy(const nks_problem *H, int slot, double *out)
{
    Problem *P = const_cast<Problem *>(&H->P);
    int rc = check_slot(P, slot, true);
    if (rc) return rc;
    *out = P->is[slot].E;
    return NKS_OK;
}

int nks_batch_mass(const nks_problem *H, int slot, double *out)
{
    Problem *P = const_cast<Problem *>(&H->P);
    int rc = check_slot(P, slot, true);
    if (rc) return rc;
    std::vector<double> parts, mass;
    rc = energy_mass(P, P->Xn, only(P->nb, slot), parts, mass);
    if (!rc) *out = mass[slot];
    return rc;
}

int nks_batch_get_fields(const nks_problem *H, int slot, double *c, double *eta, double *u)
{
    Problem *P = const_cast<Problem *>(&H->P);
    int rc = check_slot(P, slot, true);
    if (rc) return rc;
    const size_t fb = sizeof(double) * (size_t)P->N;
    const double *Xn = shift(P->Xn, (long long)slot * P->stride);
    if (c) cudaMemcpyAsync(c, Xn, fb, cudaMemcpyDeviceToHost, P->stream);
    if (eta) cudaMemcpyAsync(eta, Xn + P->N, fb * P->k.ne, cudaMemcpyDeviceToHost, P->stream);
    if (u && P->k.elastic)
        cudaMemcpyAsync(u, Xn + (1 + P->k.ne) * P->N, fb * P->g.dim, cudaMemcpyDeviceToHost, P->stream);
    return P->sync_check("get_fields");
}

int nks_energy(const nks_problem *H, double *out) { return nks_batch_energy(H, 0, out); }

int nks_mass(const nks_problem *H, double *out) { return nks_batch_mass(H, 0, out); }

int nks_get_fields(const nks_problem *H, double *c, double *eta, double *u)
{
    return nks_batch_get_fields(H, 0, c, eta, u);
}

int nks_model3_point(const nks_coeffs *coeffs, const double *x1, const double *x0, double *G, double *dG)
{
    if (!coeffs || !x1 || !x0 || !G || !dG || coeffs->S < 1 || coeffs->S > 16) return NKS_EINVAL;
    const DCoef k = derive_coefficients(*coeffs, 1, 0.0);
    model3_block(k, x1, x0, G, dG);
    return NKS_OK;
}

int nks_debug_withhold_copy(nks_problem *H, int on)
{
    if (!H) return NKS_EINVAL;
    H->P.withhold_copy = on ? 1 : 0;
    // replayed graphs hold the flag in their kernel arguments: capture them again
    destroy_graphs(&H->P);
    return NKS_OK;
}

size_t nks_device_bytes(const nks_problem *H)
{
    const Problem *P = &H->P;
    return (size_t)P->stride * P->nb;
}

struct StateHeader {
    char magic[8];
    long long nvec, nstep;
    double t, dt_prev, zeta, E, Eprev, cbar0;
};

size_t nks_state_size(const nks_problem *H) { return sizeof(StateHeader) + 2 * sizeof(double) * (size_t)H->P.nvec; }

int nks_batch_get_state(const nks_problem *H, int slot, void *buf, size_t bytes)
{
    Problem *P = const_cast<Problem *>(&H->P);
    int rc = check_slot(P, slot, true);
    if (rc) return rc;
    if (!buf || bytes < nks_state_size(H)) {
        P->err = "state buffer too small";
        return NKS_EINVAL;
    }
    const IState &s = P->is[slot];
    StateHeader hd;
    memcpy(hd.magic, "NKSSTAT2", 8);
    hd.nvec = P->nvec;
    hd.nstep = s.nstep;
    hd.t = s.t;
    hd.dt_prev = s.dt_prev;
    hd.zeta = s.zeta;
    hd.E = s.E;
    hd.Eprev = s.Eprev;
    hd.cbar0 = s.cbar0;
    memcpy(buf, &hd, sizeof(hd));
    char *b = (char *)buf + sizeof(hd);
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    const long long io = (long long)slot * P->stride;
    cudaMemcpyAsync(b, shift(P->Xn, io), vb, cudaMemcpyDeviceToHost, P->stream);
    cudaMemcpyAsync(b + vb, shift(P->Xprev, io), vb, cudaMemcpyDeviceToHost, P->stream);
    return P->sync_check("get_state");
}

int nks_batch_set_state(nks_problem *H, int slot, const void *buf, size_t bytes)
{
    Problem *P = &H->P;
    int rc = check_slot(P, slot, false);
    if (rc) return rc;
    StateHeader hd;
    if (!buf || bytes < sizeof(hd)) {
        P->err = "state buffer too small";
        return NKS_EINVAL;
    }
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "NKSSTAT2", 8) != 0 || hd.nvec != P->nvec || bytes < nks_state_size(H)) {
        P->err = "state buffer does not match this problem";
        return NKS_EINVAL;
    }
    const char *b = (const char *)buf + sizeof(hd);
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    const long long io = (long long)slot * P->stride;
    cudaMemcpyAsync(shift(P->Xn, io), b, vb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(shift(P->Xprev, io), b + vb, vb, cudaMemcpyHostToDevice, P->stream);
    IState &s = P->is[slot];
    s = IState{};
    s.nstep = hd.nstep;
    s.t = hd.t;
    s.dt_prev = hd.dt_prev;
    s.zeta = hd.zeta;
    s.E = hd.E;
    s.Eprev = hd.Eprev;
    s.cbar0 = hd.cbar0;
    s.lam = 1.0;
    s.loaded = true;
    P->upload_isc();
    return P->sync_check("set_state");
}

int nks_get_state(const nks_problem *H, void *buf, size_t bytes) { return nks_batch_get_state(H, 0, buf, bytes); }

int nks_set_state(nks_problem *H, const void *buf, size_t bytes) { return nks_batch_set_state(H, 0, buf, bytes); }

int nks_get_stats(const nks_problem *H, nks_stats *out)
{
    *out = H->P.stats;
    return NKS_OK;
}

int nks_reset_stats(nks_problem *H)
{
    nks_stats keep = H->P.stats;  // plan figures survive a reset
    memset(&H->P.stats, 0, sizeof(nks_stats));
    H->P.stats.factor_bytes = keep.factor_bytes;
    H->P.stats.schwarz_points = keep.schwarz_points;
    H->P.stats.schwarz_bytes = keep.schwarz_bytes;
    H->P.stats.schwarz_flops = keep.schwarz_flops;
    return NKS_OK;
}

void nks_destroy(nks_problem *H)
{
    if (!H) return;
    Problem *P = &H->P;
    if (P->stream) cudaStreamSynchronize(P->stream);
    harvest_timers(P);
    destroy_timers(P);
    destroy_graphs(P);
    ras_plan_destroy(P);
    P->dfree_all();
    if (P->hread) cudaFreeHost(P->hread);
    if (P->hflags) cudaFreeHost(P->hflags);
    if (P->hmask_ring) cudaFreeHost(P->hmask_ring);
    if (P->hsc_ring) cudaFreeHost(P->hsc_ring);
    if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
    delete H;
}

const char *nks_last_error(const nks_problem *H)
{
    if (!H) return g_create_error.c_str();
    return H->P.err.c_str();
}

// ---------------------------------------------------------------------------
// operator-level entry points (instance 0)
// ---------------------------------------------------------------------------

static int op_setup(Problem *P, const double *X1, const double *X0, double dt, int mode)
{
    P->err.clear();
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    cudaMemcpyAsync(P->X, X1, vb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(P->Xt, X0, vb, cudaMemcpyHostToDevice, P->stream);
    P->cur_mode = mode;
    P->is[0].dt = dt;
    P->upload_isc();
    const std::vector<char> on = only(P->nb, 0);
    const Bat bt = P->set_mask(M_X2, on);
    P->tick(8);
    P->count(launch_mobility(P->g, P->k, P->Xt, P->mob, P->stream, bt));
    if (P->k.elastic) P->count(launch_trace0(P->g, P->k, P->isc, P->Xt, P->tr0, P->stream, bt));
    P->tock(8);
    std::vector<double> fn;
    std::vector<char> dok;
    return residual(P, mode, P->X, P->Xt, P->F, P->part, on, fn, dok);
}

static int op_finish(Problem *P, int rc)
{
    int r2 = P->sync_check("operator");
    harvest_timers(P);
    return rc ? rc : r2;
}

int nks_eval_residual(nks_problem *H, const double *X1, const double *X0, double dt, int mode, double *F)
{
    Problem *P = &H->P;
    int rc = op_setup(P, X1, X0, dt, mode);
    if (!rc) {
        cudaMemcpyAsync(F, P->F, sizeof(double) * (size_t)P->nvec, cudaMemcpyDeviceToHost, P->stream);
        rc = P->sync_check("eval_residual");
    }
    return op_finish(P, rc);
}

int nks_apply_jacobian(nks_problem *H, const double *X1, const double *X0, double dt, int mode, const double *v,
                       double *Jv)
{
    Problem *P = &H->P;
    int rc = op_setup(P, X1, X0, dt, mode);
    if (!rc) {
        const size_t vb = sizeof(double) * (size_t)P->nvec;
        const Bat bt = P->set_mask(M_X2, only(P->nb, 0));
        cudaMemcpyAsync(P->B, v, vb, cudaMemcpyHostToDevice, P->stream);
        P->tick(1);
        if (P->opts.precision == NKS_MIXED) {
            // as the Arnoldi step applies it: FP32 vectors, coefficients and arithmetic
            refresh_f32_coefficients(P, bt);
            P->count(launch_convert(P->nvec, P->B, P->Zf, P->stream, bt));
            P->count(launch_jv32(P->g, P->k, P->isc, mode, P->partf, P->mobf, P->Zf, P->Wf, P->stream, bt, nullptr));
            P->count(launch_convert(P->nvec, P->Wf, P->W, P->stream, bt));
        } else {
            P->count(launch_jv64(P->g, P->k, P->isc, mode, P->part, P->mob, P->B, P->Gc, P->sig, P->W, P->stream,
                                 bt));
        }
        P->tock(1);
        cudaMemcpyAsync(Jv, P->W, vb, cudaMemcpyDeviceToHost, P->stream);
        rc = P->sync_check("apply_jacobian");
    }
    return op_finish(P, rc);
}

int nks_apply_preconditioner(nks_problem *H, const double *X1, const double *X0, double dt, const double *r, double *z)
{
    Problem *P = &H->P;
    int rc = op_setup(P, X1, X0, dt, 0);
    const std::vector<char> on = only(P->nb, 0);
    const Bat bt = P->set_mask(M_X2, on);
    P->is[0].nst = 1;
    if (!rc) rc = ras_factor(P, 0, bt, on);
    if (!rc && P->is[0].nst < 0) {
        P->err = P->is[0].err;
        rc = -P->is[0].nst;
    }
    if (!rc) {
        const size_t vb = sizeof(double) * (size_t)P->nvec;
        cudaMemcpyAsync(P->B, r, vb, cudaMemcpyHostToDevice, P->stream);
        if (P->opts.precision == NKS_MIXED) {
            // as the solver applies it: FP32 vectors and factors
            P->count(launch_convert(P->nvec, P->B, P->Wf, P->stream, bt));
            ras_apply_projected<float>(P, P->Wf, P->Zf, bt);
            P->count(launch_convert(P->nvec, P->Zf, P->Z, P->stream, bt));
        } else {
            ras_apply(P, P->B, P->Z, bt);
        }
        cudaMemcpyAsync(z, P->Z, vb, cudaMemcpyDeviceToHost, P->stream);
        rc = P->sync_check("apply_preconditioner");
    }
    return op_finish(P, rc);
}

int nks_linear_solve(nks_problem *H, const double *X1, const double *X0, double dt, int mode, const double *b,
                     double *x, double tol, int *its, double *res)
{
    Problem *P = &H->P;
    int rc = op_setup(P, X1, X0, dt, mode);
    const std::vector<char> on = only(P->nb, 0);
    const Bat bt = P->set_mask(M_X2, on);
    P->is[0].nst = 1;
    if (!rc) rc = ras_factor(P, mode, bt, on);
    if (!rc && P->is[0].nst < 0) {
        P->err = P->is[0].err;
        rc = -P->is[0].nst;
    }
    if (!rc) {
        const size_t vb = sizeof(double) * (size_t)P->nvec;
        cudaMemcpyAsync(P->B, b, vb, cudaMemcpyHostToDevice, P->stream);
        for (int i = 0; i < P->nb; i++) P->is[i].gin = i == 0;
        P->is[0].gtol = tol;
        rc = gmres_solve(P, mode, P->B, P->S);
        if (!rc) {
            if (its) *its = P->is[0].gits;
            if (res) *res = P->is[0].res;
            cudaMemcpyAsync(x, P->S, vb, cudaMemcpyDeviceToHost, P->stream);
            rc = P->sync_check("linear_solve");
        }
    }
    return op_finish(P, rc);
}

int nks_eval_energy(nks_problem *H, const double *X, double *parts, double *mass)
{
    Problem *P = &H->P;
    cudaMemcpyAsync(P->W, X, sizeof(double) * (size_t)P->nvec, cudaMemcpyHostToDevice, P->stream);
    std::vector<double> pv, mv;
    int rc = energy_mass(P, P->W, only(P->nb, 0), pv, mv);
    if (!rc) {
        if (parts)
            for (int q = 0; q < 5; q++) parts[q] = pv[q];
        if (mass) *mass = mv[0];
    }
    harvest_timers(P);
    return rc;
}

// ---------------------------------------------------------------------------
// autotuner of the Schwarz decomposition
// ---------------------------------------------------------------------------

// built-in candidates: owned boxes of side b per axis (squares / cubes) with
// overlap 1 or 2, for the sides that give at least two boxes per axis
static std::vector<int> default_candidates(const nks_grid *g)
{
    static const int sides2[] = {16, 24, 32, 48, 64, 128};
    static const int sides3[] = {8, 12, 16, 24, 32};
    std::vector<int> out;
    const int *sides = g->dim == 3 ? sides3 : sides2;
    const int ns = g->dim == 3 ? 5 : 6;
    int nmin = g->n[0];
    for (int J = 1; J < g->dim; J++) nmin = std::min(nmin, g->n[J]);
    for (int q = 0; q < ns; q++) {
        const int b = g->dim == 1 ? sides[q] * 4 : sides[q];
        if (2 * b > nmin) continue;
        for (int ov = 1; ov <= 2; ov++) {
            int sub[3] = {1, 1, 1};
            for (int J = 0; J < g->dim; J++) sub[J] = std::max(1, (g->n[J] + b / 2) / b);
            out.insert(out.end(), {sub[0], sub[1], sub[2], ov});
        }
    }
    return out;
}

int nks_autotune(const nks_grid *grid, const double *c, const double *eta, const nks_coeffs *coeffs,
                 const nks_opts *base, const int *cands, int ncand, double dt_trial, nks_opts *best, double *times,
                 int *chosen)
{
    g_create_error.clear();
    if (!grid || !c || !eta || !coeffs || !base || !best || !(dt_trial > 0.0) || (cands && ncand < 1)) {
        g_create_error = "nks_autotune: invalid argument";
        return NKS_EINVAL;
    }
    std::vector<int> list = cands ? std::vector<int>(cands, cands + 4 * ncand) : default_candidates(grid);
    const int nc = (int)list.size() / 4;
    if (nc == 0) {
        g_create_error = "nks_autotune: no candidate decomposition fits this grid";
        return NKS_EINVAL;
    }
    double best_t = -1.0;
    int best_q = -1;
    for (int q = 0; q < nc; q++) {
        nks_opts o = *base;
        for (int J = 0; J < 3; J++) o.sub[J] = list[4 * q + J];
        o.overlap = list[4 * q + 3];
        o.timing = 0;
        double t = -1.0;
        nks_problem *H = nullptr;
        if (nks_create_problem(grid, c, eta, coeffs, &o, nullptr, nullptr, &H) == NKS_OK) {
            // the first step captures the iteration graphs; the second is timed
            nks_step_info info{};
            if (nks_step(H, dt_trial, &info) == NKS_OK) {
                const auto t0 = std::chrono::steady_clock::now();
                const int rc = nks_step(H, dt_trial, &info);
                const auto t1 = std::chrono::steady_clock::now();
                if (rc == NKS_OK) t = std::chrono::duration<double>(t1 - t0).count();
            }
            nks_destroy(H);
        }
        cudaGetLastError();
        if (times) times[q] = t;
        if (t > 0.0 && (best_q < 0 || t < best_t)) {
            best_t = t;
            best_q = q;
        }
    }
    if (best_q < 0) {
        g_create_error = "nks_autotune: every candidate failed";
        return NKS_EDIVERGED;
    }
    *best = *base;
    for (int J = 0; J < 3; J++) best->sub[J] = list[4 * best_q + J];
    best->overlap = list[4 * best_q + 3];
    if (chosen) *chosen = best_q;
    return NKS_OK;
}

}  // extern "C"
