// nks_api.cu -- C ABI, Newton iteration (Sec. 4) and adaptive time stepping.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "nks_internal.cuh"

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
    k.nf = 2 + (k.elastic ? dim : 0);
    k.S = c.S;
    for (int i = 1; i < 16; i++) {
        k.ser_c[i] = 1.0 / ((2.0 * i) * (2.0 * i + 1.0));
        k.ser_e[i] = 1.0 / (2.0 * i + 1.0);
    }
    k.cbar0 = cbar0;
    return k;
}

// ||F||^2 after launch_residual; returns the domain flag too
static int residual(Problem *P, double dt, int mode, const double *X1, const double *X0, double *F, double *part,
                    double *fn, bool *domain_ok)
{
    cudaMemsetAsync(P->dflag, 0, sizeof(int), P->stream);
    P->tick(0);
    P->count(launch_residual(P->g, P->k, dt, mode, X1, X0, P->tr0, P->mob, P->Gc, P->sig, part, F, P->dflag,
                             P->partials, P->stream));
    P->count(launch_finalize(P->partials, kRedBlocks, 1, P->dscal, P->stream));
    P->tock(0);
    cudaMemcpyAsync(P->hscal, P->dscal, sizeof(double), cudaMemcpyDeviceToHost, P->stream);
    cudaMemcpyAsync(P->hscal + 1, P->dflag, sizeof(int), cudaMemcpyDeviceToHost, P->stream);
    int rc = P->sync_check("residual");
    if (rc) return rc;
    int flag = 0;
    memcpy(&flag, P->hscal + 1, sizeof(int));
    *fn = sqrt(P->hscal[0]);
    *domain_ok = (flag & 1) == 0;
    return NKS_OK;
}

// level-n quantities used by every residual of the step
static void prepare_level(Problem *P, const double *X0)
{
    P->tick(8);
    P->count(launch_mobility(P->g, P->k, X0, P->mob, P->stream));
    if (P->k.elastic) P->count(launch_trace0(P->g, P->k, X0, P->tr0, P->stream));
    P->tock(8);
}

// One NKS solve (Sec. 4) for X^{n+1} from X = X^n on entry; P->Xn holds X^n.
// mode 1 solves the displacement-only system (initial equilibrium).
static int newton(Problem *P, double dt, int mode, double rtol, double atol, int maxit, nks_step_info *info)
{
    const long long n = P->nvec;
    P->cur_dt = dt;
    P->cur_mode = mode;
    P->factored = false;
    double fn0;
    bool ok;
    int rc = residual(P, dt, mode, P->X, P->Xn, P->F, P->part, &fn0, &ok);
    if (rc) return rc;
    info->fnorm0 = fn0;
    info->fnorm = fn0;
    info->newton_its = 0;
    info->gmres_its = 0;
    if (!ok) {
        P->err = "state outside the domain of the logarithms";
        return NKS_EDOMAIN;
    }
    if (!(fn0 == fn0) || isinf(fn0)) {
        P->err = "non-finite residual";
        return NKS_EDIVERGED;
    }
    const double tol = std::max(rtol * fn0, atol);
    if (fn0 <= tol) return NKS_OK;
    double fn = fn0;
    for (int it = 0; it < maxit; it++) {
        if (!P->factored || !P->opts.ilu_reuse) {
            rc = ras_factor(P, mode);
            if (rc) return rc;
        }
        P->tick(8);
        P->count(launch_axpby(n, -1.0, P->F, 0.0, P->B, P->stream));
        P->tock(8);
        int gits = 0;
        double gres = 0.0;
        rc = gmres_solve(P, mode, P->B, P->S, std::max(P->opts.gmres_rtol * fn, P->opts.gmres_atol), &gits, &gres);
        if (rc) return rc;
        info->gmres_its += gits;
        P->stats.gmres_its += gits;
        double lam = 1.0, ftn = 0.0;
        bool accepted = false;
        while (lam >= P->opts.ls_lambda_min) {
            P->tick(8);
            P->count(launch_waxpy(n, P->X, lam, P->S, P->Xt, P->stream));
            P->tock(8);
            bool dok;
            rc = residual(P, dt, mode, P->Xt, P->Xn, P->Ft, P->part_t, &ftn, &dok);
            if (rc) return rc;
            if (dok && ftn == ftn && !isinf(ftn) && ftn * ftn <= (1.0 - 2.0 * P->opts.ls_alpha * lam) * fn * fn) {
                accepted = true;
                break;
            }
            lam *= 0.5;
        }
        info->newton_its = it + 1;
        P->stats.newton_its++;
        if (!accepted) {
            P->err = "line search failed";
            return NKS_EDIVERGED;
        }
        std::swap(P->X, P->Xt);
        std::swap(P->F, P->Ft);
        std::swap(P->part, P->part_t);
        fn = ftn;
        info->fnorm = fn;
        if (fn <= tol) return NKS_OK;
    }
    P->err = "Newton iteration limit reached";
    return NKS_EDIVERGED;
}

static int energy_mass(Problem *P, const double *X, double *parts5, double *mass)
{
    P->tick(7);
    P->count(launch_energy(P->g, P->k, X, P->partials, P->stream));
    P->count(launch_finalize(P->partials, kRedBlocks, 5, P->dscal, P->stream));
    P->tock(7);
    cudaMemcpyAsync(P->hscal, P->dscal, 5 * sizeof(double), cudaMemcpyDeviceToHost, P->stream);
    int rc = P->sync_check("energy");
    if (rc) return rc;
    double v = 1.0;
    for (int J = 0; J < P->g.dim; J++) v *= P->g.h;
    const double *s = P->hscal;
    if (parts5) {
        for (int i = 0; i < 4; i++) parts5[i] = s[i] * v;
        parts5[4] = (s[0] + s[1] + s[2] + s[3]) * v;
    }
    if (mass) *mass = s[4] * v;
    return NKS_OK;
}

static int equilibrate(Problem *P)
{
    if (!P->k.elastic) return NKS_OK;
    cudaMemcpyAsync(P->X, P->Xn, sizeof(double) * P->nvec, cudaMemcpyDeviceToDevice, P->stream);
    prepare_level(P, P->Xn);
    nks_step_info info{};
    int rc = newton(P, 1.0, 1, P->opts.u0_rtol, P->opts.u0_atol, P->opts.u0_maxit, &info);
    if (rc) return rc;
    std::swap(P->Xn, P->X);
    return NKS_OK;
}

static bool host_in_domain(long long N, const double *c, const double *e)
{
    for (long long p = 0; p < N; p++) {
        const double pp = c[p] * e[p], q = c[p] * (4.0 - 3.0 * e[p]);
        if (!(c[p] > 0.0 && c[p] < 1.0 && pp > 0.0 && pp < 1.0 && q > 0.0 && q < 1.0)) return false;
    }
    return true;
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
}

int nks_create_problem(const nks_grid *grid, const double *c, const double *eta, const nks_coeffs *coeffs,
                       const nks_opts *opts, const nks_allocator *alloc, void *stream, nks_problem **out)
{
    *out = nullptr;
    g_create_error.clear();
    if (!grid || !c || !eta || !coeffs || !opts) {
        g_create_error = "null argument";
        return NKS_EINVAL;
    }
    if (grid->dim < 1 || grid->dim > 3 || !(grid->h > 0.0)) {
        g_create_error = "grid: dim must be 1..3 and h > 0";
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
    if (npts * (2 + grid->dim) >= (1LL << 31)) {
        // stencil kernels index the field planes with 32-bit offsets
        g_create_error = "grid: (2 + dim) * points must be below 2^31";
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
    nks_problem *H = new nks_problem();
    Problem *P = &H->P;
    cudaGetDevice(&P->device);
    P->grid = *grid;
    P->coeffs = *coeffs;
    P->opts = *opts;
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
    g.N = (long long)g.n[0] * g.n[1] * g.n[2];
    g.h = grid->h;
    P->N = g.N;
    if (!host_in_domain(g.N, c, eta)) {
        g_create_error = "initial state outside the domain: c, c*eta and c*(4-3*eta) must lie in (0, 1)";
        nks_destroy(H);
        return NKS_EDOMAIN;
    }
    double s = 0.0;
    for (long long p = 0; p < g.N; p++) s += c[p];
    P->cbar0 = s / (double)g.N;
    P->k = derive_coefficients(*coeffs, g.dim, P->cbar0);
    P->nf = P->k.nf;
    P->nvec = P->nf * g.N;
    P->ldv = (P->nvec + 1) & ~1LL;
    P->ldvf = (P->nvec + 3) & ~3LL;
    // every work vector holds ldv entries; the entry past nvec stays zero (16-byte pair loads)
    const size_t vb = sizeof(double) * (size_t)P->ldv, fb = sizeof(double) * (size_t)g.N;
    const int m = opts->gmres_restart;
    double **vecs[] = {&P->Xn, &P->Xprev, &P->X, &P->Xt, &P->F, &P->Ft, &P->S, &P->B, &P->W, &P->Z, &P->R};
    bool ok = true;
    for (double **v : vecs) ok = ok && ((*v = (double *)P->dalloc(vb)) != nullptr);
    ok = ok && (P->part = (double *)P->dalloc(4 * fb)) && (P->part_t = (double *)P->dalloc(4 * fb)) &&
         (P->mob = (double *)P->dalloc(3 * fb)) && (P->tr0 = (double *)P->dalloc(fb)) &&
         (P->Gc = (double *)P->dalloc(fb)) && (P->sig = (double *)P->dalloc(6 * fb)) &&
         (P->partials = (double *)P->dalloc(sizeof(double) * kRedBlocks * 64)) &&
         (P->dscal = (double *)P->dalloc(sizeof(double) * 64)) && (P->dflag = (int *)P->dalloc(sizeof(int) * 4)) &&
         (P->tickets = (unsigned int *)P->dalloc(sizeof(unsigned int) * 16)) &&
         (P->zsum = (double *)P->dalloc(sizeof(double) * 8)) && (P->Jec = (double *)P->dalloc(vb)) &&
         (P->ec = (double *)P->dalloc(vb)) &&
         (P->V = (double *)P->dalloc(vb * (opts->precision == NKS_MIXED ? 1 : m + 1))) &&
         (P->T64 = (double *)P->dalloc(vb)) &&
         (P->gm = (double *)P->dalloc(sizeof(double) * gmres_state_doubles(m)));
    if (ok && opts->precision == NKS_MIXED) {
        const size_t fvb = sizeof(float) * (size_t)P->ldvf;
        ok = (P->Vf = (float *)P->dalloc(fvb * (m + 1))) && (P->Wf = (float *)P->dalloc(fvb)) &&
             (P->Zf = (float *)P->dalloc(fvb)) &&
             (P->partf = (float *)P->dalloc(sizeof(float) * 4 * (size_t)g.N)) &&
             (P->mobf = (float *)P->dalloc(sizeof(float) * g.dim * (size_t)g.N)) &&
             (P->Jecf = (float *)P->dalloc(sizeof(float) * 2 * (size_t)g.N));
        if (ok) {
            cudaMemsetAsync(P->Vf, 0, fvb * (m + 1), P->stream);
            cudaMemsetAsync(P->Wf, 0, fvb, P->stream);
            cudaMemsetAsync(P->Zf, 0, fvb, P->stream);
        }
    }
    if (ok && cudaMallocHost((void **)&P->hscal, 64 * sizeof(double)) != cudaSuccess) ok = false;
    if (!ok) {
        g_create_error = "out of device memory";
        nks_destroy(H);
        return NKS_ENOMEM;
    }
    for (double **v : vecs) cudaMemsetAsync(*v, 0, vb, P->stream);
    cudaMemsetAsync(P->V, 0, vb * (opts->precision == NKS_MIXED ? 1 : m + 1), P->stream);
    cudaMemsetAsync(P->T64, 0, vb, P->stream);
    cudaMemcpyAsync(P->Xn, c, fb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(P->Xn + g.N, eta, fb, cudaMemcpyHostToDevice, P->stream);
    cudaMemsetAsync(P->tr0, 0, fb, P->stream);
    cudaMemsetAsync(P->tickets, 0, sizeof(unsigned int) * 16, P->stream);
    cudaMemsetAsync(P->zsum, 0, sizeof(double) * 8, P->stream);
    cudaMemsetAsync(P->Jec, 0, vb, P->stream);
    cudaMemsetAsync(P->ec, 0, vb, P->stream);
    {
        const std::vector<double> ones((size_t)g.N, 1.0);
        cudaMemcpyAsync(P->ec, ones.data(), fb, cudaMemcpyHostToDevice, P->stream);
        cudaStreamSynchronize(P->stream);
    }
    std::string err;
    int rc = ras_plan_create(P, err);
    if (rc) {
        g_create_error = err;
        nks_destroy(H);
        return rc;
    }
    rc = P->sync_check("create");
    if (!rc) rc = equilibrate(P);
    if (!rc) {
        cudaMemcpyAsync(P->Xprev, P->Xn, vb, cudaMemcpyDeviceToDevice, P->stream);
        double parts[5] = {0, 0, 0, 0, 0};
        rc = energy_mass(P, P->Xn, parts, nullptr);
        P->E = P->Eprev = parts[4];
    }
    if (rc) {
        g_create_error = P->err.empty() ? "initial equilibrium failed" : P->err;
        nks_destroy(H);
        return rc;
    }
    P->zeta = opts->zeta;
    P->dt_prev = opts->dt_init;
    harvest_timers(P);
    *out = H;
    return NKS_OK;
}

int nks_step(nks_problem *H, double dt_arg, nks_step_info *info_out)
{
    Problem *P = &H->P;
    P->err.clear();
    nks_step_info info{};
    const long long n = P->nvec;
    double dt;
    if (dt_arg > 0.0) {
        dt = dt_arg;
    } else if (P->nstep == 0 || P->opts.dt_mode == NKS_DT_FIXED) {
        dt = P->opts.dt_init;
    } else {
        double Xd;
        if (P->opts.dt_mode == NKS_DT_SOLUTION) {
            P->count(launch_waxpy(n, P->Xn, -1.0, P->Xprev, P->W, P->stream));
            P->count(launch_dot2(n, P->W, P->W, P->partials, P->stream));
            P->count(launch_finalize(P->partials, kRedBlocks, 2, P->dscal, P->stream));
            cudaMemcpyAsync(P->hscal, P->dscal + 1, sizeof(double), cudaMemcpyDeviceToHost, P->stream);
            int rc = P->sync_check("dt");
            if (rc) return rc;
            Xd = sqrt(P->hscal[0]) / P->dt_prev;
        } else {
            Xd = fabs(P->E - P->Eprev) / P->dt_prev;
        }
        // Eq. sencondt
        dt = std::max(P->opts.dt_min, P->opts.dt_max / sqrt(1.0 + P->zeta * Xd * Xd));
    }
    if (!P->opts.zeta_persist) P->zeta = P->opts.zeta;
    int rc = NKS_OK;
    int retries = 0;
    for (;;) {
        cudaMemcpyAsync(P->X, P->Xn, sizeof(double) * n, cudaMemcpyDeviceToDevice, P->stream);
        prepare_level(P, P->Xn);
        rc = newton(P, dt, 0, P->opts.newton_rtol, P->opts.newton_atol, P->opts.newton_maxit, &info);
        if (rc == NKS_OK) break;
        if (rc == NKS_ECUDA || dt_arg > 0.0 || retries >= P->opts.max_retries) break;
        // Sec. 4: a diverged NKS solve restarts with dt / sqrt(2) and zeta doubled
        dt /= sqrt(2.0);
        P->zeta *= 2.0;
        retries++;
        P->stats.retries++;
    }
    info.dt = dt;
    info.retries = retries;
    if (rc != NKS_OK) {
        info.status = rc;
        info.t = P->t;
        info.energy = P->E;
        if (info_out) *info_out = info;
        harvest_timers(P);
        return rc;
    }
    std::swap(P->Xprev, P->Xn);  // X^{n-1} <- X^n
    std::swap(P->Xn, P->X);      // X^n <- X^{n+1}
    double parts[5], mass;
    rc = energy_mass(P, P->Xn, parts, &mass);
    if (rc) return rc;
    P->Eprev = P->E;
    P->E = parts[4];
    P->t += dt;
    P->dt_prev = dt;
    P->nstep++;
    P->stats.steps++;
    info.t = P->t;
    info.energy = P->E;
    info.mass = mass;
    info.status = NKS_OK;
    if (info_out) *info_out = info;
    harvest_timers(P);
    return NKS_OK;
}

int nks_energy(const nks_problem *H, double *out)
{
    *out = H->P.E;
    return NKS_OK;
}

int nks_mass(const nks_problem *H, double *out)
{
    Problem *P = const_cast<Problem *>(&H->P);
    return energy_mass(P, P->Xn, nullptr, out);
}

int nks_get_fields(const nks_problem *H, double *c, double *eta, double *u)
{
    Problem *P = const_cast<Problem *>(&H->P);
    const size_t fb = sizeof(double) * (size_t)P->N;
    if (c) cudaMemcpyAsync(c, P->Xn, fb, cudaMemcpyDeviceToHost, P->stream);
    if (eta) cudaMemcpyAsync(eta, P->Xn + P->N, fb, cudaMemcpyDeviceToHost, P->stream);
    if (u && P->k.elastic) cudaMemcpyAsync(u, P->Xn + 2 * P->N, fb * P->g.dim, cudaMemcpyDeviceToHost, P->stream);
    return P->sync_check("get_fields");
}

struct StateHeader {
    char magic[8];
    long long nvec, nstep;
    double t, dt_prev, zeta, E, Eprev;
};

size_t nks_state_size(const nks_problem *H) { return sizeof(StateHeader) + 2 * sizeof(double) * (size_t)H->P.nvec; }

int nks_get_state(const nks_problem *H, void *buf, size_t bytes)
{
    Problem *P = const_cast<Problem *>(&H->P);
    if (bytes < nks_state_size(H)) {
        P->err = "state buffer too small";
        return NKS_EINVAL;
    }
    StateHeader hd;
    memcpy(hd.magic, "NKSSTAT1", 8);
    hd.nvec = P->nvec;
    hd.nstep = P->nstep;
    hd.t = P->t;
    hd.dt_prev = P->dt_prev;
    hd.zeta = P->zeta;
    hd.E = P->E;
    hd.Eprev = P->Eprev;
    memcpy(buf, &hd, sizeof(hd));
    char *b = (char *)buf + sizeof(hd);
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    cudaMemcpyAsync(b, P->Xn, vb, cudaMemcpyDeviceToHost, P->stream);
    cudaMemcpyAsync(b + vb, P->Xprev, vb, cudaMemcpyDeviceToHost, P->stream);
    return P->sync_check("get_state");
}

int nks_set_state(nks_problem *H, const void *buf, size_t bytes)
{
    Problem *P = &H->P;
    StateHeader hd;
    if (bytes < sizeof(hd)) {
        P->err = "state buffer too small";
        return NKS_EINVAL;
    }
    memcpy(&hd, buf, sizeof(hd));
    if (memcmp(hd.magic, "NKSSTAT1", 8) != 0 || hd.nvec != P->nvec || bytes < nks_state_size(H)) {
        P->err = "state buffer does not match this problem";
        return NKS_EINVAL;
    }
    const char *b = (const char *)buf + sizeof(hd);
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    cudaMemcpyAsync(P->Xn, b, vb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(P->Xprev, b + vb, vb, cudaMemcpyHostToDevice, P->stream);
    P->nstep = hd.nstep;
    P->t = hd.t;
    P->dt_prev = hd.dt_prev;
    P->zeta = hd.zeta;
    P->E = hd.E;
    P->Eprev = hd.Eprev;
    return P->sync_check("set_state");
}

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
    ras_plan_destroy(P);
    P->dfree_all();
    if (P->hscal) cudaFreeHost(P->hscal);
    if (P->own_stream && P->stream) cudaStreamDestroy(P->stream);
    delete H;
}

const char *nks_last_error(const nks_problem *H)
{
    if (!H) return g_create_error.c_str();
    return H->P.err.c_str();
}

// ---------------------------------------------------------------------------
// operator-level entry points
// ---------------------------------------------------------------------------

static int op_setup(Problem *P, const double *X1, const double *X0, double dt, int mode)
{
    const size_t vb = sizeof(double) * (size_t)P->nvec;
    cudaMemcpyAsync(P->X, X1, vb, cudaMemcpyHostToDevice, P->stream);
    cudaMemcpyAsync(P->Xt, X0, vb, cudaMemcpyHostToDevice, P->stream);
    P->cur_dt = dt;
    P->cur_mode = mode;
    P->tick(8);
    P->count(launch_mobility(P->g, P->k, P->Xt, P->mob, P->stream));
    if (P->k.elastic) P->count(launch_trace0(P->g, P->k, P->Xt, P->tr0, P->stream));
    P->tock(8);
    double fn;
    bool ok;
    return residual(P, dt, mode, P->X, P->Xt, P->F, P->part, &fn, &ok);
}

static int op_finish(Problem *P, int rc)
{
    // the operator calls reuse the step's work buffers: level-n data must be rebuilt
    prepare_level(P, P->Xn);
    P->factored = false;
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
        cudaMemcpyAsync(P->B, v, vb, cudaMemcpyHostToDevice, P->stream);
        P->tick(1);
        if (P->opts.precision == NKS_MIXED) {
            // as the Arnoldi step applies it: FP32 vectors, coefficients and arithmetic
            refresh_f32_coefficients(P);
            P->count(launch_convert(P->nvec, P->B, P->Zf, P->stream));
            P->count(launch_jv32(P->g, P->k, dt, mode, P->partf, P->mobf, P->Zf, P->Wf, P->stream, nullptr, nullptr));
            P->count(launch_convert(P->nvec, P->Wf, P->W, P->stream));
        } else {
            P->count(launch_jv(P->g, P->k, dt, mode, P->part, P->mob, P->B, P->Gc, P->sig, P->W, P->stream));
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
    if (!rc) rc = ras_factor(P, 0);
    if (!rc) {
        const size_t vb = sizeof(double) * (size_t)P->nvec;
        cudaMemcpyAsync(P->B, r, vb, cudaMemcpyHostToDevice, P->stream);
        if (P->opts.precision == NKS_MIXED) {
            // as the solver applies it: FP32 vectors and factors
            P->count(launch_convert(P->nvec, P->B, P->Wf, P->stream));
            ras_apply_projected<float>(P, P->Wf, P->Zf);
            P->count(launch_convert(P->nvec, P->Zf, P->Z, P->stream));
        } else {
            ras_apply(P, P->B, P->Z);
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
    if (!rc) rc = ras_factor(P, mode);
    if (!rc) {
        const size_t vb = sizeof(double) * (size_t)P->nvec;
        cudaMemcpyAsync(P->B, b, vb, cudaMemcpyHostToDevice, P->stream);
        rc = gmres_solve(P, mode, P->B, P->S, tol, its, res);
        if (!rc) {
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
    int rc = energy_mass(P, P->W, parts, mass);
    harvest_timers(P);
    return rc;
}

}  // extern "C"
