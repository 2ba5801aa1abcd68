/*
 * nks.h -- C ABI of the GB300 Newton-Krylov-Schwarz solver for the
 * semi-implicit discrete-variational-derivative (DVD) scheme NSOA-1 of
 * Huang & Yang, "Parallel energy stable phase field simulations of Ni-based
 * alloys system" (arXiv 2209.08001).
 *
 * The solver advances the coupled Cahn-Hilliard / Allen-Cahn (Ginzburg-Landau)
 * system for the Al composition c, the long-range order (one parameter eta, the
 * reduced model of Sec. 2-5, or the three eta_1..eta_3 of App. A) and the
 * elastic displacement u on a cell-centred, uniform grid, periodic or with
 * homogeneous Neumann boundaries (Sec. 2-3).
 * Every time step solves the nonlinear system F(X) = 0 of Eq. NSOA-1 by an
 * inexact Newton method with line search (Sec. 4), whose Jacobian systems are
 * solved by restarted GMRES preconditioned with restricted additive Schwarz
 * and ILU(0) subdomain solves (Sec. 4, Sec. 5.4).  The step size is adaptive
 * (Sec. 4, Eq. sencondt) with divergence retries.
 *
 * Conventions for every entry point:
 *   - Grids are x-fastest: point p = x + nx*(y + ny*z).  A "field" array holds
 *     N = nx*ny*nz doubles in that order.
 *   - A "state" array (X) holds the fields one after another (SoA): c, then
 *     the n_eta order parameters (nks_coeffs.n_eta: 1 or 3) and, when
 *     elasticity is on (any of C11, C12, C44 non-zero), u_1..u_d.  Its length
 *     is nf*N with nf = 1 + n_eta + d (elastic) or 1 + n_eta.  An "eta" array
 *     holds the n_eta order-parameter fields one after another (n_eta*N).
 *   - Pointers marked HOST are read or written with synchronous copies before
 *     the call returns; the caller keeps ownership.  Pointers marked DEVICE
 *     must be device memory on the problem's device.
 *   - Every int-returning function returns NKS_OK (0) or a negative-free
 *     error code below; nks_last_error() then describes the failure.
 *   - A problem is bound to the CUDA device and stream given at creation and
 *     is not thread safe; distinct problems may be used from distinct threads.
 */
#ifndef NKS_H
#define NKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define NKS_OK 0
#define NKS_EINVAL 1     /* invalid argument or unsupported configuration        */
#define NKS_EDOMAIN 2    /* c, c*eta or c*(4-3*eta) outside (0, 1); with three order
                            parameters c, c*eta_i (i = 1..4, eta_4 = 4 - sum) */
#define NKS_ENOMEM 3     /* device allocation failed                              */
#define NKS_EDIVERGED 4  /* Newton failed and the retry budget is spent (Sec. 4)  */
#define NKS_ETIMEOUT 5   /* an iteration cap was reached                          */
#define NKS_ECUDA 6      /* CUDA runtime error                                    */
#define NKS_EPIVOT 7     /* zero pivot in an ILU(0) subdomain factorisation       */

/* Schwarz preconditioner types (nks_opts.ras_variant, Sec. 4) */
#define NKS_LEFT_RAS 0
#define NKS_AS 1
#define NKS_RIGHT_RAS 2

/* precision modes */
#define NKS_FP64 0       /* everything in FP64                                     */
#define NKS_MIXED 1      /* FP32 Schwarz factors/sub-solves and Krylov basis;
                            FP64 residual, update, log terms, energy and mass      */

/* step-size drivers (Sec. 4, Eq. sencondt) */
#define NKS_DT_FIXED 0
#define NKS_DT_SOLUTION 1 /* X'_d = ||X^n - X^{n-1}||_2 / dt_{n-1}                */
#define NKS_DT_ENERGY 2   /* X'_d = |E^n - E^{n-1}| / dt_{n-1}                    */

/* boundary conditions (nks_grid.bc) */
#define NKS_PERIODIC 0
#define NKS_NEUMANN 1    /* homogeneous Neumann (Sec. 2, Eq. boundaryequ)              */

/*
 * Cell-centred grid x_i = (i - 1/2) h on each axis (Sec. 3).
 *   bc  NKS_PERIODIC: periodic in every axis.
 *       NKS_NEUMANN: homogeneous Neumann boundaries, n.grad c = n.grad eta =
 *       n.M grad mu = 0 and n.sigma = 0 (Eq. boundaryequ).  The ghost cell beyond
 *       a boundary cell mirrors it, so D^+ / D^- across a boundary face vanish and
 *       the flux form has no boundary flux (Sec. 3's summation by parts holds as
 *       stated); the displacement rows are the exact variation -dE_3/du of the
 *       discrete elastic energy (strains by the centred difference with mirrored
 *       ghosts), whose natural boundary condition is the traction-free one; the
 *       Schwarz boxes stop at the boundary; the null modes of the strain, which
 *       the Newton corrections are kept free of, are the d translations and, for
 *       each pair of axes that both have an even number of cells, a discrete
 *       rotation (u_I = -S(x_J), u_J = S(x_I), S(x) = floor((x+1)/2) - n/4).
 */
typedef struct {
    int dim;     /* 1, 2 or 3                                        */
    int n[3];    /* cells per axis; entries >= dim are ignored        */
    double h;    /* mesh size (the same on every axis)                */
    int bc;      /* NKS_PERIODIC or NKS_NEUMANN                       */
} nks_grid;

/*
 * Dimensionless coefficients (App. A scaling by V_m*dE and the length 1.5 nm).
 *   kappa       mobility parameter, M = kappa c (1 - c)            (Eq. CHGL)
 *   gamma_c     gradient coefficient of c                          (Eq. simple free energy-1)
 *   gamma_eta   gradient coefficient of eta; enters as 3*gamma_eta
 *   theta       R T / (V_m dE), weight of the entropy terms        (Eq. neq:01)
 *   w_psi       weight of theta*Psi(c) inside E_2 (1 in Sec. 2-3; App. A cancels it)
 *   dE0         (E0_Al - E0_Ni)/(V_m dE)                           (App. A)
 *   L[4], U1, U4  excess and ordering parameters / (V_m dE)        (App. A)
 *   eps0        composition expansion coefficient of the lattice   (App. A)
 *   C11, C12, C44  cubic Hooke constants / dE; multiplied by Lscale (Sec. 5.1).
 *               All three zero switches elasticity (and the u fields) off.
 *   S           Taylor order of Psi_S (Sec. 3, S = 10 in Sec. 5); must be >= 1
 *   n_eta       order parameters: 1 (0 reads as 1) for the reduced model of the
 *               main text, 3 for the model of App. A (E_1 = dis(c) + a(c) S(eta)
 *               + b(c) T(eta), E_2 over the four sublattices, gamma_eta/2 per
 *               |grad eta_j|^2, Allen-Cahn rows with the kinetic factor 3, so
 *               that eta_1 = eta_2 = eta_3 = eta is the reduced model)
 */
typedef struct {
    double kappa, gamma_c, gamma_eta, theta, w_psi, dE0;
    double L[4];
    double U1, U4, eps0;
    double C11, C12, C44, Lscale;
    int S;
    int n_eta;
} nks_coeffs;

/*
 * Solver options (Sec. 4; Sec. 5.4 for the Schwarz settings).
 *   newton_rtol/atol   eps_r, eps_a: stop when ||F|| <= max(eps_r ||F(X_0)||, eps_a)
 *   newton_maxit       Newton iterations before the step counts as diverged
 *   ls_alpha, ls_lambda_min  backtracking: halve lambda while
 *                      ||F(X + lambda S)||^2 > (1 - 2 alpha lambda) ||F||^2 or the
 *                      trial leaves the domain; fail below lambda_min
 *   gmres_restart, gmres_maxit  GMRES(m) and the total iteration cap per solve
 *   gmres_rtol/atol    xi_r, xi_a: ||J S + F|| <= max(xi_r ||F||, xi_a)
 *   sub[3], overlap    box decomposition (subdomains per axis) and delta (layers
 *                      per side); each overlapped box must be at least 2 cells
 *                      shorter than the grid along every axis
 *   ilu_reuse          1: factor once per time step (ILU(0)-reuse, Table 1)
 *   precision          NKS_FP64 or NKS_MIXED
 *   dt_init            dt of the first step (Sec. 5.1: 0.01)
 *   dt_min, dt_max, zeta  predictor parameters (Eq. sencondt)
 *   dt_mode            NKS_DT_FIXED / NKS_DT_SOLUTION / NKS_DT_ENERGY
 *   zeta_persist       0: a doubled zeta is used for the next prediction only
 *   max_retries        divergence retries (dt /= sqrt 2, zeta *= 2) per step
 *   u0_rtol/atol/maxit initial mechanical equilibrium solve
 *   timing             1: record per-kernel CUDA-event times (nks_get_stats)
 *   ras_variant        Schwarz type (Sec. 4, Table 2): NKS_LEFT_RAS (default,
 *                      sum_i R_i^0T A_i^-1 R_i^delta), NKS_AS (classical,
 *                      sum_i R_i^deltaT A_i^-1 R_i^delta), NKS_RIGHT_RAS
 *                      (sum_i R_i^deltaT A_i^-1 R_i^0); overlaps of the last two
 *                      are summed in box order; all coincide for overlap 0
 *   graphs             1: each GMRES iteration replays a CUDA graph captured on
 *                      its first use (kernels of all batch slots and the read-back
 *                      of the iteration's scalars); ignored when timing = 1
 *   u0_mixed           1: the displacement-only solves (the initial mechanical
 *                      equilibrium, mode 1) run their GMRES in the NKS_MIXED form
 *                      (FP32 factors, sweeps, basis) even when precision is
 *                      NKS_FP64; their Newton residual, update and tolerance stay
 *                      FP64, so the equilibrium meets the same u0_rtol/atol.  The
 *                      time steps keep `precision`.  0 (default): `precision`.
 *                      Costs the FP32 buffers of the mixed mode in FP64 mode.
 */
typedef struct {
    double newton_rtol, newton_atol;
    int newton_maxit;
    double ls_alpha, ls_lambda_min;
    int gmres_restart, gmres_maxit;
    double gmres_rtol, gmres_atol;
    int sub[3];
    int overlap;
    int ilu_reuse;
    int precision;
    double dt_init, dt_min, dt_max, zeta;
    int dt_mode;
    int zeta_persist;
    int max_retries;
    double u0_rtol, u0_atol;
    int u0_maxit;
    int timing;
    int graphs;
    int ras_variant;
    int u0_mixed;
} nks_opts;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns device memory of at least `bytes` bytes (NULL on failure);
 * free releases it.  Both are called on the creating thread. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} nks_allocator;

typedef struct nks_problem nks_problem; /* opaque, owned by the library */

/* Outcome of one accepted (or failed) time step. */
typedef struct {
    double dt;         /* accepted step size                                   */
    double t;          /* time after the step                                  */
    double energy;     /* discrete energy E^{n+1} (Eq. freeenergy)             */
    double mass;       /* <c^{n+1}> = h^d sum c                                */
    double fnorm0;     /* ||F(X_0)|| of the accepted attempt                   */
    double fnorm;      /* final ||F||                                          */
    int retries;       /* divergence retries taken                             */
    int newton_its;    /* Newton iterations of the accepted attempt            */
    int gmres_its;     /* GMRES iterations of the accepted attempt             */
    int status;        /* NKS_OK or the failure code                           */
} nks_step_info;

/* Per-kernel-class counters (launches and, with opts.timing, device time). */
#define NKS_NCLASS 11
typedef struct {
    long long launches[NKS_NCLASS];
    double ms[NKS_NCLASS];          /* summed CUDA-event durations (timing = 1) */
    long long newton_its, gmres_its, steps, retries;
    long long factor_bytes;         /* bytes of stored Schwarz factors          */
    double schwarz_points;          /* overlapped points of all subdomains      */
    double schwarz_bytes;           /* algorithmic bytes of one Schwarz sweep:
                                       factors of every overlapped point, the
                                       gathered sub-vectors and the owned output */
    double schwarz_flops;           /* algorithmic FLOPs of one Schwarz sweep   */
    long long kernel_launches;      /* CUDA kernels this problem launched       */
    long long reorth;               /* Gram-Schmidt second passes taken         */
    double cgs_bytes;               /* algorithmic bytes of the Gram-Schmidt
                                       passes: (2j + 5) basis-vector reads and
                                       writes for Arnoldi step j, per pass      */
} nks_stats;
/* kernel classes: 0 residual, 1 Jacobian action of the Arnoldi steps (FP32 in
 * mixed precision), 2 Schwarz apply, 3 assembly + ILU(0), 4 Gram-Schmidt dots,
 * 5 Gram-Schmidt update, 6 projection, 7 energy/mass, 8 vector ops, 9 small
 * dense (Hessenberg), 10 FP64 Jacobian action of the true residual b - J x at
 * the end of each GMRES cycle */

/* Fill *o with the default solver settings (Sec. 4-5): eps_r = 1e-10,
 * GMRES(30), 4x4 subdomains with overlap 1, ILU(0)-reuse, dt_1 = dt_min =
 * 0.01, dt_max = 2, zeta = 100, fixed dt. */
void nks_default_opts(nks_opts *o);

/*
 * Create a problem from the initial fields and solve the initial mechanical
 * equilibrium for u (reading: the energy law of Theorem 3.1 assumes u in
 * equilibrium at level n).  The mean composition cbar0 of Sec. 3 is taken from c.
 *   c, eta   HOST, N and n_eta*N doubles (x-fastest)
 *   alloc    NULL: cudaMalloc / cudaFree
 *   stream   a cudaStream_t, or NULL for a stream the library creates and owns
 * Fails with NKS_EDOMAIN when an initial value leaves the domain of the
 * logarithms, NKS_EINVAL for an unsupported grid or decomposition.
 */
int nks_create_problem(const nks_grid *grid, const double *c, const double *eta, const nks_coeffs *coeffs,
                       const nks_opts *opts, const nks_allocator *alloc, void *stream, nks_problem **out);

/*
 * Advance one time step of NSOA-1.  dt > 0: that step size (no retries);
 * dt <= 0: step size from opts (dt_init for the first step, then the
 * predictor of Eq. sencondt) with divergence retries.  On failure the state
 * stays at X^n and info->status holds the code.  info may be NULL.
 */
int nks_step(nks_problem *p, double dt, nks_step_info *info);

/* Discrete energy E^n of Eq. freeenergy (Sec. 3). */
int nks_energy(const nks_problem *p, double *out);

/* Mass <c^n> = h^d sum_i c_i (Theorem 3.1). */
int nks_mass(const nks_problem *p, double *out);

/* Copy the current fields to HOST arrays (c: N doubles, eta: n_eta*N; u: d*N
 * doubles, component-major, or NULL; ignored without elasticity). */
int nks_get_fields(const nks_problem *p, double *c, double *eta, double *u);

/* Checkpoint: bytes needed, then save / restore X^n, X^{n-1}, t, step count,
 * dt_{n-1}, zeta, the two last energies and cbar0 (HOST buffer). Restoring
 * gives a bitwise-identical continuation. */
size_t nks_state_size(const nks_problem *p);
int nks_get_state(const nks_problem *p, void *buf, size_t bytes);
int nks_set_state(nks_problem *p, const void *buf, size_t bytes);

/* Counters since creation or the last reset. */
int nks_get_stats(const nks_problem *p, nks_stats *out);
int nks_reset_stats(nks_problem *p);

void nks_destroy(nks_problem *p);

/* Message of the last failure on this problem ("" if none); p may be NULL for
 * failures of nks_create_problem / nks_create_batch on the calling thread. */
const char *nks_last_error(const nks_problem *p);

/* ------------------------------------------------------------------------ */
/* Batches: nb independent problems of the same grid, coefficients and       */
/* options in one object (no counterpart in the paper, which solves one      */
/* problem at a time).  Each phase of the solver (residual, Jacobian action, */
/* Schwarz factorisation and sweeps, Gram-Schmidt passes, small GMRES        */
/* kernels) is ONE kernel launch over all instances; every instance keeps    */
/* its own Newton / GMRES iteration, step size and retries, and an instance  */
/* that has converged is masked out of the remaining launches, so each      */
/* instance's result is bitwise the result of solving it alone.  The        */
/* problem API above acts on slot 0 (a problem is a batch of one).  Device  */
/* memory: one allocation of nks_device_bytes() for all slots.              */
/* ------------------------------------------------------------------------ */

/* Create a batch of nb slots (1 <= nb <= 65535; in 3-D n_z * nb <= 65535).
 *   c, eta   HOST, nb * N and nb * n_eta * N doubles (slot-major), or both NULL: every slot
 *            starts empty (fill slots with nks_batch_load).
 * Each loaded slot takes its own mean composition cbar0 and initial
 * mechanical equilibrium, as nks_create_problem does.  Errors as there. */
int nks_create_batch(const nks_grid *grid, int nb, const double *c, const double *eta, const nks_coeffs *coeffs,
                     const nks_opts *opts, const nks_allocator *alloc, void *stream, nks_problem **out);

/* Number of slots. */
int nks_batch_size(const nks_problem *p);

/* Load initial fields (HOST, N and n_eta*N doubles) into a slot: resets its time,
 * step count and step-size state, solves its initial equilibrium.  Other
 * slots are untouched.  NKS_EINVAL for a bad slot, NKS_EDOMAIN as above. */
int nks_batch_load(nks_problem *p, int slot, const double *c, const double *eta);

/* Mark a slot empty (its buffers stay allocated for the next load). */
int nks_batch_unload(nks_problem *p, int slot);

/* 1 when the slot holds a problem, else 0. */
int nks_batch_loaded(const nks_problem *p, int slot);

/* One time step of every loaded slot with active[slot] != 0 (active NULL: all
 * loaded slots).  dt: nb step sizes (> 0 fixed, <= 0 adaptive as in nks_step)
 * or NULL (all adaptive).  infos: nb entries (written for the stepped slots).
 * Returns NKS_OK unless a CUDA error stops the batch; per-slot failures are
 * in infos[slot].status (the slot then stays at its X^n). */
int nks_batch_step(nks_problem *p, const int *active, const double *dt, nks_step_info *infos);

/* Per-slot versions of nks_energy, nks_mass, nks_get_fields, nks_get_state
 * and nks_set_state (set_state also marks the slot loaded). */
int nks_batch_energy(const nks_problem *p, int slot, double *out);
int nks_batch_mass(const nks_problem *p, int slot, double *out);
int nks_batch_get_fields(const nks_problem *p, int slot, double *c, double *eta, double *u);
int nks_batch_get_state(const nks_problem *p, int slot, void *buf, size_t bytes);
int nks_batch_set_state(nks_problem *p, int slot, const void *buf, size_t bytes);

/* Device bytes of the per-slot buffers of all slots (state, Krylov basis,
 * Schwarz factors, scratch). */
size_t nks_device_bytes(const nks_problem *p);

/* Pointwise DVD derivative of the model with three order parameters (App. A:
 * eta_1..eta_3, eta_4 = 4 - sum), the part of the residual the kernels of that
 * model evaluate per point.  Host computation, no device needed.
 *   x1, x0  HOST, 4 doubles each: (c, eta_1, eta_2, eta_3) at levels n+1 and n;
 *           c and the four site fractions c eta_i must lie in (0, 1)
 *   G       HOST, 4 doubles out: G^1 + G^{2,S} = (G_c, G_eta_1, G_eta_2, G_eta_3),
 *           the product terms split symmetrically with exact polynomial quotients
 *           and average-vector-field gradients, the logarithms by Psi_S (Sec. 3)
 *   dG      HOST, 16 doubles out: dG[a * 4 + b] = dG_a / dx1_b
 * coeffs as for nks_create_problem (the Hooke constants are not used).
 * Returns NKS_EINVAL for a null pointer or S outside 1..16. */
int nks_model3_point(const nks_coeffs *coeffs, const double *x1, const double *x0, double *G, double *dG);

/* Testing hook for failure detection (no counterpart in the paper): on != 0
 * makes every Schwarz sweep withhold the first bulk copy of factors in each
 * block, so the block's bounded mbarrier wait expires (about a second), the
 * block writes nothing and flags the failure, and the running solve returns
 * NKS_ETIMEOUT with the state left at X^n; the GPU context stays usable.
 * on = 0 restores normal sweeps. */
int nks_debug_withhold_copy(nks_problem *p, int on);

/* ------------------------------------------------------------------------ */
/* Serving: a request loop for many simulations on one GPU (no counterpart   */
/* in the paper).  Requests of the same grid shape share one batch (above)   */
/* with a fixed number of slots, a CUDA stream and a worker thread; between  */
/* two batch steps the worker loads newly admitted requests into free slots, */
/* steps every occupied slot, and retires finished requests (continuous      */
/* batching).  Shape groups run concurrently, so their kernels overlap on    */
/* the device.  Admission is by device memory: a group reserves slots x the  */
/* measured bytes of one slot out of mem_budget and returns them when it     */
/* empties.  Each result is bitwise the result of the request run alone.     */
/* Thread-safe: submit and wait may be called from any host threads.         */
/* ------------------------------------------------------------------------ */

typedef struct nks_server nks_server;

typedef struct {
    nks_opts opts;         /* solver options of every request (sub is set per shape) */
    size_t mem_budget;     /* device bytes for all batches; 0: 80% of the free memory */
    int max_slots;         /* slots per shape group */
    int max_groups;        /* shape groups alive at once (worker threads / streams) */
    int box_side_2d;       /* owned Schwarz box side for 2-D (and 4x for 1-D) grids */
    int box_side_3d;       /* owned Schwarz box side for 3-D grids */
} nks_server_opts;

typedef struct {
    long long id;
    int status;            /* NKS_OK or the failure code of the request */
    int steps;             /* steps completed */
    int newton_its, gmres_its, retries;   /* summed over the steps */
    long long points;      /* grid points */
    double t_submit, t_admit, t_done;     /* seconds since nks_server_create */
    double t, energy, mass;               /* after the last step */
} nks_request_result;

typedef struct {
    int waiting;           /* submitted, not yet in a group */
    int groups;            /* live shape groups */
    int in_flight;         /* requests in groups (loaded or queued) */
    size_t bytes_reserved, mem_budget;
} nks_server_state;

/* mixed precision, energy-driven dt, 16 slots, 8 groups, boxes 32 (2-D) / 16 (3-D) */
void nks_server_default_opts(nks_server_opts *o);
int nks_server_create(const nks_coeffs *coeffs, const nks_server_opts *opts, nks_server **out);

/* Queue a request: grid, initial fields (HOST, N and n_eta*N doubles; copied),
 * number of time steps (adaptive dt).  Never blocks on the GPU work. */
int nks_server_submit(nks_server *s, const nks_grid *grid, const double *c, const double *eta, int steps,
                      long long *id);

/* Wait for a request (timeout_s < 0: no limit; NKS_ETIMEOUT on expiry), copy its
 * result and final fields (c: N, eta: n_eta N, u: d N doubles; any may be NULL)
 * and release it. */
int nks_server_wait(nks_server *s, long long id, nks_request_result *res, double *c, double *eta, double *u,
                    double timeout_s);

int nks_server_status(nks_server *s, nks_server_state *st);

/* Finish every submitted request, stop the workers, free everything. */
void nks_server_destroy(nks_server *s);

/* Autotuner of the Schwarz decomposition (no counterpart in the paper, which
 * fixes it per experiment): for each candidate (owned-box counts per axis and
 * overlap delta) a problem is created from c, eta (HOST, N doubles each) and
 * base, one step of dt_trial is taken (it captures the iteration graphs), and
 * the wall time of a second step is measured; best receives base with the
 * fastest candidate's sub and overlap.
 *   cands   ncand x 4 ints (sub_x, sub_y, sub_z, overlap), or NULL for the
 *           built-in list: square / cubic owned boxes of side 16..128 (2-D) or
 *           8..32 (3-D) that give at least two boxes per axis, overlap 1 and 2
 *   times   seconds of each candidate's timed step (-1: rejected or failed),
 *           as many entries as candidates (the built-in list has at most 12);
 *           may be NULL
 *   chosen  index of the chosen candidate, may be NULL
 * Returns NKS_OK, NKS_EINVAL, or NKS_EDIVERGED when every candidate failed. */
int nks_autotune(const nks_grid *grid, const double *c, const double *eta, const nks_coeffs *coeffs,
                 const nks_opts *base, const int *cands, int ncand, double dt_trial, nks_opts *best, double *times,
                 int *chosen);

/* ------------------------------------------------------------------------ */
/* Operator-level entry points (the stages of one Newton iteration).         */
/* They use the problem's grid, coefficients and decomposition and leave its */
/* state untouched.  All arrays are HOST state arrays of length nf*N.        */
/* ------------------------------------------------------------------------ */

/* F(X1; X0, dt) of Eq. NSOA-1 (mode 0), or the displacement-only residual
 * (mode 1: F_c = F_eta = 0) used for the initial equilibrium; without
 * elasticity mode 1 gives F = 0. */
int nks_eval_residual(nks_problem *p, const double *X1, const double *X0, double dt, int mode, double *F);

/* Jv = J(X1; X0, dt) v with J = dF/dX1 (Sec. 4, J_m = grad F(X_m)).  In the
 * NKS_MIXED mode the action runs as the solver's Arnoldi step runs it: v
 * rounded to FP32, FP32 copies of the pointwise coefficients, FP32 arithmetic;
 * the result is widened to FP64 (the FP64 form is used for true residuals). */
int nks_apply_jacobian(nks_problem *p, const double *X1, const double *X0, double dt, int mode, const double *v,
                       double *Jv);

/* z = P sum_i R_i^0T (L_i U_i)^-1 R_i^delta r: restricted additive Schwarz
 * (Sec. 4, left-RAS) with ILU(0) factors of J(X1; X0, dt) restricted to each
 * overlapped box, followed by the projection P (mean of z_c removed; the
 * null modes of the centred-difference strain removed from z_u).  In the
 * NKS_MIXED mode the sweeps run as the solver runs them: FP32 factors and
 * vectors (r rounded to FP32 on input). */
int nks_apply_preconditioner(nks_problem *p, const double *X1, const double *X0, double dt, const double *r,
                             double *z);

/* Solve J(X1; X0, dt) x = b from x = 0 by right-preconditioned GMRES(m)
 * (Sec. 4) to ||b - J x|| <= tol; its/res receive the iteration count and the
 * final true residual norm. */
int nks_linear_solve(nks_problem *p, const double *X1, const double *X0, double dt, int mode, const double *b,
                     double *x, double tol, int *its, double *res);

/* Energy parts of X (Eq. relations: E1, E2, E3, E4 summed times h^d), their
 * total, and the mass; parts has 5 entries. */
int nks_eval_energy(nks_problem *p, const double *X, double *parts, double *mass);

/* ------------------------------------------------------------------------ */
/* Residual evaluation that allocates no device memory.                      */
/* ------------------------------------------------------------------------ */

/* Largest grid (points) nks_residual_noalloc accepts. */
#define NKS_NOALLOC_MAX_POINTS 65536

/*
 * F(X1; X0, dt) as nks_eval_residual computes it, but on DEVICE arrays and
 * without allocating: no cudaMalloc, cudaFree or allocating library call is
 * made.  The paper has no counterpart; this entry point serves callers that
 * cannot allocate device memory when they evaluate the residual, for example
 * a host application whose memory manager owns the whole device, or a
 * latency-critical loop that must not allocate because allocation can
 * synchronise the device.
 *
 *   grid, coeffs   as for nks_create_problem; grid->n[0]*n[1]*n[2] must not
 *                  exceed NKS_NOALLOC_MAX_POINTS (NKS_EINVAL otherwise); every
 *                  axis needs at least 3 cells
 *   cbar0          mean composition of the initial state (Sec. 3)
 *   dt, mode       as for nks_eval_residual (mode 1: displacement-only system;
 *                  without elasticity that system is empty and F = 0)
 *   X1, X0, F      DEVICE state arrays of nf*N doubles (layout of this header)
 *   fnorm2         DEVICE pointer receiving ||F||^2, or NULL
 *   stream         cudaStream_t to run on (NULL: the legacy default stream)
 * Serves the model with one order parameter (coeffs->n_eta 0 or 1; NKS_EINVAL
 * for 3).
 * Returns NKS_OK, NKS_EINVAL, NKS_EDOMAIN (X1 outside the domain of the
 * logarithms; F is still written) or NKS_ECUDA; nks_last_error(NULL) gives
 * the message.  The call synchronises the stream before it returns.  A CUDA
 * error already pending from the caller's earlier work makes the call return
 * NKS_ECUDA at once, leaving that error pending for its owner.
 *
 * Scratch: a fixed array of 15 * NKS_NOALLOC_MAX_POINTS doubles (7.5 MiB) plus
 * reduction space, held in device memory by every GPU that loads the library
 * until the process exits.  The first call on a device looks up the array's
 * device address (once per device, with that device current); make that first
 * call before any stream capture.  The address belongs to the device's primary
 * context: after cudaDeviceReset, or from another context on the same device,
 * it is no longer valid, so do not call this function there.  All calls share
 * the array and it keeps the previous call's contents, so calls that overlap
 * on the GPU (from several threads or streams) race: serialise them.
 */
int nks_residual_noalloc(const nks_grid *grid, const nks_coeffs *coeffs, double cbar0, double dt, int mode,
                         const double *X1, const double *X0, double *F, double *fnorm2, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NKS_H */
