// nks_noalloc.cu -- residual evaluation that allocates no device memory.
//
// nks_residual_noalloc() evaluates F(X1; X0, dt) of the scheme on caller-owned
// device arrays without ever calling cudaMalloc / cudaFree or an allocating
// library routine.  It exists for callers that cannot allocate device memory
// at the point of the call: a host application whose memory manager owns the
// whole device and hands out fixed pools, or a latency-critical loop that must
// not allocate because an allocation can synchronise the device and stall
// other work.  Its intermediate grid functions (edge mobilities, level-n strain
// trace, G_c, the stress, the pointwise derivatives) and the reduction
// partials live in the file-scope array below, which every GPU that loads this
// library keeps for the life of the process.
#include <mutex>
#include <string>

#include "nks_internal.cuh"

namespace nks {

namespace {

// scratch per point: 3 mobilities + 1 trace + 1 G_c + 6 stress + 4 derivatives
constexpr long long kPerPoint = 15;
constexpr long long kScratchDoubles = kPerPoint * NKS_NOALLOC_MAX_POINTS + kRedBlocks * 64 + 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::once_flag g_once[kMaxDevices];
double *g_scratch_ptr[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices];

}  // namespace

}  // namespace nks

using namespace nks;

extern "C" int nks_residual_noalloc(const nks_grid *grid, const nks_coeffs *coeffs, double cbar0, double dt, int mode,
                                    const double *X1, const double *X0, double *F, double *fnorm2, void *stream)
{
    if (!grid || !coeffs || !X1 || !X0 || !F || grid->dim < 1 || grid->dim > 3 || !(grid->h > 0.0) ||
        coeffs->S < 1 || coeffs->S > 16 || !(dt > 0.0) || (mode != 0 && mode != 1)) {
        set_thread_error("nks_residual_noalloc: invalid argument");
        return NKS_EINVAL;
    }
    if (grid->bc != NKS_PERIODIC && grid->bc != NKS_NEUMANN) {
        set_thread_error("nks_residual_noalloc: invalid argument");
        return NKS_EINVAL;
    }
    // the scratch holds the 2 x 2 pointwise block of one order parameter
    if (coeffs->n_eta != 0 && coeffs->n_eta != 1) {
        set_thread_error("nks_residual_noalloc: serves the model with one order parameter (n_eta 0 or 1)");
        return NKS_EINVAL;
    }
    DGrid g{};
    g.dim = grid->dim;
    g.bc = grid->bc;
    for (int J = 0; J < 3; J++) g.n[J] = J < grid->dim ? grid->n[J] : 1;
    for (int J = 0; J < g.dim; J++) {
        if (g.n[J] < 3) {
            set_thread_error("nks_residual_noalloc: at least 3 cells per axis");
            return NKS_EINVAL;
        }
        // each axis on its own first, so that the product below cannot overflow
        if (g.n[J] > NKS_NOALLOC_MAX_POINTS) {
            set_thread_error("nks_residual_noalloc: grid larger than NKS_NOALLOC_MAX_POINTS points; use the problem API");
            return NKS_EINVAL;
        }
    }
    g.N = (long long)g.n[0] * g.n[1] * g.n[2];
    set_spacing(g, grid->h);
    if (g.N > NKS_NOALLOC_MAX_POINTS) {
        set_thread_error("nks_residual_noalloc: grid larger than NKS_NOALLOC_MAX_POINTS points; use the problem API");
        return NKS_EINVAL;
    }
    // an error left pending by the caller's earlier work is theirs: fail without consuming it
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        set_thread_error((std::string("nks_residual_noalloc: a CUDA error of earlier work is pending: ") +
                          cudaGetErrorString(pending)).c_str());
        return NKS_ECUDA;
    }
    // set-up once per device, with that device current: the device address of the scratch array
    // (an address in the device's primary context, which a cudaDeviceReset invalidates)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_thread_error("nks_residual_noalloc: no usable CUDA device");
        return NKS_ECUDA;
    }
    std::call_once(g_once[dev], [dev] {
        g_setup_err[dev] = cudaGetSymbolAddress((void **)&g_scratch_ptr[dev], g_noalloc_scratch);
    });
    if (g_setup_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) {
        set_thread_error("nks_residual_noalloc: cudaGetSymbolAddress failed for the scratch array");
        return NKS_ECUDA;
    }
    const DCoef k = derive_coefficients(*coeffs, g.dim, cbar0);
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = g.N;
    double *base = g_scratch_ptr[dev];
    double *mob = base, *tr0 = mob + 3 * N, *Gc = tr0 + N, *sig = Gc + N, *part = sig + 6 * N;
    double *partials = base + kPerPoint * NKS_NOALLOC_MAX_POINTS;
    double *sums = partials + kRedBlocks * 64;  // 64 doubles after the partials
    int *flag = reinterpret_cast<int *>(sums + 8);
    double *isc = sums + 16;  // the kernels' per-instance scalars (dt, cbar0)
    auto fail = [](cudaError_t e, const char *what) {
        set_thread_error((std::string("nks_residual_noalloc: ") + what + ": " + cudaGetErrorString(e)).c_str());
        return NKS_ECUDA;
    };
    // the scratch keeps the previous call's contents: only the domain flag must start at zero
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(e, "clearing the domain flag");
    double hisc[I_NSC] = {0.0};
    hisc[I_DT] = dt;
    hisc[I_IDT] = 1.0 / dt;
    hisc[I_CBAR0] = cbar0;
    // from pageable memory: the source is staged before the call returns
    e = cudaMemcpyAsync(isc, hisc, sizeof(hisc), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(e, "uploading dt and cbar0");
    const Bat one{};
    launch_mobility(g, k, X0, mob, st, one);
    if (k.elastic) launch_trace0(g, k, isc, X0, tr0, st, one);
    launch_residual(g, k, isc, mode, X1, X0, tr0, mob, Gc, sig, part, F, flag, partials, kRedBlocks, st, one);
    launch_finalize(partials, kRedBlocks, 1, fnorm2 ? fnorm2 : sums, st, one);
    // nothing was pending at entry, so a launch error here is this call's
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "kernel launch");
    int hflag = 0;
    e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(e, "reading the domain flag");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e, "synchronising the stream");
    if (hflag & 1) {
        set_thread_error("nks_residual_noalloc: X1 leaves the domain of the logarithms");
        return NKS_EDOMAIN;
    }
    return NKS_OK;
}
