// noalloc.cu -- mfc_rhs_noalloc: the FP64 right-hand side without any device
// allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// right-hand side: code running inside a framework that owns every byte of
// the GPU through its own pool allocator and forbids side allocations, a
// long-running service that must not grow its footprint or hit cudaMalloc's
// implicit device synchronisation after start-up, or a host that has no
// handle through which to create and keep a solver context.  For them this
// entry point evaluates L(q) for caller-owned input and output buffers and
// keeps its only scratch -- the RHS accumulator that the direction sweeps add
// into, and the non-physical status word -- in one fixed array of device
// memory that is part of the library image itself.
//
// That array is a file-scope __device__ variable of MFC_NOALLOC_MAX_DOUBLES
// doubles (16 MiB).  Every device that loads the library holds it until the
// process exits.  In host code its name is only a host-side stand-in, not a
// device address, so its address is looked up per device with
// cudaGetSymbolAddress on the first call made with that device current, and
// kept for the life of the process: that first call should come before any
// stream capture, and the library must not be called again on a device after
// cudaDeviceReset() (the array is then reloaded at an address the cache does
// not know).  All calls share the array and it keeps the previous call's
// contents: the status word is cleared at the start of every call (the
// accumulator is fully rewritten by the first sweep).  Calls whose kernels
// overlap on the GPU -- on different streams, or from different host
// threads -- race on the array and must be serialised by the caller.  Every
// call synchronises its stream before returning, to read the status word.
// The output must not overlap the input: the last sweep writes L into cells
// whose neighbours other warps are still reading as stencil input.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "mfc.h"
#include "mfc_internal.cuh"

using namespace mfc5;

// The fixed scratch: a file-scope device array of the library image.
static __device__ __align__(256) double g_noalloc_scratch[MFC_NOALLOC_MAX_DOUBLES];

namespace {

// First 32 doubles: the control block (status word); the rest: accumulator.
constexpr long long kCtrlDoubles = 32;
static_assert(sizeof(DevCtrl) <= kCtrlDoubles * sizeof(double), "control block does not fit");

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MFC_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return MFC_EINVAL;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MFC_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return MFC_OK;
}

int check_params(const mfc_params* p) {
    if (!p || p->ndim < 1 || p->ndim > 3) return MFC_EINVAL;
    for (int d = 0; d < p->ndim; ++d) {
        if (p->n[d] < 1) return MFC_EINVAL;
        if (!(p->hi[d] > p->lo[d]) || !isfinite(p->hi[d] - p->lo[d])) return MFC_EINVAL;
        int b0 = p->bc[d][0], b1 = p->bc[d][1];
        if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b0 != b1) return MFC_EINVAL;
    }
    if (p->nfluids != 0 && (p->nfluids < 2 || p->nfluids > MFC_MAX_FLUIDS)) return MFC_EINVAL;
    for (int i = 0; i < params_nfluids(p->nfluids); ++i)
        if (!(p->gamma[i] > 1.0) || !isfinite(p->gamma[i]) || !(p->pi_inf[i] >= 0.0) || !isfinite(p->pi_inf[i]))
            return MFC_EINVAL;
    if (!(p->weno_eps > 0.0) || !isfinite(p->weno_eps)) return MFC_EINVAL;
    if (p->precision != MFC_FP64) return MFC_EINVAL;
    if (p->weno_order != 0 && p->weno_order != 3 && p->weno_order != 5) return MFC_EINVAL;
    return MFC_OK;
}

}  // namespace

extern "C" int mfc_rhs_noalloc(const mfc_params* params, const double* q, double* rhs, void* cuda_stream) {
    if (!q || !rhs) return MFC_EINVAL;
    int st = check_params(params);
    if (st) return st;
    const int ndim = params->ndim, neq = 2 * params_nfluids(params->nfluids) + ndim;
    // neq * ncell against the scratch, checked per factor so that no product
    // can overflow (each n[d] >= 1)
    const long long cap = ((long long)MFC_NOALLOC_MAX_DOUBLES - kCtrlDoubles) / neq;
    int n[3];
    long long ncell = 1;
    for (int d = 0; d < 3; ++d) {
        n[d] = d < ndim ? params->n[d] : 1;
        if (ncell > cap / n[d]) return MFC_ETOOBIG;
        ncell *= n[d];
    }
    // input and output ranges must be disjoint (compared as addresses; the
    // byte count is below 16 MiB, so no sum wraps)
    const uintptr_t qa = (uintptr_t)q, ra = (uintptr_t)rhs;
    const uintptr_t bytes = (uintptr_t)(neq * ncell) * sizeof(double);
    if (qa < ra + bytes && ra < qa + bytes) return MFC_EINVAL;

    double* scratch = nullptr;
    st = scratch_for_current_device(&scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DevCtrl* ctrl = reinterpret_cast<DevCtrl*>(scratch);
    if (cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), s) != cudaSuccess) return MFC_ECUDA;


    SweepArgs a;
    memset(&a, 0, sizeof(a));
    for (int d = 0; d < 3; ++d) {
        a.n[d] = n[d];
        a.inv_dx[d] = d < ndim ? (double)n[d] / (params->hi[d] - params->lo[d]) : 0.0;
        a.dx[d] = d < ndim ? (params->hi[d] - params->lo[d]) / (double)n[d] : 1.0;
        a.rdx[d] = 1.0 / a.dx[d];
    }
    a.ncell = ncell;
    a.eos = make_eos(params->gamma, params->pi_inf, params_nfluids(params->nfluids));
    a.eps = params->weno_eps;
    a.order = params->weno_order == 3 ? 3 : 5;
    a.ctrl = ctrl;
    a.acc = scratch + kCtrlDoubles;
    a.qin = q;
    a.qout = rhs;
    for (int d = 0; d < ndim; ++d) {
        a.periodic = params->bc[d][0] == MFC_BC_PERIODIC;
        int mode = d == ndim - 1 ? SW_LAST_RHS : (d == 0 ? SW_FIRST : SW_MID);
        if (launch_sweep_fp64x(ndim, d, mode, a, s) != cudaSuccess) return MFC_ECUDA;
    }
    unsigned int status = 0;
    if (cudaMemcpyAsync(&status, &ctrl->status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MFC_ECUDA;
    return status ? MFC_ENONPHYSICAL : MFC_OK;
}
