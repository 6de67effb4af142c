// sweep_gated.cu -- the MLP-gated form: the mixed-precision sweep with a
// troubled-cell network (evaluated on the tensor cores) choosing
// linear-weight reconstruction in smooth cells; plain WENO5-JS elsewhere and
// wherever a linear face state is non-physical.  Built with the same fast
// FP32 division/square root as the mixed form.
#include "mfc.h"
#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_gated(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep_any<FORM_GATED>(ndim, dir, mode, a, s);
}

// Batched logits with the sweep's tensor-core evaluation: each warp takes 64
// samples per pass (rows 0-31 in the density slot, 32-63 in the pressure slot).
__global__ void __launch_bounds__(128) gate_forward_tc_kernel(const float* __restrict__ X, long long n,
                                                              const float* __restrict__ theta, float* z) {
    __shared__ GateSmem g;
    __shared__ uint4 tile[4 * 128];
    gate_fill(g, theta);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nwarps = (long long)gridDim.x * 4;
    for (long long base = ((long long)blockIdx.x * 4 + warp) * 64; base < n; base += nwarps * 64) {
        float xr[5], xp[5], zr, zp;
        const long long sr = base + lane, sp = base + 32 + lane;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            xr[k] = sr < n ? X[sr * 5 + k] : 0.f;
            xp[k] = sp < n ? X[sp * 5 + k] : 0.f;
        }
        gate_logits(g, tile + warp * 128, xr, xp, sr < n, sp < n, false, zr, zp);
        if (sr < n) z[sr] = zr;
        if (sp < n) z[sp] = zp;
    }
}
}  // namespace mfc5

extern "C" int mfc_mlp_forward_tc(const float* X, long long n, const float* theta, float* z, void* cuda_stream) {
    if (!X || !theta || !z || n <= 0) return MFC_EINVAL;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    mfc5::gate_forward_tc_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)cuda_stream>>>(X, n, theta, z);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ECUDA;
}
