// sweep_mixed.cu -- mixed-precision instantiation of the fused sweep kernels
// (FP32 stencils and Riemann solves; FP64 pressure numerator and RK update).
// Built with fast FP32 division and square root: the FP32 results are
// reported against the FP64 oracle with their measured error.
#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_mixed(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep_any<FORM_MIXED>(ndim, dir, mode, a, s);
}
}  // namespace mfc5
