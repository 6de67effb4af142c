// sweep_fp64x.cu -- FP64 sweep kernels in the reference operation order
// (physics_exact.cuh).  Built with -fmad=false so that no a*b+c is
// contracted: every result is bit-identical to the serial formula order.
#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_fp64x(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep_any<FORM_FP64_EXACT>(ndim, dir, mode, a, s);
}
}  // namespace mfc5
