// sweep_fp64.cu -- FP64 sweep kernels with the reorganised (fewer-instruction)
// formulas of physics.cuh; agree with the reference order to rounding.
#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_fp64(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep_any<FORM_FP64_FAST>(ndim, dir, mode, a, s);
}
}  // namespace mfc5
