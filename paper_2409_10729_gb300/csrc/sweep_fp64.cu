// sweep_fp64.cu -- FP64 instantiation of the fused sweep kernels.
#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_fp64(int ndim, int dir, int mode, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep_any<double>(ndim, dir, mode, a, s);
}
}  // namespace mfc5
