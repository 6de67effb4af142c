// sweep_gated.cu -- the MLP-gated form: the mixed-precision sweep with a
// troubled-cell network choosing linear-weight reconstruction in smooth cells
// (plain WENO5-JS elsewhere and wherever a linear face state is non-physical).
// Built with the same fast FP32 division/square root as the mixed form.
#include <string.h>

#include "sweep.cuh"

namespace mfc5 {
cudaError_t launch_sweep_gated(int ndim, int dir, int mode, const SweepArgs& a, const GateWeights& g, cudaStream_t s) {
    static_assert(sizeof(GateArg<FORM_GATED>) == sizeof(GateWeights), "gate weights layout");
    GateArg<FORM_GATED> arg;
    memcpy(arg.w, g.w, sizeof(arg.w));
    return launch_sweep_any<FORM_GATED>(ndim, dir, mode, a, arg, s);
}
}  // namespace mfc5
