// Warp-task kernels with 2 pieces per lane (the templates are in unit_kernels.cuh;
// one translation unit per lane mapping so that they compile in parallel).
#include "unit_kernels.cuh"

namespace hines {

cudaError_t unit_prepare_p2(DevPlan& P) { return UnitKernels<2>::prepare(P); }
cudaError_t unit_run_p2(const DevPlan& P, const UnitCall& c, cudaStream_t s) { return UnitKernels<2>::run(P, c, s); }

}  // namespace hines
