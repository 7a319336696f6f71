// Warp-task kernels with 1 piece per lane (the templates are in unit_kernels.cuh;
// one translation unit per lane mapping so that they compile in parallel).
#include "unit_kernels.cuh"

namespace hines {

cudaError_t unit_prepare_p1(DevPlan& P) { return UnitKernels<1>::prepare(P); }
cudaError_t unit_run_p1(const DevPlan& P, const UnitCall& c, cudaStream_t s) { return UnitKernels<1>::run(P, c, s); }

}  // namespace hines
