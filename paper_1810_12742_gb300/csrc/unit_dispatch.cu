// Entry points of the warp-task solves: each builds a UnitCall and hands it to
// the kernels of the plan's lane mapping (one or two pieces per lane).
#include <cuda_runtime.h>

#include "kernels.h"

namespace hines {

cudaError_t unit_prepare_p1(DevPlan& P);
cudaError_t unit_prepare_p2(DevPlan& P);
cudaError_t unit_run_p1(const DevPlan& P, const UnitCall& c, cudaStream_t s);
cudaError_t unit_run_p2(const DevPlan& P, const UnitCall& c, cudaStream_t s);

namespace {
cudaError_t run(const DevPlan& P, const UnitCall& c, cudaStream_t s) {
  return P.per_lane == 2 ? unit_run_p2(P, c, s) : unit_run_p1(P, c, s);
}
UnitCall call(UnitOp op) {
  UnitCall c;
  c.op = op;
  return c;
}
}  // namespace

cudaError_t prepare_unit_kernels(DevPlan& P) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  P.sms = sms > 0 ? sms : 1;
  return P.per_lane == 2 ? unit_prepare_p2(P) : unit_prepare_p1(P);
}

cudaError_t launch_unit_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s) {
  UnitCall c = call(UnitOp::F64);
  c.d = d, c.u = u, c.x = b;
  return run(P, c, s);
}
cudaError_t launch_unit_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s) {
  UnitCall c = call(UnitOp::F32);
  c.d = d, c.u = u, c.x = b;
  return run(P, c, s);
}
cudaError_t launch_unit_resolve_f32(const DevPlan& P, const float* u, float* b, cudaStream_t s) {
  UnitCall c = call(UnitOp::F32Resolve);
  c.u = u, c.x = b;
  return run(P, c, s);
}
cudaError_t launch_unit_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                          cudaStream_t s) {
  UnitCall c = call(UnitOp::Comp);
  c.d = d, c.u = u, c.b = b, c.x = x;
  return run(P, c, s);
}
cudaError_t launch_unit_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, bool rhs_from_V, cudaStream_t s) {
  UnitCall c = call(UnitOp::Cable);
  c.s = sv, c.g = g, c.u = u, c.x = V, c.dt = dt, c.E = E, c.theta = theta, c.rhs_from_V = rhs_from_V;
  return run(P, c, s);
}
cudaError_t launch_unit_solve_f32_rhs(const DevPlan& P, const float* d, const float* u, const float* rhs, float* x,
                                      cudaStream_t s) {
  UnitCall c = call(UnitOp::F32);
  c.d = d, c.u = u, c.rhs = rhs, c.x = x;
  return run(P, c, s);
}
cudaError_t launch_unit_refine_step(const DevPlan& P, const float* d, const float* u, const float* b, const void* x,
                                    bool x_pairs, void* xo, bool final, float* bcorr, cudaStream_t s) {
  UnitCall c = call(x_pairs ? (final ? UnitOp::Refine2to64 : UnitOp::Refine2to2)
                            : (final ? UnitOp::Refine32to64 : UnitOp::Refine32to2));
  c.d = d, c.u = u, c.b = b, c.rhs = x, c.x = xo, c.rw = static_cast<float*>(P.rw), c.bcorr = bcorr;
  return run(P, c, s);
}
cudaError_t launch_pk_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s) {
  UnitCall c = call(UnitOp::PkF64);
  c.d = d, c.u = u, c.x = b;
  return run(P, c, s);
}
cudaError_t launch_pk_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s) {
  UnitCall c = call(UnitOp::PkF32);
  c.d = d, c.u = u, c.x = b;
  return run(P, c, s);
}
cudaError_t launch_pk_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                        cudaStream_t s) {
  UnitCall c = call(UnitOp::PkComp);
  c.d = d, c.u = u, c.b = b, c.x = x;
  return run(P, c, s);
}
cudaError_t launch_pk_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V, double dt,
                            double E, int theta, bool rhs_from_V, cudaStream_t s) {
  UnitCall c = call(UnitOp::PkCable);
  c.s = sv, c.g = g, c.u = u, c.x = V, c.dt = dt, c.E = E, c.theta = theta, c.rhs_from_V = rhs_from_V;
  return run(P, c, s);
}
cudaError_t launch_unit_cable_reuse(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                                    double dt, double E, int theta, bool packed, cudaStream_t s) {
  UnitCall c = call(packed ? UnitOp::PkCableReuse : UnitOp::CableReuse);
  c.s = sv, c.g = g, c.u = u, c.x = V, c.dt = dt, c.E = E, c.theta = theta;
  return run(P, c, s);
}

}  // namespace hines
