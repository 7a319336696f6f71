// FP32 elimination with residual refinement on the warp-task kernels
// (internal to libhines).
//
// x0 = A^{-1} b by the FP32 solve, which leaves the reciprocal eliminated
// diagonal in the workspace; then, per step, one pass of the task kernels in
// refinement mode: its elimination visit forms the residual r = b - A x
// (exact products and error-free sums of the FP32 inputs, in FP32 words) and
// eliminates it with the stored factor, its substitution visit solves for the
// correction c and writes x + c (a double-float pair between steps, FP64
// after the last).  The per-cell residual norms, when asked for, come from an
// FP64 residual of the final x.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hines.h"
#include "device_common.cuh"
#include "kernels.h"

namespace hines {
namespace {

using dev::ff_to_double;
using dev::kFull;

__device__ __forceinline__ double half_max(double v) {  // over the 16 lanes of a half-warp
  for (int o = 8; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// FP32 -> FP64 exactly on the integer pipe (the FP64 pipe is scarce)
__device__ __forceinline__ double widen(float v) { return ff_to_double(v, 0.f); }

// x = (double) xf
__global__ void k_widen(const float* __restrict__ xf, double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = widen(xf[i]);
}

// Residual r = b - A x in FP64 for every compartment, two branches per warp
// (branches are at most 16 long).  kStats = false: r rounded to FP32 into rf.
// kStats = true: per branch max |r|, max row sum |A| and max |x| into bstat.
template <bool kStats>
__global__ void k_residual(DevPlan P, const float* __restrict__ d, const float* __restrict__ u,
                           const float* __restrict__ b, const double* __restrict__ x, float* __restrict__ rf,
                           double* __restrict__ bstat) {
  const int lane = threadIdx.x & 31, half = lane >> 4, t = lane & 15;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nb = P.n_branches, pairs = (nb + 1) / 2;
  for (int64_t pr = gw; pr < pairs; pr += nw) {
    const int64_t br = 2 * pr + half;
    const bool vb = br < nb;
    const int64_t f0 = vb ? P.br_first[br] : 0;
    const int len = vb ? P.br_len[br] : 0;
    double r = 0.0, a = 0.0, xa = 0.0;
    if (t < len) {
      const int64_t i = f0 + t;
      const int32_t pb = P.br_parent[br];
      const double xi = x[i], di = widen(d[i]);
      r = fma(-di, xi, widen(b[i]));
      if (kStats) a = fabs(di);
      const int64_t pi = t > 0 ? i - 1 : (pb >= 0 ? (int64_t)P.br_first[pb] + P.br_len[pb] - 1 : -1);
      if (pi >= 0) {
        const double ui = widen(u[i]);
        r = fma(-ui, x[pi], r);
        if (kStats) a += fabs(ui);
      }
      if (t < len - 1) {
        const double un = widen(u[i + 1]);
        r = fma(-un, x[i + 1], r);
        if (kStats) a += fabs(un);
      } else {
        for (int32_t c = P.child_ptr[br]; c < P.child_ptr[br + 1]; ++c) {
          const int64_t fc = P.br_first[P.child[c]];
          const double uc = widen(u[fc]);
          r = fma(-uc, x[fc], r);
          if (kStats) a += fabs(uc);
        }
      }
      if (!kStats) rf[i] = (float)r;
      xa = fabs(xi);
    }
    if (kStats) {
      const double rm = half_max(fabs(r)), am = half_max(a), xm = half_max(xa);
      if (vb && t == 0) {
        bstat[3 * br] = rm;
        bstat[3 * br + 1] = am;
        bstat[3 * br + 2] = xm;
      }
    }
  }
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// One warp per cell: the cell's largest correction of this step from the
// per-branch maxima; HINES_WARN_REFINE when it grew since the last step.
__global__ void k_growth(DevPlan P, const float* __restrict__ bcorr, double* __restrict__ prev) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < P.n_cells; c += nw) {
    double m = 0.0;
    for (int64_t br = P.cell_br_off[c] + lane; br < P.cell_br_off[c + 1]; br += 32)
      m = fmax(m, widen(bcorr[br]));
    m = warp_max(m);
    if (lane == 0) {
      if (m > prev[c]) atomicMax(P.status, (int)HINES_WARN_REFINE);
      prev[c] = m;
    }
  }
}

// One warp per cell: ||b - A x||_inf / (||A||_inf ||x||_inf) from the per-branch maxima
__global__ void k_relres(DevPlan P, const double* __restrict__ bstat, double* __restrict__ relres) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < P.n_cells; c += nw) {
    double rm = 0.0, am = 0.0, xm = 0.0;
    for (int64_t br = P.cell_br_off[c] + lane; br < P.cell_br_off[c + 1]; br += 32) {
      rm = fmax(rm, bstat[3 * br]);
      am = fmax(am, bstat[3 * br + 1]);
      xm = fmax(xm, bstat[3 * br + 2]);
    }
    rm = warp_max(rm);
    am = warp_max(am);
    xm = warp_max(xm);
    if (lane == 0) relres[c] = (am > 0.0 && xm > 0.0) ? rm / (am * xm) : rm;
  }
}

// enough blocks to cover the items, at most 32 per multiprocessor of the plan's device
int grid_for(const DevPlan& P, int64_t items, int per_block) {
  const int64_t b = (items + per_block - 1) / per_block, cap = (int64_t)P.sms * 32;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

cudaError_t launch_unit_refine(const DevPlan& P, const float* d, const float* u, const float* b, double* x, int steps,
                               double* relres, cudaStream_t s) {
  const int64_t n = P.n_unknowns;
  const int32_t nc = P.n_cells;
  cudaError_t e = cudaSuccess;
  if (n == 0) {
    if (relres && nc > 0) e = cudaMemsetAsync(relres, 0, (size_t)nc * sizeof(double), s);
    return e;
  }
  float* x0 = static_cast<float*>(P.fac) + (n > P.n_packed ? n : P.n_packed);  // after the FP32 factor
  double* prev = static_cast<double*>(P.red);  // [n_cells] largest correction of the last step
  float* bcorr = static_cast<float*>(P.cb);    // [nb] largest correction per branch
  double* bstat = static_cast<double*>(P.cb) + P.n_branches;  // [nb][3] residual maxima per branch
  const int blocks_b = grid_for(P, (P.n_branches + 1) / 2 * 32, 256);
  const int blocks_n = grid_for(P, n, 256);
  const int blocks_c = grid_for(P, (int64_t)nc * 32, 256);
  e = launch_unit_solve_f32_rhs(P, d, u, b, x0, s);
  if (e == cudaSuccess && steps == 0) {
    k_widen<<<blocks_n, 256, 0, s>>>(x0, x, n);
    e = cudaGetLastError();
  }
  // the "last step" maxima start huge, so that the first step never warns
  if (e == cudaSuccess && steps > 0) e = cudaMemsetAsync(prev, 0x7F, (size_t)nc * sizeof(double), s);
  for (int step = 1; step <= steps && e == cudaSuccess; ++step) {
    const bool pairs = step > 1;  // after the first step x is a double-float pair, kept in x's 8 bytes
    e = launch_unit_refine_step(P, d, u, b, pairs ? static_cast<const void*>(x) : static_cast<const void*>(x0), pairs,
                                x, step == steps, bcorr, s);
    if (e != cudaSuccess) break;
    k_growth<<<blocks_c, 256, 0, s>>>(P, bcorr, prev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && relres) {
    k_residual<true><<<blocks_b, 256, 0, s>>>(P, d, u, b, x, nullptr, bstat);
    k_relres<<<blocks_c, 256, 0, s>>>(P, bstat, relres);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace hines
