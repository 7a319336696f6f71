// CUDA kernels of the adjoint (internal to libhines): the elementwise
// gathers of the gradient and the rollout loss terms, one warp per branch
// over the natural layout.  The solves themselves are the warp-task kernels.
#include <cfloat>

#include "kernels.h"
#include "../../include/hines.h"

namespace hines {
namespace {

// ----------------------------------------------------------------------------
// Per-compartment kernels that need the parent of every compartment: one warp
// per branch, lanes over the branch's compartments.
// ----------------------------------------------------------------------------
template <typename F>
__device__ __forceinline__ void for_each_branch_compartment(const DevPlan& P, F&& f) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t br = warp; br < P.n_branches; br += nwarps) {
    const int64_t f0 = P.br_first[br];
    const int32_t len = P.br_len[br];
    const int32_t pb = P.br_parent[br];
    const int64_t pcomp = pb >= 0 ? P.br_first[pb] + P.br_len[pb] - 1 : -1;
    for (int32_t j = lane; j < len; j += 32) {
      const int64_t i = f0 + j;
      f(i, j > 0 ? i - 1 : pcomp);
    }
  }
}

__global__ void k_grad_du(DevPlan P, const double* __restrict__ lam, const double* __restrict__ x,
                          double* __restrict__ gd, double* __restrict__ gu) {
  for_each_branch_compartment(P, [&](int64_t i, int64_t pi) {
    gd[i] = -lam[i] * x[i];
    gu[i] = pi >= 0 ? -(lam[i] * x[pi] + lam[pi] * x[i]) : 0.0;
  });
}

__global__ void k_cable_adjoint_step(DevPlan P, const double* __restrict__ lam, const double* __restrict__ Vk,
                                     const double* __restrict__ Vm, const double* __restrict__ sv,
                                     const double* __restrict__ g, double dt, double E, double theta,
                                     double* __restrict__ grad_g, double* __restrict__ grad_a,
                                     double* __restrict__ vbar) {
  for_each_branch_compartment(P, [&](int64_t i, int64_t pi) {
    const double li = lam[i], si = sv[i], gi = g[i];
    grad_g[i] += li * si * dt * (E - (1.0 - theta) * Vm[i]) - theta * si * dt * li * Vk[i];
    if (pi >= 0) grad_a[i] += -(li - lam[pi]) * (Vk[i] - Vk[pi]);
    vbar[i] = li * si * (1.0 - (1.0 - theta) * dt * gi);
  });
}

__global__ void k_cable_loss_seed(DevPlan P, const double* __restrict__ V, const double* __restrict__ target,
                                  double* __restrict__ vbar) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n_cells) return;
  const int64_t lo = P.cell_off[c];
  if (P.cell_off[c + 1] > lo) vbar[lo] += 2.0 * (V[lo] - target[c]);
}

__global__ void k_cable_loss_accumulate(DevPlan P, const double* __restrict__ V, const double* __restrict__ target,
                                        double* __restrict__ loss) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n_cells) return;
  const int64_t lo = P.cell_off[c];
  if (P.cell_off[c + 1] > lo) {
    const double e = V[lo] - target[c];
    loss[c] += e * e;
  }
}

int grid_for_branches(const DevPlan& P) {
  const int64_t warps = P.n_branches;
  const int64_t blocks = (warps * 32 + 255) / 256;
  const int64_t cap = (int64_t)P.sms * 16;  // 16 blocks of 256 threads per multiprocessor at most
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

cudaError_t launch_grad_du(const DevPlan& P, const double* lam, const double* x, double* gd, double* gu,
                           cudaStream_t s) {
  if (P.n_branches == 0) return cudaSuccess;
  k_grad_du<<<grid_for_branches(P), 256, 0, s>>>(P, lam, x, gd, gu);
  return cudaGetLastError();
}

cudaError_t launch_cable_adjoint_step(const DevPlan& P, const double* lam, const double* Vk, const double* Vkm1,
                                      const double* sv, const double* g, const double* target, double dt, double E,
                                      int theta, int add_loss, double* grad_g, double* grad_a, double* vbar,
                                      cudaStream_t s) {
  if (P.n_branches == 0) return cudaSuccess;
  k_cable_adjoint_step<<<grid_for_branches(P), 256, 0, s>>>(P, lam, Vk, Vkm1, sv, g, dt, E, (double)theta, grad_g,
                                                             grad_a, vbar);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !add_loss) return e;
  return launch_cable_loss_seed(P, Vkm1, target, vbar, s);
}

cudaError_t launch_cable_loss_accumulate(const DevPlan& P, const double* V, const double* target, double* loss,
                                         cudaStream_t s) {
  if (P.n_cells == 0) return cudaSuccess;
  k_cable_loss_accumulate<<<(P.n_cells + 255) / 256, 256, 0, s>>>(P, V, target, loss);
  return cudaGetLastError();
}

cudaError_t launch_cable_loss_seed(const DevPlan& P, const double* V, const double* target, double* vbar,
                                   cudaStream_t s) {
  if (P.n_cells == 0) return cudaSuccess;
  k_cable_loss_seed<<<(P.n_cells + 255) / 256, 256, 0, s>>>(P, V, target, vbar);
  return cudaGetLastError();
}

}  // namespace hines
