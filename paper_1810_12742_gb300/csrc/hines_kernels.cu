// CUDA kernels of the batched Hines solver, sm_103a: the FP32 + FP64
// refinement solve and the adjoint's elementwise gathers.
//
// k_solve_refine is level-synchronous and branch-parallel (Section 3): one CTA
// owns one cell; the branches of a level are processed in parallel, one
// thread per branch, deepest level first for the elimination and root level
// first for the substitution, with a CTA barrier between levels.  Inside a
// branch the parent of compartment i is i - 1 (Section 5), so a thread runs a
// Thomas chain (Listing 1); at the branch's proximal end the elimination
// produces one contribution to the parent compartment (Listing 2's parent
// lookup), which the parent branch's thread folds in before its own chain
// starts.  Child contributions go through per-branch slots, so siblings never
// write the same word and the fold order is fixed (children by first
// compartment, descending).
#include <cfloat>

#include "kernels.h"
#include "../../include/hines.h"

namespace hines {
namespace {

// ----------------------------------------------------------------------------
// Mixed precision: FP32 elimination, FP64 residual and correction.
// Workspace: fac32 = eliminated diagonal (float[N]), w32 = working vector
// (float[N]), cd32/cb32 per-branch contributions (float).
// ----------------------------------------------------------------------------
__device__ __forceinline__ double block_max(double v, double* sh) {
  // sh: at least 32 doubles
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int j = 0; j < nw; ++j) r = fmax(r, sh[j]);
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_solve_refine(DevPlan P, const float* __restrict__ d,
                                                        const float* __restrict__ u, const float* __restrict__ b,
                                                        double* __restrict__ x, int steps, double* relres) {
  __shared__ double sh[32];
  const int32_t cell = P.task_cell[blockIdx.x];
  const int32_t nl = P.cell_nlvl[cell];
  if (nl == 0) {
    if (relres && threadIdx.x == 0) relres[cell] = 0.0;
    return;
  }
  const int32_t* lp = P.lvl_ptr + P.cell_lvl_off[cell];
  float* fac = static_cast<float*>(P.fac);
  float* w = fac + P.n_unknowns;
  float* cd = static_cast<float*>(P.cd);
  float* cb = static_cast<float*>(P.cb);
  double prev_corr = DBL_MAX;

  for (int pass = 0; pass <= steps; ++pass) {
    const bool first_pass = (pass == 0);
    // backward: FP32 elimination of the right-hand side (pass 0: b and the
    // diagonal; later passes: the FP64 residual of the current x)
    for (int l = nl - 1; l >= 0; --l) {
      for (int k = lp[l] + (int)threadIdx.x; k < lp[l + 1]; k += blockDim.x) {
        const int32_t br = P.order[k];
        const int64_t f0 = P.br_first[br];
        const int64_t last = f0 + P.br_len[br] - 1;
        const int32_t pb = P.br_parent[br];
        const int64_t pcomp = pb >= 0 ? P.br_first[pb] + P.br_len[pb] - 1 : -1;
        // residual r_i = b_i - d_i x_i - u_i x_p(i) - sum over children u_c x_c, in FP64
        auto resid = [&](int64_t i) -> float {
          double r = (double)b[i] - (double)d[i] * x[i];
          if (i > f0) r -= (double)u[i] * x[i - 1];
          else if (pcomp >= 0) r -= (double)u[i] * x[pcomp];
          if (i < last) {
            r -= (double)u[i + 1] * x[i + 1];
          } else {
            for (int32_t c = P.child_ptr[br]; c < P.child_ptr[br + 1]; ++c) {
              const int64_t fc = P.br_first[P.child[c]];
              r -= (double)u[fc] * x[fc];
            }
          }
          return (float)r;
        };
        int64_t i = last;
        float cur_b = first_pass ? b[i] : resid(i);
        float cur_d = first_pass ? d[i] : 0.f;
        for (int32_t c = P.child_ptr[br]; c < P.child_ptr[br + 1]; ++c) {
          const int32_t ch = P.child[c];
          if (first_pass) cur_d -= cd[ch];
          cur_b -= cb[ch];
        }
        for (; i > f0; --i) {
          if (first_pass) fac[i] = cur_d; else cur_d = fac[i];
          w[i] = cur_b;
          const float ui = u[i];
          const float f = ui / cur_d;
          if (first_pass) cur_d = d[i - 1] - f * ui;
          cur_b = (first_pass ? b[i - 1] : resid(i - 1)) - f * cur_b;
        }
        if (first_pass) fac[f0] = cur_d; else cur_d = fac[f0];
        if (pb >= 0) {
          w[f0] = cur_b;
          const float ui = u[f0];
          const float f = ui / cur_d;
          if (first_pass) cd[br] = f * ui;
          cb[br] = f * cur_b;
        } else {
          w[f0] = cur_b / cur_d;
        }
      }
      __syncthreads();
    }
    // forward: FP32 substitution, then x = w (pass 0) or x += w, in FP64
    double corr = 0.0;
    for (int l = 0; l < nl; ++l) {
      for (int k = lp[l] + (int)threadIdx.x; k < lp[l + 1]; k += blockDim.x) {
        const int32_t br = P.order[k];
        const int64_t f0 = P.br_first[br];
        const int64_t end = f0 + P.br_len[br];
        const int32_t pb = P.br_parent[br];
        int64_t i = f0;
        float wp;
        if (pb < 0) {
          wp = w[f0];
          if (first_pass) x[f0] = (double)wp; else x[f0] += (double)wp;
          corr = fmax(corr, fabs((double)wp));
          ++i;
        } else {
          wp = w[P.br_first[pb] + P.br_len[pb] - 1];
        }
        for (; i < end; ++i) {
          const float wi = (w[i] - u[i] * wp) / fac[i];
          w[i] = wi;
          wp = wi;
          if (first_pass) x[i] = (double)wi; else x[i] += (double)wi;
          corr = fmax(corr, fabs((double)wi));
        }
      }
      __syncthreads();
    }
    if (!first_pass) {
      corr = block_max(corr, sh);
      if (corr > prev_corr && threadIdx.x == 0) atomicMax(P.status, (int)HINES_WARN_REFINE);
      prev_corr = corr;
    }
  }
  if (relres) {
    // scaled residual of the returned x, FP64
    double rmax = 0.0, amax = 0.0, xmax = 0.0;
    const int64_t lo = P.cell_off[cell], hi = P.cell_off[cell + 1];
    for (int l = 0; l < nl; ++l) {
      for (int k = lp[l] + (int)threadIdx.x; k < lp[l + 1]; k += blockDim.x) {
        const int32_t br = P.order[k];
        const int64_t f0 = P.br_first[br];
        const int64_t last = f0 + P.br_len[br] - 1;
        const int32_t pb = P.br_parent[br];
        const int64_t pcomp = pb >= 0 ? P.br_first[pb] + P.br_len[pb] - 1 : -1;
        for (int64_t i = f0; i <= last; ++i) {
          double r = (double)b[i] - (double)d[i] * x[i];
          double a = fabs((double)d[i]);
          const int64_t pi = i > f0 ? i - 1 : pcomp;
          if (pi >= 0) {
            r -= (double)u[i] * x[pi];
            a += fabs((double)u[i]);
          }
          if (i < last) {
            r -= (double)u[i + 1] * x[i + 1];
            a += fabs((double)u[i + 1]);
          } else {
            for (int32_t c = P.child_ptr[br]; c < P.child_ptr[br + 1]; ++c) {
              const int64_t fc = P.br_first[P.child[c]];
              r -= (double)u[fc] * x[fc];
              a += fabs((double)u[fc]);
            }
          }
          rmax = fmax(rmax, fabs(r));
          amax = fmax(amax, a);
          xmax = fmax(xmax, fabs(x[i]));
        }
      }
    }
    (void)lo;
    (void)hi;
    rmax = block_max(rmax, sh);
    amax = block_max(amax, sh);
    xmax = block_max(xmax, sh);
    if (threadIdx.x == 0) relres[cell] = (amax > 0.0 && xmax > 0.0) ? rmax / (amax * xmax) : rmax;
  }
}

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
  return (int)(blocks < 152 * 16 ? (blocks > 0 ? blocks : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_solve_refine(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                int steps, double* relres, cudaStream_t s) {
  if (P.n_tasks == 0) return cudaSuccess;
  k_solve_refine<<<P.n_tasks, P.cta_threads, 0, s>>>(P, d, u, b, x, steps, relres);
  return cudaGetLastError();
}

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
