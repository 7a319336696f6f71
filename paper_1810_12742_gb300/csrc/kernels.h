// Device-side plan view and kernel launchers (internal to libhines).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hines {

// Per-branch metadata in warp-task order (one entry per position of torder).
struct __align__(16) BrMetaT {
  int64_t first;  // natural-layout index of the proximal compartment
  int64_t pcomp;  // natural-layout index of the parent compartment, -1 for a cell's root branch
  int32_t len;    // compartments (1..32)
  int32_t cbeg;   // children: positions tchild[cbeg .. cend)
  int32_t cend;
  int32_t ppos;   // position of the parent branch, -1 for a root branch
};

// Device copy of the host plan (pointers into one metadata allocation) and
// the plan's workspace.
struct DevPlan {
  int32_t n_cells = 0;
  int32_t n_tasks = 0;
  int32_t cta_threads = 256;
  int64_t n_unknowns = 0;
  int64_t n_branches = 0;
  const int64_t* cell_off = nullptr;      // [n_cells + 1]
  const int32_t* task_cell = nullptr;     // [n_tasks]
  const int32_t* cell_nlvl = nullptr;     // [n_cells]
  const int64_t* cell_lvl_off = nullptr;  // [n_cells]
  const int32_t* lvl_ptr = nullptr;       // per cell nlvl + 1
  const int32_t* order = nullptr;         // [nb]
  const int64_t* br_first = nullptr;      // [nb]
  const int32_t* br_len = nullptr;        // [nb]
  const int32_t* br_parent = nullptr;     // [nb]
  const int32_t* child_ptr = nullptr;     // [nb + 1]
  const int32_t* child = nullptr;         // [nb - n_roots]
  // warp tasks
  int32_t n_wtasks = 0;
  const int32_t* task_nlvl = nullptr;     // [n_wtasks]
  const int64_t* task_lvl_off = nullptr;  // [n_wtasks]
  const int32_t* tlvl_ptr = nullptr;      // per task nlvl + 1 positions
  const BrMetaT* tmeta = nullptr;         // [nb] by position
  const int32_t* tchild = nullptr;        // child positions
  int32_t* counter = nullptr;             // work counter (workspace)
  int32_t grid_f64 = 1, grid_f32 = 1, grid_cable = 1, grid_comp = 1;  // persistent grid sizes
  // workspace
  void* fac = nullptr;    // n_unknowns * 8 bytes: eliminated diagonal (FP64), or two FP32 arrays
  void* cd = nullptr;     // n_branches * 8 bytes: child-to-parent diagonal contribution
  void* cb = nullptr;     // n_branches * 8 bytes: child-to-parent right-hand-side contribution
  void* red = nullptr;    // n_cells * 8 bytes: per-cell reductions
  int32_t* status = nullptr;  // device status word
};

// warp-task kernels; prepare_warp_kernels sets their shared-memory limits and
// persistent grid sizes once per plan (outside any stream capture)
cudaError_t prepare_warp_kernels(DevPlan& P);
cudaError_t launch_warp_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s);
cudaError_t launch_warp_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s);
cudaError_t launch_warp_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                          cudaStream_t s);
cudaError_t launch_warp_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, bool rhs_from_V, cudaStream_t s);

cudaError_t launch_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s);
cudaError_t launch_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s);
cudaError_t launch_solve_refine(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                int steps, double* relres, cudaStream_t s);
cudaError_t launch_cable_step(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, cudaStream_t s);
cudaError_t launch_cable_solve(const DevPlan& P, const double* sv, const double* g, const double* u, double* y,
                               double dt, int theta, cudaStream_t s);
cudaError_t launch_grad_du(const DevPlan& P, const double* lam, const double* x, double* gd, double* gu,
                           cudaStream_t s);
cudaError_t launch_cable_adjoint_step(const DevPlan& P, const double* lam, const double* Vk, const double* Vkm1,
                                      const double* sv, const double* g, const double* target, double dt, double E,
                                      int theta, int add_loss, double* grad_g, double* grad_a, double* vbar,
                                      cudaStream_t s);
cudaError_t launch_cable_loss_accumulate(const DevPlan& P, const double* V, const double* target, double* loss,
                                         cudaStream_t s);
cudaError_t launch_cable_loss_seed(const DevPlan& P, const double* V, const double* target, double* vbar,
                                   cudaStream_t s);

}  // namespace hines
