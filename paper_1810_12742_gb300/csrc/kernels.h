// Device-side plan view and kernel launchers (internal to libhines).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hines {

// Per-branch metadata in task order (one entry per position of torder).
struct __align__(16) BrMetaT {
  int64_t first;    // natural-layout index of the proximal compartment
  int64_t pcomp;    // natural-layout index of the parent compartment, -1 for a cell's root branch
  int32_t ppos;     // position of the parent branch, -1 for a cell's root branch
  int32_t cpos;     // children: first child position if contiguous, else first index into tchild
  int16_t len;      // compartments (1..16)
  int16_t nchild;   // children
  int16_t ccontig;  // 1: the children are positions cpos .. cpos + nchild - 1
  int16_t xtask;    // 1: some child is in another task (written by another warp in the same launch)
};

// Device copy of the host plan (pointers into one metadata allocation) and
// the plan's workspace.
struct DevPlan {
  int32_t n_cells = 0;
  int64_t n_unknowns = 0;
  int64_t n_branches = 0;
  // branches in the natural layout (refinement residual, adjoint gathers)
  const int64_t* cell_off = nullptr;      // [n_cells + 1]
  const int64_t* br_first = nullptr;      // [nb]
  const int32_t* br_len = nullptr;        // [nb]
  const int32_t* br_parent = nullptr;     // [nb]
  const int32_t* br_cell = nullptr;       // [nb]
  const int64_t* cell_br_off = nullptr;   // [n_cells + 1] branches of each cell
  const int32_t* child_ptr = nullptr;     // [nb + 1]
  const int32_t* child = nullptr;         // [nb - roots]
  // warp tasks over units (whole cells, subtrees, top parts)
  int32_t n_wtasks = 0;
  const int32_t* task_nlvl = nullptr;     // [n_wtasks]
  const int64_t* task_lvl_off = nullptr;  // [n_wtasks]
  const int32_t* tlvl_ptr = nullptr;      // per task nlvl + 1 positions
  const BrMetaT* tmeta = nullptr;         // [nb] by position
  const int32_t* tchild = nullptr;        // child positions (non-contiguous children)
  const int32_t* phase_entry = nullptr;   // 4 * task + visits, phases A, B (empty), C concatenated
  int32_t phase_off[4] = {0, 0, 0, 0};
  int32_t* counter = nullptr;             // [4 + n_cells] work counters, then cell_pending (workspace)
  const int32_t* counter_init = nullptr;  // [4 + n_cells] values restored before every solve
  const int32_t* cell_top_task = nullptr; // [n_cells] task of the cell's top part, -1 if not cut
  const int32_t* task_sub = nullptr;      // [2 * n_wtasks] (cell, subtree units) of a subtree task
  const int32_t* pos_branch = nullptr;    // [nb] branch id (natural numbering) of each position
  int32_t* cell_pending = nullptr;        // counter + 4: subtree units whose elimination is still to finish
  // solver layout (Section 5's interleaving per chunk)
  int64_t n_packed = 0;
  const longlong2* pk_meta = nullptr;     // [nb] per position: (chunk block offset, parent's solver-layout index)
  const int64_t* pk_perm = nullptr;       // [n_packed] natural index of each solver-layout slot, -1 for padding
  const int64_t* pk_edge = nullptr;       // [n_packed] natural index of each slot's coupling (pk_perm unless re-rooted)
  int32_t grid[8] = {1, 1, 1, 1, 1, 1, 1, 1};  // persistent grid size per kernel kind
  int32_t grid_nf[4] = {1, 1, 1, 1};           // the same for the FP64 kinds keeping the factor at natural positions
  int32_t fp64_blocks = 0;                     // 1: FP64 factors in block order (hines_plan_opts.fp64_factor)
  int32_t sms = 1;                             // multiprocessors of the plan's device
  int32_t per_lane = 2;                        // branch pieces per warp lane (the plan's lane mapping)
  int32_t grid_refine = 1;                     // persistent grid size of the refinement steps
  // workspace
  void* fac = nullptr;    // 8 bytes per natural or solver-layout slot: factor (FP64 / FP32 solves), FP32 working
                          // arrays (refine)
  void* cd = nullptr;     // n_branches * 16 bytes: child-to-parent contribution (or root solution) per position
  void* cb = nullptr;     // n_branches * 32 bytes: per-branch reductions of the refinement
  void* xlast = nullptr;  // n_branches * 8 bytes: solution at the distal compartment per position
  void* red = nullptr;    // n_cells * 8 bytes: per-cell reductions
  void* rw = nullptr;     // 4 bytes per natural or solver-layout slot: the refinement's eliminated residual
  void* ff4 = nullptr;    // 16 bytes per solver-layout slot: the compensated solve's factor (y, g as pairs)
  int32_t* status = nullptr;  // device status word
};

// One call of the warp-task kernels (unit_kernels.cuh): the mode and its arrays.
enum class UnitOp {
  F64, F32, F32Resolve, Comp, Cable, CableReuse, PkF64, PkF32, PkComp, PkCable, PkCableReuse,
  // refinement steps on the FP32 factor (natural layout): x in FP32 or as a
  // double-float pair, x + c out as a pair or in FP64
  Refine32to2, Refine32to64, Refine2to2, Refine2to64
};
struct UnitCall {
  UnitOp op = UnitOp::F64;
  const void* d = nullptr;
  const void* u = nullptr;
  const void* b = nullptr;
  void* x = nullptr;  // right-hand side in / solution out (compensated: the FP64 solution)
  const void* s = nullptr;
  const void* g = nullptr;
  double dt = 0.0, E = 0.0;
  int theta = 1;
  bool rhs_from_V = true;
  const void* rhs = nullptr;  // FP32 factor solve: right-hand side read instead of x (x then receives the solution)
  float* rw = nullptr;        // refinement: eliminated residual per compartment
  float* bcorr = nullptr;     // refinement: per branch the largest |correction| of the step
};

// Warp-task kernels (unit_kernels.cuh, unit_dispatch.cu).  prepare_unit_kernels
// sets their shared-memory limits and persistent grid sizes once per plan.
cudaError_t prepare_unit_kernels(DevPlan& P);
cudaError_t launch_unit_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s);
cudaError_t launch_unit_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s);
// FP32 solve of a new right-hand side with the factor launch_unit_solve_f32 left in the workspace.
cudaError_t launch_unit_resolve_f32(const DevPlan& P, const float* u, float* b, cudaStream_t s);
cudaError_t launch_unit_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                          cudaStream_t s);
cudaError_t launch_unit_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, bool rhs_from_V, cudaStream_t s);

cudaError_t launch_pk_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s);
cudaError_t launch_pk_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s);
cudaError_t launch_pk_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                        cudaStream_t s);
cudaError_t launch_pk_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V, double dt,
                            double E, int theta, bool rhs_from_V, cudaStream_t s);
// Passive-cable step with the factor the last full step left (natural or solver layout).
cudaError_t launch_unit_cable_reuse(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                                    double dt, double E, int theta, bool packed, cudaStream_t s);
// Natural <-> solver layout permutations (elem_bytes 4 or 8).
// coupling: gather through pk_edge (coupling arrays of a re-rooted plan) instead of pk_perm
cudaError_t launch_pack(const DevPlan& P, int elem_bytes, const void* natural, void* packed, cudaStream_t s,
                        bool coupling = false);
cudaError_t launch_unpack(const DevPlan& P, int elem_bytes, const void* packed, void* natural, cudaStream_t s);

// FP32 solve of rhs into x (x receives the solution; rhs is not modified).
cudaError_t launch_unit_solve_f32_rhs(const DevPlan& P, const float* d, const float* u, const float* rhs, float* x,
                                      cudaStream_t s);
// One refinement step on the FP32 factor (natural layout): x (FP32, or double-float pairs when x_pairs) in,
// x + c out (double-float pairs, or FP64 when final); per branch the largest |c| into bcorr.
cudaError_t launch_unit_refine_step(const DevPlan& P, const float* d, const float* u, const float* b, const void* x,
                                    bool x_pairs, void* xo, bool final, float* bcorr, cudaStream_t s);

// FP32 elimination + residual refinement on the warp-task kernels (refine_kernels.cu).
cudaError_t launch_unit_refine(const DevPlan& P, const float* d, const float* u, const float* b, double* x, int steps,
                               double* relres, cudaStream_t s);

// Adjoint gathers and loss terms (hines_kernels.cu).
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
