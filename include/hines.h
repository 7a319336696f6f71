/*
 * libhines -- batched direct solver for Hines matrices on one GB300 GPU.
 *
 * A Hines matrix (Huber, "Efficient Tree Solver for Hines Matrices on the
 * GPU", Sections 1-2) is the symmetric, strictly diagonally dominant matrix of
 * the implicit-Euler finite-volume discretisation of the cable equation on a
 * neuron's dendritic tree.  For one cell with N compartments:
 *
 *     A[i][i] = d[i],   A[i][p[i]] = A[p[i]][i] = u[i]   (i > 0),
 *
 * with the parent array p in Hines numbering: p[0] = -1 and 0 <= p[i] < i
 * (Section 2).  u[i] is the coupling of compartment i to its parent; u[0] is
 * never read.  The solve is the Hines algorithm (Section 2, Listing 2): one
 * leaf-to-root elimination and one root-to-leaf substitution, O(N).
 *
 * Layout ("natural layout").  A batch of n_cells cells is stored with the
 * cells concatenated in the order they were given to hines_plan_create; cell c
 * occupies [off[c], off[c+1]) (see hines_plan_layout) and its parent indices
 * are cell-local.  All per-compartment device arrays use this layout.
 *
 * Ownership.  Device arrays passed to the solve calls belong to the caller.
 * The plan owns its device metadata and a device workspace; it is created
 * on the device that is current at hines_plan_create and every call must be
 * made with that device current.
 *
 * Asynchrony.  Calls that take a stream only enqueue work on it and return;
 * argument errors are returned synchronously, before anything is enqueued.
 * Calls that share a plan must be ordered on one stream (they share the
 * plan's workspace).  Nothing is allocated inside the solve calls.
 *
 * Errors.  Every entry point returns a hines_status; hines_status_string
 * gives its text.  Device-side errors raise the plan's status word, read with
 * hines_plan_status.
 */
#ifndef HINES_H
#define HINES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *hines_stream_t;

/* Opaque plan handle; owned by the library, released by hines_plan_destroy. */
typedef struct hines_plan_s *hines_plan_t;

typedef enum {
  HINES_OK = 0,
  HINES_ERR_INVALID_ARG = 1,     /* null pointer, negative size, bad dtype or option, host-only plan */
  HINES_ERR_NOT_HINES_ORDER = 2, /* a cell violates p[0] = -1, 0 <= p[i] < i */
  HINES_ERR_OOM = 3,             /* host or device allocation failed (plan creation only) */
  HINES_ERR_CUDA = 4,            /* a CUDA runtime call failed */
  HINES_ERR_TIMEOUT = 5,         /* a bounded device wait ran out (status word) */
  HINES_WARN_REFINE = 6,         /* iterative refinement did not contract in some cell (status word) */
  HINES_ERR_DEVICE = 7           /* the plan was created on another device than the current one */
} hines_status;

/* Element types of the solve arrays. */
enum { HINES_F64 = 0, HINES_F32 = 1 };

/* Plan options; pass NULL for the defaults (all zero). */
typedef struct {
  int32_t host_only;       /* 1: build the host-side plan only (no CUDA calls); it can be
                              inspected with hines_plan_info / hines_plan_export but not solved */
  int32_t split_branches;  /* 1: split branches longer than their level's mean over the batch
                              (Section 6); 2: longer than their level's mean within their own
                              cell (a local variant, the per-block averages of the paper's
                              outlook after Section 7); 0: no split */
  int32_t pieces_per_lane; /* branch pieces a warp lane owns in a chunk: 0 or 1 (default) for
                              one (chunks of up to 32 pieces), 2 for two (chunks of up to 64;
                              the lane runs both chains at once, the compensated solve with
                              packed FP32-pair instructions); other values HINES_ERR_INVALID_ARG */
  int32_t sort_by_length;  /* 1: among ready branches equally far from their unit root, take the
                              longer first (Section 4, Fig. 4.1); 0: by cell and branch index,
                              so that a chunk of a breadth-first numbered cell reads contiguous runs */
  int32_t pack_compartments; /* warp tasks are filled with units up to this many compartments
                                (0: 24576, or total / 2048 for smaller batches, so that they still
                                give one task per warp); -1: Section 4's rule instead (a unit joins a task
                                while every level of the task holds at most a chunk of branches).
                                Applies to the subtrees of large cells, and to whole cells unless
                                pack_whole is set */
  int32_t reroot;          /* 1: re-root every cell at its centre (Section 6, balancing the
                              dependency tree; see hines_plan_export_reroot).  Such a plan
                              numbers compartments its own way and takes solver-layout
                              arrays only: the natural-layout entry points return
                              HINES_ERR_INVALID_ARG, and hines_pack / hines_pack_coupling /
                              hines_unpack map straight between the caller's numbering
                              and its solver layout */
  int32_t even_cuts;       /* 0: branches longer than 16 are cut from the proximal end at the
                              farthest multiple of 8 (natural layout) within 16 compartments, so
                              that pieces share no 32-byte sector; 1: into ceil(len / 16) pieces
                              of near-equal length, wherever their boundaries fall */
  int32_t pack_whole;      /* the same fill for tasks of whole cells (cells of at most 4096
                              compartments; the other size class is the subtrees of larger cells):
                              0 as pack_compartments, a count, or -1 for Section 4's rule */
  int32_t fp64_factor;     /* where the FP64 solves and cable steps keep their factor between the
                              elimination and the substitution: 1 at natural positions (the
                              reciprocal pivot in the workspace, the eliminated right-hand side in
                              place), 2 in the chunks' block order (both as one 16-byte pair,
                              staged back by bulk copies: faster on large batches, slower on
                              latency-bound small ones), 0 (default) 2 for batches of at least
                              50,331,648 compartments, else 1; other values HINES_ERR_INVALID_ARG.
                              Results are the same bit for bit */
  int32_t reserved[1];     /* must be zero */
} hines_plan_opts;

/* Plan summary. */
typedef struct {
  int32_t n_cells;
  int32_t max_levels;       /* deepest branch dependency tree (levels of Section 3) */
  int32_t n_tasks;          /* warp tasks: groups of cells solved together by one warp */
  int32_t reserved;
  int64_t n_unknowns;       /* total compartments */
  int64_t n_branches;       /* unbranched runs after optional splitting */
  int64_t workspace_bytes;  /* device workspace owned by the plan */
  int64_t metadata_bytes;   /* device metadata owned by the plan */
  int64_t n_packed;         /* length of a solver-layout array (n_unknowns plus block padding) */
} hines_plan_info_t;

/*
 * Build a plan for a batch of cells (host, once per morphology; Section 4:
 * the distribution is computed once during setup).
 *   n_cells  >= 0
 *   ncomp    host int32[n_cells], compartments per cell (each >= 0)
 *   parent   host int32[sum ncomp], cell-local parent arrays, concatenated
 *   opts     NULL or options
 * Validates every cell (HINES_ERR_NOT_HINES_ORDER names no cell; use a
 * per-cell check on the host to find it), decomposes each tree into branches
 * (maximal unbranched runs: compartment i starts a branch when i = 0,
 * p[i] != i-1, or p[i] has two or more children), optionally splits branches
 * longer than their level's mean (Section 6), cuts every branch longer than
 * 16 compartments into chained pieces (see even_cuts), assigns levels (number of
 * ancestor branches), cuts cells of more than 4096 compartments into a top
 * part and subtrees, packs these units into warp tasks (by size, or by
 * Section 4's greedy rule with the lanes of a warp), cuts every task into
 * chunks of at most 32 * pieces_per_lane branches by Hu's list schedule (a
 * branch joins a chunk once its children in the task are in earlier chunks,
 * deepest first; within a chunk, longest first), lays out the solver layout
 * (Section 5), and uploads the metadata and a workspace to the current
 * device.  Branches longer than 16 are cut from their proximal end into
 * pieces that each reach the farthest multiple of 8 (in the natural layout)
 * within 16 compartments, or the branch's end.  On success *out receives the
 * plan; on failure *out is NULL.
 */
hines_status hines_plan_create(hines_plan_t *out, int32_t n_cells, const int32_t *ncomp, const int32_t *parent,
                               const hines_plan_opts *opts);

/* Release a plan (NULL is a no-op).  Synchronises the plan's device. */
hines_status hines_plan_destroy(hines_plan_t plan);

/* Host int64[n_cells + 1]: offset of each cell in the natural layout. */
hines_status hines_plan_layout(hines_plan_t plan, int64_t *cell_offsets);

/* Fill *info with the plan's sizes. */
hines_status hines_plan_info(hines_plan_t plan, hines_plan_info_t *info);

/*
 * Copy the planner's branch decomposition to host arrays (all int64 so that
 * one call serves any batch size; every pointer may be NULL to skip it):
 *   first[nb], len[nb], parent_branch[nb], level[nb], cell[nb]  per branch,
 *        branches numbered cell by cell in order of their first compartment;
 *        first is the natural-layout index of the proximal compartment,
 *        parent_branch is -1 for a cell's root branch
 *   order[nb]  the processing order: cell by cell, level by level from 0,
 *        within a level by length descending then branch index
 * nb = info.n_branches.
 */
hines_status hines_plan_export(hines_plan_t plan, int64_t *first, int64_t *len, int64_t *parent_branch,
                               int64_t *level, int64_t *cell, int64_t *order);

/*
 * Copy the warp-task schedule to host arrays (NULL skips an array).  A cell of
 * at most 4096 compartments is one unit; a larger cell is cut into its top
 * part (the branches whose subtree holds more than 4096 compartments) and one
 * unit per subtree hanging below the top part.  Units of one kind are packed
 * into tasks, largest first (subtrees per cell), up to pack_compartments
 * compartments, or with the lane rule while every level (counted from each
 * unit's root branch) holds at most 32 branches (Section 4's rule).
 *   branch_task[nb]  task of each branch
 *   branch_kind[nb]  kind of the branch's unit: 0 whole cell, 1 subtree, 2 top part
 *   task_order[nb]   branches in processing order: tasks whole-cell, then
 *        subtree, then top kind; within a task the chunks of Hu's list schedule
 *        (at most 32 branches each; a branch follows all its children in the
 *        task; ready branches farthest from the unit root first, ties by
 *        length descending with sort_by_length, then cell, then branch index),
 *        listed root-side chunk first
 */
hines_status hines_plan_export_tasks(hines_plan_t plan, int64_t *branch_task, int64_t *branch_kind,
                                     int64_t *task_order);

/*
 * The solver layout (Section 5: the data of the branches a warp solves
 * together, interleaved so that each step reads one contiguous run).  Every
 * chunk of a warp task owns a block starting on a multiple of 4 slots.  With
 * one piece per lane, row r of the block holds the r-th compartment counted
 * from the distal end of every branch of the chunk longer than r, in chunk
 * order.  With two pieces per lane the chunk's branches pair up (2j, 2j + 1,
 * the first the longer), the two aligned at their proximal ends: row r holds
 * two slots for every pair whose longer branch is longer than r -- that
 * branch's r-th compartment from its distal end, and the compartment of the
 * shorter one at the same distance from the proximal end, or a padding slot.
 * A solver-layout array has info.n_packed elements (n_unknowns plus padding
 * slots) and must be 16-byte aligned.
 *
 * hines_plan_export_packed: host int64[n_packed], the natural-layout index
 * held by each slot, -1 for a padding slot (for a re-rooted plan: the index in
 * the caller's numbering).
 */
hines_status hines_plan_export_packed(hines_plan_t plan, int64_t *slot_natural);

/*
 * The re-rooting of a plan created with opts.reroot = 1 (Section 6: a new root
 * that minimises the depth of each cell's compartment tree, then a renumbering
 * that keeps every branch on consecutive indices).  Per cell the new root is
 * the centre of the tree: the compartment whose largest distance, in edges, to
 * any other compartment is smallest (the smaller index when two tie).  The
 * renumbering visits branches breadth first from the root branch, each branch
 * proximal to distal, the children of a compartment in ascending caller index.
 * Host arrays, global indices in the caller's natural layout:
 *   parent[n_unknowns]  int32, cell-local parent arrays of the re-rooted cells
 *                       (the morphology that hines_plan_export describes)
 *   perm[n_unknowns]    caller's index of each re-rooted compartment
 *   edge[n_unknowns]    caller's index at which the coupling between a
 *                       re-rooted compartment and its new parent is stored,
 *                       -1 at a root
 *   centre[n_cells]     int32, cell-local caller's index of each new root
 * HINES_ERR_INVALID_ARG for a plan that is not re-rooted.
 */
hines_status hines_plan_export_reroot(hines_plan_t plan, int32_t *parent, int64_t *perm, int64_t *edge,
                                      int32_t *centre);

/*
 * Permute one array between the layouts (device arrays; elem_bytes 4 or 8).
 * hines_pack writes every slot of packed[n_packed] (padding slots: zero) from
 * natural[n_unknowns]; hines_unpack writes natural[n_unknowns] from the
 * non-padding slots of packed.  Stream-ordered.
 *
 * hines_pack_coupling packs an array of couplings u (u[i] = A[i, p(i)], stored
 * at the child end of its edge).  For a plan that is not re-rooted it equals
 * hines_pack.  For a re-rooted plan the edges between a cell's old and new
 * root change direction, so each slot takes the coupling of the edge between
 * its compartment and that compartment's new parent (zero at a new root).
 */
hines_status hines_pack(hines_plan_t plan, int32_t elem_bytes, const void *natural, void *packed,
                        hines_stream_t stream);
hines_status hines_pack_coupling(hines_plan_t plan, int32_t elem_bytes, const void *natural, void *packed,
                                 hines_stream_t stream);
hines_status hines_unpack(hines_plan_t plan, int32_t elem_bytes, const void *packed, void *natural,
                          hines_stream_t stream);

/*
 * hines_solve and hines_solve_compensated on solver-layout arrays (each
 * n_packed elements, 16-byte aligned; padding slots are read and ignored,
 * and padding slots of the output are left unspecified).  The arithmetic is
 * the same; only where each value lives differs, so a batch kept in the
 * solver layout between solves (a simulation's state) needs no permutation.
 */
hines_status hines_solve_packed(hines_plan_t plan, int32_t dtype, const void *d, const void *u, void *b_inout,
                                hines_stream_t stream);
hines_status hines_solve_compensated_packed(hines_plan_t plan, const float *d, const float *u, const float *b,
                                            double *x_out, hines_stream_t stream);

/*
 * Solve A x = b for every cell (Section 2, Listing 2), in place.
 *   dtype   HINES_F64 (arithmetic in FP64) or HINES_F32 (arithmetic in FP32)
 *   d       device [n_unknowns] diagonal, not modified
 *   u       device [n_unknowns] parent couplings, not modified (u[first of cell] unused)
 *   b_inout device [n_unknowns] right-hand side on entry, solution x on return
 * Stream-ordered; uses the plan's workspace.
 */
hines_status hines_solve(hines_plan_t plan, int32_t dtype, const void *d, const void *u, void *b_inout,
                         hines_stream_t stream);

/*
 * Compensated mixed-precision solve: FP32 inputs, FP64 solution, and the
 * elimination and substitution of Listing 2 carried out in double-float
 * arithmetic (each quantity an unevaluated sum of two FP32 numbers, products
 * and sums made exact by error-free transformations), so that no FP64
 * instruction is needed.  Accuracy is that of a solve in about 48-bit
 * precision: relative error about cond(A) * 2^-50.  No paper counterpart.
 *   d, u, b   device float[n_unknowns], not modified
 *   x_out     device double[n_unknowns], the solution
 * Stream-ordered; uses the plan's workspace.
 */
hines_status hines_solve_compensated(hines_plan_t plan, const float *d, const float *u, const float *b,
                                     double *x_out, hines_stream_t stream);

/*
 * Mixed-precision solve: elimination in FP32 on FP32 inputs (the FP32
 * factor is kept in the plan's workspace), then refine_steps (0..4) steps of
 * iterative refinement.  A step forms the residual r = b - A x of the
 * current solution exactly enough for FP64 accuracy without FP64
 * instructions (products split by FMA into exact pairs, sums compensated),
 * eliminates it with the stored factor on the same staged chunk, then
 * substitutes the correction and adds it to x; between steps x is kept as a
 * double-float pair, the last step writes it in FP64.  A and b are the FP32
 * inputs taken exactly.  No paper counterpart (Section 2 gives the FP64
 * algorithm only).
 *   d, u, b      device float[n_unknowns], not modified
 *   x_out        device double[n_unknowns], the solution
 *   cell_relres  device double[n_cells] or NULL: per cell the scaled residual
 *                ||b - A x||_inf / (||A||_inf ||x||_inf) of the returned x, in FP64
 * If a refinement step grows the correction in some cell the plan's status
 * word receives HINES_WARN_REFINE.
 */
hines_status hines_solve_refine(hines_plan_t plan, const float *d, const float *u, const float *b, double *x_out,
                                int32_t refine_steps, double *cell_relres, hines_stream_t stream);

/*
 * One implicit-Euler step of a passive cable for every cell: the system of
 * Section 1 (finite volume, implicit Euler) is rebuilt from V and solved,
 * fused in one pass:
 *   d_i = s_i (1 + theta dt g_i) + sum_{j in N(i)} a_ij,   A[i][p[i]] = u_i = -a_i
 *   b_i = s_i V_i + s_i dt g_i (E - (1 - theta) V_i)
 * theta = 0 evaluates the membrane current at the old step as the paper's
 * equation does; theta = 1 takes the leak at the new step.  s_i = sigma_i
 * c_m,i / dt.  All arrays device double[n_unknowns]; V_inout holds V^k on
 * entry and V^{k+1} on return.
 */
hines_status hines_cable_step(hines_plan_t plan, const double *s, const double *g, const double *u, double *V_inout,
                              double dt, double E, int32_t theta, hines_stream_t stream);

/*
 * Solve with the passive-cable matrix of hines_cable_step (same d and u, any
 * right-hand side), in place: rhs_inout holds y on entry and A^{-1} y on
 * return.  The adjoint of a step is this solve, A being symmetric.
 */
hines_status hines_cable_solve(hines_plan_t plan, const double *s, const double *g, const double *u,
                               double *rhs_inout, double dt, int32_t theta, hines_stream_t stream);

/*
 * hines_cable_step and hines_cable_solve on solver-layout arrays (n_packed
 * elements each, 16-byte aligned; padding slots ignored), so that a rollout
 * keeps s, g, u and V in the solver layout from the first step to the last.
 * Same arithmetic, bit for bit, as the natural-layout calls.
 */
hines_status hines_cable_step_packed(hines_plan_t plan, const double *s, const double *g, const double *u,
                                     double *V_inout, double dt, double E, int32_t theta, hines_stream_t stream);
hines_status hines_cable_solve_packed(hines_plan_t plan, const double *s, const double *g, const double *u,
                                      double *rhs_inout, double dt, int32_t theta, hines_stream_t stream);

/*
 * A passive-cable step that re-uses the factor of the last full step.  With
 * s, g, u, dt and theta unchanged, the step's matrix is the same at every
 * step (only b depends on V), so after one hines_cable_step (or
 * hines_cable_step_packed) has left its factor -- the reciprocal eliminated
 * diagonal -- in the plan's workspace, a step only rebuilds b from V and
 * eliminates it: no reciprocal, about half the FP64 work.  The result equals
 * a full step bit for bit.  The caller guarantees that s, g, u, dt and theta
 * are those of the last full step on this plan, in the same layout, and that
 * no other call has used the plan's workspace since.  No paper counterpart
 * (the paper solves each step afresh; factor reuse is the constant-matrix
 * special case of the passive cable).
 *   solver_layout  0: natural-layout arrays (n_unknowns); 1: solver layout
 *                  (n_packed, 16-byte aligned)
 */
hines_status hines_cable_step_reuse(hines_plan_t plan, const double *s, const double *g, const double *u,
                                    double *V_inout, double dt, double E, int32_t theta, int32_t solver_layout,
                                    hines_stream_t stream);

/*
 * Adjoint gather for x = A^{-1} b with lambda = A^{-1} xbar (A symmetric, so
 * lambda is a second Hines solve):
 *   grad_d[i] = -lambda_i x_i
 *   grad_u[i] = -(lambda_i x_{p(i)} + lambda_{p(i)} x_i)   (i > 0; 0 at a cell's root)
 * All arrays device double[n_unknowns].  No paper counterpart.
 */
hines_status hines_grad_du(hines_plan_t plan, const double *lambda, const double *x, double *grad_d, double *grad_u,
                           hines_stream_t stream);

/*
 * Reverse step of a passive-cable rollout with loss
 * L = sum_cells sum_k (V^k_root - target_cell)^2, for the step V^{k-1} -> V^k
 * of hines_cable_step.  Given lambda = A^{-1} Vbar^k, accumulates
 *   grad_g[i] += lambda_i s_i dt (E - (1 - theta) V^{k-1}_i) - theta s_i dt lambda_i V^k_i
 *   grad_a[i] += -(lambda_i - lambda_{p(i)}) (V^k_i - V^k_{p(i)})     (i > 0)
 * and writes Vbar^{k-1} = lambda s (1 - (1 - theta) dt g), plus
 * 2 (V^{k-1}_root - target) at every cell root when add_loss_term != 0.
 *   target  device double[n_cells]; other arrays device double[n_unknowns].
 */
hines_status hines_cable_adjoint_step(hines_plan_t plan, const double *lambda, const double *V_k, const double *V_km1,
                                      const double *s, const double *g, const double *target, double dt, double E,
                                      int32_t theta, int32_t add_loss_term, double *grad_g, double *grad_a,
                                      double *vbar_out, hines_stream_t stream);

/*
 * Rollout loss term: loss_cells[c] += (V[root of c] - target[c])^2 for every
 * cell.  Device arrays (V: n_unknowns; target, loss_cells: n_cells).
 */
hines_status hines_cable_loss_accumulate(hines_plan_t plan, const double *V, const double *target,
                                         double *loss_cells, hines_stream_t stream);

/*
 * Loss seed: vbar[root of c] += 2 (V[root of c] - target[c]) for every cell.
 * Device arrays; used for the last step of a rollout.
 */
hines_status hines_cable_loss_seed(hines_plan_t plan, const double *V, const double *target, double *vbar,
                                   hines_stream_t stream);

/*
 * Allocation-free FP64 solve, for callers that may not allocate device
 * memory (a host runtime whose device allocator is fixed at start-up, a
 * memory pool that forbids new allocations, code that must not change the
 * process's device footprint).  Such callers cannot create a plan, because
 * plan creation allocates; this call needs none.  The paper has no
 * counterpart: it is a plain serial tree solve run by one GPU thread per
 * cell (each unbranched run eliminated as a chain, folded into its parent
 * row where a branch starts, then substituted from the root outwards), with
 * its scratch -- the eliminated diagonal and one validity word -- kept in a
 * fixed device array inside the library (16 MiB per GPU that loads the
 * library, held until the process exits).
 *   n_unknowns    total compartments, 0 .. 2,097,152 (larger: HINES_ERR_INVALID_ARG)
 *   n_cells       >= 0 (0: nothing to do, HINES_OK)
 *   cell_offsets  device int64[n_cells + 1], natural-layout offsets: off[0] = 0,
 *                 non-decreasing, off[n_cells] <= n_unknowns
 *   parent        device int32[n_unknowns], cell-local parent arrays
 *   d, u          device double[n_unknowns], not modified
 *   b_inout       device double[n_unknowns]: right-hand side in, solution out
 * Stream-ordered.  The checks of the device arrays run on the GPU, so they
 * cannot be returned: offsets that break the rule above leave every entry of
 * b_inout NaN and solve nothing; a cell whose parent array breaks Hines order
 * is left NaN while the other cells are solved.  The first call on a device
 * looks up the device address of the scratch array, so make it before any
 * stream capture.  All calls share the scratch array: calls whose work may
 * overlap on the GPU (unordered streams) race on it.
 */
hines_status hines_solve_f64_noalloc(int64_t n_unknowns, int32_t n_cells, const int64_t *cell_offsets,
                                     const int32_t *parent, const double *d, const double *u, double *b_inout,
                                     hines_stream_t stream);

/* Read (synchronously) and clear the plan's device status word. */
hines_status hines_plan_status(hines_plan_t plan, int32_t *status_out);

/*
 * Host pipeline: hines_solve_compensated from arrays in host memory, with
 * the host-device transfers overlapped with the solve.  No paper
 * counterpart.  Creation cuts the batch into `pieces` runs of consecutive
 * cells of about equal compartment counts (fewer where cells are few or
 * large), builds one plan per run (opts as for hines_plan_create; host_only
 * is rejected) and allocates the runs' device copies of d, u, b and x on the
 * current device (the pipeline owns them; hines_pipeline_destroy releases
 * everything, after its streams are idle).
 *   out       receives the pipeline, NULL on failure
 *   n_cells, ncomp, parent   as for hines_plan_create (host arrays)
 *   pieces    >= 1
 * Errors: those of hines_plan_create, HINES_ERR_OOM for the buffers,
 * HINES_ERR_CUDA for streams or events.
 */
typedef struct hines_pipeline_s *hines_pipeline_t;
hines_status hines_pipeline_create(hines_pipeline_t *out, int32_t n_cells, const int32_t *ncomp,
                                   const int32_t *parent, int32_t pieces, const hines_plan_opts *opts);

/* The number of runs the batch was cut into, and the batch's compartments. */
hines_status hines_pipeline_info(hines_pipeline_t pipeline, int32_t *pieces, int64_t *n_unknowns);

/*
 * The compensated solve of the whole batch from host arrays (natural layout
 * of the batch, as for hines_solve_compensated):
 *   d, u, b   host float[n_unknowns], not modified
 *   x_out     host double[n_unknowns], the solution
 * Per run: the three input copies on one internal stream, the device solve
 * on a second, the copy of x back on a third, joined by events; the work is
 * ordered after everything enqueued on `stream` before the call, and
 * `stream` waits for all of it (x_out is complete when the stream reaches
 * that point).  The transfers overlap only when the host arrays are
 * page-locked (cudaHostAlloc, cudaHostRegister, pinned torch tensors); with
 * pageable memory the copies still complete, without overlap.  Calls on one
 * pipeline must be ordered on one stream (they share its buffers).  Results
 * are those of hines_solve_compensated on each run's plan.
 * Errors: HINES_ERR_INVALID_ARG (null pipeline or array), HINES_ERR_DEVICE
 * (another device current than at creation), HINES_ERR_CUDA.
 */
hines_status hines_pipeline_solve_compensated(hines_pipeline_t pipeline, const float *d, const float *u,
                                              const float *b, double *x_out, hines_stream_t stream);

/* Read (synchronously) and clear the runs' plan status words; the largest. */
hines_status hines_pipeline_status(hines_pipeline_t pipeline, int32_t *status_out);

hines_status hines_pipeline_destroy(hines_pipeline_t pipeline);

/*
 * Check of the bounded device wait the solves use when they stage blocks with
 * bulk copies (no paper counterpart).  One CTA on the current device sets up
 * a shared-memory barrier that expects one arrival and polls it `polls`
 * times (1 .. 65536); with arrive = 0 nothing ever arrives (no copy is
 * issued), so the polls run out and the kernel records HINES_ERR_TIMEOUT in
 * *status_out, as a solve records it in its plan's status word, and returns;
 * with arrive = 1 the CTA makes the arrival itself and *status_out is
 * HINES_OK.  *elapsed_ns (if not NULL) receives the time the polls took.
 * Synchronous; allocates and frees a few bytes of device memory.  Nothing
 * faults or hangs, and the context stays usable afterwards.
 */
hines_status hines_check_bounded_wait(int32_t polls, int32_t arrive, int32_t *status_out, int64_t *elapsed_ns);

/* Static text of a status code. */
const char *hines_status_string(int32_t status);

#ifdef __cplusplus
}
#endif

#endif /* HINES_H */
