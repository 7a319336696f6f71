// Host-side plan of the batched Hines solver (internal to libhines).
#pragma once
#include <cstdint>
#include <vector>

namespace hines {

// Branch decomposition and schedule of a batch of cells.  Branch ids are
// global: the branches of cell c are [cell_br_off[c], cell_br_off[c+1]),
// numbered by their first compartment.
struct HostPlan {
  int32_t n_cells = 0;
  int64_t n_unknowns = 0;
  int32_t max_levels = 0;
  std::vector<int64_t> cell_off;     // [n_cells + 1] natural-layout offsets
  std::vector<int64_t> cell_br_off;  // [n_cells + 1]
  std::vector<int64_t> br_first;     // natural-layout index of the proximal compartment
  std::vector<int32_t> br_len;       // compartments
  std::vector<int32_t> br_parent;    // global parent branch id, -1 for a root branch
  std::vector<int32_t> br_level;     // ancestor branches
  std::vector<int32_t> br_cell;      // owning cell
  std::vector<int32_t> child_ptr;    // [nb + 1] CSR of children per branch
  std::vector<int32_t> child;        // children, by first compartment descending
  std::vector<int32_t> order;        // per cell, level 0..L-1, length desc then id
  std::vector<int32_t> cell_nlvl;    // [n_cells]
  std::vector<int64_t> cell_lvl_off; // [n_cells] index of the cell's first entry in lvl_ptr
  std::vector<int32_t> lvl_ptr;      // per cell nlvl + 1 indices into order
  std::vector<int32_t> task_cell;    // cells in processing order (cost descending)

  // warp tasks (Section 4 packing with 32 lanes): groups of cells processed
  // by one warp level by level, largest task first
  int32_t n_tasks = 0;
  std::vector<int32_t> cell_task;    // [n_cells] task of each cell
  std::vector<int32_t> task_nlvl;    // [n_tasks]
  std::vector<int64_t> task_lvl_off; // [n_tasks] index of the task's first entry in tlvl_ptr
  std::vector<int32_t> tlvl_ptr;     // per task nlvl + 1 indices into torder
  std::vector<int32_t> torder;       // [nb] per task, level ascending, within a level
                                     // length desc, then cell, then branch id
  std::vector<int32_t> tpos;         // [nb] position of each branch in torder
  std::vector<int32_t> tchild_ptr;   // [nb + 1] children of the branch at each position, CSR
  std::vector<int32_t> tchild;       // child positions (by first compartment descending)
};

constexpr int kLanes = 32;       // branches per chunk (one per lane)
constexpr int kBranchCap = 32;   // maximum compartments per branch after capping

// Return codes follow hines_status.
int build_host_plan(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, int split_branches,
                    HostPlan& out);

}  // namespace hines
