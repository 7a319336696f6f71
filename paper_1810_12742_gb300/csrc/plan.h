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

  // units and warp tasks.  A unit is a whole cell of at most kUnitMax
  // compartments, or, for a larger cell, its top part (kind 2) or one of the
  // subtrees hanging below it (kind 1).  Units of one kind are packed into warp
  // tasks (Section 4's rule with 32 lanes: every level, counted from the
  // unit's root, holds at most 32 branches), so each level of a task is one
  // chunk of at most 32 branches, one per lane.
  std::vector<int32_t> br_kind;      // [nb] kind of the branch's unit (0 whole, 1 subtree, 2 top)
  std::vector<int32_t> br_rlevel;    // [nb] level relative to the unit's root branch
  std::vector<int32_t> br_task;      // [nb] task of the branch
  int32_t n_tasks = 0;
  std::vector<int32_t> task_kind;    // [n_tasks]
  std::vector<int32_t> task_nlvl;    // [n_tasks]
  std::vector<int64_t> task_lvl_off; // [n_tasks] index of the task's first entry in tlvl_ptr
  std::vector<int32_t> tlvl_ptr;     // per task nlvl + 1 positions into torder
  std::vector<int32_t> torder;       // [nb] per task, relative level ascending, within a level
                                     // cell then branch id (length desc first if sorted)
  std::vector<int32_t> tpos;         // [nb] position of each branch in torder
  std::vector<int32_t> tchild_ptr;   // [nb + 1] children of the branch at each position, CSR
  std::vector<int32_t> tchild;       // child positions (by first compartment descending)
  // launch phases: entries 4 * task + visits (0 both, 1 elimination, 2 substitution)
  std::vector<int32_t> phase_off;    // [4]
  std::vector<int32_t> phase_entry;
  // top-part hand-over
  std::vector<int32_t> cell_top_task;  // [n_cells] task of the cell's top part, -1 if not cut
  std::vector<int32_t> cell_nsub;      // [n_cells] subtree units of the cell
  std::vector<int32_t> counter_init;   // [4 + n_cells] work counters (0) then cell_nsub
  std::vector<int32_t> task_sub;       // [2 * n_tasks] (cell, subtree units) of a subtree task, else (-1, 0)

  // Pieces per lane: a chunk holds at most 32 * per_lane pieces; lane j of a
  // warp owns the chunk's pieces per_lane * j .. per_lane * j + per_lane - 1.
  // Within a chunk the pieces are sorted by length, longest first.
  int32_t per_lane = 1;

  // Solver layout (Section 5's interleaving, per chunk): each chunk owns a
  // block.  One piece per lane: row r of the block holds the r-th compartment
  // from the distal end of every piece of the chunk longer than r, in chunk
  // order.  Two pieces per lane: the pieces pair up as the lanes own them
  // (2j, 2j + 1; the first is the longer); a pair spans as many rows as its
  // longer piece has compartments, the two pieces aligned at their proximal
  // ends, and row r holds two slots for every pair longer than r: the longer
  // piece's r-th compartment from its distal end, and the shorter piece's
  // compartment at the same distance from the proximal end (a padding slot
  // where the shorter piece has none).  So a warp reads a row as one
  // contiguous run, each lane its two values as one 8-byte word.  Blocks start
  // on multiples of kPackAlign compartments.
  int64_t n_packed = 0;
  std::vector<int64_t> pk_blk;    // [nb] block offset of the chunk of each position
  std::vector<int64_t> pk_pcomp;  // [nb] solver-layout index of the parent branch's distal compartment, -1 at a root
  std::vector<int64_t> pk_perm;   // [n_packed] natural index held by each solver-layout slot, -1 for padding
};

constexpr int kLanes = 32;       // lanes of a warp; a chunk holds 32 * per_lane pieces
constexpr int kBranchCap = 16;   // maximum compartments per branch after capping
constexpr int kWarpsPerCta = 2;  // warps per CTA of the task kernels (each warp runs its own task)
constexpr int64_t kCutAlign = 8; // pieces of a cut branch start on multiples of 8 natural indices (32-byte sectors)
constexpr int64_t kUnitMax = 4096;  // largest unit (compartments); larger cells are cut
constexpr int64_t kPackAlign = 4;   // solver-layout blocks start on multiples of 4 compartments
constexpr int64_t kTaskCompartments = 24576;  // default fill of a warp task
constexpr int64_t kMinTasks = 2048;           // smaller tasks for batches below kMinTasks * kTaskCompartments

// Return codes follow hines_status.
int build_host_plan(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, int split_branches,
                    int sort_by_length, int pack_compartments, int pieces_per_lane, int even_cuts,
                    int pack_whole, HostPlan& out);

}  // namespace hines
