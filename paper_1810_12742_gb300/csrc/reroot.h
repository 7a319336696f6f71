// Re-rooting of a cell at its centre (Section 6); internal to libhines.
#pragma once
#include <cstdint>
#include <vector>

namespace hines {

// Centre of the tree given by a valid cell-local parent array (p[0] = -1,
// 0 <= p[i] < i): the compartment of smallest eccentricity, the smaller index
// of two.
int32_t tree_centre(int32_t n, const int32_t* parent);

// Renumbering of the cell rooted at `root` (old index).  Outputs, per new index
// j: new_parent[j] (-1 at the root), perm[j] = old index of compartment j, and
// edge[j] = old index at which the coupling of the edge between j and its new
// parent is stored (the child end in the old orientation; -1 at the root).
void reroot_cell(int32_t n, const int32_t* parent, int32_t root, int32_t* new_parent, int32_t* perm,
                 int32_t* edge);

// Every cell of a batch re-rooted at its centre; indices are global (natural
// layout, cells concatenated).
struct RerootMap {
  std::vector<int32_t> parent;  // [n] cell-local parent arrays of the re-rooted cells
  std::vector<int64_t> perm;    // [n] caller's index of each re-rooted compartment
  std::vector<int64_t> edge;    // [n] caller's index holding the coupling to the new parent, -1 at a root
  std::vector<int32_t> centre;  // [n_cells] cell-local caller's index of the new root
};

// Validates like plan creation (hines_status codes) and fills `out`.
int reroot_batch(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, RerootMap& out);

}  // namespace hines
