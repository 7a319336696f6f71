// Host planner of the batched Hines solver.
//
// Section 2: with breadth-first branch numbering every cell's matrix is a
// Hines matrix, eliminated leaves-to-root and substituted root-to-leaves.
// Section 3: the branches form a dependency tree; all branches of one level
// can be processed in parallel once the deeper level is done.
// Section 4: the schedule is computed once at setup; the branches of a level
// are sorted by size to reduce divergence (Fig. 4.1).
// Section 5: only one parent index per branch is needed; inside a branch the
// parent of compartment i is i - 1.
// Section 6: optional splitting of branches longer than their level's mean.
#include "plan.h"

#include <algorithm>
#include <numeric>

#include "../../include/hines.h"

namespace hines {
namespace {

struct Br {
  int64_t first;  // cell-local index of the proximal compartment
  int32_t len;
  int32_t parent;  // cell-local branch id, -1 for the root branch
  int32_t level;
};

// Decompose one validated cell into branches (maximal unbranched runs).
// Compartment i starts a branch iff i == 0, p[i] != i - 1, or p[i] has two
// or more children; such a parent is always the last compartment of its run.
void decompose(int64_t n, const int32_t* p, std::vector<int32_t>& nchild, std::vector<int32_t>& branch_of,
               std::vector<Br>& out) {
  out.clear();
  if (n == 0) return;
  nchild.assign((size_t)n, 0);
  branch_of.resize((size_t)n);
  for (int64_t i = 1; i < n; ++i) nchild[(size_t)p[i]]++;
  for (int64_t i = 0; i < n; ++i) {
    bool start = (i == 0) || (p[i] != i - 1) || (nchild[(size_t)p[i]] >= 2);
    if (start) {
      Br b;
      b.first = i;
      b.len = 1;
      b.parent = (i == 0) ? -1 : branch_of[(size_t)p[i]];
      b.level = (i == 0) ? 0 : out[(size_t)b.parent].level + 1;
      out.push_back(b);
    } else {
      out.back().len++;
    }
    branch_of[(size_t)i] = (int32_t)out.size() - 1;
  }
}

// One level of Section 6's splitting over the whole batch: every branch on
// `level` longer than the level's mean length (mean in FP64, strict >) is cut
// after ceil(len/2) compartments; the distal piece becomes a child branch one
// level deeper and takes over the children.  Returns true if the level exists.
bool split_level(std::vector<std::vector<Br>>& cells, int32_t level) {
  double sum = 0.0;
  int64_t cnt = 0;
  for (auto& bs : cells)
    for (auto& b : bs)
      if (b.level == level) {
        sum += (double)b.len;
        cnt++;
      }
  if (cnt == 0) return false;
  const double mean = sum / (double)cnt;
  std::vector<Br> nb;
  std::vector<int32_t> remap_prox, remap_dist;
  for (auto& bs : cells) {
    bool any = false;
    for (auto& b : bs)
      if (b.level == level && (double)b.len > mean && b.len >= 2) any = true;
    if (!any) continue;
    nb.clear();
    remap_prox.assign(bs.size(), -1);
    remap_dist.assign(bs.size(), -1);
    for (size_t j = 0; j < bs.size(); ++j) {
      const Br& b = bs[j];
      remap_prox[j] = (int32_t)nb.size();
      if (b.level == level && (double)b.len > mean && b.len >= 2) {
        int32_t k = (b.len + 1) / 2;
        Br prox = b, dist = b;
        prox.len = k;
        dist.first = b.first + k;
        dist.len = b.len - k;
        dist.parent = -2 - (int32_t)j;  // resolved below: child of the proximal piece
        nb.push_back(prox);
        remap_dist[j] = (int32_t)nb.size();
        nb.push_back(dist);
      } else {
        remap_dist[j] = remap_prox[j];
        nb.push_back(b);
      }
    }
    for (auto& b : nb) {
      if (b.parent <= -2)
        b.parent = remap_prox[(size_t)(-2 - b.parent)];
      else if (b.parent >= 0)
        b.parent = remap_dist[(size_t)b.parent];  // old children hang below the distal piece
    }
    for (auto& b : nb) b.level = (b.parent < 0) ? 0 : nb[(size_t)b.parent].level + 1;
    bs.swap(nb);
  }
  return true;
}

}  // namespace

int build_host_plan(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, int split_branches,
                    HostPlan& P) {
  if (n_cells < 0 || (n_cells > 0 && !ncomp)) return HINES_ERR_INVALID_ARG;
  P = HostPlan();
  P.n_cells = n_cells;
  P.cell_off.assign((size_t)n_cells + 1, 0);
  for (int32_t c = 0; c < n_cells; ++c) {
    if (ncomp[c] < 0) return HINES_ERR_INVALID_ARG;
    P.cell_off[(size_t)c + 1] = P.cell_off[(size_t)c] + ncomp[c];
  }
  P.n_unknowns = P.cell_off[(size_t)n_cells];
  if (P.n_unknowns > 0 && !parent) return HINES_ERR_INVALID_ARG;
  if (P.n_unknowns > (int64_t)INT32_MAX * 8) return HINES_ERR_INVALID_ARG;

  // validate and decompose
  std::vector<std::vector<Br>> cells((size_t)n_cells);
  std::vector<int32_t> nchild, branch_of;
  for (int32_t c = 0; c < n_cells; ++c) {
    const int64_t n = ncomp[c];
    const int32_t* p = parent + P.cell_off[(size_t)c];
    if (n > 0) {
      if (p[0] != -1) return HINES_ERR_NOT_HINES_ORDER;
      for (int64_t i = 1; i < n; ++i)
        if (p[i] < 0 || (int64_t)p[i] >= i) return HINES_ERR_NOT_HINES_ORDER;
    }
    decompose(n, p, nchild, branch_of, cells[(size_t)c]);
  }
  if (split_branches)
    for (int32_t level = 0; split_level(cells, level); ++level) {
    }

  // flatten to global branch ids (cell by cell, by first compartment)
  P.cell_br_off.assign((size_t)n_cells + 1, 0);
  for (int32_t c = 0; c < n_cells; ++c)
    P.cell_br_off[(size_t)c + 1] = P.cell_br_off[(size_t)c] + (int64_t)cells[(size_t)c].size();
  const int64_t nb = P.cell_br_off[(size_t)n_cells];
  if (nb > INT32_MAX - 1) return HINES_ERR_INVALID_ARG;
  P.br_first.resize((size_t)nb);
  P.br_len.resize((size_t)nb);
  P.br_parent.resize((size_t)nb);
  P.br_level.resize((size_t)nb);
  P.br_cell.resize((size_t)nb);
  P.cell_nlvl.assign((size_t)n_cells, 0);
  for (int32_t c = 0; c < n_cells; ++c) {
    const int64_t base = P.cell_br_off[(size_t)c];
    int32_t nl = 0;
    for (size_t j = 0; j < cells[(size_t)c].size(); ++j) {
      const Br& b = cells[(size_t)c][j];
      const size_t g = (size_t)(base + (int64_t)j);
      P.br_first[g] = P.cell_off[(size_t)c] + b.first;
      P.br_len[g] = b.len;
      P.br_parent[g] = b.parent < 0 ? -1 : (int32_t)(base + b.parent);
      P.br_level[g] = b.level;
      P.br_cell[g] = c;
      nl = std::max(nl, b.level + 1);
    }
    P.cell_nlvl[(size_t)c] = nl;
    P.max_levels = std::max(P.max_levels, nl);
  }

  // children, by first compartment descending (the order in which a serial
  // leaves-to-root sweep over decreasing compartment index meets them)
  P.child_ptr.assign((size_t)nb + 1, 0);
  for (int64_t b = 0; b < nb; ++b)
    if (P.br_parent[(size_t)b] >= 0) P.child_ptr[(size_t)P.br_parent[(size_t)b] + 1]++;
  for (int64_t b = 0; b < nb; ++b) P.child_ptr[(size_t)b + 1] += P.child_ptr[(size_t)b];
  P.child.resize((size_t)P.child_ptr[(size_t)nb]);
  {
    std::vector<int32_t> fill(P.child_ptr.begin(), P.child_ptr.end() - 1);
    for (int64_t b = nb - 1; b >= 0; --b) {  // descending ids = descending first compartment
      int32_t pb = P.br_parent[(size_t)b];
      if (pb >= 0) P.child[(size_t)fill[(size_t)pb]++] = (int32_t)b;
    }
  }

  // level-major order per cell: level ascending, length descending, id ascending
  P.order.resize((size_t)nb);
  P.cell_lvl_off.resize((size_t)n_cells);
  int64_t lvl_total = 0;
  for (int32_t c = 0; c < n_cells; ++c) {
    P.cell_lvl_off[(size_t)c] = lvl_total;
    lvl_total += P.cell_nlvl[(size_t)c] + 1;
  }
  P.lvl_ptr.assign((size_t)lvl_total, 0);
  for (int32_t c = 0; c < n_cells; ++c) {
    const int64_t lo = P.cell_br_off[(size_t)c], hi = P.cell_br_off[(size_t)c + 1];
    for (int64_t b = lo; b < hi; ++b) P.order[(size_t)b] = (int32_t)b;
    std::stable_sort(P.order.begin() + lo, P.order.begin() + hi, [&](int32_t x, int32_t y) {
      if (P.br_level[(size_t)x] != P.br_level[(size_t)y]) return P.br_level[(size_t)x] < P.br_level[(size_t)y];
      if (P.br_len[(size_t)x] != P.br_len[(size_t)y]) return P.br_len[(size_t)x] > P.br_len[(size_t)y];
      return x < y;
    });
    const int64_t lb = P.cell_lvl_off[(size_t)c];
    const int32_t nl = P.cell_nlvl[(size_t)c];
    int64_t k = lo;
    for (int32_t l = 0; l <= nl; ++l) {
      while (k < hi && P.br_level[(size_t)P.order[(size_t)k]] < l) ++k;
      P.lvl_ptr[(size_t)(lb + l)] = (int32_t)k;
    }
  }

  // processing order of cells: most compartments first, ties by index
  P.task_cell.resize((size_t)n_cells);
  std::iota(P.task_cell.begin(), P.task_cell.end(), 0);
  std::stable_sort(P.task_cell.begin(), P.task_cell.end(),
                   [&](int32_t x, int32_t y) { return ncomp[x] > ncomp[y]; });
  return HINES_OK;
}

}  // namespace hines
