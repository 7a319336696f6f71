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
#include <queue>

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

// One level of Section 6's splitting: every branch on `level` longer than
// the level's mean length (mean in FP64, strict >) is cut after ceil(len/2)
// compartments; the distal piece becomes a child branch one level deeper and
// takes over the children.  The mean is taken over the whole batch (global),
// or, with `local`, over each cell's own branches on the level (the local
// heuristic of the paper's outlook: averages per block of work instead of
// over all trees).  Returns true if some cell has the level.
bool split_level(std::vector<std::vector<Br>>& cells, int32_t level, bool local) {
  double sum = 0.0;
  int64_t cnt = 0;
  for (auto& bs : cells)
    for (auto& b : bs)
      if (b.level == level) {
        sum += (double)b.len;
        cnt++;
      }
  if (cnt == 0) return false;
  const double global_mean = sum / (double)cnt;
  std::vector<Br> nb;
  std::vector<int32_t> remap_prox, remap_dist;
  for (auto& bs : cells) {
    double mean = global_mean;
    if (local) {
      double csum = 0.0;
      int64_t ccnt = 0;
      for (auto& b : bs)
        if (b.level == level) {
          csum += (double)b.len;
          ccnt++;
        }
      if (ccnt == 0) continue;
      mean = csum / (double)ccnt;
    }
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

// Cut every branch longer than `cap` into chained pieces of at most `cap`
// compartments whose boundaries fall on multiples of kCutAlign natural
// indices (`base` is the cell's offset in the natural layout): from the
// proximal end, each piece reaches the farthest such boundary within `cap`
// compartments, or the branch's end.  A piece then never shares a 32-byte
// sector of an FP32 array with the next piece of its branch, so the chunks
// that load them (at different times) do not fetch a sector twice.  The
// system is unchanged; only the schedule is.
// With `even`, the pieces are instead ceil(len / cap) of near-equal length
// (the first len % pieces, from the proximal end, one longer), wherever their
// boundaries fall.
void cap_branches(std::vector<Br>& bs, int32_t cap, int64_t base, bool even) {
  bool any = false;
  for (auto& b : bs) any |= b.len > cap;
  if (!any) return;
  std::vector<Br> nb;
  std::vector<int32_t> last_piece(bs.size());
  for (size_t j = 0; j < bs.size(); ++j) {
    const Br b = bs[j];
    int32_t parent = b.parent < 0 ? -1 : last_piece[(size_t)b.parent];
    const int64_t end = b.first + b.len;
    const int32_t pieces = (b.len + cap - 1) / cap, plen = b.len / pieces, rem = b.len % pieces;
    int64_t start = b.first;
    for (int32_t k = 0; start < end; ++k) {
      int64_t stop = std::min<int64_t>(end, start + cap);
      if (even) {
        stop = start + plen + (k < rem ? 1 : 0);
      } else if (stop < end) {
        const int64_t down = stop - (base + stop) % kCutAlign;  // aligned boundary at or below stop
        if (down > start) stop = down;
      }
      Br q;
      q.first = start;
      q.len = (int32_t)(stop - start);
      q.parent = parent;
      q.level = parent < 0 ? 0 : nb[(size_t)parent].level + 1;
      parent = (int32_t)nb.size();
      nb.push_back(q);
      start = stop;
    }
    last_piece[j] = parent;
  }
  bs.swap(nb);
}

}  // namespace

int build_host_plan(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, int split_branches,
                    int sort_by_length, int pack_compartments, int pieces_per_lane, int even_cuts, int pack_whole,
                    HostPlan& P) {
  if (n_cells < 0 || (n_cells > 0 && !ncomp)) return HINES_ERR_INVALID_ARG;
  if (pieces_per_lane != 1 && pieces_per_lane != 2) return HINES_ERR_INVALID_ARG;
  P = HostPlan();
  P.n_cells = n_cells;
  P.per_lane = pieces_per_lane;
  const int32_t width = kLanes * pieces_per_lane;  // pieces per chunk
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
  if (split_branches < 0 || split_branches > 2) return HINES_ERR_INVALID_ARG;
  if (split_branches)
    for (int32_t level = 0; split_level(cells, level, split_branches == 2); ++level) {
    }
  for (int32_t c = 0; c < n_cells; ++c)
    cap_branches(cells[(size_t)c], kBranchCap, P.cell_off[(size_t)c], even_cuts != 0);

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

  // units: a cell of at most kUnitMax compartments is one unit; a larger cell
  // is cut into its top part (the branches whose subtree holds more than
  // kUnitMax compartments; connected, contains the root) and one subtree unit
  // per remaining branch whose parent is in the top part
  std::vector<int64_t> sub((size_t)nb, 0);
  for (int64_t b = nb - 1; b >= 0; --b) {
    sub[(size_t)b] += P.br_len[(size_t)b];
    if (P.br_parent[(size_t)b] >= 0) sub[(size_t)P.br_parent[(size_t)b]] += sub[(size_t)b];
  }
  struct Unit {
    int32_t cell, root, kind;
    int64_t size;
    int32_t nlvl;
  };
  std::vector<Unit> units;
  std::vector<int32_t> unit_of((size_t)nb, -1);
  P.br_kind.assign((size_t)nb, 0);
  for (int32_t c = 0; c < n_cells; ++c) {
    const int64_t lo = P.cell_br_off[(size_t)c], hi = P.cell_br_off[(size_t)c + 1];
    if (lo == hi) continue;
    const bool split = ncomp[c] > kUnitMax;
    int32_t top_unit = -1;
    for (int64_t b = lo; b < hi; ++b) {  // parents before children
      const int32_t pb = P.br_parent[(size_t)b];
      int32_t u;
      if (!split) {
        if (b == lo) units.push_back({c, (int32_t)b, 0, 0, 0});
        u = (int32_t)units.size() - 1;
      } else if (sub[(size_t)b] > kUnitMax) {
        if (top_unit < 0) {
          units.push_back({c, (int32_t)b, 2, 0, 0});
          top_unit = (int32_t)units.size() - 1;
        }
        u = top_unit;
      } else if (pb < 0 || P.br_kind[(size_t)pb] == 2) {
        units.push_back({c, (int32_t)b, 1, 0, 0});
        u = (int32_t)units.size() - 1;
      } else {
        u = unit_of[(size_t)pb];
      }
      unit_of[(size_t)b] = u;
      P.br_kind[(size_t)b] = units[(size_t)u].kind;
    }
  }
  P.br_rlevel.assign((size_t)nb, 0);
  std::vector<std::vector<int32_t>> unit_br(units.size());
  for (int64_t b = 0; b < nb; ++b) {
    const int32_t u = unit_of[(size_t)b];
    if (u < 0) continue;
    const int32_t rl = P.br_level[(size_t)b] - P.br_level[(size_t)units[(size_t)u].root];
    P.br_rlevel[(size_t)b] = rl;
    units[(size_t)u].size += P.br_len[(size_t)b];
    units[(size_t)u].nlvl = std::max(units[(size_t)u].nlvl, rl + 1);
    unit_br[(size_t)u].push_back((int32_t)b);
  }

  // tasks: per kind, units largest first (ties by cell, then root branch),
  // packed next-fit up to pack_compartments compartments per task (levels of
  // more than 32 branches become several chunks), or, with the lane rule,
  // while every relative level holds at most kLanes branches (Section 4's
  // rule with the 32 lanes of a warp)
  // The fill is chosen per size class: whole cells (pack_whole, or as the
  // subtrees when 0) and the subtrees of large cells (pack_compartments).
  // default fill: kTaskCompartments, but small enough that a small batch
  // still gives kMinTasks tasks (one per warp of a full GPU) where its units allow
  const int64_t pack_default =
      std::min<int64_t>(kTaskCompartments, std::max<int64_t>(1, (P.n_unknowns + kMinTasks - 1) / kMinTasks));
  auto fill_of = [&](int32_t opt) { return opt > 0 ? (int64_t)opt : pack_default; };
  const int32_t whole_opt = pack_whole != 0 ? pack_whole : pack_compartments;
  P.n_tasks = 0;
  P.task_kind.clear();
  P.task_nlvl.clear();
  P.task_lvl_off.clear();
  P.tlvl_ptr.clear();
  P.torder.clear();
  P.torder.reserve((size_t)nb);
  P.br_task.assign((size_t)nb, -1);
  std::vector<int64_t> task_size;
  for (int32_t kind = 0; kind < 3; ++kind) {
    const int32_t opt = kind == 0 ? whole_opt : pack_compartments;
    const bool lane_rule = opt < 0;
    const int64_t pack_max = fill_of(opt);
    std::vector<int32_t> us;
    for (size_t u = 0; u < units.size(); ++u)
      if (units[u].kind == kind) us.push_back((int32_t)u);
    // subtrees are packed per cell (a task finishes at most one cell)
    std::stable_sort(us.begin(), us.end(), [&](int32_t x, int32_t y) {
      if (kind == 1 && units[(size_t)x].cell != units[(size_t)y].cell)
        return units[(size_t)x].cell < units[(size_t)y].cell;
      if (units[(size_t)x].size != units[(size_t)y].size) return units[(size_t)x].size > units[(size_t)y].size;
      if (units[(size_t)x].cell != units[(size_t)y].cell) return units[(size_t)x].cell < units[(size_t)y].cell;
      return units[(size_t)x].root < units[(size_t)y].root;
    });
    std::vector<std::vector<int32_t>> groups;
    std::vector<int32_t> cnt, ucnt;
    int64_t gsize = 0;
    for (int32_t u : us) {
      ucnt.assign((size_t)units[(size_t)u].nlvl, 0);
      for (int32_t b : unit_br[(size_t)u]) ucnt[(size_t)P.br_rlevel[(size_t)b]]++;
      bool fits = !groups.empty() && kind != 2;  // top parts are never packed
      if (fits && kind == 1 && units[(size_t)groups.back()[0]].cell != units[(size_t)u].cell) fits = false;
      if (fits && lane_rule) {
        for (size_t l = 0; l < ucnt.size(); ++l)
          if ((l < cnt.size() ? cnt[l] : 0) + ucnt[l] > width) {
            fits = false;
            break;
          }
      } else if (fits) {
        fits = gsize + units[(size_t)u].size <= pack_max;
      }
      if (!fits) {
        groups.emplace_back();
        cnt.clear();
        gsize = 0;
      }
      gsize += units[(size_t)u].size;
      groups.back().push_back(u);
      if (cnt.size() < ucnt.size()) cnt.resize(ucnt.size(), 0);
      for (size_t l = 0; l < ucnt.size(); ++l) cnt[l] += ucnt[l];
    }
    std::vector<int32_t> ids;
    std::vector<int32_t> pend((size_t)nb, 0);
    for (const auto& g : groups) {
      const int32_t t = P.n_tasks++;
      int32_t nl = 0;
      int64_t size = 0;
      ids.clear();
      for (int32_t u : g) {
        nl = std::max(nl, units[(size_t)u].nlvl);
        size += units[(size_t)u].size;
        ids.insert(ids.end(), unit_br[(size_t)u].begin(), unit_br[(size_t)u].end());
      }
      // chunks by Hu's list schedule for in-forests: a branch is ready once
      // all its children in the task sit in earlier chunks; each chunk takes
      // the (at most 32 per lane) ready branches farthest from their unit's
      // root, ties by length (with sort_by_length), cell, branch.  This needs
      // the fewest chunks for the task's dependency forest; levels of the
      // kernel are these chunks, stored root-side first.  Within a chunk the
      // branches are then ordered by length, longest first (stable), so that
      // the lanes' pieces shrink together and the rows of the solver layout
      // are prefixes of the chunk.
      for (int32_t b : ids) P.br_task[(size_t)b] = t;
      auto later = [&](int32_t x, int32_t y) {  // priority-queue order: true if x goes after y
        if (P.br_rlevel[(size_t)x] != P.br_rlevel[(size_t)y]) return P.br_rlevel[(size_t)x] < P.br_rlevel[(size_t)y];
        if (sort_by_length && P.br_len[(size_t)x] != P.br_len[(size_t)y])
          return P.br_len[(size_t)x] < P.br_len[(size_t)y];
        if (P.br_cell[(size_t)x] != P.br_cell[(size_t)y]) return P.br_cell[(size_t)x] > P.br_cell[(size_t)y];
        return x > y;
      };
      std::priority_queue<int32_t, std::vector<int32_t>, decltype(later)> ready(later);
      for (int32_t b : ids) {
        int32_t k = 0;
        for (int32_t q = P.child_ptr[(size_t)b]; q < P.child_ptr[(size_t)b + 1]; ++q)
          if (P.br_task[(size_t)P.child[(size_t)q]] == t) ++k;
        pend[(size_t)b] = k;
        if (k == 0) ready.push(b);
      }
      std::vector<std::vector<int32_t>> chunks;
      std::vector<int32_t> done;
      while (!ready.empty()) {
        chunks.emplace_back();
        while (!ready.empty() && (int)chunks.back().size() < width) {
          chunks.back().push_back(ready.top());
          ready.pop();
        }
        std::stable_sort(chunks.back().begin(), chunks.back().end(),
                         [&](int32_t x, int32_t y) { return P.br_len[(size_t)x] > P.br_len[(size_t)y]; });
        for (int32_t b : chunks.back()) {
          const int32_t pb = P.br_parent[(size_t)b];
          if (pb >= 0 && P.br_task[(size_t)pb] == t && --pend[(size_t)pb] == 0) done.push_back(pb);
        }
        for (int32_t b : done) ready.push(b);
        done.clear();
      }
      nl = (int32_t)chunks.size();
      ids.clear();
      P.task_kind.push_back(kind);
      P.task_nlvl.push_back(nl);
      P.task_lvl_off.push_back((int64_t)P.tlvl_ptr.size());
      const int32_t base = (int32_t)P.torder.size();
      for (int32_t l = nl - 1; l >= 0; --l) {
        P.tlvl_ptr.push_back(base + (int32_t)ids.size());
        ids.insert(ids.end(), chunks[(size_t)l].begin(), chunks[(size_t)l].end());
      }
      P.tlvl_ptr.push_back(base + (int32_t)ids.size());
      P.torder.insert(P.torder.end(), ids.begin(), ids.end());
      task_size.push_back(size);
    }
  }
  // phases: A = whole-cell tasks (both visits) and subtree tasks
  // (elimination), heaviest first; a cell's top part runs in phase A too,
  // taken over by the warp that finishes the cell's last subtree (it has no
  // list entry); C = subtree tasks (substitution), heaviest first.
  // Entry = 4 * task + visits (0: both, 1: elimination, 2: substitution).
  {
    std::vector<int32_t> a, c;
    for (int32_t t = 0; t < P.n_tasks; ++t) {
      if (P.task_kind[(size_t)t] == 0) a.push_back(4 * t + 0);
      if (P.task_kind[(size_t)t] == 1) {
        a.push_back(4 * t + 1);
        c.push_back(4 * t + 2);
      }
    }
    auto work = [&](int32_t e) { return task_size[(size_t)(e >> 2)] * ((e & 3) == 0 ? 2 : 1); };
    auto heavy_first = [&](std::vector<int32_t>& v) {
      std::stable_sort(v.begin(), v.end(), [&](int32_t x, int32_t y) { return work(x) > work(y); });
    };
    heavy_first(a);
    heavy_first(c);
    P.phase_off = {0, (int32_t)a.size(), (int32_t)a.size(), (int32_t)(a.size() + c.size())};
    P.phase_entry = a;
    P.phase_entry.insert(P.phase_entry.end(), c.begin(), c.end());
  }
  // top-part hand-over: per cell its top task and number of subtree units;
  // per subtree task the cells of its units with their counts
  P.cell_top_task.assign((size_t)n_cells, -1);
  P.cell_nsub.assign((size_t)n_cells, 0);
  for (const auto& u : units)
    if (u.kind == 1) P.cell_nsub[(size_t)u.cell]++;
  P.counter_init.assign(4, 0);
  P.counter_init.insert(P.counter_init.end(), P.cell_nsub.begin(), P.cell_nsub.end());
  for (int64_t b = 0; b < nb; ++b)
    if (P.br_kind[(size_t)b] == 2) P.cell_top_task[(size_t)P.br_cell[(size_t)b]] = P.br_task[(size_t)b];
  // per task the cell its subtree units belong to (subtree tasks hold one
  // cell's units only) and their number; -1 / 0 for other tasks
  P.task_sub.assign(2 * (size_t)P.n_tasks, 0);
  for (int32_t t = 0; t < P.n_tasks; ++t) P.task_sub[2 * (size_t)t] = -1;
  for (const auto& u : units) {
    if (u.kind != 1) continue;
    const size_t t = (size_t)P.br_task[(size_t)u.root];
    P.task_sub[2 * t] = u.cell;
    P.task_sub[2 * t + 1]++;
  }

  P.tpos.assign((size_t)nb, -1);
  for (size_t k = 0; k < P.torder.size(); ++k) P.tpos[(size_t)P.torder[k]] = (int32_t)k;
  P.tchild_ptr.assign((size_t)nb + 1, 0);
  P.tchild.resize(P.child.size());
  for (size_t k = 0; k < P.torder.size(); ++k) {
    const int32_t b = P.torder[k];
    P.tchild_ptr[k + 1] = P.tchild_ptr[k] + (P.child_ptr[(size_t)b + 1] - P.child_ptr[(size_t)b]);
    int32_t w = P.tchild_ptr[k];
    for (int32_t c = P.child_ptr[(size_t)b]; c < P.child_ptr[(size_t)b + 1]; ++c) P.tchild[(size_t)w++] = P.tpos[(size_t)P.child[(size_t)c]];
  }
  // solver layout: blocks in task order, levels ascending, chunks of the
  // chunk width; row layout as described in plan.h
  {
    const int32_t per = pieces_per_lane;
    P.pk_blk.assign((size_t)nb, 0);
    P.pk_pcomp.assign((size_t)nb, -1);
    std::vector<int64_t> distal((size_t)nb, -1);  // solver-layout index of each position's distal compartment
    std::vector<int64_t> slots;
    int64_t off = 0;
    for (int32_t t = 0; t < P.n_tasks; ++t) {
      const int32_t* lp = P.tlvl_ptr.data() + P.task_lvl_off[(size_t)t];
      for (int32_t l = 0; l < P.task_nlvl[(size_t)t]; ++l) {
        for (int32_t c0 = lp[l]; c0 < lp[l + 1]; c0 += width) {
          const int32_t c1 = std::min(c0 + width, lp[l + 1]);
          const int32_t n = c1 - c0, lanes = (n + per - 1) / per;
          auto len_at = [&](int32_t i) { return i < n ? P.br_len[(size_t)P.torder[(size_t)(c0 + i)]] : 0; };
          int64_t e = 0;
          for (int32_t r = 0; r < kBranchCap; ++r) {
            for (int32_t j = 0; j < lanes; ++j) {
              const int32_t rows = len_at(per * j);  // the lane's rows: its longer (first) piece
              if (rows <= r) continue;
              for (int32_t h = 0; h < per; ++h) {
                const int32_t i = per * j + h, len = len_at(i);
                // distance from the proximal end of the piece at row r (pieces
                // of a pair are aligned at their proximal ends)
                const int32_t t_prox = rows - 1 - r;
                int64_t nat = -1;
                if (i < n && t_prox < len) {
                  nat = P.br_first[(size_t)P.torder[(size_t)(c0 + i)]] + t_prox;
                  if (t_prox == len - 1) distal[(size_t)(c0 + i)] = off + e;
                }
                slots.push_back(nat);
                ++e;
              }
            }
          }
          for (int32_t q = c0; q < c1; ++q) P.pk_blk[(size_t)q] = off;
          const int64_t padded = (e + kPackAlign - 1) / kPackAlign * kPackAlign;
          for (int64_t k = e; k < padded; ++k) slots.push_back(-1);
          off += padded;
        }
      }
    }
    P.n_packed = off;
    P.pk_perm.swap(slots);
    for (int32_t q = 0; q < (int32_t)nb; ++q) {
      const int32_t pb = P.br_parent[(size_t)P.torder[(size_t)q]];
      if (pb >= 0) P.pk_pcomp[(size_t)q] = distal[(size_t)P.tpos[(size_t)pb]];
    }
  }
  return HINES_OK;
}

}  // namespace hines
