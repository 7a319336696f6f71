// Re-rooting of each cell at its centre (Section 6, balancing the dependency
// tree).  Internal to libhines.
//
// The compartments of a cell and their couplings form a tree.  Choosing another
// compartment as the root changes only the direction of the edges on the path
// between the old and the new root, so the system stays the same up to a
// renumbering; the renumbering below keeps every branch on consecutive indices
// and every parent before its children, which is what makes it a Hines matrix
// again.
//
//   centre     the compartment whose largest distance (in edges) to any other
//              compartment is smallest; when two compartments tie -- a tree has
//              one or two centres, the middle of every longest path -- the one
//              with the smaller old index.
//   numbering  branches in breadth-first order from the root branch; within a
//              branch proximal to distal.  The children of a compartment are
//              visited in ascending old index.
#include "reroot.h"

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <exception>
#include <new>
#include <thread>
#include <vector>

#include "../../include/hines.h"

namespace hines {
namespace {

// Breadth-first distances from src over the undirected tree (CSR adjacency);
// returns the farthest compartment (smallest index among the farthest).
int32_t bfs_far(const std::vector<int32_t>& adj_ptr, const std::vector<int32_t>& adj, int32_t n, int32_t src,
                std::vector<int32_t>& dist, std::vector<int32_t>& from, std::vector<int32_t>& queue) {
  std::fill(dist.begin(), dist.begin() + n, -1);
  queue.clear();
  queue.push_back(src);
  dist[src] = 0;
  from[src] = -1;
  int32_t far = src;
  for (size_t h = 0; h < queue.size(); ++h) {
    const int32_t x = queue[h];
    if (dist[x] > dist[far] || (dist[x] == dist[far] && x < far)) far = x;
    for (int32_t k = adj_ptr[x]; k < adj_ptr[x + 1]; ++k) {
      const int32_t y = adj[k];
      if (dist[y] < 0) {
        dist[y] = dist[x] + 1;
        from[y] = x;
        queue.push_back(y);
      }
    }
  }
  return far;
}

}  // namespace

int32_t tree_centre(int32_t n, const int32_t* parent) {
  if (n <= 2) return 0;
  std::vector<int32_t> adj_ptr(n + 1, 0), adj(2 * (size_t)(n - 1)), dist(n), from(n), queue;
  queue.reserve(n);
  for (int32_t i = 1; i < n; ++i) {
    ++adj_ptr[i + 1];
    ++adj_ptr[parent[i] + 1];
  }
  for (int32_t i = 0; i < n; ++i) adj_ptr[i + 1] += adj_ptr[i];
  std::vector<int32_t> fill(adj_ptr.begin(), adj_ptr.end() - 1);
  for (int32_t i = 1; i < n; ++i) {
    adj[fill[i]++] = parent[i];
    adj[fill[parent[i]]++] = i;
  }
  // a longest path runs between the farthest compartment a from any start and
  // the farthest b from a; its middle compartment(s) are the centre(s)
  const int32_t a = bfs_far(adj_ptr, adj, n, 0, dist, from, queue);
  const int32_t b = bfs_far(adj_ptr, adj, n, a, dist, from, queue);
  const int32_t len = dist[b];
  std::vector<int32_t> path;
  for (int32_t x = b; x >= 0; x = from[x]) path.push_back(x);  // path[k] at distance len - k from a
  const int32_t c0 = path[len / 2];
  const int32_t c1 = path[(len + 1) / 2];
  return std::min(c0, c1);
}

void reroot_cell(int32_t n, const int32_t* parent, int32_t root, int32_t* new_parent, int32_t* perm,
                 int32_t* edge) {
  if (n == 0) return;
  // children of each compartment in the re-rooted orientation, ascending old
  // index: the old children, plus the old parent for compartments on the path
  // from the new root to the old one, minus the compartment's new parent
  std::vector<int32_t> up(n, -1);  // new parent (old index)
  {
    // the path root -> old root reverses; everything else keeps its parent
    for (int32_t i = 0; i < n; ++i) up[i] = parent[i];
    int32_t x = root, prev = -1;
    while (x >= 0) {
      const int32_t nx = parent[x];
      up[x] = prev;
      prev = x;
      x = nx;
    }
  }
  std::vector<int32_t> cnt(n + 1, 0), kids;
  for (int32_t i = 0; i < n; ++i)
    if (up[i] >= 0) ++cnt[up[i] + 1];
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  kids.assign(cnt[n], 0);
  {
    std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
    for (int32_t i = 0; i < n; ++i)  // ascending i: each child list comes out sorted
      if (up[i] >= 0) kids[fill[up[i]]++] = i;
  }
  std::vector<int32_t> new_of(n, -1);
  std::vector<int32_t> starts;  // branch starts in breadth-first order (old indices)
  starts.reserve(n);
  starts.push_back(root);
  int32_t next = 0;
  for (size_t h = 0; h < starts.size(); ++h) {
    int32_t x = starts[h];
    for (;;) {
      new_of[x] = next;
      perm[next] = x;
      new_parent[next] = up[x] >= 0 ? new_of[up[x]] : -1;
      // the coupling of the edge (x, up[x]) is stored at whichever end is the
      // child in the old orientation
      edge[next] = up[x] < 0 ? -1 : (parent[x] == up[x] ? x : up[x]);
      ++next;
      const int32_t nk = cnt[x + 1] - cnt[x];
      if (nk == 1) {
        x = kids[cnt[x]];
        continue;
      }
      for (int32_t k = cnt[x]; k < cnt[x + 1]; ++k) starts.push_back(kids[k]);
      break;
    }
  }
}

int reroot_batch(int32_t n_cells, const int32_t* ncomp, const int32_t* parent, RerootMap& out) {
  if (n_cells < 0 || (n_cells > 0 && !ncomp)) return HINES_ERR_INVALID_ARG;
  int64_t n = 0;
  for (int32_t c = 0; c < n_cells; ++c) {
    if (ncomp[c] < 0) return HINES_ERR_INVALID_ARG;
    n += ncomp[c];
  }
  if (n > 0 && !parent) return HINES_ERR_INVALID_ARG;
  for (int64_t off = 0, c = 0; c < n_cells; off += ncomp[c], ++c) {
    const int32_t* p = parent + off;
    if (ncomp[c] > 0 && p[0] != -1) return HINES_ERR_NOT_HINES_ORDER;
    for (int32_t i = 1; i < ncomp[c]; ++i)
      if (p[i] < 0 || p[i] >= i) return HINES_ERR_NOT_HINES_ORDER;
  }
  out.parent.resize((size_t)n);
  out.perm.resize((size_t)n);
  out.edge.resize((size_t)n);
  out.centre.resize((size_t)n_cells);
  std::vector<int64_t> off((size_t)n_cells + 1, 0);
  for (int32_t c = 0; c < n_cells; ++c) off[(size_t)c + 1] = off[(size_t)c] + ncomp[c];
  // cells are independent: worker threads take cells in turn and write
  // disjoint ranges of the outputs
  std::atomic<int32_t> next_cell{0};
  std::atomic<bool> oom{false};
  auto work = [&]() {
    try {
      std::vector<int32_t> perm, edge;
      for (int32_t c = next_cell++; c < n_cells && !oom; c = next_cell++) {
        const int64_t o = off[(size_t)c];
        const int32_t m = ncomp[c];
        perm.resize((size_t)m);
        edge.resize((size_t)m);
        const int32_t root = m > 0 ? tree_centre(m, parent + o) : 0;
        out.centre[(size_t)c] = root;
        reroot_cell(m, parent + o, root, out.parent.data() + o, perm.data(), edge.data());
        for (int32_t j = 0; j < m; ++j) {
          out.perm[(size_t)(o + j)] = o + perm[(size_t)j];
          out.edge[(size_t)(o + j)] = edge[(size_t)j] >= 0 ? o + edge[(size_t)j] : -1;
        }
      }
    } catch (const std::bad_alloc&) {
      oom = true;
    }
  };
  const unsigned hw = std::thread::hardware_concurrency();
  const int64_t by_size = n / 65536 + 1;  // no thread for less than about 64K compartments
  const int n_threads = (int)std::min<int64_t>({(int64_t)(hw > 0 ? hw : 1), 32, by_size, (int64_t)n_cells});
  std::vector<std::thread> pool;
  try {  // fewer workers if threads cannot be had; this thread works too
    pool.reserve((size_t)n_threads);
    for (int t = 1; t < n_threads; ++t) pool.emplace_back(work);
  } catch (const std::exception&) {
  }
  work();
  for (auto& th : pool) th.join();
  if (oom) return HINES_ERR_OOM;
  return HINES_OK;
}

}  // namespace hines
