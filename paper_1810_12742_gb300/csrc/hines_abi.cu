// C-ABI of libhines: plan lifetime, argument checks and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hines.h"
#include "kernels.h"
#include "plan.h"
#include "reroot.h"

struct hines_plan_s {
  hines::HostPlan host;
  hines::DevPlan dev;
  int device = -1;
  bool host_only = false;
  bool rerooted = false;         // cells re-rooted at their centres (Section 6)
  hines::RerootMap rr;           // re-rooted numbering -> caller's numbering
  std::vector<int64_t> pk_edge;  // [n_packed] caller's index of each slot's coupling (re-rooted plans)
  void* meta = nullptr;
  void* work = nullptr;
  int64_t meta_bytes = 0;
  int64_t work_bytes = 0;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Copy the host plan's arrays into one device allocation and point the
// device view at them; allocate the workspace.
hines_status upload(hines_plan_t p) {
  const hines::HostPlan& H = p->host;
  struct Item {
    const void* src;
    size_t bytes;
    const void** dst;
  };
  hines::DevPlan& D = p->dev;
  // per-branch metadata in task order
  std::vector<hines::BrMetaT> tmeta(H.torder.size());
  for (size_t k = 0; k < H.torder.size(); ++k) {
    const int32_t b = H.torder[k];
    hines::BrMetaT& m = tmeta[k];
    m.first = H.br_first[(size_t)b];
    m.len = (int16_t)H.br_len[(size_t)b];
    const int32_t pb = H.br_parent[(size_t)b];
    m.pcomp = pb < 0 ? -1 : H.br_first[(size_t)pb] + H.br_len[(size_t)pb] - 1;
    m.ppos = pb < 0 ? -1 : H.tpos[(size_t)pb];
    const int32_t cb = H.tchild_ptr[k], ce = H.tchild_ptr[k + 1];
    m.nchild = (int16_t)(ce - cb);
    int32_t lo = INT32_MAX, hi = -1;
    m.xtask = 0;
    for (int32_t q = cb; q < ce; ++q) {
      lo = std::min(lo, H.tchild[(size_t)q]);
      hi = std::max(hi, H.tchild[(size_t)q]);
      if (H.br_task[(size_t)H.torder[(size_t)H.tchild[(size_t)q]]] != H.br_task[(size_t)b]) m.xtask = 1;
    }
    m.ccontig = (int16_t)(ce > cb && hi - lo + 1 == ce - cb);
    m.cpos = m.ccontig ? lo : cb;
  }
  // solver layout: per position (block offset, parent's solver-layout index)
  std::vector<int64_t> pkm(2 * H.torder.size());
  for (size_t k = 0; k < H.torder.size(); ++k) {
    pkm[2 * k] = H.pk_blk[k];
    pkm[2 * k + 1] = H.pk_pcomp[k];
  }
  std::vector<Item> items = {
      {tmeta.data(), tmeta.size() * sizeof(hines::BrMetaT), (const void**)&D.tmeta},
      {pkm.data(), pkm.size() * 8, (const void**)&D.pk_meta},
      {H.pk_perm.data(), H.pk_perm.size() * 8, (const void**)&D.pk_perm},
      {p->pk_edge.data(), p->pk_edge.size() * 8, (const void**)&D.pk_edge},
      {H.task_nlvl.data(), H.task_nlvl.size() * 4, (const void**)&D.task_nlvl},
      {H.task_lvl_off.data(), H.task_lvl_off.size() * 8, (const void**)&D.task_lvl_off},
      {H.tlvl_ptr.data(), H.tlvl_ptr.size() * 4, (const void**)&D.tlvl_ptr},
      {H.tchild.data(), H.tchild.size() * 4, (const void**)&D.tchild},
      {H.phase_entry.data(), H.phase_entry.size() * 4, (const void**)&D.phase_entry},
      {H.cell_top_task.data(), H.cell_top_task.size() * 4, (const void**)&D.cell_top_task},
      {H.counter_init.data(), H.counter_init.size() * 4, (const void**)&D.counter_init},
      {H.task_sub.data(), H.task_sub.size() * 4, (const void**)&D.task_sub},
      {H.torder.data(), H.torder.size() * 4, (const void**)&D.pos_branch},
      {H.cell_off.data(), H.cell_off.size() * 8, (const void**)&D.cell_off},
      {H.br_first.data(), H.br_first.size() * 8, (const void**)&D.br_first},
      {H.br_len.data(), H.br_len.size() * 4, (const void**)&D.br_len},
      {H.br_parent.data(), H.br_parent.size() * 4, (const void**)&D.br_parent},
      {H.br_cell.data(), H.br_cell.size() * 4, (const void**)&D.br_cell},
      {H.cell_br_off.data(), H.cell_br_off.size() * 8, (const void**)&D.cell_br_off},
      {H.child_ptr.data(), H.child_ptr.size() * 4, (const void**)&D.child_ptr},
      {H.child.data(), H.child.size() * 4, (const void**)&D.child},
  };
  size_t total = 256;  // status word first
  for (auto& it : items) total += align256(it.bytes > 0 ? it.bytes : 1);
  if (cudaMalloc(&p->meta, total) != cudaSuccess) {
    cudaGetLastError();
    p->meta = nullptr;
    return HINES_ERR_OOM;
  }
  p->meta_bytes = (int64_t)total;
  char* base = static_cast<char*>(p->meta);
  if (cudaMemset(base, 0, 256) != cudaSuccess) return HINES_ERR_CUDA;
  D.status = reinterpret_cast<int32_t*>(base);
  size_t off = 256;
  for (auto& it : items) {
    if (it.bytes > 0 && cudaMemcpy(base + off, it.src, it.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
      return HINES_ERR_CUDA;
    *it.dst = base + off;
    off += align256(it.bytes > 0 ? it.bytes : 1);
  }
  if (!p->rerooted) D.pk_edge = D.pk_perm;  // a coupling sits at its child compartment
  const size_t n = (size_t)H.n_unknowns, nb = H.br_first.size(), nc = (size_t)H.n_cells;
  // the factor is indexed by natural or solver-layout position
  const size_t fac_b = align256(std::max(n, (size_t)H.n_packed) * 8 + 8), cd_b = align256(nb * 16 + 16),
               cb_b = align256(nb * 32 + 32),
               xl_b = align256(nb * 8 + 8), red_b = align256(nc * 8 + 8),
               cnt_b = align256((nc + 4) * 4), rw_b = align256(std::max(n, (size_t)H.n_packed) * 4 + 4),
               ff4_b = align256((size_t)H.n_packed * 16 + 16);
  const size_t wtotal = fac_b + cd_b + cb_b + xl_b + red_b + cnt_b + rw_b + ff4_b;
  if (cudaMalloc(&p->work, wtotal) != cudaSuccess) {
    cudaGetLastError();
    p->work = nullptr;
    return HINES_ERR_OOM;
  }
  p->work_bytes = (int64_t)wtotal;
  char* w = static_cast<char*>(p->work);
  D.fac = w;
  w += fac_b;
  D.cd = w;
  w += cd_b;
  D.cb = w;
  w += cb_b;
  D.xlast = w;
  w += xl_b;
  D.red = w;
  w += red_b;
  D.counter = reinterpret_cast<int32_t*>(w);
  D.cell_pending = D.counter + 4;
  w += cnt_b;
  D.rw = w;
  w += rw_b;
  D.ff4 = w;
  D.n_wtasks = H.n_tasks;
  D.per_lane = H.per_lane;
  D.n_packed = H.n_packed;
  for (int k = 0; k < 4; ++k) D.phase_off[k] = H.phase_off.empty() ? 0 : H.phase_off[(size_t)k];
  D.n_cells = H.n_cells;
  D.n_unknowns = H.n_unknowns;
  D.n_branches = (int64_t)nb;
  if (hines::prepare_unit_kernels(D) != cudaSuccess) return HINES_ERR_CUDA;
  return HINES_OK;
}

hines_status check_plan(hines_plan_t p) {
  if (!p || p->host_only) return HINES_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HINES_ERR_CUDA;
  if (dev != p->device) return HINES_ERR_DEVICE;
  return HINES_OK;
}

// Entry points that take natural-layout arrays: a re-rooted plan numbers the
// compartments differently from the caller, so it accepts the solver layout only.
hines_status check_natural(hines_plan_t p) {
  const hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  return p->rerooted ? HINES_ERR_INVALID_ARG : HINES_OK;
}

hines_status launched(cudaError_t e) { return e == cudaSuccess ? HINES_OK : HINES_ERR_CUDA; }

bool need(hines_plan_t p, const void* a) { return a != nullptr || p->host.n_unknowns == 0; }

}  // namespace

extern "C" {

hines_status hines_plan_create(hines_plan_t* out, int32_t n_cells, const int32_t* ncomp, const int32_t* parent,
                               const hines_plan_opts* opts) {
  if (!out) return HINES_ERR_INVALID_ARG;
  *out = nullptr;
  hines_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.reserved[0] != 0) return HINES_ERR_INVALID_ARG;
  if (o.pack_whole < -1) return HINES_ERR_INVALID_ARG;
  if (o.even_cuts != 0 && o.even_cuts != 1) return HINES_ERR_INVALID_ARG;
  if (o.pack_compartments < -1) return HINES_ERR_INVALID_ARG;
  if (o.pieces_per_lane == 0) o.pieces_per_lane = 1;
  if (o.pieces_per_lane != 1 && o.pieces_per_lane != 2) return HINES_ERR_INVALID_ARG;
  if (o.fp64_factor < 0 || o.fp64_factor > 2) return HINES_ERR_INVALID_ARG;
  hines_plan_t p = new (std::nothrow) hines_plan_s();
  if (!p) return HINES_ERR_OOM;
  int rc;
  try {
    p->rerooted = o.reroot != 0;
    rc = p->rerooted ? hines::reroot_batch(n_cells, ncomp, parent, p->rr) : HINES_OK;
    if (rc == HINES_OK)
      rc = hines::build_host_plan(n_cells, ncomp, p->rerooted ? p->rr.parent.data() : parent, o.split_branches,
                                  o.sort_by_length, o.pack_compartments, o.pieces_per_lane, o.even_cuts,
                                  o.pack_whole, p->host);
    if (rc == HINES_OK && p->rerooted) {
      // the solver layout maps straight to the caller's numbering: node arrays
      // through the renumbering, couplings through the edge map
      std::vector<int64_t>& perm = p->host.pk_perm;
      p->pk_edge.assign(perm.size(), -1);
      for (size_t k = 0; k < perm.size(); ++k) {
        if (perm[k] < 0) continue;
        p->pk_edge[k] = p->rr.edge[(size_t)perm[k]];
        perm[k] = p->rr.perm[(size_t)perm[k]];
      }
    }
  } catch (const std::bad_alloc&) {
    rc = HINES_ERR_OOM;
  }
  if (rc != HINES_OK) {
    delete p;
    return (hines_status)rc;
  }
  p->host_only = o.host_only != 0;
  // FP64 factors in block order where the batch fills default-size tasks
  // (the planner's small-batch bound), or as asked
  p->dev.fp64_blocks = o.fp64_factor == 2 || (o.fp64_factor == 0 && p->host.n_unknowns >=
                                                                       hines::kMinTasks * hines::kTaskCompartments);
  if (!p->host_only) {
    if (cudaGetDevice(&p->device) != cudaSuccess) {
      cudaGetLastError();
      delete p;
      return HINES_ERR_CUDA;
    }
    hines_status st = upload(p);
    if (st != HINES_OK) {
      hines_plan_destroy(p);
      return st;
    }
  }
  *out = p;
  return HINES_OK;
}

hines_status hines_plan_destroy(hines_plan_t p) {
  if (!p) return HINES_OK;
  hines_status st = HINES_OK;
  if (p->meta || p->work) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    if (cudaDeviceSynchronize() != cudaSuccess) st = HINES_ERR_CUDA;
    if (p->meta) cudaFree(p->meta);
    if (p->work) cudaFree(p->work);
    if (cur != p->device && cur >= 0) cudaSetDevice(cur);
  }
  delete p;
  return st;
}

hines_status hines_plan_layout(hines_plan_t p, int64_t* cell_offsets) {
  if (!p || !cell_offsets) return HINES_ERR_INVALID_ARG;
  std::memcpy(cell_offsets, p->host.cell_off.data(), p->host.cell_off.size() * sizeof(int64_t));
  return HINES_OK;
}

hines_status hines_plan_info(hines_plan_t p, hines_plan_info_t* info) {
  if (!p || !info) return HINES_ERR_INVALID_ARG;
  info->n_cells = p->host.n_cells;
  info->max_levels = p->host.max_levels;
  info->n_tasks = p->host.n_tasks;
  info->reserved = 0;
  info->n_unknowns = p->host.n_unknowns;
  info->n_branches = (int64_t)p->host.br_first.size();
  info->workspace_bytes = p->work_bytes;
  info->metadata_bytes = p->meta_bytes;
  info->n_packed = p->host.n_packed;
  return HINES_OK;
}

hines_status hines_plan_export(hines_plan_t p, int64_t* first, int64_t* len, int64_t* parent_branch, int64_t* level,
                               int64_t* cell, int64_t* order) {
  if (!p) return HINES_ERR_INVALID_ARG;
  const hines::HostPlan& H = p->host;
  const size_t nb = H.br_first.size();
  for (size_t b = 0; b < nb; ++b) {
    if (first) first[b] = H.br_first[b];
    if (len) len[b] = H.br_len[b];
    if (parent_branch) parent_branch[b] = H.br_parent[b];
    if (level) level[b] = H.br_level[b];
    if (cell) cell[b] = H.br_cell[b];
    if (order) order[b] = H.order[b];
  }
  return HINES_OK;
}

hines_status hines_plan_export_tasks(hines_plan_t p, int64_t* branch_task, int64_t* branch_kind, int64_t* task_order) {
  if (!p) return HINES_ERR_INVALID_ARG;
  const hines::HostPlan& H = p->host;
  for (size_t b = 0; b < H.br_task.size(); ++b) {
    if (branch_task) branch_task[b] = H.br_task[b];
    if (branch_kind) branch_kind[b] = H.br_kind[b];
  }
  if (task_order)
    for (size_t b = 0; b < H.torder.size(); ++b) task_order[b] = H.torder[b];
  return HINES_OK;
}

hines_status hines_solve(hines_plan_t p, int32_t dtype, const void* d, const void* u, void* b_inout,
                         hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, d) || !need(p, u) || !need(p, b_inout)) return HINES_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == HINES_F64)
    return launched(hines::launch_unit_solve_f64(p->dev, (const double*)d, (const double*)u, (double*)b_inout, s));
  if (dtype == HINES_F32)
    return launched(hines::launch_unit_solve_f32(p->dev, (const float*)d, (const float*)u, (float*)b_inout, s));
  return HINES_ERR_INVALID_ARG;
}

hines_status hines_solve_compensated(hines_plan_t p, const float* d, const float* u, const float* b, double* x_out,
                                     hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, d) || !need(p, u) || !need(p, b) || !need(p, x_out)) return HINES_ERR_INVALID_ARG;
  return launched(
      hines::launch_unit_solve_compensated(p->dev, d, u, b, x_out, reinterpret_cast<cudaStream_t>(stream)));
}

// Solver-layout arrays: n_packed elements, 16-byte aligned (blocks are copied
// with 16-byte transfers).
bool need_pk(hines_plan_t p, const void* a) {
  if (p->host.n_packed == 0) return true;
  return a != nullptr && (reinterpret_cast<uintptr_t>(a) & 15u) == 0;
}

hines_status hines_plan_export_packed(hines_plan_t p, int64_t* slot_natural) {
  if (!p || (!slot_natural && p->host.n_packed > 0)) return HINES_ERR_INVALID_ARG;
  for (size_t k = 0; k < p->host.pk_perm.size(); ++k) slot_natural[k] = p->host.pk_perm[k];
  return HINES_OK;
}

hines_status hines_pack(hines_plan_t p, int32_t elem_bytes, const void* natural, void* packed, hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if ((elem_bytes != 4 && elem_bytes != 8) || !need(p, natural) || !need_pk(p, packed)) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_pack(p->dev, elem_bytes, natural, packed, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_pack_coupling(hines_plan_t p, int32_t elem_bytes, const void* natural, void* packed,
                                 hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if ((elem_bytes != 4 && elem_bytes != 8) || !need(p, natural) || !need_pk(p, packed)) return HINES_ERR_INVALID_ARG;
  return launched(
      hines::launch_pack(p->dev, elem_bytes, natural, packed, reinterpret_cast<cudaStream_t>(stream), true));
}

hines_status hines_plan_export_reroot(hines_plan_t p, int32_t* parent, int64_t* perm, int64_t* edge,
                                      int32_t* centre) {
  if (!p || !p->rerooted) return HINES_ERR_INVALID_ARG;
  const size_t n = p->rr.perm.size(), nc = p->rr.centre.size();
  if (n > 0 && (!parent || !perm || !edge)) return HINES_ERR_INVALID_ARG;
  if (nc > 0 && !centre) return HINES_ERR_INVALID_ARG;
  std::memcpy(parent, p->rr.parent.data(), n * sizeof(int32_t));
  std::memcpy(perm, p->rr.perm.data(), n * sizeof(int64_t));
  std::memcpy(edge, p->rr.edge.data(), n * sizeof(int64_t));
  std::memcpy(centre, p->rr.centre.data(), nc * sizeof(int32_t));
  return HINES_OK;
}

hines_status hines_unpack(hines_plan_t p, int32_t elem_bytes, const void* packed, void* natural,
                          hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if ((elem_bytes != 4 && elem_bytes != 8) || !need(p, natural) || !need_pk(p, packed)) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_unpack(p->dev, elem_bytes, packed, natural, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_solve_packed(hines_plan_t p, int32_t dtype, const void* d, const void* u, void* b_inout,
                                hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (!need_pk(p, d) || !need_pk(p, u) || !need_pk(p, b_inout)) return HINES_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == HINES_F64)
    return launched(hines::launch_pk_solve_f64(p->dev, (const double*)d, (const double*)u, (double*)b_inout, s));
  if (dtype == HINES_F32)
    return launched(hines::launch_pk_solve_f32(p->dev, (const float*)d, (const float*)u, (float*)b_inout, s));
  return HINES_ERR_INVALID_ARG;
}

hines_status hines_solve_compensated_packed(hines_plan_t p, const float* d, const float* u, const float* b,
                                            double* x_out, hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (!need_pk(p, d) || !need_pk(p, u) || !need_pk(p, b) || !need_pk(p, x_out)) return HINES_ERR_INVALID_ARG;
  return launched(
      hines::launch_pk_solve_compensated(p->dev, d, u, b, x_out, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_solve_refine(hines_plan_t p, const float* d, const float* u, const float* b, double* x_out,
                                int32_t refine_steps, double* cell_relres, hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, d) || !need(p, u) || !need(p, b) || !need(p, x_out)) return HINES_ERR_INVALID_ARG;
  if (refine_steps < 0 || refine_steps > 4) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_unit_refine(p->dev, d, u, b, x_out, refine_steps, cell_relres,
                                            reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_step(hines_plan_t p, const double* s, const double* g, const double* u, double* V_inout,
                              double dt, double E, int32_t theta, hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, s) || !need(p, g) || !need(p, u) || !need(p, V_inout)) return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_unit_cable(p->dev, s, g, u, V_inout, dt, E, theta, true,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_solve(hines_plan_t p, const double* s, const double* g, const double* u, double* rhs_inout,
                               double dt, int32_t theta, hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, s) || !need(p, g) || !need(p, u) || !need(p, rhs_inout)) return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_unit_cable(p->dev, s, g, u, rhs_inout, dt, 0.0, theta, false,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_step_packed(hines_plan_t p, const double* s, const double* g, const double* u,
                                     double* V_inout, double dt, double E, int32_t theta, hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (!need_pk(p, s) || !need_pk(p, g) || !need_pk(p, u) || !need_pk(p, V_inout)) return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_pk_cable(p->dev, s, g, u, V_inout, dt, E, theta, true,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_solve_packed(hines_plan_t p, const double* s, const double* g, const double* u,
                                      double* rhs_inout, double dt, int32_t theta, hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (!need_pk(p, s) || !need_pk(p, g) || !need_pk(p, u) || !need_pk(p, rhs_inout)) return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_pk_cable(p->dev, s, g, u, rhs_inout, dt, 0.0, theta, false,
                                         reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_step_reuse(hines_plan_t p, const double* s, const double* g, const double* u,
                                    double* V_inout, double dt, double E, int32_t theta, int32_t solver_layout,
                                    hines_stream_t stream) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (solver_layout != 0 && solver_layout != 1) return HINES_ERR_INVALID_ARG;
  if (!solver_layout && p->rerooted) return HINES_ERR_INVALID_ARG;
  if (solver_layout ? (!need_pk(p, s) || !need_pk(p, g) || !need_pk(p, u) || !need_pk(p, V_inout))
                    : (!need(p, s) || !need(p, g) || !need(p, u) || !need(p, V_inout)))
    return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_unit_cable_reuse(p->dev, s, g, u, V_inout, dt, E, theta, solver_layout != 0,
                                                 reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_grad_du(hines_plan_t p, const double* lambda, const double* x, double* grad_d, double* grad_u,
                           hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, lambda) || !need(p, x) || !need(p, grad_d) || !need(p, grad_u)) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_grad_du(p->dev, lambda, x, grad_d, grad_u, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_adjoint_step(hines_plan_t p, const double* lambda, const double* V_k, const double* V_km1,
                                      const double* s, const double* g, const double* target, double dt, double E,
                                      int32_t theta, int32_t add_loss_term, double* grad_g, double* grad_a,
                                      double* vbar_out, hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, lambda) || !need(p, V_k) || !need(p, V_km1) || !need(p, s) || !need(p, g) || !need(p, grad_g) ||
      !need(p, grad_a) || !need(p, vbar_out))
    return HINES_ERR_INVALID_ARG;
  if (add_loss_term && !target && p->host.n_cells > 0) return HINES_ERR_INVALID_ARG;
  if (theta != 0 && theta != 1) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_cable_adjoint_step(p->dev, lambda, V_k, V_km1, s, g, target, dt, E, theta,
                                                   add_loss_term, grad_g, grad_a, vbar_out,
                                                   reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_loss_seed(hines_plan_t p, const double* V, const double* target, double* vbar,
                                   hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, V) || !need(p, vbar) || (!target && p->host.n_cells > 0)) return HINES_ERR_INVALID_ARG;
  return launched(hines::launch_cable_loss_seed(p->dev, V, target, vbar, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_cable_loss_accumulate(hines_plan_t p, const double* V, const double* target, double* loss_cells,
                                         hines_stream_t stream) {
  hines_status st = check_natural(p);
  if (st != HINES_OK) return st;
  if (!need(p, V) || ((!target || !loss_cells) && p->host.n_cells > 0)) return HINES_ERR_INVALID_ARG;
  return launched(
      hines::launch_cable_loss_accumulate(p->dev, V, target, loss_cells, reinterpret_cast<cudaStream_t>(stream)));
}

hines_status hines_plan_status(hines_plan_t p, int32_t* status_out) {
  hines_status st = check_plan(p);
  if (st != HINES_OK) return st;
  if (!status_out) return HINES_ERR_INVALID_ARG;
  if (cudaMemcpy(status_out, p->dev.status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HINES_ERR_CUDA;
  if (cudaMemset(p->dev.status, 0, sizeof(int32_t)) != cudaSuccess) return HINES_ERR_CUDA;
  return HINES_OK;
}

const char* hines_status_string(int32_t status) {
  switch (status) {
    case HINES_OK: return "ok";
    case HINES_ERR_INVALID_ARG: return "invalid argument";
    case HINES_ERR_NOT_HINES_ORDER: return "parent array not in Hines order (need p[0] = -1, 0 <= p[i] < i)";
    case HINES_ERR_OOM: return "out of memory";
    case HINES_ERR_CUDA: return "CUDA runtime error";
    case HINES_ERR_TIMEOUT: return "bounded device wait timed out";
    case HINES_WARN_REFINE: return "iterative refinement did not contract";
    case HINES_ERR_DEVICE: return "plan belongs to another device";
    default: return "unknown status";
  }
}

}  // extern "C"
