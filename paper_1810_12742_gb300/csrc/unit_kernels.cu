// Warp-task kernels of the batched Hines solver, sm_103a.
//
// The planner cuts every cell into units -- whole small cells, or the top part
// and the subtrees of a large cell -- and packs units into tasks (by size, or
// by Section 4's rule with the 32 lanes of a warp).  A warp owns a task and
// walks its levels, one level = chunks of at most 32 branches, one per lane:
// deepest level first for the elimination, root level first for the
// substitution (Section 3).  Inside a branch the parent of compartment i is
// i - 1 (Section 5): each lane runs a Thomas chain (Listing 1) and leaves one
// contribution for its parent compartment (Listing 2's parent lookup).
//
// A solve is two launches: (A) whole-cell tasks (both sweeps), the
// elimination of subtree tasks and, taken over by the warp that finishes a
// cell's last subtree, that cell's top part (both sweeps); (C) the
// substitution of subtree tasks.  No warp ever waits for another.
//
// The levels of a task follow one another in the same warp, so a chunk's
// children are the lanes of the chunk just before it (elimination) and its
// parents likewise (substitution): those values pass through a small shared
// memory cache; only values crossing task boundaries go through global
// memory.  The next chunk's inputs are staged with cp.async into a second
// buffer while the current one is computed, in an interleaved layout
// (Section 5) whose column is XOR-swizzled by the row so that the warp's
// copies and the lanes' chain steps are free of bank conflicts.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hines.h"
#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hines {
namespace {

using namespace dev;

constexpr int kL = kBranchCap;      // compartments per branch, at most
constexpr int kSlots = 32 * kL;     // one staged array of one chunk
constexpr int kWarps = kWarpsPerCta;
constexpr int kSmemPerSm = 227 * 1024;  // shared memory one SM gives its CTAs

struct Meta {
  long long first, pcomp;  // solver layout: the chunk's block offset, the parent's solver-layout index
  int ppos, cpos, len, nchild, ccontig, xtask;
  float4 ds;  // compensated substitution: folded distal state left by the elimination
};

template <bool kPk>
__device__ __forceinline__ Meta load_meta(const DevPlan& P, int pos, bool valid, bool want_ds) {
  Meta m{0, -1, -1, 0, 0, 0, 0, 0, make_float4(0.f, 0.f, 0.f, 0.f)};
  if (valid) {
    if (want_ds) m.ds = static_cast<const float4*>(P.dstate)[pos];
    const BrMetaT t = P.tmeta[pos];
    if (kPk) {
      const longlong2 q = P.pk_meta[pos];
      m.first = q.x;
      m.pcomp = q.y;
    } else {
      m.first = t.first;
      m.pcomp = t.pcomp;
    }
    m.ppos = t.ppos;
    m.cpos = t.cpos;
    m.len = t.len;
    m.nchild = t.nchild;
    m.ccontig = t.ccontig;
    m.xtask = t.xtask;
  }
  return m;
}

__device__ __forceinline__ int child_pos(const DevPlan& P, const Meta& m, int i) {
  return m.ccontig ? m.cpos + i : __ldg(P.tchild + m.cpos + i);
}

// A child's contribution slot: through L2 when another warp may have written
// it in this launch (a top part's subtree children), else the ordinary path.
template <typename V>
__device__ __forceinline__ V slot_load(const V* p, const Meta& m) {
  return m.xtask ? __ldcg(p) : *p;
}

// The chunk processed just before the current one in the same sweep.
struct Prev {
  int c0, n, which;  // n = 0: none
};

// Per-element work over a chunk's branches in the natural layout: sixteen
// lanes per branch, two branches per step (branches are at most 16 long), so a
// step's copies read two contiguous runs.  kPc: also pass the branch's parent
// compartment.
template <bool kPc = false, typename F>
__device__ __forceinline__ void for_branch_elements(const Meta& m, int n, int lane, F&& f) {
  const int half = lane >> 4, t = lane & 15;
  for (int j = 0; j < n; j += 2) {
    const int jj = j + half;
    const long long fj = __shfl_sync(kFull, m.first, jj & 31);
    const int lj = __shfl_sync(kFull, m.len, jj & 31);
    const long long pc = kPc ? __shfl_sync(kFull, m.pcomp, jj & 31) : -1;
    if (jj < n && t < lj) f(jj, t, lj, fj, pc);
  }
}

// Staged-chunk index of row k (counted from the distal end) of a lane's branch.
// Natural layout: the XOR-swizzled interleaving built while staging.
struct NatIdx {
  __device__ __forceinline__ int operator()(int k, int lane) const { return sidx(k, lane); }
};
// Solver layout: the chunk's block as stored, row r holding the lanes whose
// branch is longer than r, in lane order: offset of row r plus the rank of the
// lane among them.  Consecutive active lanes read consecutive words.
struct PkIdx {
  const uint2* tab;  // per row: (lanes present, row offset)
  unsigned lt;       // mask of the lanes below this one
  __device__ __forceinline__ int operator()(int k, int) const {
    const uint2 t = tab[k];
    return (int)t.y + __popc(t.x & lt);
  }
};
constexpr int kTabBytes = kL * 8;

// Builds the row table of the current chunk (every lane of the warp calls it).
__device__ __forceinline__ PkIdx pk_index(const Meta& m, int n, int lane, unsigned char* tabmem) {
  uint2* tab = reinterpret_cast<uint2*>(tabmem);
  const int len = lane < n ? m.len : 0;
  unsigned off = 0;
#pragma unroll
  for (int r = 0; r < kL; ++r) {
    const unsigned mk = __ballot_sync(kFull, len > r);
    if (lane == r) tab[r] = make_uint2(mk, off);
    off += __popc(mk);
  }
  __syncwarp();
  return PkIdx{tab, (1u << lane) - 1u};
}

template <bool kPk>
struct IdxOf;
template <>
struct IdxOf<false> {
  using type = NatIdx;
  __device__ static NatIdx make(const Meta&, int, int, unsigned char*) { return NatIdx{}; }
};
template <>
struct IdxOf<true> {
  using type = PkIdx;
  __device__ static PkIdx make(const Meta& m, int n, int lane, unsigned char* t) { return pk_index(m, n, lane, t); }
};

// Solver layout: compartments in the chunk's block (every lane calls it).
__device__ __forceinline__ int chunk_elems(const Meta& m, int n, int lane) {
  return __reduce_add_sync(kFull, lane < n ? m.len : 0);
}

// Solver layout: copy the chunk's block of one array into shared memory with
// 16-byte copies (blocks start on multiples of 4 compartments and are padded).
template <typename T>
__device__ __forceinline__ void stage_block(T* dst, const T* src, long long blk, int e, int lane) {
  constexpr int V = 16 / (int)sizeof(T);
  const int nv = (e + V - 1) / V;
  for (int v = lane; v < nv; v += 32) cp_async16(dst + v * V, src + blk + (long long)v * V);
}

// ============================================================================
// Compensated mode: FP32 inputs, double-float arithmetic from FP32 error-free
// transformations, FP64 solution.  The elimination keeps nothing per
// compartment: it leaves, per branch, its contribution to the parent (or the
// root's solution) and its folded distal state; the substitution re-stages the
// chunk and re-eliminates it from that state before substituting.
// ============================================================================
template <bool kPk>
struct CompModeT {
  static constexpr bool kPacked = kPk;
  struct Args {
    const float* d;
    const float* u;
    const float* b;
    double* x;
  };
  static constexpr int kStageBytes = 3 * kSlots * 4;
  static constexpr int kStages = 2;
  static constexpr int kCacheBytes = 2 * 32 * 16 + 2 * 32 * 8 + kTabBytes;
  static constexpr int kWarpBytes = kStages * kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = kSmemPerSm / (kWarps * kWarpBytes);  // CTAs per SM that shared memory allows

  static constexpr bool kWantDs = true;

  __device__ static void stage(const DevPlan&, const Args& A, int, const Meta& m, int n, int lane,
                               unsigned char* buf) {
    float* sd = reinterpret_cast<float*>(buf);
    float* su = sd + kSlots;
    float* sb = su + kSlots;
    if (kPk) {
      const long long blk = __shfl_sync(kFull, m.first, 0);
      const int e = chunk_elems(m, n, lane);
      stage_block(sd, A.d, blk, e, lane);
      stage_block(su, A.u, blk, e, lane);
      stage_block(sb, A.b, blk, e, lane);
    } else {
      for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
        const int q = sidx(lj - 1 - t, jj);
        cp_async4(&sd[q], A.d + fj + t);
        cp_async4(&su[q], A.u + fj + t);
        cp_async4(&sb[q], A.b + fj + t);
      });
    }
    cp_commit();
  }

  __device__ static void compute(const DevPlan& P, const Args&, int visit, int c0, int n, int lane, const Meta& m,
                                 unsigned char* buf, const Prev& pv, unsigned char* cache, int cur) {
    float* sd = reinterpret_cast<float*>(buf);
    const float* su = sd + kSlots;
    float* sb = sd + 2 * kSlots;
    float4* cslot = reinterpret_cast<float4*>(cache);        // [2][32] contributions
    float2* cx = reinterpret_cast<float2*>(cache + 2 * 32 * 16);  // [2][32] distal solutions
    float4* slot = static_cast<float4*>(P.cd);
    float4* dst = static_cast<float4*>(P.dstate);
    float2* xlast = static_cast<float2*>(P.xlast);
    const auto Q = IdxOf<kPk>::make(m, n, lane, cache + 2 * 32 * 16 + 2 * 32 * 8);
    if (lane >= n) return;
    const int pos = c0 + lane;
    const int len = m.len;
    if (visit == 0) {
      ff Dv = {sd[Q(0, lane)], 0.f}, Bv = {sb[Q(0, lane)], 0.f};
      for (int i = 0; i < m.nchild; ++i) {
        const int cp = child_pos(P, m, i);
        const int loc = cp - pv.c0;
        const float4 v = (loc >= 0 && loc < pv.n) ? cslot[pv.which * 32 + loc] : slot_load(slot + cp, m);
        Dv = ff_sub(Dv, v.x, v.y);
        Bv = ff_sub(Bv, v.z, v.w);
      }
      dst[pos] = make_float4(Dv.h, Dv.l, Bv.h, Bv.l);
      for (int k = 0; k < len - 1; ++k) {
        const float uk = su[Q(k, lane)];
        const ff f = ff_div_f(uk, Dv);
        const ff fu = ff_mul_f(f, uk);
        const ff fb = ff_mul(f, Bv);
        Dv = ff_sub_dom(sd[Q(k + 1, lane)], fu.h, fu.l);
        Bv = ff_sub({sb[Q(k + 1, lane)], 0.f}, fb.h, fb.l);
      }
      float4 out;
      if (m.pcomp >= 0) {
        const float uk = su[Q(len - 1, lane)];
        const ff f = ff_div_f(uk, Dv);
        const ff fu = ff_mul_f(f, uk);
        const ff fb = ff_mul(f, Bv);
        out = make_float4(fu.h, fu.l, fb.h, fb.l);
      } else {
        const ff x0 = ff_div(Bv, Dv);  // solve root
        out = make_float4(x0.h, x0.l, 0.f, 0.f);
      }
      slot[pos] = out;
      cslot[cur * 32 + lane] = out;
      return;
    }
    ff Dv = {m.ds.x, m.ds.y}, Bv = {m.ds.z, m.ds.w};
    float el[kL], bl[kL];
#pragma unroll
    for (int k = 0; k < kL; ++k) {
      if (k < len) {
        const int q = Q(k, lane);
        sd[q] = Dv.h;
        el[k] = Dv.l;
        sb[q] = Bv.h;
        bl[k] = Bv.l;
        if (k < len - 1) {
          const float uk = su[q];
          const ff f = ff_div_f(uk, Dv);
          const ff fu = ff_mul_f(f, uk);
          const ff fb = ff_mul(f, Bv);
          const int q1 = Q(k + 1, lane);
          Dv = ff_sub_dom(sd[q1], fu.h, fu.l);
          Bv = ff_sub({sb[q1], 0.f}, fb.h, fb.l);
        }
      }
    }
    ff xp = {0.f, 0.f};
    if (m.pcomp >= 0) {
      const int loc = m.ppos - pv.c0;
      const float2 t = (loc >= 0 && loc < pv.n) ? cx[pv.which * 32 + loc] : xlast[m.ppos];
      xp = {t.x, t.y};
    }
#pragma unroll
    for (int k = kL - 1; k >= 0; --k) {
      if (k < len) {
        const int q = Q(k, lane);
        ff xi;
        if (m.pcomp < 0 && k == len - 1) {
          const float4 t = slot[pos];
          xi = {t.x, t.y};
        } else {
          const float uk = su[q];
          const float M = __fmul_rn(uk, xp.h);
          float mm = fmaf(uk, xp.h, -M);
          mm = fmaf(uk, xp.l, mm);
          const ff num = ff_sub({sb[q], bl[k]}, M, mm);
          xi = ff_div(num, {sd[q], el[k]});
        }
        const double xd = ff_to_double(xi.h, xi.l);
        sd[q] = __int_as_float(__double2loint(xd));
        sb[q] = __int_as_float(__double2hiint(xd));
        xp = xi;
      }
    }
    const float2 xo = make_float2(xp.h, xp.l);
    xlast[pos] = xo;
    cx[cur * 32 + lane] = xo;
  }

  __device__ static void copy_out(const DevPlan&, const Args& A, int visit, const Meta& m, int n, int lane,
                                  unsigned char* buf) {
    if (visit == 0) return;
    const float* sd = reinterpret_cast<const float*>(buf);
    const float* sb = sd + 2 * kSlots;
    if (kPk) {
      const long long blk = __shfl_sync(kFull, m.first, 0);
      const int e = chunk_elems(m, n, lane);
      for (int i = lane; i < e; i += 32) A.x[blk + i] = __hiloint2double(__float_as_int(sb[i]), __float_as_int(sd[i]));
      return;
    }
    for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
      const int q = sidx(lj - 1 - t, jj);
      A.x[fj + t] = __hiloint2double(__float_as_int(sb[q]), __float_as_int(sd[q]));
    });
  }
};

// ============================================================================
// Factor mode (FP64, FP32, passive cable): the elimination writes the
// reciprocal eliminated diagonal to the workspace and the eliminated
// right-hand side in place; the substitution reads them back.  In cable mode
// the system is rebuilt while staging (Section 1's implicit-Euler system):
// d_i = s_i (1 + theta dt g_i) + sum of a over the edges at i (a = -u),
// b_i = s_i V_i + s_i dt g_i (E - (1 - theta) V_i).
// ============================================================================
// kReuse: the elimination of a new right-hand side with the factor a previous
// solve of the same plan and matrix left in the workspace (the reciprocal
// eliminated diagonal): only b is eliminated (the refinement's correction
// solves; passive-cable steps after the first, the matrix being constant).
template <typename T, bool kCable, bool kPk, bool kReuse = false>
struct FactorMode {
  // the reciprocal eliminated diagonal: FP64 as rcp_t gives it; FP32 with one
  // more Newton step on the hardware approximation, so that the stored factor
  // is that of an FP32 elimination to the last bit or so, which the
  // refinement's re-solves depend on
  __device__ static T rcp_solve(T x) {
    T r = rcp_t(x);
    if (sizeof(T) == 4) r = fma(r, fma(-x, r, T(1)), r);
    return r;
  }
  static constexpr bool kPacked = kPk;
  struct Args {
    const T* d;
    const T* u;
    const T* s;  // cable: s, g
    const T* g;
    T* x;        // right-hand side in, solution out (cable: V in, V out)
    T dt, E, theta;
    bool rhs_from_V;
  };
  static constexpr int kStageBytes = 3 * kSlots * (int)sizeof(T);
  // FP64 chunks are large and the FP64 pipe is slow: one staging buffer, so
  // that twice as many warps share an SM
  static constexpr int kStages = sizeof(T) == 8 ? 1 : 2;
  static constexpr int kCacheBytes = 2 * 32 * 2 * (int)sizeof(T) + 2 * 32 * (int)sizeof(T) + kTabBytes;
  static constexpr int kWarpBytes = kStages * kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = kSmemPerSm / (kWarps * kWarpBytes);  // CTAs per SM that shared memory allows

  static constexpr bool kWantDs = false;

  // Section 1's implicit-Euler system: the membrane part of the diagonal,
  // s (1 + theta dt g), and the right-hand side s (V + dt g (E - (1 - theta) V)),
  // each in the fewest operations (theta = 1: s (V + dt E g))
  __device__ static T cable_diag(const Args& A, T si, T gi) { return si * fma(A.theta * A.dt, gi, T(1)); }
  __device__ static T cable_rhs(const Args& A, T si, T gi, T vi) {
    if (A.theta == T(1)) return si * fma(A.dt * A.E, gi, vi);
    return si * fma(A.dt * gi, fma(A.theta - T(1), vi, A.E), vi);
  }

  __device__ static void stage(const DevPlan& P, const Args& A, int visit, const Meta& m, int n, int lane,
                               unsigned char* buf) {
    T* sd = reinterpret_cast<T*>(buf);
    T* su = sd + kSlots;
    T* sb = su + kSlots;
    if (kPk && kCable && visit == 0) {
      // the block's rows in place; the own edge to the parent is taken off
      // the diagonal in compute(), where the cell's root compartment is known
      const long long blk = __shfl_sync(kFull, m.first, 0);
      const int e = chunk_elems(m, n, lane);
      if (kReuse) {  // the stored factor; only the right-hand side is rebuilt
        stage_block(sd, static_cast<const T*>(P.fac), blk, e, lane);
        stage_block(su, A.u, blk, e, lane);
      }
      for (int i = lane; i < e; i += 32) {
        const long long g = blk + i;
        const T vi = A.x[g];
        if (kReuse) {
          sb[i] = A.rhs_from_V ? cable_rhs(A, A.s[g], A.g[g], vi) : vi;
        } else {
          const T si = A.s[g], gi = A.g[g], ui = A.u[g];
          sd[i] = cable_diag(A, si, gi);
          su[i] = ui;
          sb[i] = A.rhs_from_V ? cable_rhs(A, si, gi, vi) : vi;
        }
      }
    } else if (kPk) {
      const long long blk = __shfl_sync(kFull, m.first, 0);
      const int e = chunk_elems(m, n, lane);
      stage_block(sd, (visit == 1 || kReuse) ? static_cast<const T*>(P.fac) : A.d, blk, e, lane);
      stage_block(su, A.u, blk, e, lane);
      stage_block(sb, static_cast<const T*>(A.x), blk, e, lane);
    } else if (visit == 1) {
      const T* fac = static_cast<const T*>(P.fac);
      for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
        const int q = sidx(lj - 1 - t, jj);
        cp_async(&sd[q], fac + fj + t);
        cp_async(&su[q], A.u + fj + t);
        cp_async(&sb[q], A.x + fj + t);
      });
    } else if (!kCable) {
      const T* dsrc = kReuse ? static_cast<const T*>(P.fac) : A.d;
      for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
        const int q = sidx(lj - 1 - t, jj);
        cp_async(&sd[q], dsrc + fj + t);
        cp_async(&su[q], A.u + fj + t);
        cp_async(&sb[q], A.x + fj + t);
      });
    } else if (kReuse) {  // cable, stored factor: only the right-hand side is rebuilt
      const T* fac = static_cast<const T*>(P.fac);
      for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
        const long long i = fj + t;
        const int q = sidx(lj - 1 - t, jj);
        cp_async(&sd[q], fac + i);
        cp_async(&su[q], A.u + i);
        const T vi = A.x[i];
        sb[q] = A.rhs_from_V ? cable_rhs(A, A.s[i], A.g[i], vi) : vi;
      });
    } else {
      for_branch_elements<true>(m, n, lane, [&](int jj, int t, int lj, long long fj, long long pc) {
        const long long i = fj + t;
        const T si = A.s[i], gi = A.g[i], ui = A.u[i], vi = A.x[i];
        T dd = cable_diag(A, si, gi);
        if (!(pc < 0 && t == 0)) dd -= ui;  // own edge to the parent
        const T bb = A.rhs_from_V ? cable_rhs(A, si, gi, vi) : vi;
        const int q = sidx(lj - 1 - t, jj);
        sd[q] = dd;
        su[q] = ui;
        sb[q] = bb;
      });
    }
    cp_commit();
  }

  __device__ static void compute(const DevPlan& P, const Args& A, int visit, int c0, int n, int lane, const Meta& m,
                                 unsigned char* buf, const Prev& pv, unsigned char* cache, int cur) {
    T* sd = reinterpret_cast<T*>(buf);
    const T* su = sd + kSlots;
    T* sb = sd + 2 * kSlots;
    T* cslot = reinterpret_cast<T*>(cache);                   // [2][32][2] contributions
    T* cx = cslot + 2 * 32 * 2;                               // [2][32] distal solutions
    T* slot = static_cast<T*>(P.cd);                          // [nb][2]
    const auto Q = IdxOf<kPk>::make(m, n, lane, cache + kCacheBytes - kTabBytes);
    if (lane >= n) return;
    const int pos = c0 + lane;
    const int len = m.len;
    if (kReuse && visit == 0) {  // sd holds the stored reciprocals; eliminate b only
      T B = sb[Q(0, lane)];
      for (int i = 0; i < m.nchild; ++i) {
        const int cp = child_pos(P, m, i);
        const int loc = cp - pv.c0;
        const bool local = loc >= 0 && loc < pv.n;
        B -= local ? cslot[(pv.which * 32 + loc) * 2 + 1] : slot_load(slot + 2 * cp + 1, m);
      }
      for (int k = 0; k < len - 1; ++k) {
        const int q = Q(k, lane);
        sb[q] = B;
        const T f = su[q] * sd[q];
        B = sb[Q(k + 1, lane)] - f * B;
      }
      const int q = Q(len - 1, lane);
      T c1v = T(0);
      if (m.pcomp >= 0) {
        sb[q] = B;
        c1v = su[q] * sd[q] * B;
      } else {
        sb[q] = B * sd[q];  // solve root
      }
      slot[2 * pos] = T(0);
      slot[2 * pos + 1] = c1v;
      cslot[(cur * 32 + lane) * 2] = T(0);
      cslot[(cur * 32 + lane) * 2 + 1] = c1v;
      return;
    }
    if (visit == 0) {
      if (kPk && kCable) {  // own edge to the parent, except at the cell's root compartment
        for (int k = 0; k < len; ++k)
          if (!(m.pcomp < 0 && k == len - 1)) sd[Q(k, lane)] -= su[Q(k, lane)];
      }
      T D = sd[Q(0, lane)], B = sb[Q(0, lane)];
      for (int i = 0; i < m.nchild; ++i) {
        const int cp = child_pos(P, m, i);
        const int loc = cp - pv.c0;
        const bool local = loc >= 0 && loc < pv.n;
        D -= local ? cslot[(pv.which * 32 + loc) * 2] : slot_load(slot + 2 * cp, m);
        B -= local ? cslot[(pv.which * 32 + loc) * 2 + 1] : slot_load(slot + 2 * cp + 1, m);
      }
      for (int k = 0; k < len - 1; ++k) {
        const T uk = su[Q(k, lane)];
        const T r = rcp_solve(D);
        sd[Q(k, lane)] = r;
        sb[Q(k, lane)] = B;
        const T f = uk * r;
        D = sd[Q(k + 1, lane)] - f * uk;
        if (kCable) D -= uk;  // the edge to the chain child
        B = sb[Q(k + 1, lane)] - f * B;
      }
      const int k = len - 1;
      const T r = rcp_solve(D);
      sd[Q(k, lane)] = r;
      T c0v = T(0), c1v = T(0);
      if (m.pcomp >= 0) {
        sb[Q(k, lane)] = B;
        const T uk = su[Q(k, lane)];
        const T f = uk * r;
        c0v = kCable ? f * uk + uk : f * uk;
        c1v = f * B;
      } else {
        sb[Q(k, lane)] = B * r;  // solve root
      }
      slot[2 * pos] = c0v;
      slot[2 * pos + 1] = c1v;
      cslot[(cur * 32 + lane) * 2] = c0v;
      cslot[(cur * 32 + lane) * 2 + 1] = c1v;
      return;
    }
    T xp = T(0);
    if (m.pcomp >= 0) {
      const int loc = m.ppos - pv.c0;
      xp = (loc >= 0 && loc < pv.n) ? cx[pv.which * 32 + loc] : A.x[m.pcomp];
    }
    for (int k = len - 1; k >= 0; --k) {
      const int q = Q(k, lane);
      const T xi = (m.pcomp < 0 && k == len - 1) ? sb[q] : (sb[q] - su[q] * xp) * sd[q];
      sb[q] = xi;
      xp = xi;
    }
    cx[cur * 32 + lane] = xp;
  }

  __device__ static void copy_out(const DevPlan& P, const Args& A, int visit, const Meta& m, int n, int lane,
                                  unsigned char* buf) {
    const T* sd = reinterpret_cast<const T*>(buf);
    const T* sb = sd + 2 * kSlots;
    T* fac = static_cast<T*>(P.fac);
    if (kPk) {
      const long long blk = __shfl_sync(kFull, m.first, 0);
      const int e = chunk_elems(m, n, lane);
      for (int i = lane; i < e; i += 32) {
        if (visit == 0 && !kReuse) fac[blk + i] = sd[i];
        A.x[blk + i] = sb[i];
      }
      return;
    }
    for_branch_elements(m, n, lane, [&](int jj, int t, int lj, long long fj, long long) {
      const int q = sidx(lj - 1 - t, jj);
      if (visit == 0 && !kReuse) fac[fj + t] = sd[q];
      A.x[fj + t] = sb[q];
    });
  }
};

// ============================================================================
// Task driver
// ============================================================================
// Position in a task's chunk sequence: levels deepest-first for the
// elimination (visit 0), root-first for the substitution (visit 1); a level of
// more than 32 branches is several chunks.
struct Pos {
  int visit, l, c0, n;  // visit == ve: past the end
};

__device__ __forceinline__ Pos pos_level(int visit, int l, const int32_t* lp) {
  const int c0 = __ldg(lp + l), e = __ldg(lp + l + 1) - c0;
  return {visit, l, c0, e < 32 ? e : 32};
}

__device__ __forceinline__ Pos pos_next(Pos p, const int32_t* lp, int nl, int ve) {
  const int end = __ldg(lp + p.l + 1);
  if (p.c0 + 32 < end) {
    p.c0 += 32;
    p.n = end - p.c0 < 32 ? end - p.c0 : 32;
    return p;
  }
  if (p.visit == 0) {
    if (p.l > 0) return pos_level(0, p.l - 1, lp);
    if (ve == 1) return {ve, 0, 0, 0};
    return pos_level(1, 0, lp);
  }
  if (p.l + 1 < nl) return pos_level(1, p.l + 1, lp);
  return {ve, 0, 0, 0};
}

template <class M>
__device__ void run_task(const DevPlan& P, const typename M::Args& A, int t, int code, int lane, unsigned char* wbase) {
  const int nl = P.task_nlvl[t];
  const int32_t* lp = P.tlvl_ptr + P.task_lvl_off[t];
  const int vb = code == 2 ? 1 : 0, ve = code == 1 ? 1 : 2;
  unsigned char* cache = wbase + M::kStages * M::kStageBytes;
  auto buf = [wbase](int which) { return wbase + (M::kStages == 2 ? which : 0) * M::kStageBytes; };
  auto meta = [&](const Pos& p) {
    return load_meta<M::kPacked>(P, p.c0 + lane, p.visit < ve && lane < p.n, M::kWantDs && p.visit == 1);
  };
  Pos cur = pos_level(vb, vb == 0 ? nl - 1 : 0, lp);
  Meta m_cur = meta(cur);
  M::stage(P, A, cur.visit, m_cur, cur.n, lane, buf(0));
  Pos nxt = pos_next(cur, lp, nl, ve);
  Meta m_nxt = meta(nxt);
  Prev pv{0, 0, 0};  // last chunk of the previous level in this sweep
  int which = 0;
  while (cur.visit < ve) {
    cp_wait_all();
    __syncwarp();
    // nothing of the substitution is read before the elimination has finished:
    // its first chunks reuse positions the elimination is still writing
    const bool crossing = nxt.visit != cur.visit;
    // two staging buffers: the next chunk is copied in while this one is
    // computed; one buffer: after this one is done (more warps per SM instead)
    if (M::kStages == 2 && nxt.visit < ve && !crossing) M::stage(P, A, nxt.visit, m_nxt, nxt.n, lane, buf(which ^ 1));
    const Pos nn = nxt.visit < ve ? pos_next(nxt, lp, nl, ve) : nxt;
    Meta m_nn = meta(nn);
    M::compute(P, A, cur.visit, cur.c0, cur.n, lane, m_cur, buf(which), pv, cache, cur.l & 1);
    __syncwarp();
    M::copy_out(P, A, cur.visit, m_cur, cur.n, lane, buf(which));
    __syncwarp();
    if (crossing && nxt.visit < ve) {
      m_nxt = meta(nxt);
      m_nn = meta(nn);
    }
    if (nxt.visit < ve && (crossing || M::kStages == 1)) M::stage(P, A, nxt.visit, m_nxt, nxt.n, lane, buf(which ^ 1));
    // predecessor of the next chunk: the last chunk of the level before its level, same sweep
    if (crossing) {
      pv = Prev{0, 0, 0};
    } else if (nxt.l != cur.l) {
      pv = Prev{cur.c0, cur.n, cur.l & 1};
    }
    cur = nxt;
    m_cur = m_nxt;
    nxt = nn;
    m_nxt = m_nn;
    which ^= 1;
  }
}

// After a subtree task's elimination: count its units off their cell's
// pending count; the warp that finishes the cell's last subtree takes over
// the cell's top part (both visits) as its next task.  Nothing waits: the
// hand-over goes to whoever arrives last.  Release: every lane fences its slot
// writes before lane 0's atomic; acquire: the fence after it, and the top
// part reads those slots through L2.  Returns the top task, or -1.
__device__ __forceinline__ int hand_over(const DevPlan& P, int t, int lane) {
  __threadfence();
  __syncwarp();
  const int cell = __ldg(P.task_sub + 2 * t);
  if (cell < 0) return -1;
  int last = 0;
  if (lane == 0) {
    const int cnt = __ldg(P.task_sub + 2 * t + 1);
    last = atomicSub(P.cell_pending + cell, cnt) == cnt;
  }
  if (!__shfl_sync(kFull, last, 0)) return -1;
  __threadfence();
  return __ldg(P.cell_top_task + cell);
}

template <class M>
__global__ void __launch_bounds__(32 * kWarps, M::kMinBlocks) k_units(DevPlan P, typename M::Args A, int phase) {
  extern __shared__ __align__(16) unsigned char smem_u[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* wbase = smem_u + w * M::kWarpBytes;
  const int e0 = P.phase_off[phase], ne = P.phase_off[phase + 1] - e0;
  int next = -1;  // a top part handed over to this warp
  for (;;) {
    int t, code;
    if (next >= 0) {
      t = next;
      code = 0;
      next = -1;
    } else {
      int k = 0;
      if (lane == 0) k = atomicAdd(P.counter + phase, 1);
      k = __shfl_sync(kFull, k, 0);
      if (k >= ne) break;
      const int e = P.phase_entry[e0 + k];
      t = e >> 2;
      code = e & 3;
    }
    run_task<M>(P, A, t, code, lane, wbase);
    if (code == 1) next = hand_over(P, t, lane);
  }
}

template <class M>
cudaError_t grid_of(const DevPlan& P, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  const size_t smem = (size_t)kWarps * M::kWarpBytes;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_units<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_units<M>, 32 * kWarps, smem);
  if (e != cudaSuccess) return e;
  *grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  return cudaSuccess;
}

template <class M>
cudaError_t launch_phases(const DevPlan& P, const typename M::Args& A, int grid, cudaStream_t s) {
  if (P.n_wtasks == 0) return cudaSuccess;
  const size_t smem = (size_t)kWarps * M::kWarpBytes;
  // work counters to 0 and per-cell subtree counts to their full values
  cudaError_t e = cudaMemcpyAsync(P.counter, P.counter_init, (4 + (size_t)P.n_cells) * sizeof(int32_t),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  for (int phase = 0; phase < 3; ++phase) {
    const int ne = P.phase_off[phase + 1] - P.phase_off[phase];
    if (ne == 0) continue;
    const int warps = ne < grid * kWarps ? ne : grid * kWarps;
    const int blocks = (warps + kWarps - 1) / kWarps;
    k_units<M><<<blocks, 32 * kWarps, smem, s>>>(P, A, phase);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

using F64 = FactorMode<double, false, false>;
using F32 = FactorMode<float, false, false>;
using Cable = FactorMode<double, true, false>;
using CompMode = CompModeT<false>;
using PkF64 = FactorMode<double, false, true>;
using PkF32 = FactorMode<float, false, true>;
using PkComp = CompModeT<true>;
using PkCable = FactorMode<double, true, true>;
using F32Reuse = FactorMode<float, false, false, true>;
using CableReuse = FactorMode<double, true, false, true>;
using PkCableReuse = FactorMode<double, true, true, true>;

}  // namespace

cudaError_t prepare_unit_kernels(DevPlan& P) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  P.sms = sms > 0 ? sms : 1;
  e = grid_of<F64>(P, &P.grid[0]);
  if (e == cudaSuccess) e = grid_of<F32>(P, &P.grid[1]);
  if (e == cudaSuccess) e = grid_of<Cable>(P, &P.grid[2]);
  if (e == cudaSuccess) e = grid_of<CompMode>(P, &P.grid[3]);
  if (e == cudaSuccess) e = grid_of<PkF64>(P, &P.grid[4]);
  if (e == cudaSuccess) e = grid_of<PkF32>(P, &P.grid[5]);
  if (e == cudaSuccess) e = grid_of<PkComp>(P, &P.grid[6]);
  if (e == cudaSuccess) e = grid_of<PkCable>(P, &P.grid[7]);
  int g_reuse = 0;  // same footprint as the FP32 solve
  if (e == cudaSuccess) e = grid_of<F32Reuse>(P, &g_reuse);
  if (e == cudaSuccess) e = grid_of<CableReuse>(P, &g_reuse);
  if (e == cudaSuccess) e = grid_of<PkCableReuse>(P, &g_reuse);
  return e;
}

cudaError_t launch_unit_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s) {
  F64::Args A{d, u, nullptr, nullptr, b, 0.0, 0.0, 0.0, false};
  return launch_phases<F64>(P, A, P.grid[0], s);
}

cudaError_t launch_unit_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s) {
  F32::Args A{d, u, nullptr, nullptr, b, 0.f, 0.f, 0.f, false};
  return launch_phases<F32>(P, A, P.grid[1], s);
}

cudaError_t launch_unit_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, bool rhs_from_V, cudaStream_t s) {
  Cable::Args A{nullptr, u, sv, g, V, dt, E, (double)theta, rhs_from_V};
  return launch_phases<Cable>(P, A, P.grid[2], s);
}

cudaError_t launch_unit_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                          cudaStream_t s) {
  CompMode::Args A{d, u, b, x};
  return launch_phases<CompMode>(P, A, P.grid[3], s);
}

cudaError_t launch_pk_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s) {
  PkF64::Args A{d, u, nullptr, nullptr, b, 0.0, 0.0, 0.0, false};
  return launch_phases<PkF64>(P, A, P.grid[4], s);
}

cudaError_t launch_pk_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s) {
  PkF32::Args A{d, u, nullptr, nullptr, b, 0.f, 0.f, 0.f, false};
  return launch_phases<PkF32>(P, A, P.grid[5], s);
}

cudaError_t launch_pk_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                        cudaStream_t s) {
  PkComp::Args A{d, u, b, x};
  return launch_phases<PkComp>(P, A, P.grid[6], s);
}

cudaError_t launch_pk_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V, double dt,
                            double E, int theta, bool rhs_from_V, cudaStream_t s) {
  PkCable::Args A{nullptr, u, sv, g, V, dt, E, (double)theta, rhs_from_V};
  return launch_phases<PkCable>(P, A, P.grid[7], s);
}

cudaError_t launch_unit_resolve_f32(const DevPlan& P, const float* u, float* b, cudaStream_t s) {
  F32Reuse::Args A{nullptr, u, nullptr, nullptr, b, 0.f, 0.f, 0.f, false};
  return launch_phases<F32Reuse>(P, A, P.grid[1], s);
}

cudaError_t launch_unit_cable_reuse(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                                    double dt, double E, int theta, bool packed, cudaStream_t s) {
  if (packed) {
    PkCableReuse::Args A{nullptr, u, sv, g, V, dt, E, (double)theta, true};
    return launch_phases<PkCableReuse>(P, A, P.grid[7], s);
  }
  CableReuse::Args A{nullptr, u, sv, g, V, dt, E, (double)theta, true};
  return launch_phases<CableReuse>(P, A, P.grid[2], s);
}

}  // namespace hines
