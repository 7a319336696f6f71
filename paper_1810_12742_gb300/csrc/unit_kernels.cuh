// Warp-task kernels of the batched Hines solver, sm_103a.
//
// The planner cuts every cell into units -- whole small cells, or the top part
// and the subtrees of a large cell -- and packs units into tasks.  A warp owns
// a task and walks its chunks (Hu's list schedule of the task's pieces, at
// most 32 * P pieces each, longest first): deepest chunk first for the
// elimination, root-side chunk first for the substitution (Section 3).  Lane
// j owns the chunk's pieces P j .. P j + P - 1 (P = 1 or 2 pieces per lane).
// Inside a piece the parent of compartment i is i - 1 (Section 5): the lane
// runs a Thomas chain (Listing 1) and leaves one contribution for its parent
// compartment (Listing 2's parent lookup).  With P = 2 the lane runs its two
// chains at once, the two pieces aligned at their proximal ends (the shorter
// one joins the chain when its distal row comes up), so that both halves of
// every value live in one 8-byte register pair and the compensated
// arithmetic runs on packed FP32-pair instructions.
//
// A solve is two launches: (A) whole-cell tasks (both sweeps), the
// elimination of subtree tasks and, taken over by the warp that finishes a
// cell's last subtree, that cell's top part (both sweeps); (C) the
// substitution of subtree tasks.  No warp ever waits for another.
//
// The chunks of a task follow one another in the same warp, so a chunk's
// children are usually in the chunk just before it (elimination) and its
// parents likewise (substitution): those values pass through a small shared
// memory cache; other values go through global memory.  A chunk's inputs are
// staged into shared memory in the row layout of Section 5 (row r: the
// compartments r rows from each pair's distal start, one word per piece), so
// that a lane reads its P values of a row as one word: gathered with cp.async
// from the natural layout, or, where they are one contiguous block (the
// solver layout, and the factor blocks the eliminations leave in block
// order), by bulk copies one lane issues (BulkStage).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hines.h"
#include "device_common.cuh"
#include "kernels.h"
#include "plan.h"

namespace hines {
namespace {

using namespace dev;

constexpr int kL = kBranchCap;          // rows (compartments per piece), at most
constexpr int kWarps = kWarpsPerCta;
constexpr int kSmemPerSm = 227 * 1024;  // shared memory one SM gives its CTAs

template <int P>
struct Geo {
  static constexpr int kChunk = 32 * P;              // pieces per chunk
  static constexpr int kS = P == 2 ? 66 : 32;        // natural staging: words per row
  static constexpr int kSlots = kL * kS + 4;         // words per staged array (holds a padded solver-layout block)
};
// Natural-layout staging: the word of piece i's compartment in row r.  One
// piece per lane: rows of 32 words, the column XOR-swizzled by the row, so
// that the warp's staging copies (sixteen consecutive rows of one piece per
// half-warp) and the lanes' row reads are both free of bank conflicts.  Two
// pieces per lane: rows of 66 words (64 + 2), so that a lane's pair is one
// aligned 8-byte word and the staging copies spread over the banks.
template <int P>
__device__ __forceinline__ int nidx(int r, int i) {
  if constexpr (P == 2)
    return r * 66 + i;
  else
    return (r << 5) + (i ^ (r & 31));
}
template <int P>
struct VOf {
  using type = float;
};
template <>
struct VOf<2> {
  using type = F2;
};

// ---- per-lane metadata ------------------------------------------------------
struct Piece {
  long long first, pcomp;  // natural: proximal compartment, parent compartment; solver layout: the chunk's
                           // block offset, the parent's solver-layout index (-1 at a cell's root)
  int ppos, cpos, len, nchild, ccontig, xtask;
};
// A parent's solution fetched ahead: a double-float pair (compensated and
// refinement modes) or one value of the solve's type (factor modes).
union PreX {
  float2 ff;
  float f;
  double d;
};
__device__ __forceinline__ float pre_get(const PreX& v, float) { return v.f; }
__device__ __forceinline__ double pre_get(const PreX& v, double) { return v.d; }
__device__ __forceinline__ void pre_set(PreX& v, float x) { v.f = x; }
__device__ __forceinline__ void pre_set(PreX& v, double x) { v.d = x; }

template <int P>
struct Meta {
  long long blk;  // the chunk's block offset in the solver layout
  Piece p[P];
  // substitution: the parent's solution when another chunk than the cached
  // predecessor left it, fetched while the chunk is staged so that its
  // latency overlaps the staging copies
  PreX xpre[P];
  int L;         // rows of the lane: length of its first (longer) piece, 0 for a lane without pieces
};

template <bool kPk, int P>
__device__ __forceinline__ Meta<P> load_meta(const DevPlan& Pl, int c0, int n, int lane, bool active,
                                             bool want_blk = false) {
  Meta<P> m;
  m.blk = 0;
  if (want_blk && active && n > 0) m.blk = Pl.pk_meta[c0].x;  // every piece of a chunk shares it
#pragma unroll
  for (int h = 0; h < P; ++h) {
    const int i = P * lane + h;
    Piece q{0, -1, -1, 0, 0, 0, 0, 0};
    m.xpre[h].d = 0.0;
    if (active && i < n) {
      const int pos = c0 + i;
      const BrMetaT t = Pl.tmeta[pos];
      if (kPk) {
        const longlong2 w = Pl.pk_meta[pos];
        q.first = w.x;
        q.pcomp = w.y;
      } else {
        q.first = t.first;
        q.pcomp = t.pcomp;
      }
      q.ppos = t.ppos;
      q.cpos = t.cpos;
      q.len = t.len;
      q.nchild = t.nchild;
      q.ccontig = t.ccontig;
      q.xtask = t.xtask;
    }
    m.p[h] = q;
  }
  m.L = m.p[0].len;
  return m;
}

__device__ __forceinline__ int child_pos(const DevPlan& Pl, const Piece& q, int c) {
  return q.ccontig ? q.cpos + c : __ldg(Pl.tchild + q.cpos + c);
}

// A child's contribution slot: through L2 when another warp may have written
// it in this launch (a top part's subtree children), else the ordinary path.
template <typename W>
__device__ __forceinline__ W slot_load(const W* p, const Piece& q) {
  return q.xtask ? __ldcg(p) : *p;
}

// The chunk processed just before the current one in the same sweep.
struct Prev {
  int c0, n, which;  // n = 0: none
};

// ---- rows of the staged chunk -------------------------------------------------
// Word index of row r's first slot: natural layout, the fixed stride of the
// staging buffer; solver layout, the block's row offsets (a per-warp table).
template <bool kPk, int P>
struct Rows {
  const int* tab;
  // word of chunk position j (a lane's first piece: P * lane) in row r
  __device__ __forceinline__ int slot(int r, int j) const {
    if constexpr (kPk)
      return tab[r] + j;
    else
      return nidx<P>(r, j);
  }
};

// Solver layout: the row offsets of the current chunk's block from the lanes'
// row counts (every lane calls it); tab[kL] is the block's slot count.
template <int P>
__device__ __forceinline__ void build_row_table(int L, int lane, int* tab) {
  int acc = 0;
#pragma unroll
  for (int r = 0; r < kL; ++r) {
    const int nl = __popc(__ballot_sync(kFull, L > r));
    if (lane == r) tab[r] = acc;
    acc += P * nl;
  }
  if (lane == 0) tab[kL] = acc;
  __syncwarp();
}

// Every element of the chunk's pieces in the natural layout: sixteen lanes
// per piece, two pieces per step (pieces are at most 16 long); the owner
// lane's metadata comes by shuffle.  f(i, t, row, g, root) for piece i,
// distance t from its proximal end, row of the staged chunk, natural index g,
// and whether the piece holds its cell's root compartment (its parent is none).
template <int P, typename F>
__device__ __forceinline__ void for_chunk_elements(const Meta<P>& m, int n, int lane, F&& f) {
  const int half = lane >> 4, t = lane & 15;
  for (int j = 0; j < n; j += 2) {
    const int i = j + half, src = (i / P) & 31;
    long long first = __shfl_sync(kFull, m.p[0].first, src);
    int len = __shfl_sync(kFull, m.p[0].len, src);
    int root = __shfl_sync(kFull, (int)(m.p[0].pcomp < 0), src);
    const int rows = P == 2 ? __shfl_sync(kFull, m.L, src) : len;
    if constexpr (P == 2) {
      const long long f1 = __shfl_sync(kFull, m.p[1].first, src);
      const int l1 = __shfl_sync(kFull, m.p[1].len, src);
      const int r1 = __shfl_sync(kFull, (int)(m.p[1].pcomp < 0), src);
      if (i & 1) {
        first = f1;
        len = l1;
        root = r1;
      }
    }
    if (i < n && t < len) f(i, t, rows - 1 - t, first + t, root != 0);
  }
}

// Solver layout: copy the chunk's block of one array into shared memory with
// 16-byte copies (blocks start on multiples of 4 slots and are padded).
template <typename T>
__device__ __forceinline__ void stage_block(T* dst, const T* src, long long blk, int e, int lane) {
  constexpr int V = 16 / (int)sizeof(T);
  const int nv = (e + V - 1) / V;
  for (int v = lane; v < nv; v += 32) cp_async16(dst + v * V, src + blk + (long long)v * V);
}

// ---- one or two values of a row -------------------------------------------------
__device__ __forceinline__ float ldv(const float* s, int idx, float) { return s[idx]; }
__device__ __forceinline__ F2 ldv(const float* s, int idx, F2) { return *reinterpret_cast<const F2*>(s + idx); }
__device__ __forceinline__ void stv(float* s, int idx, float v) { s[idx] = v; }
__device__ __forceinline__ void stv(float* s, int idx, F2 v) { *reinterpret_cast<F2*>(s + idx) = v; }
__device__ __forceinline__ float vget(float v, int) { return v; }
__device__ __forceinline__ float vget(F2 v, int h) { return h == 0 ? f2_lo(v) : f2_hi(v); }
template <int P>
__device__ __forceinline__ typename VOf<P>::type vpack(const float* a) {
  if constexpr (P == 2)
    return f2_make(a[0], a[1]);
  else
    return a[0];
}
// the second half of v replaced by w (the shorter piece joins its chain)
__device__ __forceinline__ F2 vset_hi(F2 v, float w) { return f2_make(f2_lo(v), w); }

// ---- bulk staging -------------------------------------------------------------
// Contiguous blocks are staged by one-dimensional bulk copies that one lane
// issues, completing on a per-warp shared-memory barrier at byte kOff of the
// warp's region (then its phase parity and a failure flag).  A mode with one
// staging buffer has at most one staging in flight, so one barrier does.
template <int kOff>
struct BulkStage {
  static_assert(kOff % 8 == 0, "barrier alignment");
  static constexpr int kBytes = 16;  // barrier, parity word, failure flag
  // bounded wait: a poll that sees nothing suspends about 3.75 us on a GB300
  // (hines_check_bounded_wait measures it), so about one second in all, far
  // beyond any real copy latency
  static constexpr int kWaitPolls = 1 << 18;
  __device__ static uint64_t* barrier(unsigned char* wbase) { return reinterpret_cast<uint64_t*>(wbase + kOff); }
  __device__ static unsigned* words(unsigned char* wbase) { return reinterpret_cast<unsigned*>(barrier(wbase) + 1); }
  // once per warp, before its first task
  __device__ static void init(unsigned char* wbase, int lane) {
    if (lane == 0) {
      mbar_init(barrier(wbase));
      words(wbase)[0] = 0u;  // parity of the next phase
      words(wbase)[1] = 0u;  // a wait of this warp has run out
    }
    __syncwarp();
  }
  // one arrival with the expected bytes, then the copies.  Every lane fences
  // its earlier ordinary accesses first: the buffer's previous contents, and
  // factors this warp wrote in an earlier chunk of the same task, which the
  // copies may read.
  template <int N>
  __device__ static void issue(unsigned char* wbase, int lane, unsigned bytes, void* d0, const void* s0,
                               void* d1 = nullptr, const void* s1 = nullptr, void* d2 = nullptr,
                               const void* s2 = nullptr) {
    fence_async();
    __syncwarp();
    if (lane == 0) {
      uint64_t* bar = barrier(wbase);
      mbar_expect_tx(bar, N * bytes);
      if (bytes > 0) {
        bulk_g2s(d0, s0, bytes, bar);
        if (N > 1) bulk_g2s(d1, s1, bytes, bar);
        if (N > 2) bulk_g2s(d2, s2, bytes, bar);
      }
    }
  }
  // every lane waits for the staged copies; a wait that runs out raises the
  // plan's timeout status and goes on (no access leaves its buffer), and the
  // warp's later waits poll only once, so that a failed launch ends within
  // about a second instead of a second per chunk
  __device__ static void wait(const DevPlan& Pl, unsigned char* wbase, int lane) {
    unsigned* w = words(wbase);
    const unsigned parity = w[0];
    const bool ok = mbar_wait(barrier(wbase), parity, w[1] ? 1 : kWaitPolls);
    if (!ok && lane == 0 && Pl.status) atomicCAS(Pl.status, 0, (int)HINES_ERR_TIMEOUT);
    __syncwarp();
    if (lane == 0) {
      w[0] = parity ^ 1u;
      if (!ok) w[1] = 1u;
    }
    __syncwarp();
  }
};

// ============================================================================
// Compensated mode: FP32 inputs, double-float arithmetic from FP32 error-free
// transformations, FP64 solution.  The elimination leaves, per compartment k,
// the two double-float numbers the substitution needs, y_k = B_k / D_k and
// g_k = u_k / D_k (D, B: the eliminated pivot and right-hand side), written
// in the chunk's block order of the solver layout (16 bytes a slot, each row
// a contiguous run); per piece its contribution to the parent.  The
// substitution stages the block with 16-byte copies and runs
// x_k = y_k - g_k x_{k+1} from the proximal row (x of the parent's distal
// compartment) to the distal one: no inputs are read again.
// ============================================================================
template <bool kPk, int P>
struct CompMode {
  using V = typename VOf<P>::type;
  using G = Geo<P>;
  static constexpr bool kPacked = kPk;
  static constexpr bool kNeedsBlk = true;
  static constexpr int kPer = P;
  struct Args {
    const float* d;
    const float* u;
    const float* b;
    double* x;
  };
  // a staging buffer: elimination, d, u, b (3 words a slot); substitution,
  // the factor block (4 words a slot, the FP64 solution written over its
  // first two); then the block's row table
  static constexpr int kArr = 3 * G::kSlots * 4, kFac = G::kSlots * 16;
  static constexpr int kTab = kArr > kFac ? kArr : kFac;
  static constexpr int kStageBytes = kTab + 80;
  static constexpr int kStages = 1;
  // contiguous blocks (the factor block; d, u, b in the solver layout) are
  // staged by bulk copies (BulkStage, its barrier after the caches)
  static constexpr bool kBulk = true;
  static constexpr int kCslot = 0, kCx = 2 * G::kChunk * 16, kBar = kCx + 2 * G::kChunk * 8;
  static constexpr int kCacheBytes = kBar + 16;
  static constexpr int kWarpBytes = kStages * kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = kSmemPerSm / (kWarps * kWarpBytes) < 12 ? kSmemPerSm / (kWarps * kWarpBytes) : 12;
  static_assert(kStages == 1 && kStageBytes % 16 == 0, "one staging buffer, 16-byte aligned");
  using Bulk = BulkStage<kStageBytes + kBar>;

  __device__ static bool bulk_staged(int visit) { return kBulk && (visit == 1 || kPk); }
  __device__ static void init_warp(unsigned char* wbase, int lane) {
    if (kBulk) Bulk::init(wbase, lane);
  }

  __device__ static void stage(const DevPlan& Pl, const Args& A, int visit, Meta<P>& m, int n, int lane,
                               unsigned char* buf, const Prev& pv) {
    int* tab = reinterpret_cast<int*>(buf + kTab);
    build_row_table<P>(m.L, lane, tab);
    const int e = tab[kL];
    if (visit == 1) {
      if (kBulk) {
        Bulk::template issue<1>(buf, lane, (unsigned)e * 16u, buf, static_cast<const float4*>(Pl.ff4) + m.blk);
      } else {
        stage_block(reinterpret_cast<float4*>(buf), static_cast<const float4*>(Pl.ff4), m.blk, e, lane);
        cp_commit();
      }
      // the parent's solution, unless the predecessor chunk's cache holds it
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        const int loc = q.ppos - pv.c0;
        if (q.len > 0 && q.pcomp >= 0 && !(loc >= 0 && loc < pv.n))
          m.xpre[h].ff = static_cast<const float2*>(Pl.xlast)[q.ppos];
      }
      return;
    }
    float* sd = reinterpret_cast<float*>(buf);
    float* su = sd + G::kSlots;
    float* sb = su + G::kSlots;
    if (kPk) {
      const long long blk = __shfl_sync(kFull, m.p[0].first, 0);
      if (kBulk) {
        // whole 16-byte words: the block's padding (blocks start on multiples
        // of 4 slots, and the layout's length is one) completes the last
        Bulk::template issue<3>(buf, lane, (unsigned)((e + 3) & ~3) * 4u, sd, A.d + blk, su, A.u + blk, sb,
                                A.b + blk);
        return;
      }
      stage_block(sd, A.d, blk, e, lane);
      stage_block(su, A.u, blk, e, lane);
      stage_block(sb, A.b, blk, e, lane);
    } else {
      for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
        const int q = nidx<P>(row, i);
        cp_async4(&sd[q], A.d + g);
        cp_async4(&su[q], A.u + g);
        cp_async4(&sb[q], A.b + g);
      });
    }
    cp_commit();
  }

  __device__ static void compute(const DevPlan& Pl, const Args&, int visit, int c0, int n, int lane,
                                 const Meta<P>& m, unsigned char* buf, const Prev& pv, unsigned char* cache, int cur) {
    float4* cslot = reinterpret_cast<float4*>(cache + kCslot);  // [2][kChunk] contributions
    float2* cx = reinterpret_cast<float2*>(cache + kCx);        // [2][kChunk] distal solutions
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    float4* slot = static_cast<float4*>(Pl.cd);
    float2* xlast = static_cast<float2*>(Pl.xlast);
    if (bulk_staged(visit)) Bulk::wait(Pl, buf, lane);
    const int L = m.L;
    if (L == 0) return;
    const int me = P * lane;
    // the second piece's distal row (it joins the chain there); L: none
    const int delta = P == 2 ? L - m.p[P - 1].len : 0;
    if (visit == 0) {
      const float* sd = reinterpret_cast<const float*>(buf);
      const float* su = sd + G::kSlots;
      const float* sb = su + G::kSlots;
      float4* fac = static_cast<float4*>(Pl.ff4) + m.blk;
      const Rows<kPk, P> rows{tab};
      float d0h[P], d0l[P], b0h[P], b0l[P];
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        d0h[h] = 1.f;
        d0l[h] = b0h[h] = b0l[h] = 0.f;
        if (q.len == 0) continue;
        const int idx = rows.slot(L - q.len, me + h);
        ff Dv = {sd[idx], 0.f}, Bv = {sb[idx], 0.f};
        for (int c = 0; c < q.nchild; ++c) {
          const int cp = child_pos(Pl, q, c);
          const int loc = cp - pv.c0;
          const float4 v = (loc >= 0 && loc < pv.n) ? cslot[pv.which * G::kChunk + loc] : slot_load(slot + cp, q);
          Dv = ff_sub(Dv, v.x, v.y);
          Bv = ff_sub(Bv, v.z, v.w);
        }
        d0h[h] = Dv.h;
        d0l[h] = Dv.l;
        b0h[h] = Bv.h;
        b0l[h] = Bv.l;
      }
      FFV<V> D{vpack<P>(d0h), vpack<P>(d0l)}, B{vpack<P>(b0h), vpack<P>(b0l)};
      // row r: g = u / D, y = B / D into the factor block; then the chain to row r + 1
#pragma unroll
      for (int r = 0; r < kL - 1; ++r) {
        if (r < L - 1) {
          const V uk = ldv(su, rows.slot(r, me), V{});
          const FFV<V> g = vdiv_f(uk, D);
          const FFV<V> y = vdiv(B, D);
          const int f0 = tab[r] + me;
#pragma unroll
          for (int h = 0; h < P; ++h)
            fac[f0 + h] = make_float4(vget(y.h, h), vget(y.l, h), vget(g.h, h), vget(g.l, h));
          const FFV<V> fu = vmul_f(g, uk);
          const FFV<V> fb = vmul_ff(g, B);
          const int i1 = rows.slot(r + 1, me);
          D = vsub_dom(ldv(sd, i1, V{}), fu.h, fu.l);
          B = vsub_ff(ldv(sb, i1, V{}), fb.h, fb.l);
          if constexpr (P == 2) {
            if (r + 1 == delta) {
              D = {vset_hi(D.h, d0h[1]), vset_hi(D.l, d0l[1])};
              B = {vset_hi(B.h, b0h[1]), vset_hi(B.l, b0l[1])};
            }
          }
        }
      }
      // the proximal row: its factor, and the contribution to the parent (a
      // root's solution is its y, the factor's first number)
      const V uk = ldv(su, rows.slot(L - 1, me), V{});
      const FFV<V> g = vdiv_f(uk, D);
      const FFV<V> y = vdiv(B, D);
      const FFV<V> fu = vmul_f(g, uk);
      const FFV<V> fb = vmul_ff(g, B);
      const int f0 = tab[L - 1] + me;
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const bool root = m.p[h].pcomp < 0;  // a cell's root: no coupling to a parent
        fac[f0 + h] = make_float4(vget(y.h, h), vget(y.l, h), root ? 0.f : vget(g.h, h), root ? 0.f : vget(g.l, h));
        if (m.p[h].len == 0 || root) continue;
        const float4 out = make_float4(vget(fu.h, h), vget(fu.l, h), vget(fb.h, h), vget(fb.l, h));
        slot[c0 + me + h] = out;
        cslot[cur * G::kChunk + me + h] = out;
      }
      return;
    }
    // substitution: x = y - g x_parent from the proximal row down; the FP64
    // solution goes over the slot's first two words
    float4* sf = reinterpret_cast<float4*>(buf);
    float xph[P], xpl[P];
#pragma unroll
    for (int h = 0; h < P; ++h) {
      const Piece& q = m.p[h];
      xph[h] = xpl[h] = 0.f;
      if (q.len > 0 && q.pcomp >= 0) {
        const int loc = q.ppos - pv.c0;
        const float2 t = (loc >= 0 && loc < pv.n) ? cx[pv.which * G::kChunk + loc] : m.xpre[h].ff;
        xph[h] = t.x;
        xpl[h] = t.y;
      }
    }
    FFV<V> X{vpack<P>(xph), vpack<P>(xpl)};
    float xbh = 0.f, xbl = 0.f;  // the second piece's distal solution
#pragma unroll
    for (int r = kL - 1; r >= 0; --r) {
      if (r < L) {
        const int q = tab[r] + me;
        float yh[P], yl[P], gh[P], gl[P];
#pragma unroll
        for (int h = 0; h < P; ++h) {
          const float4 f = sf[q + h];
          yh[h] = f.x;
          yl[h] = f.y;
          gh[h] = f.z;
          gl[h] = f.w;
        }
        const FFV<V> gx = vmul_ff(FFV<V>{vpack<P>(gh), vpack<P>(gl)}, X);
        X = vsub_ffff(FFV<V>{vpack<P>(yh), vpack<P>(yl)}, gx.h, gx.l);
#pragma unroll
        for (int h = 0; h < P; ++h)
          reinterpret_cast<double*>(sf + q + h)[0] = ff_to_double(vget(X.h, h), vget(X.l, h));
        if constexpr (P == 2) {
          if (r == delta) {
            xbh = f2_hi(X.h);
            xbl = f2_hi(X.l);
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < P; ++h) {
      if (m.p[h].len == 0) continue;
      const float2 xo = h == 0 ? make_float2(vget(X.h, 0), vget(X.l, 0)) : make_float2(xbh, xbl);
      xlast[c0 + me + h] = xo;
      cx[cur * G::kChunk + me + h] = xo;
    }
  }

  __device__ static void copy_out(const DevPlan&, const Args& A, int visit, const Meta<P>& m, int n, int lane,
                                  unsigned char* buf) {
    if (visit == 0) return;
    const double* sx = reinterpret_cast<const double*>(buf);  // two per slot: the solution, then g
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    if (kPk) {
      const long long blk = __shfl_sync(kFull, m.p[0].first, 0);
      const int e = tab[kL];
      for (int s = lane; s < e; s += 32) A.x[blk + s] = sx[2 * s];
      return;
    }
    for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) { A.x[g] = sx[2 * (tab[row] + i)]; });
  }
};

// ============================================================================
// Factor mode (FP64, FP32, passive cable): the elimination leaves, per
// compartment, the reciprocal eliminated diagonal and the eliminated
// right-hand side; the substitution reads them back.  FP64 writes the pair
// as 16 bytes into the plan's factor block, in the chunk's block order of the
// solver layout (each row a contiguous run), and the substitution stages it
// with bulk copies in either layout; FP32 writes the reciprocal to the
// workspace at natural positions and the right-hand side in place (the
// refinement reads that factor).  In cable mode
// the system is rebuilt while staging (Section 1's implicit-Euler system):
// d_i = s_i (1 + theta dt g_i) + sum of a over the edges at i (a = -u),
// b_i = s_i V_i + s_i dt g_i (E - (1 - theta) V_i).
// The lane's pieces are handled one after the other in the same loop step
// (no packed FP64 instructions exist), their rows aligned as in the compensated
// mode; a piece's rows before its distal row are skipped.
// ============================================================================
// kReuse: the elimination of a new right-hand side with the factor a previous
// solve of the same plan and matrix left in the workspace (the reciprocal
// eliminated diagonal): only b is eliminated (the refinement's correction
// solves; passive-cable steps after the first, the matrix being constant).
// kBlk: FP64 keeps its factor in block order (else at natural positions, as
// FP32 always does).
template <typename T, bool kCable, bool kPk, int P, bool kReuse = false, bool kBlk = true>
struct FactorMode {
  using G = Geo<P>;
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
  static constexpr bool kBF = kBlk && sizeof(T) == 8;  // the factor in block order (FP64)
  static constexpr bool kNeedsBlk = kBF;
  static constexpr int kPer = P;
  struct Args {
    const T* d;
    const T* u;
    const T* s;  // cable: s, g
    const T* g;
    T* x;        // right-hand side in, solution out (cable: V in, V out)
    T dt, E, theta;
    bool rhs_from_V;
    const T* rhs = nullptr;  // non-null: the right-hand side is read from here (x receives the solution)
  };
  // a staging buffer: d (or the factor), u, b, then the row table (solver layout)
  static constexpr int kTab = 3 * G::kSlots * (int)sizeof(T);
  static constexpr int kStageBytes = kTab + 80;
  // FP64 chunks are large and the FP64 pipe is slow: one staging buffer, so
  // that more warps share an SM; FP32 with one piece per lane: two
  static constexpr int kStages = (sizeof(T) == 4 && P == 1) ? 2 : 1;
  static constexpr int kCslot = 0, kCx = 2 * G::kChunk * 2 * (int)sizeof(T);
  static constexpr int kBar = kCx + 2 * G::kChunk * (int)sizeof(T);
  static constexpr int kCacheBytes = kBar + (kBF ? 16 : 0);
  static constexpr int kWarpBytes = kStages * kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = kSmemPerSm / (kWarps * kWarpBytes);
  // the factor block is staged by bulk copies (FP64 has one staging buffer)
  static constexpr bool kBulk = kBF;
  static_assert(!kBF || (kStages == 1 && kStageBytes % 16 == 0), "one staging buffer, 16-byte aligned");
  using Bulk = BulkStage<kStageBytes + kBar>;
  __device__ static void init_warp(unsigned char* wbase, int lane) {
    if (kBulk) Bulk::init(wbase, lane);
  }
  __device__ static double2* factor_block(const DevPlan& Pl) { return static_cast<double2*>(Pl.ff4); }

  // Section 1's implicit-Euler system, each part in the fewest operations:
  // the diagonal less the compartment's own edge to its parent,
  // s (1 + theta dt g) - a_own, in one FMA (a cell's root, which has no such
  // edge, adds its u back: the same operations in both layouts), and the
  // right-hand side s (V + dt g (E - (1 - theta) V)) (theta = 1: s (V + dt E g))
  __device__ static T cable_diag_edge(const Args& A, T si, T gi, T ui) {
    return fma(si, fma(A.theta * A.dt, gi, T(1)), -ui);
  }
  __device__ static T cable_rhs(const Args& A, T si, T gi, T vi) {
    if (A.theta == T(1)) return si * fma(A.dt * A.E, gi, vi);
    return si * fma(A.dt * gi, fma(A.theta - T(1), vi, A.E), vi);
  }

  __device__ static void stage(const DevPlan& Pl, const Args& A, int visit, Meta<P>& m, int n, int lane,
                               unsigned char* buf, const Prev& pv) {
    T* sd = reinterpret_cast<T*>(buf);
    T* su = sd + G::kSlots;
    T* sb = su + G::kSlots;
    const T* fac = static_cast<const T*>(Pl.fac);
    if (visit == 1) {
      // the parent's solution, unless the predecessor chunk's cache holds it
      // (a chunk staged before its predecessor is computed finds that
      // predecessor's solutions in the cache, so it never reads them here)
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        const int loc = q.ppos - pv.c0;
        if (q.len > 0 && q.pcomp >= 0 && !(loc >= 0 && loc < pv.n)) pre_set(m.xpre[h], A.x[q.pcomp]);
      }
    }
    if constexpr (kBF) {
      int* tab = reinterpret_cast<int*>(buf + kTab);
      build_row_table<P>(m.L, lane, tab);
      const int e = tab[kL];
      const long long blk = kPk ? __shfl_sync(kFull, m.p[0].first, 0) : 0;
      if (visit == 1) {
        // the factor block (reciprocal pivot, eliminated right-hand side) over
        // the first two arrays, u in the third
        Bulk::template issue<1>(buf, lane, (unsigned)e * 16u, buf, factor_block(Pl) + m.blk);
        if (kPk) {
          stage_block(sb, A.u, blk, e, lane);
        } else {
          for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
            cp_async(&sb[nidx<P>(row, i)], A.u + g);
          });
        }
        cp_commit();
        return;
      }
      if (kReuse) {
        // the stored reciprocal pivots from the block, u, and b rebuilt
        const double* rp = reinterpret_cast<const double*>(factor_block(Pl) + m.blk);
        if (kPk) {
          for (int i = lane; i < e; i += 32) cp_async(&sd[i], rp + 2 * i);
          stage_block(su, A.u, blk, e, lane);
          for (int i = lane; i < e; i += 32) {
            const long long g = blk + i;
            const T vi = A.x[g];
            sb[i] = A.rhs_from_V ? cable_rhs(A, A.s[g], A.g[g], vi) : vi;
          }
        } else {
          for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
            const int q = nidx<P>(row, i);
            cp_async(&sd[q], rp + 2 * (tab[row] + i));
            cp_async(&su[q], A.u + g);
            const T vi = A.x[g];
            sb[q] = A.rhs_from_V ? cable_rhs(A, A.s[g], A.g[g], vi) : vi;
          });
        }
        cp_commit();
        return;
      }
    }
    if (kPk) {
      int* tab = reinterpret_cast<int*>(buf + kTab);
      if constexpr (!kBF) build_row_table<P>(m.L, lane, tab);
      const long long blk = __shfl_sync(kFull, m.p[0].first, 0);
      const int e = tab[kL];
      if (kCable && visit == 0) {
        // the block's rows in place; every diagonal loses its own edge here,
        // and compute() gives it back to a cell's root compartment (known there)
        if (kReuse) {  // the stored factor; only the right-hand side is rebuilt
          stage_block(sd, fac, blk, e, lane);
          stage_block(su, A.u, blk, e, lane);
        }
        for (int i = lane; i < e; i += 32) {
          const long long g = blk + i;
          const T vi = A.x[g];
          if (kReuse) {
            sb[i] = A.rhs_from_V ? cable_rhs(A, A.s[g], A.g[g], vi) : vi;
          } else {
            const T si = A.s[g], gi = A.g[g], ui = A.u[g];
            sd[i] = cable_diag_edge(A, si, gi, ui);
            su[i] = ui;
            sb[i] = A.rhs_from_V ? cable_rhs(A, si, gi, vi) : vi;
          }
        }
      } else {
        stage_block(sd, (visit == 1 || kReuse) ? fac : A.d, blk, e, lane);
        stage_block(su, A.u, blk, e, lane);
        stage_block(sb, (visit == 0 && A.rhs) ? A.rhs : static_cast<const T*>(A.x), blk, e, lane);
      }
      cp_commit();
      return;
    }
    if (visit == 1 || !kCable) {
      const T* dsrc = (visit == 1 || kReuse) ? fac : A.d;
      const T* bsrc = (visit == 0 && A.rhs) ? A.rhs : A.x;
      for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
        const int q = nidx<P>(row, i);
        cp_async(&sd[q], dsrc + g);
        cp_async(&su[q], A.u + g);
        cp_async(&sb[q], bsrc + g);
      });
    } else if (kReuse) {  // cable, stored factor: only the right-hand side is rebuilt
      for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
        const int q = nidx<P>(row, i);
        cp_async(&sd[q], fac + g);
        cp_async(&su[q], A.u + g);
        const T vi = A.x[g];
        sb[q] = A.rhs_from_V ? cable_rhs(A, A.s[g], A.g[g], vi) : vi;
      });
    } else {
      // the own edge to the parent comes off every diagonal but a cell root's
      for_chunk_elements(m, n, lane, [&](int i, int t, int row, long long g, bool root) {
        const T si = A.s[g], gi = A.g[g], ui = A.u[g], vi = A.x[g];
        T dd = cable_diag_edge(A, si, gi, ui);
        if (root && t == 0) dd += ui;  // a cell's root: no edge to a parent
        const int q = nidx<P>(row, i);
        sd[q] = dd;
        su[q] = ui;
        sb[q] = A.rhs_from_V ? cable_rhs(A, si, gi, vi) : vi;
      });
    }
    cp_commit();
  }

  __device__ static void compute(const DevPlan& Pl, const Args& A, int visit, int c0, int n, int lane,
                                 const Meta<P>& m, unsigned char* buf, const Prev& pv, unsigned char* cache, int cur) {
    T* sd = reinterpret_cast<T*>(buf);
    T* su = sd + G::kSlots;
    T* sb = su + G::kSlots;
    T* cslot = reinterpret_cast<T*>(cache + kCslot);  // [2][kChunk][2] contributions
    T* cx = reinterpret_cast<T*>(cache + kCx);        // [2][kChunk] distal solutions
    T* slot = static_cast<T*>(Pl.cd);                 // [nb][2]
    const int* tab = reinterpret_cast<const int*>(buf + kTab);
    const Rows<kPk, P> rows{tab};
    if (kBulk && visit == 1) Bulk::wait(Pl, buf, lane);
    const int L = m.L;
    if (L == 0) return;
    const int me = P * lane;
    double2* bf = kBF ? factor_block(Pl) + m.blk : nullptr;  // the chunk's factor block
    int first_row[P];  // each piece's distal row
#pragma unroll
    for (int h = 0; h < P; ++h) first_row[h] = m.p[h].len > 0 ? L - m.p[h].len : kL;
    if (visit == 0) {
      if (kPk && kCable && !kReuse) {
        // solver layout: a cell's root compartment (the proximal compartment
        // of a root piece, row L - 1) gets back the edge staging took off
#pragma unroll
        for (int h = 0; h < P; ++h) {
          if (m.p[h].len > 0 && m.p[h].pcomp < 0) {
            const int i = rows.slot(L - 1, me + h);
            sd[i] += su[i];
          }
        }
      }
      T D[P], B[P];
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        D[h] = T(1);
        B[h] = T(0);
        if (q.len == 0) continue;
        const int idx = rows.slot(first_row[h], me + h);
        if (!kReuse) D[h] = sd[idx];
        B[h] = sb[idx];
        for (int c = 0; c < q.nchild; ++c) {
          const int cp = child_pos(Pl, q, c);
          const int loc = cp - pv.c0;
          const bool local = loc >= 0 && loc < pv.n;
          if (!kReuse) D[h] -= local ? cslot[(pv.which * G::kChunk + loc) * 2] : slot_load(slot + 2 * cp, q);
          B[h] -= local ? cslot[(pv.which * G::kChunk + loc) * 2 + 1] : slot_load(slot + 2 * cp + 1, q);
        }
      }
      // rows from the distal end: store the reciprocal pivot (or, reusing the
      // factor, read it) and the eliminated right-hand side, then pass the
      // chain on; at the proximal row leave the contribution to the parent
#pragma unroll
      for (int r = 0; r < kL - 1; ++r) {
        if (r < L - 1) {
          const int i = rows.slot(r, me);
#pragma unroll
          for (int h = 0; h < P; ++h) {
            if (r < first_row[h]) continue;
            const T uk = su[i + h];
            const T rr = kReuse ? sd[i + h] : rcp_solve(D[h]);
            if constexpr (kBF) {
              bf[tab[r] + me + h] = make_double2(rr, B[h]);
            } else {
              if (!kReuse) sd[i + h] = rr;
              sb[i + h] = B[h];
            }
            const T f = uk * rr;
            const int i1 = rows.slot(r + 1, me + h);
            if (!kReuse) {
              D[h] = sd[i1] - f * uk;
              if (kCable) D[h] -= uk;  // the edge to the chain child
            }
            B[h] = sb[i1] - f * B[h];
          }
        }
      }
      T c0v[P], c1v[P];
      {
        const int i = rows.slot(L - 1, me);
#pragma unroll
        for (int h = 0; h < P; ++h) {
          c0v[h] = c1v[h] = T(0);
          if (m.p[h].len == 0) continue;
          const T uk = su[i + h];
          const T rr = kReuse ? sd[i + h] : rcp_solve(D[h]);
          if constexpr (kBF) bf[tab[L - 1] + me + h] = make_double2(rr, B[h]);  // a root's x is B rr
          else if (!kReuse) sd[i + h] = rr;
          if (m.p[h].pcomp >= 0) {
            const T f = uk * rr;
            if constexpr (!kBF) sb[i + h] = B[h];
            c0v[h] = kReuse ? T(0) : (kCable ? f * uk + uk : f * uk);
            c1v[h] = f * B[h];
          } else if constexpr (!kBF) {
            sb[i + h] = B[h] * rr;  // solve root
          }
        }
      }
#pragma unroll
      for (int h = 0; h < P; ++h) {
        if (m.p[h].len == 0) continue;
        const int pos = c0 + me + h;
        slot[2 * pos] = c0v[h];
        slot[2 * pos + 1] = c1v[h];
        cslot[(cur * G::kChunk + me + h) * 2] = c0v[h];
        cslot[(cur * G::kChunk + me + h) * 2 + 1] = c1v[h];
      }
      return;
    }
    T xp[P];
#pragma unroll
    for (int h = 0; h < P; ++h) {
      const Piece& q = m.p[h];
      xp[h] = T(0);
      if (q.len > 0 && q.pcomp >= 0) {
        const int loc = q.ppos - pv.c0;
        xp[h] = (loc >= 0 && loc < pv.n) ? cx[pv.which * G::kChunk + loc] : pre_get(m.xpre[h], T{});
      }
    }
    if constexpr (kBF) {
      // the staged block: (reciprocal pivot, eliminated right-hand side) per
      // slot in block order, u in the third array; x goes over the pivot
      const double2* fb = reinterpret_cast<const double2*>(buf);
      double* sx = reinterpret_cast<double*>(buf);
#pragma unroll
      for (int r = kL - 1; r >= 0; --r) {
        if (r < L) {
          const int i = rows.slot(r, me), q = tab[r] + me;
#pragma unroll
          for (int h = 0; h < P; ++h) {
            if (r < first_row[h]) continue;
            const double2 f = fb[q + h];
            const T xi = (m.p[h].pcomp < 0 && r == L - 1) ? f.y * f.x : (f.y - sb[i + h] * xp[h]) * f.x;
            sx[2 * (q + h)] = xi;
            xp[h] = xi;
          }
        }
      }
    } else {
#pragma unroll
      for (int r = kL - 1; r >= 0; --r) {
        if (r < L) {
          const int i = rows.slot(r, me);
#pragma unroll
          for (int h = 0; h < P; ++h) {
            if (r < first_row[h]) continue;
            const T xi = (m.p[h].pcomp < 0 && r == L - 1) ? sb[i + h] : (sb[i + h] - su[i + h] * xp[h]) * sd[i + h];
            sb[i + h] = xi;
            xp[h] = xi;
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < P; ++h)
      if (m.p[h].len > 0) cx[cur * G::kChunk + me + h] = xp[h];
  }

  __device__ static void copy_out(const DevPlan& Pl, const Args& A, int visit, const Meta<P>& m, int n, int lane,
                                  unsigned char* buf) {
    const T* sd = reinterpret_cast<const T*>(buf);
    const T* sb = sd + 2 * G::kSlots;
    T* fac = static_cast<T*>(Pl.fac);
    if constexpr (kBF) {
      // the elimination wrote its factor block directly; the substitution
      // left x over each slot's pivot
      if (visit == 0) return;
      const double* sx = reinterpret_cast<const double*>(buf);
      const int* tab = reinterpret_cast<const int*>(buf + kTab);
      if (kPk) {
        const long long blk = __shfl_sync(kFull, m.p[0].first, 0);
        const int e = tab[kL];
        for (int s = lane; s < e; s += 32) A.x[blk + s] = sx[2 * s];
        return;
      }
      for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) { A.x[g] = sx[2 * (tab[row] + i)]; });
      return;
    }
    if (kPk) {
      const int* tab = reinterpret_cast<const int*>(buf + kTab);
      const long long blk = __shfl_sync(kFull, m.p[0].first, 0);
      const int e = tab[kL];
      for (int s = lane; s < e; s += 32) {
        if (visit == 0 && !kReuse) fac[blk + s] = sd[s];
        A.x[blk + s] = sb[s];
      }
      return;
    }
    for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
      const int q = nidx<P>(row, i);
      if (visit == 0 && !kReuse) fac[g] = sd[q];
      A.x[g] = sb[q];
    });
  }
};

// ============================================================================
// Refinement mode (natural layout): one step of iterative refinement on the
// FP32 factor that a FactorMode<float> solve of the same plan left in the
// workspace (the reciprocal pivots).  The elimination visit forms the
// residual r = b - A x of the current x (the FP32 inputs taken exactly;
// products and sums by error-free transformations, so that r keeps FP32
// accuracy although it is tiny next to b) and eliminates it with the stored
// factor, as the FP32 solve eliminated b.  A compartment's residual needs its
// parent's x (the next row; at the proximal row, the parent piece's distal
// compartment) and its children's (the previous row; at a piece's distal
// row, the child pieces pass their products u x up with their
// contributions).  The substitution visit solves for the correction c with
// the same factor and writes x + c.  kIn: x is FP32 (0) or a double-float
// pair (1); kOut: x + c as a pair (0, for another step) or in FP64 (1).
// ============================================================================
template <int P, int kIn, int kOut>
struct RefineMode {
  using V = typename VOf<P>::type;
  using G = Geo<P>;
  static constexpr bool kPacked = false;
  static constexpr bool kNeedsBlk = false;
  static constexpr int kPer = P;
  struct Args {
    const float* d;
    const float* u;
    const float* b;
    const void* x;     // kIn 0: float[n]; 1: float2[n]
    float* rw;         // the eliminated residual (the correction's right-hand side)
    void* xo;          // kOut 0: float2[n]; 1: double[n]
    float* bcorr;      // per piece (branch id): largest |c| of this step
  };
  // staged words: d, u, b (visit 1: the eliminated residual), the factor, and
  // x as pairs (two words per slot; FP32 x uses the first)
  static constexpr int kTab = 6 * G::kSlots * 4;
  static constexpr int kStageBytes = kTab + 80;
  // one staging buffer: six staged arrays per chunk, and twice as many warps
  // per SM hide the loads better than a second buffer at half the warps
  // (measured on the 228M-compartment batch: 12.6 ms against 13.7 ms per
  // one-step solve)
  static constexpr int kStages = 1;
  static constexpr int kCslot = 0, kCx = 2 * G::kChunk * 16;
  static constexpr int kCacheBytes = kCx + 2 * G::kChunk * 8;
  static constexpr int kWarpBytes = kStages * kStageBytes + kCacheBytes;
  static constexpr int kMinBlocks = kSmemPerSm / (kWarps * kWarpBytes);
  static constexpr bool kBulk = false;
  __device__ static void init_warp(unsigned char*, int) {}

  __device__ static void stage(const DevPlan& Pl, const Args& A, int visit, Meta<P>& m, int n, int lane,
                               unsigned char* buf, const Prev& pv) {
    float* sd = reinterpret_cast<float*>(buf);
    float* su = sd + G::kSlots;
    float* sb = su + G::kSlots;
    float* sf = sb + G::kSlots;
    float* sx = sf + G::kSlots;  // [2 * kSlots]
    const float* fac = static_cast<const float*>(Pl.fac);
    if (visit == 1) {
      // the parent's correction, unless the predecessor chunk's cache holds it
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        const int loc = q.ppos - pv.c0;
        if (q.len > 0 && q.pcomp >= 0 && !(loc >= 0 && loc < pv.n))
          m.xpre[h].f = static_cast<const float2*>(Pl.xlast)[q.ppos].x;
      }
    }
    for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
      const int q = nidx<P>(row, i);
      if (visit == 0) {
        cp_async4(&sd[q], A.d + g);
        cp_async4(&sb[q], A.b + g);
      } else {
        cp_async4(&sb[q], A.rw + g);
      }
      cp_async4(&su[q], A.u + g);
      cp_async4(&sf[q], fac + g);
      if (kIn == 1)
        cp_async8(&sx[2 * q], static_cast<const float2*>(A.x) + g);
      else
        cp_async4(&sx[2 * q], static_cast<const float*>(A.x) + g);
    });
    cp_commit();
  }

  // x of a row: the lane's P values as a double-float pair
  __device__ static FFV<V> ldx(const float* sx, int idx) {
    if constexpr (P == 2) {
      const float4 v = *reinterpret_cast<const float4*>(sx + 2 * idx);
      return {f2_make(v.x, v.z), kIn == 1 ? f2_make(v.y, v.w) : f2_make(0.f, 0.f)};
    } else {
      const float2 v = *reinterpret_cast<const float2*>(sx + 2 * idx);
      return {v.x, kIn == 1 ? v.y : 0.f};
    }
  }
  // x of a compartment in global memory (a parent's distal compartment)
  __device__ static float2 gx(const Args& A, long long g) {
    if (kIn == 1) return static_cast<const float2*>(A.x)[g];
    return make_float2(static_cast<const float*>(A.x)[g], 0.f);
  }
  // acc -= t, accumulating the rounding errors of the leading parts exactly
  // (two-sum) and everything else in the second word
  __device__ static void acc_sub(V& s, V& e, const FFV<V>& t) {
    const V s1 = vsub(s, t.h);
    const V bb = vsub(s1, s);
    const V err = vsub(vsub(s, vsub(s1, bb)), vadd(t.h, bb));
    e = vadd(e, vsub(err, t.l));
    s = s1;
  }

  __device__ static void compute(const DevPlan& Pl, const Args& A, int visit, int c0, int n, int lane,
                                 const Meta<P>& m, unsigned char* buf, const Prev& pv, unsigned char* cache, int cur) {
    float* sd = reinterpret_cast<float*>(buf);
    float* su = sd + G::kSlots;
    float* sb = su + G::kSlots;
    float* sf = sb + G::kSlots;
    float* sx = sf + G::kSlots;
    float4* cslot = reinterpret_cast<float4*>(cache + kCslot);  // [2][kChunk] (u x up, eliminated residual up)
    float* cx = reinterpret_cast<float*>(cache + kCx);          // [2][kChunk] distal corrections
    float4* slot = static_cast<float4*>(Pl.cd);
    float2* xlast = static_cast<float2*>(Pl.xlast);
    const int L = m.L;
    if (L == 0) return;
    const int me = P * lane;
    const int delta = P == 2 ? L - m.p[P - 1].len : 0;
    // a cell's root has no parent: its coupling is not part of the system
#pragma unroll
    for (int h = 0; h < P; ++h)
      if (m.p[h].len > 0 && m.p[h].pcomp < 0) su[nidx<P>(L - 1, me + h)] = 0.f;
    if (visit == 0) {
      // per piece: the parent's x, and the children's u x and eliminated residuals
      float xph[P], xpl[P], crh[P], crl[P], ce[P];
#pragma unroll
      for (int h = 0; h < P; ++h) {
        const Piece& q = m.p[h];
        xph[h] = xpl[h] = crh[h] = crl[h] = ce[h] = 0.f;
        if (q.len == 0) continue;
        if (q.pcomp >= 0) {
          const float2 t = gx(A, q.pcomp);
          xph[h] = t.x;
          xpl[h] = t.y;
        }
        ff acc = {0.f, 0.f};
        for (int c = 0; c < q.nchild; ++c) {
          const int cp = child_pos(Pl, q, c);
          const int loc = cp - pv.c0;
          const float4 v = (loc >= 0 && loc < pv.n) ? cslot[pv.which * G::kChunk + loc] : slot_load(slot + cp, q);
          acc = ff_sub(acc, -v.x, -v.y);
          ce[h] += v.z;
        }
        crh[h] = acc.h;
        crl[h] = acc.l;
      }
      FFV<V> tc{vpack<P>(crh), vpack<P>(crl)};  // the children's u x (at a distal row), or the chain child's
      V cev = vpack<P>(ce);                    // the children's eliminated residuals times their multipliers
      FFV<V> un{}, en{};                       // the proximal row's u x and eliminated residual times multiplier
#pragma unroll
      for (int r = 0; r < kL; ++r) {
        if (r < L) {
          if constexpr (P == 2) {
            if (r > 0 && r == delta) {
              tc = {vset_hi(tc.h, crh[1]), vset_hi(tc.l, crl[1])};
              cev = vset_hi(cev, ce[1]);
            }
          }
          const int i = nidx<P>(r, me);
          const V dk = ldv(sd, i, V{}), uk = ldv(su, i, V{}), bk = ldv(sb, i, V{}), fk = ldv(sf, i, V{});
          const FFV<V> xk = ldx(sx, i);
          FFV<V> xn;
          if (r < L - 1)
            xn = ldx(sx, nidx<P>(r + 1, me));
          else
            xn = {vpack<P>(xph), vpack<P>(xpl)};
          V s = bk, e = vsplat(0.f, V{});
          acc_sub(s, e, vmul_f(xk, dk));
          acc_sub(s, e, vmul_f(xn, uk));
          acc_sub(s, e, tc);
          const V rp = vsub(vadd(s, e), cev);  // the residual, less the children's eliminated residuals
          stv(sb, i, rp);
          tc = vmul_f(xk, uk);                 // this row's u x, for the next row (or the parent)
          cev = vmul(vmul(uk, fk), rp);        // multiplier u / pivot times the eliminated residual
          un = tc;
          en = {cev, vsplat(0.f, V{})};
        }
      }
#pragma unroll
      for (int h = 0; h < P; ++h) {
        if (m.p[h].len == 0) continue;
        const float4 out = m.p[h].pcomp >= 0 ? make_float4(vget(un.h, h), vget(un.l, h), vget(en.h, h), 0.f)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
        slot[c0 + me + h] = out;
        cslot[cur * G::kChunk + me + h] = out;
      }
      return;
    }
    // the correction from the proximal row down, and x + c
    float cph[P];
#pragma unroll
    for (int h = 0; h < P; ++h) {
      const Piece& q = m.p[h];
      cph[h] = 0.f;
      if (q.len > 0 && q.pcomp >= 0) {
        const int loc = q.ppos - pv.c0;
        cph[h] = (loc >= 0 && loc < pv.n) ? cx[pv.which * G::kChunk + loc] : m.xpre[h].f;
      }
    }
    V cp = vpack<P>(cph);
    float cm[P], cb = 0.f;
#pragma unroll
    for (int h = 0; h < P; ++h) cm[h] = 0.f;
#pragma unroll
    for (int r = kL - 1; r >= 0; --r) {
      if (r < L) {
        const int i = nidx<P>(r, me);
        const V uk = ldv(su, i, V{}), rk = ldv(sb, i, V{}), fk = ldv(sf, i, V{});
        const V c = vmul(vfma(vneg(uk), cp, rk), fk);
        const FFV<V> xk = ldx(sx, i);
        // x + c: two-sum of the leading parts, the rest into the low word
        const V s = vadd(xk.h, c);
        const V bb = vsub(s, xk.h);
        const V err = vadd(vsub(xk.h, vsub(s, bb)), vsub(c, bb));
        const FFV<V> xn = vrenorm(s, vadd(err, xk.l));
#pragma unroll
        for (int h = 0; h < P; ++h) {
          const int q = i + h;
          if (r >= L - m.p[h].len) cm[h] = fmaxf(cm[h], fabsf(vget(c, h)));
          if (kOut == 1)
            reinterpret_cast<double*>(sx)[q] = ff_to_double(vget(xn.h, h), vget(xn.l, h));
          else
            reinterpret_cast<float2*>(sx)[q] = make_float2(vget(xn.h, h), vget(xn.l, h));
        }
        if constexpr (P == 2) {
          if (r == delta) cb = f2_hi(c);
        }
        cp = c;
      }
    }
#pragma unroll
    for (int h = 0; h < P; ++h) {
      if (m.p[h].len == 0) continue;
      const float cd = h == 0 ? vget(cp, 0) : cb;
      const int pos = c0 + me + h;
      xlast[pos] = make_float2(cd, 0.f);
      cx[cur * G::kChunk + me + h] = cd;
      if (A.bcorr) A.bcorr[Pl.pos_branch[pos]] = cm[h];
    }
  }

  __device__ static void copy_out(const DevPlan&, const Args& A, int visit, const Meta<P>& m, int n, int lane,
                                  unsigned char* buf) {
    const float* sd = reinterpret_cast<const float*>(buf);
    const float* sb = sd + 2 * G::kSlots;
    const float* sx = sd + 4 * G::kSlots;
    for_chunk_elements(m, n, lane, [&](int i, int, int row, long long g, bool) {
      const int q = nidx<P>(row, i);
      if (visit == 0)
        A.rw[g] = sb[q];
      else if (kOut == 1)
        static_cast<double*>(A.xo)[g] = reinterpret_cast<const double*>(sx)[q];
      else
        static_cast<float2*>(A.xo)[g] = reinterpret_cast<const float2*>(sx)[q];
    });
  }
};

// ============================================================================
// Task driver
// ============================================================================
// Position in a task's chunk sequence: chunks deepest-first for the
// elimination (visit 0), root-side first for the substitution (visit 1); a
// level of more than one chunk's pieces is several chunks.
struct Pos {
  int visit, l, c0, n;  // visit == ve: past the end
};

template <int W>
__device__ __forceinline__ Pos pos_level(int visit, int l, const int32_t* lp) {
  const int c0 = __ldg(lp + l), e = __ldg(lp + l + 1) - c0;
  return {visit, l, c0, e < W ? e : W};
}

template <int W>
__device__ __forceinline__ Pos pos_next(Pos p, const int32_t* lp, int nl, int ve) {
  const int end = __ldg(lp + p.l + 1);
  if (p.c0 + W < end) {
    p.c0 += W;
    p.n = end - p.c0 < W ? end - p.c0 : W;
    return p;
  }
  if (p.visit == 0) {
    if (p.l > 0) return pos_level<W>(0, p.l - 1, lp);
    if (ve == 1) return {ve, 0, 0, 0};
    return pos_level<W>(1, 0, lp);
  }
  if (p.l + 1 < nl) return pos_level<W>(1, p.l + 1, lp);
  return {ve, 0, 0, 0};
}

template <class M>
__device__ void run_task(const DevPlan& Pl, const typename M::Args& A, int t, int code, int lane,
                         unsigned char* wbase) {
  constexpr int P = M::kPer, W = 32 * P;
  const int nl = Pl.task_nlvl[t];
  const int32_t* lp = Pl.tlvl_ptr + Pl.task_lvl_off[t];
  const int vb = code == 2 ? 1 : 0, ve = code == 1 ? 1 : 2;
  unsigned char* cache = wbase + M::kStages * M::kStageBytes;
  auto buf = [wbase](int which) { return wbase + (M::kStages == 2 ? which : 0) * M::kStageBytes; };
  auto meta = [&](const Pos& p) {
    return load_meta<M::kPacked, P>(Pl, p.c0, p.n, lane, p.visit < ve, M::kNeedsBlk);
  };
  // metadata runs two chunks ahead; with two staging buffers the next chunk
  // is staged while this one is computed, with one right after this one's
  // results are out
  Pos cur = pos_level<W>(vb, vb == 0 ? nl - 1 : 0, lp);
  Meta<P> m_cur = meta(cur);
  Prev pv{0, 0, 0};  // last chunk of the previous level in this sweep
  M::stage(Pl, A, cur.visit, m_cur, cur.n, lane, buf(0), pv);
  Pos nxt = pos_next<W>(cur, lp, nl, ve);
  Meta<P> m_nxt = meta(nxt);
  int which = 0;
  while (cur.visit < ve) {
    cp_wait_all();
    __syncwarp();
    // nothing of the substitution is read before the elimination has
    // finished: its first chunks reuse positions the elimination is still
    // writing (and read the folded states it leaves)
    const bool crossing = nxt.visit != cur.visit;
    // predecessor of the next chunk: the last chunk of the level before its level, same sweep
    const Prev pn = crossing ? Prev{0, 0, 0} : nxt.l != cur.l ? Prev{cur.c0, cur.n, cur.l & 1} : pv;
    // (staged before this chunk is computed: a mode with two buffers reads
    // nothing in stage that this chunk writes)
    if (M::kStages == 2 && nxt.visit < ve && !crossing)
      M::stage(Pl, A, nxt.visit, m_nxt, nxt.n, lane, buf(which ^ 1), pn);
    const Pos nn = nxt.visit < ve ? pos_next<W>(nxt, lp, nl, ve) : nxt;
    Meta<P> m_nn = meta(nn);
    M::compute(Pl, A, cur.visit, cur.c0, cur.n, lane, m_cur, buf(which), pv, cache, cur.l & 1);
    __syncwarp();
    M::copy_out(Pl, A, cur.visit, m_cur, cur.n, lane, buf(which));
    __syncwarp();
    if (crossing && nxt.visit < ve) {
      // the substitution reads what the elimination wrote (through L2)
      __threadfence();
      __syncwarp();
      m_nxt = meta(nxt);
      m_nn = meta(nn);
    }
    if (nxt.visit < ve && (crossing || M::kStages == 1))
      M::stage(Pl, A, nxt.visit, m_nxt, nxt.n, lane, buf(which ^ 1), pn);
    pv = pn;
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
  M::init_warp(wbase, lane);
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
  int per_sm = 0;
  const size_t smem = (size_t)kWarps * M::kWarpBytes;
  cudaError_t e = cudaFuncSetAttribute(k_units<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_units<M>, 32 * kWarps, smem);
  if (e != cudaSuccess) return e;
  *grid = P.sms * (per_sm > 0 ? per_sm : 1);
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

// ---- the modes' instantiations for P pieces per lane --------------------------
template <int PL>
struct UnitKernels {
  using F64 = FactorMode<double, false, false, PL>;
  using F32 = FactorMode<float, false, false, PL>;
  using Cable = FactorMode<double, true, false, PL>;
  using Comp = CompMode<false, PL>;
  using PkF64 = FactorMode<double, false, true, PL>;
  using PkF32 = FactorMode<float, false, true, PL>;
  using PkComp = CompMode<true, PL>;
  using PkCable = FactorMode<double, true, true, PL>;
  using F32Reuse = FactorMode<float, false, false, PL, true>;
  using CableReuse = FactorMode<double, true, false, PL, true>;
  using PkCableReuse = FactorMode<double, true, true, PL, true>;
  // the FP64 kinds with the factor at natural positions (small batches)
  using F64N = FactorMode<double, false, false, PL, false, false>;
  using CableN = FactorMode<double, true, false, PL, false, false>;
  using PkF64N = FactorMode<double, false, true, PL, false, false>;
  using PkCableN = FactorMode<double, true, true, PL, false, false>;
  using CableReuseN = FactorMode<double, true, false, PL, true, false>;
  using PkCableReuseN = FactorMode<double, true, true, PL, true, false>;
  using R32to2 = RefineMode<PL, 0, 0>;
  using R32to64 = RefineMode<PL, 0, 1>;
  using R2to2 = RefineMode<PL, 1, 0>;
  using R2to64 = RefineMode<PL, 1, 1>;

  static cudaError_t prepare(DevPlan& P) {
    cudaError_t e = grid_of<F64>(P, &P.grid[0]);
    if (e == cudaSuccess) e = grid_of<F32>(P, &P.grid[1]);
    if (e == cudaSuccess) e = grid_of<Cable>(P, &P.grid[2]);
    if (e == cudaSuccess) e = grid_of<Comp>(P, &P.grid[3]);
    if (e == cudaSuccess) e = grid_of<PkF64>(P, &P.grid[4]);
    if (e == cudaSuccess) e = grid_of<PkF32>(P, &P.grid[5]);
    if (e == cudaSuccess) e = grid_of<PkComp>(P, &P.grid[6]);
    if (e == cudaSuccess) e = grid_of<PkCable>(P, &P.grid[7]);
    int g_reuse = 0;  // same footprint as the plain modes
    if (e == cudaSuccess) e = grid_of<F32Reuse>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<CableReuse>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<PkCableReuse>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<R32to2>(P, &P.grid_refine);
    if (e == cudaSuccess) e = grid_of<R32to64>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<R2to2>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<R2to64>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<F64N>(P, &P.grid_nf[0]);
    if (e == cudaSuccess) e = grid_of<CableN>(P, &P.grid_nf[1]);
    if (e == cudaSuccess) e = grid_of<PkF64N>(P, &P.grid_nf[2]);
    if (e == cudaSuccess) e = grid_of<PkCableN>(P, &P.grid_nf[3]);
    if (e == cudaSuccess) e = grid_of<CableReuseN>(P, &g_reuse);
    if (e == cudaSuccess) e = grid_of<PkCableReuseN>(P, &g_reuse);
    return e;
  }

  static cudaError_t run(const DevPlan& P, const UnitCall& c, cudaStream_t s) {
    const double* d8 = static_cast<const double*>(c.d);
    const double* u8 = static_cast<const double*>(c.u);
    const double* s8 = static_cast<const double*>(c.s);
    const double* g8 = static_cast<const double*>(c.g);
    double* x8 = static_cast<double*>(c.x);
    const float* d4 = static_cast<const float*>(c.d);
    const float* u4 = static_cast<const float*>(c.u);
    const float* b4 = static_cast<const float*>(c.b);
    float* x4 = static_cast<float*>(c.x);
    const double th = (double)c.theta;
    const bool blk = P.fp64_blocks != 0;
    switch (c.op) {
      case UnitOp::F64:
        if (!blk) return launch_phases<F64N>(P, {d8, u8, nullptr, nullptr, x8, 0.0, 0.0, 0.0, false}, P.grid_nf[0], s);
        return launch_phases<F64>(P, {d8, u8, nullptr, nullptr, x8, 0.0, 0.0, 0.0, false}, P.grid[0], s);
      case UnitOp::F32:
        return launch_phases<F32>(P, {d4, u4, nullptr, nullptr, x4, 0.f, 0.f, 0.f, false,
                                      static_cast<const float*>(c.rhs)}, P.grid[1], s);
      case UnitOp::F32Resolve:
        return launch_phases<F32Reuse>(P, {nullptr, u4, nullptr, nullptr, x4, 0.f, 0.f, 0.f, false}, P.grid[1], s);
      case UnitOp::Comp:
        return launch_phases<Comp>(P, {d4, u4, b4, x8}, P.grid[3], s);
      case UnitOp::Cable:
        if (!blk)
          return launch_phases<CableN>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, c.rhs_from_V}, P.grid_nf[1], s);
        return launch_phases<Cable>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, c.rhs_from_V}, P.grid[2], s);
      case UnitOp::CableReuse:
        if (!blk) return launch_phases<CableReuseN>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, true}, P.grid_nf[1], s);
        return launch_phases<CableReuse>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, true}, P.grid[2], s);
      case UnitOp::PkF64:
        if (!blk)
          return launch_phases<PkF64N>(P, {d8, u8, nullptr, nullptr, x8, 0.0, 0.0, 0.0, false}, P.grid_nf[2], s);
        return launch_phases<PkF64>(P, {d8, u8, nullptr, nullptr, x8, 0.0, 0.0, 0.0, false}, P.grid[4], s);
      case UnitOp::PkF32:
        return launch_phases<PkF32>(P, {d4, u4, nullptr, nullptr, x4, 0.f, 0.f, 0.f, false}, P.grid[5], s);
      case UnitOp::PkComp:
        return launch_phases<PkComp>(P, {d4, u4, b4, x8}, P.grid[6], s);
      case UnitOp::PkCable:
        if (!blk)
          return launch_phases<PkCableN>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, c.rhs_from_V}, P.grid_nf[3], s);
        return launch_phases<PkCable>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, c.rhs_from_V}, P.grid[7], s);
      case UnitOp::PkCableReuse:
        if (!blk)
          return launch_phases<PkCableReuseN>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, true}, P.grid_nf[3], s);
        return launch_phases<PkCableReuse>(P, {nullptr, u8, s8, g8, x8, c.dt, c.E, th, true}, P.grid[7], s);
      case UnitOp::Refine32to2:
        return launch_phases<R32to2>(P, {d4, u4, b4, c.rhs, c.rw, c.x, c.bcorr}, P.grid_refine, s);
      case UnitOp::Refine32to64:
        return launch_phases<R32to64>(P, {d4, u4, b4, c.rhs, c.rw, c.x, c.bcorr}, P.grid_refine, s);
      case UnitOp::Refine2to2:
        return launch_phases<R2to2>(P, {d4, u4, b4, c.rhs, c.rw, c.x, c.bcorr}, P.grid_refine, s);
      case UnitOp::Refine2to64:
        return launch_phases<R2to64>(P, {d4, u4, b4, c.rhs, c.rw, c.x, c.bcorr}, P.grid_refine, s);
    }
    return cudaErrorInvalidValue;
  }
};

}  // namespace
}  // namespace hines
