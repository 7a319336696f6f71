// Warp-task kernels of the batched Hines solver, sm_103a.
//
// One warp owns one task (a cell, or several small cells packed so that no
// level holds more than 32 branches; Section 4).  The warp walks the task's
// levels -- deepest first for the elimination, root level first for the
// substitution (Section 3) -- in chunks of at most 32 branches of one level,
// one branch per lane.  Branches of a level are sorted by length so the 32
// chains of a chunk have similar lengths (Section 4, Fig. 4.1), and no branch
// is longer than 32 compartments (the planner cuts longer ones; Section 6).
//
// A chunk is staged in shared memory in the interleaved layout of Section 5:
// step k of the chain of lane j (k = 0 at the distal end) lives at row k,
// column j, with the column XOR-swizzled by k so that the warp's copy of one
// branch (lanes over k) and the lanes' chain steps (lanes over j) are both
// free of bank conflicts.  Inside a branch the parent of compartment i is
// i - 1 (Section 5); at the proximal end the elimination produces one
// contribution to the parent compartment (Listing 2's parent lookup), kept in
// a per-branch slot that the parent's lane folds in when its level comes.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hines.h"
#include "kernels.h"

namespace hines {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSlots = 1024;  // 32 lanes x 32 steps

__device__ __forceinline__ int sidx(int k, int j) { return (k << 5) + (j ^ (k & 31)); }

// ---- asynchronous global -> shared copies (LDGSTS) --------------------------
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
  if constexpr (sizeof(T) == 8)
    cp_async8(smem, gmem);
  else
    cp_async4(smem, gmem);
}

// ---- reciprocals -------------------------------------------------------------
// FP64: hardware approximation of the high word, then two Newton steps.
__device__ __forceinline__ double rcp_t(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
__device__ __forceinline__ float rcp_t(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---- double-float arithmetic from FP32 error-free transformations -------------
// A value is an unevaluated pair hi + lo; every product and sum below uses the
// _rn intrinsics so the compiler cannot contract them into FMAs, which would
// break the exactness the transformations rely on.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff ff_renorm(float h, float l) {  // fast two-sum, |h| >= |l|
  const float s = __fadd_rn(h, l);
  return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
// x - (yh + yl), two-sum on the leading parts
__device__ __forceinline__ ff ff_sub(ff x, float yh, float yl) {
  const float s = __fsub_rn(x.h, yh);
  const float bb = __fsub_rn(s, x.h);
  const float e = __fadd_rn(__fsub_rn(x.h, __fsub_rn(s, bb)), __fsub_rn(-yh, bb));
  return ff_renorm(s, __fadd_rn(e, __fsub_rn(x.l, yl)));
}
// f = u / d for an FP32 u
__device__ __forceinline__ ff ff_div_f(float u, ff d) {
  const float r = rcp_t(d.h);
  const float F = __fmul_rn(u, r);
  float t = fmaf(-F, d.h, u);
  t = fmaf(-F, d.l, t);
  return ff_renorm(F, __fmul_rn(t, r));
}
// n / d
__device__ __forceinline__ ff ff_div(ff n, ff d) {
  const float r = rcp_t(d.h);
  const float X = __fmul_rn(n.h, r);
  float t = fmaf(-X, d.h, n.h);
  t = __fadd_rn(t, n.l);
  t = fmaf(-X, d.l, t);
  return ff_renorm(X, __fmul_rn(t, r));
}
// f * u for an FP32 u (exact leading product plus the lo term)
__device__ __forceinline__ ff ff_mul_f(ff f, float u) {
  const float P = __fmul_rn(f.h, u);
  float p = fmaf(f.h, u, -P);
  p = fmaf(f.l, u, p);
  return {P, p};
}
// f * b
__device__ __forceinline__ ff ff_mul(ff f, ff b) {
  const float Q = __fmul_rn(f.h, b.h);
  float q = fmaf(f.h, b.h, -Q);
  q = fmaf(f.h, b.l, q);
  q = fmaf(f.l, b.h, q);
  return {Q, q};
}

// hi + lo rounded to FP64 with integer operations on the bit pattern (no FP64
// pipe): hi is widened exactly by re-biasing its exponent, lo is scaled to
// units of the last place of that double and added to the bit pattern.  Rare
// cases (tiny or huge hi, large lo, a sum crossing below hi's binade) take the
// FP64 path.
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
  const uint32_t hb = __float_as_uint(hi);
  const uint32_t ex = (hb >> 23) & 0xFFu;
  if (ex < 64u || ex > 253u) return (double)hi + (double)lo;
  const float q = __fmul_rn(lo, __uint_as_float((306u - ex) << 23));  // lo / ulp_double(hi), exact
  if (!(fabsf(q) < 1073741824.0f)) return (double)hi + (double)lo;
  int32_t k = __float2int_rn(q);
  if (hb & 0x80000000u) k = -k;  // bits hold the magnitude
  if (k < 0 && (hb & 0x7FFFFFu) == 0u) return (double)hi + (double)lo;
  const uint64_t db = ((uint64_t)(hb & 0x80000000u) << 32) | ((uint64_t)(ex + 896u) << 52) |
                      ((uint64_t)(hb & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)(db + (uint64_t)(int64_t)k));
}

// ---- task / chunk iteration -------------------------------------------------
struct Chunk {
  int visit;  // 0: leaves-to-root elimination, 1: root-to-leaves substitution, 2: done
  int l;      // level
  int c0;     // first position of the chunk
};

__device__ __forceinline__ Chunk chunk_first(const int32_t* lp, int nl) { return {0, nl - 1, __ldg(lp + nl - 1)}; }

__device__ __forceinline__ Chunk chunk_next(Chunk c, const int32_t* lp, int nl) {
  if (c.visit == 2) return c;
  c.c0 += 32;
  if (c.c0 < __ldg(lp + c.l + 1)) return c;
  if (c.visit == 0) {
    if (c.l == 0) return {1, 0, __ldg(lp)};
    c.l -= 1;
  } else {
    c.l += 1;
    if (c.l == nl) return {2, nl, 0};
  }
  c.c0 = __ldg(lp + c.l);
  return c;
}

__device__ __forceinline__ int chunk_size(Chunk c, const int32_t* lp) {
  const int e = __ldg(lp + c.l + 1) - c.c0;
  return e < 32 ? e : 32;
}

struct LaneMeta {
  long long first, pcomp;
  int len, cbeg, cend, ppos;
};

__device__ __forceinline__ LaneMeta load_meta(const DevPlan& P, Chunk c, int nbc, int lane) {
  LaneMeta m{0, -1, 0, 0, 0, -1};
  if (c.visit < 2 && lane < nbc) {
    const BrMetaT t = P.tmeta[c.c0 + lane];
    m.first = t.first;
    m.pcomp = t.pcomp;
    m.len = t.len;
    m.cbeg = t.cbeg;
    m.cend = t.cend;
    m.ppos = t.ppos;
  }
  return m;
}

__device__ __forceinline__ int next_task(const DevPlan& P, int lane) {
  int t = 0;
  if (lane == 0) t = atomicAdd(P.counter, 1);
  return __shfl_sync(kFull, t, 0);
}

// ============================================================================
// Factor-storing solve (FP64, FP32, passive cable): the elimination writes the
// reciprocal eliminated diagonal to the workspace and the eliminated
// right-hand side in place; the substitution reads them back.
// ============================================================================
template <typename T, bool kCable>
struct FactorArgs {
  const T* d;   // plain: diagonal
  const T* b;   // plain: right-hand side (== x)
  const T* s;   // cable: s, g
  const T* g;
  const T* u;
  T* x;         // in/out
  T dt, E, theta;
  bool rhs_from_V;
};

template <typename T, bool kCable>
__device__ __forceinline__ void stage_backward(const FactorArgs<T, kCable>& A, const LaneMeta& m, int nbc, int lane,
                                               T* sd, T* su, T* sb) {
  if constexpr (!kCable) {
    for (int j = 0; j < nbc; ++j) {
      const long long fj = __shfl_sync(kFull, m.first, j);
      const int lj = __shfl_sync(kFull, m.len, j);
      if (lane < lj) {
        const int q = sidx(lj - 1 - lane, j);
        cp_async(&sd[q], A.d + fj + lane);
        cp_async(&su[q], A.u + fj + lane);
        cp_async(&sb[q], A.b + fj + lane);
      }
    }
    cp_commit();
    cp_wait_all();
  } else {
#pragma unroll 4
    for (int j = 0; j < nbc; ++j) {
      const long long fj = __shfl_sync(kFull, m.first, j);
      const int lj = __shfl_sync(kFull, m.len, j);
      const bool root_branch = __shfl_sync(kFull, m.pcomp, j) < 0;
      if (lane < lj) {
        const long long i = fj + lane;
        const T si = A.s[i], gi = A.g[i], ui = A.u[i], vi = A.x[i];
        T dd = si * (T(1) + A.theta * A.dt * gi);
        if (!(root_branch && lane == 0)) dd -= ui;  // own edge to the parent
        const T bb = A.rhs_from_V ? si * vi + si * A.dt * gi * (A.E - (T(1) - A.theta) * vi) : vi;
        const int q = sidx(lj - 1 - lane, j);
        sd[q] = dd;
        su[q] = ui;
        sb[q] = bb;
      }
    }
  }
  __syncwarp();
}

template <typename T, bool kCable>
__global__ void __launch_bounds__(32) k_warp_factor(DevPlan P, FactorArgs<T, kCable> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sd = reinterpret_cast<T*>(smem_raw);
  T* su = sd + kSlots;
  T* sb = su + kSlots;
  const int lane = threadIdx.x;
  T* cd = static_cast<T*>(P.cd);  // per position: (diag, rhs) contribution pairs
  T* fac = static_cast<T*>(P.fac);
  for (int task = next_task(P, lane); task < P.n_wtasks; task = next_task(P, lane)) {
    const int nl = P.task_nlvl[task];
    const int32_t* lp = P.tlvl_ptr + P.task_lvl_off[task];
    for (Chunk c = chunk_first(lp, nl); c.visit < 2; c = chunk_next(c, lp, nl)) {
      const int nbc = chunk_size(c, lp);
      const LaneMeta m = load_meta(P, c, nbc, lane);
      const int pos = c.c0 + lane;
      if (c.visit == 0) {
        stage_backward<T, kCable>(A, m, nbc, lane, sd, su, sb);
        if (lane < nbc) {
          T D = sd[sidx(0, lane)], B = sb[sidx(0, lane)];
          for (int q = m.cbeg; q < m.cend; ++q) {
            const int cp = P.tchild[q];
            D -= cd[2 * cp];
            B -= cd[2 * cp + 1];
          }
          for (int k = 0; k < m.len - 1; ++k) {
            const T uk = su[sidx(k, lane)];
            const T r = rcp_t(D);
            sd[sidx(k, lane)] = r;
            sb[sidx(k, lane)] = B;
            const T f = uk * r;
            D = sd[sidx(k + 1, lane)] - f * uk;
            if (kCable) D -= uk;  // the edge to the chain child
            B = sb[sidx(k + 1, lane)] - f * B;
          }
          const int k = m.len - 1;
          const T r = rcp_t(D);
          sd[sidx(k, lane)] = r;
          if (m.pcomp >= 0) {
            sb[sidx(k, lane)] = B;
            const T uk = su[sidx(k, lane)];
            const T f = uk * r;
            cd[2 * pos] = kCable ? f * uk + uk : f * uk;
            cd[2 * pos + 1] = f * B;
          } else {
            sb[sidx(k, lane)] = B * r;  // solve root
          }
        }
        __syncwarp();
        for (int j = 0; j < nbc; ++j) {  // write the factor back
          const long long fj = __shfl_sync(kFull, m.first, j);
          const int lj = __shfl_sync(kFull, m.len, j);
          if (lane < lj) {
            const int q = sidx(lj - 1 - lane, j);
            fac[fj + lane] = sd[q];
            A.x[fj + lane] = sb[q];
          }
        }
      } else {
        for (int j = 0; j < nbc; ++j) {
          const long long fj = __shfl_sync(kFull, m.first, j);
          const int lj = __shfl_sync(kFull, m.len, j);
          if (lane < lj) {
            const int q = sidx(lj - 1 - lane, j);
            cp_async(&sd[q], fac + fj + lane);
            cp_async(&su[q], A.u + fj + lane);
            cp_async(&sb[q], A.x + fj + lane);
          }
        }
        cp_commit();
        cp_wait_all();
        __syncwarp();
        if (lane < nbc) {
          T xp = m.pcomp >= 0 ? A.x[m.pcomp] : T(0);
          for (int k = m.len - 1; k >= 0; --k) {
            const int q = sidx(k, lane);
            T xi;
            if (m.pcomp < 0 && k == m.len - 1)
              xi = sb[q];
            else
              xi = (sb[q] - su[q] * xp) * sd[q];
            sb[q] = xi;
            xp = xi;
          }
        }
        __syncwarp();
        for (int j = 0; j < nbc; ++j) {
          const long long fj = __shfl_sync(kFull, m.first, j);
          const int lj = __shfl_sync(kFull, m.len, j);
          if (lane < lj) A.x[fj + lane] = sb[sidx(lj - 1 - lane, j)];
        }
      }
      __syncwarp();
    }
  }
}

// ============================================================================
// Compensated solve: FP32 inputs, double-float arithmetic built from FP32
// error-free transformations, FP64 solution.  Nothing per compartment is kept
// between the two visits: the elimination leaves only per-branch
// contributions, and the substitution re-stages the chunk and recomputes its
// chains before substituting.  Staging is double buffered.
// ============================================================================
struct MixedBuf {
  float* d;
  float* u;
  float* b;
};

__device__ __forceinline__ void stage_mixed(const float* d, const float* u, const float* b, const LaneMeta& m,
                                            int nbc, int lane, MixedBuf B) {
  for (int j = 0; j < nbc; ++j) {
    const long long fj = __shfl_sync(kFull, m.first, j);
    const int lj = __shfl_sync(kFull, m.len, j);
    if (lane < lj) {
      const int q = sidx(lj - 1 - lane, j);
      cp_async4(&B.d[q], d + fj + lane);
      cp_async4(&B.u[q], u + fj + lane);
      cp_async4(&B.b[q], b + fj + lane);
    }
  }
  cp_commit();
}

__global__ void __launch_bounds__(32) k_warp_compensated(DevPlan P, const float* __restrict__ d,
                                                         const float* __restrict__ u, const float* __restrict__ b,
                                                         double* __restrict__ x) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* base = reinterpret_cast<float*>(smem_raw);
  auto buf = [base](int w) -> MixedBuf {
    float* p = base + w * 3 * kSlots;
    return {p, p + kSlots, p + 2 * kSlots};
  };
  float* se = base + 6 * kSlots;  // lo part of the eliminated diagonal
  float* sbl = base + 7 * kSlots; // lo part of the eliminated right-hand side
  const int lane = threadIdx.x;
  float4* slot = static_cast<float4*>(P.cd);   // per position: (diag contribution, rhs contribution) or root x
  float2* xlast = static_cast<float2*>(P.cb);  // per position: x at the branch's distal compartment
  for (int task = next_task(P, lane); task < P.n_wtasks; task = next_task(P, lane)) {
    const int nl = P.task_nlvl[task];
    const int32_t* lp = P.tlvl_ptr + P.task_lvl_off[task];
    Chunk cur = chunk_first(lp, nl);
    int ncur = chunk_size(cur, lp);
    LaneMeta mcur = load_meta(P, cur, ncur, lane);
    stage_mixed(d, u, b, mcur, ncur, lane, buf(0));
    Chunk nxt = chunk_next(cur, lp, nl);
    int nnxt = nxt.visit < 2 ? chunk_size(nxt, lp) : 0;
    LaneMeta mnxt = load_meta(P, nxt, nnxt, lane);
    int which = 0;
    while (cur.visit < 2) {
      cp_wait_all();
      __syncwarp();
      if (nxt.visit < 2) stage_mixed(d, u, b, mnxt, nnxt, lane, buf(which ^ 1));
      const Chunk nn = chunk_next(nxt, lp, nl);
      const int nnn = nn.visit < 2 ? chunk_size(nn, lp) : 0;
      const LaneMeta mnn = load_meta(P, nn, nnn, lane);
      const MixedBuf B = buf(which);
      const int pos = cur.c0 + lane;
      if (lane < ncur) {
        ff Dv = {B.d[sidx(0, lane)], 0.f}, Bv = {B.b[sidx(0, lane)], 0.f};
        for (int q = mcur.cbeg; q < mcur.cend; ++q) {
          const float4 v = slot[P.tchild[q]];
          Dv = ff_sub(Dv, v.x, v.y);
          Bv = ff_sub(Bv, v.z, v.w);
        }
        const bool store = cur.visit == 1;
        for (int k = 0; k < mcur.len - 1; ++k) {
          const int q = sidx(k, lane);
          if (store) {
            B.d[q] = Dv.h;
            se[q] = Dv.l;
            B.b[q] = Bv.h;
            sbl[q] = Bv.l;
          }
          const float uk = B.u[q];
          const ff f = ff_div_f(uk, Dv);
          const ff fu = ff_mul_f(f, uk);
          const ff fb = ff_mul(f, Bv);
          const int q1 = sidx(k + 1, lane);
          Dv = ff_sub({B.d[q1], 0.f}, fu.h, fu.l);
          Bv = ff_sub({B.b[q1], 0.f}, fb.h, fb.l);
        }
        const int kp = mcur.len - 1, qp = sidx(kp, lane);
        if (cur.visit == 0) {
          if (mcur.pcomp >= 0) {
            const float uk = B.u[qp];
            const ff f = ff_div_f(uk, Dv);
            const ff fu = ff_mul_f(f, uk);
            const ff fb = ff_mul(f, Bv);
            slot[pos] = make_float4(fu.h, fu.l, fb.h, fb.l);
          } else {
            const ff x0 = ff_div(Bv, Dv);  // solve root
            slot[pos] = make_float4(x0.h, x0.l, 0.f, 0.f);
          }
        } else {
          B.d[qp] = Dv.h;
          se[qp] = Dv.l;
          B.b[qp] = Bv.h;
          sbl[qp] = Bv.l;
          ff xp = {0.f, 0.f};
          if (mcur.pcomp >= 0) {
            const float2 t = xlast[mcur.ppos];
            xp = {t.x, t.y};
          }
          for (int k = kp; k >= 0; --k) {
            const int q = sidx(k, lane);
            ff xi;
            if (mcur.pcomp < 0 && k == kp) {
              const float4 t = slot[pos];
              xi = {t.x, t.y};
            } else {
              const float uk = B.u[q];
              const float M = __fmul_rn(uk, xp.h);
              float mm = fmaf(uk, xp.h, -M);
              mm = fmaf(uk, xp.l, mm);
              const ff num = ff_sub({B.b[q], sbl[q]}, M, mm);
              xi = ff_div(num, {B.d[q], se[q]});
            }
            B.d[q] = xi.h;
            se[q] = xi.l;
            xp = xi;
          }
          xlast[pos] = make_float2(xp.h, xp.l);
        }
      }
      __syncwarp();
      if (cur.visit == 1) {
        for (int j = 0; j < ncur; ++j) {
          const long long fj = __shfl_sync(kFull, mcur.first, j);
          const int lj = __shfl_sync(kFull, mcur.len, j);
          if (lane < lj) {
            const int q = sidx(lj - 1 - lane, j);
            x[fj + lane] = ff_to_double(B.d[q], se[q]);
          }
        }
        __syncwarp();
      }
      cur = nxt;
      ncur = nnxt;
      mcur = mnxt;
      nxt = nn;
      nnxt = nnn;
      mnxt = mnn;
      which ^= 1;
    }
  }
}

// ---- launch helpers ----------------------------------------------------------
template <typename K>
cudaError_t grid_for(K kernel, size_t smem, const DevPlan& P, int32_t* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, smem);
  if (e != cudaSuccess) return e;
  long long g = (long long)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  if (g > P.n_wtasks) g = P.n_wtasks;
  *grid = (int32_t)(g > 0 ? g : 1);
  return cudaSuccess;
}

template <typename T, bool kCable>
cudaError_t launch_factor(const DevPlan& P, const FactorArgs<T, kCable>& A, int grid, cudaStream_t s) {
  if (P.n_wtasks == 0) return cudaSuccess;
  const size_t smem = 3 * kSlots * sizeof(T);
  cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_warp_factor<T, kCable><<<grid, 32, smem, s>>>(P, A);
  return cudaGetLastError();
}

constexpr size_t kSmemComp = 8 * kSlots * sizeof(float);

}  // namespace

cudaError_t prepare_warp_kernels(DevPlan& P) {
  cudaError_t e = grid_for(k_warp_factor<double, false>, 3 * kSlots * sizeof(double), P, &P.grid_f64);
  if (e == cudaSuccess) e = grid_for(k_warp_factor<float, false>, 3 * kSlots * sizeof(float), P, &P.grid_f32);
  if (e == cudaSuccess) e = grid_for(k_warp_factor<double, true>, 3 * kSlots * sizeof(double), P, &P.grid_cable);
  if (e == cudaSuccess) e = grid_for(k_warp_compensated, kSmemComp, P, &P.grid_comp);
  return e;
}

cudaError_t launch_warp_solve_f64(const DevPlan& P, const double* d, const double* u, double* b, cudaStream_t s) {
  FactorArgs<double, false> A{d, b, nullptr, nullptr, u, b, 0.0, 0.0, 0.0, false};
  return launch_factor(P, A, P.grid_f64, s);
}

cudaError_t launch_warp_solve_f32(const DevPlan& P, const float* d, const float* u, float* b, cudaStream_t s) {
  FactorArgs<float, false> A{d, b, nullptr, nullptr, u, b, 0.f, 0.f, 0.f, false};
  return launch_factor(P, A, P.grid_f32, s);
}

cudaError_t launch_warp_cable(const DevPlan& P, const double* sv, const double* g, const double* u, double* V,
                              double dt, double E, int theta, bool rhs_from_V, cudaStream_t s) {
  FactorArgs<double, true> A{nullptr, nullptr, sv, g, u, V, dt, E, (double)theta, rhs_from_V};
  return launch_factor(P, A, P.grid_cable, s);
}

cudaError_t launch_warp_solve_compensated(const DevPlan& P, const float* d, const float* u, const float* b, double* x,
                                          cudaStream_t s) {
  if (P.n_wtasks == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.counter, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  k_warp_compensated<<<P.grid_comp, 32, kSmemComp, s>>>(P, d, u, b, x);
  return cudaGetLastError();
}

}  // namespace hines
