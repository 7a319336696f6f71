// Device helpers shared by the solve kernels (internal to libhines).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"

namespace hines {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;
// ---- asynchronous global -> shared copies (LDGSTS) --------------------------
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {  // both 16-byte aligned
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// ---- bulk (TMA, one-dimensional) copies global -> shared, completing on a
// shared-memory barrier -------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// a barrier for one arriving thread (the copy's issuer) plus the copies' bytes
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// orders this thread's earlier ordinary memory accesses (shared and global)
// before later bulk copies: their reads of global data it wrote, and their
// writes into shared memory it used
__device__ __forceinline__ void fence_async() { asm volatile("fence.proxy.async;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// dst and src 16-byte aligned, bytes a positive multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// waits until the barrier's phase of the given parity has completed; false
// when `limit` polls did not see it (the caller reports a timeout)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int limit) {
  for (int k = 0; k < limit; ++k) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
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
// FP64: hardware approximation of the high word, then one cubically
// convergent correction (the series 1/x = r (1 + e + e^2 + ...) with
// e = 1 - x r, cut after e^2): an approximation good to about 2^-20 leaves a
// relative error near 2^-60, below FP64 rounding, in three FMAs where two
// Newton steps take four.  The FP64 pipe bounds the FP64 elimination on
// this part, so the FMA saved there is time saved.
__device__ __forceinline__ double rcp_t(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, fma(e, e, e), r);
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
// ---- one or two independent values per thread -------------------------------
// The solve kernels give a lane one or two branch pieces.  Their arithmetic is
// written once over a value type V: float for one piece, F2 for two, whose
// operations are the packed FP32 pair instructions of sm_100 and later (one
// instruction performs the operation on both halves, each rounded to nearest
// like its FP32 counterpart; no fusing or contraction happens across them).
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 f2_make(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f2_lo(F2 a) { return __uint_as_float((unsigned)a.v); }
__device__ __forceinline__ float f2_hi(F2 a) { return __uint_as_float((unsigned)(a.v >> 32)); }
__device__ __forceinline__ F2 vadd(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 vsub(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 vmul(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ F2 vneg(F2 a) { return vmul(a, f2_make(-1.f, -1.f)); }
__device__ __forceinline__ F2 vrcp(F2 a) { return f2_make(rcp_t(f2_lo(a)), rcp_t(f2_hi(a))); }
__device__ __forceinline__ F2 vsplat(float a, F2) { return f2_make(a, a); }

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float vrcp(float a) { return rcp_t(a); }
__device__ __forceinline__ float vsplat(float a, float) { return a; }

// Double-float over V: the same error-free transformations as ff above.
template <typename V>
struct FFV {
  V h, l;
};
// fast two-sum, |h| >= |l|
template <typename V>
__device__ __forceinline__ FFV<V> vrenorm(V h, V l) {
  const V s = vadd(h, l);
  return {s, vsub(l, vsub(s, h))};
}
// (x, 0) - (yh + yl) with a full two-sum on the leading parts
template <typename V>
__device__ __forceinline__ FFV<V> vsub_ff(V x, V yh, V yl) {
  const V s = vsub(x, yh);
  const V bb = vsub(s, x);
  const V e = vsub(vsub(x, vsub(s, bb)), vadd(yh, bb));
  return vrenorm(s, vsub(e, yl));
}
// (x, 0) - (yh + yl) when |x| >= |yh| (the diagonal chain of a diagonally
// dominant matrix: d_{i-1} > u_i^2 / d'_i), fast two-sum on the leading parts
template <typename V>
__device__ __forceinline__ FFV<V> vsub_dom(V x, V yh, V yl) {
  const V s = vsub(x, yh);
  const V e = vsub(vsub(x, s), yh);
  return vrenorm(s, vsub(e, yl));
}
// (x.h + x.l) - (yh + yl), full two-sum on the leading parts
template <typename V>
__device__ __forceinline__ FFV<V> vsub_ffff(FFV<V> x, V yh, V yl) {
  const V s = vsub(x.h, yh);
  const V bb = vsub(s, x.h);
  const V e = vsub(vsub(x.h, vsub(s, bb)), vadd(yh, bb));
  return vrenorm(s, vadd(e, vsub(x.l, yl)));
}
// u / D for a plain u: r = 1/D.h, F = u r, t = u - F D (exact leading part by
// FMA), quotient F + t r, renormalised.  nF = -F carries the sign so that
// both FMAs take their operands as they are.
template <typename V>
__device__ __forceinline__ FFV<V> vdiv_f(V u, FFV<V> D) {
  const V r = vrcp(D.h);
  const V F = vmul(u, r);
  const V nF = vneg(F);
  V t = vfma(nF, D.h, u);
  t = vfma(nF, D.l, t);
  return vrenorm(F, vmul(t, r));
}
// N / D
template <typename V>
__device__ __forceinline__ FFV<V> vdiv(FFV<V> N, FFV<V> D) {
  const V r = vrcp(D.h);
  const V X = vmul(N.h, r);
  const V nX = vneg(X);
  V t = vfma(nX, D.h, N.h);
  t = vadd(t, N.l);
  t = vfma(nX, D.l, t);
  return vrenorm(X, vmul(t, r));
}
// f * u for a plain u: the leading product, its exact error by FMA, plus f.l u
template <typename V>
__device__ __forceinline__ FFV<V> vmul_f(FFV<V> f, V u) {
  const V P = vmul(f.h, u);
  V p = vfma(f.h, u, vneg(P));
  p = vfma(f.l, u, p);
  return {P, p};
}
// f * b
template <typename V>
__device__ __forceinline__ FFV<V> vmul_ff(FFV<V> f, FFV<V> b) {
  const V Q = vmul(f.h, b.h);
  V q = vfma(f.h, b.h, vneg(Q));
  q = vfma(f.h, b.l, q);
  q = vfma(f.l, b.h, q);
  return {Q, q};
}

// hi + lo rounded to FP64 with integer operations on the bit pattern (no FP64
// pipe): hi is widened exactly by re-biasing its exponent, lo is scaled to
// units of the last place of that double and added to the bit pattern.  Rare
// cases (tiny or huge hi, large lo, a sum crossing below hi's binade) take an
// FP64 path kept out of line, so the compiler cannot evaluate it
// speculatively for every element.
static __device__ __noinline__ double ff_to_double_slow(float hi, float lo) { return (double)hi + (double)lo; }

__device__ __forceinline__ double ff_to_double(float hi, float lo) {
  const uint32_t hb = __float_as_uint(hi);
  const uint32_t ex = (hb >> 23) & 0xFFu;
  // lo / ulp_double(hi), signed against hi's magnitude: lo * (+-2^(179 - e)) with hi's sign
  const float q = __fmul_rn(lo, __uint_as_float(((306u - ex) << 23) | (hb & 0x80000000u)));
  const int32_t k = __float2int_rn(q);
  // out of line: hi tiny or huge (biased exponent outside [64, 253]), lo not
  // below hi's last place (or NaN), or a sum that drops below hi's binade
  const bool slow = (ex - 64u) > 189u || !(fabsf(q) < 1073741824.0f) || (k < 0 && (hb & 0x7FFFFFu) == 0u);
  if (slow) return ff_to_double_slow(hi, lo);
  // hi widened: exponent re-biased by 1023 - 127, mantissa moved up by 29 bits
  const uint32_t whi = (((hb & 0x7FFFFFFFu) >> 3) + (896u << 20)) | (hb & 0x80000000u);
  const uint64_t db = ((uint64_t)whi << 32) | (uint64_t)(hb << 29);
  return __longlong_as_double((long long)(db + (uint64_t)(int64_t)k));
}

}  // namespace dev
}  // namespace hines
