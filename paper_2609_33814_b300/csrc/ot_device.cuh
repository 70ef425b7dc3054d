// Device-side building blocks for the sm_103a sweep kernels: packed f32x2 arithmetic,
// three-input max, MUFU exp2, TMA bulk copies with mbarrier completion, and error-free
// floating-point transforms for the compensated (float-float) sweep.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "ot_exp2_poly.cuh"

namespace ot {

typedef unsigned long long u64;

// ---------------------------------------------------------------------------------------
// Packed pairs of FP32 (f32x2): one instruction issues two FP32 lane operations.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ u64 pk2(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void up2(u64 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// 2^x on the special-function unit (flush-to-zero for tiny results).
__device__ __forceinline__ float ex2_mufu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Exact 2^-k for an integer-valued float k >= 0 (0 when the result would be subnormal).
__device__ __forceinline__ float exp2_neg_int(float k) {
  int e = 127 - (int)k;
  return e > 0 ? __int_as_float(e << 23) : 0.0f;
}

// ---------------------------------------------------------------------------------------
// Error-free transforms (Knuth TwoSum, FMA-based TwoProd).  Used by the compensated sweep.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// ---------------------------------------------------------------------------------------
// mbarrier + bulk (TMA) copy, global -> shared, completion counted in bytes.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Acquire load / release store of a 64-bit counter at GPU scope (phase signals between CTAs of
// one launch; they also bypass the SM's L1, which is not coherent).
__device__ __forceinline__ long long ld_acquire(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(long long* p, long long v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Orders this thread's view of global memory (generic proxy) before its later bulk copies (async
// proxy): needed before a TMA copy reads data that another CTA of the same launch wrote.
__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Bounded wait: returns false after `limit` polls (the caller records an error and stops).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 2^x for a pair, on the FP32/INT pipes: x = n + f with n = round(x) (magic-number rounding),
// 2^f by the fitted polynomial (|f| <= 1/2), 2^n added into the exponent bits.  x is clamped to
// [-125, 126] so the result stays a normal float (an overflow still shows up as a huge value).
__device__ __forceinline__ u64 exp2_poly2(u64 v) {
  float lo, hi;
  up2(v, lo, hi);
  lo = fminf(fmaxf(lo, -125.0f), 126.0f);
  hi = fminf(fmaxf(hi, -125.0f), 126.0f);
  const u64 x = pk2(lo, hi);
  const u64 magic = pk2(12582912.0f, 12582912.0f);  // 1.5 * 2^23
  const u64 t = add2(x, magic);
  const u64 f = sub2(x, sub2(t, magic));
  u64 p = fma2(pk2(kExp2Poly[5], kExp2Poly[5]), f, pk2(kExp2Poly[4], kExp2Poly[4]));
  p = fma2(p, f, pk2(kExp2Poly[3], kExp2Poly[3]));
  p = fma2(p, f, pk2(kExp2Poly[2], kExp2Poly[2]));
  p = fma2(p, f, pk2(kExp2Poly[1], kExp2Poly[1]));
  p = fma2(p, f, pk2(kExp2Poly[0], kExp2Poly[0]));
  float t0, t1, p0, p1;
  up2(t, t0, t1);
  up2(p, p0, p1);
  p0 = __int_as_float(__float_as_int(p0) + (__float_as_int(t0) << 23));
  p1 = __int_as_float(__float_as_int(p1) + (__float_as_int(t1) << 23));
  return pk2(p0, p1);
}

}  // namespace ot
