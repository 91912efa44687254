// Device helpers shared by the scattering kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include "plan.h"

namespace scatter {
namespace dev {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Phase arithmetic
// ---------------------------------------------------------------------------

// x - rint(x) for |x| < 2^22, exactly, on the FMA pipe.  (cvt.rni runs on a
// 16/clk/SM pipe on this GPU, the same rate as the MUFU sin/cos the kernels
// are bound by, so it is avoided in the inner loops.)  The add/sub of
// 1.5 * 2^23 rounds x to an integer in round-to-nearest-even.
// Order-preserving map of doubles to unsigned integers (atomicMin/Max on
// the bounding box) and its inverse.
__device__ __forceinline__ unsigned long long ordered(double x) {
  long long i = __double_as_longlong(x);
  return (unsigned long long)(i >= 0 ? (i ^ (long long)0x8000000000000000ULL) : ~i);
}
__device__ __forceinline__ double unordered(unsigned long long u) {
  long long i = (u & 0x8000000000000000ULL) ? (long long)(u ^ 0x8000000000000000ULL) : (long long)~u;
  return __longlong_as_double(i);
}

__device__ __forceinline__ float frac_rn(float x) {
  const float kMagic = 12582912.0f;  // 1.5 * 2^23
  const float n = __fsub_rn(__fadd_rn(x, kMagic), kMagic);
  return __fsub_rn(x, n);
}

// frac_rn(p) + (err + acc): a rounded value's fractional part, then its
// rounding error and a small addend
__device__ __forceinline__ float dev_frac_plus(float p, float err, float acc) {
  return frac_rn(p) + (err + acc);
}

// Exact-product phases for long crystals.  A phase s . x' computed with FP32
// products errs by up to |s . x'| 2^-24 cycles: below 128 cycles that is
// under 8e-6 cycles (5e-5 rad) per pair, well inside the FP32 paths' 1e-4;
// above it (crystals hundreds to thousands of cells long) the rounding of
// the products, structured along a lattice row, sets the noise floor of the
// map.  The kernels then restore each product's rounding error (exact by
// FMA) after its integer part is removed.
constexpr double kPhaseExactLim = 128.0;  // cycles

// True when |s . x'| + |c| can exceed kPhaseExactLim for positions inside
// `bbox` (ordered min xyz, max xyz) centred on `shift` with |s_d| <= smax_d;
// false without atoms or without a box.
__device__ __forceinline__ bool phase_needs_exact(const unsigned long long* bbox, const double* shift,
                                                  const float* smax) {
  if (!bbox) return false;
  double b = 0.5;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const unsigned long long lo = bbox[d], hi = bbox[3 + d];
    if (lo == ~0ULL || hi == 0ULL) return false;
    const double e = fmax(fabs(unordered(lo) - shift[d]), fabs(unordered(hi) - shift[d]));
    b += (double)smax[d] * (e + 1.0);
  }
  return b > kPhaseExactLim;
}

// x - rint(x) of a product a b with its rounding error restored: the pair
// (frac of the rounded product, exact error) summed into `acc`.
__device__ __forceinline__ float frac_product_plus(float a, float b, float acc) {
  const float p = a * b;
  return dev_frac_plus(p, fmaf(a, b, -p), acc);
}

// frac_product_plus for a double-float multiplier a + alo (alo the FP32
// rounding error of a, |alo| <= ulp(a)/2): the low part's product joins the
// rounding error.  Without it the multiplier's own rounding, |a| 2^-24 per
// component, errs by that much times |b| cycles, coherently for one point.
__device__ __forceinline__ float frac_product2_plus(float a, float alo, float b, float acc) {
  const float p = a * b;
  return dev_frac_plus(p, fmaf(alo, b, fmaf(a, b, -p)), acc);
}

// a b - rint(a b) with the product's rounding error restored (|result|
// <= 1/2 + 2^-24 |a b|): the argument of the per-call tables' sincospif
__device__ __forceinline__ float frac_of_product(float a, float b) {
  const float p = a * b;
  return (p - rintf(p)) + fmaf(a, b, -p);
}

// frac_of_product for a double-float multiplier a + alo
__device__ __forceinline__ float frac_of_product2(float a, float alo, float b) {
  const float p = a * b;
  return (p - rintf(p)) + fmaf(alo, b, fmaf(a, b, -p));
}

// Running sum as an unevaluated FP32 pair hi + lo (about 2^-44 relative to
// the partial sums, against FP64's 2^-53) on the FP32 pipe, for the places
// where an FP64 accumulator would issue at GB300's small FP64 rate.  Each
// addition is Knuth's branch-free TwoSum: the exact rounding error of
// hi + x gathers in lo.  A product enters with its own exact rounding error
// (FMA), so hi + lo equals the FP64 sum of the exact products up to the
// rounding of lo.  The _rn intrinsics keep the compiler from contracting or
// reordering the error terms.
struct DFloatSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void add_product(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(hi, lo); }
};

// sin and cos of 2*pi*f for |f| <= 1/2 (cycles) on the MUFU pipe
// (sin.approx/cos.approx: absolute error below 1e-6 on [-pi, pi]).
__device__ __forceinline__ void sincos_cycles_mufu(float f, float* s, float* c) {
  const float kTwoPi = 6.28318530717958647692f;
  const float th = __fmul_rn(f, kTwoPi);
  *s = __sinf(th);
  *c = __cosf(th);
}

// ---------------------------------------------------------------------------
// Scattering factor (Section 3, pynx.fthomson form; Section 4.2 f', f'', DW)
//   f(s) = (sum_i a_i exp(-b_i s^2) + c + f' + i f'') exp(-B s^2),
// evaluated in FP32 with s^2 = |S|^2 / (4 a^2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 form_factor(const float* __restrict__ cf, float s2) {
  float f0 = __ldg(cf + 8);
#pragma unroll
  for (int i = 0; i < 4; ++i) f0 = fmaf(__ldg(cf + i), __expf(-__ldg(cf + 4 + i) * s2), f0);
  const float dw = __expf(-__ldg(cf + 11) * s2);
  return make_float2((f0 + __ldg(cf + 9)) * dw, __ldg(cf + 10) * dw);
}

// Two FP32 values in one 64-bit register pair, for the packed f32x2 FMA
// (one instruction for two lanes' worth of FP32 FMAs, each rounded as
// fmaf: the FMA pipe's lane rate is unchanged, the issue slots halve).
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// d = a * b + d on both halves
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
// a * b + c on both halves
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// a + b, a - b, a * b on both halves (round to nearest, like the scalar forms)
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// e^{2 pi i s.t} for the integer centring t, reduced in FP64 (O(M) work).
__device__ __forceinline__ float2 shift_phase(double s0, double s1, double s2, const double* t) {
  const double ph = s0 * t[0] + s1 * t[1] + s2 * t[2];
  const float f = (float)(ph - rint(ph));
  float sn, cs;
  sincospif(2.0f * f, &sn, &cs);
  return make_float2(cs, sn);
}

// The same phase without FP64 arithmetic (GB300 issues FP64 at a small
// fraction of the FP32 rate): offsets as double-floats s_hi + s_lo, t_d
// integers below 2^24 in FP32.  Each s_d t_d has its fractional part taken
// with the product's rounding error restored (error ~2^-24 per term, as the
// FP64 form's final rounding to FP32).
__device__ __forceinline__ float2 shift_phase2(const float (&s_hi)[3], const float (&s_lo)[3], const float (&t)[3]) {
  float f = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) f += frac_of_product2(s_hi[d], s_lo[d], t[d]);
  float sn, cs;
  sincospif(2.0f * frac_rn(f), &sn, &cs);
  return make_float2(cs, sn);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (TMA engine) with bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of `bar` to complete, giving up after roughly
// `budget_cycles` SM clocks.  Returns false on timeout (the caller records
// kStatusTimeout and leaves the loop).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long budget_cycles = (1LL << 31)) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > budget_cycles) return false;
  }
  return true;
}

// 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled on `bar` as transaction bytes.  dst, src and bytes must be
// multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void set_status(unsigned* status, unsigned bit) {
  if (status) atomicOr(status, bit);
}

}  // namespace dev
}  // namespace scatter
