// Loss and adjoint of Eq. 2 with respect to the atom positions.
//
//   L        = sum_S (|A(S)|^2 - I_obs(S))^2
//   g(S)     = 4 (|A|^2 - I_obs) conj(A)        (or conj(G) for a general VJP)
//   dL/dr_j  = -2 pi w_j sum_S S Im( g(S) f_s(|S|) exp(2 i pi S.r_j) )
//
// With the forward's split S.r_j = s.t + c_j + s.x'_j (mod 1) the factor
// exp(2 i pi s.t) and f_s(|S|) are folded into one weight per (species, S):
//   gF_s(S) = g(S) f_s(|S|) exp(2 i pi s.t)
// so the per-pair work is the forward's phase + MUFU sincos plus
//   v = Im(gF e^{2 i pi phi}) = gF.re sin + gF.im cos,   acc_d += S_d v.
//
// k_loss_weights  O(M): L partials (FP64, fixed grid, fixed order), the
//                 expanded S table {s, gF.re | S, gF.im} per species.
// k_adjoint       atom-parallel (the paper's alternative decomposition,
//                 Section 2.2): each thread holds RA atoms in registers, S
//                 tiles are staged in shared memory by the TMA engine; inner
//                 sums per tile in FP32, outer sums in FP64 (the terms over
//                 millions of S nearly cancel).  The exponentials are
//                 recomputed, nothing of size N x M is stored.
// k_adjoint_final sums the S-chunk partials in a fixed order, scales by
//                 -2 pi w_j and writes the caller's atom order.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <vector>
#include <type_traits>
#include "device_common.cuh"
#include "launch.h"

namespace scatter {

constexpr int kSTile = 256;        // S points per shared-memory stage
constexpr int kAdjThreads = 128;
constexpr int kAdjRA = 8;          // atoms per thread
constexpr int kLossThreads = 256;

struct LossArgs {
  const float2* A;        // forward amplitude (loss mode) or null
  const float* I_obs;
  const float2* G;        // upstream gradient (vjp mode) or null
  int64_t n_s;
  int grid;
  const float* s_hi;       // list: [3][M] offsets s = S - H, FP32
  const float* s_lo;       //       their rounding errors
  const float* axis_s;     // grid: [n0 | n1 | n2] offsets, FP32
  const float* axis_lo;    //       their rounding errors
  int64_t n0, n1, n2;
  double H[3];
  const double* shift;
  const float* coef;
  const float2* ftab;     // Eq. 4 factor table [n_species][M] (F_t(S) of block types), or null
  int n_species;
  float inv4a2;
  int layout;             // 0: rows {s, gF.re | S, gF.im} for k_adjoint; 1: compact rows
                          // (s_z, S_z, gF.re, gF.im) for k_adjoint_line; 2: gF alone (adjoint_sep.cu)
  float4* table;          // [n_species][M][2] (layout 0), [n_species][M] (layout 1)
  float2* gf;             // [n_species][M] (layout 2)
  double* loss_part;      // [gridDim.x]
};

// FP32 arithmetic throughout (GB300 issues FP64 at ~2 operations per SM and
// clock): S as the plan's double-float offsets s = S - H, the centring phase
// from them and the integer shift, the misfit d = |A|^2 - I_obs exactly
// (products with their rounding errors, TwoSum) before its one rounding,
// and the loss as a double-float sum, folded into FP64 once per thread.
__global__ void __launch_bounds__(kLossThreads) k_loss_weights(const LossArgs a) {
  __shared__ float sh_t[3];
  __shared__ int sh_shifted;
  if (threadIdx.x == 0) {
    sh_t[0] = (float)a.shift[0];
    sh_t[1] = (float)a.shift[1];
    sh_t[2] = (float)a.shift[2];
    sh_shifted = a.shift[0] != 0.0 || a.shift[1] != 0.0 || a.shift[2] != 0.0;
  }
  __syncthreads();
  const float H0 = (float)a.H[0], H1 = (float)a.H[1], H2 = (float)a.H[2];
  dev::DFloatSum lsum;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < a.n_s;
       m += (int64_t)gridDim.x * blockDim.x) {
    float s_hi[3], s_lo[3];
    if (a.grid) {
      const int64_t i2 = m % a.n2, line = m / a.n2, i1 = line % a.n1, i0 = line / a.n1;
      const int64_t ia[3] = {i0, a.n0 + i1, a.n0 + a.n1 + i2};
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        s_hi[d] = a.axis_s[ia[d]];
        s_lo[d] = a.axis_lo[ia[d]];
      }
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        s_hi[d] = a.s_hi[d * a.n_s + m];
        s_lo[d] = a.s_lo[d * a.n_s + m];
      }
    }
    float2 g;
    if (a.A) {
      const float2 A = a.A[m];
      // d = A.x^2 + A.y^2 - I_obs from the exact products and TwoSums
      const float p1 = __fmul_rn(A.x, A.x), p2 = __fmul_rn(A.y, A.y);
      dev::DFloatSum dd;
      dd.hi = p1;
      dd.add(p2);
      dd.add(-a.I_obs[m]);
      dd.lo = __fadd_rn(dd.lo, __fadd_rn(__fmaf_rn(A.x, A.x, -p1), __fmaf_rn(A.y, A.y, -p2)));
      const float d = dd.value();
      lsum.add_product(d, d);
      g = make_float2(4.f * d * A.x, -4.f * d * A.y);
    } else {
      const float2 G = a.G[m];
      g = make_float2(G.x, -G.y);
    }
    const float2 ph = sh_shifted ? dev::shift_phase2(s_hi, s_lo, sh_t) : make_float2(1.f, 0.f);
    const float2 gp = dev::cmul(g, ph);
    const float sx = s_hi[0] + s_lo[0], sy = s_hi[1] + s_lo[1], sz = s_hi[2] + s_lo[2];
    const float Sx = H0 + sx, Sy = H1 + sy, Sz = H2 + sz;
    const float s2 = (Sx * Sx + Sy * Sy + Sz * Sz) * a.inv4a2;
    for (int sp = 0; sp < a.n_species; ++sp) {
      const float2 F = a.ftab ? a.ftab[(int64_t)sp * a.n_s + m] : dev::form_factor(a.coef + kNCoef * sp, s2);
      const float2 gF = dev::cmul(gp, F);
      if (a.layout == 2) {
        a.gf[(int64_t)sp * a.n_s + m] = gF;
      } else if (a.layout == 1) {
        a.table[(int64_t)sp * a.n_s + m] = make_float4(sz, Sz, gF.x, gF.y);
      } else {
        float4* row = a.table + 2 * ((int64_t)sp * a.n_s + m);
        row[0] = make_float4(sx, sy, sz, gF.x);
        row[1] = make_float4(Sx, Sy, Sz, gF.y);
      }
    }
  }
  double lpart = (double)lsum.hi + (double)lsum.lo;
  // deterministic block reduction of the misfit
  __shared__ double sh[kLossThreads / 32];
  for (int o = 16; o > 0; o >>= 1) lpart += __shfl_xor_sync(0xffffffffu, lpart, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lpart;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kLossThreads / 32; ++w) v += sh[w];
    a.loss_part[blockIdx.x] = v;
  }
}

// One warp: lane l sums the partials l, l + 32, ... in order, then a fixed
// butterfly; the order does not depend on timing, so the loss is reproducible.
__global__ void k_loss_final(const double* part, int n, double* out) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < n; i += 32) v += part[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

struct AdjArgs {
  const float4* atom4;
  const AdjBlock* blocks;
  const float4* table;     // [n_species][M][2]
  int64_t n_s;
  int64_t s_per_chunk;
  float* partial;          // [split][n_slots][3]
  int64_t n_slots;
  const unsigned long long* bbox;  // [6] this call's ordered min / max xyz
  const double* shift;             // [3] its centring t
  float smax[3];                   // max |S_d - H_d| over the points
  unsigned* status;
};

// Outer sums of a thread's atoms (over S tiles), double-float, in shared
// memory: hi and lo of component d of the thread's atom r at [d][r][thread].
// Every thread owns its slots (no synchronisation) and consecutive threads
// use consecutive words; a slot is touched once per tile, so keeping the
// 3 x kAdjRA pairs out of the registers costs little and lets four CTAs
// share an SM.
struct OuterSums {
  float2 (*g)[kAdjRA][kAdjThreads];
  int t;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int r = 0; r < kAdjRA; ++r) g[d][r][t] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(int d, int r, float x) {
    const float2 v = g[d][r][t];
    dev::DFloatSum a;
    a.hi = v.x;
    a.lo = v.y;
    a.add(x);
    g[d][r][t] = make_float2(a.hi, a.lo);
  }
  __device__ __forceinline__ void add_product(int d, int r, float x, float y) {
    const float2 v = g[d][r][t];
    dev::DFloatSum a;
    a.hi = v.x;
    a.lo = v.y;
    a.add_product(x, y);
    g[d][r][t] = make_float2(a.hi, a.lo);
  }
  __device__ __forceinline__ float value(int d, int r) const {
    const float2 v = g[d][r][t];
    return __fadd_rn(v.x, v.y);
  }
};

__global__ void __launch_bounds__(kAdjThreads, 4) k_adjoint(const AdjArgs a) {
  __shared__ __align__(128) float4 sh_s[2][kSTile * 2];
  __shared__ __align__(8) uint64_t sh_bar[2];
  const int tid = threadIdx.x;
  const AdjBlock blk = a.blocks[blockIdx.x];
  const int chunk = blockIdx.y;
  const int64_t m0 = (int64_t)chunk * a.s_per_chunk;
  const int64_t m1 = dev::min64(a.n_s, m0 + a.s_per_chunk);
  const float4* tab = a.table + 2 * (int64_t)blk.species * a.n_s;

  float x[kAdjRA], y[kAdjRA], z[kAdjRA], c[kAdjRA];
#pragma unroll
  for (int r = 0; r < kAdjRA; ++r) {
    const int i = r * kAdjThreads + tid;
    const float4 at = i < blk.count ? a.atom4[blk.begin + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    x[r] = at.x;
    y[r] = at.y;
    z[r] = at.z;
    c[r] = at.w;
  }
  // the atoms in packed pairs for the plain phase form
  unsigned long long x2[kAdjRA / 2], y2[kAdjRA / 2], z2[kAdjRA / 2], c2[kAdjRA / 2];
#pragma unroll
  for (int pp = 0; pp < kAdjRA / 2; ++pp) {
    x2[pp] = dev::pack2(x[2 * pp], x[2 * pp + 1]);
    y2[pp] = dev::pack2(y[2 * pp], y[2 * pp + 1]);
    z2[pp] = dev::pack2(z[2 * pp], z[2 * pp + 1]);
    c2[pp] = dev::pack2(c[2 * pp], c[2 * pp + 1]);
  }
  // outer sums over the tiles: double-float on the FP32 pipe, in shared memory
  __shared__ float2 sh_g[3][kAdjRA][kAdjThreads];
  OuterSums g{sh_g, tid};
  g.zero();

  if (tid == 0) {
    dev::mbar_init(&sh_bar[0], 1);
    dev::mbar_init(&sh_bar[1], 1);
    dev::mbar_fence_init();
  }
  __syncthreads();
  const int64_t n_tiles = m1 > m0 ? (m1 - m0 + kSTile - 1) / kSTile : 0;
  // long crystals: every product of the phase with its rounding error restored
  const bool exact = dev::phase_needs_exact(a.bbox, a.shift, a.smax);
  auto issue = [&](int64_t k) {
    if (k >= n_tiles) return;
    const int64_t b = m0 + k * kSTile;
    const int cnt = (int)dev::min64(kSTile, m1 - b);
    const int st = (int)(k & 1);
    dev::mbar_arrive_expect_tx(&sh_bar[st], (uint32_t)cnt * 32u);
    dev::bulk_g2s(&sh_s[st][0], tab + 2 * b, (uint32_t)cnt * 32u, &sh_bar[st]);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  bool aborted = false;
  for (int64_t k = 0; k < n_tiles; ++k) {
    const int st = (int)(k & 1);
    const int cnt = (int)dev::min64(kSTile, m1 - (m0 + k * kSTile));
    const bool ok = dev::mbar_wait_bounded(&sh_bar[st], (uint32_t)((k >> 1) & 1));
    float ax[kAdjRA], ay[kAdjRA], az[kAdjRA];
#pragma unroll
    for (int r = 0; r < kAdjRA; ++r) ax[r] = ay[r] = az[r] = 0.f;
    // one loop body per phase form: the choice stays out of the unrolled
    // pair loop, whose eight atoms' chains then interleave freely
    auto tile = [&](auto exact_tag) {
      constexpr bool kExact = decltype(exact_tag)::value;
      const float4* sv = sh_s[st];
      if (!kExact) {
        // two atoms per packed register pair: every step of the plain form is
        // elementwise over the atoms, so one f32x2 operation does two atoms'
        // (the same roundings as the scalar fmaf / __fadd_rn / __fmul_rn);
        // the point's values are broadcast into both halves
        using u64 = unsigned long long;
        const u64 magic2 = dev::pack2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: rint by addition
        const u64 twopi2 = dev::pack2(6.28318530717958647692f, 6.28318530717958647692f);
        u64 ax2[kAdjRA / 2], ay2[kAdjRA / 2], az2[kAdjRA / 2];
#pragma unroll
        for (int pp = 0; pp < kAdjRA / 2; ++pp) ax2[pp] = ay2[pp] = az2[pp] = 0ull;
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
          const float4 p = sv[2 * j];      // s, gF.re
          const float4 q = sv[2 * j + 1];  // S, gF.im
          const u64 px = dev::pack2(p.x, p.x), py = dev::pack2(p.y, p.y), pz = dev::pack2(p.z, p.z);
          const u64 pw = dev::pack2(p.w, p.w), qw = dev::pack2(q.w, q.w);
          const u64 qx = dev::pack2(q.x, q.x), qy = dev::pack2(q.y, q.y), qz = dev::pack2(q.z, q.z);
#pragma unroll
          for (int pp = 0; pp < kAdjRA / 2; ++pp) {
            const u64 ph = dev::fma2(pz, z2[pp], dev::fma2(py, y2[pp], dev::fma2(px, x2[pp], c2[pp])));
            const u64 f = dev::sub2(ph, dev::sub2(dev::add2(ph, magic2), magic2));  // ph - rint(ph)
            float t0, t1;
            dev::unpack2(dev::mul2(f, twopi2), t0, t1);
            const u64 sn = dev::pack2(__sinf(t0), __sinf(t1)), cs = dev::pack2(__cosf(t0), __cosf(t1));
            const u64 v = dev::fma2(pw, sn, dev::mul2(qw, cs));
            ax2[pp] = dev::fma2(qx, v, ax2[pp]);
            ay2[pp] = dev::fma2(qy, v, ay2[pp]);
            az2[pp] = dev::fma2(qz, v, az2[pp]);
          }
        }
#pragma unroll
        for (int pp = 0; pp < kAdjRA / 2; ++pp) {
          dev::unpack2(ax2[pp], ax[2 * pp], ax[2 * pp + 1]);
          dev::unpack2(ay2[pp], ay[2 * pp], ay[2 * pp + 1]);
          dev::unpack2(az2[pp], az[2 * pp], az[2 * pp + 1]);
        }
        return;
      }
#pragma unroll 2
      for (int j = 0; j < cnt; ++j) {
        const float4 p = sv[2 * j];      // s, gF.re
        const float4 q = sv[2 * j + 1];  // S, gF.im
#pragma unroll
        for (int r = 0; r < kAdjRA; ++r) {
          const float f =
              kExact ? dev::frac_rn(dev::frac_product_plus(
                           p.x, x[r], dev::frac_product_plus(p.y, y[r], dev::frac_product_plus(p.z, z[r], c[r]))))
                     : dev::frac_rn(fmaf(p.z, z[r], fmaf(p.y, y[r], fmaf(p.x, x[r], c[r]))));
          float sn, cs;
          dev::sincos_cycles_mufu(f, &sn, &cs);
          const float v = fmaf(p.w, sn, q.w * cs);
          ax[r] = fmaf(q.x, v, ax[r]);
          ay[r] = fmaf(q.y, v, ay[r]);
          az[r] = fmaf(q.z, v, az[r]);
        }
      }
    };
    if (ok) {
      if (exact)
        tile(std::true_type{});
      else
        tile(std::false_type{});
    }
#pragma unroll
    for (int r = 0; r < kAdjRA; ++r) {
      g.add(0, r, ax[r]);
      g.add(1, r, ay[r]);
      g.add(2, r, az[r]);
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      if (tid == 0) {
        dev::set_status(a.status, kStatusTimeout);
        for (int64_t kk = k; kk < dev::min64(k + 2, n_tiles); ++kk)
          dev::mbar_wait_bounded(&sh_bar[kk & 1], (uint32_t)((kk >> 1) & 1), 1LL << 28);
      }
      break;
    }
    if (tid == 0) issue(k + 2);
  }
  if (aborted) return;
  float* out = a.partial + (int64_t)chunk * a.n_slots * 3;
#pragma unroll
  for (int r = 0; r < kAdjRA; ++r) {
    const int i = r * kAdjThreads + tid;
    if (i < blk.count) {
      const int64_t slot = blk.begin + i;
      out[3 * slot] = g.value(0, r);
      out[3 * slot + 1] = g.value(1, r);
      out[3 * slot + 2] = g.value(2, r);
    }
  }
}

// Grid variant of k_adjoint for an l axis of uniform step ds.  S tiles are
// segments of one l line (fixed h, k), so s_x, s_y, S_x, S_y are constants
// of the tile and the table row per point shrinks to (s_z, S_z, gF.re,
// gF.im).  Along the line the phase advances by ds z'_j per point, so
// e^{2 i pi phi} is carried from point to point by one complex multiply
// with w_j = e^{2 i pi ds z'_j} instead of a MUFU sin/cos per pair (four
// FMA-pipe ops; the pair costs eight in all, no MUFU).  Every 128 points the
// exponential is re-seeded from the exactly reduced phase, which bounds the
// rounding drift of the recurrence to ~128 products with w accurate to ~1
// ulp (~1e-5 relative, against the 1e-3 tolerance of the gradients).  Per tile: FP32 line sums
// sum v and sum S_z v, folded into double-float outer sums (FP32 pairs on
// the FMA pipe) as S_x sum v, S_y sum v, sum S_z v.
struct AdjLineArgs {
  const float4* atom4;
  const AdjBlock* blocks;
  const float4* table;      // [n_species][M]: (s_z, S_z, gF.re, gF.im)
  const float* axis_s;      // [n0 | n1 | n2] offsets s = axis - H
  float H[3];
  int64_t n0, n1, n2;
  float ds;                 // step of the l axis
  int64_t lines_per_chunk;
  float* partial;           // [split][n_slots][3]
  int64_t n_slots;
  unsigned* status;
};

constexpr int kReseed = 128;  // points between exact re-seeds of the recurrence

__global__ void __launch_bounds__(kAdjThreads, 4) k_adjoint_line(const AdjLineArgs a) {
  __shared__ __align__(128) float4 sh_s[2][kSTile];
  __shared__ __align__(8) uint64_t sh_bar[2];
  const int tid = threadIdx.x;
  const AdjBlock blk = a.blocks[blockIdx.x];
  const int chunk = blockIdx.y;
  const int64_t n_lines = a.n0 * a.n1;
  const int64_t L0 = (int64_t)chunk * a.lines_per_chunk;
  const int64_t L1 = dev::min64(n_lines, L0 + a.lines_per_chunk);
  const int64_t segs = (a.n2 + kSTile - 1) / kSTile;  // tiles per line
  const float4* tab = a.table + (int64_t)blk.species * n_lines * a.n2;

  float x[kAdjRA], y[kAdjRA], z[kAdjRA], c[kAdjRA], wr[kAdjRA], wi[kAdjRA];
#pragma unroll
  for (int r = 0; r < kAdjRA; ++r) {
    const int i = r * kAdjThreads + tid;
    const float4 at = i < blk.count ? a.atom4[blk.begin + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    x[r] = at.x;
    y[r] = at.y;
    z[r] = at.z;
    c[r] = at.w;
    float sn, cs;
    // rotation per l step, accurate to ~1 ulp (its error compounds along
    // the line between re-seeds)
    sincospif(2.0f * dev::frac_of_product(a.ds, z[r]), &sn, &cs);
    wr[r] = cs;
    wi[r] = sn;
  }
  // outer sums over the lines: double-float on the FP32 pipe, in shared memory
  __shared__ float2 sh_g[3][kAdjRA][kAdjThreads];
  OuterSums g{sh_g, tid};
  g.zero();

  if (tid == 0) {
    dev::mbar_init(&sh_bar[0], 1);
    dev::mbar_init(&sh_bar[1], 1);
    dev::mbar_fence_init();
  }
  __syncthreads();
  const int64_t n_tiles = L1 > L0 ? (L1 - L0) * segs : 0;
  auto issue = [&](int64_t k) {
    if (k >= n_tiles) return;
    const int64_t line = L0 + k / segs, j0 = (k % segs) * kSTile;
    const int cnt = (int)dev::min64(kSTile, a.n2 - j0);
    const int st = (int)(k & 1);
    dev::mbar_arrive_expect_tx(&sh_bar[st], (uint32_t)cnt * 16u);
    dev::bulk_g2s(&sh_s[st][0], tab + line * a.n2 + j0, (uint32_t)cnt * 16u, &sh_bar[st]);
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }
  bool aborted = false;
  for (int64_t k = 0; k < n_tiles; ++k) {
    const int st = (int)(k & 1);
    const int64_t line = L0 + k / segs, j0 = (k % segs) * kSTile;
    const int cnt = (int)dev::min64(kSTile, a.n2 - j0);
    const bool ok = dev::mbar_wait_bounded(&sh_bar[st], (uint32_t)((k >> 1) & 1));
    const int64_t i0 = line / a.n1, i1 = line % a.n1;
    const float sx = a.axis_s[i0], sy = a.axis_s[a.n0 + i1];
    float base[kAdjRA], er[kAdjRA], ei[kAdjRA], sv[kAdjRA], szv[kAdjRA];
#pragma unroll
    for (int r = 0; r < kAdjRA; ++r) {
      // once per atom and tile: the products with their rounding errors
      base[r] = dev::frac_product_plus(sx, x[r], dev::frac_product_plus(sy, y[r], c[r]));
      sv[r] = szv[r] = 0.f;
    }
    if (ok) {
      // two atoms per packed register pair: every operation of the recurrence
      // is elementwise over the atoms, so one fma.rn.f32x2 does two atoms'
      // FMA (the same rounding as fmaf); the point's values are broadcast
      using u64 = unsigned long long;
      constexpr int kP = kAdjRA / 2;
      u64 wr2[kP], wi2[kP], nwi2[kP], sv2[kP], szv2[kP];
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        wr2[p] = dev::pack2(wr[2 * p], wr[2 * p + 1]);
        wi2[p] = dev::pack2(wi[2 * p], wi[2 * p + 1]);
        nwi2[p] = dev::pack2(-wi[2 * p], -wi[2 * p + 1]);
        sv2[p] = szv2[p] = 0ull;
      }
      const u64 one2 = dev::pack2(1.f, 1.f), zero2 = 0ull;
      const float4* sv4 = sh_s[st];
      for (int jb = 0; jb < cnt; jb += kReseed) {
        // exact exponential at the first point of every 64
        const float qz = sv4[jb].x;
#pragma unroll
        for (int r = 0; r < kAdjRA; ++r)
          dev::sincos_cycles_mufu(dev::frac_rn(dev::frac_product_plus(qz, z[r], base[r])), &ei[r], &er[r]);
        u64 er2[kP], ei2[kP];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
          er2[p] = dev::pack2(er[2 * p], er[2 * p + 1]);
          ei2[p] = dev::pack2(ei[2 * p], ei[2 * p + 1]);
        }
        const int je = min(cnt, jb + kReseed);
#pragma unroll 2
        for (int j = jb; j < je; ++j) {
          const float4 q = sv4[j];  // s_z, S_z, gF.re, gF.im
          const u64 qy2 = dev::pack2(q.y, q.y), qz2 = dev::pack2(q.z, q.z), qw2 = dev::pack2(q.w, q.w);
#pragma unroll
          for (int p = 0; p < kP; ++p) {
            const u64 v = dev::fma2(qz2, ei2[p], dev::fma2(qw2, er2[p], zero2));  // Im(gF e)
            sv2[p] = dev::fma2(v, one2, sv2[p]);
            szv2[p] = dev::fma2(qy2, v, szv2[p]);
            const u64 nr = dev::fma2(er2[p], wr2[p], dev::fma2(ei2[p], nwi2[p], zero2));
            ei2[p] = dev::fma2(er2[p], wi2[p], dev::fma2(ei2[p], wr2[p], zero2));
            er2[p] = nr;
          }
        }
      }
#pragma unroll
      for (int p = 0; p < kP; ++p) {
        dev::unpack2(sv2[p], sv[2 * p], sv[2 * p + 1]);
        dev::unpack2(szv2[p], szv[2 * p], szv[2 * p + 1]);
      }
    }
    const float Sx = a.H[0] + sx, Sy = a.H[1] + sy;
#pragma unroll
    for (int r = 0; r < kAdjRA; ++r) {
      g.add_product(0, r, Sx, sv[r]);
      g.add_product(1, r, Sy, sv[r]);
      g.add(2, r, szv[r]);
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      if (tid == 0) {
        dev::set_status(a.status, kStatusTimeout);
        for (int64_t kk = k; kk < dev::min64(k + 2, n_tiles); ++kk)
          dev::mbar_wait_bounded(&sh_bar[kk & 1], (uint32_t)((kk >> 1) & 1), 1LL << 28);
      }
      break;
    }
    if (tid == 0) issue(k + 2);
  }
  if (aborted) return;
  float* out = a.partial + (int64_t)chunk * a.n_slots * 3;
#pragma unroll
  for (int r = 0; r < kAdjRA; ++r) {
    const int i = r * kAdjThreads + tid;
    if (i < blk.count) {
      const int64_t slot = blk.begin + i;
      out[3 * slot] = g.value(0, r);
      out[3 * slot + 1] = g.value(1, r);
      out[3 * slot + 2] = g.value(2, r);
    }
  }
}

__global__ void k_adjoint_final(const float* partial, int split, int64_t n_slots, const int32_t* slot_src,
                                const float* atom_w, float* grad) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n_slots) return;
  const int32_t src = slot_src[slot];
  if (src < 0) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int c = 0; c < split; ++c)
    for (int d = 0; d < 3; ++d) v[d] += (double)partial[((int64_t)c * n_slots + slot) * 3 + d];
  const double scale = -2.0 * 3.14159265358979323846 * (double)atom_w[slot];
  for (int d = 0; d < 3; ++d) grad[3 * (int64_t)src + d] = (float)(scale * v[d]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

scatter_status prepare_adjoint(scatter_plan_s* p) {
  if (p->adj_ready) return SCATTER_OK;
  if (p->batch != 1) return fail(SCATTER_ERR_UNSUPPORTED, "backward is available for single instances");
  // a SEPARABLE grid plan contracts on the tensor cores when its workspace fits
  scatter_status ss = prepare_adjoint_sep(p);
  if (ss != SCATTER_OK) return ss;
  if (p->adj_sep) {
    p->adj_ready = true;
    return SCATTER_OK;
  }
  std::vector<AdjBlock> blocks;
  const int per = kAdjThreads * kAdjRA;
  for (const Segment& s : p->all_segs)
    for (int64_t b = s.begin; b < s.end; b += per)
      blocks.push_back(AdjBlock{b, (int32_t)dev::min64(per, s.end - b), s.species});
  // a grid whose l axis has a uniform step runs the line-recurrence kernel
  p->adj_line = false;
  if (p->s_kind == SCATTER_S_GRID && p->n_axis[2] >= 1) {
    const std::vector<double>& l = p->axis_host[2];
    const int64_t n2 = (int64_t)l.size();
    const double ds = n2 > 1 ? (l[n2 - 1] - l[0]) / (double)(n2 - 1) : 0.0;
    bool uniform = true;
    for (int64_t i = 0; i < n2 && uniform; ++i)
      uniform = std::fabs(l[i] - (l[0] + (double)i * ds)) <= 1e-9 * std::max(1.0, std::fabs(l[i]));
    p->adj_line = uniform;
    p->adj_ds = (float)ds;
  }
  // split over S so that the grid fills the GPU a few times over
  int bps = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, p->adj_line ? (const void*)k_adjoint_line
                                                                      : (const void*)k_adjoint,
                                                    kAdjThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    bps = 1;
  }
  const int64_t nb = std::max<int64_t>(1, (int64_t)blocks.size());
  const int64_t cap = (int64_t)p->n_sm * std::max(1, bps);  // resident CTAs
  // S chunks (in whole l lines, or 256-point tiles) per atom block: the split
  // that minimises waves x work per CTA, among those giving >= 2 waves
  const int64_t unit = p->adj_line ? p->n_axis[2] : (int64_t)kSTile;
  const int64_t n_units = p->adj_line ? std::max<int64_t>(1, p->n_axis[0] * p->n_axis[1])
                                      : std::max<int64_t>(1, (p->n_s + kSTile - 1) / kSTile);
  int64_t best_per = n_units;
  double best_cost = 1e300;
  for (int64_t split = 1; split <= std::min<int64_t>(n_units, 64 * cap / nb + 1); ++split) {
    const int64_t per = (n_units + split - 1) / split;
    const int64_t chunks = (n_units + per - 1) / per;
    const double waves = std::ceil((double)(nb * chunks) / (double)cap);
    // a fixed per-CTA cost (atom loads, outer sums, partial write) of ~2 units
    const double cost = waves * (double)(per + 2) + (nb * chunks < 2 * cap ? 1e200 : 0.0);
    if (cost < best_cost * 0.999) {
      best_cost = cost;
      best_per = per;
    }
  }
  if (best_cost >= 1e199) best_per = std::max<int64_t>(1, n_units / std::max<int64_t>(1, 2 * cap / nb));
  const int64_t split = (n_units + best_per - 1) / best_per;
  if (p->adj_line) {
    p->adj_lines_per_chunk = best_per;
    p->adj_s_per_chunk = best_per * unit;
  } else {
    p->adj_s_per_chunk = best_per * kSTile;
  }
  p->adj_split = (int)split;
  p->adj_blocks = (int)blocks.size();
  cudaError_t e;
  const size_t tab_bytes = (size_t)p->n_species * (size_t)p->n_s * 2 * sizeof(float4);
  const size_t part_bytes = (size_t)split * (size_t)p->n_slots * 3 * sizeof(float);
  if (!blocks.empty()) {
    if ((e = cudaMalloc(&p->d.adj_blocks, blocks.size() * sizeof(AdjBlock))) != cudaSuccess)
      return cuda_status(e, "cudaMalloc");
    if ((e = cudaMemcpy(p->d.adj_blocks, blocks.data(), blocks.size() * sizeof(AdjBlock), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
      return cuda_status(e, "cudaMemcpy");
  }
  if (tab_bytes && (e = cudaMalloc(&p->d.adj_table, tab_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc");
  if (part_bytes && (e = cudaMalloc(&p->d.adj_partial, part_bytes)) != cudaSuccess)
    return cuda_status(e, "cudaMalloc");
  p->base_bytes += (int64_t)(tab_bytes + part_bytes + blocks.size() * sizeof(AdjBlock));
  p->adj_ready = true;
  return SCATTER_OK;
}

scatter_status launch_backward(scatter_plan_t p, const double* xyz, const float* occ, const float2* A,
                               const float* I_obs, const float2* G, double* loss_out, float* grad,
                               cudaStream_t st) {
  if (p->path == SCATTER_PATH_FP64_REF)
    return fail(SCATTER_ERR_UNSUPPORTED, "backward runs on the generic path; plan with SCATTER_PATH_GENERIC");
  scatter_status s = SCATTER_OK;
  if (grad) {
    if ((s = prepare_adjoint(p)) != SCATTER_OK) return s;
    // positions (and the centring t) exactly as the forward used them
    if ((s = launch_prep(p, xyz, occ, st)) != SCATTER_OK) return s;
  } else if (p->n_s > 0 && p->n_atoms > 0) {
    // loss only: the shift is not needed, but the table write is skipped too
  }
  if (p->n_s == 0) {
    if (loss_out) cudaMemsetAsync(loss_out, 0, sizeof(double), st);
    if (grad && p->n_atoms) cudaMemsetAsync(grad, 0, sizeof(float) * 3 * p->n_atoms, st);
    return cuda_status(cudaGetLastError(), "backward (empty)");
  }
  LossArgs la{};
  la.A = A;
  la.I_obs = I_obs;
  la.G = G;
  la.n_s = p->n_s;
  la.grid = p->s_kind == SCATTER_S_GRID;
  la.s_hi = p->d.s_hi;
  la.s_lo = p->d.s_lo;
  la.axis_s = p->d.axis_s;
  la.axis_lo = p->d.axis_lo;
  la.n0 = p->n_axis[0];
  la.n1 = p->n_axis[1];
  la.n2 = p->n_axis[2];
  for (int d = 0; d < 3; ++d) la.H[d] = p->inst[0].H[d];
  la.shift = p->d.inst_shift;
  la.coef = p->d.coef;
  la.ftab = p->d.ftab;  // Eq. 4: the block factors F_t(S) in place of f_s(|S|), held fixed
  la.n_species = grad ? p->n_species : 0;
  la.inv4a2 = (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a));
  la.layout = !grad ? 0 : (p->adj_sep ? 2 : (p->adj_line ? 1 : 0));
  la.table = p->d.adj_table;
  la.gf = p->d.adj_gf;
  la.loss_part = p->d.loss_part;
  k_loss_weights<<<kLossParts, kLossThreads, 0, st>>>(la);
  p->last_launches += 1;
  if (A && loss_out) {
    k_loss_final<<<1, 32, 0, st>>>(p->d.loss_part, kLossParts, loss_out);
    p->last_launches += 1;
  }
  if (grad && p->n_atoms > 0 && p->adj_sep) return launch_adjoint_sep(p, grad, st);
  if (grad && p->n_atoms > 0) {
    AdjArgs aa{};
    aa.atom4 = p->d.atom4;
    aa.blocks = p->d.adj_blocks;
    aa.table = p->d.adj_table;
    aa.n_s = p->n_s;
    aa.s_per_chunk = p->adj_s_per_chunk;
    aa.partial = p->d.adj_partial;
    aa.n_slots = p->n_slots;
    aa.bbox = p->d.inst_bbox;
    aa.shift = p->d.inst_shift;
    for (int d = 0; d < 3; ++d) aa.smax[d] = (float)p->s_max[d];
    aa.status = p->d.status;
    if (p->adj_blocks > 0) {
      dim3 gridd((unsigned)p->adj_blocks, (unsigned)p->adj_split);
      timing_begin(p, st);
      if (p->adj_line) {
        AdjLineArgs al{};
        al.atom4 = p->d.atom4;
        al.blocks = p->d.adj_blocks;
        al.table = p->d.adj_table;
        al.axis_s = p->d.axis_s;
        for (int d = 0; d < 3; ++d) al.H[d] = (float)p->inst[0].H[d];
        al.n0 = p->n_axis[0];
        al.n1 = p->n_axis[1];
        al.n2 = p->n_axis[2];
        al.ds = p->adj_ds;
        al.lines_per_chunk = p->adj_lines_per_chunk;
        al.partial = p->d.adj_partial;
        al.n_slots = p->n_slots;
        al.status = p->d.status;
        k_adjoint_line<<<gridd, kAdjThreads, 0, st>>>(al);
      } else {
        k_adjoint<<<gridd, kAdjThreads, 0, st>>>(aa);
      }
      timing_end(p, st);
      p->last_launches += 1;
    }
    const int64_t nb = (p->n_slots + 255) / 256;
    k_adjoint_final<<<(unsigned)nb, 256, 0, st>>>(p->d.adj_partial, p->adj_split, p->n_slots, p->d.slot_src,
                                                  p->d.atom_w, grad);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "backward launch");
}

}  // namespace scatter
