// The generic kernel's inner pipeline, shared by the one-shot kernel
// (forward.cu) and the persistent batched kernel (batch.cu).
#pragma once

#include "device_common.cuh"

namespace scatter {

constexpr int kTile = 256;  // atoms per shared-memory stage

enum { kModeList = 0, kModeGrid = 1 };

struct GenericArgs {
  const float4* atom4;
  const float4* atom_lo;  // FP32 rounding errors of (x', y', z') (exact-product phases), 0
  const float* atom_w;
  const Segment* segs;
  const int32_t* chunk_seg_off;
  const float* coef;
  int64_t n_s;
  const float* s_hi;      // LIST [3][M]
  const float* s_lo;      // LIST [3][M] FP32 rounding error of s_hi (exact-product phases)
  const double* S64;      // LIST [M][3]
  const float* axis_s;    // GRID [n0 | n1 | n2]
  const float* axis_lo;   // GRID [n0 | n1 | n2] FP32 rounding error of axis_s
  const double* axis64;   // GRID [n0 | n1 | n2]
  int64_t n0, n1, n2;
  float H[3];
  double H64[3];
  float inv4a2;
  const double* shift;    // [3] device, written by prep
  const unsigned long long* bbox;  // [6] device, this call's ordered min / max xyz (null: never exact)
  float smax[3];          // max |S_d - H_d| over the points
  const float* smax_dev;  // the same maxima in device memory [3] (written by an earlier kernel), or null
  const float2* ftab;     // Eq. 4 factor table [n_species][M], or null (form factors)
  float2* out_amp;
  float* out_int;
  float2* partial;        // split-K partials [chunk][M] (or null)
  unsigned* status;
};

// LIST-mode generic kernel (+ split-K reduction) on prepared arguments.
scatter_status launch_generic_args(GenericArgs a, int R, int threads, int n_chunks, cudaStream_t st);

// Sum over the atoms of one chunk (a list of species segments) for the R
// S points of this thread: atom tiles are staged in shared memory by the TMA
// engine (two stages, mbarrier completion, bounded waits), the per-pair work
// is the split phase + MUFU sincos + 2 FFMA into tile-blocked FP32 sums, and
// f_s(|S|) is folded in at the end of every species segment (or, with an
// Eq. 4 factor table, F_s(S) at the thread's point indices pbase + r pstride,
// clamped to the map).  EXACT: crystals whose phases can pass
// dev::kPhaseExactLim cycles take every product of the phase with its
// rounding error restored, with s as a double-float (s + lo: lx, ly, lz) and
// the positions as double-floats (x' + e, e staged from atom_lo into sh_lo);
// the lo parts are read only then.  A position rounded to FP32 errs by
// |x'| 2^-24 cells, which at thousands of cells moves s.x' by ~1e-4 rad.  `k` counts the
// tiles this CTA has consumed so far (it sets the stage and mbarrier parity
// and carries over between chunks of a persistent CTA).  Returns false if a
// wait gave up (the CTA then drains its copies and must stop).
template <int MODE, int R, bool EXACT = false>
__device__ __forceinline__ bool chunk_sum(const float4* __restrict__ atom4, const float4* __restrict__ atom_lo,
                                          const float* __restrict__ atom_w,
                                          const Segment* __restrict__ segs, int seg_lo, int seg_hi,
                                          const float* __restrict__ coef, const float H[3], float inv4a2,
                                          const float (&sx)[R], const float (&sy)[R], const float (&sz)[R],
                                          const float (&lx)[R], const float (&ly)[R], const float (&lz)[R],
                                          float4 (*sh_atom)[kTile], float4 (*sh_lo)[kTile], float (*sh_w)[kTile],
                                          uint64_t* sh_bar, int& k, float2 (&tot)[R], unsigned* status,
                                          const float2* __restrict__ ftab, int64_t n_s, int64_t pbase,
                                          int64_t pstride) {
  const int tid = threadIdx.x;
  // loader state (used by thread 0 only)
  int l_seg = seg_lo;
  int64_t l_begin = seg_lo < seg_hi ? segs[seg_lo].begin : 0;
  auto issue = [&](int stage) {
    if (l_seg >= seg_hi) return;
    const int64_t end = segs[l_seg].end;
    const int cnt = (int)dev::min64(kTile, end - l_begin);
    dev::mbar_arrive_expect_tx(&sh_bar[stage], (uint32_t)cnt * (EXACT ? 36u : 20u));
    dev::bulk_g2s(&sh_atom[stage][0], atom4 + l_begin, (uint32_t)cnt * 16u, &sh_bar[stage]);
    dev::bulk_g2s(&sh_w[stage][0], atom_w + l_begin, (uint32_t)cnt * 4u, &sh_bar[stage]);
    if (EXACT) dev::bulk_g2s(&sh_lo[stage][0], atom_lo + l_begin, (uint32_t)cnt * 16u, &sh_bar[stage]);
    l_begin += cnt;
    if (l_begin >= end && ++l_seg < seg_hi) l_begin = segs[l_seg].begin;
  };
  if (tid == 0) {
    issue(k & 1);
    issue((k + 1) & 1);
  }

  float2 sacc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) tot[r] = sacc[r] = make_float2(0.f, 0.f);

  int c_seg = seg_lo;
  int64_t c_begin = seg_lo < seg_hi ? segs[seg_lo].begin : 0;
  while (c_seg < seg_hi) {
    const int64_t end = segs[c_seg].end;
    const int cnt = (int)dev::min64(kTile, end - c_begin);
    const int st = k & 1;
    const bool ok = dev::mbar_wait_bounded(&sh_bar[st], (uint32_t)((k >> 1) & 1));
    float2 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = make_float2(0.f, 0.f);
    if (ok && !EXACT && R % 2 == 0) {
      // the plain phase for two points per packed register pair: each half
      // runs one point's operations with the scalar form's roundings (the
      // atom's values broadcast into both halves), so every point's sum is
      // the scalar loop's bit for bit, in half the issue slots
      using u64 = unsigned long long;
      constexpr int RP = R / 2 > 0 ? R / 2 : 1;
      const float4* at4 = sh_atom[st];
      const float* atw = sh_w[st];
      const u64 magic2 = dev::pack2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: rint by addition
      const u64 twopi2 = dev::pack2(6.28318530717958647692f, 6.28318530717958647692f);
      u64 px[RP], py[RP], pz[RP], are[RP], aim[RP];
#pragma unroll
      for (int q = 0; q < RP; ++q) {
        px[q] = dev::pack2(sx[2 * q], sx[2 * q + 1]);
        py[q] = dev::pack2(sy[2 * q], sy[2 * q + 1]);
        pz[q] = dev::pack2(sz[2 * q], sz[2 * q + 1]);
        are[q] = aim[q] = 0ull;
      }
#pragma unroll 2
      for (int j = 0; j < cnt; ++j) {
        const float4 at = at4[j];
        const float w = atw[j];
        const u64 w2 = dev::pack2(w, w), az = dev::pack2(at.z, at.z);
        u64 b2 = 0ull, ax = 0ull, ay = 0ull, aw = 0ull;
        if (MODE == kModeGrid) {
          const float base = fmaf(sy[0], at.y, fmaf(sx[0], at.x, at.w));
          b2 = dev::pack2(base, base);
        } else {
          ax = dev::pack2(at.x, at.x);
          ay = dev::pack2(at.y, at.y);
          aw = dev::pack2(at.w, at.w);
        }
#pragma unroll
        for (int q = 0; q < RP; ++q) {
          const u64 ph = MODE == kModeGrid ? dev::fma2(pz[q], az, b2)
                                           : dev::fma2(pz[q], az, dev::fma2(py[q], ay, dev::fma2(px[q], ax, aw)));
          const u64 f = dev::sub2(ph, dev::sub2(dev::add2(ph, magic2), magic2));  // ph - rint(ph)
          float t0, t1;
          dev::unpack2(dev::mul2(f, twopi2), t0, t1);
          are[q] = dev::fma2(w2, dev::pack2(__cosf(t0), __cosf(t1)), are[q]);
          aim[q] = dev::fma2(w2, dev::pack2(__sinf(t0), __sinf(t1)), aim[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < RP; ++q) {
        dev::unpack2(are[q], acc[2 * q].x, acc[2 * q + 1].x);
        dev::unpack2(aim[q], acc[2 * q].y, acc[2 * q + 1].y);
      }
    } else if (ok) {
      const float4* at4 = sh_atom[st];
      const float4* atl = sh_lo[st];
      const float* atw = sh_w[st];
#pragma unroll 2
      for (int j = 0; j < cnt; ++j) {
        const float4 at = at4[j];
        const float4 e = EXACT ? atl[j] : at;  // position rounding errors (EXACT only)
        const float w = atw[j];
        if (MODE == kModeGrid) {
          const float base =
              EXACT ? dev::frac_product2_plus(sx[0], lx[0], at.x,
                                              dev::frac_product2_plus(sy[0], ly[0], at.y,
                                                                      fmaf(sx[0], e.x, fmaf(sy[0], e.y, at.w))))
                    : fmaf(sy[0], at.y, fmaf(sx[0], at.x, at.w));
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float f = EXACT ? dev::frac_rn(dev::frac_product2_plus(sz[r], lz[r], at.z, fmaf(sz[r], e.z, base)))
                                  : dev::frac_rn(fmaf(sz[r], at.z, base));
            float sn, cs;
            dev::sincos_cycles_mufu(f, &sn, &cs);
            acc[r].x = fmaf(w, cs, acc[r].x);
            acc[r].y = fmaf(w, sn, acc[r].y);
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float f =
                EXACT ? dev::frac_rn(dev::frac_product2_plus(
                            sx[r], lx[r], at.x,
                            dev::frac_product2_plus(
                                sy[r], ly[r], at.y,
                                dev::frac_product2_plus(sz[r], lz[r], at.z,
                                                        fmaf(sx[r], e.x, fmaf(sy[r], e.y, fmaf(sz[r], e.z, at.w)))))))
                      : dev::frac_rn(fmaf(sz[r], at.z, fmaf(sy[r], at.y, fmaf(sx[r], at.x, at.w))));
            float sn, cs;
            dev::sincos_cycles_mufu(f, &sn, &cs);
            acc[r].x = fmaf(w, cs, acc[r].x);
            acc[r].y = fmaf(w, sn, acc[r].y);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      sacc[r].x += acc[r].x;
      sacc[r].y += acc[r].y;
    }
    c_begin += cnt;
    if (c_begin >= end) {
      // end of a species segment: fold f_s(|S|)
      const float* cf = coef + kNCoef * segs[c_seg].species;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float Sx = H[0] + sx[r], Sy = H[1] + sy[r], Sz = H[2] + sz[r];
        const float s2 = (Sx * Sx + Sy * Sy + Sz * Sz) * inv4a2;
        const float2 F = ftab ? ftab[(int64_t)segs[c_seg].species * n_s + dev::min64(pbase + r * pstride, n_s - 1)]
                              : dev::form_factor(cf, s2);
        const float2 v = dev::cmul(F, sacc[r]);
        tot[r].x += v.x;
        tot[r].y += v.y;
        sacc[r] = make_float2(0.f, 0.f);
      }
      if (++c_seg < seg_hi) c_begin = segs[c_seg].begin;
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        dev::set_status(status, kStatusTimeout);
        // drain the copies this CTA still has in flight (bounded)
        for (int kk = k; kk < k + 2; ++kk)
          dev::mbar_wait_bounded(&sh_bar[kk & 1], (uint32_t)((kk >> 1) & 1), 1LL << 28);
      }
      return false;
    }
    if (tid == 0) issue(st);
    ++k;
  }
  return true;
}

// The exact-product sum of chunk_sum for R points, run as two passes of R/2
// points over the chunk's atoms.  The exact phases need the low parts of s
// besides everything the plain loop holds; halving the points per pass keeps
// the exact branch within the registers of the plain one, so the plain
// loop, the one that runs on common maps, keeps its register allocation.
// lo(r, &x, &y, &z) yields the low parts of point r.  Returns false if a
// wait gave up.
template <int MODE, int R, class LoFn>
__device__ __forceinline__ bool chunk_sum_exact_halves(
    const float4* __restrict__ atom4, const float4* __restrict__ atom_lo, const float* __restrict__ atom_w,
    const Segment* __restrict__ segs,
    int seg_lo, int seg_hi, const float* __restrict__ coef, const float H[3], float inv4a2, const float (&sx)[R],
    const float (&sy)[R], const float (&sz)[R], LoFn lo, float4 (*sh_atom)[kTile], float4 (*sh_lo)[kTile],
    float (*sh_w)[kTile], uint64_t* sh_bar, int& k, float2 (&tot)[R], unsigned* status, const float2* __restrict__ ftab, int64_t n_s,
    int64_t pbase, int64_t pstride) {
  static_assert(R % 2 == 0, "two halves of the thread's points");
  constexpr int R2 = R / 2;
#pragma unroll 1
  for (int half = 0; half < 2; ++half) {
    float hx[R2], hy[R2], hz[R2], lx[R2], ly[R2], lz[R2];
    float2 t2[R2];
#pragma unroll
    for (int r = 0; r < R2; ++r) {
      const int q = half * R2 + r;
      hx[r] = sx[q];
      hy[r] = sy[q];
      hz[r] = sz[q];
      lo(q, lx[r], ly[r], lz[r]);
    }
    if (!chunk_sum<MODE, R2, true>(atom4, atom_lo, atom_w, segs, seg_lo, seg_hi, coef, H, inv4a2, hx, hy, hz, lx,
                                   ly, lz, sh_atom, sh_lo, sh_w, sh_bar, k, t2, status, ftab, n_s,
                                   pbase + half * R2 * pstride, pstride))
      return false;
    // the next pass re-stages the chunk's tiles: every thread is done with
    // the shared stages of this one
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R2; ++r) tot[half * R2 + r] = t2[r];
  }
  return true;
}

}  // namespace scatter
