// Grazing-incidence scattering in the distorted-wave Born approximation
// (Section 4.3): four beams, incident and exit waves each direct or
// reflected by the substrate, summed in one pass.
//
// For a map over (h, k, alpha_f) at fixed alpha_i (a/lambda = scale):
//   Sz1 = scale (sin a_i + sin a_f)   W1 = 1          (direct in, direct out)
//   Sz2 = scale (sin a_f - sin a_i)   W2 = R_i        (reflected in)
//   Sz3 = -Sz2                        W3 = R_f        (reflected out)
//   Sz4 = -Sz1                        W4 = R_i R_f    (reflected in and out)
//   A = sum_t W_t sum_s f_s(|S_t|) sum_{j in s} w_j exp(2 i pi S_t . r_j)
// with R the Fresnel reflection coefficient of the substrate.
//
// exp(2 i pi S_t . r) = E(h,k,r) Z_t(alpha_f, z) where
//   E   = w exp(2 i pi (c + s_h x' + s_k y'))      one MUFU sincos per atom and
//                                                  (h,k), shared by 4 alpha_f
//   Z1  = exp(2 i pi Sz1 z'), Z2 = exp(2 i pi Sz2 z'), Z3 = conj Z2, Z4 = conj Z1
// Z1, Z2 depend on (atom, alpha_f) only: a per-call table (accurate sincospif)
// streamed through shared memory by the TMA engine.  A warp's 32 lanes are
// 32 (h,k) points sharing the same alpha_f values, so the table reads are
// shared-memory broadcasts.  E Z and E conj(Z) are made of the same four real
// products, E Z = (P - Q, R + T) and E conj(Z) = (P + Q, T - R) with
// P = Er Zr, Q = Ei Zi, R = Er Zi, T = Ei Zr, and every beam is linear in the
// atom sums, so the kernel accumulates P, Q, R, T of Z1 and Z2 (8 FFMA per
// (atom, S point)) and forms the four beams once per 64-atom tile.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>
#include "device_common.cuh"
#include "launch.h"

namespace scatter {

constexpr int kDwbaTile = 64;      // atoms per stage
constexpr int kDwbaR = 4;          // alpha_f points per thread
constexpr int kDwbaWarps = 8;      // 8 warps x 4 = 32 alpha_f per CTA
constexpr int kDwbaThreads = 32 * kDwbaWarps;
constexpr int kAfBlock = kDwbaR * kDwbaWarps;  // 32
// stage: Z table tile (occupancy folded in), atom records, position rounding
// errors (exact instance)
constexpr size_t kDwbaStageBytes = (size_t)kDwbaTile * kAfBlock * 16 + kDwbaTile * 16 + kDwbaTile * 16;
constexpr size_t kDwbaSmem = 2 * kDwbaStageBytes;

struct DwbaArgs {
  const float4* atom4;
  const float4* atom_lo;   // FP32 rounding errors of the positions (exact instance)
  const float* atom_w;
  const Segment* segs;
  const int32_t* chunk_seg_off;
  const float* coef;
  const float4* ztab;      // [n_afb][n_slots][32] (Z1.re, Z1.im, Z2.re, Z2.im)
  int64_t n_slots;
  const float* axis_s;     // [n0 | n1 | n_af]: s_h, s_k (r.l.u. minus H), unused
  const float* axis_lo;    // rounding errors of axis_s (double-float s of the exact phases)
  const double* axis64;    // [n0 | n1 | n_af]: h, k, alpha_f
  const float* gid_sz;     // [2][n_af] Sz1, Sz2 (r.l.u.)
  const double* gid_sz64;  // [2][n_af]
  const float* gid_szf;    // [4][n_af] S_z of each beam's form factor
  const double* gid_sz64_im;  // [n_af] Im sigma of a buried object's beam, 0 on the substrate
  const float2* gid_w;     // [4][n_af]
  int64_t n0, n1, n_af;
  float H[3];
  double H64[3];
  float inv4a2;
  const double* shift;
  const unsigned long long* bbox;  // [6] this call's ordered min / max xyz
  float smax[3];                   // max |s_h|, |s_k| over the map (z: the table's business), 0
  float2* out_amp;
  float* out_int;
  float2* partial;
  int64_t n_s;
  unsigned* status;
};

// Z table of the call: w Z1, w Z2 for every slot and alpha_f (padded to 32),
// the atom's occupancy folded in.
__global__ void k_dwba_ztable(const float4* __restrict__ atom4, const float4* __restrict__ atom_lo,
                              const float* __restrict__ atom_w, const float* __restrict__ sz,
                              const float* __restrict__ sz_lo, const float* __restrict__ sz_im, int64_t n_slots,
                              int64_t n_af, int64_t n_afb, float4* __restrict__ ztab) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = n_afb * n_slots * kAfBlock;
  if (i >= total) return;
  const int af_l = (int)(i % kAfBlock);
  const int64_t slot = (i / kAfBlock) % n_slots;
  const int64_t afb = i / (kAfBlock * n_slots);
  const int64_t af = afb * kAfBlock + af_l;
  if (af >= n_af) {
    ztab[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // Sz z with Sz and z as double-floats (the products' low parts are far
  // below FP32 resolution unless the crystal is tall; they cost nothing here)
  const float z = atom4[slot].z, ez = atom_lo[slot].z;
  float s1, c1, s2, c2;
  sincospif(2.0f * (dev::frac_of_product2(sz[af], sz_lo[af], z) + sz[af] * ez), &s1, &c1);
  sincospif(2.0f * (dev::frac_of_product2(sz[n_af + af], sz_lo[n_af + af], z) + sz[n_af + af] * ez), &s2, &c2);
  // the occupancy rides in the table: w Z1, w Z2; a buried object's beam is
  // attenuated in the medium, |Z1| = exp(-2 pi Im(sigma) z') (Im sz = 0 otherwise)
  const float w = atom_w[slot];
  const float w1 = w * expf(-6.28318530717958647692f * sz_im[af] * (z + ez));
  const float w2 = w * expf(-6.28318530717958647692f * sz_im[n_af + af] * (z + ez));
  ztab[i] = make_float4(w1 * c1, w1 * s1, w2 * c2, w2 * s2);
}

// Tile sums of the four real products of E_j = w_j e^{2 pi i (s_h x'_j + s_k y'_j + c_j)}
// with each Z of the thread's rows: [P, Q, R, T] of Z1, then of Z2.  The
// products that share a factor of E run as packed pairs: (P, R) += Er (Zr, Zi)
// and (T, Q) += Ei (Zr, Zi), so the eight FMAs per (atom, point) issue as four
// fma.rn.f32x2 (the pipe's lane rate is unchanged; the issue slots halve,
// and the kernel is issue-bound).  EXACT: the phase with its products'
// rounding errors restored and s_h, s_k as double-floats (shl, skl their low
// parts; long crystals).
template <bool EXACT>
__device__ __forceinline__ void dwba_tile_products(const float4* zs, const float4* as, const float4* es, int cnt,
                                                   int af_l0, float sh, float sk, float shl, float skl,
                                                   float (&acc)[kDwbaR][8]) {
  unsigned long long pk[kDwbaR][4];  // (P1, R1), (T1, Q1), (P2, R2), (T2, Q2)
#pragma unroll
  for (int r = 0; r < kDwbaR; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) pk[r][q] = 0ull;
#pragma unroll 2
  for (int j = 0; j < cnt; ++j) {
    const float4 at = as[j];
    float f;
    if (EXACT) {
      const float4 e = es[j];  // the positions' FP32 rounding errors
      f = dev::frac_rn(dev::frac_product2_plus(
          sh, shl, at.x, dev::frac_product2_plus(sk, skl, at.y, fmaf(sh, e.x, fmaf(sk, e.y, at.w)))));
    } else {
      f = dev::frac_rn(fmaf(sk, at.y, fmaf(sh, at.x, at.w)));
    }
    float er, ei;  // E / w (the table carries w)
    dev::sincos_cycles_mufu(f, &ei, &er);
    const unsigned long long er2 = dev::pack2(er, er), ei2 = dev::pack2(ei, ei);
    const float4* zr = zs + j * kAfBlock + af_l0;
#pragma unroll
    for (int r = 0; r < kDwbaR; ++r) {
      const float4 z = zr[r];  // Z1 (re, im), Z2 (re, im)
      const unsigned long long z1 = dev::pack2(z.x, z.y), z2 = dev::pack2(z.z, z.w);
      dev::ffma2(pk[r][0], er2, z1);
      dev::ffma2(pk[r][1], ei2, z1);
      dev::ffma2(pk[r][2], er2, z2);
      dev::ffma2(pk[r][3], ei2, z2);
    }
  }
#pragma unroll
  for (int r = 0; r < kDwbaR; ++r) {
    dev::unpack2(pk[r][0], acc[r][0], acc[r][2]);  // P1, R1
    dev::unpack2(pk[r][1], acc[r][3], acc[r][1]);  // T1, Q1
    dev::unpack2(pk[r][2], acc[r][4], acc[r][6]);  // P2, R2
    dev::unpack2(pk[r][3], acc[r][7], acc[r][5]);  // T2, Q2
  }
}

// Launched twice per call, EXACT = false and true: every CTA of a call
// reaches the same phase bound, and the instance that does not match it
// returns at once, so each loop body is compiled on its own.
template <bool EXACT>
__global__ void __launch_bounds__(kDwbaThreads) k_dwba(const DwbaArgs a) {
  // long crystals: the per-atom phase with its products' rounding errors restored
  if (dev::phase_needs_exact(a.bbox, a.shift, a.smax) != EXACT) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t sh_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t hk = (int64_t)blockIdx.x * 32 + lane;
  const bool hk_ok = hk < a.n0 * a.n1;
  const int64_t i_h = hk_ok ? hk / a.n1 : 0, i_k = hk_ok ? hk % a.n1 : 0;
  const float sh = a.axis_s[i_h], sk = a.axis_s[a.n0 + i_k];
  const float shl = EXACT ? a.axis_lo[i_h] : 0.f, skl = EXACT ? a.axis_lo[a.n0 + i_k] : 0.f;
  const int64_t afb = blockIdx.y;
  const int af_l0 = warp * kDwbaR;
  const int64_t af0 = afb * kAfBlock + af_l0;
  const int chunk = blockIdx.z;

  auto stage_z = [&](int s) { return reinterpret_cast<float4*>(smem + s * kDwbaStageBytes); };
  auto stage_a = [&](int s) {
    return reinterpret_cast<float4*>(smem + s * kDwbaStageBytes + (size_t)kDwbaTile * kAfBlock * 16);
  };
  auto stage_e = [&](int s) {
    return reinterpret_cast<float4*>(smem + s * kDwbaStageBytes + (size_t)kDwbaTile * kAfBlock * 16 + kDwbaTile * 16);
  };

  const int seg_lo = a.chunk_seg_off[chunk], seg_hi = a.chunk_seg_off[chunk + 1];
  if (tid == 0) {
    dev::mbar_init(&sh_bar[0], 1);
    dev::mbar_init(&sh_bar[1], 1);
    dev::mbar_fence_init();
  }
  __syncthreads();
  int l_seg = seg_lo;
  int64_t l_begin = seg_lo < seg_hi ? a.segs[seg_lo].begin : 0;
  const float4* zbase = a.ztab + afb * a.n_slots * kAfBlock;
  auto issue = [&](int st) {
    if (l_seg >= seg_hi) return;
    const int64_t end = a.segs[l_seg].end;
    const int cnt = (int)dev::min64(kDwbaTile, end - l_begin);
    dev::mbar_arrive_expect_tx(&sh_bar[st], (uint32_t)cnt * (kAfBlock * 16u + (EXACT ? 32u : 16u)));
    dev::bulk_g2s(stage_z(st), zbase + l_begin * kAfBlock, (uint32_t)cnt * kAfBlock * 16u, &sh_bar[st]);
    dev::bulk_g2s(stage_a(st), a.atom4 + l_begin, (uint32_t)cnt * 16u, &sh_bar[st]);
    if (EXACT) dev::bulk_g2s(stage_e(st), a.atom_lo + l_begin, (uint32_t)cnt * 16u, &sh_bar[st]);
    l_begin += cnt;
    if (l_begin >= end && ++l_seg < seg_hi) l_begin = a.segs[l_seg].begin;
  };
  if (tid == 0) {
    issue(0);
    issue(1);
  }

  float2 seg[kDwbaR][4], tot[kDwbaR];
#pragma unroll
  for (int r = 0; r < kDwbaR; ++r) {
    tot[r] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < 4; ++t) seg[r][t] = make_float2(0.f, 0.f);
  }
  int c_seg = seg_lo;
  int64_t c_begin = seg_lo < seg_hi ? a.segs[seg_lo].begin : 0;
  int k = 0;
  bool aborted = false;
  while (c_seg < seg_hi) {
    const int64_t end = a.segs[c_seg].end;
    const int cnt = (int)dev::min64(kDwbaTile, end - c_begin);
    const int st = k & 1;
    const bool ok = dev::mbar_wait_bounded(&sh_bar[st], (uint32_t)((k >> 1) & 1));
    // tile sums of the four real products per Z: [P, Q, R, T] of Z1, then of Z2
    float acc[kDwbaR][8];
#pragma unroll
    for (int r = 0; r < kDwbaR; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[r][q] = 0.f;
    if (ok) {
      dwba_tile_products<EXACT>(stage_z(st), stage_a(st), stage_e(st), cnt, af_l0, sh, sk, shl, skl, acc);
    }
    // beams of the tile: E Z1, E Z2, E conj(Z2), E conj(Z1)
#pragma unroll
    for (int r = 0; r < kDwbaR; ++r) {
      const float* q = acc[r];
      seg[r][0].x += q[0] - q[1];
      seg[r][0].y += q[2] + q[3];
      seg[r][1].x += q[4] - q[5];
      seg[r][1].y += q[6] + q[7];
      seg[r][2].x += q[4] + q[5];
      seg[r][2].y += q[7] - q[6];
      seg[r][3].x += q[0] + q[1];
      seg[r][3].y += q[3] - q[2];
    }
    c_begin += cnt;
    if (c_begin >= end) {
      // fold W_t f_s(|S_t|) e^{2 pi i s_t . t} into the map
      const float* cf = a.coef + kNCoef * a.segs[c_seg].species;
      const double* tt = a.shift;
      const bool shifted = tt[0] != 0.0 || tt[1] != 0.0 || tt[2] != 0.0;
      const float Sx = a.H[0] + sh, Sy = a.H[1] + sk;
#pragma unroll
      for (int r = 0; r < kDwbaR; ++r) {
        const int64_t af = af0 + r < a.n_af ? af0 + r : a.n_af - 1;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float szf = a.gid_szf[t * a.n_af + af];
          const float s2 = (Sx * Sx + Sy * Sy + szf * szf) * a.inv4a2;
          float2 wf = dev::cmul(a.gid_w[t * a.n_af + af], dev::form_factor(cf, s2));
          if (shifted) {
            const double z64 = (t == 0 || t == 3 ? a.gid_sz64[af] : a.gid_sz64[a.n_af + af]) * (t < 2 ? 1.0 : -1.0);
            wf = dev::cmul(dev::shift_phase(a.axis64[i_h] - a.H64[0], a.axis64[a.n0 + i_k] - a.H64[1], z64, tt), wf);
            if (t == 0) {  // a buried object's attenuation over the centring shift
              const float att = (float)exp(-6.283185307179586 * a.gid_sz64_im[af] * tt[2]);
              wf.x *= att;
              wf.y *= att;
            }
          }
          const float2 v = dev::cmul(wf, seg[r][t]);
          tot[r].x += v.x;
          tot[r].y += v.y;
          seg[r][t] = make_float2(0.f, 0.f);
        }
      }
      if (++c_seg < seg_hi) c_begin = a.segs[c_seg].begin;
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      break;
    }
    if (tid == 0) issue(st);
    ++k;
  }
  if (aborted) {
    if (tid == 0) {
      dev::set_status(a.status, kStatusTimeout);
      for (int kk = k; kk < k + 2; ++kk) dev::mbar_wait_bounded(&sh_bar[kk & 1], (uint32_t)((kk >> 1) & 1), 1LL << 28);
    }
    return;
  }
  if (!hk_ok) return;
#pragma unroll
  for (int r = 0; r < kDwbaR; ++r) {
    if (af0 + r >= a.n_af) continue;
    const int64_t m = hk * a.n_af + af0 + r;
    if (a.partial) {
      a.partial[(int64_t)chunk * a.n_s + m] = tot[r];
    } else {
      if (a.out_amp) a.out_amp[m] = tot[r];
      if (a.out_int) a.out_int[m] = tot[r].x * tot[r].x + tot[r].y * tot[r].y;
    }
  }
}

__global__ void k_dwba_reduce(const float2* partial, int split, int64_t n_s, float2* out_amp, float* out_int) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_s) return;
  float2 v = make_float2(0.f, 0.f);
  for (int c = 0; c < split; ++c) {
    const float2 p = partial[(int64_t)c * n_s + m];
    v.x += p.x;
    v.y += p.y;
  }
  if (out_amp) out_amp[m] = v;
  if (out_int) out_int[m] = v.x * v.x + v.y * v.y;
}

// Plain FP64 four-beam sum (no tables, no splitting), the GPU comparator.
__global__ void __launch_bounds__(128) k_f64_gid(const double* __restrict__ xyz, const float* __restrict__ occ,
                                                 const int32_t* __restrict__ slot_src, const Segment* __restrict__ segs,
                                                 int n_segs, const double* __restrict__ coef64,
                                                 const double* __restrict__ axis64, const double* __restrict__ sz64,
                                                 const double* __restrict__ szf64, const double* __restrict__ sz64_im,
                                                 const double2* __restrict__ w64, int64_t n0, int64_t n1,
                                                 int64_t n_af, double inv4a2, float2* out_amp, float* out_int) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n0 * n1 * n_af) return;
  const int64_t af = m % n_af, hk = m / n_af, i_k = hk % n1, i_h = hk / n1;
  const double h = axis64[i_h], kk = axis64[n0 + i_k];
  const double sz1 = sz64[af], sz2 = sz64[n_af + af];
  const double szt[4] = {sz1, sz2, -sz2, -sz1};
  double are = 0.0, aim = 0.0;
  for (int t = 0; t < 4; ++t) {
    const double2 W = w64[t * n_af + af];
    if (W.x == 0.0 && W.y == 0.0) continue;  // a buried object: one beam
    const double szf = szf64[t * n_af + af];
    const double s2 = (h * h + kk * kk + szf * szf) * inv4a2;
    const double im = t == 0 ? sz64_im[af] : 0.0;
    double tr_all = 0.0, ti_all = 0.0;
    for (int g = 0; g < n_segs; ++g) {
      const Segment sg = segs[g];
      const double* cf = coef64 + kNCoef * sg.species;
      double f0 = cf[8];
      for (int i = 0; i < 4; ++i) f0 += cf[i] * exp(-cf[4 + i] * s2);
      const double dw = exp(-cf[11] * s2);
      const double fr = (f0 + cf[9]) * dw, fi = cf[10] * dw;
      double tr = 0.0, ti = 0.0;
      for (int64_t slot = sg.begin; slot < sg.end; ++slot) {
        const int32_t j = slot_src[slot];
        if (j < 0) continue;
        const double* r = xyz + 3 * (int64_t)j;
        const double w = occ ? (double)occ[j] : 1.0;
        double sn, cs;
        sincospi(2.0 * (h * r[0] + kk * r[1] + szt[t] * r[2]), &sn, &cs);
        const double wa = im != 0.0 ? w * exp(-2.0 * 3.14159265358979323846 * im * r[2]) : w;
        tr += wa * cs;
        ti += wa * sn;
      }
      tr_all += fr * tr - fi * ti;
      ti_all += fr * ti + fi * tr;
    }
    are += W.x * tr_all - W.y * ti_all;
    aim += W.x * ti_all + W.y * tr_all;
  }
  if (out_amp) out_amp[m] = make_float2((float)are, (float)aim);
  if (out_int) out_int[m] = (float)(are * are + aim * aim);
}

// Beam combination of a map computed on the virtual grid (h, k, beams x
// alpha_f): [Sz1 | Sz2 | -Sz2 | -Sz1] on the substrate, [Re sigma] for a
// buried object:  A = sum_t W_t(alpha_f) T_t.  f_s(|S_t|), the translation
// phase and (buried) the attenuation are already in T.
__global__ void k_gid_combine(const float2* __restrict__ virt, const float2* __restrict__ w, int64_t n_hk,
                              int64_t n_af, int n_beams, float2* out_amp, float* out_int) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_hk * n_af) return;
  const int64_t af = m % n_af, hk = m / n_af;
  const float2* row = virt + hk * n_beams * n_af + af;
  float2 v = make_float2(0.f, 0.f);
  for (int t = 0; t < n_beams; ++t) {
    const float2 c = dev::cmul(w[t * n_af + af], row[t * n_af]);
    v.x += c.x;
    v.y += c.y;
  }
  if (out_amp) out_amp[m] = v;
  if (out_int) out_int[m] = v.x * v.x + v.y * v.y;
}

scatter_status launch_gid_combine(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st) {
  const int64_t n_hk = p->n_axis[0] * p->n_axis[1], n_af = p->n_axis[2];
  k_gid_combine<<<(unsigned)((n_hk * n_af + 255) / 256), 256, 0, st>>>(p->d.sep_virt, p->d.gid_w, n_hk, n_af,
                                                                      (int)p->sep_beams, amp_out, int_out);
  p->last_launches += 1;
  return cuda_status(cudaGetLastError(), "gid combine launch");
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

std::complex<double> fresnel_r(double alpha, double delta, double beta) {
  const std::complex<double> n(1.0 - delta, beta);
  const double ca = std::cos(alpha);
  const std::complex<double> kz(std::sin(alpha), 0.0);
  const std::complex<double> kt = std::sqrt(n * n - ca * ca);  // principal branch: Im >= 0 here
  return (kz - kt) / (kz + kt);
}

// sin of the refracted angle in the substrate, q = sqrt(n^2 - cos^2 alpha)
// (principal branch: Im q >= 0, the field decays into the substrate)
std::complex<double> refracted_sin(double alpha, double delta, double beta) {
  const std::complex<double> n(1.0 - delta, beta);
  const double ca = std::cos(alpha);
  return std::sqrt(n * n - ca * ca);
}

}  // namespace

int dwba_blocks_per_sm() {
  static int cached = 0;
  if (cached) return cached;
  cudaFuncSetAttribute(k_dwba<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwbaSmem);
  cudaFuncSetAttribute(k_dwba<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDwbaSmem);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_dwba<false>, kDwbaThreads, kDwbaSmem) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  cached = nb > 0 ? nb : 1;
  return cached;
}

int64_t dwba_num_tiles(const scatter_plan_s* p) {
  return ((p->n_axis[0] * p->n_axis[1] + 31) / 32) * ((p->n_axis[2] + kAfBlock - 1) / kAfBlock);
}

// Host tables of a grazing-incidence plan: Sz1, Sz2 per alpha_f and the four
// beam weights (Fresnel coefficients in FP64), plus the Z-table workspace.
scatter_status prepare_gid(scatter_plan_s* p) {
  const int64_t n_af = p->n_axis[2];
  const double scale = p->lattice_a / p->wavelength;
  const std::complex<double> Ri = fresnel_r(p->alpha_i, p->delta, p->beta);
  const std::complex<double> qi = refracted_sin(p->alpha_i, p->delta, p->beta);
  const bool buried = p->gid_mode == 1;
  std::vector<double> sz64(2 * n_af), szf64(4 * n_af), sz64_im(n_af, 0.0);
  std::vector<float> sz(2 * n_af), sz_lo(2 * n_af), sz_im(2 * n_af, 0.f), szf(4 * n_af);
  std::vector<double2> w64(4 * n_af);
  std::vector<float2> w32(4 * n_af);
  for (int64_t i = 0; i < n_af; ++i) {
    const double af = p->axis_host[2][i];
    const double s1 = scale * (std::sin(p->alpha_i) + std::sin(af)), s2 = scale * (std::sin(af) - std::sin(p->alpha_i));
    const std::complex<double> Rf = fresnel_r(af, p->delta, p->beta);
    std::complex<double> W[4] = {1.0, Ri, Rf, Ri * Rf};
    double szf_t[4] = {s1, s2, -s2, -s1};
    if (!buried) {
      sz64[i] = s1;
      sz64[n_af + i] = s2;
    } else {
      // one beam, transmitted in and out, refracted and attenuated in the medium
      const std::complex<double> sigma = scale * (std::conj(qi) + std::conj(refracted_sin(af, p->delta, p->beta)));
      sz64[i] = sigma.real();
      sz64[n_af + i] = 0.0;
      sz64_im[i] = sigma.imag();
      sz_im[i] = (float)sigma.imag();
      W[0] = (1.0 + Ri) * (1.0 + Rf);
      W[1] = W[2] = W[3] = 0.0;
      szf_t[1] = szf_t[2] = szf_t[3] = 0.0;
    }
    for (int t = 0; t < 4; ++t) {
      w64[t * n_af + i] = make_double2(W[t].real(), W[t].imag());
      w32[t * n_af + i] = make_float2((float)W[t].real(), (float)W[t].imag());
      szf64[t * n_af + i] = szf_t[t];
      szf[t * n_af + i] = (float)szf_t[t];
    }
    p->s_max[2] = std::max(p->s_max[2], std::fabs(sz64[i]));
    for (int64_t q : {i, n_af + i}) {
      sz[q] = (float)sz64[q];
      sz_lo[q] = (float)(sz64[q] - (double)sz[q]);
    }
  }
  cudaError_t e;
  auto up = [&](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t r = cudaMalloc(dst, bytes);
    if (r != cudaSuccess) return r;
    p->base_bytes += (int64_t)bytes;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  p->gid_sz_host = sz64;
  p->gid_sz_im_host = sz64_im;
  p->gid_szf_host = szf64;
  if ((e = up((void**)&p->d.gid_sz, sz.data(), sz.size() * sizeof(float))) != cudaSuccess) return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_sz_lo, sz_lo.data(), sz_lo.size() * sizeof(float))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_sz_im, sz_im.data(), sz_im.size() * sizeof(float))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_szf, szf.data(), szf.size() * sizeof(float))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_szf64, szf64.data(), szf64.size() * sizeof(double))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_sz64_im, sz64_im.data(), sz64_im.size() * sizeof(double))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_sz64, sz64.data(), sz64.size() * sizeof(double))) != cudaSuccess)
    return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_w, w32.data(), w32.size() * sizeof(float2))) != cudaSuccess) return cuda_status(e, "gid");
  if ((e = up((void**)&p->d.gid_w64, w64.data(), w64.size() * sizeof(double2))) != cudaSuccess)
    return cuda_status(e, "gid");
  const int64_t n_afb = (n_af + kAfBlock - 1) / kAfBlock;
  const size_t zbytes = (size_t)n_afb * (size_t)std::max<int64_t>(p->n_slots, 1) * kAfBlock * sizeof(float4);
  if ((e = cudaMalloc((void**)&p->d.ztab, zbytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc z table");
  p->base_bytes += (int64_t)zbytes;
  return SCATTER_OK;
}

int dwba_best_split(const scatter_plan_s* p) {
  const double tiles = (double)dwba_num_tiles(p);
  const double cap = (double)p->n_sm * dwba_blocks_per_sm();
  const double n = (double)std::max<int64_t>(p->n_slots, 1);
  double best = 1e300;
  int best_k = 1;
  for (int k = 1; k <= 64; ++k) {
    if (k > 1 && n / k < 256) break;
    const double cost = std::ceil(tiles * k / cap) * (n / k + 128.0) + (k > 1 ? 0.02 * k * (double)p->n_s / cap : 0.0);
    if (cost < best * 0.995) {
      best = cost;
      best_k = k;
    }
  }
  return best_k;
}

scatter_status launch_dwba(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st) {
  const int64_t n_af = p->n_axis[2];
  const int64_t n_afb = (n_af + kAfBlock - 1) / kAfBlock;
  if (p->n_slots > 0) {
    const int64_t total = n_afb * p->n_slots * kAfBlock;
    k_dwba_ztable<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(p->d.atom4, p->d.atom_lo, p->d.atom_w,
                                                                    p->d.gid_sz, p->d.gid_sz_lo, p->d.gid_sz_im,
                                                                    p->n_slots, n_af, n_afb, p->d.ztab);
    p->last_launches += 1;
  }
  DwbaArgs a{};
  a.atom4 = p->d.atom4;
  a.atom_lo = p->d.atom_lo;
  a.atom_w = p->d.atom_w;
  a.segs = p->d.segs;
  a.chunk_seg_off = p->d.chunk_seg_off;
  a.coef = p->d.coef;
  a.ztab = p->d.ztab;
  a.n_slots = p->n_slots;
  a.axis_s = p->d.axis_s;
  a.axis_lo = p->d.axis_lo;
  a.axis64 = p->d.axis64;
  a.gid_sz = p->d.gid_sz;
  a.gid_sz64 = p->d.gid_sz64;
  a.gid_szf = p->d.gid_szf;
  a.gid_sz64_im = p->d.gid_sz64_im;
  a.gid_w = p->d.gid_w;
  a.n0 = p->n_axis[0];
  a.n1 = p->n_axis[1];
  a.n_af = n_af;
  for (int d = 0; d < 3; ++d) {
    a.H[d] = (float)p->inst[0].H[d];
    a.H64[d] = p->inst[0].H[d];
  }
  a.inv4a2 = (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a));
  a.shift = p->d.inst_shift;
  a.bbox = p->d.inst_bbox;
  a.smax[0] = (float)p->s_max[0];
  a.smax[1] = (float)p->s_max[1];
  a.smax[2] = 0.f;  // the Z table takes exact products itself
  a.n_s = p->n_s;
  a.status = p->d.status;
  const int n_chunks = (int)p->chunk_seg_off.size() - 1;
  if (n_chunks > 1) {
    a.partial = p->d.partial;
  } else {
    a.out_amp = amp_out;
    a.out_int = int_out;
  }
  dwba_blocks_per_sm();  // sets the dynamic shared memory attribute
  dim3 grid((unsigned)((p->n_axis[0] * p->n_axis[1] + 31) / 32), (unsigned)n_afb, (unsigned)std::max(n_chunks, 1));
  timing_begin(p, st);
  k_dwba<false><<<grid, kDwbaThreads, kDwbaSmem, st>>>(a);
  k_dwba<true><<<grid, kDwbaThreads, kDwbaSmem, st>>>(a);
  timing_end(p, st);
  p->last_launches += 2;
  if (n_chunks > 1) {
    k_dwba_reduce<<<(unsigned)((p->n_s + 255) / 256), 256, 0, st>>>(p->d.partial, n_chunks, p->n_s, amp_out, int_out);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "dwba launch");
}

scatter_status launch_f64_gid(scatter_plan_t p, const double* xyz, const float* occ, float2* amp_out, float* int_out,
                              cudaStream_t st) {
  const int64_t nb = (p->n_s + 127) / 128;
  timing_begin(p, st);
  k_f64_gid<<<(unsigned)nb, 128, 0, st>>>(xyz, occ, p->d.slot_src, p->d.segs, (int)p->segs.size(), p->d.coef64,
                                          p->d.axis64, p->d.gid_sz64, p->d.gid_szf64, p->d.gid_sz64_im, p->d.gid_w64,
                                          p->n_axis[0], p->n_axis[1],
                                          p->n_axis[2], 1.0 / (4.0 * p->lattice_a * p->lattice_a), amp_out, int_out);
  timing_end(p, st);
  p->last_launches += 1;
  return cuda_status(cudaGetLastError(), "fp64 gid launch");
}

}  // namespace scatter
