// Atom-parallel form of the generic sum, for many atoms and few reflections.
//
// The S-parallel kernel (forward.cu) gives every thread R reflections and
// streams all atoms past them; with a short S list it has too few threads to
// fill the GPU.  Section 3 names the alternative for that case: parallelise
// over the atoms and share the reflections.  Here a CTA holds one block of
// kApThreads * K atoms of a single species (K per thread, in registers) and
// one tile of up to kApPts reflections (in shared memory).  For every
// reflection each thread sums its K atoms (the same split phase, exact mod-1
// reduction and MUFU sincos as the generic kernel), the warp reduces by
// shuffles and the eight warps' sums meet in shared memory.  The CTA writes
// f_s(|S|) x T_block(S) to the partials [block][M]; k_reduce sums the blocks
// in order and applies the translation phase, as for split-K.
#include <cuda_runtime.h>
#include <algorithm>
#include <vector>
#include "device_common.cuh"
#include "generic_impl.cuh"
#include "launch.h"

namespace scatter {

constexpr int kApThreads = 256;
constexpr int kApWarps = kApThreads / 32;
constexpr int kApPts = 128;  // reflections per CTA tile

struct ApArgs {
  const float4* atom4;
  const float4* atom_lo;  // position rounding errors (exact-product phases)
  const float* atom_w;
  const Segment* blocks;  // species-uniform atom blocks of <= kApThreads * K slots
  const float* coef;
  int64_t n_s;
  const float* s_hi;      // LIST [3][M]
  const float* s_lo;      // LIST [3][M] rounding error of s_hi
  const float* axis_s;    // GRID [n0 | n1 | n2]
  const float* axis_lo;   // GRID [n0 | n1 | n2] rounding error of axis_s
  int64_t n0, n1, n2;
  int grid_mode;
  float H[3];
  float inv4a2;
  const float2* ftab;     // Eq. 4 factor table [n_species][M], or null (form factors)
  const unsigned long long* bbox;  // [6] this call's ordered min / max xyz
  const double* shift;             // [3] the call's centring t
  float smax[3];                   // max |S_d - H_d| over the points
  float2* partial;        // [block][M]
  int tile;               // reflections per CTA (<= kApPts)
};

// EXACT: the phase with its products' rounding errors restored and s and the
// positions as double-floats; the positions' low parts are read from L1
// (atom_lo at the thread's slots) rather than held in registers, which keeps
// the plain loop's register allocation.
template <int K, bool EXACT>
__device__ __forceinline__ void atompar_sums(const float4* sh_s, const float4* sh_slo, int np, const float (&x)[K],
                                             const float (&y)[K], const float (&z)[K], const float (&c)[K],
                                             const float (&w)[K], const float4* __restrict__ lo_base, int nk,
                                             float2 (*sh_part)[kApPts], int lane, int warp) {
  if constexpr (!EXACT && K % 2 == 0) {
    // two atoms per packed register pair (atoms 2k and 2k + 1 in the low and
    // high halves): every step is elementwise over the atoms and rounds like
    // its scalar form, and the halves of the packed sums are exactly the two
    // accumulator pairs (even and odd atoms) of the scalar loop below
    using u64 = unsigned long long;
    constexpr int KP = K / 2 > 0 ? K / 2 : 1;
    u64 x2[KP], y2[KP], z2[KP], c2[KP], w2[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      x2[k] = dev::pack2(x[2 * k], x[2 * k + 1]);
      y2[k] = dev::pack2(y[2 * k], y[2 * k + 1]);
      z2[k] = dev::pack2(z[2 * k], z[2 * k + 1]);
      c2[k] = dev::pack2(c[2 * k], c[2 * k + 1]);
      w2[k] = dev::pack2(w[2 * k], w[2 * k + 1]);
    }
    const u64 magic2 = dev::pack2(12582912.0f, 12582912.0f);  // 1.5 * 2^23: rint by addition
    const u64 twopi2 = dev::pack2(6.28318530717958647692f, 6.28318530717958647692f);
    for (int p = 0; p < np; ++p) {
      const float4 s = sh_s[p];
      const u64 sx = dev::pack2(s.x, s.x), sy = dev::pack2(s.y, s.y), sz = dev::pack2(s.z, s.z);
      u64 re2 = 0ull, im2 = 0ull;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        const u64 ph = dev::fma2(sz, z2[k], dev::fma2(sy, y2[k], dev::fma2(sx, x2[k], c2[k])));
        const u64 f = dev::sub2(ph, dev::sub2(dev::add2(ph, magic2), magic2));  // ph - rint(ph)
        float t0, t1;
        dev::unpack2(dev::mul2(f, twopi2), t0, t1);
        re2 = dev::fma2(w2[k], dev::pack2(__cosf(t0), __cosf(t1)), re2);
        im2 = dev::fma2(w2[k], dev::pack2(__sinf(t0), __sinf(t1)), im2);
      }
      float re0, re1, im0, im1;
      dev::unpack2(re2, re0, re1);
      dev::unpack2(im2, im0, im1);
      float re = re0 + re1, im = im0 + im1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) sh_part[warp][p] = make_float2(re, im);
    }
  } else {
    for (int p = 0; p < np; ++p) {
      const float4 s = sh_s[p];
      const float4 sl = EXACT ? sh_slo[p] : s;
      // two accumulator pairs halve the dependent FFMA chain
      float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (EXACT && k < nk) e = __ldg(lo_base + k * kApThreads);  // slots past the block's end: weight 0
        const float f = EXACT ? dev::frac_rn(dev::frac_product2_plus(
                                    s.x, sl.x, x[k],
                                    dev::frac_product2_plus(
                                        s.y, sl.y, y[k],
                                        dev::frac_product2_plus(s.z, sl.z, z[k],
                                                                fmaf(s.x, e.x, fmaf(s.y, e.y, fmaf(s.z, e.z, c[k])))))))
                              : dev::frac_rn(fmaf(s.z, z[k], fmaf(s.y, y[k], fmaf(s.x, x[k], c[k]))));
        float sn, cs;
        dev::sincos_cycles_mufu(f, &sn, &cs);
        if (k & 1) {
          re1 = fmaf(w[k], cs, re1);
          im1 = fmaf(w[k], sn, im1);
        } else {
          re0 = fmaf(w[k], cs, re0);
          im0 = fmaf(w[k], sn, im0);
        }
      }
      float re = re0 + re1, im = im0 + im1;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane == 0) sh_part[warp][p] = make_float2(re, im);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kApThreads, 2) k_atompar(const ApArgs a) {
  __shared__ float4 sh_s[kApPts];
  __shared__ float4 sh_slo[kApPts];  // rounding errors of sh_s (exact-product phases)
  __shared__ float2 sh_part[kApWarps][kApPts];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Segment blk = a.blocks[blockIdx.y];
  const int64_t p0 = (int64_t)blockIdx.x * a.tile;
  const int np = (int)dev::min64(a.tile, a.n_s - p0);

  // the tile's S offsets s = S - H
  for (int i = tid; i < np; i += kApThreads) {
    const int64_t m = p0 + i;
    float4 s, sl;
    if (a.grid_mode) {
      const int64_t i2 = m % a.n2, line = m / a.n2, i1 = line % a.n1, i0 = line / a.n1;
      s = make_float4(a.axis_s[i0], a.axis_s[a.n0 + i1], a.axis_s[a.n0 + a.n1 + i2], 0.f);
      sl = make_float4(a.axis_lo[i0], a.axis_lo[a.n0 + i1], a.axis_lo[a.n0 + a.n1 + i2], 0.f);
    } else {
      s = make_float4(a.s_hi[m], a.s_hi[a.n_s + m], a.s_hi[2 * a.n_s + m], 0.f);
      sl = make_float4(a.s_lo[m], a.s_lo[a.n_s + m], a.s_lo[2 * a.n_s + m], 0.f);
    }
    sh_s[i] = s;
    sh_slo[i] = sl;
  }
  // this thread's atoms (zero weight past the block's end)
  float x[K], y[K], z[K], c[K], w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int64_t slot = blk.begin + (int64_t)k * kApThreads + tid;
    const bool in = slot < blk.end;
    const float4 at = in ? a.atom4[slot] : make_float4(0.f, 0.f, 0.f, 0.f);
    x[k] = at.x;
    y[k] = at.y;
    z[k] = at.z;
    c[k] = at.w;
    w[k] = in ? a.atom_w[slot] : 0.f;
  }
  __syncthreads();

  // phases that can pass kPhaseExactLim cycles take the exact-product route
  // (one decision per call: every CTA computes the same)
  if (dev::phase_needs_exact(a.bbox, a.shift, a.smax))
    atompar_sums<K, true>(sh_s, sh_slo, np, x, y, z, c, w, a.atom_lo + blk.begin + tid,
                          (int)dev::max64(0, (blk.end - blk.begin - tid + kApThreads - 1) / kApThreads), sh_part, lane,
                          warp);
  else
    atompar_sums<K, false>(sh_s, sh_slo, np, x, y, z, c, w, a.atom_lo, 0, sh_part, lane, warp);
  __syncthreads();

  // the block's T(S) for this tile, times f_s(|S|) of its species
  const float* cf = a.coef + kNCoef * blk.species;
  for (int i = tid; i < np; i += kApThreads) {
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kApWarps; ++q) {
      v.x += sh_part[q][i].x;
      v.y += sh_part[q][i].y;
    }
    const float4 s = sh_s[i];
    const float Sx = a.H[0] + s.x, Sy = a.H[1] + s.y, Sz = a.H[2] + s.z;
    const float2 F = a.ftab ? a.ftab[(int64_t)blk.species * a.n_s + p0 + i]
                            : dev::form_factor(cf, (Sx * Sx + Sy * Sy + Sz * Sz) * a.inv4a2);
    a.partial[(int64_t)blockIdx.y * a.n_s + p0 + i] = dev::cmul(F, v);
  }
}

namespace {

void* pick_atompar(int K) {
  switch (K) {
    case 1: return (void*)&k_atompar<1>;
    case 2: return (void*)&k_atompar<2>;
    case 4: return (void*)&k_atompar<4>;
    case 8: return (void*)&k_atompar<8>;
    case 16: return (void*)&k_atompar<16>;
    default: return nullptr;
  }
}

// Species-uniform blocks of at most kApThreads * K slots of instance 0.
std::vector<Segment> atompar_blocks(const scatter_plan_s* p, int K) {
  std::vector<Segment> blocks;
  const int64_t cap = (int64_t)kApThreads * K;
  for (const Segment& sg : p->all_segs) {
    if (sg.instance != 0) continue;
    for (int64_t b = sg.begin; b < sg.end; b += cap)
      blocks.push_back(Segment{b, std::min(sg.end, b + cap), sg.species, 0});
  }
  return blocks;
}

}  // namespace

// Reflections per CTA.  Every CTA of a block costs the same (each thread
// runs all K of its atoms), so the call lasts ceil(CTAs / resident CTAs)
// waves of one CTA's time, which scales with its reflections plus a fixed
// part (its atoms' loads, the tile's S offsets, the block sums).  The tile
// that minimises that product fills the last wave: for 245 blocks x 1000
// reflections on 304 resident CTAs, 11 tiles of 91 (9 waves) instead of 8
// of 125 (7 waves, the last under half full).
int atompar_tile(int64_t n_s, int64_t n_blocks, int64_t resident) {
  if (n_s <= 0 || n_blocks <= 0 || resident <= 0) return kApPts;
  constexpr double kFixed = 6.0;  // the fixed part, in reflections
  const int64_t t_min = (n_s + kApPts - 1) / kApPts;
  double best = 1e300;
  int best_tile = kApPts;
  for (int64_t t = t_min; t <= 4 * t_min; ++t) {
    const int64_t tile = (n_s + t - 1) / t;
    const int64_t tiles = (n_s + tile - 1) / tile;
    const double waves = (double)((tiles * n_blocks + resident - 1) / resident);
    const double cost = waves * ((double)tile + kFixed);
    if (cost < best * 0.999) {
      best = cost;
      best_tile = (int)tile;
    }
  }
  return best_tile;
}

bool atompar_applicable(const scatter_plan_s* p) {
  return p->batch == 1 && (p->s_kind == SCATTER_S_LIST || p->s_kind == SCATTER_S_GRID) && p->n_s > 0;
}

int atompar_choose_k(const scatter_plan_s* p) {
  // the largest K that still gives two CTAs per SM
  const int64_t tiles = (p->n_s + kApPts - 1) / kApPts;
  for (int K : {16, 8, 4, 2})
    if (tiles * (int64_t)atompar_blocks(p, K).size() >= 2 * (int64_t)p->n_sm) return K;
  return atompar_blocks(p, 1).size() <= 65535 ? 1 : 16;
}

bool atompar_preferred(const scatter_plan_s* p, const Tiling& s_parallel) {
  if (!atompar_applicable(p)) return false;
  // warps the S-parallel kernel keeps busy: R reflections per thread, split-K
  // chunks per tile; below one warp per SM sub-partition it cannot hide the
  // MUFU latency, while the atom-parallel form spreads the atoms instead
  const double warps = std::ceil((double)p->n_s / s_parallel.R / 32.0) * s_parallel.split_k;
  return warps < 4.0 * p->n_sm && p->n_slots >= 16 * kApThreads;
}

scatter_status prepare_atompar(scatter_plan_s* p, int K) {
  if (!atompar_applicable(p)) return fail(SCATTER_ERR_UNSUPPORTED, "the atom-parallel form needs one instance");
  if (!pick_atompar(K)) return fail(SCATTER_ERR_INVALID_ARG, "atoms per thread must be 1, 2, 4, 8 or 16");
  std::vector<Segment> blocks = atompar_blocks(p, K);
  if (blocks.empty()) blocks.push_back(Segment{0, 0, 0, 0});  // no atoms: one empty block, zero map
  if (blocks.size() > 65535)
    return fail(SCATTER_ERR_UNSUPPORTED, "%zu atom blocks exceed the grid's y extent: use more atoms per thread",
                blocks.size());
  const size_t part = blocks.size() * (size_t)p->n_s;
  if (part * sizeof(float2) > ((size_t)1 << 31))
    return fail(SCATTER_ERR_UNSUPPORTED, "atom-parallel partials would exceed 2 GiB (%zu blocks x %lld points)",
                blocks.size(), (long long)p->n_s);
  cudaError_t e;
  if (p->d.ap_blocks) cudaFree(p->d.ap_blocks);
  p->d.ap_blocks = nullptr;
  if ((e = cudaMalloc(&p->d.ap_blocks, blocks.size() * sizeof(Segment))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc atom blocks");
  if ((e = cudaMemcpy(p->d.ap_blocks, blocks.data(), blocks.size() * sizeof(Segment), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return cuda_status(e, "atom blocks upload");
  if (p->d.partial) cudaFree(p->d.partial);
  p->d.partial = nullptr;
  if ((e = cudaMalloc(&p->d.partial, part * sizeof(float2))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc atom-parallel partials");
  p->tiling_bytes += (int64_t)(blocks.size() * sizeof(Segment) + part * sizeof(float2));
  p->ap_n_blocks = (int32_t)blocks.size();
  p->tiling.atom_k = K;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick_atompar(K), kApThreads, 0)) != cudaSuccess)
    return cuda_status(e, "atom-parallel occupancy");
  p->ap_tile = atompar_tile(p->n_s, (int64_t)blocks.size(), (int64_t)std::max(per_sm, 1) * p->n_sm);
  return SCATTER_OK;
}

scatter_status launch_atompar(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st) {
  void* fn = pick_atompar(p->tiling.atom_k);
  if (!fn || !p->d.ap_blocks) return fail(SCATTER_ERR_UNSUPPORTED, "atom-parallel tiling not prepared");
  ApArgs a{};
  a.atom4 = p->d.atom4;
  a.atom_lo = p->d.atom_lo;
  a.atom_w = p->d.atom_w;
  a.blocks = p->d.ap_blocks;
  a.coef = p->d.coef;
  a.n_s = p->n_s;
  a.s_hi = p->d.s_hi;
  a.s_lo = p->d.s_lo;
  a.axis_lo = p->d.axis_lo;
  a.axis_s = p->d.axis_s;
  a.n0 = p->n_axis[0];
  a.n1 = p->n_axis[1];
  a.n2 = p->n_axis[2];
  a.grid_mode = p->s_kind == SCATTER_S_GRID;
  for (int d = 0; d < 3; ++d) a.H[d] = (float)p->inst[0].H[d];
  a.inv4a2 = (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a));
  a.ftab = p->d.ftab;
  a.bbox = p->d.inst_bbox;
  a.shift = p->d.inst_shift;
  for (int d = 0; d < 3; ++d) a.smax[d] = (float)p->s_max[d];
  a.partial = p->d.partial;
  a.tile = p->ap_tile > 0 ? p->ap_tile : kApPts;
  dim3 grid((unsigned)((p->n_s + a.tile - 1) / a.tile), (unsigned)p->ap_n_blocks);
  void* args[] = {&a};
  timing_begin(p, st);
  cudaError_t e = cudaLaunchKernel(fn, grid, dim3(kApThreads), args, 0, st);
  timing_end(p, st);
  if (e != cudaSuccess) return cuda_status(e, "atom-parallel kernel launch");
  p->last_launches += 1;
  return launch_generic_reduce(p, p->ap_n_blocks, amp_out, int_out, st);
}

}  // namespace scatter
