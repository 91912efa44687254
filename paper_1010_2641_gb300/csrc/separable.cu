// Separable tensor-core path for axis-aligned S grids (tcgen05, sm_103a).
//
// On a grid S = H + (s_a, s_b, s_c) the phase of Eq. 2 separates,
//   w_j exp(2 i pi (c_j + s_a x'_j + s_b y'_j + s_c z'_j)) = Xw[a,j] B[(b,c),j]
// with Xw = w e^{2 pi i s_a x'} and B = e^{2 pi i (s_b y' + s_c z' + c)},
// so the per-species sum is a complex matrix product over the atoms:
//   T_s[a, (b,c)] = sum_{j in s} Xw[a,j] B[(b,c), j].
// It runs as a real GEMM D = A B^T on the 5th-generation tensor cores:
//   A  (M = 2 n_a rows: Re/Im of each a) x (K = 2 per atom: Re/Im):
//      rows 2a: [Xwr, -Xwi], rows 2a+1: [Xwi, Xwr]  -> D[2a] = Re T, D[2a+1] = Im T
//   B  (N = (b,c) points) x (K): [Br, Bi]
// Both operands are split into f16 hi + lo parts and three products
// (hi.hi + hi.lo + lo.hi) accumulate in FP32 in tensor memory (TMEM), which
// keeps the result near FP32 accuracy (the lo.lo term is below 2^-22).
//
// Per call: k_sep_tab_a writes the A operand (hi/lo, already in the
// canonical no-swizzle K-major shared-memory layout, one 16 KB block per
// (M tile, 16-atom step), the two tiles of a pair adjacent).
// k_sep: CTA = a pair of 128-row M tiles (two 128 x 256 FP32
// accumulators filling the 512 TMEM columns) x one 256-point N tile x one
// atom chunk; per 16-atom step the TMA engine copies the pair's A blocks
// and the step's 16 atom records (y', z', c), every thread computes its
// point's row of B from them (FP32 phase, exact reduction mod 1, MUFU
// sincos, f16 split) into shared memory once for both tiles, and one
// thread issues 12 tcgen05.mma (2 tiles x 2 K16 sub-steps x 3 products,
// M=128 N=256).  Warp roles: eight warps form B (and read the accumulators
// out), one warp issues the MMAs, one warp issues the copies (a 32 KB bulk
// copy holds its issuing thread for ~1000 cycles, so it must not be the MMA
// thread).  A four-stage ring for the A blocks, an eight-stage ring for the
// atom records and a two-stage ring for the B blocks, each stage with a
// full and an empty mbarrier, keep the formation of step k+1 and the copies
// of later steps overlapped with the MMAs of step k.  The MMAs read ~96 B/clk of shared memory on their own;
// computing B from the atom records, instead of loading tabulated factors
// through L1, keeps the rest of the shared-memory traffic to the A copies
// and the B stores.
// Atom chunks (grid y) hold one species each.  Every 256 steps and at the
// end of the chunk the accumulator is read from TMEM (tcgen05.ld) and added
// into FP32 partials owned by the CTA, in the accumulator's 32 x 32 blocks
// (sep_part_off; shorter groups keep the
// tensor core's FP32 accumulation error down); k_sep_reduce sums the chunks
// in order, each times its species' f_s(|S|), and applies the translation
// phase.
// The same kernel, with the roles of the operands swapped, runs the adjoint
// on grids (adjoint_sep.cu); the arguments in sep_common.cuh cover both.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>
#include "launch.h"
#include "sep_common.cuh"
#include "tuner.h"

namespace scatter {

// -------------------------------------------------------------------------
// tables
// -------------------------------------------------------------------------

struct SepTabArgs {
  const float4* atom4;
  const float4* atom_lo;  // position rounding errors
  const float* atom_w;
  const float* axis_s;  // [n0 | n1 | n2] s values
  const float* axis_lo; // their FP32 rounding errors (s as a double-float)
  int64_t n0, n1, n2;
  int64_t n_slots, n_steps, n_mt;
  uint4* A;             // [n_mt/2][n_steps][2 tiles][hi|lo][4 kb][16 mg][8 rows] of 16 B
};

// One thread per 16-byte row of a core matrix of the A operand (4 atoms x
// Re/Im of one row m), hi and lo parts; the weight w_j is folded in here.
__global__ void k_sep_tab_a(const SepTabArgs t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = t.n_mt * t.n_steps * 4 * kSepM;
  // total is a multiple of 512: whole warps leave here, the shuffles below
  // always see all 32 lanes
  if (i >= total) return;
  const int r = (int)(i % 8), mg = (int)((i / 8) % 16), kb = (int)((i / 128) % 4);
  const int64_t ks = (i / 512) % t.n_steps, mt = i / (512 * t.n_steps);
  const int64_t m = mt * kSepM + mg * 8 + r;
  const int64_t a = m >> 1;
  const int ri = (int)(m & 1);
  const bool ok = a < t.n0;
  const float sa = ok ? t.axis_s[a] : 0.f, sal = ok ? t.axis_lo[a] : 0.f;
  float x[2] = {0.f, 0.f}, xl[2] = {0.f, 0.f}, w[2] = {0.f, 0.f};
  if (ok) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t slot = ks * kSepStep + kb * 4 + 2 * ri + u;
      x[u] = t.atom4[slot].x;
      xl[u] = t.atom_lo[slot].x;
      w[u] = t.atom_w[slot];
    }
  }
  uint4 hi, lo;
  sep_a_row(sa, sal, ok, ri, x, xl, w, hi, lo);
  uint4* blk = t.A + (((mt >> 1) * t.n_steps + ks) * kSepPair + (mt & 1)) * (kSepABytes / 16);
  const int64_t off = (int64_t)(kb * 16 + mg) * 8 + r;
  blk[off] = hi;
  blk[512 + off] = lo;
}

// -------------------------------------------------------------------------
// main kernel
// -------------------------------------------------------------------------


// Warp roles: warps 0..7 form the B rows (one point per thread) and read the
// accumulators out at every group end; warp 8 (one lane) issues the MMAs;
// warp 9 (one lane) issues the TMA copies.  Hand-offs go through mbarriers
// only:
//   bar_full[a]   A block of a step arrived            (TMA, 1 arrival + bytes)
//   bar_done[a]   MMAs of the step done (one commit per step); frees the A
//                 stage of that step and the B stage it read
//   bar_atom[t]   atom records of a step arrived       (TMA)
//   bar_tempty[t] atom records read by the formation   (8 warps)
//   bar_bfull[b]  B block of a step formed             (8 warps)
//   bar_tfree     accumulators read out after a group end (8 warps)
__global__ void __maxnreg__(168) k_sep(const SepArgs a) {
  // a B stage is freed by the done barrier of the step that read it: the A
  // ring (and with it the done ring) must be at least as deep as the B ring
  static_assert(kSepBStages <= kSepAStages, "B-stage reuse is tracked on the done ring");
  extern __shared__ __align__(1024) unsigned char sep_smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kSepAStages];
  __shared__ __align__(8) uint64_t bar_done[kSepAStages];
  __shared__ __align__(8) uint64_t bar_atom[kSepTStages];
  __shared__ __align__(8) uint64_t bar_tempty[kSepTStages];
  __shared__ __align__(8) uint64_t bar_bfull[kSepBStages];
  __shared__ __align__(8) uint64_t bar_tfree;
  __shared__ __align__(16) float4 ring_atom[kSepTStages][kSepStep];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(sep_smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ringA = smem;
  unsigned char* ringB = smem + kSepAStages * kSepPair * kSepABytes;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == kSepFormWarps, copy_warp = warp == kSepFormWarps + 1;
  const int64_t n_mp = a.mp_count > 0 ? a.mp_count : (a.n_mt + 1) / 2;  // pairs of this launch
  const int64_t mp = a.mp_first + blockIdx.x % n_mp, nt = blockIdx.x / n_mp;
  const int ntp = 2 * mp + 1 < a.n_mt ? 2 : 1;  // M tiles of this CTA with rows
  const int chunk = blockIdx.y;
  const int64_t nbc = a.n1 * a.n2;
  // this CTA's columns [col_base, col_end) and the species of its A table
  int64_t col_base = nt * kSepN, col_end = nbc;
  int a_species = 0;
  if (a.ntiles) {
    const Segment t = a.ntiles[nt];
    col_base = t.begin;
    col_end = t.end;
    a_species = t.species;
  }

  if (mma_warp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dev::smem_addr(&tmem_slot)),
                 "r"(kSepTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kSepAStages; ++s) {
      dev::mbar_init(&bar_full[s], 1);
      dev::mbar_init(&bar_done[s], 1);
    }
    for (int s = 0; s < kSepTStages; ++s) {
      dev::mbar_init(&bar_atom[s], 1);
      dev::mbar_init(&bar_tempty[s], kSepFormWarps);
    }
    for (int s = 0; s < kSepBStages; ++s) {
      dev::mbar_init(&bar_bfull[s], kSepFormWarps);
    }
    dev::mbar_init(&bar_tfree, kSepFormWarps);
    s_abort = 0;
    dev::mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // the chunk's steps (record bounds on step edges)
  const int64_t ks_begin = a.chunks[chunk].begin / kSepStep, ks_end = a.chunks[chunk].end / kSepStep;
  SepGroups grp{ks_end, ks_begin};
  bool ok = true;
  // copies issued and MMA steps committed (steps), for the drain on abort
  int64_t a_issued = 0, t_issued = 0, g_committed = 0;

  if (copy_warp) {
    if (lane == 0) {
      // A block and K records of every step, in step order; a stage is
      // refilled once its previous contents were consumed
      const uint4* Ablk = a.A + a_species * a.a_sp_stride + mp * a.n_steps * (kSepPair * kSepABytes / 16);
      const uint32_t a_bytes = (uint32_t)ntp * kSepABytes;
      int64_t g = 0;
      for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
        if (s_abort) {
          ok = false;
          break;
        }
        const int tst = (int)(g % kSepTStages), ast = (int)(g % kSepAStages);
        if (g >= kSepTStages &&
            !dev::mbar_wait_bounded(&bar_tempty[tst], (uint32_t)(((g - kSepTStages) / kSepTStages) & 1))) {
          ok = false;
          break;
        }
        dev::mbar_arrive_expect_tx(&bar_atom[tst], kSepStep * sizeof(float4));
        dev::bulk_g2s(&ring_atom[tst][0], a.rec + ks * kSepStep, kSepStep * sizeof(float4), &bar_atom[tst]);
        t_issued = g + 1;
        if (g >= kSepAStages &&
            !dev::mbar_wait_bounded(&bar_done[ast], (uint32_t)(((g - kSepAStages) / kSepAStages) & 1))) {
          ok = false;
          break;
        }
        dev::mbar_arrive_expect_tx(&bar_full[ast], a_bytes);
        dev::bulk_g2s(ringA + ast * kSepPair * kSepABytes, Ablk + ks * (kSepPair * kSepABytes / 16), a_bytes,
                      &bar_full[ast]);
        a_issued = g + 1;
      }
    }
  } else if (mma_warp) {
    if (lane == 0) {
      // descriptors of A stage 0 tile 0 and B stage 0 (hi and lo of the two
      // K16 halves); other stages and tiles add their byte offset / 16 to the
      // address field (every shared-memory address here is below 2^18)
      const uint32_t a0 = dev::smem_addr(ringA), b0 = dev::smem_addr(ringB);
      const uint64_t dah[2] = {smem_desc(a0, 2048, 128), smem_desc(a0 + 4096, 2048, 128)};
      const uint64_t dal[2] = {smem_desc(a0 + 8192, 2048, 128), smem_desc(a0 + 8192 + 4096, 2048, 128)};
      const uint64_t dbh[2] = {smem_desc(b0, 4096, 128), smem_desc(b0 + 8192, 4096, 128)};
      const uint64_t dbl[2] = {smem_desc(b0 + 16384, 4096, 128), smem_desc(b0 + 16384 + 8192, 4096, 128)};
      int64_t flushes = 0;  // groups read out before the current one
      int64_t g = 0;
      for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
        if ((g & 15) == 0 && s_abort) {  // waits are bounded; a prompt exit is a bonus
          ok = false;
          break;
        }
        if (ks == grp.grp_start && flushes > 0 &&
            !dev::mbar_wait_bounded(&bar_tfree, (uint32_t)((flushes - 1) & 1))) {
          ok = false;
          break;
        }
        const int ast = (int)(g % kSepAStages), bst = (int)(g % kSepBStages);
        if (!dev::mbar_wait_bounded(&bar_full[ast], (uint32_t)((g / kSepAStages) & 1)) ||
            !dev::mbar_wait_bounded(&bar_bfull[bst], (uint32_t)((g / kSepBStages) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t offB = (uint64_t)((bst * kSepBBytes) >> 4);
        for (int tp = 0; tp < ntp; ++tp) {
          const uint64_t offA = (uint64_t)(((ast * kSepPair + tp) * kSepABytes) >> 4);
          const uint32_t d = tmem + (uint32_t)(tp * kSepN);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const uint32_t acc0 = (ks > grp.grp_start || u > 0) ? 1u : 0u;
            mma_f16(d, dah[u] + offA, dbh[u] + offB, acc0);
            mma_f16(d, dah[u] + offA, dbl[u] + offB, 1u);
            mma_f16(d, dal[u] + offA, dbh[u] + offB, 1u);
          }
        }
        mma_commit(&bar_done[ast]);
        g_committed = g + 1;
        if (grp.ends_at(ks)) {
          grp.advance(ks);
          ++flushes;
        }
      }
    }
  } else {
    // ---- formation warps ---------------------------------------------------
    // this thread's B row (column col of D): forward the point (b, c) with
    // offsets (s_b, s_c) from H, adjoint the atom's (y', z')
    const int64_t col = col_base + tid;
    const bool row_ok = col < col_end;
    float sb, sc, sbl = 0.f, scl = 0.f;  // sbl, scl: low parts of a double-float s (forward)
    float att = 0.f;                     // buried object: 2 pi Im(sigma) of the column's beam
    bool att_over = false;               // an attenuation exponent passed kSepAttMax
    if (a.ntiles) {
      const float4 at = row_ok ? a.atom4[col] : make_float4(0.f, 0.f, 0.f, 0.f);
      sb = at.y;
      sc = at.z;
    } else {
      const int64_t rb = row_ok ? col / a.n2 : 0, rc = row_ok ? col % a.n2 : 0;
      sb = a.axis_s[a.n0 + rb];
      sc = a.axis_s[a.n0 + a.n1 + rc];
      if (a.axis_att) att = a.axis_att[rc];
      if (a.axis_lo) {
        sbl = a.axis_lo[a.n0 + rb];
        scl = a.axis_lo[a.n0 + a.n1 + rc];
      }
    }
    const uint32_t b_row_off = (uint32_t)((tid >> 3) * 128 + (tid & 7) * 16);
    // |s_b y' + s_c z' + c| of every B element of this call stays below
    // kSepPhaseLim cycles when the centred extent is small: the exact mod-1
    // reduction is then skipped (MUFU sin/cos of an argument of L cycles errs
    // by ~L 2^-24 cycles, 6e-6 rad at the limit, below this path's 1e-4)
    // (and above dev::kPhaseExactLim cycles, crystals hundreds of cells long,
    // each product is taken with its rounding error restored)
    bool reduce = true, exact = false;
    {
      const unsigned long long ylo = a.bbox[1], zlo = a.bbox[2], yhi = a.bbox[4], zhi = a.bbox[5];
      if (ylo != ~0ULL && zlo != ~0ULL && yhi != 0ULL && zhi != 0ULL) {
        const double ey = fmax(fabs(dev::unordered(ylo) - a.shift[1]), fabs(dev::unordered(yhi) - a.shift[1]));
        const double ez = fmax(fabs(dev::unordered(zlo) - a.shift[2]), fabs(dev::unordered(zhi) - a.shift[2]));
        const double bound = (double)a.smax_b * (ey + 1.0) + (double)a.smax_c * (ez + 1.0) + 0.5;
        reduce = bound > kSepPhaseLim;
        exact = bound > dev::kPhaseExactLim;
      }
    }
    float* part = a.partial + (int64_t)chunk * a.chunk_floats;
    bool first_flush = true;
    int64_t g = 0;
    for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
      const int bst = (int)(g % kSepBStages), tst = (int)(g % kSepTStages);
      // B stage bst is free once the MMAs of step g - kSepBStages completed;
      // every lane waits, the warp agrees on the outcome
      bool w = !s_abort;
      if (w && g >= kSepBStages)
        w = dev::mbar_wait_bounded(&bar_done[(g - kSepBStages) % kSepAStages],
                                   (uint32_t)(((g - kSepBStages) / kSepAStages) & 1));
      if (w) w = dev::mbar_wait_bounded(&bar_atom[tst], (uint32_t)((g / kSepTStages) & 1));
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      // B[col, k] = e^{2 pi i (s_b y' + s_c z' + c)}, zero past the last column
      unsigned char* sB = ringB + bst * kSepBBytes;
      const float4* at = ring_atom[tst];
      // mode 0: raw phase, 1: reduced mod 1, 2: exact products, reduced
      // kAtt: a buried object's rows carry exp(-att z')
      auto form = [&](auto mode_tag, auto att_tag) {
        constexpr int kMode = decltype(mode_tag)::value;
        constexpr bool kAtt = decltype(att_tag)::value;
#pragma unroll
        for (int kb = 0; kb < 4; ++kb) {
          uint32_t hi[4] = {0u, 0u, 0u, 0u}, lo[4] = {0u, 0u, 0u, 0u};
          if (row_ok) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 v = at[kb * 4 + q];
              const float ph =
                  kMode == 2 ? dev::frac_rn(dev::frac_product2_plus(sb, sbl, v.y,
                                                                    dev::frac_product2_plus(sc, scl, v.z, v.w)))
                  : kMode == 1 ? dev::frac_rn(fmaf(sb, v.y, fmaf(sc, v.z, v.w)))
                               : fmaf(sb, v.y, fmaf(sc, v.z, v.w));
              float sn, cs;
              dev::sincos_cycles_mufu(ph, &sn, &cs);
              if (kAtt) {
                float ex = -att * v.z;
                if (ex > kSepAttMax) {
                  ex = kSepAttMax;
                  att_over = true;
                }
                const float gz = __expf(ex);
                sn *= gz;
                cs *= gz;
              }
              split2(cs, sn, hi[q], lo[q]);
            }
          }
          *reinterpret_cast<uint4*>(sB + kb * 4096 + b_row_off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(sB + 16384 + kb * 4096 + b_row_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      };
      auto form_all = [&](auto att_tag) {
        if (exact)
          form(std::integral_constant<int, 2>{}, att_tag);
        else if (reduce)
          form(std::integral_constant<int, 1>{}, att_tag);
        else
          form(std::integral_constant<int, 0>{}, att_tag);
      };
      if (a.axis_att)
        form_all(std::true_type{});
      else
        form_all(std::false_type{});
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bar_bfull[bst]);
        mbar_arrive(&bar_tempty[tst]);
      }
      if (!grp.ends_at(ks)) continue;

      // ---- group end: TMEM -> blocked partials -------------------------------
      // the commit of step g covers every earlier MMA of the group
      w = dev::mbar_wait_bounded(&bar_done[g % kSepAStages], (uint32_t)((g / kSepAStages) & 1));
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      tc_fence_after();
      // TMEM lane = row (2 pa + ri) of this CTA's tile: one 32 x 32 block of
      // the partials per load; padding rows and columns are written too
      const int sub = warp & 3;
      const int col0 = (warp >> 2) * 128;
      for (int tp = 0; tp < ntp; ++tp) {
        const int64_t m0 = (2 * mp + tp) * kSepM + sub * 32;
#pragma unroll 1
        for (int cc = 0; cc < 128; cc += 32) {
          const int64_t bc0 = col_base + col0 + cc;
          if (bc0 >= col_end) break;
          float4* blk = reinterpret_cast<float4*>(part + sep_part_off(m0, bc0, a.n_cb)) + lane;
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(tp * kSepN + col0 + cc), v);
          // the first read-out stores, later ones add in L2 (reductions, no
          // load round trip); every element belongs to this CTA and its
          // updates come from this thread in program order, so the sum is
          // deterministic
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 x = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            if (first_flush)
              blk[q * 32] = x;
            else
              atomicAdd(blk + q * 32, x);
          }
        }
      }
      first_flush = false;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bar_tfree);
      grp.advance(ks);
    }
    if (att_over) dev::set_status(a.status, kStatusNonFinite);
    if (ok && first_flush) {
      // empty chunk: its partials are zero
      const int sub = warp & 3;
      const int col0 = (warp >> 2) * 128;
      for (int tp = 0; tp < ntp; ++tp) {
        const int64_t m0 = (2 * mp + tp) * kSepM + sub * 32;
        for (int cc = 0; cc < 128 && col_base + col0 + cc < col_end; cc += 32) {
          float4* blk = reinterpret_cast<float4*>(part + sep_part_off(m0, col_base + col0 + cc, a.n_cb)) + lane;
          for (int q = 0; q < 8; ++q) blk[q * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
  }
  if (!ok) {
    s_abort = 1;
    dev::set_status(a.status, kStatusTimeout);
  }
  __syncthreads();
  // on abort, wait (bounded) for MMAs and copies still in flight before
  // releasing TMEM and shared memory; phases already complete return at once
  if (mma_warp && lane == 0 && s_abort && g_committed > 0) {
    const int64_t gl = g_committed - 1;
    dev::mbar_wait_bounded(&bar_done[gl % kSepAStages], (uint32_t)((gl / kSepAStages) & 1), 1LL << 28);
  }
  if (copy_warp && lane == 0 && s_abort) {
    for (int64_t s = a_issued > kSepAStages ? a_issued - kSepAStages : 0; s < a_issued; ++s)
      dev::mbar_wait_bounded(&bar_full[s % kSepAStages], (uint32_t)((s / kSepAStages) & 1), 1LL << 28);
    for (int64_t s = t_issued > kSepTStages ? t_issued - kSepTStages : 0; s < t_issued; ++s)
      dev::mbar_wait_bounded(&bar_atom[s % kSepTStages], (uint32_t)((s / kSepTStages) & 1), 1LL << 28);
  }
  tc_fence_before();
  __syncthreads();
  if (mma_warp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSepTmemCols));
}

// Sum over the chunks in order of f_s(|S|) x T_chunk (Eq. 2: each chunk holds
// one species s), translation phase, outputs.
// Sum of the chunks' partials with f_s(|S|) per chunk's species, the
// centring phase and |A|^2.  One CTA per 32 x 32 block of the blocked
// partials (16 h values x 32 (k, l) columns, 512 points): each chunk's block
// is 4 KB contiguous and is read as one float4 per thread, thread t holding
// D row t % 32 (Re of h row (t % 32) / 2 for even t % 32, Im for odd) of the
// columns 4 (t / 32) .. +3.  One exchange between the two lanes of a row
// pair gives lane 2i columns 4q, 4q+1 and lane 2i+1 columns 4q+2, 4q+3 (two
// points each).  The sum over chunks runs in chunk order, eight chunks' loads
// in flight.
__global__ void __launch_bounds__(256) k_sep_reduce(const float* __restrict__ partial, int64_t chunk_floats,
                                                    int64_t n_cb, const Segment* __restrict__ chunks, int n_chunks,
                                                    const float* __restrict__ coef, const float2* __restrict__ ftab,
                                                    float inv4a2, const float* __restrict__ axis_s,
                                                    const float* __restrict__ axis_lo, int64_t n0, int64_t n1,
                                                    int64_t n2, float3 H, const double* __restrict__ shift,
                                                    const float* __restrict__ att, const float* __restrict__ szf,
                                                    int64_t bm_base, float2* out_amp, float* out_int) {
  // the centring shift of the call (integers), once per block
  __shared__ float sh_t[3];
  __shared__ int sh_shifted;
  if (threadIdx.x == 0) {
    sh_t[0] = (float)shift[0];
    sh_t[1] = (float)shift[1];
    sh_t[2] = (float)shift[2];
    sh_shifted = shift[0] != 0.0 || shift[1] != 0.0 || shift[2] != 0.0;
  }
  __syncthreads();
  const int t = threadIdx.x, lane = t & 31, odd = lane & 1;
  const int64_t bm = bm_base + blockIdx.y, bc = blockIdx.x;
  const int64_t ncols = n1 * n2, n_s = n0 * ncols;
  const int64_t i0 = bm * 16 + (lane >> 1);
  const int64_t col0 = bc * 32 + (t >> 5) * 4 + odd * 2;  // the thread's two columns
  // per point: double-float offsets s, |S|^2 / (4 a^2) in FP32 (S = H + s)
  float s_hi[2][3], s_lo[2][3], s2[2];
  bool ok[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int64_t col = col0 + u;
    ok[u] = i0 < n0 && col < ncols;
    const int64_t ia[3] = {ok[u] ? i0 : 0, n0 + (ok[u] ? col / n2 : 0), n0 + n1 + (ok[u] ? col % n2 : 0)};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      s_hi[u][d] = axis_s[ia[d]];
      s_lo[u][d] = axis_lo[ia[d]];
    }
    // (a buried object's form factor is taken at the vacuum beam's S_z)
    const int64_t il = ia[2] - n0 - n1;
    const float S0 = H.x + (s_hi[u][0] + s_lo[u][0]), S1 = H.y + (s_hi[u][1] + s_lo[u][1]),
                S2 = szf ? szf[il] : H.z + (s_hi[u][2] + s_lo[u][2]);
    s2[u] = (S0 * S0 + S1 * S1 + S2 * S2) * inv4a2;
  }
  const int64_t m0 = i0 * ncols + col0;
  const float* blk = partial + (bm * n_cb + bc) * 1024 + 4 * t;
  float2 v[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}, F[2] = {v[0], v[1]};
  int cur = -1;
  constexpr int kU = 8;
  for (int c0 = 0; c0 < n_chunks; c0 += kU) {
    float4 x[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u)
      x[u] = c0 + u < n_chunks ? __ldcs(reinterpret_cast<const float4*>(blk + (int64_t)(c0 + u) * chunk_floats))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      if (c0 + u >= n_chunks) break;  // uniform over the block
      // even lane: Re of columns 4q..4q+3, needs Im of 4q, 4q+1; odd lane:
      // Im, needs Re of 4q+2, 4q+3
      const float sx = odd ? x[u].x : x[u].z, sy = odd ? x[u].y : x[u].w;
      const float rx = __shfl_xor_sync(0xffffffffu, sx, 1), ry = __shfl_xor_sync(0xffffffffu, sy, 1);
      const float re[2] = {odd ? rx : x[u].x, odd ? ry : x[u].y};
      const float im[2] = {odd ? x[u].z : rx, odd ? x[u].w : ry};
      const int sp = chunks[c0 + u].species;
      if (sp != cur) {
#pragma unroll
        for (int w = 0; w < 2; ++w)
          F[w] = ftab ? (ok[w] ? ftab[(int64_t)sp * n_s + m0 + w] : make_float2(0.f, 0.f))
                      : dev::form_factor(coef + kNCoef * sp, s2[w]);
        cur = sp;
      }
#pragma unroll
      for (int w = 0; w < 2; ++w) {
        v[w].x += F[w].x * re[w] - F[w].y * im[w];
        v[w].y += F[w].x * im[w] + F[w].y * re[w];
      }
    }
  }
#pragma unroll
  for (int w = 0; w < 2; ++w) {
    if (!ok[w]) continue;
    float2 a = v[w];
    if (sh_shifted) a = dev::cmul(dev::shift_phase2(s_hi[w], s_lo[w], sh_t), a);
    if (att) {
      // a buried object's attenuation over the centring shift t_z (the rows
      // carried exp(-2 pi Im(sigma) z') of the centred z')
      const float g = __expf(-att[(col0 + w) % n2] * sh_t[2]);
      a.x *= g;
      a.y *= g;
    }
    if (out_amp) out_amp[m0 + w] = a;
    if (out_int) out_int[m0 + w] = a.x * a.x + a.y * a.y;
  }
}

// -------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------

cudaError_t sep_prepare_kernel() {
  static_assert(kSepSmem + 4096 <= 227 * 1024, "dynamic + static shared memory of k_sep");
  const cudaError_t e = cudaFuncSetAttribute(k_sep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSepSmem);
  return e != cudaSuccess ? e : sep_pair_prepare_kernel();
}

// grid: x = M-tile pairs x N tiles, y = chunks.  The CTA-pair kernel
// (sep_pair.cu) covers the same tiles with two M-tile pairs per cluster.  An
// odd last pair runs on the one-CTA kernel (a pair cluster with one
// accumulator tile would form all of its B columns for half the MMA work),
// on the side stream where one is given, so that its CTAs take the SMs the
// pair kernel's last clusters leave idle.
cudaError_t sep_launch_core(const SepArgs& a, dim3 grid, cudaStream_t st, cudaStream_t side, cudaEvent_t fork,
                            cudaEvent_t join) {
  const int64_t n_mp = (a.n_mt + 1) / 2;
  const int64_t n_nt = (int64_t)grid.x / n_mp;
  const int64_t n_even = n_mp & ~int64_t(1);
  if (!sep_pair_enabled() || n_even == 0) {
    k_sep<<<grid, kSepThreads, kSepSmem, st>>>(a);
    return cudaGetLastError();
  }
  SepArgs pa = a;
  pa.mp_first = 0;
  pa.mp_count = n_even;
  SepArgs sa = a;
  sa.mp_first = n_even;
  sa.mp_count = 1;
  const bool split = n_even < n_mp;
  const bool beside = split && side && fork && join;
  cudaError_t e = cudaSuccess;
  if (beside && ((e = cudaEventRecord(fork, st)) != cudaSuccess || (e = cudaStreamWaitEvent(side, fork, 0)) != cudaSuccess))
    return e;
  e = sep_pair_launch_core(pa, n_nt, (int)grid.y, st);
  if (split) {
    if (e == cudaSuccess) {
      k_sep<<<dim3((unsigned)n_nt, grid.y), kSepThreads, kSepSmem, beside ? side : st>>>(sa);
      e = cudaGetLastError();
    }
    if (beside) {  // join even after a failed launch: a capture needs the side stream back
      const cudaError_t ej = cudaEventRecord(join, side);
      const cudaError_t ew = ej == cudaSuccess ? cudaStreamWaitEvent(st, join, 0) : ej;
      if (e == cudaSuccess) e = ew;
    }
  }
  return e;
}

scatter_status sep_prepare_side(scatter_plan_s* p, int64_t n_mt) {
  if (sep_core_launches(n_mt) < 2 || p->side_stream) return SCATTER_OK;
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&p->side_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_status(e, "side stream");
  if ((e = cudaEventCreateWithFlags(&p->side_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&p->side_join, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_status(e, "side stream events");
  return SCATTER_OK;
}

int sep_core_launches(int64_t n_mt) {
  const int64_t n_mp = (n_mt + 1) / 2;
  return (sep_pair_enabled() && n_mp >= 2 && n_mp % 2 == 1) ? 2 : 1;
}

namespace {

int sep_best_split(const scatter_plan_s* p, int64_t tiles) {
  const double cap = (double)p->n_sm;  // one CTA per SM (TMEM + shared memory)
  const double steps = (double)std::max<int64_t>(p->n_slots / kSepStep, 1);
  double best = 1e300;
  int best_k = 1;
  // up to two chunks per SM: a grid of one N tile and one M quad (a few
  // columns, a long atom list) needs ~n_sm / 2 chunks to give every SM a CTA
  for (int k = 1; k <= 2 * p->n_sm; ++k) {
    if (k > 1 && steps / k < 64) break;
    // one step ~1 us of MMA; an extra chunk costs one partial of the
    // map (8 B per point written once, read once by the reduction)
    const double part_steps = 16.0 * (double)p->sep_ns / 6.0e12 / 1.0e-6;
    const double cost = std::ceil((double)tiles * k / cap) * (steps / k + 40.0) + (k > 1 ? k * part_steps : 0.0);
    if (cost < best * 0.995) {
      best = cost;
      best_k = k;
    }
  }
  return best_k;
}

}  // namespace

// The separable grid: the plan's own axes, or for a grazing-incidence plan
// the virtual grid (h, k, l) whose l axis stacks the four beams' Sz values
// [Sz1 | Sz2 | -Sz2 | -Sz1] over alpha_f, so each beam is a plain grid sum.
// A buried object has one beam, l = Re(sigma) per alpha_f; its formed rows
// carry the attenuation exp(-2 pi Im(sigma) z') and its form factor is taken
// at the vacuum beam S_1 (the per-column tables sep_att and sep_szf).
scatter_status prepare_separable(scatter_plan_s* p, int split_override) {
  const bool gid = p->s_kind == SCATTER_S_GID_GRID;
  if ((p->s_kind != SCATTER_S_GRID && !gid) || p->batch != 1)
    return fail(SCATTER_ERR_UNSUPPORTED, "the separable path needs a single axis-aligned grid");
  if (p->n_slots % kSepStep) return fail(SCATTER_ERR_UNSUPPORTED, "slot padding is not a multiple of 16");
  std::vector<double> ax64[3];
  for (int d = 0; d < 2; ++d) ax64[d] = p->axis_host[d];
  const bool buried = gid && p->gid_mode == 1;
  std::vector<float> att, szf;
  p->sep_beams = buried ? 1 : 4;
  if (buried) {
    const int64_t n_af = p->n_axis[2];
    ax64[2].assign(p->gid_sz_host.begin(), p->gid_sz_host.begin() + n_af);
    for (int64_t i = 0; i < n_af; ++i) {
      att.push_back((float)(6.283185307179586 * p->gid_sz_im_host[i]));
      szf.push_back((float)p->gid_szf_host[i]);
    }
  } else if (gid) {
    const int64_t n_af = p->n_axis[2];
    ax64[2].resize(4 * n_af);
    for (int64_t i = 0; i < n_af; ++i) {
      const double z1 = p->gid_sz_host[i], z2 = p->gid_sz_host[n_af + i];
      ax64[2][i] = z1;
      ax64[2][n_af + i] = z2;
      ax64[2][2 * n_af + i] = -z2;
      ax64[2][3 * n_af + i] = -z1;
    }
  } else {
    ax64[2] = p->axis_host[2];
  }
  std::vector<float> alls, alls_lo;
  for (int d = 0; d < 3; ++d) {
    p->sep_n[d] = (int64_t)ax64[d].size();
    for (double v : ax64[d]) {
      const double sv = v - p->inst[0].H[d];
      alls.push_back((float)sv);
      alls_lo.push_back((float)(sv - (double)(float)sv));
    }
  }
  p->sep_ns = p->sep_n[0] * p->sep_n[1] * p->sep_n[2];
  p->sep_smax[0] = p->sep_smax[1] = 0.f;
  for (int64_t i = 0; i < p->sep_n[1]; ++i)
    p->sep_smax[0] = std::max(p->sep_smax[0], std::fabs(alls[p->sep_n[0] + i]));
  for (int64_t i = 0; i < p->sep_n[2]; ++i)
    p->sep_smax[1] = std::max(p->sep_smax[1], std::fabs(alls[p->sep_n[0] + p->sep_n[1] + i]));
  const int64_t n_steps = p->n_slots / kSepStep;
  const int64_t n_mt = (2 * p->sep_n[0] + kSepM - 1) / kSepM;
  const int64_t n_nt = (p->sep_n[1] * p->sep_n[2] + kSepN - 1) / kSepN;
  const int64_t n_mp = (n_mt + 1) / 2;
  const int split = split_override > 0 ? split_override : sep_best_split(p, n_mp * n_nt);
  Tiling t;
  t.threads = 256;
  t.R = 8;
  t.split_k = split;
  // chunk tables (segments) as for the generic path; the partial buffer is blocked
  scatter_status st = apply_tiling(p, t);
  if (st != SCATTER_OK) return st;
  if (p->d.partial) {  // the generic path's partials are not used here
    cudaFree(p->d.partial);
    p->d.partial = nullptr;
  }
  p->sep_mt = n_mt;
  p->sep_nt = n_nt;
  p->sep_steps = n_steps;
  cudaError_t e;
  // With one N tile every A tile is read by one cluster only: the CTA pair
  // then forms its A tiles itself from the atom records (the same arithmetic
  // as k_sep_tab_a), and the table, written and read once, is not kept.
  // With several N tiles that formation would repeat per tile, so the table
  // stays; an odd pair count runs its last pair on the one-CTA kernel, which
  // reads the table.
  p->sep_form_a = sep_pair_enabled() && n_mp % 2 == 0 && n_nt == 1;
  const size_t a_bytes =
      p->sep_form_a ? 0 : (size_t)(2 * n_mp) * (size_t)std::max<int64_t>(n_steps, 1) * kSepABytes;
  // atom chunks: every species segment split into step-aligned pieces, about
  // `split` pieces in all, so that each chunk carries a single form factor
  std::vector<Segment> chunks;
  int64_t total_steps = 0;
  for (const Segment& sg : p->all_segs)
    if (sg.instance == 0 && sg.end > sg.begin) total_steps += (sg.end - sg.begin) / kSepStep;
  for (const Segment& sg : p->all_segs) {
    if (sg.instance != 0 || sg.end <= sg.begin) continue;
    const int64_t steps = (sg.end - sg.begin) / kSepStep;
    const int64_t k = std::max<int64_t>(1, std::llround((double)split * (double)steps / (double)total_steps));
    const int64_t per = (steps + k - 1) / k;
    for (int64_t b = 0; b < steps; b += per)
      chunks.push_back(Segment{sg.begin + b * kSepStep, sg.begin + std::min(steps, b + per) * kSepStep, sg.species, 0});
  }
  if (chunks.empty()) chunks.push_back(Segment{0, 0, 0, 0});  // no atoms: one empty chunk, zero partials
  p->sep_n_chunks = (int32_t)chunks.size();
  const size_t part_bytes =
      (size_t)p->sep_n_chunks * (size_t)sep_part_floats(n_mt, p->sep_n[1] * p->sep_n[2]) * sizeof(float);
  const size_t chunk_bytes = chunks.size() * sizeof(Segment);
  if (a_bytes) {
    if ((e = cudaMalloc(&p->d.sep_A, a_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc separable A");
    // tiles past the last row are never written by the table kernel: zero
    // them once (the CTA-pair kernel streams the second tile of a pair always)
    if ((e = cudaMemset(p->d.sep_A, 0, a_bytes)) != cudaSuccess) return cuda_status(e, "memset separable A");
  }
  if ((e = cudaMalloc(&p->d.sep_partial, part_bytes)) != cudaSuccess)
    return cuda_status(e, "cudaMalloc separable partials");
  if ((e = cudaMalloc(&p->d.sep_chunks, chunk_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc chunks");
  cudaMemcpy(p->d.sep_chunks, chunks.data(), chunk_bytes, cudaMemcpyHostToDevice);
  if ((e = cudaMalloc(&p->d.sep_axis_s, alls.size() * sizeof(float))) != cudaSuccess) return cuda_status(e, "axes");
  if ((e = cudaMalloc(&p->d.sep_axis_lo, alls_lo.size() * sizeof(float))) != cudaSuccess) return cuda_status(e, "axes");
  cudaMemcpy(p->d.sep_axis_s, alls.data(), alls.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(p->d.sep_axis_lo, alls_lo.data(), alls_lo.size() * sizeof(float), cudaMemcpyHostToDevice);
  size_t virt_bytes = 0;
  if (gid) {
    virt_bytes = (size_t)p->sep_ns * sizeof(float2);
    if ((e = cudaMalloc(&p->d.sep_virt, virt_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc virtual map");
  }
  if (buried) {
    const size_t tb = att.size() * sizeof(float);
    if ((e = cudaMalloc(&p->d.sep_att, tb)) != cudaSuccess) return cuda_status(e, "attenuation table");
    if ((e = cudaMalloc(&p->d.sep_szf, tb)) != cudaSuccess) return cuda_status(e, "form-factor Sz table");
    cudaMemcpy(p->d.sep_att, att.data(), tb, cudaMemcpyHostToDevice);
    cudaMemcpy(p->d.sep_szf, szf.data(), tb, cudaMemcpyHostToDevice);
    virt_bytes += 2 * tb;
  }
  p->base_bytes += (int64_t)(a_bytes + part_bytes + chunk_bytes + virt_bytes);
  if ((e = sep_prepare_kernel()) != cudaSuccess) return cuda_status(e, "separable shared memory attribute");
  return sep_prepare_side(p, n_mt);
}

scatter_status launch_separable(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st) {
  SepTabArgs t{};
  t.atom4 = p->d.atom4;
  t.atom_lo = p->d.atom_lo;
  t.atom_w = p->d.atom_w;
  t.axis_s = p->d.sep_axis_s;
  t.axis_lo = p->d.sep_axis_lo;
  t.n0 = p->sep_n[0];
  t.n1 = p->sep_n[1];
  t.n2 = p->sep_n[2];
  t.n_slots = p->n_slots;
  t.n_steps = p->sep_steps;
  t.n_mt = p->sep_mt;
  t.A = static_cast<uint4*>(p->d.sep_A);
  const int n_chunks = p->sep_n_chunks;
  if (p->n_slots > 0 && !p->sep_form_a) {
    const int64_t na = p->sep_mt * p->sep_steps * 4 * kSepM;  // real tiles; a padding tile is never read
    k_sep_tab_a<<<(unsigned)((na + 255) / 256), 256, 0, st>>>(t);
    p->last_launches += 1;
  }
  SepArgs a{};
  a.A = static_cast<const uint4*>(p->d.sep_A);
  a.a_sp_stride = 0;
  a.rec = p->d.atom4;
  a.chunks = p->d.sep_chunks;
  a.ntiles = nullptr;
  a.bbox = p->d.inst_bbox;
  a.shift = p->d.inst_shift;
  a.smax_b = p->sep_smax[0];
  a.smax_c = p->sep_smax[1];
  a.axis_s = p->d.sep_axis_s;
  a.axis_lo = p->d.sep_axis_lo;
  a.n0 = p->sep_n[0];
  a.n1 = p->sep_n[1];
  a.n2 = p->sep_n[2];
  a.n_cb = (p->sep_n[1] * p->sep_n[2] + 31) / 32;
  a.chunk_floats = sep_part_floats(p->sep_mt, p->sep_n[1] * p->sep_n[2]);
  a.n_steps = p->sep_steps;
  a.n_mt = p->sep_mt;
  a.partial = p->d.sep_partial;
  a.status = p->d.status;
  a.axis_att = p->d.sep_att;
  a.form_a = p->sep_form_a ? 1 : 0;
  a.rec_lo = p->d.atom_lo;
  a.rec_w = p->d.atom_w;
  dim3 grid((unsigned)(((p->sep_mt + 1) / 2) * p->sep_nt), (unsigned)n_chunks);
  timing_begin(p, st);
  const cudaError_t le = sep_launch_core(a, grid, st, p->side_stream, p->side_fork, p->side_join);
  timing_end(p, st);
  if (le != cudaSuccess) return cuda_status(le, "separable kernel launch");
  p->last_launches += sep_core_launches(p->sep_mt);
  const bool gid = p->s_kind == SCATTER_S_GID_GRID;
  const int64_t n_cb = (p->sep_n[1] * p->sep_n[2] + 31) / 32;
  const int64_t n_bm = (2 * p->sep_n[0] + 31) / 32;  // 32-row blocks holding map rows
  // a host call copies each row range to the host while the next is reduced
  const bool pieces = p->host_out && !gid;
  const int n_pieces = pieces ? (int)std::min<int64_t>(kHostPieces, n_bm) : 1;
  const int64_t ncols = p->sep_n[1] * p->sep_n[2];
  for (int k = 0; k < n_pieces; ++k) {
    const int64_t b0 = n_bm * k / n_pieces, b1 = n_bm * (k + 1) / n_pieces;
    const dim3 rgrid((unsigned)n_cb, (unsigned)(b1 - b0));
    k_sep_reduce<<<rgrid, 256, 0, st>>>(
        p->d.sep_partial, sep_part_floats(p->sep_mt, ncols), n_cb, p->d.sep_chunks, n_chunks, p->d.coef, p->d.ftab,
        (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a)), p->d.sep_axis_s, p->d.sep_axis_lo, p->sep_n[0],
        p->sep_n[1], p->sep_n[2],
        make_float3((float)p->inst[0].H[0], (float)p->inst[0].H[1], (float)p->inst[0].H[2]), p->d.inst_shift,
        p->d.sep_att, p->d.sep_szf, b0, gid ? p->d.sep_virt : amp_out, gid ? nullptr : int_out);
    p->last_launches += 1;
    if (pieces) {
      // h rows 16 b0 .. 16 b1 of the map: a contiguous range of points
      const int64_t m0 = std::min<int64_t>(16 * b0, p->sep_n[0]) * ncols;
      const int64_t m1 = std::min<int64_t>(16 * b1, p->sep_n[0]) * ncols;
      cudaError_t e = cudaEventRecord(p->copy_ev[k], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_stream, p->copy_ev[k], 0);
      if (e == cudaSuccess && m1 > m0)
        e = cudaMemcpyAsync(static_cast<float2*>(p->host_out) + m0, amp_out + m0, (size_t)(m1 - m0) * sizeof(float2),
                            cudaMemcpyDeviceToHost, p->copy_stream);
      if (e != cudaSuccess) return cuda_status(e, "map range to the host");
    }
  }
  if (pieces) {
    // the caller's stream resumes once the last range is on the host
    cudaError_t e = cudaEventRecord(p->copy_ev[kHostPieces], p->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, p->copy_ev[kHostPieces], 0);
    if (e != cudaSuccess) return cuda_status(e, "host copy completion");
  }
  if (gid) {
    scatter_status s2 = launch_gid_combine(p, amp_out, int_out, st);
    if (s2 != SCATTER_OK) return s2;
  }
  return cuda_status(cudaGetLastError(), "separable launch");
}

}  // namespace scatter
