// k_sep on a CTA pair: the separable contraction with tcgen05.mma.cta_group::2.
//
// The one-CTA kernel (separable.cu) spends a step of 16 atoms on 12 MMAs of
// M = 128, N = 256, each reading 4 KB of A and 8 KB of B from shared memory,
// plus 64 KB of A and B writes: ~208 KB of shared-memory traffic against
// 1536 tensor cycles, which the SM's ~128 B/clk cannot carry, so a step
// takes ~2070 cycles.  Here two CTAs of a cluster (two SMs) share one
// accumulator tile of M = 256 rows: each CTA holds its own 128 rows of A
// and half of the 256 B columns, and the pair's tensor cores each compute
// their 128 rows x 256 columns, reading the other SM's B half through the
// pair's connection.  Per SM and step: 8 KB of operand reads per MMA (96 KB
// per step) and 48 KB of writes, and half the B formation (128 columns x 16
// atoms instead of 256 x 16), for the same tensor work per SM.
//
// Roles (320 threads per CTA, both CTAs):
//   warps 0..7  form the CTA's 128 B columns (two threads per column, eight
//               atoms each) and read its accumulators out at group ends
//   warp 8      rank 0: issues the pair's MMAs (cta_group::2) and one commit
//               per step, multicast to both CTAs' done barriers;
//               rank 1: the relay (below)
//   warp 9      copies the CTA's A blocks and the step's atom records (TMA)
// Every role signals on barriers of its own CTA (release at CTA scope).  In
// rank 1 one relay thread waits for its CTA's A stage and B stage of each
// step (and its TMEM read-out at group ends) and forwards each event to
// rank 0 with one remote arrive (release at cluster scope; rank 0 waits
// with acquire at cluster scope): per step one cluster-scope release from a
// thread with no memory traffic of its own, instead of one per formation
// warp (which stalled those warps on the fence behind their stores and
// L2 reductions).  The MMA completion reaches both CTAs through the
// multicast commit.  Every wait is bounded; a CTA that gives up tells its
// peer through a remote store, both drain their copies and MMAs in flight,
// meet at a cluster barrier and release TMEM together.
//
// Rows: the pair covers the M-tile pairs p = 2 q + tp (tp = 0, 1) of its
// M quad q; in pair p rank r owns tile 2 p + r, i.e. the half r of the
// A table's 32 KB (pair, step) block.  Columns: N tile nt of 256 columns,
// rank r forms columns nt * 256 + r * 128 + [0, 128).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <type_traits>
#include "launch.h"
#include "sep_common.cuh"

namespace scatter {

namespace {

constexpr int kPairHalfN = kSepN / 2;                  // B columns formed per CTA
constexpr uint32_t kPairBBytes = 16384;                // B half stage: hi + lo, 128 x 32 f16 each
constexpr uint32_t kPairTileBytes = kSepABytes;        // one CTA's A tile per step (hi + lo)
constexpr int kPairAStages = 4;
constexpr int kPairBStages = kPairAStages;  // a step's A and B stages share one "ready" barrier
constexpr int kPairTStages = 8;
constexpr int kPairAWarps = 8;  // FORM_A: warps that form the A tiles (beside the B warps)
constexpr int kPairThreadsA = kSepThreads + 32 * kPairAWarps;
constexpr size_t kPairSmem = kPairAStages * 2 * kPairTileBytes + kPairBStages * kPairBBytes + 1024;
// kind::f16, D f32, K-major A and B, N = 256 (>> 3 at bit 17), M = 256 (>> 4 at bit 24)
constexpr uint32_t kPairIdesc = (1u << 4) | ((uint32_t)(kSepN >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of `p` (a shared variable of this CTA) in CTA `rank`
__device__ __forceinline__ uint32_t peer_addr(const void* p, uint32_t rank) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(dev::smem_addr(p)), "r"(rank));
  return ra;
}

// arrive on the barrier at `bar`'s offset in CTA `rank` (release, cluster scope)
__device__ __forceinline__ void arrive_at(uint64_t* bar, uint32_t rank) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(peer_addr(bar, rank)) : "memory");
}

__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(dev::smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on a barrier that other CTAs of the cluster arrive on
__device__ __forceinline__ bool wait_cluster_bounded(uint64_t* bar, uint32_t parity,
                                                     long long budget = (1LL << 31)) {
  if (try_wait_cluster(bar, parity)) return true;
  const long long t0 = clock64();
  while (!try_wait_cluster(bar, parity)) {
    if (clock64() - t0 > budget) return false;
  }
  return true;
}

__device__ __forceinline__ void mma_pair(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kPairIdesc), "r"(acc));
}

// completion of every MMA issued so far, signalled on `bar` in both CTAs
__device__ __forceinline__ void commit_pair(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          dev::smem_addr(bar)),
      "h"((uint16_t)0x3)
      : "memory");
}

}  // namespace

// Barriers (every CTA holds the full set; the ones marked "rank 0" only carry
// arrivals in rank 0):
//   bar_ready[s]  stage s of a step is ready: this CTA's A blocks arrived
//                 (TMA: the copy warp's arrival + bytes), its B half formed
//                 (8 warps) and, in rank 0, rank 1's stage ready (relay):
//                 the MMA thread's only wait per step
//   bar_done[s]   the pair's MMAs of the step completed         (multicast commit)
//   bar_atom[t]   atom records of a step arrived                (TMA)
//   bar_tempty[t] atom records read by this CTA's formation     (8 warps)
//   bar_tread     this CTA's accumulators read out              (8 warps)
//   bar_pfree     rank 0: rank 1's accumulators read out        (relay)
// FORM_A: eight more warps (10..17, kPairThreadsA threads per CTA) form this
// CTA's A tiles from the step's atom records (with their x' errors and
// occupancies) instead of the copy warp streaming them from the table (a
// grid of one N tile, where the table would be written and read once); they
// wait and signal like the B warps, and take no part in the read-outs.
template <bool FORM_A>
__global__ void __cluster_dims__(2, 1, 1) __maxnreg__(FORM_A ? 112 : 168) k_sep_pair(const SepArgs a) {
  extern __shared__ __align__(1024) unsigned char pair_smem_raw[];
  __shared__ __align__(8) uint64_t bar_ready[kPairAStages];
  __shared__ __align__(8) uint64_t bar_done[kPairAStages];
  __shared__ __align__(8) uint64_t bar_atom[kPairTStages];
  __shared__ __align__(8) uint64_t bar_tempty[kPairTStages];
  __shared__ __align__(8) uint64_t bar_tread;
  __shared__ __align__(8) uint64_t bar_pfree;
  __shared__ __align__(16) float4 ring_atom[kPairTStages][kSepStep];
  // FORM_A: the records' x' errors and occupancies (one unused stage otherwise)
  __shared__ __align__(16) float4 ring_lo[FORM_A ? kPairTStages : 1][kSepStep];
  __shared__ __align__(16) float ring_w[FORM_A ? kPairTStages : 1][kSepStep];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(pair_smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ringA = smem;                                    // [stage][tp][hi|lo 16 KB]
  unsigned char* ringB = smem + kPairAStages * 2 * kPairTileBytes;  // [stage][hi 8 KB | lo 8 KB]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool mma_warp = warp == kSepFormWarps, copy_warp = warp == kSepFormWarps + 1;
  const bool a_warp = FORM_A && warp >= kSepFormWarps + 2;
  const uint32_t rank = cluster_rank();
  const int64_t n_mp = a.mp_count > 0 ? a.mp_count : (a.n_mt + 1) / 2;  // M-tile pairs of this launch
  const int64_t n_mq = (n_mp + 1) / 2;       // M quads (one per cluster)
  const int64_t cl = blockIdx.x >> 1;
  const int64_t mq = cl % n_mq, nt = cl / n_mq;
  const int ntp = 2 * mq + 1 < n_mp ? 2 : 1;  // tile pairs of this quad with rows
  const int64_t mp0 = a.mp_first + 2 * mq;   // the quad's first M-tile pair
  const int chunk = blockIdx.y;
  const int64_t nbc = a.n1 * a.n2;
  int64_t col_base = nt * kSepN, col_end = nbc;
  int a_species = 0;
  if (a.ntiles) {
    const Segment t = a.ntiles[nt];
    col_base = t.begin;
    col_end = t.end;
    a_species = t.species;
  }

  if (mma_warp) {
    // one warp of each CTA of the pair allocates collectively: the same 512
    // columns in both SMs' tensor memory
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dev::smem_addr(&tmem_slot)),
                 "r"(kSepTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  if (tid == 0) {
    for (int s = 0; s < kPairAStages; ++s) {
      dev::mbar_init(&bar_ready[s], (FORM_A ? kPairAWarps : 1) + kSepFormWarps + (rank == 0 ? 1 : 0));
      dev::mbar_init(&bar_done[s], 1);
    }
    for (int s = 0; s < kPairTStages; ++s) {
      dev::mbar_init(&bar_atom[s], 1);
      dev::mbar_init(&bar_tempty[s], kSepFormWarps + (FORM_A ? kPairAWarps : 0));
    }
    dev::mbar_init(&bar_tread, kSepFormWarps);
    dev::mbar_init(&bar_pfree, 1);
    s_abort = 0;
    dev::mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers initialised before any remote arrival
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const int64_t ks_begin = a.chunks[chunk].begin / kSepStep, ks_end = a.chunks[chunk].end / kSepStep;
  SepGroups grp{ks_end, ks_begin};
  bool ok = true;
  int64_t a_issued = 0, t_issued = 0, g_committed = 0;

  if (copy_warp) {
    if (lane == 0) {
      // this CTA's A tile of each pair with rows (half `rank` of the pair's
      // (pair, step) block) and the step's K records, in step order
      // (FORM_A: no A table, a.A is null and never read)
      const uint4* Abase = FORM_A ? nullptr : a.A + a_species * a.a_sp_stride + rank * (kPairTileBytes / 16);
      const int64_t pair_stride = a.n_steps * (kSepPair * kSepABytes / 16);
      int64_t g = 0;
      for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
        if (s_abort) {
          ok = false;
          break;
        }
        const int tst = (int)(g % kPairTStages), ast = (int)(g % kPairAStages);
        if (g >= kPairTStages &&
            !dev::mbar_wait_bounded(&bar_tempty[tst], (uint32_t)(((g - kPairTStages) / kPairTStages) & 1))) {
          ok = false;
          break;
        }
        if constexpr (FORM_A) {
          // the records, their x' errors and occupancies: the formation warps
          // build the step's A tiles from them
          dev::mbar_arrive_expect_tx(&bar_atom[tst], kSepStep * (2 * sizeof(float4) + sizeof(float)));
          dev::bulk_g2s(&ring_atom[tst][0], a.rec + ks * kSepStep, kSepStep * sizeof(float4), &bar_atom[tst]);
          dev::bulk_g2s(&ring_lo[tst][0], a.rec_lo + ks * kSepStep, kSepStep * sizeof(float4), &bar_atom[tst]);
          dev::bulk_g2s(&ring_w[tst][0], a.rec_w + ks * kSepStep, kSepStep * sizeof(float), &bar_atom[tst]);
          t_issued = g + 1;
          continue;
        }
        dev::mbar_arrive_expect_tx(&bar_atom[tst], kSepStep * sizeof(float4));
        dev::bulk_g2s(&ring_atom[tst][0], a.rec + ks * kSepStep, kSepStep * sizeof(float4), &bar_atom[tst]);
        t_issued = g + 1;
        if (g >= kPairAStages &&
            !dev::mbar_wait_bounded(&bar_done[ast], (uint32_t)(((g - kPairAStages) / kPairAStages) & 1))) {
          ok = false;
          break;
        }
        dev::mbar_arrive_expect_tx(&bar_ready[ast], (uint32_t)ntp * kPairTileBytes);
        for (int tp = 0; tp < ntp; ++tp)
          dev::bulk_g2s(ringA + (ast * 2 + tp) * kPairTileBytes,
                        Abase + (mp0 + tp) * pair_stride + ks * (kSepPair * kSepABytes / 16), kPairTileBytes,
                        &bar_ready[ast]);
        a_issued = g + 1;
      }
    }
  } else if (mma_warp) {
    if (lane == 0 && rank == 0) {
      // descriptors of A stage 0 tile 0 and B stage 0 (hi and lo of the two
      // K16 halves); other stages and tiles add their byte offset / 16
      const uint32_t a0 = dev::smem_addr(ringA), b0 = dev::smem_addr(ringB);
      const uint64_t dah[2] = {smem_desc(a0, 2048, 128), smem_desc(a0 + 4096, 2048, 128)};
      const uint64_t dal[2] = {smem_desc(a0 + 8192, 2048, 128), smem_desc(a0 + 8192 + 4096, 2048, 128)};
      const uint64_t dbh[2] = {smem_desc(b0, 2048, 128), smem_desc(b0 + 4096, 2048, 128)};
      const uint64_t dbl[2] = {smem_desc(b0 + 8192, 2048, 128), smem_desc(b0 + 8192 + 4096, 2048, 128)};
      int64_t flushes = 0;
      int64_t g = 0;
      for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
        if ((g & 15) == 0 && s_abort) {
          ok = false;
          break;
        }
        if (ks == grp.grp_start && flushes > 0 &&
            (!dev::mbar_wait_bounded(&bar_tread, (uint32_t)((flushes - 1) & 1)) ||
             !wait_cluster_bounded(&bar_pfree, (uint32_t)((flushes - 1) & 1)))) {
          ok = false;
          break;
        }
        const int ast = (int)(g % kPairAStages), bst = ast;
        if (!wait_cluster_bounded(&bar_ready[ast], (uint32_t)((g / kPairAStages) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t offB = (uint64_t)((bst * kPairBBytes) >> 4);
        for (int tp = 0; tp < ntp; ++tp) {
          const uint64_t offA = (uint64_t)(((ast * 2 + tp) * kPairTileBytes) >> 4);
          const uint32_t d = tmem + (uint32_t)(tp * kSepN);
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const uint32_t acc0 = (ks > grp.grp_start || u > 0) ? 1u : 0u;
            mma_pair(d, dah[u] + offA, dbh[u] + offB, acc0);
            mma_pair(d, dah[u] + offA, dbl[u] + offB, 1u);
            mma_pair(d, dal[u] + offA, dbh[u] + offB, 1u);
          }
        }
        commit_pair(&bar_done[ast]);
        g_committed = g + 1;
        if (grp.ends_at(ks)) {
          grp.advance(ks);
          ++flushes;
        }
      }
    } else if (lane == 0) {
      // rank 1, the relay: per step "my A and B are ready", per group end
      // "my accumulators are read out", each forwarded to rank 0 once
      int64_t g = 0, flushes = 0;
      for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
        if ((g & 15) == 0 && s_abort) {
          ok = false;
          break;
        }
        const int ast = (int)(g % kPairAStages);
        if (!dev::mbar_wait_bounded(&bar_ready[ast], (uint32_t)((g / kPairAStages) & 1))) {
          ok = false;
          break;
        }
        arrive_at(&bar_ready[ast], 0);
        if (grp.ends_at(ks)) {
          if (!dev::mbar_wait_bounded(&bar_tread, (uint32_t)(flushes & 1))) {
            ok = false;
            break;
          }
          arrive_at(&bar_pfree, 0);
          ++flushes;
          grp.advance(ks);
        }
      }
    }
  } else if (a_warp) {
    // ---- FORM_A: the A warps -------------------------------------------------
    // unit i * 256 + atid of the CTA's 2 x 512 16-byte rows of a step's A
    // tiles (the table kernel's units: 4 atoms of one row m in one K block);
    // m = 2 a + {Re, Im}, and the two lanes of a row pair share
    // X = w e^{2 pi i s_a x'} of their 4 atoms
    const int atid = tid - 32 * (kSepFormWarps + 2);
    constexpr int kAUnits = 4;
    float a_s[kAUnits], a_sl[kAUnits];
    bool a_ok[kAUnits];
#pragma unroll
    for (int i = 0; i < kAUnits; ++i) {
      const int unit = i * 256 + atid, tp = unit >> 9, u = unit & 511;
      const int64_t m = (int64_t)(2 * (mp0 + tp) + (int)rank) * kSepM + ((u >> 3) & 15) * 8 + (u & 7);
      const int64_t ah = m >> 1;
      a_ok[i] = tp < ntp && ah < a.n0;
      a_s[i] = a_ok[i] ? a.axis_s[ah] : 0.f;
      a_sl[i] = a_ok[i] ? a.axis_lo[ah] : 0.f;
    }
    int64_t g = 0;
    for (int64_t ks = ks_begin; ks < ks_end; ++ks, ++g) {
      const int bst = (int)(g % kPairBStages), tst = (int)(g % kPairTStages);
      bool w = !s_abort;
      if (w && g >= kPairBStages)
        w = dev::mbar_wait_bounded(&bar_done[(g - kPairBStages) % kPairAStages],
                                   (uint32_t)(((g - kPairBStages) / kPairAStages) & 1));
      if (w) w = dev::mbar_wait_bounded(&bar_atom[tst], (uint32_t)((g / kPairTStages) & 1));
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      // the step's A tiles of this CTA (rows of M tile 2 (mp0 + tp) + rank of
      // every tile pair with rows), as the table kernel writes them: the
      // phase s_a x' with its products' rounding errors restored, MUFU
      // sin/cos, the occupancy, rows Re (Xr, -Xi) and Im (Xi, Xr), f16 hi, lo
      const float4* atl = ring_lo[tst];
      const float* atw = ring_w[tst];
#pragma unroll
      for (int i = 0; i < kAUnits; ++i) {
        const int unit = i * 256 + atid, tp = unit >> 9, u = unit & 511;
        if (tp >= ntp) continue;  // the same for the whole warp
        const int kb = u >> 7, ri = u & 1;
        float x[2], xl[2], w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = kb * 4 + 2 * ri + h;
          x[h] = ring_atom[tst][j].x;
          xl[h] = atl[j].x;
          w[h] = atw[j];
        }
        uint4 hi, lo;
        sep_a_row(a_s[i], a_sl[i], a_ok[i], ri, x, xl, w, hi, lo);
        uint4* blk = reinterpret_cast<uint4*>(ringA + (bst * 2 + tp) * kPairTileBytes);
        blk[u] = hi;
        blk[512 + u] = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&bar_ready[bst]);
        mbar_arrive(&bar_tempty[tst]);
      }
    }
  } else {
    // ---- formation warps ---------------------------------------------------
    // column col of this CTA's half: forward the point (b, c) with offsets
    // (s_b, s_c) from H, adjoint the atom's (y', z'); two threads per column,
    // thread half h forms the step's atoms 8 h .. 8 h + 7 (K blocks 2 h, 2 h + 1)
    const int c_loc = tid & (kPairHalfN - 1), half = tid / kPairHalfN;
    const int64_t col = col_base + (int64_t)rank * kPairHalfN + c_loc;
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
    const uint32_t b_row_off = (uint32_t)((c_loc >> 3) * 128 + (c_loc & 7) * 16);
    // phase bound of the call, as in the one-CTA kernel: below kSepPhaseLim
    // cycles the mod-1 reduction is skipped, above dev::kPhaseExactLim every
    // product is taken with its rounding error restored
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
      const int bst = (int)(g % kPairBStages), tst = (int)(g % kPairTStages);
      // B stage bst is free once the pair's MMAs of step g - kPairBStages completed
      bool w = !s_abort;
      if (w && g >= kPairBStages)
        w = dev::mbar_wait_bounded(&bar_done[(g - kPairBStages) % kPairAStages],
                                   (uint32_t)(((g - kPairBStages) / kPairAStages) & 1));
      if (w) w = dev::mbar_wait_bounded(&bar_atom[tst], (uint32_t)((g / kPairTStages) & 1));
      if (!__all_sync(0xffffffffu, w)) {
        ok = false;
        break;
      }
      unsigned char* sB = ringB + bst * kPairBBytes;
      const float4* at = ring_atom[tst] + half * 8;
      // mode 0: raw phase, 1: reduced mod 1, 2: exact products, reduced
      // kAtt: a buried object's rows carry exp(-att z')
      auto form = [&](auto mode_tag, auto att_tag) {
        constexpr int kMode = decltype(mode_tag)::value;
        constexpr bool kAtt = decltype(att_tag)::value;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          uint32_t hi[4] = {0u, 0u, 0u, 0u}, lo[4] = {0u, 0u, 0u, 0u};
          if (row_ok) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 v = at[kq * 4 + q];
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
          const int kb = 2 * half + kq;
          *reinterpret_cast<uint4*>(sB + kb * 2048 + b_row_off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(sB + 8192 + kb * 2048 + b_row_off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
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
        mbar_arrive(&bar_ready[bst]);
        mbar_arrive(&bar_tempty[tst]);
      }
      if (!grp.ends_at(ks)) continue;

      // ---- group end: this CTA's TMEM -> blocked partials ----------------------
      w = dev::mbar_wait_bounded(&bar_done[g % kPairAStages], (uint32_t)((g / kPairAStages) & 1));
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
        const int64_t m0 = (2 * (mp0 + tp) + rank) * kSepM + sub * 32;
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
      if (lane == 0) mbar_arrive(&bar_tread);
      grp.advance(ks);
    }
    if (att_over) dev::set_status(a.status, kStatusNonFinite);
    if (ok && first_flush) {
      // empty chunk: its partials are zero
      const int sub = warp & 3;
      const int col0 = (warp >> 2) * 128;
      for (int tp = 0; tp < ntp; ++tp) {
        const int64_t m0 = (2 * (mp0 + tp) + rank) * kSepM + sub * 32;
        for (int cc = 0; cc < 128 && col_base + col0 + cc < col_end; cc += 32) {
          float4* blk = reinterpret_cast<float4*>(part + sep_part_off(m0, col_base + col0 + cc, a.n_cb)) + lane;
          for (int q = 0; q < 8; ++q) blk[q * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
  }
  if (!ok) {
    s_abort = 1;
    // tell the peer, whose waits on this CTA would otherwise run to their limit
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_addr((const void*)&s_abort, rank ^ 1u)), "r"(1)
                 : "memory");
    dev::set_status(a.status, kStatusTimeout);
  }
  __syncthreads();
  // on abort: wait (bounded) for this CTA's MMAs and copies in flight; phases
  // already complete return at once
  if (mma_warp && lane == 0 && rank == 0 && s_abort && g_committed > 0) {
    const int64_t gl = g_committed - 1;
    dev::mbar_wait_bounded(&bar_done[gl % kPairAStages], (uint32_t)((gl / kPairAStages) & 1), 1LL << 28);
  }
  if (copy_warp && lane == 0 && s_abort) {
    for (int64_t s = a_issued > kPairAStages ? a_issued - kPairAStages : 0; s < a_issued; ++s)
      dev::mbar_wait_bounded(&bar_ready[s % kPairAStages], (uint32_t)((s / kPairAStages) & 1), 1LL << 28);
    for (int64_t s = t_issued > kPairTStages ? t_issued - kPairTStages : 0; s < t_issued; ++s)
      dev::mbar_wait_bounded(&bar_atom[s % kPairTStages], (uint32_t)((s / kPairTStages) & 1), 1LL << 28);
  }
  tc_fence_before();
  __syncthreads();
  // neither CTA leaves (or releases tensor memory) while the pair's MMAs or
  // the peer's remote arrivals may still touch its shared memory
  cluster_sync();
  if (mma_warp)
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSepTmemCols));
}

cudaError_t sep_pair_prepare_kernel() {
  static_assert(kPairSmem + 8192 <= 227 * 1024, "dynamic + static shared memory of k_sep_pair");
  const cudaError_t e =
      cudaFuncSetAttribute(k_sep_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem);
  return e != cudaSuccess
             ? e
             : cudaFuncSetAttribute(k_sep_pair<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem);
}

// Grid: x = 2 CTAs x M quads x N tiles (cluster pairs along x), y = chunks.
cudaError_t sep_pair_launch_core(const SepArgs& a, int64_t n_nt, int n_chunks, cudaStream_t st) {
  const int64_t n_mq = ((a.mp_count > 0 ? a.mp_count : (a.n_mt + 1) / 2) + 1) / 2;
  dim3 grid((unsigned)(2 * n_mq * n_nt), (unsigned)n_chunks);
  if (a.form_a)
    k_sep_pair<true><<<grid, kPairThreadsA, kPairSmem, st>>>(a);
  else
    k_sep_pair<false><<<grid, kSepThreads, kPairSmem, st>>>(a);
  return cudaGetLastError();
}

// The CTA-pair kernel is used unless SCATTER_SEP_PAIR=0 (the one-CTA kernel,
// kept for comparison).
bool sep_pair_enabled() {
  static const int on = [] {
    const char* v = std::getenv("SCATTER_SEP_PAIR");
    return (v && v[0] == '0') ? 0 : 1;
  }();
  return on != 0;
}

}  // namespace scatter
