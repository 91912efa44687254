// Shared pieces of the tcgen05 contraction kernel k_sep: tile constants,
// descriptors, the MMA / TMEM wrappers, the f16 hi/lo split and the kernel
// arguments.  k_sep computes, for one CTA, D[rows, cols] = sum_K A[rows, K]
// B[cols, K] with A read as precomputed f16 hi/lo blocks and B formed in
// the kernel: B[col, (k, Re|Im)] = e^{2 pi i (u_col v_k + w_col z_k + c_k)}
// from a per-column pair (u, w) and a per-K record (., v, z, c).
//   forward (Eq. 2):  cols = grid points (s_b, s_c), K = atoms (y', z', c)
//   adjoint:          cols = atoms (y', z'),        K = grid points (s_b, s_c, 0)
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include "device_common.cuh"
#include "plan.h"

namespace scatter {

constexpr int kSepFormWarps = 8;           // warps forming B rows (one N column per thread)
constexpr int kSepThreads = 32 * (kSepFormWarps + 2);  // + the MMA warp + the copy warp
constexpr int kSepM = 128;                 // MMA M (rows of A per CTA)
constexpr int kSepN = 256;                 // MMA N (columns per CTA)
constexpr int kSepStep = 16;               // K records per pipeline step (K' = 32)
constexpr int kSepFlush = 256;             // steps between TMEM flushes
constexpr uint32_t kSepABytes = 16384;     // A block of one M tile: hi + lo, 128 x 32 f16 each
constexpr int kSepPair = 2;                // M tiles per CTA (one formed B tile feeds both)
constexpr uint32_t kSepBBytes = 32768;     // B block: hi + lo, 256 x 32 f16 each
constexpr int kSepAStages = 4;             // A ring (full / empty barrier per stage)
constexpr int kSepBStages = 2;             // B ring: formation of step k+1 overlaps MMAs of k
constexpr int kSepTStages = 8;             // K-record ring (256 B per step)
constexpr size_t kSepSmem = kSepAStages * kSepPair * kSepABytes + kSepBStages * kSepBBytes + 1024;  // + align
constexpr uint32_t kSepTmemCols = 512;     // two 128 x 256 FP32 accumulators
constexpr double kSepPhaseLim = 16.0;      // cycles: B phases below this skip the mod-1 reduction
// largest exponent of a formed row's attenuation exp(-2 pi Im(sigma) z'): e^10
// keeps hi + lo inside f16's range; beyond it the call reports NUMERIC
constexpr float kSepAttMax = 10.0f;

// -------------------------------------------------------------------------
// descriptors (PTX tcgen05 shared-memory and instruction descriptors)
// -------------------------------------------------------------------------

// No-swizzle K-major operand: 8-row x 16-byte core matrices; lbo = byte
// stride between core matrices along K, sbo = along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor core
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// kind::f16: D f32, A and B f16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kSepIdesc = (1u << 4) | ((uint32_t)(kSepN >> 3) << 17) | ((uint32_t)(kSepM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kSepIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   dev::smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t addr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// f16 hi/lo split of two floats packed as f16x2 each.
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(y), "f"(x));
  const __half2 h = *reinterpret_cast<const __half2*>(&hi);
  const float2 hf = __half22float2(h);
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(y - hf.y), "f"(x - hf.x));
}

// One 16-byte row of the A operand's core matrix, hi and lo: row m = 2 a +
// ri (Re or Im of axis value a, offset s_a = sa + sal) over one K block of 4
// atoms.  Lanes l and l ^ 1 hold rows 2 a and 2 a + 1 of the same a and
// share X_j = w_j e^{2 i pi s_a x'_j}: lane ri evaluates atoms 2 ri, 2 ri + 1
// of the block (x'_j with its rounding error xl_j, weight w_j) and takes the
// other two from its neighbour.  The phase is reduced exactly mod 1 (the
// products' rounding errors restored) before the MUFU sin/cos: |error| <
// 4e-7, below the hi + lo split's resolution.  Row 2 a holds (Xr, -Xi), row
// 2 a + 1 (Xi, Xr).  All 32 lanes of the warp must call it together (ok
// false gives a zero row).  The table kernel and the CTA pair's A warps
// both form A through it, so the two routes agree bit for bit.
__device__ __forceinline__ void sep_a_row(float sa, float sal, bool ok, int ri, const float (&x)[2],
                                          const float (&xl)[2], const float (&w)[2], uint4& hi, uint4& lo) {
  float sq[2], cq[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float sn = 0.f, cs = 0.f;
    if (ok) {
      dev::sincos_cycles_mufu(dev::frac_of_product2(sa, sal, x[h]) + sa * xl[h], &sn, &cs);
      sn *= w[h];
      cs *= w[h];
    }
    sq[h] = sn;
    cq[h] = cs;
  }
  float v[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int h = q & 1;
    const float ps = __shfl_xor_sync(0xffffffffu, sq[h], 1), pc = __shfl_xor_sync(0xffffffffu, cq[h], 1);
    const bool own = (q >> 1) == ri;
    const float sn = own ? sq[h] : ps, cs = own ? cq[h] : pc;
    v[2 * q] = ri ? sn : cs;
    v[2 * q + 1] = ri ? cs : -sn;
  }
  split2(v[0], v[1], hi.x, lo.x);
  split2(v[2], v[3], hi.y, lo.y);
  split2(v[4], v[5], hi.z, lo.z);
  split2(v[6], v[7], hi.w, lo.w);
}

struct SepArgs {
  const uint4* A;         // A blocks [species][M-tile pair][step][2 tiles][hi|lo] of 16 KB per tile
  int64_t a_sp_stride;    // uint4 per species table of A (0: one table, the forward)
  const float4* rec;      // K records, 16 per step: forward the atom slots (x', y', z', c),
                          // adjoint the grid points (0, s_b, s_c, 0)
  const Segment* chunks;  // per blockIdx.y: K range in records (multiples of 16)
  const Segment* ntiles;  // adjoint: slot range and species of each N tile; null: N = grid points
  const float4* atom4;    // adjoint: the columns' atoms (y', z' read)
  const float* axis_s;    // forward: the columns' points, s = axis - H ([n0 | n1 | n2])
  const float* axis_lo;   // forward: rounding errors of axis_s (double-float s, exact formation); adjoint null
  const unsigned long long* bbox;  // instance 0: ordered min xyz, max xyz of this call's positions
  const double* shift;             // instance 0: its centring t
  float smax_b, smax_c;            // max |s| of the b and c axes
  int64_t n0, n1, n2;     // grid shape
  int64_t n_steps, n_mt;  // K steps per A table, M tiles
  int64_t n_cb;           // 32-column blocks of the partials (ceil(columns / 32))
  int64_t chunk_floats;   // floats of one chunk's partials (sep_part_floats)
  float* partial;         // [chunk] blocked as sep_part_off, raw D (no f_s)
  unsigned* status;
  const float* axis_att;  // forward of a buried object: per l, 2 pi Im(sigma); the formed
                          // rows carry exp(-axis_att[l] z'); null otherwise
  int64_t mp_first;       // M-tile pairs of this launch: [mp_first, mp_first + mp_count)
  int64_t mp_count;       // (0: all (n_mt + 1) / 2 of them)
  int form_a;             // CTA-pair forward: 1 = the A tiles are formed in the kernel from the
                          // records (rec_lo, rec_w beside them) instead of streamed from `A`
  const float4* rec_lo;   //   the records' position rounding errors (x' error read)
  const float* rec_w;     //   the atoms' occupancies
};

// Partials in the accumulator's own blocking.  D row m (TMEM lane of its M
// tile: m = 2 pa + ri, Re or Im of row pa) and column c live at
//   (((m / 32) n_cb + c / 32) 8 + (c % 32) / 4) 128 + (m % 32) 4 + c % 4
// floats into a chunk's partials: the 32 x 32 block a warp reads from TMEM
// with one 32x32b.x32 load is 4 KB contiguous, and each of the warp's eight
// float4 stores or reductions covers 512 contiguous bytes (lane l holds row
// m0 + l, columns 4 q .. 4 q + 3 at float4 q * 32 + l of the block).
__host__ __device__ __forceinline__ int64_t sep_part_off(int64_t m, int64_t c, int64_t n_cb) {
  return ((((m >> 5) * n_cb + (c >> 5)) * 8 + ((c & 31) >> 2)) << 7) + ((m & 31) << 2) + (c & 3);
}
// floats per chunk: every row of n_mt M tiles rounded up to pairs, columns
// rounded up to blocks of 32
inline int64_t sep_part_floats(int64_t n_mt, int64_t n_cols) {
  return ((n_mt + 1) / 2) * 2 * 128 * ((n_cols + 31) / 32) * 32;
}

// Accumulation groups: the steps between two TMEM flushes (every kSepFlush
// steps and at the end of the chunk).  Every role walks them identically.
struct SepGroups {
  int64_t ks_end, grp_start;
  __device__ bool ends_at(int64_t ks) const { return ks + 1 == ks_end || ks + 1 - grp_start >= kSepFlush; }
  __device__ void advance(int64_t ks) { grp_start = ks + 1; }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(dev::smem_addr(bar)) : "memory");
}

// Launches k_sep on `st` (its shared-memory attribute set by sep_prepare_kernel).
// side, fork, join: where an odd M-tile pair count splits between the two
// kernels, the one-CTA kernel's launch runs on `side`, forked from `st` by
// `fork` and joined back by `join`, beside the CTA-pair kernel (null: after
// it on `st`)
cudaError_t sep_launch_core(const SepArgs& a, dim3 grid, cudaStream_t st, cudaStream_t side = nullptr,
                            cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
// kernels sep_launch_core launches for n_mt M tiles (1, or 2 when an odd
// M-tile pair count splits between the CTA-pair and the one-CTA kernel)
int sep_core_launches(int64_t n_mt);
// creates the plan's side stream and its events where n_mt M tiles split
scatter_status sep_prepare_side(scatter_plan_s* p, int64_t n_mt);
cudaError_t sep_prepare_kernel();
// The CTA-pair form (sep_pair.cu): n_nt N tiles, n_chunks atom chunks.
cudaError_t sep_pair_launch_core(const SepArgs& a, int64_t n_nt, int n_chunks, cudaStream_t st);
cudaError_t sep_pair_prepare_kernel();
bool sep_pair_enabled();

}  // namespace scatter
