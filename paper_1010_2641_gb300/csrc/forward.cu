// Generic forward path of the direct scattering sum (Eq. 2) on sm_103a.
//
//   prep     per call: integer centring t of each instance (rint of the
//            bounding-box centre of its atoms), split r - t = n + delta with
//            n = rint(r - t), and the per-atom phase c = frac(H . delta) in
//            FP64, stored as fp32 slots (x', y', z', c) with x' = r - t.
//            Because H . n is an integer, for S = H + s
//              S . r = S . t + H . delta + s . (r - t)  (mod 1)
//            so only the small quantities c and s . x' reach FP32.
//   generic  CTA = a tile of S points, THREADS x R points in registers; atom
//            tiles (20 B/atom) staged in shared memory by the TMA engine
//            (cp.async.bulk, double buffered on mbarriers, bounded waits).
//            Per pair: phase = c + s . x' (FFMA), reduction mod 1 (FADD),
//            sin/cos of 2 pi phase on MUFU, two FFMA into tile-blocked FP32
//            accumulators.  Species segments fold f_s(|S|) in-kernel
//            (Section 4.2: f factors out of the sum over atoms of a species).
//   reduce   split-K partials summed in a fixed order (deterministic), then
//            the translation phase e^{2 pi i s.t} and |A|^2 if requested.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include "device_common.cuh"
#include "generic_impl.cuh"
#include "launch.h"

namespace scatter {


// ---------------------------------------------------------------------------
// prep
// ---------------------------------------------------------------------------

using dev::ordered;
using dev::unordered;

__global__ void k_bbox_init(unsigned long long* bbox, int batch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch * 6) bbox[i] = (i % 6) < 3 ? ~0ULL : 0ULL;  // min slots: max value; max slots: 0
}

// One grid row per instance; each CTA reduces a strided share of the
// instance's atoms and merges with order-independent atomic min/max.
__global__ void k_bbox(const double* __restrict__ xyz, const int64_t* __restrict__ atom_off,
                       unsigned long long* bbox, unsigned* status) {
  const int inst = blockIdx.y;
  const int64_t b = atom_off[inst], e = atom_off[inst + 1];
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t j = b + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < e;
       j += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double v = xyz[3 * j + d];
      if (!isfinite(v)) {
        bad = true;
        continue;
      }
      lo[d] = fmin(lo[d], v);
      hi[d] = fmax(hi[d], v);
    }
  }
  if (bad) dev::set_status(status, kStatusNonFinite);
  __shared__ double sh[6][32];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
      hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sh[d][warp] = lo[d];
      sh[3 + d][warp] = hi[d];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int d = threadIdx.x;
    double v = sh[d][0];
    for (int w = 1; w < nw; ++w) v = d < 3 ? fmin(v, sh[d][w]) : fmax(v, sh[d][w]);
    if (isfinite(v)) {
      if (d < 3) atomicMin(&bbox[6 * inst + d], ordered(v));
      else atomicMax(&bbox[6 * inst + d], ordered(v));
    }
  }
}

__global__ void k_prep(const double* __restrict__ xyz, const float* __restrict__ occ,
                       const int32_t* __restrict__ slot_src, const int32_t* __restrict__ slot_inst,
                       const int64_t* __restrict__ inst_slot_begin, const double* __restrict__ inst_H,
                       const unsigned long long* __restrict__ bbox, double* inst_shift, float4* atom4,
                       float4* atom_lo, float* atom_w, int64_t n_slots, unsigned* status) {
  const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= n_slots) return;
  const int inst = slot_inst[slot];
  double t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const unsigned long long ulo = bbox[6 * inst + d], uhi = bbox[6 * inst + 3 + d];
    t[d] = (ulo == ~0ULL || uhi == 0ULL) ? 0.0 : rint(0.5 * (unordered(ulo) + unordered(uhi)));
  }
  if (slot == inst_slot_begin[inst]) {
#pragma unroll
    for (int d = 0; d < 3; ++d) inst_shift[3 * inst + d] = t[d];
  }
  const int32_t src = slot_src[slot];
  if (src < 0) {
    atom4[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    atom_lo[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    atom_w[slot] = 0.f;
    return;
  }
  const double* H = inst_H + 3 * inst;
  double r[3];
  bool ok = true;
  double c = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    r[d] = xyz[3 * (int64_t)src + d] - t[d];
    ok = ok && isfinite(r[d]);
    const double delta = r[d] - rint(r[d]);
    c = fma(H[d], delta, c);
  }
  float w = occ ? occ[src] : 1.0f;
  ok = ok && isfinite(w);
  if (!ok) {
    dev::set_status(status, kStatusNonFinite);
    atom4[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    atom_lo[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    atom_w[slot] = 0.f;
    return;
  }
  c -= rint(c);
  const float x0 = (float)r[0], x1 = (float)r[1], x2 = (float)r[2];
  atom4[slot] = make_float4(x0, x1, x2, (float)c);
  atom_lo[slot] = make_float4((float)(r[0] - (double)x0), (float)(r[1] - (double)x1), (float)(r[2] - (double)x2), 0.f);
  atom_w[slot] = w;
}

// ---------------------------------------------------------------------------
// generic kernel
// ---------------------------------------------------------------------------

template <int MODE, int R, int THREADS>
__global__ void __launch_bounds__(THREADS) k_generic(const GenericArgs a) {
  __shared__ __align__(128) float4 sh_atom[2][kTile];
  __shared__ __align__(128) float4 sh_lo[2][kTile];  // position rounding errors (exact-product phases)
  __shared__ __align__(128) float sh_w[2][kTile];
  __shared__ __align__(8) uint64_t sh_bar[2];

  const int tid = threadIdx.x;
  const int chunk = blockIdx.y;

  // ---- S points of this thread -------------------------------------------
  float sx[R], sy[R], sz[R];
  int64_t idx0 = 0;      // GRID: output index of point 0; LIST: tile base
  int nvalid = 0;        // GRID: number of valid points (prefix)
  bool valid[R];
  if (MODE == kModeGrid) {
    const int64_t q = (a.n2 + R - 1) / R;
    const int64_t g = (int64_t)blockIdx.x * THREADS + tid;
    const bool active = g < a.n0 * a.n1 * q;
    const int64_t line = active ? g / q : 0, blk = active ? g % q : 0;
    const int64_t i0 = line / a.n1, i1 = line % a.n1, i2 = blk * R;
    const float x = a.axis_s[i0], y = a.axis_s[a.n0 + i1];
    nvalid = active ? (int)dev::min64(R, a.n2 - i2) : 0;
    idx0 = line * a.n2 + i2;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      sx[r] = x;
      sy[r] = y;
      sz[r] = a.axis_s[a.n0 + a.n1 + dev::min64(i2 + r, a.n2 - 1)];
      valid[r] = r < nvalid;
    }
  } else {
    idx0 = (int64_t)blockIdx.x * THREADS * R;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t m = idx0 + (int64_t)r * THREADS + tid;
      valid[r] = m < a.n_s;
      const int64_t mm = valid[r] ? m : 0;
      sx[r] = a.s_hi[mm];
      sy[r] = a.s_hi[a.n_s + mm];
      sz[r] = a.s_hi[2 * a.n_s + mm];
    }
  }

  if (tid == 0) {
    dev::mbar_init(&sh_bar[0], 1);
    dev::mbar_init(&sh_bar[1], 1);
    dev::mbar_fence_init();
  }
  __syncthreads();
  // output index of point r: pbase + r pstride (for a factor table)
  const int64_t pbase = MODE == kModeGrid ? idx0 : idx0 + tid;
  const int64_t pstride = MODE == kModeGrid ? 1 : THREADS;
  float2 tot[R];
  int k = 0;
  // one decision per call (every CTA computes the same): phases that can
  // pass kPhaseExactLim cycles take the exact-product route, with s as a
  // double-float
  bool ok;
  if (dev::phase_needs_exact(a.bbox, a.shift, a.smax_dev ? a.smax_dev : a.smax)) {
    int64_t i0 = 0, i1 = 0, i2 = 0;
    if (MODE == kModeGrid) {
      const int64_t q = (a.n2 + R - 1) / R;
      const int64_t g = (int64_t)blockIdx.x * THREADS + tid;
      const int64_t line = g < a.n0 * a.n1 * q ? g / q : 0;
      i0 = line / a.n1;
      i1 = line % a.n1;
      i2 = idx0 - line * a.n2;
    }
    auto lo = [&](int r, float& x, float& y, float& z) {
      if (MODE == kModeGrid) {
        x = a.axis_lo[i0];
        y = a.axis_lo[a.n0 + i1];
        z = a.axis_lo[a.n0 + a.n1 + dev::min64(i2 + r, a.n2 - 1)];
      } else {
        const int64_t m = valid[r] ? idx0 + (int64_t)r * THREADS + tid : 0;
        x = a.s_lo[m];
        y = a.s_lo[a.n_s + m];
        z = a.s_lo[2 * a.n_s + m];
      }
    };
    ok = chunk_sum_exact_halves<MODE, R>(a.atom4, a.atom_lo, a.atom_w, a.segs, a.chunk_seg_off[chunk],
                                         a.chunk_seg_off[chunk + 1], a.coef, a.H, a.inv4a2, sx, sy, sz, lo, sh_atom,
                                         sh_lo, sh_w, sh_bar, k, tot, a.status, a.ftab, a.n_s, pbase, pstride);
  } else {
    ok = chunk_sum<MODE, R, false>(a.atom4, a.atom_lo, a.atom_w, a.segs, a.chunk_seg_off[chunk],
                                   a.chunk_seg_off[chunk + 1], a.coef, a.H, a.inv4a2, sx, sy, sz, sx, sy, sz, sh_atom,
                                   sh_lo, sh_w, sh_bar, k, tot, a.status, a.ftab, a.n_s, pbase, pstride);
  }
  if (!ok) return;

  // ---- epilogue -----------------------------------------------------------------
  if (a.partial) {
    float2* out = a.partial + (int64_t)chunk * a.n_s;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!valid[r]) continue;
      const int64_t m = MODE == kModeGrid ? idx0 + r : idx0 + (int64_t)r * THREADS + tid;
      out[m] = tot[r];
    }
    return;
  }
  const double* t = a.shift;
  const bool shifted = t[0] != 0.0 || t[1] != 0.0 || t[2] != 0.0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (!valid[r]) continue;
    int64_t m;
    float2 v = tot[r];
    if (MODE == kModeGrid) {
      m = idx0 + r;
      if (shifted) {
        const int64_t i2 = m % a.n2, line = m / a.n2, i1 = line % a.n1, i0 = line / a.n1;
        v = dev::cmul(dev::shift_phase(a.axis64[i0] - a.H64[0], a.axis64[a.n0 + i1] - a.H64[1],
                                       a.axis64[a.n0 + a.n1 + i2] - a.H64[2], t),
                      v);
      }
    } else {
      m = idx0 + (int64_t)r * THREADS + tid;
      if (shifted)
        v = dev::cmul(dev::shift_phase(a.S64[3 * m] - a.H64[0], a.S64[3 * m + 1] - a.H64[1],
                                       a.S64[3 * m + 2] - a.H64[2], t),
                      v);
    }
    if (a.out_amp) a.out_amp[m] = v;
    if (a.out_int) a.out_int[m] = v.x * v.x + v.y * v.y;
  }
}

// Sum of split-K partials in chunk order, translation phase, outputs.
__global__ void k_reduce(GenericArgs a, int split_k, int grid_mode) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.n_s) return;
  float2 v = make_float2(0.f, 0.f);
  for (int c = 0; c < split_k; ++c) {
    const float2 p = a.partial[(int64_t)c * a.n_s + m];
    v.x += p.x;
    v.y += p.y;
  }
  const double* t = a.shift;
  if (t[0] != 0.0 || t[1] != 0.0 || t[2] != 0.0) {
    if (grid_mode) {
      const int64_t i2 = m % a.n2, line = m / a.n2, i1 = line % a.n1, i0 = line / a.n1;
      v = dev::cmul(dev::shift_phase(a.axis64[i0] - a.H64[0], a.axis64[a.n0 + i1] - a.H64[1],
                                     a.axis64[a.n0 + a.n1 + i2] - a.H64[2], t),
                    v);
    } else {
      v = dev::cmul(dev::shift_phase(a.S64[3 * m] - a.H64[0], a.S64[3 * m + 1] - a.H64[1],
                                     a.S64[3 * m + 2] - a.H64[2], t),
                    v);
    }
  }
  if (a.out_amp) a.out_amp[m] = v;
  if (a.out_int) a.out_int[m] = v.x * v.x + v.y * v.y;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

template <int MODE, int R, int THREADS>
void* generic_fn() {
  return (void*)&k_generic<MODE, R, THREADS>;
}

void* pick_generic(int mode, int R, int threads) {
#define SCATTER_CASE(M, RR, TT) \
  if (mode == M && R == RR && threads == TT) return generic_fn<M, RR, TT>();
  SCATTER_CASE(kModeList, 4, 128) SCATTER_CASE(kModeList, 4, 256)
  SCATTER_CASE(kModeList, 8, 128) SCATTER_CASE(kModeList, 8, 256)
  SCATTER_CASE(kModeList, 16, 128) SCATTER_CASE(kModeList, 16, 256)
  SCATTER_CASE(kModeGrid, 4, 128) SCATTER_CASE(kModeGrid, 4, 256)
  SCATTER_CASE(kModeGrid, 8, 128) SCATTER_CASE(kModeGrid, 8, 256)
  SCATTER_CASE(kModeGrid, 16, 128) SCATTER_CASE(kModeGrid, 16, 256)
#undef SCATTER_CASE
  return nullptr;
}

int mode_of(const scatter_plan_s* p) { return p->s_kind == SCATTER_S_GRID ? kModeGrid : kModeList; }

GenericArgs make_args(scatter_plan_t p) {
  GenericArgs a{};
  a.atom4 = p->d.atom4;
  a.atom_lo = p->d.atom_lo;
  a.atom_w = p->d.atom_w;
  a.segs = p->d.segs;
  a.chunk_seg_off = p->d.chunk_seg_off;
  a.coef = p->d.coef;
  a.n_s = p->n_s;
  a.s_hi = p->d.s_hi;
  a.s_lo = p->d.s_lo;
  a.S64 = p->d.S64;
  a.axis_s = p->d.axis_s;
  a.axis_lo = p->d.axis_lo;
  a.axis64 = p->d.axis64;
  a.n0 = p->n_axis[0];
  a.n1 = p->n_axis[1];
  a.n2 = p->n_axis[2];
  for (int d = 0; d < 3; ++d) {
    a.H[d] = (float)p->inst[0].H[d];
    a.H64[d] = p->inst[0].H[d];
  }
  a.inv4a2 = (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a));
  a.shift = p->d.inst_shift;
  a.bbox = p->d.inst_bbox;
  for (int d = 0; d < 3; ++d) a.smax[d] = (float)p->s_max[d];
  a.ftab = p->d.ftab;
  a.status = p->d.status;
  return a;
}

}  // namespace

bool generic_tiling_supported(const Tiling& t) {
  return pick_generic(kModeList, t.R, t.threads) != nullptr && t.split_k >= 1;
}

int64_t generic_num_tiles(const scatter_plan_s* p, const Tiling& t) {
  if (mode_of(p) == kModeGrid) {
    const int64_t q = (p->n_axis[2] + t.R - 1) / t.R;
    return (p->n_axis[0] * p->n_axis[1] * q + t.threads - 1) / t.threads;
  }
  const int64_t per = (int64_t)t.threads * t.R;
  return (p->n_s + per - 1) / per;
}

int generic_blocks_per_sm(const scatter_plan_s* p, const Tiling& t) {
  void* fn = pick_generic(mode_of(p), t.R, t.threads);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, t.threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

scatter_status launch_prep(scatter_plan_t p, const double* xyz, const float* occ, cudaStream_t st) {
  const int batch = p->batch;
  k_bbox_init<<<(batch * 6 + 255) / 256, 256, 0, st>>>(p->d.inst_bbox, batch);
  p->last_launches += 2;
  int64_t max_atoms = 0;
  for (const auto& in : p->inst) max_atoms = std::max<int64_t>(max_atoms, in.atom_end - in.atom_begin);
  const int bx = (int)dev::min64(std::max<int64_t>((max_atoms + 255) / 256, 1), 64);
  k_bbox<<<dim3(bx, batch), 256, 0, st>>>(xyz, p->d.atom_off, p->d.inst_bbox, p->d.status);
  if (p->n_slots > 0) {
    const int64_t nb = (p->n_slots + 255) / 256;
    k_prep<<<(unsigned)nb, 256, 0, st>>>(xyz, occ, p->d.slot_src, p->d.slot_inst, p->d.inst_slot_begin,
                                         p->d.inst_H, p->d.inst_bbox, p->d.inst_shift, p->d.atom4,
                                         p->d.atom_lo, p->d.atom_w, p->n_slots, p->d.status);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "prep launch");
}

scatter_status launch_bbox_raw(const double* xyz, const int64_t* atom_off, int batch, int64_t max_atoms,
                               unsigned long long* bbox, unsigned* status, cudaStream_t st) {
  const int bx = (int)dev::min64(std::max<int64_t>((max_atoms + 255) / 256, 1), 64);
  k_bbox<<<dim3(bx, batch), 256, 0, st>>>(xyz, atom_off, bbox, status);
  return cuda_status(cudaGetLastError(), "bounding-box launch");
}

scatter_status launch_generic_reduce(scatter_plan_t p, int n_chunks, float2* amp_out, float* int_out,
                                     cudaStream_t st) {
  GenericArgs a = make_args(p);
  a.partial = p->d.partial;
  a.out_amp = amp_out;
  a.out_int = int_out;
  const int64_t nb = (p->n_s + 255) / 256;
  if (nb > 0) {
    k_reduce<<<(unsigned)nb, 256, 0, st>>>(a, n_chunks, mode_of(p) == kModeGrid);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "generic reduction launch");
}

scatter_status launch_generic(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st) {
  if (p->tiling.atom_k > 0) return launch_atompar(p, amp_out, int_out, st);
  const Tiling& t = p->tiling;
  void* fn = pick_generic(mode_of(p), t.R, t.threads);
  if (!fn) return fail(SCATTER_ERR_UNSUPPORTED, "no generic kernel for R=%d threads=%d", t.R, t.threads);
  GenericArgs a = make_args(p);
  const int n_chunks = (int)p->chunk_seg_off.size() - 1;
  if (n_chunks > 1) {
    a.partial = p->d.partial;
  } else {
    a.out_amp = amp_out;
    a.out_int = int_out;
  }
  const int64_t tiles = generic_num_tiles(p, t);
  if (tiles > 0 && n_chunks > 0) {
    dim3 grid((unsigned)tiles, (unsigned)n_chunks);
    void* args[] = {&a};
    timing_begin(p, st);
    cudaError_t e = cudaLaunchKernel(fn, grid, dim3(t.threads), args, 0, st);
    timing_end(p, st);
    if (e != cudaSuccess) return cuda_status(e, "generic kernel launch");
    p->last_launches += 1;
  }
  if (n_chunks > 1) {
    a.partial = p->d.partial;
    a.out_amp = amp_out;
    a.out_int = int_out;
    const int64_t nb = (p->n_s + 255) / 256;
    k_reduce<<<(unsigned)nb, 256, 0, st>>>(a, n_chunks, mode_of(p) == kModeGrid);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "generic launch");
}

// Launches the LIST-mode generic kernel (and the split-K reduction) on fully
// prepared arguments; used by callers that own their buffers.
scatter_status launch_generic_args(GenericArgs a, int R, int threads, int n_chunks, cudaStream_t st) {
  void* fn = pick_generic(kModeList, R, threads);
  if (!fn) return fail(SCATTER_ERR_UNSUPPORTED, "no generic kernel for R=%d threads=%d", R, threads);
  float2* out_amp = a.out_amp;
  float* out_int = a.out_int;
  float2* partial = a.partial;
  if (n_chunks > 1) {
    a.out_amp = nullptr;
    a.out_int = nullptr;
  } else {
    a.partial = nullptr;
  }
  const int64_t per = (int64_t)threads * R;
  const int64_t tiles = (a.n_s + per - 1) / per;
  if (tiles > 0 && n_chunks > 0) {
    void* args[] = {&a};
    cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)tiles, (unsigned)n_chunks), dim3(threads), args, 0, st);
    if (e != cudaSuccess) return cuda_status(e, "generic kernel launch");
  }
  if (n_chunks > 1 && a.n_s > 0) {
    a.partial = partial;
    a.out_amp = out_amp;
    a.out_int = out_int;
    k_reduce<<<(unsigned)((a.n_s + 255) / 256), 256, 0, st>>>(a, n_chunks, 0);
  }
  return cuda_status(cudaGetLastError(), "generic launch");
}

}  // namespace scatter
