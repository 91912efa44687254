// Many independent crystals of uneven size in one persistent launch.
//
// The paper cut the atom list into batches short enough for the display
// watchdog (Section 5); here the unit of work is an item (instance, S tile,
// atom chunk).  Big instances are split over several atom chunks so that no
// item dominates, items are sorted longest-first (LPT), and a persistent grid
// of (#SMs x resident CTAs) pulls them from one atomic counter.  Items of an
// instance with one chunk write the map directly; split instances write
// partials that a second kernel sums in chunk order (deterministic).  The
// whole per-call sequence (counter reset, prep, persistent kernel, reduce) is
// captured once into a CUDA graph on a plan-owned stream and replayed while
// the caller's pointers stay the same.
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <vector>
#include "device_common.cuh"
#include "generic_impl.cuh"
#include "launch.h"

namespace scatter {

struct BatchArgs {
  const float4* atom4;
  const float4* atom_lo;  // position rounding errors (exact-product phases)
  const float* atom_w;
  const Segment* segs;
  const int32_t* chunk_seg_off;
  const float* coef;
  const float2* ftab;   // Eq. 4 factor table [n_species][M], or null (form factors)
  const float* s_hi;
  const float* s_lo;  // rounding error of s_hi (double-float s of the exact-product phases)
  const double* S64;
  int64_t n_s;
  const BatchInst* inst;
  const BatchItem* items;
  int32_t n_items;
  const double* inst_H;
  const double* inst_shift;
  const unsigned long long* inst_bbox;  // [batch][6] ordered min / max xyz of this call
  float smax[3];                        // max |S_d - H_d| over every instance's points
  float inv4a2;
  int* counter;
  float2* partial;
  float2* out_amp;
  float* out_int;
  unsigned* status;
};

template <int R, int THREADS>
__global__ void __launch_bounds__(THREADS) k_batch(const BatchArgs a) {
  __shared__ __align__(128) float4 sh_atom[2][kTile];
  __shared__ __align__(128) float4 sh_lo[2][kTile];
  __shared__ __align__(128) float sh_w[2][kTile];
  __shared__ __align__(8) uint64_t sh_bar[2];
  __shared__ int sh_item;
  const int tid = threadIdx.x;
  if (tid == 0) {
    dev::mbar_init(&sh_bar[0], 1);
    dev::mbar_init(&sh_bar[1], 1);
    dev::mbar_fence_init();
  }
  int k = 0;
  for (;;) {
    __syncthreads();  // previous item fully done (and barrier init visible)
    if (tid == 0) sh_item = atomicAdd(a.counter, 1);
    __syncthreads();
    const int it = sh_item;
    if (it >= a.n_items) break;
    const BatchItem w = a.items[it];
    const BatchInst in = a.inst[w.inst];
    float sx[R], sy[R], sz[R];
    bool valid[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t m = w.p0 + (int64_t)r * THREADS + tid;
      valid[r] = m < in.s_end;
      const int64_t mm = valid[r] ? m : in.s_begin;
      sx[r] = a.s_hi[mm];
      sy[r] = a.s_hi[a.n_s + mm];
      sz[r] = a.s_hi[2 * a.n_s + mm];
    }
    const int chunk = in.chunk0 + w.chunk;
    float2 tot[R];
    // a long crystal takes the exact-product phases with s as a double-float;
    // an Eq. 4 table holds one factor per (type, point) of the whole batch
    bool ok;
    if (dev::phase_needs_exact(a.inst_bbox + 6 * w.inst, a.inst_shift + 3 * w.inst, a.smax)) {
      auto lo = [&](int r, float& x, float& y, float& z) {
        const int64_t m = w.p0 + (int64_t)r * THREADS + tid;
        const int64_t mm = valid[r] ? m : in.s_begin;
        x = a.s_lo[mm];
        y = a.s_lo[a.n_s + mm];
        z = a.s_lo[2 * a.n_s + mm];
      };
      ok = chunk_sum_exact_halves<kModeList, R>(a.atom4, a.atom_lo, a.atom_w, a.segs, a.chunk_seg_off[chunk],
                                                a.chunk_seg_off[chunk + 1], a.coef, in.H, a.inv4a2, sx, sy, sz, lo,
                                                sh_atom, sh_lo, sh_w, sh_bar, k, tot, a.status, a.ftab, a.n_s,
                                                w.p0 + tid, THREADS);
    } else {
      ok = chunk_sum<kModeList, R, false>(a.atom4, a.atom_lo, a.atom_w, a.segs, a.chunk_seg_off[chunk],
                                          a.chunk_seg_off[chunk + 1], a.coef, in.H, a.inv4a2, sx, sy, sz, sx, sy, sz,
                                          sh_atom, sh_lo, sh_w, sh_bar, k, tot, a.status, a.ftab, a.n_s, w.p0 + tid,
                                          THREADS);
    }
    if (!ok) return;
    const int64_t M_b = in.s_end - in.s_begin;
    const double* t = a.inst_shift + 3 * w.inst;
    const double* H64 = a.inst_H + 3 * w.inst;
    const bool shifted = t[0] != 0.0 || t[1] != 0.0 || t[2] != 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!valid[r]) continue;
      const int64_t m = w.p0 + (int64_t)r * THREADS + tid;
      if (in.split > 1) {
        a.partial[in.part_off + (int64_t)w.chunk * M_b + (m - in.s_begin)] = tot[r];
        continue;
      }
      float2 v = tot[r];
      if (shifted)
        v = dev::cmul(dev::shift_phase(a.S64[3 * m] - H64[0], a.S64[3 * m + 1] - H64[1], a.S64[3 * m + 2] - H64[2], t),
                      v);
      if (a.out_amp) a.out_amp[m] = v;
      if (a.out_int) a.out_int[m] = v.x * v.x + v.y * v.y;
    }
  }
}

__global__ void k_batch_reduce(const BatchArgs a, const int32_t* __restrict__ s_inst) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.n_s) return;
  const int b = s_inst[m];
  const BatchInst in = a.inst[b];
  if (in.split <= 1) return;
  const int64_t M_b = in.s_end - in.s_begin;
  float2 v = make_float2(0.f, 0.f);
  for (int c = 0; c < in.split; ++c) {
    const float2 p = a.partial[in.part_off + (int64_t)c * M_b + (m - in.s_begin)];
    v.x += p.x;
    v.y += p.y;
  }
  const double* t = a.inst_shift + 3 * b;
  const double* H64 = a.inst_H + 3 * b;
  if (t[0] != 0.0 || t[1] != 0.0 || t[2] != 0.0)
    v = dev::cmul(dev::shift_phase(a.S64[3 * m] - H64[0], a.S64[3 * m + 1] - H64[1], a.S64[3 * m + 2] - H64[2], t), v);
  if (a.out_amp) a.out_amp[m] = v;
  if (a.out_int) a.out_int[m] = v.x * v.x + v.y * v.y;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

template <int R, int THREADS>
void* batch_fn() {
  return (void*)&k_batch<R, THREADS>;
}

void* pick_batch(int R, int threads) {
#define SCATTER_BCASE(RR, TT) \
  if (R == RR && threads == TT) return batch_fn<RR, TT>();
  SCATTER_BCASE(4, 128) SCATTER_BCASE(4, 256) SCATTER_BCASE(8, 128) SCATTER_BCASE(8, 256)
  SCATTER_BCASE(16, 128) SCATTER_BCASE(16, 256)
#undef SCATTER_BCASE
  return nullptr;
}

template <class T>
cudaError_t upload_vec(T** dst, const std::vector<T>& v, int64_t* bytes) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)dst, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  *bytes += (int64_t)(v.size() * sizeof(T));
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

int batch_blocks_per_sm(int R, int threads) {
  void* fn = pick_batch(R, threads);
  if (!fn) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return std::max(nb, 1);
}

// Work list of a batch plan for the plan's (threads, R): per-instance atom
// splits so that no item exceeds ~1/8 of a wave's share of the total work,
// chunks cut at species boundaries, items sorted longest-first.
scatter_status prepare_batch(scatter_plan_s* p) {
  const Tiling& t = p->tiling;
  if (!pick_batch(t.R, t.threads)) return fail(SCATTER_ERR_INVALID_ARG, "unsupported batch tiling");
  const int64_t P = (int64_t)t.threads * t.R;
  const int B = p->batch;
  const int bps = batch_blocks_per_sm(t.R, t.threads);
  const double ctas = (double)p->n_sm * bps;
  double total = 0.0;
  for (const Instance& in : p->inst)
    total += (double)(in.s_end - in.s_begin) * (double)std::max<int64_t>(in.slot_end - in.slot_begin, 0);
  const double target = std::max(total / (ctas * 8.0), (double)P * 256.0);

  std::vector<int32_t> chunk_seg_off(1, 0);
  std::vector<Segment> segs;
  std::vector<BatchInst> binst(B);
  std::vector<BatchItem> items;
  std::vector<double> cost;
  int64_t part = 0;
  int32_t chunk0 = 0;
  for (int b = 0; b < B; ++b) {
    const Instance& in = p->inst[b];
    const int64_t n = in.slot_end - in.slot_begin;
    const int64_t M_b = in.s_end - in.s_begin;
    int split = (int)std::ceil((double)std::min<int64_t>(P, M_b) * (double)n / target);
    split = std::max(1, std::min(split, 64));
    while (split > 1 && n / split < 256) --split;
    int64_t per = (n + split - 1) / std::max(split, 1);
    per = std::max<int64_t>(kSlotAlign, (per + kSlotAlign - 1) / kSlotAlign * kSlotAlign);
    std::vector<Segment> sp;
    for (const Segment& s : p->all_segs)
      if (s.instance == b) sp.push_back(s);
    std::vector<int64_t> chunk_cnt;
    for (int c = 0; c < split; ++c) {
      const int64_t lo = in.slot_begin + c * per, hi = std::min(in.slot_end, lo + per);
      int64_t cnt = 0;
      for (const Segment& s : sp) {
        const int64_t b2 = std::max(lo, s.begin), e2 = std::min(hi, s.end);
        if (b2 < e2) {
          segs.push_back(Segment{b2, e2, s.species, s.instance});
          cnt += e2 - b2;
        }
      }
      chunk_seg_off.push_back((int32_t)segs.size());
      chunk_cnt.push_back(cnt);
    }
    BatchInst bi{};
    bi.s_begin = in.s_begin;
    bi.s_end = in.s_end;
    bi.split = split;
    bi.chunk0 = chunk0;
    bi.part_off = split > 1 ? part : 0;
    for (int d = 0; d < 3; ++d) bi.H[d] = (float)in.H[d];
    binst[b] = bi;
    if (split > 1) part += (int64_t)split * M_b;
    chunk0 += split;
    for (int64_t p0 = in.s_begin; p0 < in.s_end; p0 += P)
      for (int c = 0; c < split; ++c) {
        items.push_back(BatchItem{p0, b, c});
        cost.push_back((double)std::min<int64_t>(P, in.s_end - p0) * (double)(chunk_cnt[c] + 64));
      }
  }
  std::vector<size_t> order(items.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  std::vector<BatchItem> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];

  p->segs = segs;
  p->chunk_seg_off = chunk_seg_off;
  p->batch_items = (int32_t)sorted.size();
  p->batch_ctas = (int)ctas;
  int64_t bytes = 0;
  cudaError_t e;
  if ((e = upload_vec(&p->d.segs, segs, &bytes)) != cudaSuccess) return cuda_status(e, "batch tables");
  if ((e = upload_vec(&p->d.chunk_seg_off, chunk_seg_off, &bytes)) != cudaSuccess) return cuda_status(e, "batch tables");
  if ((e = upload_vec(&p->d.batch_inst, binst, &bytes)) != cudaSuccess) return cuda_status(e, "batch tables");
  if ((e = upload_vec(&p->d.batch_items, sorted, &bytes)) != cudaSuccess) return cuda_status(e, "batch tables");
  if (p->d.partial) cudaFree(p->d.partial);
  p->d.partial = nullptr;
  if (part > 0) {
    if ((e = cudaMalloc(&p->d.partial, (size_t)part * sizeof(float2))) != cudaSuccess)
      return cuda_status(e, "batch partials");
    bytes += part * (int64_t)sizeof(float2);
  }
  if (!p->d.counter) {
    if ((e = cudaMalloc(&p->d.counter, sizeof(int))) != cudaSuccess) return cuda_status(e, "counter");
    bytes += sizeof(int);
  }
  p->tiling_bytes = bytes;
  p->batch_has_split = part > 0;
  // a tiling change invalidates a captured graph
  if (p->graph_exec) {
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  return SCATTER_OK;
}

// Counter reset, persistent kernel and (for split instances) the reduction,
// on prepared slots.
scatter_status enqueue_batch_kernels(scatter_plan_t p, float2* amp, float* inten, cudaStream_t st) {
  BatchArgs a{};
  a.atom4 = p->d.atom4;
  a.atom_lo = p->d.atom_lo;
  a.atom_w = p->d.atom_w;
  a.segs = p->d.segs;
  a.chunk_seg_off = p->d.chunk_seg_off;
  a.coef = p->d.coef;
  a.ftab = p->d.ftab;
  a.s_hi = p->d.s_hi;
  a.s_lo = p->d.s_lo;
  a.S64 = p->d.S64;
  a.n_s = p->n_s;
  a.inst = p->d.batch_inst;
  a.items = p->d.batch_items;
  a.n_items = p->batch_items;
  a.inst_H = p->d.inst_H;
  a.inst_shift = p->d.inst_shift;
  a.inst_bbox = p->d.inst_bbox;
  for (int d = 0; d < 3; ++d) a.smax[d] = (float)p->s_max[d];
  a.inv4a2 = (float)(1.0 / (4.0 * p->lattice_a * p->lattice_a));
  a.counter = p->d.counter;
  a.partial = p->d.partial;
  a.out_amp = amp;
  a.out_int = inten;
  a.status = p->d.status;
  cudaError_t e = cudaMemsetAsync(p->d.counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_status(e, "counter reset");
  void* fn = pick_batch(p->tiling.R, p->tiling.threads);
  void* args[] = {&a};
  if (p->batch_items > 0) {
    e = cudaLaunchKernel(fn, dim3((unsigned)std::max(1, std::min(p->batch_ctas, p->batch_items))),
                         dim3(p->tiling.threads), args, 0, st);
    if (e != cudaSuccess) return cuda_status(e, "batch kernel launch");
    p->last_launches += 1;
  }
  if (p->batch_has_split) {
    k_batch_reduce<<<(unsigned)((p->n_s + 255) / 256), 256, 0, st>>>(a, p->d.s_inst);
    p->last_launches += 1;
  }
  return cuda_status(cudaGetLastError(), "batch launch");
}

namespace {

scatter_status enqueue_batch(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                             cudaStream_t st) {
  scatter_status s = launch_prep(p, xyz, occ, st);
  if (s != SCATTER_OK) return s;
  return enqueue_batch_kernels(p, amp, inten, st);
}

}  // namespace

scatter_status launch_batch(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                            cudaStream_t st) {
  if (!p->use_graph) {
    timing_begin(p, st);
    scatter_status s = enqueue_batch(p, xyz, occ, amp, inten, st);
    timing_end(p, st);
    return s;
  }
  cudaError_t e;
  const void* key[4] = {xyz, occ, amp, inten};
  bool same = p->graph_exec != nullptr;
  for (int i = 0; i < 4 && same; ++i) same = p->graph_key[i] == key[i];
  if (!same) {
    if (!p->graph_stream) {
      if ((e = cudaStreamCreateWithFlags(&p->graph_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_status(e, "graph stream");
      if ((e = cudaEventCreateWithFlags(&p->graph_in, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_status(e, "graph event");
      if ((e = cudaEventCreateWithFlags(&p->graph_out, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_status(e, "graph event");
    }
    if (p->graph_exec) {
      cudaStreamSynchronize(p->graph_stream);
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(p->graph_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_status(e, "begin capture");
    const int32_t before = p->last_launches;
    scatter_status s = enqueue_batch(p, xyz, occ, amp, inten, p->graph_stream);
    p->graph_launches = p->last_launches - before;
    e = cudaStreamEndCapture(p->graph_stream, &g);
    if (s != SCATTER_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "end capture");
    e = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "graph instantiate");
    for (int i = 0; i < 4; ++i) p->graph_key[i] = key[i];
    p->last_launches = 0;
  }
  if ((e = cudaEventRecord(p->graph_in, st)) != cudaSuccess) return cuda_status(e, "event record");
  if ((e = cudaStreamWaitEvent(p->graph_stream, p->graph_in, 0)) != cudaSuccess) return cuda_status(e, "stream wait");
  timing_begin(p, p->graph_stream);
  if ((e = cudaGraphLaunch(p->graph_exec, p->graph_stream)) != cudaSuccess) return cuda_status(e, "graph launch");
  timing_end(p, p->graph_stream);
  p->last_launches = p->graph_launches;
  if ((e = cudaEventRecord(p->graph_out, p->graph_stream)) != cudaSuccess) return cuda_status(e, "event record");
  if ((e = cudaStreamWaitEvent(st, p->graph_out, 0)) != cudaSuccess) return cuda_status(e, "stream wait");
  return SCATTER_OK;
}

}  // namespace scatter
