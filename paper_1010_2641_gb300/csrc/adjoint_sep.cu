// Adjoint of Eq. 2 on axis-aligned grids, on the tensor cores.
//
// With gF_s(S) = g(S) f_s(|S|) e^{2 i pi s.t} (k_loss_weights) the gradient is
//   dL/dr_j = -2 pi w_j sum_S S Im( gF_s(S) e^{2 i pi (c_j + s.x'_j)} ).
// On a grid s = (s_a, s_b, s_c) the exponential separates as in the forward.
// Define, for the weights omega_0 = 1, omega_1 = s_b, omega_2 = s_c,
//   U_w[a, j] = sum_{(b,c)} gF_s[a,b,c] omega_w(b,c) e^{2 i pi (s_b y'_j + s_c z'_j)}
// a complex matrix product of (a, w) rows by atom columns over the n1 n2
// points of each a-plane.  Every sum the gradient needs is then a short sum
// over a with E[a, j] = e^{2 i pi s_a x'_j}:
//   V = sum_a E U_0,  W_a = sum_a s_a E U_0,  W_b = sum_a E U_1,  W_c = sum_a E U_2
//   dL/dr_j,d = -2 pi w_j Im( e^{2 i pi c_j} (H_d V + W_d) ).
// The product runs on k_sep with the operands' roles swapped: A holds gF
// omega (f16 hi/lo, rows 2 pa + {Re, Im} for pa = w n0 + a, K = points),
// B is formed per step from the columns' atoms (y', z') and the step's 16
// point records (s_b, s_c).  gF spans many decades across a map, so every
// A row is scaled by a power of two that puts its largest element near
// 2^14 (f16 keeps 22 bits of it in hi + lo down to 2^-17 of the row's
// maximum); the epilogue undoes the scale exactly.
//
// k_adj_sep_scale  per (species, a): the exponents of the three rows' scales
// k_adj_sep_tab    A blocks of every species in the tcgen05 no-swizzle layout
// k_sep            U for every (M-tile pair, 256-atom tile, point chunk)
// k_adj_sep_final  per atom: the sum over a and the chunks, gradient
#include <algorithm>
#include <cmath>
#include <vector>
#include "launch.h"
#include "sep_common.cuh"

namespace scatter {

constexpr int kAdjSepRowMax = 14;  // binary exponent of a row's largest |element| after scaling

// One CTA per (species, a): the largest |Re|, |Im| of gF, s_b gF and s_c gF
// over the plane's n1 n2 points, as the exponent e of 2^e >= max (frexp),
// stored as the shift k = e - kAdjSepRowMax of the row's scale 2^k.
__global__ void __launch_bounds__(256) k_adj_sep_scale(const float2* __restrict__ gf, const float* __restrict__ axis_s,
                                                       int64_t n0, int64_t n1, int64_t n2, int64_t n_s,
                                                       int* __restrict__ sexp) {
  const int64_t sp = blockIdx.x / n0, a = blockIdx.x % n0;
  const int64_t nbc = n1 * n2;
  const float2* row = gf + sp * n_s + a * nbc;
  float m0 = 0.f, m1 = 0.f, m2 = 0.f;
  for (int64_t p = threadIdx.x; p < nbc; p += blockDim.x) {
    const float2 v = row[p];
    const float g = fmaxf(fabsf(v.x), fabsf(v.y));
    m0 = fmaxf(m0, g);
    m1 = fmaxf(m1, g * fabsf(axis_s[n0 + p / n2]));
    m2 = fmaxf(m2, g * fabsf(axis_s[n0 + n1 + p % n2]));
  }
  __shared__ float sh[3][8];
  for (int o = 16; o > 0; o >>= 1) {
    m0 = fmaxf(m0, __shfl_xor_sync(0xffffffffu, m0, o));
    m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][warp] = m0;
    sh[1][warp] = m1;
    sh[2][warp] = m2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float m = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmaxf(m, sh[threadIdx.x][q]);
    int e = 0;
    if (m > 0.f && m <= 3.0e38f) frexpf(m, &e);  // zero or non-finite rows: scale 2^-14
    sexp[(sp * 3 + threadIdx.x) * n0 + a] = e - kAdjSepRowMax;
  }
}

struct AdjSepTabArgs {
  const float2* gf;     // [n_species][M] gF_s, M = n0 n1 n2 row-major
  const float* axis_s;  // [n0 | n1 | n2] s = axis - H
  const int* sexp;      // [n_species][3][n0] row scale exponents
  int64_t n0, n1, n2, n_s;
  int64_t n_ksteps, n_mt, n_mp;
  int64_t total;        // threads: n_species x n_mt x n_ksteps x 512
  uint4* A;             // [species][n_mp][n_ksteps][2 tiles][hi|lo][4 kb][16 mg][8 rows] of 16 B
};

// One thread per 16-byte row of a core matrix (4 points x Re/Im of one A row).
// Row 2 pa: (Gr, -Gi); row 2 pa + 1: (Gi, Gr) with G = gF omega_w 2^-k.
__global__ void k_adj_sep_tab(const AdjSepTabArgs t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= t.total) return;
  const int r = (int)(i % 8), mg = (int)((i / 8) % 16), kb = (int)((i / 128) % 4);
  const int64_t ks = (i / 512) % t.n_ksteps, mt = (i / (512 * t.n_ksteps)) % t.n_mt;
  const int64_t sp = i / (512 * t.n_ksteps * t.n_mt);
  const int64_t m = mt * kSepM + mg * 8 + r;
  const int64_t pa = m >> 1;
  const int ri = (int)(m & 1);
  const int64_t nbc = t.n1 * t.n2;
  const bool in_row = pa < 3 * t.n0;
  const int w = in_row ? (int)(pa / t.n0) : 0;
  const int64_t a = in_row ? pa % t.n0 : 0;
  const int k = in_row ? t.sexp[(sp * 3 + w) * t.n0 + a] : 0;
  const float2* row = t.gf + sp * t.n_s + a * nbc;
  float v[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t p = ks * kSepStep + kb * 4 + q;
    float gr = 0.f, gi = 0.f;
    if (in_row && p < nbc) {
      const float2 g = row[p];
      const float om = w == 0 ? 1.f : (w == 1 ? t.axis_s[t.n0 + p / t.n2] : t.axis_s[t.n0 + t.n1 + p % t.n2]);
      gr = ldexpf(g.x * om, -k);
      gi = ldexpf(g.y * om, -k);
    }
    v[2 * q] = ri ? gi : gr;
    v[2 * q + 1] = ri ? gr : -gi;
  }
  uint4 hi, lo;
  split2(v[0], v[1], hi.x, lo.x);
  split2(v[2], v[3], hi.y, lo.y);
  split2(v[4], v[5], hi.z, lo.z);
  split2(v[6], v[7], hi.w, lo.w);
  uint4* blk = t.A + (((sp * t.n_mp + (mt >> 1)) * t.n_ksteps + ks) * kSepPair + (mt & 1)) * (kSepABytes / 16);
  const int64_t off = (int64_t)(kb * 16 + mg) * 8 + r;
  blk[off] = hi;
  blk[512 + off] = lo;
}

struct AdjSepFinalArgs {
  const float* partial;    // [chunk] blocked as sep_part_off: rows 2 (w n0 + a) + {Re, Im}, columns slots
  int64_t chunk_floats, n_cb;
  int n_chunks;
  const Segment* ntiles;
  const int* sexp;
  const float4* atom4;
  const float* atom_w;
  const int32_t* slot_src;
  const float* axis_s;
  int64_t n0, n_slots;
  double H[3];
  float* grad;             // [n_atoms][3] caller order
};

// One thread per atom slot of an N tile: the sum over a (and over the point
// chunks) with FP32 products and double-float (TwoSum) FP32 sums (FP64 runs
// at ~1/75 of the FP32 rate here; the 3 n0 terms are already contracted
// values whose own error is ~1e-6), the row factor e^{2 i pi s_a x'} from
// MUFU sin/cos of the exactly reduced phase (|error| < 4e-7), then the
// rotation by e^{2 i pi c} and the H terms in FP64.  Four values of a per
// iteration keep 24 loads in flight per thread.
__global__ void __launch_bounds__(kSepN) k_adj_sep_final(const AdjSepFinalArgs f) {
  const Segment t = f.ntiles[blockIdx.x];
  const int64_t slot = t.begin + threadIdx.x;
  if (slot >= t.end) return;
  const int32_t src = f.slot_src[slot];
  if (src < 0) return;
  const float4 at = f.atom4[slot];
  const int64_t rows = 3 * f.n0;
  const int* se = f.sexp + (int64_t)t.species * rows;
  dev::DFloatSum V[2], Wd[3][2];
  // the partials' offset of D entry (m, slot) is the column's part plus the
  // row's (sep_part_off): the column part once per thread, and rows 2 r and
  // 2 r + 1 (Re, Im) are neighbours in the same 32-row block, 4 floats apart
  const int64_t col_off = sep_part_off(0, slot, f.n_cb);
  const int64_t row_block = f.n_cb << 10;  // floats per 32-row block
  constexpr int kU = 4;
  for (int64_t a0 = 0; a0 < f.n0; a0 += kU) {
    float U[kU][3][2];
#pragma unroll
    for (int u = 0; u < kU; ++u)
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        U[u][w][0] = U[u][w][1] = 0.f;
        const int64_t a = a0 + u;
        if (a < f.n0) {
          const int64_t m = 2 * (w * f.n0 + a);
          const float* pc = f.partial + col_off + (m >> 5) * row_block + ((m & 31) << 2);
          for (int c = 0; c < f.n_chunks; ++c, pc += f.chunk_floats) {
            U[u][w][0] += pc[0];
            U[u][w][1] += pc[4];
          }
        }
      }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t a = a0 + u;
      if (a >= f.n0) break;
      const float sa = f.axis_s[a];
      float sn, cs;
      dev::sincos_cycles_mufu(dev::frac_of_product(sa, at.x), &sn, &cs);
      float P[3][2];
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        const int k = se[w * f.n0 + a];
        const float re = ldexpf(U[u][w][0], k), im = ldexpf(U[u][w][1], k);
        P[w][0] = fmaf(cs, re, -sn * im);
        P[w][1] = fmaf(cs, im, sn * re);
      }
      V[0].add(P[0][0]);
      V[1].add(P[0][1]);
      Wd[0][0].add(sa * P[0][0]);
      Wd[0][1].add(sa * P[0][1]);
      Wd[1][0].add(P[1][0]);
      Wd[1][1].add(P[1][1]);
      Wd[2][0].add(P[2][0]);
      Wd[2][1].add(P[2][1]);
    }
  }
  double sn, cs;
  sincospi(2.0 * (double)at.w, &sn, &cs);
  const double scale = -2.0 * 3.14159265358979323846 * (double)f.atom_w[slot];
  auto dval = [](const dev::DFloatSum& q) { return (double)q.hi + (double)q.lo; };
  const double vr = dval(V[0]), vi = dval(V[1]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double xr = f.H[d] * vr + dval(Wd[d][0]), xi = f.H[d] * vi + dval(Wd[d][1]);
    f.grad[3 * (int64_t)src + d] = (float)(scale * (cs * xi + sn * xr));  // Im(e^{2 i pi c} X)
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kAdjSepMaxBytes = (size_t)32 << 30;  // A tables + partials; larger maps use the FP32 adjoint

// Point chunks (split over K) that minimise waves x steps per CTA plus the
// cost of one more set of partials (written once, read once).
int adj_sep_split(const scatter_plan_s* p, int64_t tiles, int64_t n_ksteps, size_t part_bytes) {
  const double cap = (double)p->n_sm;
  const double part_steps = 2.0 * (double)part_bytes / 6.0e12 / 1.0e-6;  // ~1 us per step
  double best = 1e300;
  int best_k = 1;
  for (int k = 1; k <= 64; ++k) {
    if (k > 1 && (double)n_ksteps / k < 64) break;
    const double cost = std::ceil((double)tiles * k / cap) * ((double)n_ksteps / k + 40.0) + (k - 1) * part_steps;
    if (cost < best * 0.995) {
      best = cost;
      best_k = k;
    }
  }
  return best_k;
}

}  // namespace

bool adjoint_sep_applicable(const scatter_plan_s* p) {
  return p->path == SCATTER_PATH_SEPARABLE && p->s_kind == SCATTER_S_GRID && p->batch == 1 &&
         p->n_s > 0 && p->n_slots % kSepStep == 0;
}

// Tables and tiling of the tensor-core adjoint; leaves p->adj_sep false (and
// allocates nothing) when the map is too large for its workspace.
scatter_status prepare_adjoint_sep(scatter_plan_s* p) {
  p->adj_sep = false;
  if (!adjoint_sep_applicable(p)) return SCATTER_OK;
  const int64_t n0 = p->n_axis[0], n1 = p->n_axis[1], n2 = p->n_axis[2];
  const int64_t nbc = n1 * n2;
  const int64_t n_ksteps = (nbc + kSepStep - 1) / kSepStep;
  const int64_t n_mt = (2 * 3 * n0 + kSepM - 1) / kSepM;
  const int64_t n_mp = (n_mt + 1) / 2;
  // N tiles: 256 slots of one species
  std::vector<Segment> ntiles;
  for (const Segment& sg : p->all_segs) {
    if (sg.instance != 0) continue;
    for (int64_t b = sg.begin; b < sg.end; b += kSepN)
      ntiles.push_back(Segment{b, std::min(sg.end, b + (int64_t)kSepN), sg.species, 0});
  }
  if (ntiles.empty()) return SCATTER_OK;  // no atoms: the FP32 path writes the empty gradient
  const size_t a_bytes = (size_t)p->n_species * (size_t)n_mp * (size_t)n_ksteps * kSepPair * kSepABytes;
  const size_t part1 = (size_t)sep_part_floats(n_mt, p->n_slots) * sizeof(float);
  const int split = adj_sep_split(p, n_mp * (int64_t)ntiles.size(), n_ksteps, part1);
  std::vector<Segment> chunks;
  const int64_t per = (n_ksteps + split - 1) / split;
  for (int64_t b = 0; b < n_ksteps; b += per)
    chunks.push_back(Segment{b * kSepStep, std::min(n_ksteps, b + per) * kSepStep, 0, 0});
  const size_t part_bytes = chunks.size() * part1;
  if (a_bytes + part_bytes > kAdjSepMaxBytes) return SCATTER_OK;
  if (ntiles.size() * (size_t)n_mp > 0x7fffffffULL || chunks.size() > 65535) return SCATTER_OK;
  // point records (0, s_b, s_c, 0), zero past the last point
  std::vector<float4> rec((size_t)n_ksteps * kSepStep, make_float4(0.f, 0.f, 0.f, 0.f));
  float smax_b = 0.f, smax_c = 0.f;
  for (int64_t q = 0; q < nbc; ++q) {
    const float sb = (float)(p->axis_host[1][q / n2] - p->inst[0].H[1]);
    const float sc = (float)(p->axis_host[2][q % n2] - p->inst[0].H[2]);
    rec[q] = make_float4(0.f, sb, sc, 0.f);
    smax_b = std::max(smax_b, std::fabs(sb));
    smax_c = std::max(smax_c, std::fabs(sc));
  }
  const size_t gf_bytes = (size_t)p->n_species * (size_t)p->n_s * sizeof(float2);
  const size_t sexp_bytes = (size_t)p->n_species * 3 * (size_t)n0 * sizeof(int);
  cudaError_t e;
  if ((e = cudaMalloc(&p->d.adj_gf, gf_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc adjoint gF");
  if ((e = cudaMalloc(&p->d.adj_sexp, sexp_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc row scales");
  if ((e = cudaMalloc(&p->d.adj_sepA, a_bytes)) != cudaSuccess) return cuda_status(e, "cudaMalloc adjoint A");
  if ((e = cudaMemset(p->d.adj_sepA, 0, a_bytes)) != cudaSuccess) return cuda_status(e, "memset adjoint A");
  if ((e = cudaMalloc(&p->d.adj_sep_partial, part_bytes)) != cudaSuccess)
    return cuda_status(e, "cudaMalloc adjoint partials");
  if ((e = cudaMalloc(&p->d.adj_rec, rec.size() * sizeof(float4))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc point records");
  if ((e = cudaMalloc(&p->d.adj_ntiles, ntiles.size() * sizeof(Segment))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc atom tiles");
  if ((e = cudaMalloc(&p->d.adj_kchunks, chunks.size() * sizeof(Segment))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc point chunks");
  if ((e = cudaMemcpy(p->d.adj_rec, rec.data(), rec.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d.adj_ntiles, ntiles.data(), ntiles.size() * sizeof(Segment), cudaMemcpyHostToDevice)) !=
          cudaSuccess ||
      (e = cudaMemcpy(p->d.adj_kchunks, chunks.data(), chunks.size() * sizeof(Segment), cudaMemcpyHostToDevice)) !=
          cudaSuccess)
    return cuda_status(e, "adjoint tables upload");
  if ((e = sep_prepare_kernel()) != cudaSuccess) return cuda_status(e, "separable shared memory attribute");
  if (const scatter_status ss = sep_prepare_side(p, n_mt); ss != SCATTER_OK) return ss;
  p->base_bytes += (int64_t)(gf_bytes + sexp_bytes + a_bytes + part_bytes + rec.size() * sizeof(float4) +
                             (ntiles.size() + chunks.size()) * sizeof(Segment));
  p->adj_sep_ksteps = n_ksteps;
  p->adj_sep_mt = n_mt;
  p->adj_sep_ntiles = (int32_t)ntiles.size();
  p->adj_sep_chunks = (int32_t)chunks.size();
  p->adj_sep_smax[0] = smax_b;
  p->adj_sep_smax[1] = smax_c;
  p->adj_sep = true;
  return SCATTER_OK;
}

// After k_loss_weights wrote gF (p->d.adj_gf): scales, A tables, the
// contraction and the per-atom epilogue, all on `st`.
scatter_status launch_adjoint_sep(scatter_plan_t p, float* grad, cudaStream_t st) {
  const int64_t n0 = p->n_axis[0], n1 = p->n_axis[1], n2 = p->n_axis[2];
  const int64_t n_mp = (p->adj_sep_mt + 1) / 2;
  k_adj_sep_scale<<<(unsigned)(p->n_species * n0), 256, 0, st>>>(p->d.adj_gf, p->d.axis_s, n0, n1, n2, p->n_s,
                                                                  p->d.adj_sexp);
  AdjSepTabArgs t{};
  t.gf = p->d.adj_gf;
  t.axis_s = p->d.axis_s;
  t.sexp = p->d.adj_sexp;
  t.n0 = n0;
  t.n1 = n1;
  t.n2 = n2;
  t.n_s = p->n_s;
  t.n_ksteps = p->adj_sep_ksteps;
  t.n_mt = p->adj_sep_mt;
  t.n_mp = n_mp;
  t.total = (int64_t)p->n_species * p->adj_sep_mt * p->adj_sep_ksteps * 512;
  t.A = static_cast<uint4*>(p->d.adj_sepA);
  k_adj_sep_tab<<<(unsigned)((t.total + 255) / 256), 256, 0, st>>>(t);
  SepArgs a{};
  a.A = static_cast<const uint4*>(p->d.adj_sepA);
  a.a_sp_stride = n_mp * p->adj_sep_ksteps * (int64_t)(kSepPair * kSepABytes / 16);
  a.rec = p->d.adj_rec;
  a.chunks = p->d.adj_kchunks;
  a.ntiles = p->d.adj_ntiles;
  a.atom4 = p->d.atom4;
  a.axis_s = p->d.axis_s;
  a.bbox = p->d.inst_bbox;
  a.shift = p->d.inst_shift;
  a.smax_b = p->adj_sep_smax[0];
  a.smax_c = p->adj_sep_smax[1];
  a.n0 = n0;
  a.n1 = n1;
  a.n2 = n2;
  a.n_cb = (p->n_slots + 31) / 32;
  a.chunk_floats = sep_part_floats(p->adj_sep_mt, p->n_slots);
  a.n_steps = p->adj_sep_ksteps;
  a.n_mt = p->adj_sep_mt;
  a.partial = p->d.adj_sep_partial;
  a.status = p->d.status;
  dim3 grid((unsigned)(n_mp * p->adj_sep_ntiles), (unsigned)p->adj_sep_chunks);
  timing_begin(p, st);
  const cudaError_t le = sep_launch_core(a, grid, st, p->side_stream, p->side_fork, p->side_join);
  timing_end(p, st);
  if (le != cudaSuccess) return cuda_status(le, "adjoint contraction launch");
  AdjSepFinalArgs f{};
  f.partial = p->d.adj_sep_partial;
  f.chunk_floats = sep_part_floats(p->adj_sep_mt, p->n_slots);
  f.n_cb = (p->n_slots + 31) / 32;
  f.n_chunks = p->adj_sep_chunks;
  f.ntiles = p->d.adj_ntiles;
  f.sexp = p->d.adj_sexp;
  f.atom4 = p->d.atom4;
  f.atom_w = p->d.atom_w;
  f.slot_src = p->d.slot_src;
  f.axis_s = p->d.axis_s;
  f.n0 = n0;
  f.n_slots = p->n_slots;
  for (int d = 0; d < 3; ++d) f.H[d] = p->inst[0].H[d];
  f.grad = grad;
  k_adj_sep_final<<<(unsigned)p->adj_sep_ntiles, kSepN, 0, st>>>(f);
  p->last_launches += 3 + sep_core_launches(p->adj_sep_mt);
  return cuda_status(cudaGetLastError(), "adjoint launch");
}

}  // namespace scatter
