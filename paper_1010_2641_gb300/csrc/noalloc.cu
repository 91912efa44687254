// scatter_amplitude_noalloc: the generic kernel for callers that cannot
// allocate device memory.
//
// Every other entry point works on a plan, and creating a plan allocates
// (cudaMalloc) its tables and workspace.  Some callers cannot do that: code
// that runs while a CUDA stream is being captured into a graph, a host
// process whose device memory is owned by another runtime or pool allocator,
// or a latency-critical loop that must not enter the allocator.  This entry
// point takes only caller-owned inputs and outputs; the generic kernel's
// scratch (call header, atom slots as double-floats, the S split, split-K
// partials, the chunk table) lives in one file-scope __device__ array of fixed size that
// every GPU that loads the library holds until the process exits.
//
// Limits of the scratch (kNoallocBytes = 48 MiB): n_atoms <= 524,288 and
// n_s <= 1,048,576 (larger requests return SCATTER_ERR_INVALID_ARG).
// Calls share the array: calls that overlap on the GPU (two streams, or two
// threads) race on it and must be serialised by the caller.  Each call
// first resets the header it reads (status word, bounding box, |s| maxima)
// and rewrites every other scratch word it reads, so nothing carries over
// between calls.  The first call on a device looks the array up with
// cudaGetSymbolAddress with that device current, which may also load the
// library's device code on that device and reserve the array there; make
// that first call before any stream capture or allocation-free section.
//
// The positions are centred and split as on the plan path (integer centre t
// of the bounding box, c = frac(H . delta)), and crystals whose phases can
// pass 128 cycles take the exact-product phases with s as a double-float.
// Failures cannot be reported through a plan here, so they poison the
// output: if a position, occupancy or S point is not finite, or a bounded
// wait in the kernel gave up, every point of T_out is set to NaN.
#include <cuda_runtime.h>
#include <cmath>
#include <mutex>
#include "device_common.cuh"
#include "generic_impl.cuh"
#include "launch.h"

namespace scatter {

constexpr size_t kNoallocBytes = 48u << 20;
constexpr int64_t kNoallocMaxAtoms = 524288;
constexpr int64_t kNoallocMaxPoints = 1048576;
constexpr int kNoallocR = 8;
constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kNoallocMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Per-call header at the start of the scratch (reset by k_noalloc_init).
struct NoallocHeader {
  unsigned status;                // kStatusNonFinite | kStatusTimeout
  unsigned smax_bits[3];          // max |s_d| as FP32 bits (non-negative floats order as integers)
  unsigned long long bbox[6];     // ordered-int min xyz, max xyz
  int64_t atom_off[2];            // {0, n_atoms}: the atom range of the one instance
  double shift[3];                // integer centring t of this call
};
static_assert(sizeof(NoallocHeader) <= 256, "header fits its 256-byte slot");

// Scratch layout of one call (byte offsets into the array).
struct NoallocLayout {
  size_t header, atom4, atom_lo, atom_w, s_hi, s_lo, coef, segs, chunk_off, partial, end;
};

NoallocLayout layout(int64_t n_slots, int64_t n_s, int split) {
  NoallocLayout L{};
  size_t o = 0;
  L.header = o;    o = align256(o + sizeof(NoallocHeader));
  L.atom4 = o;     o = align256(o + sizeof(float4) * (size_t)n_slots);
  L.atom_lo = o;   o = align256(o + sizeof(float4) * (size_t)n_slots);
  L.atom_w = o;    o = align256(o + sizeof(float) * (size_t)n_slots);
  L.s_hi = o;      o = align256(o + sizeof(float) * 3 * (size_t)n_s);
  L.s_lo = o;      o = align256(o + sizeof(float) * 3 * (size_t)n_s);
  L.coef = o;      o = align256(o + sizeof(float) * kNCoef);
  L.segs = o;      o = align256(o + sizeof(Segment) * (size_t)split);
  L.chunk_off = o; o = align256(o + sizeof(int32_t) * (size_t)(split + 1));
  L.partial = o;   o = align256(o + (split > 1 ? sizeof(float2) * (size_t)split * (size_t)n_s : 0));
  L.end = o;
  return L;
}

// Resets the call header: no status bits, empty bounding box, zero maxima.
__global__ void k_noalloc_init(NoallocHeader* h, int64_t n_atoms) {
  const int i = threadIdx.x;
  if (i == 0) h->status = 0u;
  if (i < 3) h->smax_bits[i] = 0u;
  if (i < 6) h->bbox[i] = i < 3 ? ~0ULL : 0ULL;
  if (i < 2) h->atom_off[i] = i ? n_atoms : 0;
}

// Slots in caller order (one species, f = 1), padded to kSlotAlign with
// zero-weight slots; centred on t = rint of the bounding-box centre:
// x' = r - t, c = frac(H . (x' - rint x')).  Also writes s = S - H as a
// double-float (s_hi + s_lo) with its per-axis maxima, the unit scattering
// factor, t and the chunk table of `split` equal pieces.
__global__ void k_noalloc_prep(const double* __restrict__ xyz, const float* __restrict__ occ, int64_t n_atoms,
                               int64_t n_slots, const double* __restrict__ S, int64_t n_s, double H0, double H1,
                               double H2, int split, NoallocHeader* hdr, float4* atom4, float4* atom_lo,
                               float* atom_w, float* s_hi,
                               float* s_lo, float* coef, Segment* segs, int32_t* chunk_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double t[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const unsigned long long ulo = hdr->bbox[d], uhi = hdr->bbox[3 + d];
    t[d] = (ulo == ~0ULL || uhi == 0ULL) ? 0.0 : rint(0.5 * (dev::unordered(ulo) + dev::unordered(uhi)));
  }
  if (i < n_slots) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), e = a;
    float w = 0.f;
    if (i < n_atoms) {
      const double r0 = xyz[3 * i] - t[0], r1 = xyz[3 * i + 1] - t[1], r2 = xyz[3 * i + 2] - t[2];
      const float wi = occ ? occ[i] : 1.0f;
      if (isfinite(r0) && isfinite(r1) && isfinite(r2) && isfinite(wi)) {
        double c = H0 * (r0 - rint(r0)) + H1 * (r1 - rint(r1)) + H2 * (r2 - rint(r2));
        c -= rint(c);
        a = make_float4((float)r0, (float)r1, (float)r2, (float)c);
        e = make_float4((float)(r0 - (double)a.x), (float)(r1 - (double)a.y), (float)(r2 - (double)a.z), 0.f);
        w = wi;
      } else {
        atomicOr(&hdr->status, kStatusNonFinite);
      }
    }
    atom4[i] = a;
    atom_lo[i] = e;
    atom_w[i] = w;
  }
  if (i < n_s) {
    const double H[3] = {H0, H1, H2};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const double sv = S[3 * i + d] - H[d];
      const float hi = (float)sv;
      s_hi[d * n_s + i] = hi;
      s_lo[d * n_s + i] = (float)(sv - (double)hi);
      if (isfinite(sv))
        atomicMax(&hdr->smax_bits[d], __float_as_uint(fabsf(hi)));
      else
        atomicOr(&hdr->status, kStatusNonFinite);
    }
  }
  if (i == 0) {
    for (int k = 0; k < kNCoef; ++k) coef[k] = k == 8 ? 1.0f : 0.0f;
    for (int d = 0; d < 3; ++d) hdr->shift[d] = t[d];
    const int64_t per = ((n_slots + split - 1) / split + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    int n = 0;
    chunk_off[0] = 0;
    for (int c = 0; c < split; ++c) {
      const int64_t lo = c * per, hi = lo + per < n_slots ? lo + per : n_slots;
      if (lo < hi) segs[n++] = Segment{lo, hi, 0, 0};
      chunk_off[c + 1] = n;
    }
  }
}

// Poisons the whole output when any status bit of the call is set.
__global__ void k_noalloc_finish(const NoallocHeader* __restrict__ hdr, float2* T_out, int64_t n_s) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m < n_s && hdr->status != 0u) T_out[m] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
}

}  // namespace

}  // namespace scatter

using namespace scatter;

extern "C" scatter_status scatter_amplitude_noalloc(int64_t n_atoms, const double* xyz, const float* occ,
                                                    int64_t n_s, const double* S, const double* center_hkl,
                                                    void* T_out, void* stream) {
  if (n_atoms < 0 || n_atoms > kNoallocMaxAtoms)
    return fail(SCATTER_ERR_INVALID_ARG, "n_atoms must be in [0, %lld] for the allocation-free entry point",
                (long long)kNoallocMaxAtoms);
  if (n_s < 0 || n_s > kNoallocMaxPoints)
    return fail(SCATTER_ERR_INVALID_ARG, "n_s must be in [0, %lld] for the allocation-free entry point",
                (long long)kNoallocMaxPoints);
  if (!center_hkl) return fail(SCATTER_ERR_INVALID_ARG, "center_hkl is NULL");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(center_hkl[d]) || std::fabs(center_hkl[d] - std::rint(center_hkl[d])) > 1e-12)
      return fail(SCATTER_ERR_INVALID_ARG, "center_hkl must hold integers");
  if (n_s == 0) return SCATTER_OK;
  if (!S || !T_out || (n_atoms > 0 && !xyz)) return fail(SCATTER_ERR_INVALID_ARG, "NULL input or output");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(SCATTER_ERR_UNSUPPORTED, "device index too large");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(scratch)");
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_noalloc_ptr[dev];
  }

  const int64_t n_slots = (n_atoms + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
  // split-K: enough CTAs for a few waves, as many chunks as the scratch holds
  int sm = 1;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = (n_s + (int64_t)kNoallocThreads * kNoallocR - 1) / ((int64_t)kNoallocThreads * kNoallocR);
  int split = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * sm + tiles - 1) / tiles, 64));
  while (split > 1 && n_slots / split < 256) --split;
  while (split > 1 && layout(n_slots, n_s, split).end > kNoallocBytes) --split;
  const NoallocLayout L = layout(n_slots, n_s, split);
  if (L.end > kNoallocBytes) return fail(SCATTER_ERR_INVALID_ARG, "problem does not fit the 48 MiB scratch");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NoallocHeader* hdr = reinterpret_cast<NoallocHeader*>(base + L.header);
  k_noalloc_init<<<1, 32, 0, st>>>(hdr, n_atoms);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "noalloc init launch");
  if (n_atoms > 0) {
    const scatter_status bs = launch_bbox_raw(xyz, hdr->atom_off, 1, n_atoms, hdr->bbox, &hdr->status, st);
    if (bs != SCATTER_OK) return bs;
  }
  const int64_t n_thr = std::max<int64_t>(std::max<int64_t>(n_slots, n_s), 1);
  k_noalloc_prep<<<(unsigned)((n_thr + 255) / 256), 256, 0, st>>>(
      xyz, occ, n_atoms, n_slots, S, n_s, center_hkl[0], center_hkl[1], center_hkl[2], split, hdr,
      reinterpret_cast<float4*>(base + L.atom4), reinterpret_cast<float4*>(base + L.atom_lo),
      reinterpret_cast<float*>(base + L.atom_w),
      reinterpret_cast<float*>(base + L.s_hi), reinterpret_cast<float*>(base + L.s_lo),
      reinterpret_cast<float*>(base + L.coef), reinterpret_cast<Segment*>(base + L.segs),
      reinterpret_cast<int32_t*>(base + L.chunk_off));
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "noalloc prep launch");

  GenericArgs a{};
  a.atom4 = reinterpret_cast<const float4*>(base + L.atom4);
  a.atom_lo = reinterpret_cast<const float4*>(base + L.atom_lo);
  a.atom_w = reinterpret_cast<const float*>(base + L.atom_w);
  a.segs = reinterpret_cast<const Segment*>(base + L.segs);
  a.chunk_seg_off = reinterpret_cast<const int32_t*>(base + L.chunk_off);
  a.coef = reinterpret_cast<const float*>(base + L.coef);
  a.n_s = n_s;
  a.s_hi = reinterpret_cast<const float*>(base + L.s_hi);
  a.s_lo = reinterpret_cast<const float*>(base + L.s_lo);
  a.S64 = S;
  for (int d = 0; d < 3; ++d) {
    a.H[d] = (float)center_hkl[d];
    a.H64[d] = center_hkl[d];
  }
  a.inv4a2 = 0.0f;  // f == 1 does not depend on |S|
  a.shift = hdr->shift;
  a.bbox = hdr->bbox;
  a.smax_dev = reinterpret_cast<const float*>(hdr->smax_bits);
  a.out_amp = static_cast<float2*>(T_out);
  a.partial = split > 1 ? reinterpret_cast<float2*>(base + L.partial) : nullptr;
  a.status = &hdr->status;
  const scatter_status gs = launch_generic_args(a, kNoallocR, kNoallocThreads, split, st);
  if (gs != SCATTER_OK) return gs;
  k_noalloc_finish<<<(unsigned)((n_s + 255) / 256), 256, 0, st>>>(hdr, static_cast<float2*>(T_out), n_s);
  return cuda_status(cudaGetLastError(), "noalloc finish launch");
}
