// Entry points of libscatter that run on a plan: amplitude, intensity,
// backward / vjp, status check, error model and plan info.
#include <cmath>
#include <cstring>
#include "device_common.cuh"
#include "launch.h"
#include "plan.h"

using namespace scatter;

namespace {

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      ok = false;
      return;
    }
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// A device (or managed) pointer of the plan's device; NULL only if allowed.
scatter_status check_ptr(const void* ptr, int device, const char* name, bool allow_null) {
  if (!ptr) {
    if (allow_null) return SCATTER_OK;
    return fail(SCATTER_ERR_INVALID_ARG, "%s is NULL", name);
  }
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SCATTER_ERR_INVALID_ARG, "%s is not a CUDA pointer", name);
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(SCATTER_ERR_INVALID_ARG, "%s must be device memory", name);
  if (at.device != device)
    return fail(SCATTER_ERR_INVALID_ARG, "%s lives on device %d, the plan on device %d", name, at.device, device);
  return SCATTER_OK;
}

scatter_status check_inputs(scatter_plan_t p, const double* xyz, const float* occ) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  scatter_status st = check_ptr(xyz, p->device, "xyz", p->n_atoms == 0);
  if (st == SCATTER_OK) st = check_ptr(occ, p->device, "occ", true);
  return st;
}

// The launch sequence of a single-instance call: positions prep, the path's
// kernels, their reduction.
scatter_status enqueue_single(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                              cudaStream_t st) {
  scatter_status s = launch_prep(p, xyz, occ, st);
  if (s != SCATTER_OK) return s;
  if (p->path == SCATTER_PATH_SEPARABLE) return launch_separable(p, amp, inten, st);  // GRID and GID_GRID
  return p->s_kind == SCATTER_S_GID_GRID ? launch_dwba(p, amp, inten, st) : launch_generic(p, amp, inten, st);
}

// The same sequence as a CUDA graph, captured on the plan's own stream and
// replayed on the caller's stream: small maps are bound by the launches, not
// the kernels.  A call with new pointer arguments runs eagerly and only
// remembers them; the second call with the same pointers captures, later ones
// replay.  Callers whose buffers change every call never pay for a capture.
scatter_status forward_graphed(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                               cudaStream_t st) {
  const void* key[4] = {xyz, occ, amp, inten};
  bool same = true;
  for (int i = 0; i < 4 && same; ++i) same = p->graph_key[i] == key[i];
  cudaError_t e;
  if (!same) {
    if (p->graph_exec) {  // an in-flight replay is freed when it completes
      cudaGraphExecDestroy(p->graph_exec);
      p->graph_exec = nullptr;
    }
    for (int i = 0; i < 4; ++i) p->graph_key[i] = key[i];
    return enqueue_single(p, xyz, occ, amp, inten, st);
  }
  if (!p->graph_exec) {
    if (!p->graph_stream && (e = cudaStreamCreateWithFlags(&p->graph_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_status(e, "graph stream");
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(p->graph_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_status(e, "begin capture");
    const scatter_status s = enqueue_single(p, xyz, occ, amp, inten, p->graph_stream);
    p->graph_launches = p->last_launches;
    e = cudaStreamEndCapture(p->graph_stream, &g);
    if (s != SCATTER_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_status(e, "end capture");
    e = cudaGraphInstantiate(&p->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_status(e, "graph instantiate");
  }
  if ((e = cudaGraphLaunch(p->graph_exec, st)) != cudaSuccess) return cuda_status(e, "graph launch");
  p->last_launches = p->graph_launches;
  return SCATTER_OK;
}

scatter_status forward(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                       cudaStream_t st) {
  p->last_launches = 0;
  if (p->n_s == 0) return SCATTER_OK;
  const bool gid = p->s_kind == SCATTER_S_GID_GRID;
  if (p->path == SCATTER_PATH_FP64_REF)
    return gid ? launch_f64_gid(p, xyz, occ, amp, inten, st) : launch_f64(p, xyz, occ, amp, inten, st);
  if (p->batch > 1) return launch_batch(p, xyz, occ, amp, inten, st);
  // a timing plan's events bracket the main kernel of every call: it runs eagerly
  return p->use_graph && !p->timing ? forward_graphed(p, xyz, occ, amp, inten, st)
                                    : enqueue_single(p, xyz, occ, amp, inten, st);
}

}  // namespace

extern "C" scatter_status scatter_amplitude(scatter_plan_t p, const double* xyz, const float* occ, void* A_out,
                                            void* stream) {
  scatter_status st = check_inputs(p, xyz, occ);
  if (st != SCATTER_OK) return st;
  if ((st = check_ptr(A_out, p->device, "A_out", p->n_s == 0)) != SCATTER_OK) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  return forward(p, xyz, occ, static_cast<float2*>(A_out), nullptr, static_cast<cudaStream_t>(stream));
}

namespace {

// A host pointer (pinned or pageable); NULL only if allowed.
scatter_status check_host_ptr(const void* ptr, const char* name, bool allow_null) {
  if (!ptr) {
    if (allow_null) return SCATTER_OK;
    return fail(SCATTER_ERR_INVALID_ARG, "%s is NULL", name);
  }
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return SCATTER_OK;  // memory CUDA does not know: pageable host memory
  }
  if (at.type == cudaMemoryTypeDevice) return fail(SCATTER_ERR_INVALID_ARG, "%s must be host memory", name);
  return SCATTER_OK;
}

// Device copies of a host call's buffers, and the copy-out stream and events.
scatter_status ensure_host_staging(scatter_plan_t p, bool with_occ) {
  cudaError_t e;
  auto grow = [&](void** buf, size_t bytes, const char* what) -> scatter_status {
    if (*buf || bytes == 0) return SCATTER_OK;
    if ((e = cudaMalloc(buf, bytes)) != cudaSuccess) return cuda_status(e, what);
    p->base_bytes += (int64_t)bytes;
    return SCATTER_OK;
  };
  scatter_status s;
  if ((s = grow((void**)&p->d.host_xyz, (size_t)p->n_atoms * 3 * sizeof(double), "host-call positions"))) return s;
  if (with_occ && (s = grow((void**)&p->d.host_occ, (size_t)p->n_atoms * sizeof(float), "host-call occupancies")))
    return s;
  if ((s = grow((void**)&p->d.host_amp, (size_t)p->n_s * sizeof(float2), "host-call amplitudes"))) return s;
  if (!p->copy_stream && (e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_status(e, "copy stream");
  for (cudaEvent_t& ev : p->copy_ev)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_status(e, "copy events");
  return SCATTER_OK;
}

}  // namespace

extern "C" scatter_status scatter_amplitude_host(scatter_plan_t p, const double* xyz, const float* occ, void* A_out,
                                                 void* stream) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  scatter_status st = check_host_ptr(xyz, "xyz", p->n_atoms == 0);
  if (st == SCATTER_OK) st = check_host_ptr(occ, "occ", true);
  if (st == SCATTER_OK) st = check_host_ptr(A_out, "A_out", p->n_s == 0);
  if (st != SCATTER_OK) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  if ((st = ensure_host_staging(p, occ != nullptr)) != SCATTER_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (p->n_atoms > 0 &&
      (e = cudaMemcpyAsync(p->d.host_xyz, xyz, (size_t)p->n_atoms * 3 * sizeof(double), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return cuda_status(e, "positions to the device");
  if (occ && p->n_atoms > 0 &&
      (e = cudaMemcpyAsync(p->d.host_occ, occ, (size_t)p->n_atoms * sizeof(float), cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return cuda_status(e, "occupancies to the device");
  const float* docc = occ ? p->d.host_occ : nullptr;
  if (p->n_s == 0) return SCATTER_OK;
  // a separable grid copies its map out in row ranges while the rest is
  // reduced (inside launch_separable); other plans copy it after the call
  const bool pieces = p->path == SCATTER_PATH_SEPARABLE && p->s_kind == SCATTER_S_GRID && p->batch == 1;
  if (pieces) {
    p->host_out = A_out;
    p->last_launches = 0;
    st = enqueue_single(p, p->d.host_xyz, docc, p->d.host_amp, nullptr, s);
    p->host_out = nullptr;
    return st;
  }
  if ((st = forward(p, p->d.host_xyz, docc, p->d.host_amp, nullptr, s)) != SCATTER_OK) return st;
  if ((e = cudaMemcpyAsync(A_out, p->d.host_amp, (size_t)p->n_s * sizeof(float2), cudaMemcpyDeviceToHost, s)) !=
      cudaSuccess)
    return cuda_status(e, "amplitudes to the host");
  return SCATTER_OK;
}

extern "C" scatter_status scatter_intensity(scatter_plan_t p, const double* xyz, const float* occ, float* I_out,
                                            void* stream) {
  scatter_status st = check_inputs(p, xyz, occ);
  if (st != SCATTER_OK) return st;
  if ((st = check_ptr(I_out, p->device, "I_out", p->n_s == 0)) != SCATTER_OK) return st;
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  return forward(p, xyz, occ, nullptr, I_out, static_cast<cudaStream_t>(stream));
}

extern "C" scatter_status scatter_backward(scatter_plan_t p, const double* xyz, const float* occ, const void* A,
                                           const float* I_obs, double* loss_out, float* dL_dxyz, void* stream) {
  scatter_status st = check_inputs(p, xyz, occ);
  if (st != SCATTER_OK) return st;
  if ((st = check_ptr(A, p->device, "A", p->n_s == 0)) != SCATTER_OK) return st;
  if ((st = check_ptr(I_obs, p->device, "I_obs", p->n_s == 0)) != SCATTER_OK) return st;
  if ((st = check_ptr(loss_out, p->device, "loss_out", true)) != SCATTER_OK) return st;
  if ((st = check_ptr(dL_dxyz, p->device, "dL_dxyz", true)) != SCATTER_OK) return st;
  if (p->s_kind == SCATTER_S_GID_GRID) return fail(SCATTER_ERR_UNSUPPORTED, "no backward for GID grids");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  p->last_launches = 0;
  return launch_backward(p, xyz, occ, static_cast<const float2*>(A), I_obs, nullptr, loss_out, dL_dxyz,
                         static_cast<cudaStream_t>(stream));
}

extern "C" scatter_status scatter_vjp(scatter_plan_t p, const double* xyz, const float* occ, const void* G,
                                      float* dL_dxyz, void* stream) {
  scatter_status st = check_inputs(p, xyz, occ);
  if (st != SCATTER_OK) return st;
  if ((st = check_ptr(G, p->device, "G", p->n_s == 0)) != SCATTER_OK) return st;
  if ((st = check_ptr(dL_dxyz, p->device, "dL_dxyz", p->n_atoms == 0)) != SCATTER_OK) return st;
  if (p->s_kind == SCATTER_S_GID_GRID) return fail(SCATTER_ERR_UNSUPPORTED, "no vjp for GID grids");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  p->last_launches = 0;
  return launch_backward(p, xyz, occ, nullptr, nullptr, static_cast<const float2*>(G), nullptr, dL_dxyz,
                         static_cast<cudaStream_t>(stream));
}

namespace {

// Device self-check of the bounded waits: one thread waits for the first
// phase of an mbarrier that nothing arrives at, gives up after `budget`
// cycles and records TIMEOUT in the plan's status word, through the same
// helpers as every pipeline wait of the library.
__global__ void k_wait_selftest(unsigned* status, long long budget) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    dev::mbar_init(&bar, 1);
    dev::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !dev::mbar_wait_bounded(&bar, 0u, budget)) dev::set_status(status, kStatusTimeout);
}

}  // namespace

extern "C" scatter_status scatter_selftest_wait(scatter_plan_t p, void* stream) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard g(p->device);
  if (!g.ok) return fail(SCATTER_ERR_CUDA, "cannot select the plan's device");
  k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(p->d.status, 1LL << 20);
  return cuda_status(cudaGetLastError(), "wait self-check launch");
}

extern "C" scatter_status scatter_check(scatter_plan_t p, void* stream) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  DeviceGuard g(p->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_status(e, "stream synchronize");
  unsigned word = 0;
  if ((e = cudaMemcpy(&word, p->d.status, sizeof(unsigned), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_status(e, "status read");
  if (word) {
    const unsigned zero = 0;
    cudaMemcpy(p->d.status, &zero, sizeof(unsigned), cudaMemcpyHostToDevice);
  }
  if (word & kStatusTimeout) return fail(SCATTER_ERR_TIMEOUT, "a bounded device wait gave up");
  if (word & kStatusNonFinite) return fail(SCATTER_ERR_NUMERIC, "non-finite position or occupancy");
  return SCATTER_OK;
}

extern "C" scatter_status scatter_error_bound(scatter_plan_t p, double radius, double* per_pair,
                                              double* rel_l2_random) {
  if (!p || !per_pair || !rel_l2_random || !(radius >= 0) || !std::isfinite(radius))
    return fail(SCATTER_ERR_INVALID_ARG, "bad argument");
  const double u = std::ldexp(1.0, -24);  // fp32 unit roundoff
  const double pi = 3.14159265358979323846;
  if (p->path == SCATTER_PATH_SEPARABLE) {
    *rel_l2_random = separable_error_model(p, radius, p->tiling.split_k, per_pair);
    return SCATTER_OK;
  }
  if (p->path == SCATTER_PATH_FP64_REF) {
    // FP64 phases |S.r| <= |S| (radius + |t|): bounded by the output rounding
    *per_pair = u;
    *rel_l2_random = u;
    return SCATTER_OK;
  }
  const double sr = (p->s_max[0] + p->s_max[1] + p->s_max[2]) * radius;  // |s . x'|
  const double phi = 0.5 + sr;                                           // |c + s . x'|
  // phase error in cycles: stored s and x' (2 u sr), stored c (u/2), three
  // FMA roundings (3 u phi), 2 pi scaling of the reduced phase (u/2)
  const double dphi = 2.0 * u * sr + 0.5 * u + 3.0 * u * phi + 0.5 * u;
  const double mufu = std::ldexp(1.0, -20);  // sin.approx/cos.approx absolute error bound
  *per_pair = 2.0 * pi * dphi + std::sqrt(2.0) * mufu;
  // blocked FP32 accumulation: tiles of 256 atoms, then tiles summed
  const double per_seg = (double)std::max<int64_t>(p->n_slots, 1) / 256.0;
  const double acc = u * std::sqrt(256.0 + per_seg + (double)p->tiling.split_k);
  *rel_l2_random = *per_pair + acc;
  return SCATTER_OK;
}

extern "C" scatter_status scatter_plan_get_info(scatter_plan_t p, scatter_plan_info* info) {
  if (!p || !info) return fail(SCATTER_ERR_INVALID_ARG, "bad argument");
  std::memset(info, 0, sizeof(*info));
  info->path = p->path;
  info->threads = p->tiling.threads;
  info->points_per_thread = p->tiling.R;
  info->split_k = p->tiling.split_k;
  info->atoms_per_thread = p->tiling.atom_k;
  info->adjoint_form = !p->adj_ready ? 0 : (p->adj_sep ? 3 : (p->adj_line ? 2 : 1));
  info->n_sm = p->n_sm;
  info->n_atoms_padded = p->n_slots;
  info->n_s = p->n_s;
  info->workspace_bytes = p->base_bytes + p->tiling_bytes;
  for (int d = 0; d < 3; ++d) info->center_hkl[d] = p->inst.empty() ? 0.0 : p->inst[0].H[d];
  if (!p->inst.empty()) {
    double t[3] = {0, 0, 0};
    cudaMemcpy(t, p->d.inst_shift, sizeof(t), cudaMemcpyDeviceToHost);
    for (int d = 0; d < 3; ++d) info->shift[d] = t[d];
  }
  return SCATTER_OK;
}

extern "C" scatter_status scatter_plan_timing(scatter_plan_t p, double* ms_main, int32_t* kernel_launches) {
  if (!p || !ms_main || !kernel_launches) return fail(SCATTER_ERR_INVALID_ARG, "bad argument");
  *kernel_launches = p->last_launches;
  *ms_main = 0.0;
  if (!p->timing || !p->timed_call) return fail(SCATTER_ERR_UNSUPPORTED, "timing not enabled or no call made");
  DeviceGuard g(p->device);
  cudaError_t e = cudaEventSynchronize(p->ev_end);
  if (e != cudaSuccess) return cuda_status(e, "event synchronize");
  float ms = 0.f;
  if ((e = cudaEventElapsedTime(&ms, p->ev_begin, p->ev_end)) != cudaSuccess) return cuda_status(e, "elapsed time");
  *ms_main = ms;
  return SCATTER_OK;
}
