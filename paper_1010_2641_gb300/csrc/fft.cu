// Eq. 5/6: the FFT approximation of the scattered amplitude (Section 2.1).
//
// Every atom is put on the nearest node R_j of a triperiodic grid of step d
// (lattice units) from `origin`, r_j = R_j + u_j, and the factor
// exp(2 i pi (S - H).u_j) is dropped:
//   A(H + q) ~ sum_s f_s(|S|) sum_{j in s} w_j e^{2 i pi H.r_j} e^{2 i pi q.R_j},
// which for q on the grid q = k / (n d) is one discrete Fourier transform per
// species of the node field g_s(R) = sum_{j in s, R_j = R} w_j e^{2 i pi H.r_j}.
// Valid while |(S - H).u_j| << 1 (Eq. 7); the metric max_j sum_d |u_jd|
// max|q_d| is reported with every call.
//
// k_fft_deposit  per atom: node, H.r in FP64 (exact mod 1), atomic add of
//                w e^{2 i pi H.r} into the species grid, Eq. 7 metric
// cuFFT          one batched inverse C2C transform (exp(+2 i pi k.i/n))
// k_fft_post     per output point (fftshifted order): f_s(|S|), the phase
//                e^{2 i pi q.origin} of the grid origin (a product of three
//                per-axis factors tabulated at plan time), sum over species
//
// cuFFT is loaded on first use (dlopen), so the rest of the library does not
// depend on it; without it the calls return SCATTER_ERR_UNSUPPORTED.
#include <cufft.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>
#include "device_common.cuh"
#include "plan.h"

struct scatter_fft_plan_s {
  scatter_fft_problem pr{};
  int device = 0;
  int64_t n_nodes = 0;          // n0 n1 n2
  cufftHandle fft = 0;
  bool have_fft = false;
  float2* grid = nullptr;       // [n_species][n_nodes]
  float* coef = nullptr;        // [n_species][12] FP32 form-factor coefficients
  float2* ophase = nullptr;     // [n0 | n1 | n2] e^{2 i pi q_d o_d} per axis (the origin phase factorises)
  unsigned* stat = nullptr;     // [0] Eq. 7 metric (float bits), [1] atoms outside, [2] bad species
  cudaStream_t last_stream = nullptr;
};

namespace scatter {
namespace {

// ---- cuFFT entry points, resolved at first use ------------------------------
struct CufftApi {
  cufftResult (*plan_many)(cufftHandle*, int, int*, int*, int, int, int*, int, int, cufftType, int) = nullptr;
  cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
  cufftResult (*exec_c2c)(cufftHandle, cufftComplex*, cufftComplex*, int) = nullptr;
  cufftResult (*destroy)(cufftHandle) = nullptr;
  bool ok = false;
};

const CufftApi& cufft_api() {
  static CufftApi api;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libcufft.so.12", "libcufft.so",
#ifdef SCATTER_CUDA_LIBDIR
                           SCATTER_CUDA_LIBDIR "/libcufft.so.12",
#endif
                           nullptr};
    void* h = nullptr;
    for (int i = 0; names[i] && !h; ++i) h = dlopen(names[i], RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    api.plan_many = reinterpret_cast<decltype(api.plan_many)>(dlsym(h, "cufftPlanMany"));
    api.set_stream = reinterpret_cast<decltype(api.set_stream)>(dlsym(h, "cufftSetStream"));
    api.exec_c2c = reinterpret_cast<decltype(api.exec_c2c)>(dlsym(h, "cufftExecC2C"));
    api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "cufftDestroy"));
    api.ok = api.plan_many && api.set_stream && api.exec_c2c && api.destroy;
  });
  return api;
}

__global__ void k_fft_deposit(const double* __restrict__ xyz, const int32_t* __restrict__ species,
                              const float* __restrict__ occ, int64_t n_atoms, int n_species, double H0, double H1,
                              double H2, double step, double o0, double o1, double o2, int64_t n0, int64_t n1,
                              int64_t n2, float q0, float q1, float q2, float2* grid, int64_t n_nodes,
                              unsigned* stat) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_atoms) return;
  const double x = xyz[3 * j], y = xyz[3 * j + 1], z = xyz[3 * j + 2];
  if (!(isfinite(x) && isfinite(y) && isfinite(z))) {
    atomicAdd(&stat[1], 1u);
    return;
  }
  const double fx = (x - o0) / step, fy = (y - o1) / step, fz = (z - o2) / step;
  const double ix = rint(fx), iy = rint(fy), iz = rint(fz);
  // Eq. 7: max over the grid of |q.u_j| = sum_d |u_jd| max|q_d|
  const float m = (float)(fabs(fx - ix) * step) * q0 + (float)(fabs(fy - iy) * step) * q1 +
                  (float)(fabs(fz - iz) * step) * q2;
  atomicMax(&stat[0], __float_as_uint(m));  // non-negative floats order as their bits
  if (ix < 0 || iy < 0 || iz < 0 || ix >= (double)n0 || iy >= (double)n1 || iz >= (double)n2) {
    atomicAdd(&stat[1], 1u);
    return;
  }
  const int s = species ? species[j] : 0;
  if (s < 0 || s >= n_species) {
    atomicAdd(&stat[2], 1u);
    return;
  }
  // w e^{2 i pi H.r}, the phase reduced mod 1 in FP64
  double ph = H0 * x + H1 * y + H2 * z;
  ph -= rint(ph);
  double sn, cs;
  sincospi(2.0 * ph, &sn, &cs);
  const float w = occ ? occ[j] : 1.f;
  float2* cell = grid + (int64_t)s * n_nodes + ((int64_t)ix * n1 + (int64_t)iy) * n2 + (int64_t)iz;
  atomicAdd(&cell->x, w * (float)cs);
  atomicAdd(&cell->y, w * (float)sn);
}

__global__ void k_fft_post(const float2* __restrict__ grid, int n_species, const float* __restrict__ coef,
                           int64_t n0, int64_t n1, int64_t n2, float dq0, float dq1, float dq2, float H0, float H1,
                           float H2, const float2* __restrict__ ophase, float inv4a2, float2* __restrict__ out) {
  const int64_t n_nodes = n0 * n1 * n2;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const int64_t i2 = i % n2, line = i / n2, i1 = line % n1, i0 = line / n1;
  // fftshifted index -> frequency k (most negative first) -> transform bin
  const int64_t k0 = i0 - n0 / 2, k1 = i1 - n1 / 2, k2 = i2 - n2 / 2;
  const int64_t b0 = k0 < 0 ? k0 + n0 : k0, b1 = k1 < 0 ? k1 + n1 : k1, b2 = k2 < 0 ? k2 + n2 : k2;
  const int64_t bin = (b0 * n1 + b1) * n2 + b2;
  // |S| only enters the form factors: FP32 is ample (the FP64 pipe is slow)
  const float Sx = fmaf((float)k0, dq0, H0), Sy = fmaf((float)k1, dq1, H1), Sz = fmaf((float)k2, dq2, H2);
  const float s2 = (Sx * Sx + Sy * Sy + Sz * Sz) * inv4a2;
  // the grid index i counts from `origin`: q.R = q.origin + k.i / n
  const float2 e = dev::cmul(dev::cmul(ophase[i0], ophase[n0 + i1]), ophase[n0 + n1 + i2]);
  float2 v = make_float2(0.f, 0.f);
  for (int s = 0; s < n_species; ++s) {
    const float2 g = grid[(int64_t)s * n_nodes + bin];
    const float2 F = dev::form_factor(coef + kNCoef * s, s2);
    const float2 t = dev::cmul(F, g);
    v.x += t.x;
    v.y += t.y;
  }
  out[i] = dev::cmul(e, v);
}

}  // namespace
}  // namespace scatter

using namespace scatter;

extern "C" {

scatter_status scatter_fft_plan(const scatter_fft_problem* pr, scatter_fft_plan_t* out) {
  if (!out) return fail(SCATTER_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!pr) return fail(SCATTER_ERR_INVALID_ARG, "problem is NULL");
  if (pr->n_atoms < 0) return fail(SCATTER_ERR_INVALID_ARG, "n_atoms < 0");
  if (pr->n_species < 1 || pr->n_species > kMaxSpecies || !pr->species)
    return fail(SCATTER_ERR_INVALID_ARG, "n_species must be in [1, %d] with species given", kMaxSpecies);
  if (!(pr->lattice_a > 0.0) || !std::isfinite(pr->lattice_a))
    return fail(SCATTER_ERR_INVALID_ARG, "lattice_a must be positive and finite");
  if (!(pr->step > 0.0) || !std::isfinite(pr->step)) return fail(SCATTER_ERR_INVALID_ARG, "step must be positive");
  for (int d = 0; d < 3; ++d) {
    if (pr->n[d] < 2 || pr->n[d] > 4096) return fail(SCATTER_ERR_INVALID_ARG, "n[%d] must be in [2, 4096]", d);
    if (!std::isfinite(pr->origin[d]) || !std::isfinite(pr->center_hkl[d]) ||
        pr->center_hkl[d] != std::rint(pr->center_hkl[d]))
      return fail(SCATTER_ERR_INVALID_ARG, "origin must be finite and center_hkl integer");
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    cudaGetLastError();
    return fail(SCATTER_ERR_NO_DEVICE, "no CUDA device");
  }
  const CufftApi& api = cufft_api();
  if (!api.ok) return fail(SCATTER_ERR_UNSUPPORTED, "cuFFT could not be loaded");
  auto p = std::make_unique<scatter_fft_plan_s>();
  p->pr = *pr;
  p->pr.species = nullptr;
  cudaGetDevice(&p->device);
  p->n_nodes = pr->n[0] * pr->n[1] * pr->n[2];
  if ((double)p->n_nodes * pr->n_species * sizeof(float2) > 64.0 * (1ull << 30))
    return fail(SCATTER_ERR_INVALID_ARG, "grid larger than 64 GiB");
  std::vector<float> coef((size_t)kNCoef * pr->n_species);
  for (int s = 0; s < pr->n_species; ++s) {
    const scatter_species& sp = pr->species[s];
    const double v[kNCoef] = {sp.a[0], sp.a[1], sp.a[2], sp.a[3], sp.b[0], sp.b[1],
                              sp.b[2], sp.b[3], sp.c,    sp.fp,   sp.fpp,  sp.b_dw};
    for (int k = 0; k < kNCoef; ++k) {
      if (!std::isfinite(v[k])) return fail(SCATTER_ERR_INVALID_ARG, "species %d has non-finite coefficients", s);
      coef[(size_t)kNCoef * s + k] = (float)v[k];
    }
  }
  cudaError_t e;
  if ((e = cudaMalloc(&p->grid, (size_t)p->n_nodes * pr->n_species * sizeof(float2))) != cudaSuccess)
    return cuda_status(e, "cudaMalloc FFT grid");
  if ((e = cudaMalloc(&p->coef, coef.size() * sizeof(float))) != cudaSuccess) return cuda_status(e, "cudaMalloc");
  if ((e = cudaMalloc(&p->stat, 4 * sizeof(unsigned))) != cudaSuccess) return cuda_status(e, "cudaMalloc");
  if ((e = cudaMemcpy(p->coef, coef.data(), coef.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_status(e, "cudaMemcpy");
  if ((e = cudaMemset(p->stat, 0, 4 * sizeof(unsigned))) != cudaSuccess) return cuda_status(e, "cudaMemset");
  // e^{2 i pi q_d o_d} for every output index of every axis, reduced mod 1 in FP64
  std::vector<float2> oph;
  for (int d = 0; d < 3; ++d)
    for (int64_t i = 0; i < pr->n[d]; ++i) {
      const double q = (double)(i - pr->n[d] / 2) / ((double)pr->n[d] * pr->step);
      double ph = q * pr->origin[d];
      ph -= std::rint(ph);
      oph.push_back(make_float2((float)std::cos(2.0 * M_PI * ph), (float)std::sin(2.0 * M_PI * ph)));
    }
  if ((e = cudaMalloc(&p->ophase, oph.size() * sizeof(float2))) != cudaSuccess) return cuda_status(e, "cudaMalloc");
  if ((e = cudaMemcpy(p->ophase, oph.data(), oph.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_status(e, "cudaMemcpy");
  int dims[3] = {(int)pr->n[0], (int)pr->n[1], (int)pr->n[2]};
  if (api.plan_many(&p->fft, 3, dims, nullptr, 1, (int)p->n_nodes, nullptr, 1, (int)p->n_nodes, CUFFT_C2C,
                    pr->n_species) != CUFFT_SUCCESS)
    return fail(SCATTER_ERR_UNSUPPORTED, "cuFFT plan for %d x %d x %d x %d failed", dims[0], dims[1], dims[2],
                pr->n_species);
  p->have_fft = true;
  *out = p.release();
  return SCATTER_OK;
}

scatter_status scatter_fft_amplitude(scatter_fft_plan_t p, const double* xyz, const int32_t* atom_species,
                                     const float* occ, void* A_out, void* stream) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  if (!A_out || (p->pr.n_atoms > 0 && !xyz)) return fail(SCATTER_ERR_INVALID_ARG, "NULL buffer");
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != p->device) cudaSetDevice(p->device);
  const CufftApi& api = cufft_api();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last_stream = st;
  const scatter_fft_problem& pr = p->pr;
  const int64_t N = p->n_nodes;
  cudaMemsetAsync(p->grid, 0, (size_t)N * pr.n_species * sizeof(float2), st);
  cudaMemsetAsync(p->stat, 0, 4 * sizeof(unsigned), st);
  // max |q_d| over the output grid: the most negative frequency, n/2 bins
  const float q0 = (float)((double)(pr.n[0] / 2) / ((double)pr.n[0] * pr.step));
  const float q1 = (float)((double)(pr.n[1] / 2) / ((double)pr.n[1] * pr.step));
  const float q2 = (float)((double)(pr.n[2] / 2) / ((double)pr.n[2] * pr.step));
  if (pr.n_atoms > 0)
    k_fft_deposit<<<(unsigned)((pr.n_atoms + 255) / 256), 256, 0, st>>>(
        xyz, atom_species, occ, pr.n_atoms, pr.n_species, pr.center_hkl[0], pr.center_hkl[1], pr.center_hkl[2],
        pr.step, pr.origin[0], pr.origin[1], pr.origin[2], pr.n[0], pr.n[1], pr.n[2], q0, q1, q2, p->grid, N,
        p->stat);
  if (api.set_stream(p->fft, st) != CUFFT_SUCCESS ||
      api.exec_c2c(p->fft, reinterpret_cast<cufftComplex*>(p->grid), reinterpret_cast<cufftComplex*>(p->grid),
                   CUFFT_INVERSE) != CUFFT_SUCCESS) {
    if (cur != p->device) cudaSetDevice(cur);
    return fail(SCATTER_ERR_CUDA, "cuFFT execution failed");
  }
  k_fft_post<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(
      p->grid, pr.n_species, p->coef, pr.n[0], pr.n[1], pr.n[2], (float)(1.0 / ((double)pr.n[0] * pr.step)),
      (float)(1.0 / ((double)pr.n[1] * pr.step)), (float)(1.0 / ((double)pr.n[2] * pr.step)), (float)pr.center_hkl[0],
      (float)pr.center_hkl[1], (float)pr.center_hkl[2], p->ophase, (float)(1.0 / (4.0 * pr.lattice_a * pr.lattice_a)),
      static_cast<float2*>(A_out));
  const scatter_status s = cuda_status(cudaGetLastError(), "FFT approximation launch");
  if (cur != p->device) cudaSetDevice(cur);
  return s;
}

scatter_status scatter_fft_validity(scatter_fft_plan_t p, double* max_qu, int64_t* n_outside) {
  if (!p) return fail(SCATTER_ERR_INVALID_ARG, "plan is NULL");
  unsigned h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaStreamSynchronize(p->last_stream);
  if (e == cudaSuccess) e = cudaMemcpy(h, p->stat, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "FFT validity readback");
  float m;
  std::memcpy(&m, &h[0], sizeof(float));
  if (max_qu) *max_qu = (double)m;
  if (n_outside) *n_outside = (int64_t)h[1];
  if (h[2]) return fail(SCATTER_ERR_INVALID_ARG, "%u atoms had a species index outside [0, %d)", h[2],
                        p->pr.n_species);
  return SCATTER_OK;
}

void scatter_fft_plan_destroy(scatter_fft_plan_t p) {
  if (!p) return;
  if (p->have_fft) cufft_api().destroy(p->fft);
  cudaFree(p->grid);
  cudaFree(p->coef);
  cudaFree(p->stat);
  cudaFree(p->ophase);
  delete p;
}

}  // extern "C"
