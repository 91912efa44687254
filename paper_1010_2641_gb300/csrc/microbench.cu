// Roofline microbenchmarks for the direct scattering sum (Eq. 2).
//
// The generic kernel spends, per (atom, reflection) pair, two transcendental
// evaluations (sin and cos of 2*pi*phase) on the MUFU/XU pipe and a handful of
// FP32 multiply-adds on the FMA pipe (the paper counts 8 flop per pair with one
// sincos, Section 2.2).  The roofline of that kernel is therefore set by the
// per-SM issue rates of those two pipes, not by HBM.  These kernels measure the
// rates on the running GPU so that the reported roofline fraction uses a
// measured denominator:
//   kind 0  sin.approx + cos.approx      (MUFU ops)
//   kind 1  ex2.approx                    (MUFU ops)
//   kind 2  fma.rn.f32                    (FP32 FMA lane-ops)
//   kind 3  fma.rn.f32x2                  (FP32 FMA lane-ops, 2 per instruction)
//   kind 4  fma.rn.f64                    (FP64 FMA ops)
//   kind 5  2 MUFU + 7 FFMA per "pair"    (pairs: the generic-kernel mix)
//   kind 6  cvt.rni.f32.f32               (round-to-integer ops)
//   kind 7  cvt.rn.f16x2.f32              (pack ops: 2 floats -> f16x2)
//
// Every kernel runs a fixed number of independent dependency chains per thread
// so that latency is hidden; results are written out so nothing is eliminated.

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include "scatter_internal.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float mufu_sin(float x) {
  float y;
  asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_cos(float x) {
  float y;
  asm volatile("cos.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float frnd(float x) {
  float y;
  asm volatile("cvt.rni.f32.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a,
                                                   unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

template <int KIND>
__global__ void ub_kernel(float* out, int iters, long long* cycles) {
  const float seed = 1e-3f * (threadIdx.x + 1);
  float a[kChains], b[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = seed + 0.01f * i;
    b[i] = seed - 0.01f * i;
  }
  double d[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) d[i] = a[i];
  unsigned long long p[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    asm volatile("mov.b64 %0, {%1,%2};" : "=l"(p[i]) : "f"(a[i]), "f"(b[i]));
  }
  const float m = 0.999f, c0 = 1e-4f;
  unsigned long long m2, c2;
  asm volatile("mov.b64 %0, {%1,%2};" : "=l"(m2) : "f"(m), "f"(m));
  asm volatile("mov.b64 %0, {%1,%2};" : "=l"(c2) : "f"(c0), "f"(c0));

  __syncthreads();
  long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    if (KIND == 0) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        a[i] = mufu_sin(a[i]);
        b[i] = mufu_cos(b[i]);
      }
    } else if (KIND == 1) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        a[i] = mufu_ex2(a[i]);
        b[i] = mufu_ex2(b[i]);
      }
    } else if (KIND == 2) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        a[i] = fmaf(a[i], m, c0);
        b[i] = fmaf(b[i], m, c0);
      }
    } else if (KIND == 3) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) p[i] = fma2(p[i], m2, c2);
#pragma unroll
      for (int i = 0; i < kChains; ++i) p[i] = fma2(p[i], m2, c2);
    } else if (KIND == 4) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) d[i] = fma(d[i], 0.999, 1e-4);
#pragma unroll
      for (int i = 0; i < kChains; ++i) d[i] = fma(d[i], 0.999, 1e-4);
    } else if (KIND == 5) {
      // One generic pair per chain: 2 MUFU, 7 FFMA.
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        float ph = fmaf(a[i], m, c0);
        ph = fmaf(ph, m, c0);
        ph = fmaf(ph, m, c0);
        float s = mufu_sin(ph), c = mufu_cos(ph);
        b[i] = fmaf(s, m, b[i]);
        a[i] = fmaf(c, m, a[i]);
        a[i] = fmaf(a[i], m, c0);
        b[i] = fmaf(b[i], m, c0);
      }
    } else if (KIND == 7) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        uint32_t h;
        asm volatile("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(a[i]), "f"(b[i]));
        a[i] = __uint_as_float(h) + 1.0f;
        asm volatile("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b[i]), "f"(a[i]));
        b[i] = __uint_as_float(h) + 1.0f;
      }
    } else if (KIND == 6) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        a[i] = frnd(a[i]) + 0.3f;
        b[i] = frnd(b[i]) + 0.7f;
      }
    }
  }
  long long t1 = clock64();
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    float lo, hi;
    asm volatile("mov.b64 {%0,%1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[i]));
    acc += a[i] + b[i] + (float)d[i] + lo + hi;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Units of work per thread per iteration for each kind.
double ops_per_iter(int kind) {
  switch (kind) {
    case 0: return 2.0 * kChains;   // MUFU ops
    case 1: return 2.0 * kChains;   // MUFU ops
    case 2: return 2.0 * kChains;   // FFMA lane-ops
    case 3: return 4.0 * kChains;   // 2 x f32x2 per chain = 4 lane-ops
    case 4: return 2.0 * kChains;   // DFMA
    case 5: return 1.0 * kChains;   // generic pairs
    case 6: return 2.0 * kChains;   // FRND
    case 7: return 2.0 * kChains;   // F2F pack
  }
  return 0.0;
}

}  // namespace

extern "C" scatter_status scatter_microbench(int kind, int iters,
                                             scatter_microbench_result* res) {
  if (!res || kind < 0 || kind > 7 || iters <= 0) return SCATTER_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCATTER_ERR_NO_DEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return SCATTER_ERR_CUDA;
  const int threads = 256;
  const int blocks_per_sm = 4;
  const int blocks = prop.multiProcessorCount * blocks_per_sm;
  float* out = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return SCATTER_ERR_OOM;
  if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
    cudaFree(out);
    return SCATTER_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto launch = [&](int n_iter) {
    switch (kind) {
      case 0: ub_kernel<0><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 1: ub_kernel<1><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 2: ub_kernel<2><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 3: ub_kernel<3><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 4: ub_kernel<4><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 5: ub_kernel<5><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 6: ub_kernel<6><<<blocks, threads>>>(out, n_iter, cyc); break;
      case 7: ub_kernel<7><<<blocks, threads>>>(out, n_iter, cyc); break;
    }
  };
  launch(16);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  long long* hcyc = new long long[blocks];
  cudaMemcpy(hcyc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  long long maxc = 0;
  for (int i = 0; i < blocks; ++i) maxc = hcyc[i] > maxc ? hcyc[i] : maxc;
  delete[] hcyc;
  cudaFree(out);
  cudaFree(cyc);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return SCATTER_ERR_CUDA;
  const double total = ops_per_iter(kind) * (double)iters * threads * blocks;
  res->seconds = ms * 1e-3;
  res->ops_per_s = total / res->seconds;
  res->ops_per_clk_per_sm =
      total / ((double)maxc * prop.multiProcessorCount);
  res->sm_clock_hz = (double)maxc / res->seconds;
  res->n_sm = prop.multiProcessorCount;
  return SCATTER_OK;
}
