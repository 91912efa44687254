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
//   kind 8  tcgen05.mma kind::f16, M=128 N=256 K=16, operands in shared
//           memory, FP32 accumulators in TMEM  (dense f16 flop): the peak
//           of the separable path's contraction, one CTA per SM, one thread
//           issuing back-to-back MMAs into two accumulators
//
// Every kernel runs a fixed number of independent dependency chains per thread
// so that latency is hidden; results are written out so nothing is eliminated.

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include "device_common.cuh"
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

// Dense f16 MMA rate: A (128 x 16) and B (256 x 16) zero-filled in the
// canonical no-swizzle K-major layout, `iters` MMAs alternating between two
// 128 x 256 FP32 accumulators, one commit at the end; the issuing thread
// times the loop with clock64 (the MMA queue holds it back to the pipe's
// rate).  A wait that gives up sets out[0] to -1.
constexpr uint32_t kMbTcIdesc = (1u << 4) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint64_t mb_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__global__ void __launch_bounds__(128) ub_tc_kernel(float* out, int iters, long long* cycles) {
  __shared__ __align__(1024) unsigned char sm[4096 + 8192];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x;
  for (int i = tid; i < (4096 + 8192) / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     scatter::dev::smem_addr(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    scatter::dev::mbar_init(&bar, 1);
    scatter::dev::mbar_fence_init();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint64_t a = mb_desc(scatter::dev::smem_addr(sm), 2048, 128);
    const uint64_t b = mb_desc(scatter::dev::smem_addr(sm + 4096), 4096, 128);
    const long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
      const uint32_t d = tmem + (uint32_t)((it & 1) * 256);
      const uint32_t acc = it >= 2 ? 1u : 0u;
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
          "l"(a), "l"(b), "r"(kMbTcIdesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     scatter::dev::smem_addr(&bar))
                 : "memory");
    const bool ok = scatter::dev::mbar_wait_bounded(&bar, 0);
    cycles[blockIdx.x] = clock64() - t0;
    if (!ok) out[0] = -1.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
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
    case 8: return 2.0 * 128 * 256 * 16;  // flop per MMA (per CTA, not per thread)
  }
  return 0.0;
}

}  // namespace

extern "C" scatter_status scatter_microbench(int kind, int iters,
                                             scatter_microbench_result* res) {
  if (!res || kind < 0 || kind > 8 || iters <= 0) return SCATTER_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SCATTER_ERR_NO_DEVICE;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return SCATTER_ERR_CUDA;
  // kind 8: one CTA per SM (each allocates all 512 TMEM columns)
  const int threads = kind == 8 ? 128 : 256;
  const int blocks_per_sm = kind == 8 ? 1 : 4;
  const int blocks = prop.multiProcessorCount * blocks_per_sm;
  float* out = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return SCATTER_ERR_OOM;
  if (cudaMalloc(&cyc, sizeof(long long) * blocks) != cudaSuccess) {
    cudaFree(out);
    return SCATTER_ERR_OOM;
  }
  cudaMemset(out, 0, sizeof(float));  // kind 8 flags a timed-out wait in out[0]
  // kind 8: 120 KB of (unused) dynamic shared memory keeps one CTA per SM
  constexpr int kTcSmem = 120 * 1024;
  if (kind == 8 && cudaFuncSetAttribute(ub_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) !=
                       cudaSuccess) {
    cudaFree(out);
    cudaFree(cyc);
    return SCATTER_ERR_CUDA;
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
      case 8: ub_tc_kernel<<<blocks, threads, kTcSmem>>>(out, n_iter, cyc); break;
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
  float flag = 0.f;
  cudaMemcpy(&flag, out, sizeof(float), cudaMemcpyDeviceToHost);
  long long maxc = 0;
  for (int i = 0; i < blocks; ++i) maxc = hcyc[i] > maxc ? hcyc[i] : maxc;
  delete[] hcyc;
  cudaFree(out);
  cudaFree(cyc);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return SCATTER_ERR_CUDA;
  if (kind == 8 && flag < 0.f) return SCATTER_ERR_TIMEOUT;
  const double total = ops_per_iter(kind) * (double)iters * (kind == 8 ? 1 : threads) * blocks;
  res->seconds = ms * 1e-3;
  res->ops_per_s = total / res->seconds;
  res->ops_per_clk_per_sm =
      total / ((double)maxc * prop.multiProcessorCount);
  res->sm_clock_hz = (double)maxc / res->seconds;
  res->n_sm = prop.multiProcessorCount;
  return SCATTER_OK;
}
