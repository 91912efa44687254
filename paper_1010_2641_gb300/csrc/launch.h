// Host-side launch functions shared between translation units of libscatter.
#pragma once

#include "plan.h"

namespace scatter {

// Per-call position preparation (all instances): integer centring t of each
// instance (rint of its bounding-box centre), split r - t = n + delta,
// c = frac(H . delta), fp32 slots.  Enqueued on `st`.
scatter_status launch_prep(scatter_plan_t p, const double* xyz, const float* occ, cudaStream_t st);

// Bounding boxes of `batch` instances (ordered-int min / max xyz, atom ranges
// atom_off [batch+1] in device memory) into `bbox` [batch][6], which must hold
// the empty-box values (min slots ~0, max slots 0) beforehand; non-finite
// coordinates set kStatusNonFinite.  For callers that own their buffers.
scatter_status launch_bbox_raw(const double* xyz, const int64_t* atom_off, int batch, int64_t max_atoms,
                               unsigned long long* bbox, unsigned* status, cudaStream_t st);

// A(S) (and/or |A|^2) of every point with the generic FP32/MUFU kernel;
// positions must have been prepared by launch_prep on the same stream.
scatter_status launch_generic(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st);

// Ordered sum of n_chunks partials [chunk][M] (p->d.partial) with the
// translation phase, into the outputs (GenericArgs reduction of forward.cu).
scatter_status launch_generic_reduce(scatter_plan_t p, int n_chunks, float2* amp_out, float* int_out,
                                     cudaStream_t st);

// Atom-parallel form of the generic sum for short S lists (atompar.cu).
bool atompar_applicable(const scatter_plan_s* p);
bool atompar_preferred(const scatter_plan_s* p, const Tiling& s_parallel);
int atompar_choose_k(const scatter_plan_s* p);
scatter_status prepare_atompar(scatter_plan_s* p, int K);
scatter_status launch_atompar(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st);

// Plain FP64 kernel (no prep needed).
scatter_status launch_f64(scatter_plan_t p, const double* xyz, const float* occ, float2* amp_out,
                          float* int_out, cudaStream_t st);

// Loss L (loss_out), and/or gradient dL/dr (grad, caller order) from either
// (A, I_obs) [misfit] or an upstream gradient G [vjp].  Runs prep itself.
scatter_status launch_backward(scatter_plan_t p, const double* xyz, const float* occ, const float2* A,
                               const float* I_obs, const float2* G, double* loss_out, float* grad,
                               cudaStream_t st);

// Tensor-core adjoint on grids of SEPARABLE plans (adjoint_sep.cu).
bool adjoint_sep_applicable(const scatter_plan_s* p);
scatter_status prepare_adjoint_sep(scatter_plan_s* p);
scatter_status launch_adjoint_sep(scatter_plan_t p, float* grad, cudaStream_t st);

// Grazing-incidence (DWBA) path: plan tables, split choice, launches.
scatter_status prepare_gid(scatter_plan_s* p);
int dwba_best_split(const scatter_plan_s* p);
scatter_status launch_dwba(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st);
scatter_status launch_gid_combine(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st);
scatter_status launch_f64_gid(scatter_plan_t p, const double* xyz, const float* occ, float2* amp_out,
                              float* int_out, cudaStream_t st);

// Separable tensor-core path (GRID plans): tables, tiling, launches, and its
// error model (relative L2 of a map with uncorrelated per-term errors).
double separable_error_model(const scatter_plan_s* p, double radius, int split, double* per_pair);
scatter_status prepare_separable(scatter_plan_s* p, int split_override);
scatter_status launch_separable(scatter_plan_t p, float2* amp_out, float* int_out, cudaStream_t st);

// Batched persistent path (batch > 1): work list, launches (graph-captured).
scatter_status prepare_batch(scatter_plan_s* p);
scatter_status launch_batch(scatter_plan_t p, const double* xyz, const float* occ, float2* amp, float* inten,
                            cudaStream_t st);
scatter_status enqueue_batch_kernels(scatter_plan_t p, float2* amp, float* inten, cudaStream_t st);
int batch_blocks_per_sm(int R, int threads);

// Opt-in event timing around the main kernel of a call.
inline void timing_begin(scatter_plan_s* p, cudaStream_t st) {
  if (p->timing) cudaEventRecord(p->ev_begin, st);
}
inline void timing_end(scatter_plan_s* p, cudaStream_t st) {
  if (p->timing) {
    cudaEventRecord(p->ev_end, st);
    p->timed_call = true;
  }
}

// Occupancy-based residency of the generic kernel for a tiling.
int generic_blocks_per_sm(const scatter_plan_s* p, const Tiling& t);
bool generic_tiling_supported(const Tiling& t);
int64_t generic_num_tiles(const scatter_plan_s* p, const Tiling& t);

}  // namespace scatter
