// scatter_plan / scatter_plan_destroy: everything that does not depend on
// atom positions (Eq. 2 factored per species, Section 4.2; the atom list cut
// into chunks, the modern form of the paper's atom batching, Section 5).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>
#include "launch.h"
#include "plan.h"
#include "tuner.h"

using scatter::fail;

namespace scatter {
namespace {

bool finite_all(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

bool is_integer(double v) { return std::isfinite(v) && std::fabs(v - std::rint(v)) < 1e-12; }

template <class T>
scatter_status upload(T** dst, const T* src, size_t n, int64_t* bytes) {
  *dst = nullptr;
  if (n == 0) return SCATTER_OK;
  if (injected_alloc_failure()) return fail(SCATTER_ERR_OOM, "injected allocation failure (SCATTER_FAULT)");
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
  *bytes += (int64_t)(n * sizeof(T));
  if (src) {
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e, "cudaMemcpy");
  }
  return SCATTER_OK;
}

template <class T>
void release(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

scatter_status validate(const scatter_problem* pr, const scatter_options* op) {
  if (!pr) return fail(SCATTER_ERR_INVALID_ARG, "problem is NULL");
  if (pr->n_atoms < 0 || pr->n_atoms > (int64_t)INT32_MAX)
    return fail(SCATTER_ERR_INVALID_ARG, "n_atoms out of range (%lld)", (long long)pr->n_atoms);
  if (pr->n_species < 1 || pr->n_species > kMaxSpecies)
    return fail(SCATTER_ERR_INVALID_ARG, "n_species must be in [1, %d]", kMaxSpecies);
  if (!pr->species) return fail(SCATTER_ERR_INVALID_ARG, "species is NULL");
  for (int s = 0; s < pr->n_species; ++s) {
    const scatter_species& sp = pr->species[s];
    if (!finite_all(sp.a, 4) || !finite_all(sp.b, 4) || !std::isfinite(sp.c) || !std::isfinite(sp.fp) ||
        !std::isfinite(sp.fpp) || !std::isfinite(sp.b_dw))
      return fail(SCATTER_ERR_INVALID_ARG, "species %d has non-finite coefficients", s);
  }
  if (pr->atom_species) {
    for (int64_t j = 0; j < pr->n_atoms; ++j)
      if (pr->atom_species[j] < 0 || pr->atom_species[j] >= pr->n_species)
        return fail(SCATTER_ERR_INVALID_ARG, "atom %lld has species %d outside [0, %d)", (long long)j,
                    pr->atom_species[j], pr->n_species);
  }
  if (!(pr->lattice_a > 0) || !std::isfinite(pr->lattice_a))
    return fail(SCATTER_ERR_INVALID_ARG, "lattice_a must be positive and finite");
  if (pr->s_kind < SCATTER_S_LIST || pr->s_kind > SCATTER_S_GID_GRID)
    return fail(SCATTER_ERR_INVALID_ARG, "unknown s_kind %d", pr->s_kind);
  if (pr->s_kind == SCATTER_S_LIST) {
    if (pr->n_s < 0) return fail(SCATTER_ERR_INVALID_ARG, "n_s < 0");
    if (pr->n_s > 0 && !pr->s_list) return fail(SCATTER_ERR_INVALID_ARG, "s_list is NULL");
    if (pr->n_s > 0 && !finite_all(pr->s_list, 3 * pr->n_s))
      return fail(SCATTER_ERR_INVALID_ARG, "s_list has non-finite values");
  } else {
    for (int d = 0; d < 3; ++d) {
      if (pr->n_axis[d] < 1) return fail(SCATTER_ERR_INVALID_ARG, "n_axis[%d] < 1", d);
      if (!pr->axis[d]) return fail(SCATTER_ERR_INVALID_ARG, "axis[%d] is NULL", d);
      if (!finite_all(pr->axis[d], pr->n_axis[d]))
        return fail(SCATTER_ERR_INVALID_ARG, "axis[%d] has non-finite values", d);
    }
    const double m = (double)pr->n_axis[0] * pr->n_axis[1] * pr->n_axis[2];
    if (m > 4e9) return fail(SCATTER_ERR_INVALID_ARG, "grid has too many points");
  }
  if (pr->s_kind == SCATTER_S_GID_GRID) {
    if (!(pr->wavelength > 0) || !std::isfinite(pr->wavelength))
      return fail(SCATTER_ERR_INVALID_ARG, "wavelength must be positive");
    if (!std::isfinite(pr->alpha_i) || !std::isfinite(pr->delta) || !std::isfinite(pr->beta) ||
        pr->delta < 0 || pr->beta < 0)
      return fail(SCATTER_ERR_INVALID_ARG, "invalid alpha_i/delta/beta");
    if (pr->gid_mode != 0 && pr->gid_mode != 1) return fail(SCATTER_ERR_INVALID_ARG, "gid_mode must be 0 or 1");
  }
  if (pr->center_mode != 0 && pr->center_mode != 1)
    return fail(SCATTER_ERR_INVALID_ARG, "center_mode must be 0 or 1");
  if (pr->center_mode == 1)
    for (int d = 0; d < 3; ++d)
      if (!is_integer(pr->center_hkl[d]))
        return fail(SCATTER_ERR_INVALID_ARG, "center_hkl must hold integers");
  if (pr->center_mode == 1 && pr->s_kind == SCATTER_S_GID_GRID && pr->center_hkl[2] != 0.0)
    return fail(SCATTER_ERR_INVALID_ARG, "grazing-incidence maps use H_z = 0");
  if (pr->batch < 1) return fail(SCATTER_ERR_INVALID_ARG, "batch < 1");
  if (pr->batch > 1) {
    if (pr->s_kind != SCATTER_S_LIST) return fail(SCATTER_ERR_INVALID_ARG, "batches need SCATTER_S_LIST");
    if (!pr->atom_off || !pr->s_off) return fail(SCATTER_ERR_INVALID_ARG, "batch offsets are NULL");
    if (pr->atom_off[0] != 0 || pr->s_off[0] != 0 || pr->atom_off[pr->batch] != pr->n_atoms ||
        pr->s_off[pr->batch] != pr->n_s)
      return fail(SCATTER_ERR_INVALID_ARG, "batch offsets must start at 0 and end at n_atoms / n_s");
    for (int b = 0; b < pr->batch; ++b)
      if (pr->atom_off[b + 1] < pr->atom_off[b] || pr->s_off[b + 1] < pr->s_off[b])
        return fail(SCATTER_ERR_INVALID_ARG, "batch offsets must be non-decreasing");
  }
  if (pr->factor_table) {
    if (pr->s_kind == SCATTER_S_GID_GRID)
      return fail(SCATTER_ERR_UNSUPPORTED, "a factor table needs a LIST or GRID plan (one factor per point)");
    const int64_t M = pr->s_kind == SCATTER_S_LIST ? pr->n_s : pr->n_axis[0] * pr->n_axis[1] * pr->n_axis[2];
    for (int64_t i = 0; i < 2 * M * (int64_t)pr->n_species; ++i)
      if (!std::isfinite(pr->factor_table[i]))
        return fail(SCATTER_ERR_INVALID_ARG, "factor_table has non-finite values");
  }
  if (op) {
    if (op->path < SCATTER_PATH_AUTO || op->path > SCATTER_PATH_FP64_REF)
      return fail(SCATTER_ERR_INVALID_ARG, "unknown path %d", op->path);
    if (op->threads < 0 || op->points_per_thread < 0 || op->split_k < 0)
      return fail(SCATTER_ERR_INVALID_ARG, "negative tile override");
  }
  return SCATTER_OK;
}

// Error model of the separable path (the relative L2 error of a map whose
// per-term errors are uncorrelated): tables and formed rows from MUFU sin/cos
// of exactly reduced phases (|error| < 4e-7 = ~7 u each side), f16 hi + lo
// operands with three products (the dropped lo.lo term is below 2^-22 of
// each term), FP32 accumulation in TMEM and in the partials.  `radius`
// bounds |r - t|; *per_pair receives the per-term bound.
}  // namespace

double separable_error_model(const scatter_plan_s* p, double radius, int split, double* per_pair) {
  const double u = std::ldexp(1.0, -24);
  const double pi = 3.14159265358979323846;
  const double sr = (p->s_max[0] + p->s_max[1] + p->s_max[2]) * radius;
  const double pp = 2.0 * pi * u * (2.0 * sr + 2.0) + 4.0 * std::ldexp(1.0, -22) + 14.0 * u;
  if (per_pair) *per_pair = pp;
  const double steps = (double)std::max<int64_t>(p->n_slots, 1) / 16.0;
  return pp + u * std::sqrt(4096.0 + steps / 256.0 + (double)std::max(split, 1));
}

namespace {

// Measured separable map error over the model above: 3.8e-5 against 1.5e-5
// on the strained sphere (134,009 atoms, 256 x 256 x 64), i.e. 2.5; AUTO
// asks the model times this margin to meet the tolerance.
constexpr double kSepModelMargin = 4.0;

// SCATTER_PATH_AUTO on a single GRID or GID_GRID plan (S tables, instances
// and slots prepared): the separable tensor-core path when the grid fills its
// tiles well enough to beat the generic kernel and its error, by the model
// with the measured margin, stays within the caller's tolerance.
bool auto_prefers_separable(const scatter_plan_s* p, const scatter_options* op) {
  if (p->batch != 1 || (p->s_kind != SCATTER_S_GRID && p->s_kind != SCATTER_S_GID_GRID)) return false;
  if (p->gid_mode != 0) return false;  // a buried object: attenuated rows, generic path
  if (p->n_slots % 16) return false;
  const int64_t n0 = p->n_axis[0];
  const int64_t n12 = p->n_axis[1] * (p->s_kind == SCATTER_S_GID_GRID ? 4 * p->n_axis[2] : p->n_axis[2]);
  // B rows are formed once per 16 atoms for 2 x 64 values of the first axis:
  // with fewer than 16 of them, or a few hundred steps of atoms, the
  // formation and the fixed costs dominate
  if (n0 < 16 || p->n_slots < 4096) return false;
  if (n12 < 1024) {
    // less than four 256-point column tiles: only for a large sum, when the
    // contraction (three f16 products on padded 256 x 256 tiles at ~2e15
    // flop/s) and its per-call table (8 B per row and atom slot at ~5e12 B/s)
    // come out at least twice as fast as the generic kernel (~2.3e12 pairs/s)
    const double pairs = (double)p->n_atoms * (double)n0 * (double)n12;
    if (pairs < 1e10) return false;
    const double rows = std::ceil(2.0 * (double)n0 / 256.0) * 256.0, cols = std::ceil((double)n12 / 256.0) * 256.0;
    const double slots = (double)p->n_slots;
    const double sep_s = 6.0 * rows * cols * 2.0 * slots / 2.0e15 + rows * slots * 8.0 / 5.0e12 + 3.0e-5;
    if (2.0 * sep_s > pairs / 2.3e12) return false;
  }
  const double tol = op && op->tolerance > 0.0 ? op->tolerance : 1e-4;
  const double radius = op && op->radius_hint > 0.0
                            ? op->radius_hint
                            : std::cbrt(3.0 * (double)p->n_atoms / (16.0 * 3.14159265358979323846)) + 1.0;
  return separable_error_model(p, radius, 1, nullptr) * kSepModelMargin <= tol;
}

// Reference reflection H of one instance: rint of the mean S (or the given
// center).  S - H is then small, which keeps s . x' small in FP32.
void choose_H(const scatter_problem* pr, int64_t s_begin, int64_t s_end, double H[3]) {
  if (pr->center_mode == 1) {
    for (int d = 0; d < 3; ++d) H[d] = std::rint(pr->center_hkl[d]);
    return;
  }
  for (int d = 0; d < 3; ++d) {
    double sum = 0.0;
    int64_t n = 0;
    if (pr->s_kind == SCATTER_S_LIST) {
      for (int64_t m = s_begin; m < s_end; ++m) sum += pr->s_list[3 * m + d];
      n = s_end - s_begin;
    } else if (pr->s_kind == SCATTER_S_GRID || d < 2) {  // GID: H_z = 0
      for (int64_t i = 0; i < pr->n_axis[d]; ++i) sum += pr->axis[d][i];
      n = pr->n_axis[d];
    }
    H[d] = n > 0 ? std::rint(sum / (double)n) : 0.0;
  }
}

// Splits each instance's slot range into `split_k` contiguous chunks and cuts
// every chunk at species boundaries into segments.
void build_chunks(scatter_plan_s* p, int split_k) {
  p->segs.clear();
  p->chunk_seg_off.assign(1, 0);
  p->chunk_slots.clear();
  for (size_t b = 0; b < p->inst.size(); ++b) {
    const Instance& in = p->inst[b];
    // species segments of this instance
    std::vector<Segment> sp;
    for (const Segment& s : p->all_segs)
      if (s.instance == (int32_t)b) sp.push_back(s);
    const int64_t n = in.slot_end - in.slot_begin;
    int64_t per = (n + split_k - 1) / split_k;
    per = (per + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
    if (per == 0) per = kSlotAlign;
    for (int c = 0; c < split_k; ++c) {
      const int64_t lo = in.slot_begin + c * per, hi = std::min(in.slot_end, lo + per);
      int64_t cnt = 0;
      for (const Segment& s : sp) {
        const int64_t b2 = std::max(lo, s.begin), e2 = std::min(hi, s.end);
        if (b2 < e2) {
          p->segs.push_back(Segment{b2, e2, s.species, s.instance});
          cnt += e2 - b2;
        }
      }
      p->chunk_seg_off.push_back((int32_t)p->segs.size());
      p->chunk_slots.push_back(cnt);
    }
  }
}

}  // namespace

scatter_status apply_tiling(scatter_plan_s* p, const Tiling& t) {
  if (!generic_tiling_supported(t)) return fail(SCATTER_ERR_INVALID_ARG, "unsupported tiling");
  p->tiling = t;
  if (p->graph_exec) {  // a captured call graph holds the old launch shapes
    cudaGraphExecDestroy(p->graph_exec);
    p->graph_exec = nullptr;
  }
  build_chunks(p, t.split_k);
  release(p->d.segs);
  release(p->d.chunk_seg_off);
  release(p->d.partial);
  int64_t bytes = 0;
  scatter_status st = upload(&p->d.segs, p->segs.data(), p->segs.size(), &bytes);
  if (st == SCATTER_OK) st = upload(&p->d.chunk_seg_off, p->chunk_seg_off.data(), p->chunk_seg_off.size(), &bytes);
  const int n_chunks_per_inst = t.split_k;
  if (st == SCATTER_OK && n_chunks_per_inst > 1 && p->n_s > 0)
    st = upload<float2>(&p->d.partial, nullptr, (size_t)n_chunks_per_inst * (size_t)p->n_s, &bytes);
  p->tiling_bytes = bytes;
  if (st == SCATTER_OK && t.atom_k > 0) st = prepare_atompar(p, t.atom_k);
  return st;
}

}  // namespace scatter

using namespace scatter;

extern "C" void scatter_plan_destroy(scatter_plan_t p) {
  if (!p) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  DeviceBuffers& d = p->d;
  release(d.slot_src);
  release(d.slot_inst);
  release(d.atom4);
  release(d.atom_lo);
  release(d.atom_w);
  release(d.atom_species);
  release(d.segs);
  release(d.chunk_seg_off);
  release(d.coef);
  release(d.coef64);
  release(d.atom_off);
  release(d.inst_slot_begin);
  release(d.inst_H);
  release(d.inst_shift);
  release(d.inst_bbox);
  release(d.s_hi);
  release(d.s_lo);
  release(d.S64);
  release(d.s_inst);
  release(d.axis_s);
  release(d.axis_lo);
  release(d.axis64);
  release(d.partial);
  release(d.amp);
  release(d.loss_part);
  release(d.gS);
  release(d.status);
  release(d.gid_sz);
  release(d.gid_sz_lo);
  release(d.gid_sz_im);
  release(d.gid_szf);
  release(d.gid_szf64);
  release(d.gid_sz64_im);
  release(d.gid_sz64);
  release(d.gid_w);
  release(d.gid_w64);
  release(d.ztab);
  release(d.sep_A);
  release(d.sep_partial);
  release(d.sep_chunks);
  release(d.ap_blocks);
  release(d.ftab);
  release(d.ftab64);
  release(d.sep_axis_s);
  release(d.sep_axis_lo);
  release(d.sep_virt);
  release(d.batch_inst);
  release(d.batch_items);
  release(d.counter);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph_stream) cudaStreamDestroy(p->graph_stream);
  if (p->graph_in) cudaEventDestroy(p->graph_in);
  if (p->graph_out) cudaEventDestroy(p->graph_out);
  release(d.adj_blocks);
  release(d.adj_table);
  release(d.adj_partial);
  release(d.adj_gf);
  release(d.adj_sexp);
  release(d.adj_sepA);
  release(d.adj_sep_partial);
  release(d.adj_rec);
  release(d.adj_ntiles);
  release(d.adj_kchunks);
  if (p->ev_begin) cudaEventDestroy(p->ev_begin);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
  release(d.host_xyz);
  release(d.sep_att);
  release(d.sep_szf);
  release(d.host_occ);
  release(d.host_amp);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (cudaEvent_t& e : p->copy_ev)
    if (e) cudaEventDestroy(e);
  if (p->side_stream) cudaStreamDestroy(p->side_stream);
  if (p->side_fork) cudaEventDestroy(p->side_fork);
  if (p->side_join) cudaEventDestroy(p->side_join);
  if (prev >= 0) cudaSetDevice(prev);
  delete p;
}

extern "C" scatter_status scatter_plan(const scatter_problem* pr, const scatter_options* op,
                                       scatter_plan_t* out) {
  if (!out) return fail(SCATTER_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  scatter_status st = validate(pr, op);
  if (st != SCATTER_OK) return st;
  int dev = 0, ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(SCATTER_ERR_NO_DEVICE, "no CUDA device visible");
  }
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_status(e, "cudaGetDevice");

  std::unique_ptr<scatter_plan_s, void (*)(scatter_plan_t)> p(new scatter_plan_s(), scatter_plan_destroy);
  p->device = dev;
  cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
  p->s_kind = (scatter_s_kind)pr->s_kind;
  p->n_atoms = pr->n_atoms;
  p->n_species = pr->n_species;
  p->batch = pr->batch;
  p->lattice_a = pr->lattice_a;
  p->wavelength = pr->wavelength;
  p->alpha_i = pr->alpha_i;
  p->delta = pr->delta;
  p->beta = pr->beta;
  p->gid_mode = pr->s_kind == SCATTER_S_GID_GRID ? pr->gid_mode : 0;
  p->use_graph = !(op && op->use_graph < 0);
  if (op && op->timing) {
    p->timing = true;
    if ((e = cudaEventCreate(&p->ev_begin)) != cudaSuccess) return cuda_status(e, "cudaEventCreate");
    if ((e = cudaEventCreate(&p->ev_end)) != cudaSuccess) return cuda_status(e, "cudaEventCreate");
  }
  scatter_path path = op ? (scatter_path)op->path : SCATTER_PATH_AUTO;
  // AUTO: generic unless the grid test below (once S and the slots are known)
  // picks the separable path
  const bool auto_path = path == SCATTER_PATH_AUTO;
  if (auto_path) path = SCATTER_PATH_GENERIC;
  if (path == SCATTER_PATH_SEPARABLE && (pr->s_kind == SCATTER_S_LIST || pr->batch != 1))
    return fail(SCATTER_ERR_UNSUPPORTED, "the separable path needs a single axis-aligned grid (GRID or GID_GRID)");
  if (pr->batch > 1 && path != SCATTER_PATH_FP64_REF && path != SCATTER_PATH_GENERIC)
    return fail(SCATTER_ERR_UNSUPPORTED, "batches run on the generic path");
  p->path = path;

  // ---- S description --------------------------------------------------------
  if (pr->s_kind == SCATTER_S_LIST) {
    p->n_s = pr->n_s;
  } else {
    for (int d = 0; d < 3; ++d) {
      p->n_axis[d] = pr->n_axis[d];
      p->axis_host[d].assign(pr->axis[d], pr->axis[d] + pr->n_axis[d]);
    }
    p->n_s = pr->n_axis[0] * pr->n_axis[1] * pr->n_axis[2];
  }

  // ---- instances -----------------------------------------------------------------
  const int B = pr->batch;
  p->inst.resize(B);
  for (int b = 0; b < B; ++b) {
    Instance& in = p->inst[b];
    in.atom_begin = B > 1 ? pr->atom_off[b] : 0;
    in.atom_end = B > 1 ? pr->atom_off[b + 1] : pr->n_atoms;
    in.s_begin = B > 1 ? pr->s_off[b] : 0;
    in.s_end = B > 1 ? pr->s_off[b + 1] : p->n_s;
    choose_H(pr, in.s_begin, in.s_end, in.H);
  }

  // ---- species-sorted, padded slots --------------------------------------------
  std::vector<int32_t> slot_src, slot_inst;
  std::vector<int64_t> inst_slot_begin(B);
  for (int b = 0; b < B; ++b) {
    Instance& in = p->inst[b];
    in.slot_begin = (int64_t)slot_src.size();
    inst_slot_begin[b] = in.slot_begin;
    std::vector<std::vector<int32_t>> by(pr->n_species);
    for (int64_t j = in.atom_begin; j < in.atom_end; ++j)
      by[pr->atom_species ? pr->atom_species[j] : 0].push_back((int32_t)j);
    for (int s = 0; s < pr->n_species; ++s) {
      if (by[s].empty()) continue;
      Segment sg;
      sg.begin = (int64_t)slot_src.size();
      for (int32_t j : by[s]) slot_src.push_back(j);
      while (slot_src.size() % kSlotAlign) slot_src.push_back(-1);
      sg.end = (int64_t)slot_src.size();
      sg.species = s;
      sg.instance = b;
      p->all_segs.push_back(sg);
    }
    in.slot_end = (int64_t)slot_src.size();
    slot_inst.resize(slot_src.size(), b);
  }
  p->n_slots = (int64_t)slot_src.size();

  // ---- device tables --------------------------------------------------------------
  int64_t bytes = 0;
  DeviceBuffers& d = p->d;
  std::vector<float> coef32(kNCoef * pr->n_species);
  std::vector<double> coef64(kNCoef * pr->n_species);
  for (int s = 0; s < pr->n_species; ++s) {
    const scatter_species& sp = pr->species[s];
    const double v[kNCoef] = {sp.a[0], sp.a[1], sp.a[2], sp.a[3], sp.b[0], sp.b[1],
                              sp.b[2], sp.b[3], sp.c,    sp.fp,   sp.fpp,  sp.b_dw};
    for (int i = 0; i < kNCoef; ++i) {
      coef64[kNCoef * s + i] = v[i];
      coef32[kNCoef * s + i] = (float)v[i];
    }
  }
  p->coef_host = coef64;
  std::vector<int64_t> atom_off(B + 1);
  std::vector<double> inst_H(3 * B);
  for (int b = 0; b < B; ++b) {
    atom_off[b] = p->inst[b].atom_begin;
    for (int dd = 0; dd < 3; ++dd) inst_H[3 * b + dd] = p->inst[b].H[dd];
  }
  atom_off[B] = pr->n_atoms;
  std::vector<int32_t> species_caller(pr->n_atoms, 0);
  if (pr->atom_species) std::copy(pr->atom_species, pr->atom_species + pr->n_atoms, species_caller.begin());

  if ((st = upload(&d.slot_src, slot_src.data(), slot_src.size(), &bytes))) return st;
  if ((st = upload(&d.slot_inst, slot_inst.data(), slot_inst.size(), &bytes))) return st;
  if ((st = upload<float4>(&d.atom4, nullptr, slot_src.size(), &bytes))) return st;
  if ((st = upload<float4>(&d.atom_lo, nullptr, slot_src.size(), &bytes))) return st;
  if ((st = upload<float>(&d.atom_w, nullptr, slot_src.size(), &bytes))) return st;
  if ((st = upload(&d.atom_species, species_caller.data(), species_caller.size(), &bytes))) return st;
  if ((st = upload(&d.coef, coef32.data(), coef32.size(), &bytes))) return st;
  if ((st = upload(&d.coef64, coef64.data(), coef64.size(), &bytes))) return st;
  if ((st = upload(&d.atom_off, atom_off.data(), atom_off.size(), &bytes))) return st;
  if ((st = upload(&d.inst_slot_begin, inst_slot_begin.data(), inst_slot_begin.size(), &bytes))) return st;
  if ((st = upload(&d.inst_H, inst_H.data(), inst_H.size(), &bytes))) return st;
  if ((st = upload<double>(&d.inst_shift, nullptr, 3 * (size_t)B, &bytes))) return st;
  if ((st = upload<unsigned long long>(&d.inst_bbox, nullptr, 6 * (size_t)B, &bytes))) return st;
  if ((st = upload<unsigned>(&d.status, nullptr, 1, &bytes))) return st;
  if ((e = cudaMemset(d.inst_shift, 0, 3 * sizeof(double) * B)) != cudaSuccess) return cuda_status(e, "memset");
  if ((e = cudaMemset(d.status, 0, sizeof(unsigned))) != cudaSuccess) return cuda_status(e, "memset");
  if (p->n_slots > 0) {
    if ((e = cudaMemset(d.atom4, 0, sizeof(float4) * p->n_slots)) != cudaSuccess) return cuda_status(e, "memset");
    if ((e = cudaMemset(d.atom_lo, 0, sizeof(float4) * p->n_slots)) != cudaSuccess) return cuda_status(e, "memset");
    if ((e = cudaMemset(d.atom_w, 0, sizeof(float) * p->n_slots)) != cudaSuccess) return cuda_status(e, "memset");
  }

  if (pr->s_kind == SCATTER_S_LIST) {
    const int64_t M = p->n_s;
    std::vector<float> s_hi(3 * (size_t)M), s_lo(3 * (size_t)M);
    for (int b = 0; b < B; ++b) {
      const Instance& in = p->inst[b];
      for (int64_t m = in.s_begin; m < in.s_end; ++m)
        for (int dd = 0; dd < 3; ++dd) {
          const double sv = pr->s_list[3 * m + dd] - in.H[dd];
          s_hi[(size_t)dd * M + m] = (float)sv;
          s_lo[(size_t)dd * M + m] = (float)(sv - (double)(float)sv);
        }
    }
    for (int64_t m = 0; m < M; ++m)
      for (int dd = 0; dd < 3; ++dd) p->s_max[dd] = std::max(p->s_max[dd], (double)std::fabs(s_hi[(size_t)dd * M + m]));
    if ((st = upload(&d.s_hi, s_hi.data(), s_hi.size(), &bytes))) return st;
    if ((st = upload(&d.s_lo, s_lo.data(), s_lo.size(), &bytes))) return st;
    if ((st = upload(&d.S64, pr->s_list, 3 * (size_t)M, &bytes))) return st;
    if (B > 1) {
      std::vector<int32_t> s_inst(M);
      for (int b = 0; b < B; ++b)
        for (int64_t m = p->inst[b].s_begin; m < p->inst[b].s_end; ++m) s_inst[m] = b;
      if ((st = upload(&d.s_inst, s_inst.data(), s_inst.size(), &bytes))) return st;
    }
  } else {
    std::vector<float> ax, ax_lo;
    std::vector<double> ax64;
    for (int dd = 0; dd < 3; ++dd)
      for (int64_t i = 0; i < pr->n_axis[dd]; ++i) {
        ax64.push_back(pr->axis[dd][i]);
        const double sv = pr->axis[dd][i] - p->inst[0].H[dd];
        ax.push_back((float)sv);
        ax_lo.push_back((float)(sv - (double)(float)sv));
        if (pr->s_kind == SCATTER_S_GRID || dd < 2)
          p->s_max[dd] = std::max(p->s_max[dd], std::fabs(pr->axis[dd][i] - p->inst[0].H[dd]));
      }
    if ((st = upload(&d.axis_s, ax.data(), ax.size(), &bytes))) return st;
    if ((st = upload(&d.axis_lo, ax_lo.data(), ax_lo.size(), &bytes))) return st;
    if ((st = upload(&d.axis64, ax64.data(), ax64.size(), &bytes))) return st;
  }
  // Eq. 4 factor table (block structure factors), FP32 and FP64 copies
  if (pr->factor_table && p->n_s > 0) {
    const size_t n = (size_t)pr->n_species * (size_t)p->n_s;
    std::vector<float2> t32(n);
    for (size_t i = 0; i < n; ++i)
      t32[i] = make_float2((float)pr->factor_table[2 * i], (float)pr->factor_table[2 * i + 1]);
    if ((st = upload(&d.ftab, t32.data(), n, &bytes))) return st;
    if ((st = upload(&d.ftab64, pr->factor_table, 2 * n, &bytes))) return st;
  }
  // backward workspace (g(S) and per-block loss partials)
  if (p->n_s > 0) {
    if ((st = upload<float2>(&d.amp, nullptr, (size_t)p->n_s, &bytes))) return st;
    if ((st = upload<float2>(&d.gS, nullptr, (size_t)p->n_s, &bytes))) return st;
  }
  if ((st = upload<double>(&d.loss_part, nullptr, kLossParts, &bytes))) return st;
  p->base_bytes = bytes;
  if (pr->s_kind == SCATTER_S_GID_GRID && (st = prepare_gid(p.get()))) return st;
  if (auto_path && auto_prefers_separable(p.get(), op)) {
    path = SCATTER_PATH_SEPARABLE;
    p->path = path;
  }

  // ---- tiling ------------------------------------------------------------------------
  if (path == SCATTER_PATH_SEPARABLE) {
    if ((st = prepare_separable(p.get(), op ? op->split_k : 0))) return st;
  } else if (path == SCATTER_PATH_GENERIC && pr->s_kind == SCATTER_S_GID_GRID) {
    Tiling t;
    t.threads = 256;
    t.R = 4;
    t.split_k = op && op->split_k ? op->split_k : dwba_best_split(p.get());
    if ((st = apply_tiling(p.get(), t))) return st;
  } else if (path == SCATTER_PATH_GENERIC) {
    Tiling t = heuristic_tiling(p.get());
    if (op && op->threads) t.threads = op->threads;
    if (op && op->points_per_thread) t.R = op->points_per_thread;
    if (op && op->split_k) t.split_k = op->split_k;
    if (op && (op->threads || op->points_per_thread || op->split_k || op->atoms_per_thread < 0)) t.atom_k = 0;
    if (op && op->atoms_per_thread > 0) t.atom_k = op->atoms_per_thread;
    if (!generic_tiling_supported(t))
      return fail(SCATTER_ERR_INVALID_ARG, "unsupported tile override (threads=%d R=%d)", t.threads, t.R);
    if ((st = apply_tiling(p.get(), t))) return st;
    if (pr->batch > 1) {
      if ((st = prepare_batch(p.get()))) return st;
      if (op && op->autotune && !(op->threads || op->points_per_thread) &&
          (st = autotune_batch(p.get(), op->tune_cache)))
        return st;
    } else if (op && op->autotune && !(op->threads || op->points_per_thread || op->split_k || op->atoms_per_thread)) {
      if ((st = autotune_generic(p.get(), op->tune_cache))) return st;
    }
  } else {
    Tiling t;
    t.split_k = 1;
    if ((st = apply_tiling(p.get(), t))) return st;
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_status(e, "plan synchronize");
  if (log_enabled())
    fprintf(stderr, "[scatter] plan: path=%d N=%lld slots=%lld M=%lld threads=%d R=%d split_k=%d atom_k=%d\n",
            (int)p->path, (long long)p->n_atoms, (long long)p->n_slots, (long long)p->n_s, p->tiling.threads,
            p->tiling.R, p->tiling.split_k, p->tiling.atom_k);
  *out = p.release();
  return SCATTER_OK;
}
