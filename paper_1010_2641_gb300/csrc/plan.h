// Internal plan object of libscatter (not part of the public ABI).
//
// Device data layout (all owned by the plan, reused by every call):
//   atoms  : species-sorted, per-instance "slots", each segment of one
//            (instance, species) padded to a multiple of kSlotAlign with
//            zero-weight slots so every tile is full and 16-byte aligned.
//            slot_src[slot]  caller's atom index (or -1 for padding)
//            atom4[slot]     (x', y', z', c) fp32: x' = r - t (lattice units,
//                            t the per-call integer centring of the instance),
//                            c = frac(H . delta) with delta = r - t - rint(r - t)
//            atom_lo[slot]   (x, y, z) - fp32(x', y', z'), 0: the positions as
//                            double-floats for the exact-product phases
//            atom_w[slot]    occupancy (0 for padding)
//   S      : LIST  -> s_hi[3][M] fp32 (s = S - H), s_lo[3][M] its rounding
//                     error, S64[M][3] fp64 (epilogue)
//            GRID  -> axis_s[d][n_d] fp32, axis_lo[d][n_d] its rounding
//                     error, axis64[d][n_d] fp64
//   chunks : split-K partition of each instance's slots into contiguous
//            pieces; a chunk is a list of segments (slot range, species).
#pragma once

#include <cstdint>
#include <vector>
#include "scatter_internal.h"

namespace scatter {

constexpr int kSlotAlign = 32;     // padding granularity of species segments
constexpr int kNCoef = 12;         // a0..a3 b0..b3 c f' f'' B_dw
constexpr int kMaxSpecies = 64;
constexpr int kLossParts = 1024;   // per-block partial sums of the misfit

// Status bits written by kernels into plan->d_status.
enum : unsigned {
  kStatusNonFinite = 1u,
  kStatusTimeout = 2u,
};

struct Segment {
  int64_t begin;    // first slot
  int64_t end;      // one past last slot (multiple of kSlotAlign - begin aligned)
  int32_t species;
  int32_t instance;
};

struct Instance {
  int64_t atom_begin, atom_end;  // caller's atom indices
  int64_t slot_begin, slot_end;  // device slots
  int64_t s_begin, s_end;        // output points
  double H[3];                   // reference reflection (integers)
};

// Atom block of the adjoint kernel (slots of one species segment).
struct AdjBlock {
  int64_t begin;
  int32_t count;
  int32_t species;
};

// Instance and work item of the persistent batched kernel.
struct BatchInst {
  int64_t s_begin, s_end;
  int64_t part_off;  // float2 offset of this instance's partials (split > 1)
  int32_t split;
  int32_t chunk0;
  float H[3];
  float pad;
};

struct BatchItem {
  int64_t p0;        // first S point of the tile
  int32_t inst;
  int32_t chunk;     // chunk index within the instance
};

// Launch shape of the generic kernel.
struct Tiling {
  int threads = 256;
  int R = 8;          // S points per thread
  int split_k = 1;    // atom chunks per S tile
  int atom_k = 0;     // > 0: atom-parallel form, atoms per thread (atompar.cu)
};

// row ranges of a separable map reduced and copied out one after another by
// scatter_amplitude_host (at most one per 32-row block of partials): the
// more ranges, the less of the map's copy is left after the last reduction
constexpr int kHostPieces = 16;

struct DeviceBuffers {
  int32_t* slot_src = nullptr;      // [n_slots]
  int32_t* slot_inst = nullptr;     // [n_slots]
  float4* atom4 = nullptr;          // [n_slots]
  float4* atom_lo = nullptr;        // [n_slots] FP32 rounding errors of (x', y', z'), 0
  float* atom_w = nullptr;          // [n_slots]
  int32_t* atom_species = nullptr;  // [n_atoms] caller order (FP64 kernel)
  Segment* segs = nullptr;          // [n_segs] (chunked)
  int32_t* chunk_seg_off = nullptr; // [n_chunks+1]
  float* coef = nullptr;            // [n_species][12] fp32
  double* coef64 = nullptr;         // [n_species][12] fp64
  int64_t* atom_off = nullptr;      // [batch+1] caller atom ranges
  int64_t* inst_slot_begin = nullptr; // [batch]
  double* inst_H = nullptr;         // [batch][3]
  double* inst_shift = nullptr;     // [batch][3] integer centring t (per call)
  unsigned long long* inst_bbox = nullptr;  // [batch][6] ordered-int min/max
  // S
  float* s_hi = nullptr;            // LIST: [3][M]
  float* s_lo = nullptr;            // LIST: [3][M] s - s_hi (double-float s of the exact-product phases)
  double* S64 = nullptr;            // LIST: [M][3]
  int32_t* s_inst = nullptr;        // LIST batch: instance of each point (or null)
  float* axis_s = nullptr;          // GRID: concatenated axes (s = axis - H)
  float* axis_lo = nullptr;         // GRID: s - axis_s
  double* axis64 = nullptr;         // GRID: concatenated axes (full S)
  // workspace
  float2* partial = nullptr;        // [split_k][M] split-K partials
  float2* amp = nullptr;            // [M] amplitude scratch (intensity, backward)
  double* loss_part = nullptr;      // per-block loss partials
  float2* gS = nullptr;             // [M] adjoint weights g(S)
  unsigned* status = nullptr;       // [1]
  // grazing incidence (GID grids)
  float* gid_sz = nullptr;          // [2][n_af] Sz1, Sz2 r.l.u.
  float* gid_sz_lo = nullptr;       // [2][n_af] their FP32 rounding errors
  float* gid_sz_im = nullptr;       // [2][n_af] Im of a buried object's S_z (0 on the substrate)
  float* gid_szf = nullptr;         // [4][n_af] S_z of each beam's form factor (vacuum)
  double* gid_szf64 = nullptr;      // [4][n_af]
  double* gid_sz64_im = nullptr;    // [n_af] Im sigma of a buried object's beam (0 on the substrate)
  double* gid_sz64 = nullptr;       // [2][n_af]
  float2* gid_w = nullptr;          // [4][n_af] beam weights
  double2* gid_w64 = nullptr;       // [4][n_af]
  float4* ztab = nullptr;           // [n_afb][n_slots][32] Z1, Z2 per call
  // separable path
  void* sep_A = nullptr;            // A operand blocks (f16 hi/lo)
  float* sep_partial = nullptr;     // [chunk][2][sep_ns] planar
  Segment* sep_chunks = nullptr;    // separable atom chunks: one species each, step-aligned slots
  Segment* ap_blocks = nullptr;     // atom-parallel blocks: one species each, <= 256 K slots
  float2* ftab = nullptr;           // Eq. 4 factor table [n_species][M], or null (form factors)
  double* ftab64 = nullptr;         // the same in FP64 (re, im) for the FP64 kernel
  float* sep_axis_s = nullptr;      // separable grid axes, s = axis - H (virtual for GID)
  float* sep_axis_lo = nullptr;     // their FP32 rounding errors
  float2* sep_virt = nullptr;       // GID: map over the virtual (h, k, 4 beams x alpha_f) grid
  // batches
  BatchInst* batch_inst = nullptr;
  BatchItem* batch_items = nullptr;
  int* counter = nullptr;
  // adjoint workspace (allocated on first backward)
  AdjBlock* adj_blocks = nullptr;
  float4* adj_table = nullptr;      // [n_species][M][2], or [n_species][M] in line mode
  float* adj_partial = nullptr;     // [split][n_slots][3]
  // tensor-core adjoint on grids (adjoint_sep.cu)
  float2* adj_gf = nullptr;         // [n_species][M] gF_s
  int* adj_sexp = nullptr;          // [n_species][3][n0] row scale exponents
  void* adj_sepA = nullptr;         // A blocks [species][M-tile pair][point step][2][hi|lo]
  float* adj_sep_partial = nullptr; // [chunk][Re, Im][3 n0][n_slots]
  float4* adj_rec = nullptr;        // point records (0, s_b, s_c, 0), 16 per step
  Segment* adj_ntiles = nullptr;    // 256-slot atom tiles of one species
  Segment* adj_kchunks = nullptr;   // point-step chunks (split over K)
  // scatter_amplitude_host: device copies of the caller's host buffers
  double* host_xyz = nullptr;       // [n_atoms][3]
  float* host_occ = nullptr;        // [n_atoms]
  float2* host_amp = nullptr;       // [n_s]
  // separable path of a buried object: per virtual l column
  float* sep_att = nullptr;         // 2 pi Im(sigma): the formed rows carry exp(-sep_att z')
  float* sep_szf = nullptr;         // S_z of the column's form factor (the vacuum beam S_1)
};

}  // namespace scatter

struct scatter_plan_s {
  int device = 0;
  int n_sm = 0;
  scatter_path path = SCATTER_PATH_GENERIC;
  scatter_s_kind s_kind = SCATTER_S_LIST;
  int64_t n_atoms = 0;
  int64_t n_slots = 0;
  int64_t n_s = 0;
  int32_t n_species = 1;
  int32_t batch = 1;
  double lattice_a = 1.0;
  int64_t n_axis[3] = {0, 0, 0};
  std::vector<double> axis_host[3];
  std::vector<double> coef_host;                 // [n_species][12]
  std::vector<scatter::Instance> inst;
  std::vector<scatter::Segment> all_segs;        // (instance, species) segments
  std::vector<scatter::Segment> segs;            // chunk-major
  std::vector<int32_t> chunk_seg_off;            // [n_chunks+1]
  std::vector<int64_t> chunk_slots;              // slots per chunk (cost)
  scatter::Tiling tiling;
  double wavelength = 0, alpha_i = 0, delta = 0, beta = 0;
  int gid_mode = 0;                              // 0: on the substrate (four beams), 1: buried (one beam)
  scatter::DeviceBuffers d;
  int64_t base_bytes = 0;                        // tables and backward workspace
  int64_t tiling_bytes = 0;                      // chunk tables and split-K partials
  double s_max[3] = {0, 0, 0};                   // max |S - H| per axis (error model)
  bool use_graph = true;
  bool timing = false;
  cudaEvent_t ev_begin = nullptr, ev_end = nullptr;
  bool timed_call = false;
  int32_t last_launches = 0;
  // batches: work list and captured graph
  int32_t batch_items = 0;
  int batch_ctas = 0;
  bool batch_has_split = false;
  cudaGraphExec_t graph_exec = nullptr;
  const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t graph_in = nullptr, graph_out = nullptr;
  int32_t graph_launches = 0;
  int64_t sep_mt = 0, sep_nt = 0, sep_steps = 0;
  int64_t sep_n[3] = {0, 0, 0};                  // separable grid shape (GID: n_h, n_k, 4 n_af)
  int64_t sep_ns = 0;
  int32_t sep_n_chunks = 0;
  bool sep_form_a = false;                       // A formed inside the CTA-pair kernel, no A table
  float sep_smax[2] = {0.f, 0.f};               // max |s| of the separable grid's b and c axes
  int32_t ap_n_blocks = 0;
  int32_t ap_tile = 0;               // reflections per atom-parallel CTA (<= kApPts)
  std::vector<double> gid_sz_host;               // [2][n_af] Sz1, Sz2 (r.l.u.)
  std::vector<double> gid_sz_im_host;            // [n_af] Im sigma of a buried object's beam
  std::vector<double> gid_szf_host;              // [4][n_af] S_z of each beam's form factor
  int32_t sep_beams = 4;                         // beams stacked on the separable l axis (buried: 1)
  bool adj_ready = false;
  int adj_split = 1;
  int adj_blocks = 0;
  int64_t adj_s_per_chunk = 0;
  bool adj_line = false;            // uniform-l grid: k_adjoint_line (phase recurrence)
  float adj_ds = 0.f;               // its l step
  int64_t adj_lines_per_chunk = 0;
  bool adj_sep = false;             // SEPARABLE grid plan: the adjoint runs on k_sep
  int64_t adj_sep_ksteps = 0, adj_sep_mt = 0;
  int32_t adj_sep_ntiles = 0, adj_sep_chunks = 0;
  float adj_sep_smax[2] = {0.f, 0.f};
  // scatter_amplitude_host on a separable grid: the reduction runs in
  // kHostPieces row ranges and each range's copy to the host (destination
  // host_out) starts on copy_stream as soon as the range is reduced
  void* host_out = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[scatter::kHostPieces + 1] = {};
  // separable contractions with an odd M-tile pair count of 3 or more: the
  // last pair's one-CTA kernel runs on side_stream beside the CTA-pair kernel
  cudaStream_t side_stream = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
};
