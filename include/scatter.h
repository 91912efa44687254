/*
 * scatter.h — C ABI of the GB300 direct kinematic scattering library.
 *
 * The library evaluates the kinematic scattered amplitude of an atomistic
 * model (Favre-Nicolin et al., J. Appl. Cryst. 2010, Section 2.1, Eq. 2):
 *
 *     A(S) = sum_j  w_j * f_{s(j)}(|S|) * exp(+2 i pi S . r_j)
 *
 * for every atom j and every point S of reciprocal space, on one NVIDIA GB300
 * (sm_103a) GPU.  Positions r_j are in lattice units and S in reciprocal
 * lattice units (r.l.u.), so S . r_j is a phase in cycles (the convention of
 * the paper's examples, Section 4.1 and 4.2).  w_j is the occupancy of atom j
 * (Section 3: atoms may be given as x,y,z,occ).  f_s is the scattering factor
 * of species s; because it depends on |S| only it is factored out of the sum
 * over the atoms of that species (Section 4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Sign: exp(+2 i pi S . r) (Eq. 2).
 *  - |S| in 1/Angstrom is |S_rlu| / lattice_a (cubic reference lattice) and
 *    the scattering-factor argument is s = sin(theta)/lambda = |S| / 2.
 *  - Complex outputs are interleaved float32 pairs (re, im) — layout-compatible
 *    with C99 `float _Complex` and torch.complex64.
 *  - Reciprocal-space grids are row-major with the first axis slowest:
 *    index = (i0 * n1 + i1) * n2 + i2.  Lists keep the caller's order.
 *  - Device pointers must be allocated on the device that was current when
 *    the plan was created.  Host pointers are read only during the call.
 *  - All work is enqueued on the caller's stream; no call synchronises the
 *    device except scatter_plan (which uploads the problem) and
 *    scatter_check (which reads the kernels' status word).
 *  - No call aborts, traps or prints (unless SCATTER_LOG=1 is set in the
 *    environment).  Every call returns a scatter_status; argument checks run
 *    before anything is launched, and a failed check launches nothing.
 *    scatter_last_error() returns a one-line description of the last failure
 *    on the calling thread.
 */
#ifndef SCATTER_H_
#define SCATTER_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* Status codes                                                             */
/* ------------------------------------------------------------------------ */
typedef enum scatter_status {
  SCATTER_OK = 0,
  SCATTER_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad enum, ...     */
  SCATTER_ERR_UNSUPPORTED = 2,  /* valid request this path cannot serve      */
  SCATTER_ERR_OOM = 3,          /* device or host allocation failed          */
  SCATTER_ERR_CUDA = 4,         /* a CUDA runtime call failed                */
  SCATTER_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up        */
  SCATTER_ERR_NUMERIC = 6,      /* non-finite input detected                 */
  SCATTER_ERR_NO_DEVICE = 7     /* no CUDA device visible                    */
} scatter_status;

/* Kind of reciprocal-space sampling. */
typedef enum scatter_s_kind {
  SCATTER_S_LIST = 0,     /* arbitrary list of S points, [n_s][3] r.l.u.          */
  SCATTER_S_GRID = 1,     /* axis-aligned grid h x k x l (three 1-D axes, r.l.u.) */
  SCATTER_S_GID_GRID = 2  /* grazing incidence: h x k (r.l.u.) x alpha_f (rad)    */
} scatter_s_kind;

/* Kernel family that evaluates the sum. */
typedef enum scatter_path {
  SCATTER_PATH_AUTO = 0,      /* the plan picks (scatter_options.tolerance)      */
  SCATTER_PATH_GENERIC = 1,   /* FP32 + MUFU sincos, split phase reduction        */
  SCATTER_PATH_SEPARABLE = 2, /* axis-factorised contraction on tcgen05 (grids)   */
  SCATTER_PATH_FP64_REF = 3   /* plain FP64 kernel: one thread per S, no tricks   */
} scatter_path;

/* ------------------------------------------------------------------------ */
/* Problem description                                                      */
/* ------------------------------------------------------------------------ */

/*
 * Scattering factor of one species (Section 3, pynx.fthomson; Section 4.2):
 *   f(s) = ( sum_{i<4} a[i] exp(-b[i] s^2) + c + fp + i fpp ) * exp(-b_dw s^2)
 * with s = |S|/2 in 1/Angstrom.  f == 1 is a = {0}, b = {0}, c = 1,
 * fp = fpp = b_dw = 0 (the paper's speed test, Section 2.2, evaluates no f).
 */
typedef struct scatter_species {
  double a[4];
  double b[4];
  double c;
  double fp;    /* f'  (anomalous, real part)      */
  double fpp;   /* f'' (anomalous, imaginary part) */
  double b_dw;  /* Debye-Waller B, Angstrom^2      */
} scatter_species;

/*
 * Everything about a problem except the atom positions and occupancies,
 * which are passed to every call (they change between calls of an
 * optimisation loop; the rest does not).  All arrays are HOST memory and are
 * copied by scatter_plan; the caller may free them afterwards.
 *
 * Batches: batch > 1 describes independent instances b = 0..batch-1 that are
 * computed together in one persistent launch.  Atoms of instance b are
 * [atom_off[b], atom_off[b+1]) of the position array, its S points
 * [s_off[b], s_off[b+1]) of s_list and of the output.  Batches require
 * SCATTER_S_LIST.
 */
typedef struct scatter_problem {
  int64_t n_atoms;                 /* total atoms N (all instances)          */
  int32_t n_species;               /* >= 1                                   */
  const scatter_species* species;  /* [n_species]                            */
  const int32_t* atom_species;     /* [n_atoms] species of each atom, values
                                      in [0, n_species); NULL = all species 0 */
  double lattice_a;                /* Angstrom, > 0                          */

  int32_t s_kind;                  /* scatter_s_kind                         */
  int64_t n_s;                     /* LIST: total number of S points         */
  const double* s_list;            /* LIST: [n_s][3] r.l.u.                  */
  const double* axis[3];           /* GRID: h, k, l (r.l.u.);
                                      GID_GRID: h, k (r.l.u.), alpha_f (rad)  */
  int64_t n_axis[3];

  int32_t center_mode;             /* 0: reference reflection H = rint(mean S)
                                      per instance; 1: use center_hkl         */
  double center_hkl[3];            /* H when center_mode == 1 (integers)     */

  /* GID_GRID only (Section 4.3): wavelength (Angstrom), incidence angle
     (rad), substrate refractive index n = 1 - delta + i beta. */
  double wavelength;
  double alpha_i;
  double delta;
  double beta;

  int32_t batch;                   /* 1, or number of instances               */
  const int64_t* atom_off;         /* [batch+1] when batch > 1, else NULL     */
  const int64_t* s_off;            /* [batch+1] when batch > 1, else NULL     */

  /* Blocks of atoms (Eq. 4): host complex128 [n_species][M] (re, im pairs),
   * M the output points in output order.  When set, the "species" are
   * block types and F_t(S_m) = factor_table[t][m] replaces the Gaussian
   * form factor (the species coefficients are then unused); positions are
   * the displaced block origins.  LIST plans (one instance or a batch:
   * M counts the points of every instance) and GRID plans; the backward
   * and vjp give dL/d(block origin) with F held fixed.  GID_GRID plans
   * reject a table (their four beams each have their own S, so one factor
   * per point does not define the sum).  Copied at plan time.  NULL: the
   * form factors of `species`.                                            */
  const double* factor_table;

  /* GID_GRID only: where the scatterer sits (Section 4.3 names reflection
   * and transmission by the substrate):
   *   0  on the substrate, in vacuum (z >= 0 above the surface plane z = 0):
   *      four beams, direct and reflected in and out, W = (1, R_i, R_f,
   *      R_i R_f);
   *   1  buried in the substrate (z <= 0, lattice units below the surface
   *      plane z = 0; the substrate has no lower interface): one beam
   *      transmitted in and out, W = T_i T_f, refracted and attenuated in
   *      the medium: exp(2 i pi (h x + k y + sigma z)), sigma =
   *      (a / lambda)(conj q_i + conj q_f), q = sqrt(n^2 - cos^2 alpha),
   *      f at the vacuum beam S_1.  Generic and FP64 paths; the separable
   *      path when asked for (SCATTER_PATH_SEPARABLE; AUTO keeps the generic
   *      path): one beam on the virtual l axis, its formed rows carrying
   *      exp(-2 pi Im(sigma) z') of the centred z', which must stay below
   *      e^10 (a call whose crystal is too tall for the attenuation of its
   *      exit angles reports SCATTER_ERR_NUMERIC at scatter_check).        */
  int32_t gid_mode;
} scatter_problem;

/* Plan options.  Zero-initialised options mean "automatic". */
typedef struct scatter_options {
  int32_t path;              /* scatter_path                                  */
  int32_t autotune;          /* 1: time candidate tile shapes at plan time    */
  const char* tune_cache;    /* JSON file the autotuner reads/extends, or NULL */
  int32_t threads;           /* tile override: threads per CTA (0 = auto)     */
  int32_t points_per_thread; /* tile override: S points per thread (0 = auto) */
  int32_t split_k;           /* tile override: atom chunks per S tile (0 = auto) */
  int32_t use_graph;         /* capture a call's launch sequence (prep, main
                                kernels, reduction) in a CUDA graph on first
                                use and replay it while the pointer arguments
                                stay the same (default on: 0 = on, -1 = off);
                                single-instance plans with `timing` and the
                                FP64 path run eagerly                         */
  int32_t timing;            /* 1: record CUDA events around the main kernel
                                of every call (see scatter_plan_timing)       */
  int32_t atoms_per_thread;  /* generic path, one instance: 1, 2, 4, 8 or 16
                                selects the atom-parallel form (threads share
                                the reflections and split the atoms, Section 3)
                                with that many atoms per thread; 0 = chosen by
                                the heuristic / autotuner; -1 = never         */
  double tolerance;          /* SCATTER_PATH_AUTO: the relative L2 error of the
                                map the caller accepts (0 = 1e-4).  A single
                                GRID or GID_GRID plan takes the separable
                                tensor-core path when the grid is large enough
                                for it and its error model, times a margin
                                measured against the oracle, stays within the
                                tolerance; everything else takes the generic
                                FP32 path                                     */
  double radius_hint;        /* SCATTER_PATH_AUTO: bound on |r_j - t| (lattice
                                units, after the integer centring) used by
                                that error model; 0 = a compact crystal of
                                n_atoms at 4 atoms per cell                   */
} scatter_options;

typedef struct scatter_plan_s* scatter_plan_t;

/* Plan summary (for logging and benchmarks). */
typedef struct scatter_plan_info {
  int32_t path;              /* resolved scatter_path                          */
  int32_t threads;
  int32_t points_per_thread;
  int32_t split_k;
  int32_t n_sm;
  int64_t n_atoms_padded;    /* device atom slots incl. zero-weight padding    */
  int64_t n_s;               /* output points                                  */
  int64_t workspace_bytes;   /* device memory owned by the plan                */
  double center_hkl[3];      /* H of instance 0                                */
  double shift[3];           /* integer centring vector t of instance 0        */
  int32_t atoms_per_thread;  /* > 0: the atom-parallel form was chosen        */
  int32_t adjoint_form;      /* form of the gradient kernel, fixed at the first
                              * backward: 0 none yet, 1 FP32 S tiles (lists,
                              * non-uniform grids), 2 FP32 line recurrence
                              * (uniform l axis), 3 tensor-core contraction
                              * (SEPARABLE grid plans)                         */
} scatter_plan_info;

/* ------------------------------------------------------------------------ */
/* Entry points                                                             */
/* ------------------------------------------------------------------------ */

/*
 * scatter_plan — validate a problem and prepare everything that does not
 * depend on atom positions (Eq. 2 factored per species, Section 4.2; batching
 * of the atom list, Section 5).
 *
 *  problem  host, read during the call only.
 *  options  host or NULL (all automatic).
 *  out      receives the plan handle; set to NULL on failure.
 *
 * Work done here: species sort of the atoms (stable, padded to multiples of
 * 32 with zero-weight slots), choice of the reference reflection H and of the
 * S split S = H + s, per-S tables, Fresnel coefficients (GID), workspace
 * allocation, optional autotuning.  Uses the current CUDA device and
 * synchronises it.  Returns INVALID_ARG for inconsistent sizes, NaN/Inf in
 * host inputs or species indices out of range; UNSUPPORTED when a forced path
 * cannot serve the problem (e.g. SEPARABLE on a list); OOM when device memory
 * is short.  The plan owns its device memory until scatter_plan_destroy.
 */
scatter_status scatter_plan(const scatter_problem* problem,
                            const scatter_options* options,
                            scatter_plan_t* out);

/*
 * scatter_amplitude — A(S) of Eq. 2 for every S of the plan.
 *
 *  xyz    device, float64 [n_atoms][3], lattice units, in the caller's atom
 *         order (the order of problem->atom_species).
 *  occ    device, float32 [n_atoms] occupancies w_j, or NULL (all 1).
 *  A_out  device, complex64 [n_s] (interleaved re, im), written in full.
 *  stream CUDA stream (cudaStream_t) or NULL for the legacy default stream.
 *
 * Work is enqueued only.  The plan's workspace is reused by every call, so
 * calls on one plan must not overlap on the GPU (use one stream per plan).
 */
scatter_status scatter_amplitude(scatter_plan_t plan, const double* xyz,
                                 const float* occ, void* A_out, void* stream);

/*
 * scatter_amplitude_host — scatter_amplitude with host buffers, the shape of
 * the paper's own call (Section 3: positions in, amplitudes out, both
 * host arrays).
 *
 *  xyz    host float64 [n_atoms][3], lattice units, caller's atom order.
 *  occ    host float32 [n_atoms] occupancies, or NULL (all 1).
 *  A_out  host complex64 [n_s], written in full once the stream's work
 *         completes (synchronise `stream`, or scatter_check, before reading).
 *  stream CUDA stream or NULL.
 *
 * The plan copies the inputs into device buffers of its own (allocated on
 * the first host call and kept until scatter_plan_destroy: 28 n_atoms + 8 n_s
 * bytes, plus a second stream and 17 events), runs the plan's forward on
 * them and copies the map back.  On a SEPARABLE plan of a GRID the final
 * reduction runs in up to 16 ranges of map rows and each range's copy to the
 * host starts on the plan's second stream as soon as that range is reduced,
 * overlapping the rest of the reduction; `stream` waits for the last copy.
 * Pinned host memory gives asynchronous copies; pageable memory is accepted
 * and then copied synchronously by the driver.  Errors: INVALID_ARG for a
 * NULL or device pointer (a NULL xyz or A_out is allowed only when n_atoms
 * or n_s is 0); OOM when the staging buffers cannot be allocated; the
 * forward's errors otherwise.  Calls on one plan must not overlap.
 */
scatter_status scatter_amplitude_host(scatter_plan_t plan, const double* xyz,
                                      const float* occ, void* A_out, void* stream);

/*
 * scatter_intensity — I(S) = |A(S)|^2 (the quantity of the paper's maps,
 * Section 2.3).  Same inputs as scatter_amplitude; I_out is device float32
 * [n_s].  A is formed in the plan's workspace.
 */
scatter_status scatter_intensity(scatter_plan_t plan, const double* xyz,
                                 const float* occ, float* I_out, void* stream);

/*
 * scatter_backward — misfit L = sum_S (|A(S)|^2 - I_obs(S))^2 and its
 * gradient with respect to every atom position (adjoint of Eq. 2):
 *   dL/dr_j = -2 pi sum_S S * Im( g(S) * w_j f_{s(j)}(|S|) exp(2 i pi S.r_j) )
 *   g(S)    = 4 (|A(S)|^2 - I_obs(S)) conj(A(S))
 * with S the full scattering vector.  |S| is held fixed (f is treated as a
 * function of S only).
 *
 *  xyz, occ   as in scatter_amplitude (the positions A was computed from).
 *  A          device complex64 [n_s]: A from scatter_amplitude on the same
 *             positions (saved by the caller; not recomputed here).
 *  I_obs      device float32 [n_s].
 *  loss_out   device float64 scalar, or NULL.
 *  dL_dxyz    device float32 [n_atoms][3] in the caller's atom order, or NULL.
 *
 * Kernel form: on a SEPARABLE plan of one GRID the per-atom sums over S
 * factorise like the forward and run as a complex contraction on the tensor
 * cores (split-f16 products, FP32 accumulation, FP64 sum over the first
 * axis; gradient error of the split path's 1e-3 class), unless its workspace
 * (about 56 B per point and species plus 24 n0 B per atom) would exceed
 * 32 GiB; every other plan runs FP32 atom-parallel kernels
 * (scatter_plan_info.adjoint_form says which).
 * Not available for GID_GRID plans (UNSUPPORTED).
 */
scatter_status scatter_backward(scatter_plan_t plan, const double* xyz,
                                const float* occ, const void* A,
                                const float* I_obs, double* loss_out,
                                float* dL_dxyz, void* stream);

/*
 * scatter_vjp — vector-Jacobian product of Eq. 2 with respect to the atom
 * positions, for any real loss L of the amplitudes:
 *   dL/dr_j = -2 pi sum_S S * Im( conj(G(S)) * w_j f_{s(j)}(|S|) exp(2 i pi S.r_j) )
 * where G(S) is the gradient of L with respect to A(S) in the convention of
 * PyTorch's complex autograd (dL = Re(sum_S conj(G(S)) dA(S))).
 * scatter_backward is this product with G = 4 (|A|^2 - I_obs) A.
 *
 *  G        device complex64 [n_s].
 *  dL_dxyz  device float32 [n_atoms][3], caller's atom order (overwritten).
 * Not available for GID_GRID plans (UNSUPPORTED).
 */
scatter_status scatter_vjp(scatter_plan_t plan, const double* xyz, const float* occ,
                           const void* G, float* dL_dxyz, void* stream);

/*
 * scatter_selftest_wait — device self-check of the failure path: one thread
 * waits for an mbarrier phase that nothing completes, gives up after ~2^20
 * SM clocks (well under a millisecond) and sets the TIMEOUT bit of the plan's
 * status word exactly as a pipeline wait of the kernels would; the next
 * scatter_check returns SCATTER_ERR_TIMEOUT and clears the word, and the
 * context stays usable.  Enqueued on `stream`; nothing else is touched.
 */
scatter_status scatter_selftest_wait(scatter_plan_t plan, void* stream);

/*
 * scatter_check — wait for the plan's stream work and report any condition a
 * kernel recorded in the plan's device status word (a bounded wait that gave
 * up: TIMEOUT; a non-finite position or occupancy: NUMERIC).  Clears the
 * word.  Synchronises `stream`.
 */
scatter_status scatter_check(scatter_plan_t plan, void* stream);

/*
 * scatter_error_bound — a-priori error model of the plan's path.
 *
 *  radius        bound on |r_j - t| over the atoms (lattice units) after
 *                the per-instance integer centring t (about half the
 *                crystal's largest extent).
 *  per_pair      out: bound on |computed - exact| of one term
 *                exp(2 i pi S.r_j), relative to its weight |w_j f|: phase
 *                reduction in FP32 (c + s.x' with |c| <= 1/2), the 2 pi
 *                scaling and the MUFU sin/cos error.
 *  rel_l2_random out: the relative L2 error of a map whose per-pair errors
 *                are uncorrelated, including blocked FP32 accumulation
 *                (per_pair plus the summation term); correlated (coherent)
 *                errors are bounded by per_pair * sum_j |w_j f| / |A|.
 */
scatter_status scatter_error_bound(scatter_plan_t plan, double radius, double* per_pair,
                                   double* rel_l2_random);

/* scatter_plan_get_info — fill *info with the plan's resolved choices. */
scatter_status scatter_plan_get_info(scatter_plan_t plan, scatter_plan_info* info);

/*
 * scatter_plan_timing — device time of the main kernel (generic, FP64,
 * adjoint, ...) of the last call on a plan created with options.timing = 1,
 * measured with CUDA events recorded on the call's stream around that
 * kernel.  Waits for the end event.  *ms_main receives milliseconds and
 * *kernel_launches the number of the library's kernels the call enqueued.
 * UNSUPPORTED if timing was not enabled or no call was made.
 */
scatter_status scatter_plan_timing(scatter_plan_t plan, double* ms_main, int32_t* kernel_launches);

/* scatter_plan_destroy — free the plan and its device memory. NULL-safe. */
void scatter_plan_destroy(scatter_plan_t plan);

/* Human-readable name of a status code (static storage). */
const char* scatter_status_string(scatter_status status);

/* One-line description of the last failure on this thread (static storage,
   valid until the next call on this thread). */
const char* scatter_last_error(void);

/* ------------------------------------------------------------------------ */
/* Allocation-free entry point                                              */
/* ------------------------------------------------------------------------ */

/*
 * scatter_amplitude_noalloc — for callers that cannot allocate device memory.
 * The paper has no counterpart: it exists because plans allocate, and some
 * callers must not — code running while a stream is captured into a CUDA
 * graph, processes whose device memory belongs to another runtime or pool,
 * latency-critical loops that may not enter the allocator.  It calls no
 * cudaMalloc/cudaFree and no allocating library routine.
 *
 * Computes T(S) = sum_j w_j exp(+2 i pi S . r_j) for a list of S points with
 * the generic FP32/MUFU kernel (f == 1: the per-species sum that a caller
 * multiplies by f_s(|S|) itself).  Positions are centred and split as on the
 * plan path (integer centre of their bounding box), and crystals whose
 * phases can pass 128 cycles take the exact-product phases, so the result
 * holds the FP32 paths' accuracy wherever the crystal sits.
 *
 *  n_atoms     0 .. 524,288            n_s  0 .. 1,048,576
 *  xyz         device float64 [n_atoms][3] (lattice units)
 *  occ         device float32 [n_atoms] or NULL (all 1)
 *  S           device float64 [n_s][3] (r.l.u.)
 *  center_hkl  host double[3], integer reference reflection H near the S
 *              points (S = H + s with |s| small gives the accurate split)
 *  T_out       device complex64 [n_s], written in full
 *  stream      cudaStream_t or NULL
 *
 * Errors: there is no plan to carry a status word, so failures found on the
 * GPU poison the output instead: if any position, occupancy or S point is
 * not finite, or a bounded wait inside the kernel gave up, every element of
 * T_out is NaN.  Sizes beyond the limits return SCATTER_ERR_INVALID_ARG
 * without launching.
 *
 * Scratch: one file-scope __device__ array of 48 MiB per GPU (held from the
 * moment the library's device code is loaded on that GPU until process
 * exit), shared by every call; calls that overlap on the GPU race on it and
 * must be serialised by the caller.  Each call resets what it reads first.
 * The first call on a device looks the array up (cudaGetSymbolAddress) with
 * that device current; with lazy module loading that first call may also
 * load the library's device code there and reserve the 48 MiB, so make it
 * before any stream capture or allocation-free section begins.
 */
scatter_status scatter_amplitude_noalloc(int64_t n_atoms, const double* xyz, const float* occ, int64_t n_s,
                                         const double* S, const double* center_hkl, void* T_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Roofline microbenchmarks                                                 */
/* ------------------------------------------------------------------------ */

/*
 * The generic path is bound by the SM's transcendental (MUFU) and FP32 FMA
 * pipes (the paper's per-pair count: 3 mul, 4 add, 1 sincos, Section 2.2).
 * scatter_microbench measures the rate of one instruction class on the
 * current device:
 *   0 sin.approx+cos.approx (MUFU ops)   1 ex2.approx (MUFU ops)
 *   2 fma.rn.f32 (lane-ops)              3 fma.rn.f32x2 (lane-ops)
 *   4 fma.rn.f64                         5 generic pair mix (2 MUFU + 7 FFMA)
 *   6 cvt.rni.f32.f32                    7 cvt.rn.f16x2.f32 (pack ops)
 *   8 tcgen05.mma kind::f16 M=128 N=256 K=16 (dense f16 flop, one CTA per
 *     SM; the separable path's contraction peak).  TIMEOUT if its bounded
 *     completion wait gives up.
 * It allocates and frees a few KB of device memory and synchronises.
 */
typedef struct scatter_microbench_result {
  double ops_per_s;
  double ops_per_clk_per_sm;
  double sm_clock_hz;      /* clock64 cycles / event seconds during the run */
  double seconds;
  int32_t n_sm;
} scatter_microbench_result;

scatter_status scatter_microbench(int kind, int iters,
                                  scatter_microbench_result* result);

/* ---- Eq. 5/6: the FFT approximation (Section 2.1) -------------------------
 *
 * Every atom is placed on the nearest node R_j of a triperiodic grid of step
 * `step` (lattice units) starting at `origin`; with r_j = R_j + u_j the factor
 * exp(2 i pi (S - H).u_j) is dropped, so that
 *   A(H + q) ~ sum_s f_s(|S|) FT[ sum_{j in s} w_j exp(2 i pi H.r_j) ](q)
 * is one discrete Fourier transform per species (cuFFT, loaded on first use).
 * The output grid is S = H + q with q_d = (i_d - floor(n_d / 2)) / (n_d step),
 * i_d in [0, n_d): index 0 holds the most negative q.  The approximation is
 * valid while |(S - H).u_j| << 1 (Eq. 7); scatter_fft_validity reports that
 * metric.  Atoms outside the grid are dropped and counted.                   */
typedef struct scatter_fft_problem {
  int64_t n_atoms;                 /* atoms per call                           */
  int32_t n_species;               /* 1 .. 64                                  */
  const scatter_species* species;  /* host [n_species]: f_s(|S|) (copied)      */
  double lattice_a;                /* Angstrom                                 */
  double center_hkl[3];            /* H, integers                              */
  double step;                     /* grid step d, lattice units, > 0          */
  double origin[3];                /* position of node (0, 0, 0), lattice units */
  int64_t n[3];                    /* nodes per axis, 2 .. 4096                */
} scatter_fft_problem;

typedef struct scatter_fft_plan_s* scatter_fft_plan_t;

/* Plans the grid (device memory n0 n1 n2 x n_species complex64 + cuFFT
 * workspace).  SCATTER_ERR_UNSUPPORTED if cuFFT cannot be loaded or planned. */
scatter_status scatter_fft_plan(const scatter_fft_problem* problem, scatter_fft_plan_t* out);

/* A(S) on the plan's grid, device complex64 [n0][n1][n2] (A_out, caller-owned).
 *   xyz          device FP64 [n_atoms][3], lattice units
 *   atom_species device int32 [n_atoms] or NULL (all species 0); an index
 *                outside [0, n_species) is counted and reported by
 *                scatter_fft_validity
 *   occ          device float [n_atoms] or NULL (all 1)
 * Enqueued on `stream` (cudaStream_t); no device-wide synchronisation.      */
scatter_status scatter_fft_amplitude(scatter_fft_plan_t plan, const double* xyz, const int32_t* atom_species,
                                     const float* occ, void* A_out, void* stream);

/* Eq. 7 metric of the last scatter_fft_amplitude call: max over atoms and
 * over the output grid of |(S - H).u_j| (cycles), and the number of atoms
 * that fell outside the grid.  Synchronises that call's stream.  Returns
 * SCATTER_ERR_INVALID_ARG if an atom had a species index out of range.      */
scatter_status scatter_fft_validity(scatter_fft_plan_t plan, double* max_qu, int64_t* n_outside);

/* NULL-safe. */
void scatter_fft_plan_destroy(scatter_fft_plan_t plan);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* SCATTER_H_ */
