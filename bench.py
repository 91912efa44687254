"""Benchmark of the direct scattering sum on one GB300 (or N under torchrun).

Workload (one step = one pass of the hot path over the synthetic input):
strained spherical fcc nanocrystal of 134,009 atoms (radius 20 cells,
Si-like core / Ge-like shell, radial strain + thermal noise) scattering onto
a 256 x 256 x 64 grid of S points (step 0.002 r.l.u.) around (004):
per-call prep (centring, split phase), the map kernel and the epilogue,
5.6e11 atom-reflection pairs per step.  The headline uses the separable
tensor-core path (--path separable, the default) or the generic FP32/MUFU
path (--path generic); both meet the 1e-4 relative-L2 tolerance on this map,
which the CPU-baseline leg re-checks against the FP64 oracle on a sample.

Metric: atom-reflection pairs per second (whole job, all ranks), the paper's
"reflections x atoms / s" (Section 2.2).  Each rank runs its own full
instance (weak scaling, no collective on the data path).

JSON line keys beyond the base contract:
  roofline      dominant kernel: k_sep against the measured dense tensor
                peak, or k_generic against the MUFU bound
                (16 sin/cos ops / SM / clk -> 8 pairs / SM / clk x SMs x clock)
  cpu_baseline  the FP64 oracle timed on the host cores on a bounded sample
  accuracy      relative L2 error of the GPU map vs the oracle on that sample
  e2e           the same metric through the C-ABI call with host buffers,
                scatter_amplitude_host (positions H2D from pinned memory, the
                map D2H into pinned memory every step, both in the timed
                region)
  paths         the other rows on their own workloads: the other map path
                (with its roofline), the FP64 kernel, the adjoint, the DWBA
                map and the batched persistent launch (skip: --no-paths)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import pathlib
import re
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = pathlib.Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "atom·reflections/s at ≤1e-4 rel err vs FP64 oracle; fraction of FP32/MUFU peak"
UNIT = "atom·reflections/s"
MUFU_SINCOS_PER_SM_CLK = 16.0   # measured (scatter_microbench kind 0): 15.97
MUFU_OPS_PER_PAIR = 2.0         # one sin + one cos per (atom, reflection)


GRID = (256, 256, 64)


def workload():
    from paper_1010_2641_gb300 import workloads as W
    c = W.fcc_sphere()
    axes = [W.linspace_axis(0.0, GRID[0], step=0.002), W.linspace_axis(0.0, GRID[1], step=0.002),
            W.linspace_axis(4.0, GRID[2], step=0.002)]
    return c, axes


def workload_name():
    return (f"strained fcc sphere r=20 cells (134009 atoms, 2 species) x {GRID[0]}x{GRID[1]}x{GRID[2]} "
            "S grid around (004), step 0.002 r.l.u.")


def host_cpu() -> str:
    """Machine and CPU model of the host (best effort, for the report)."""
    import platform
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu part"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return f"{platform.machine()} {model} x{os.cpu_count()}".strip()


def sample_indices(n_s: int, n: int, seed: int = 7):
    return np.sort(np.random.default_rng(seed).choice(n_s, n, replace=False))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, log_dir: str | None = None):
        self.proc = None
        self.gpu = gpu_index
        base = pathlib.Path(log_dir) if log_dir else pathlib.Path(tempfile.gettempdir())
        self.path = base / f"clocks_rank{gpu_index}.csv"

    def start(self):
        try:
            self.path.parent.mkdir(parents=True, exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # nvidia-smi takes a moment to start: open the timed region only once it samples
            t0 = time.time()
            while time.time() - t0 < 5.0 and self.proc.poll() is None:
                if self.path.exists() and self.path.stat().st_size > 0:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        for line in self.path.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# profile summary -> traffic of the dominant kernel (null if stale)
# ---------------------------------------------------------------------------

def measured_peak(key: str, fallback: float):
    p = ROOT / "MEASURED_PEAKS.json"
    try:
        v = float(json.loads(p.read_text())[key])
        return v, f"MEASURED_PEAKS.json {key} = {v} (of measured)"
    except Exception:
        return fallback, f"fallback {fallback} (of fallback)"


GENERIC_SOURCES = ("forward.cu", "generic_impl.cuh", "device_common.cuh", "plan.h")


def kernel_source_hash(files=GENERIC_SOURCES) -> str:
    h = hashlib.sha1()
    for f in files:
        h.update((ROOT / "paper_1010_2641_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:12]


SEP_SOURCES = ("separable.cu", "sep_pair.cu", "sep_common.cuh", "device_common.cuh", "plan.h")


def profiled_traffic(name="generic_strained_sphere.md", files=GENERIC_SOURCES):
    """dram bytes per launch of a kernel from its committed ncu summary, if
    the summary was taken on the current kernel source."""
    p = ROOT / "profiles" / name
    if not p.exists():
        return None
    text = p.read_text()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s*\(source sha1 ([0-9a-f]+)\)", text)
    if not m or m.group(2) != kernel_source_hash(files):
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step(c, S_sample):
    import oracle
    from paper_1010_2641_gb300 import workloads as W
    return oracle.amplitude(c.xyz, S_sample, c.coef, W.LATTICE_A, species=c.species)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    from paper_1010_2641_gb300 import workloads as W
    oracle.build()
    c, axes = workload()
    n_s = GRID[0] * GRID[1] * GRID[2]
    n_sample = args.ref_sample
    idx = sample_indices(n_s, n_sample, seed=1)
    S = W.grid_points(axes)[idx]
    for _ in range(args.warmup):
        oracle_step(c, S)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(c, S)
        times.append(time.perf_counter() - t0)
    pairs = len(c.xyz) * n_sample
    v = pairs / float(np.mean(times))
    cores = oracle.num_threads()
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(), "n_atoms": len(c.xyz), "n_s": n_s,
                                           "sample_points": n_sample},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{n_sample} of {n_s} grid points (seeded), all {len(c.xyz)} atoms"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    from paper_1010_2641_gb300 import api, sharding

    __graft_entry__.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    c, axes = workload()
    n_atoms, n_s = len(c.xyz), GRID[0] * GRID[1] * GRID[2]
    pairs = n_atoms * n_s
    cache = str(pathlib.Path(args.log_dir or tempfile.gettempdir()) / "tune_cache.jsonl") if args.autotune else None
    plan = api.Plan(c.coef, 5.43, n_atoms, axes=axes, atom_species=c.species, timing=True, path=args.path,
                    autotune=args.autotune and args.path == "generic", tune_cache=cache)
    info = plan.info()
    xyz = torch.tensor(c.xyz, dtype=torch.float64, device=dev)
    A = torch.empty(n_s, dtype=torch.complex64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    for _ in range(args.warmup):
        plan.amplitude(xyz, out=A)
    torch.cuda.synchronize()
    plan.check()

    # ---- device-timed region: K steps, L2 flushed between steps -------------
    clocks = ClockSampler(local_rank, args.log_dir)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kern_ms, launches = [], 0
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        plan.amplitude(xyz, out=A)
        ev[i][1].record(stream)
        ms_k, n_k = plan.timing()
        kern_ms.append(ms_k)
        launches += n_k
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_step = float(np.mean(step_ms))
    t_kern = float(np.mean(kern_ms))
    if world > 1:
        t_step, t_kern = sharding.max_over_ranks([t_step, t_kern], device=dev)
    value = world * pairs / (t_step * 1e-3)

    # ---- end to end through the public API with host buffers -------------------
    # scatter_amplitude_host: pinned host positions in, pinned host map out;
    # the positions' copy to the device, the forward and the map's copy back
    # (overlapping the last reduction on separable grids) in the timed region
    xyz_host = torch.tensor(c.xyz, dtype=torch.float64).pin_memory()
    A_host = torch.empty(n_s, dtype=torch.complex64).pin_memory()
    for _ in range(2):
        plan.amplitude_host(xyz_host, out=A_host, stream=stream)
    torch.cuda.synchronize()
    plan.check()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = []
    for i in range(max(2, args.steps // 2)):
        flush.zero_()
        e0.record(stream)
        plan.amplitude_host(xyz_host, out=A_host, stream=stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    t_e2e = float(np.mean(e2e_ms))
    if world > 1:
        (t_e2e,) = sharding.max_over_ranks([t_e2e], device=dev)

    # ---- roofline of the dominant kernel ----------------------------------------
    sm_mhz = clk["sm_mhz"] if clk else None
    n_sm = info["n_sm"]
    roof = None
    if args.path == "separable":
        # executed tensor-pipe work: 3 split products x 2 flop x M' x N' x K'
        m_pad = -(-2 * GRID[0] // 128) * 128
        n_pad = -(-(GRID[1] * GRID[2]) // 256) * 256
        executed = 6.0 * m_pad * n_pad * 2 * info["n_atoms_padded"]
        useful = 8.0 * n_atoms * n_s
        peak, basis = measured_peak("bf16_tflops", 1900.0)
        achieved = executed / (t_kern * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None if args.grid else profiled_traffic("separable_strained_sphere.md", SEP_SOURCES),
                "kernel": ("k_sep_pair (tcgen05.mma.cta_group::2 kind::f16, M=256 N=256 on a CTA pair, "
                           "3 split products)" if os.environ.get("SCATTER_SEP_PAIR", "1") != "0" else
                           "k_sep (tcgen05.mma kind::f16, M=128 N=256, 3 split products)"),
                "kernel_ms": t_kern, "useful_tflops": useful / (t_kern * 1e-3) / 1e12,
                "peak_basis": f"{basis} (f16 and bf16 share the dense tensor rate)"}
        # cross-check: this GPU's own f16 MMA rate (back-to-back tcgen05.mma, M=128 N=256, zero operands)
        mb = api.microbench(8, iters=20000)
        roof["f16_mma_microbench_tflops"] = mb["ops_per_s"] / 1e12
        roof["frac_of_f16_mma_microbench"] = achieved / (mb["ops_per_s"] / 1e12)
    elif sm_mhz:
        peak = n_sm * MUFU_SINCOS_PER_SM_CLK / MUFU_OPS_PER_PAIR * sm_mhz * 1e6 / 1e9  # Gpair/s
        achieved = pairs / (t_kern * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": achieved / peak, "traffic": profiled_traffic(),
                "kernel": "k_generic (MUFU sin/cos, 16 ops/SM/clk)",
                "kernel_ms": t_kern, "peak_basis": f"{n_sm} SMs x 8 pairs/SM/clk x {sm_mhz:.0f} MHz (median sampled)"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32" if args.path == "generic" else "f16x3 split, f32 accumulate",
           "data": "synthetic",
           "config": {"workload": workload_name(), "n_atoms": n_atoms, "n_s": n_s, "pairs_per_step": pairs,
                      "path": args.path, "threads": info["threads"], "points_per_thread": info["points_per_thread"],
                      "split_k": info["split_k"], "l2": "flushed between steps (256 MB write, outside the events)",
                      "parallelism": f"weak x{world} (independent instance per GPU)"},
           "roofline": roof, "clocks": clk, "gpu_launches": launches,
           "e2e": {"value": world * pairs / (t_e2e * 1e-3), "unit": UNIT,
                   "h2d_bytes_per_step": int(xyz_host.numel() * 8), "d2h_bytes_per_step": int(A_host.numel() * 8)}}

    # ---- CPU baseline + accuracy on a bounded sample (rank 0, N=1) -------------
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        from paper_1010_2641_gb300 import workloads as W
        oracle.build()
        idx = sample_indices(n_s, args.cpu_sample)
        S = W.grid_points(axes)[idx]
        t0 = time.perf_counter()
        ref = oracle_step(c, S)
        dt = time.perf_counter() - t0
        got = A.cpu().numpy()[idx].astype(np.complex128)
        cores = oracle.num_threads()
        # single-thread rate on a smaller sample (compare: the paper's 122e6 pairs/s/core, SSE FP32)
        idx1 = idx[: max(1, len(idx) // 32)]
        oracle.set_threads(1)
        t1 = time.perf_counter()
        oracle_step(c, W.grid_points(axes)[idx1])
        dt1 = time.perf_counter() - t1
        oracle.set_threads(0)
        out["cpu_baseline"] = {"value": n_atoms * len(idx) / dt, "unit": UNIT, "cores": cores,
                               "kind": "oracle",
                               "sample": f"{len(idx)} of {n_s} grid points (seeded), all {n_atoms} atoms, {dt:.1f} s",
                               "per_core": n_atoms * len(idx) / dt / cores,
                               "single_thread": n_atoms * len(idx1) / dt1,
                               "host": host_cpu()}
        out["accuracy"] = {"rel_l2_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                           "points": int(len(idx)), "tolerance": 1e-4}
    if not args.no_paths and rank == 0 and world == 1:
        out["paths"] = measure_paths(args, dev, clk)
    plan.check()
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def _time_calls(fn, plan, reps=2, min_s=0.0):
    """Mean main-kernel time (plan events) of at least `reps` calls after one
    warm-up call, repeated until `min_s` seconds have passed (up to 2000 calls)."""
    import torch
    fn()
    torch.cuda.synchronize()
    ms = []
    t0 = time.time()
    while len(ms) < reps or (time.time() - t0 < min_s and len(ms) < 2000):
        fn()
        ms.append(plan.timing()[0])
    return float(np.mean(ms))


def _rate_roof(units, ms, per_sm_clk, n_sm, clk, unit, bound, basis):
    """Roofline object of a compute-bound row: `units` of work in `ms`
    against per_sm_clk units per SM per clock at the sampled SM clock."""
    if not (clk and clk.get("sm_mhz")):
        return None
    peak = n_sm * per_sm_clk * clk["sm_mhz"] * 1e6
    achieved = units / (ms * 1e-3)
    return {"bound": bound, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": unit, "frac": achieved / peak,
            "peak_basis": f"{n_sm} SMs x {per_sm_clk:g} {basis}/SM/clk x {clk['sm_mhz']:.0f} MHz (median sampled)",
            "clocks": clk}


def _tensor_roof(n0, n12, n_atoms_padded, ms, clk=None):
    """Executed-flop roofline of k_sep on an n0 x n12 separable grid."""
    m_pad = -(-2 * n0 // 128) * 128
    n_pad = -(-n12 // 256) * 256
    executed = 6.0 * m_pad * n_pad * 2 * n_atoms_padded
    peak, basis = measured_peak("bf16_tflops", 1900.0)
    achieved = executed / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_basis": f"{basis} (f16 and bf16 share the dense tensor rate)", "clocks": clk}


def _tensor_roof_adjoint(n0, n12, n_atoms_padded, ms, clk=None):
    """Executed-flop roofline of k_sep running the adjoint: rows (a, weight,
    Re/Im) = 6 n0, columns = atom slots in 256-slot tiles, K = 2 per point."""
    m_pad = -(-6 * n0 // 128) * 128
    n_pad = -(-n_atoms_padded // 256) * 256
    k_pad = -(-n12 // 16) * 16 * 2
    executed = 6.0 * m_pad * n_pad * k_pad
    peak, basis = measured_peak("bf16_tflops", 1900.0)
    achieved = executed / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_basis": f"{basis} (f16 and bf16 share the dense tensor rate)", "clocks": clk}


def _time_whole(fn, reps=3):
    """Device time of whole calls (every kernel they launch), CUDA events on
    torch's current stream, where the plan launches."""
    import torch
    fn()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        fn()
    t1.record()
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def measure_paths(args, dev, clk, only=None):
    """The other rows of the hot path, each on its own workload (device time
    of the row's main kernel, CUDA events on the launching stream), each with
    the roofline of its binding unit.  `only`: run just the row(s) of that name."""
    import torch
    from paper_1010_2641_gb300 import api
    from paper_1010_2641_gb300 import workloads as W
    res = {}
    rc = {}

    def timed(fn, plan, reps=2):
        """_time_calls over at least 0.5 s, with the SM clocks sampled while
        the calls ran kept in rc["clk"]: each row's roofline takes the clock
        its own kernel ran at.  --reps R: exactly R timed calls after the
        warm-up (a fixed launch sequence, for profilers)."""
        cs = ClockSampler(0, args.log_dir)
        cs.start()
        ms = _time_calls(fn, plan, args.reps, min_s=0.0) if args.reps else _time_calls(fn, plan, reps, min_s=0.5)
        rc["clk"] = cs.stop()
        return ms

    c, axes = workload()
    xyz = torch.tensor(c.xyz, dtype=torch.float64, device=dev)
    n_atoms, n_s = len(c.xyz), GRID[0] * GRID[1] * GRID[2]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    other = "generic" if args.path == "separable" else "separable"

    def want(name):
        return only is None or only == name or (name == "dwba_island" and only == "dwba_island_separable")

    if want(f"{other}_sphere"):
        # generic FP32/MUFU kernel on the full strained-sphere map, with its roofline
        other = "generic" if args.path == "separable" else "separable"
        plan = api.Plan(c.coef, W.LATTICE_A, n_atoms, axes=axes, atom_species=c.species, path=other, timing=True)
        ms = timed(lambda: plan.amplitude(xyz), plan)
        row = {"value": n_atoms * n_s / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms, "workload": "strained sphere, full map"}
        n_sm = plan.info()["n_sm"]
        if other == "generic":
            row["roofline"] = _rate_roof(n_atoms * n_s, ms, MUFU_SINCOS_PER_SM_CLK / MUFU_OPS_PER_PAIR, n_sm, rc.get("clk"),
                                         "Gpair/s", "alu", "pairs (2 MUFU sin/cos each)")
        else:
            row["roofline"] = _tensor_roof(GRID[0], GRID[1] * GRID[2], plan.info()["n_atoms_padded"], ms,
                                            rc.get("clk"))
        res[f"{other}_sphere"] = row
        del plan
    if want("auto_sphere"):
        # the same map with default options: the plan picks the path itself
        plan = api.Plan(c.coef, W.LATTICE_A, n_atoms, axes=axes, atom_species=c.species, timing=True)
        xa = torch.tensor(c.xyz, dtype=torch.float64, device=dev)
        ms = timed(lambda: plan.amplitude(xa), plan)
        ms_call = _time_whole(lambda: plan.amplitude(xa))
        inf = plan.info()
        # value from whole calls (every kernel of the call), like the headline's steps
        res["auto_sphere"] = {"value": n_atoms * n_s / (ms_call * 1e-3), "unit": UNIT, "call_ms": ms_call,
                              "kernel_ms": ms, "l2": "calls back to back, not flushed between them",
                              "path_chosen": {1: "generic", 2: "separable"}.get(inf["path"], str(inf["path"])),
                              "workload": "strained sphere, full map, default options (AUTO, tolerance 1e-4)",
                              "clocks": rc.get("clk")}
        del plan, xa
    if want('fp64_sphere_slice'):
        # plain FP64 kernel on a 1/16 slice of the same map (every 16th l plane)
        sub = [axes[0], axes[1], axes[2][::16]]
        n_sub = len(sub[0]) * len(sub[1]) * len(sub[2])
        plan = api.Plan(c.coef, W.LATTICE_A, n_atoms, axes=sub, atom_species=c.species, path="fp64", timing=True)
        ms = timed(lambda: plan.amplitude(xyz), plan, reps=1)
        res["fp64_sphere_slice"] = {"value": n_atoms * n_sub / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms, "n_s": n_sub}
        del plan, xyz
    if want('fft_sphere_approx'):
        # FFT approximation (Eq. 5/6) of the same crystal on a 256^3 grid of step 0.5 cells
        # (S within +-1 r.l.u. of (004)), against the direct sum on that grid
        xyz = torch.tensor(c.xyz, dtype=torch.float64, device=dev)
        sp = torch.tensor(c.species, dtype=torch.int32, device=dev)
        fp = api.FFTPlan(c.coef, W.LATTICE_A, n_atoms, center=(0, 0, 4), step=0.5,
                         origin=np.floor(c.xyz.min(0)) - 1.0, n=(256, 256, 256))
        A_fft = fp.amplitude(xyz, sp)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        torch.cuda.synchronize()
        ev[0].record()
        fp.amplitude(xyz, sp, out=A_fft)
        ev[1].record()
        torch.cuda.synchronize()
        ms_fft = ev[0].elapsed_time(ev[1])
        max_qu, outside = fp.validity()
        plan = api.Plan(c.coef, W.LATTICE_A, n_atoms, axes=fp.axes(), atom_species=c.species, path="separable",
                        timing=True)
        ms_dir = timed(lambda: plan.amplitude(xyz), plan, reps=1)
        A_dir = plan.amplitude(xyz).reshape(A_fft.shape)
        err = (torch.linalg.vector_norm(A_fft - A_dir) / torch.linalg.vector_norm(A_dir)).item()
        # the same near H: |q_d| <= 0.1 r.l.u. (12 bins of 1/128 r.l.u. each side), where |q.u| is 10x smaller
        win = slice(128 - 12, 128 + 13)
        a_w, d_w = A_fft[win, win, win], A_dir[win, win, win]
        err_near = (torch.linalg.vector_norm(a_w - d_w) / torch.linalg.vector_norm(d_w)).item()
        n_fft = 256 ** 3
        res["fft_sphere_approx"] = {"value": n_atoms * n_fft / (ms_fft * 1e-3), "unit": UNIT + " (equivalent)",
                                    "call_ms": ms_fft, "direct_separable_ms": ms_dir, "rel_l2_vs_direct": err,
                                    "rel_l2_vs_direct_within_0.1_rlu": err_near,
                                    "eq7_max_qu_cycles": max_qu, "atoms_outside": outside,
                                    "workload": "strained sphere on a 256^3 grid of step 0.5 cells: deposit + cuFFT "
                                                "(2 species) + f_s epilogue, against the separable direct sum"}
        del plan, fp, A_fft, A_dir, xyz, sp
    if want('example1_cube'):
        # Section 4's first example: the strained 100^3 simple cubic crystal
        # (1e6 atoms, f = 1) on its 200 x 200 (h, l) map at k = 0; the paper
        # quotes 0.93 s on its GPU for this map
        xe = torch.tensor(W.example_cube_100(strained=True), dtype=torch.float64, device=dev)
        axes_e = W.example_cube_axes()
        n_e = len(axes_e[0]) * len(axes_e[1]) * len(axes_e[2])
        row = {"unit": UNIT, "workload": "strained 100^3 simple cubic crystal (1e6 atoms) x 200 x 200 (h, l) "
                                         "around (004)", "paper_seconds_context": 0.93}
        for path in ("generic", "separable"):
            plan = api.Plan(W.unit_species()[None], W.LATTICE_A, xe.shape[0], axes=axes_e, path=path, timing=True)
            ms = timed(lambda: plan.amplitude(xe), plan)
            ms_call = _time_whole(lambda: plan.amplitude(xe))
            row[path] = {"value": xe.shape[0] * n_e / (ms_call * 1e-3), "call_ms": ms_call, "kernel_ms": ms}
            del plan
        row["value"] = max(row["generic"]["value"], row["separable"]["value"])
        res["example1_cube"] = row
        del xe
    if want('adjoint_cube'):
        # adjoint on the strained cube (102,400 atoms x 128^3)
        cube = W.strained_cube()
        ax = [W.linspace_axis(0.0, 128, step=0.005), W.linspace_axis(0.0, 128, step=0.005),
              W.linspace_axis(4.0, 128, step=0.005)]
        plan = api.Plan(cube.coef, W.LATTICE_A, len(cube.xyz), axes=ax, timing=True, path="generic")
        x = torch.tensor(cube.xyz, dtype=torch.float64, device=dev)
        I_obs = plan.intensity(torch.tensor(W.perturbed_copy(cube).xyz, dtype=torch.float64, device=dev))
        A = plan.amplitude(x)
        ms_f = timed(lambda: plan.amplitude(x, out=A), plan)
        ms = timed(lambda: plan.backward(x, A, I_obs), plan)
        res["adjoint_cube"] = {"value": len(cube.xyz) * 128 ** 3 / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
                               "forward_kernel_ms": ms_f, "workload": "strained cube 102400 atoms x 128^3, dL/dr",
                               # uniform l axis: the line kernel carries the phase along l by a complex multiply,
                               # 8 FMA-pipe ops per pair at 128 lane-ops per SM per clock, no MUFU
                               "roofline": _rate_roof(len(cube.xyz) * 128 ** 3, ms, 16.0, n_sm, rc.get("clk"), "Gpair/s", "alu",
                                                      "pairs (8 FMA-pipe ops each)")}
        del plan, x, A, I_obs
    if want('adjoint_list'):
        # the S-list adjoint (k_adjoint: MUFU sin/cos per pair): strained sphere x an Ewald-slice list
        c_l = W.fcc_sphere()
        S_l = W.ewald_slice(262144, seed=8101)
        plan = api.Plan(c_l.coef, W.LATTICE_A, len(c_l.xyz), s_list=S_l, atom_species=c_l.species, timing=True)
        x = torch.tensor(c_l.xyz, dtype=torch.float64, device=dev)
        I_obs = plan.intensity(torch.tensor(W.perturbed_copy(c_l).xyz, dtype=torch.float64, device=dev))
        A = plan.amplitude(x)
        ms = timed(lambda: plan.backward(x, A, I_obs), plan)
        pairs_l = len(c_l.xyz) * len(S_l)
        res["adjoint_list"] = {"value": pairs_l / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
                               "workload": "strained sphere 134009 atoms x 262144 Ewald-slice points near (111), dL/dr",
                               "roofline": _rate_roof(pairs_l, ms, MUFU_SINCOS_PER_SM_CLK / MUFU_OPS_PER_PAIR, n_sm,
                                                      rc.get("clk"), "Gpair/s", "alu", "pairs (2 MUFU sin/cos each)")}
        del plan, x, A, I_obs
    if want('adjoint_cube_separable'):
        # the same gradient on a SEPARABLE plan: the per-atom sums contract on the tensor cores
        cube = W.strained_cube()
        ax = [W.linspace_axis(0.0, 128, step=0.005), W.linspace_axis(0.0, 128, step=0.005),
              W.linspace_axis(4.0, 128, step=0.005)]
        plan = api.Plan(cube.coef, W.LATTICE_A, len(cube.xyz), axes=ax, path="separable", timing=True)
        x = torch.tensor(cube.xyz, dtype=torch.float64, device=dev)
        I_obs = plan.intensity(torch.tensor(W.perturbed_copy(cube).xyz, dtype=torch.float64, device=dev))
        A = plan.amplitude(x)
        ms_f = timed(lambda: plan.amplitude(x, out=A), plan)
        ms = timed(lambda: plan.backward(x, A, I_obs), plan)
        ms_call = _time_whole(lambda: plan.backward(x, A, I_obs))
        assert plan.info()["adjoint_form"] == 3
        res["adjoint_cube_separable"] = {
            "value": len(cube.xyz) * 128 ** 3 / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms, "call_ms": ms_call,
            "call_value": len(cube.xyz) * 128 ** 3 / (ms_call * 1e-3), "forward_kernel_ms": ms_f,
            "workload": "strained cube 102400 atoms x 128^3, dL/dr on a SEPARABLE plan (k_sep, operands swapped)",
            "roofline": _tensor_roof_adjoint(128, 128 * 128, plan.info()["n_atoms_padded"], ms,
                                                 rc.get("clk"))}
        del plan, x, A, I_obs
    if only == 'dwba_island_mid':
        # profiling case of the FFMA DWBA kernel: 127,560-atom island (base 60, height 20 cells) x 128x128x32
        isl = W.truncated_pyramid(base_cells=60, height_cells=20, top_cells=15)
        gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
        plan = api.Plan(isl.coef, W.LATTICE_A, len(isl.xyz), axes=list(W.gid_axes(128, 128, 32)),
                        atom_species=isl.species, gid=gid, path="generic", timing=True)
        x = torch.tensor(isl.xyz, dtype=torch.float64, device=dev)
        ms = timed(lambda: plan.amplitude(x), plan, reps=2)
        res["dwba_island_mid"] = {"value": 4 * len(isl.xyz) * 128 * 128 * 32 / (ms * 1e-3), "unit": UNIT + " (x4 beams)",
                                  "kernel_ms": ms, "workload": f"island {len(isl.xyz)} atoms x 128x128x32, FFMA kernel"}
        del plan, x
    if want('dwba_island'):
        # grazing-incidence four-beam map of the island (1,013,496 atoms x 512x512x32)
        isl = W.truncated_pyramid()
        gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
        plan = api.Plan(isl.coef, W.LATTICE_A, len(isl.xyz), axes=list(W.gid_axes()), atom_species=isl.species,
                        gid=gid, timing=True, path="generic")
        x = torch.tensor(isl.xyz, dtype=torch.float64, device=dev)
        ms = timed(lambda: plan.amplitude(x), plan, reps=1)
        m_gid = 512 * 512 * 32
        res["dwba_island"] = {"value": 4 * len(isl.xyz) * m_gid / (ms * 1e-3), "unit": UNIT + " (x4 beams)",
                              "kernel_ms": ms, "workload": "island 1013496 atoms x 512x512x32, 4 beams, FFMA kernel",
                              # 8 FFMA per (atom, point) for the four beams (they share the real products of
                              # E and Z1, Z2): 16 points = 64 beam-pairs per SM per clock on the FMA pipe
                              "roofline": _rate_roof(4 * len(isl.xyz) * m_gid, ms, 64.0, n_sm, rc.get("clk"), "Gbeam-pair/s",
                                                     "alu", "beam-pairs (8 FFMA per atom-point, 128 FFMA/SM/clk)")}
        del plan
        plan = api.Plan(isl.coef, W.LATTICE_A, len(isl.xyz), axes=list(W.gid_axes()), atom_species=isl.species,
                        gid=gid, path="separable", timing=True)
        ms = timed(lambda: plan.amplitude(x), plan, reps=1)
        res["dwba_island_separable"] = {"value": 4 * len(isl.xyz) * m_gid / (ms * 1e-3), "unit": UNIT + " (x4 beams)",
                                        "kernel_ms": ms,
                                        "workload": "same map, beams stacked on a virtual l axis, tensor cores",
                                        "roofline": _tensor_roof(512, 512 * 4 * 32, plan.info()["n_atoms_padded"], ms,
                                                                 rc.get("clk"))}
        del plan, x
    if want("atompar_few_reflections"):
        # many atoms, few reflections: the atom-parallel form (the paper's speed test at 1e6 x 1e3)
        rx, rS = W.random_sweep(1_000_000, 1000, seed=77)
        plan = api.Plan(W.unit_species(), W.LATTICE_A, len(rx), s_list=rS, path="generic", timing=True)
        x = torch.tensor(rx, dtype=torch.float64, device=dev)
        out = torch.empty(len(rS), dtype=torch.complex64, device=dev)
        ms = timed(lambda: plan.amplitude(x, out=out), plan, reps=5)
        pairs_a = float(len(rx) * len(rS))
        res["atompar_few_reflections"] = {
            "value": pairs_a / (ms * 1e-3), "unit": UNIT, "kernel_ms": ms,
            "atoms_per_thread": plan.info()["atoms_per_thread"],
            "workload": "1e6 random atoms x 1000 random reflections (atom-parallel form)",
            "roofline": _rate_roof(pairs_a, ms, MUFU_SINCOS_PER_SM_CLK / MUFU_OPS_PER_PAIR, n_sm, rc.get("clk"), "Gpair/s",
                                   "alu", "pairs (2 MUFU sin/cos each)")}
        del plan, x, out
    if want("dwba_ge_dot"):
        # the paper's germanium-dot example: (h, 0, alpha_f) map across (400), both DWBA paths
        dot = W.ge_dot()
        gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
        ax = list(W.ge_dot_axes())
        x = torch.tensor(dot.xyz, dtype=torch.float64, device=dev)
        m_dot = len(ax[0]) * len(ax[1]) * len(ax[2])
        row = {"unit": UNIT + " (x4 beams)", "workload": "Ge dot (669,753 atoms) x 512 h x 128 alpha_f across (400)"}
        for name, pth in (("ffma", "generic"), ("separable", "separable")):
            plan = api.Plan(dot.coef, W.LATTICE_A, len(dot.xyz), axes=ax, atom_species=dot.species, gid=gid,
                            path=pth, timing=True)
            ms = timed(lambda: plan.amplitude(x), plan, reps=2)
            row[f"{name}_ms"] = ms
            row[f"{name}_value"] = 4 * len(dot.xyz) * m_dot / (ms * 1e-3)
            del plan
        row["value"] = max(row["ffma_value"], row["separable_value"])
        res["dwba_ge_dot"] = row
        del x
    if want('batch_ewald'):
        # batched persistent launch, CUDA-graph replay (64 uneven crystals)
        bx, bs, bcoef, bS, ao, so = W.ewald_batch(n_instances=args.batch_instances)
        # tiles picked by the autotuner at plan time (the configuration's "autotuned tiles")
        bcache = str(pathlib.Path(args.log_dir) / "tune_cache_batch.jsonl") if args.log_dir else None
        plan = api.Plan(bcoef, W.LATTICE_A, len(bx), s_list=bS, atom_species=bs, atom_off=ao, s_off=so, timing=True,
                        autotune=True, tune_cache=bcache)
        x = torch.tensor(bx, dtype=torch.float64, device=dev)
        out = torch.empty(len(bS), dtype=torch.complex64, device=dev)
        ms = timed(lambda: plan.amplitude(x, out=out), plan)
        pairs_b = float(np.sum(np.diff(ao) * np.diff(so)))
        inf = plan.info()
        res["batch_ewald"] = {"value": pairs_b / (ms * 1e-3), "unit": UNIT, "graph_ms": ms, "instances": len(ao) - 1,
                              "tiling": {"threads": inf["threads"], "points_per_thread": inf["points_per_thread"],
                                         "autotuned": True},
                              "workload": f"{len(ao) - 1} fcc crystals 1e3-2e5 atoms, 1e4-1e6 Ewald-slice points each",
                              "roofline": _rate_roof(pairs_b, ms, MUFU_SINCOS_PER_SM_CLK / MUFU_OPS_PER_PAIR, n_sm, rc.get("clk"),
                                                     "Gpair/s", "alu", "pairs (2 MUFU sin/cos each)")}
    return res


def run_sweep(args):
    """The paper's speed test (Section 3, its speed figure): random atoms in a
    100^3 box, random S within +-0.5 of (004), occupancy 1, f = 1; pairs/s of
    the generic kernel for every (atoms, reflections) in {1e2 .. 1e6}^2, each
    spot-checked against the oracle.  Prints one JSON object."""
    import torch
    import oracle
    from paper_1010_2641_gb300 import api
    from paper_1010_2641_gb300 import workloads as W
    oracle.build()
    dev = "cuda:0"
    torch.cuda.set_device(0)
    sizes = [int(v) for v in args.sweep.split(",")]
    unit = W.unit_species()
    rows = []
    for n_atoms in sizes:
        for n_s in sizes:
            xyz, S = W.random_sweep(n_atoms, n_s, seed=1000 * len(str(n_atoms)) + len(str(n_s)))
            plan = api.Plan(unit, W.LATTICE_A, n_atoms, s_list=S, path="generic", timing=True,
                            autotune=args.autotune)
            x = torch.tensor(xyz, dtype=torch.float64, device=dev)
            out = torch.empty(n_s, dtype=torch.complex64, device=dev)
            ms = _time_calls(lambda: plan.amplitude(x, out=out), plan, reps=5 if n_atoms * n_s < 1e11 else 2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.amplitude(x, out=out)
            e1.record()
            torch.cuda.synchronize()
            call_ms = e0.elapsed_time(e1)
            # the same call on a plan without per-call timing replays its launch
            # sequence as a CUDA graph (first call eager, second captures)
            gplan = api.Plan(unit, W.LATTICE_A, n_atoms, s_list=S, path="generic", autotune=args.autotune)
            for _ in range(3):
                gplan.amplitude(x, out=out)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(5):
                gplan.amplitude(x, out=out)
            e1.record()
            torch.cuda.synchronize()
            graph_call_ms = e0.elapsed_time(e1) / 5
            del gplan
            idx = sample_indices(n_s, min(n_s, 16), seed=3)
            ref = oracle.amplitude(xyz, S[idx], unit, W.LATTICE_A)
            got = out.cpu().numpy()[idx].astype(np.complex128)
            err = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
            info = plan.info()
            rows.append({"atoms": n_atoms, "reflections": n_s, "value": n_atoms * n_s / (ms * 1e-3),
                         "kernel_ms": ms, "call_ms": call_ms, "graph_call_ms": graph_call_ms,
                         "rel_l2_16pts": err, "threads": info["threads"],
                         "points_per_thread": info["points_per_thread"], "split_k": info["split_k"],
                         "atoms_per_thread": info["atoms_per_thread"]})
            del plan, x, out
    print(json.dumps({"sweep": "generic kernel, random atoms x random reflections (paper's speed test)",
                      "unit": UNIT, "rows": rows}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=16384)
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=64,
                    help="crystals in the batch row (fewer: a smaller profiling case of the same kernel)")
    ap.add_argument("--log-dir", default=None,
                    help="folder for the per-rank clock samples and the autotune cache (default: the temp folder)")
    ap.add_argument("--no-paths", action="store_true", help="skip the other rows' measurements")
    ap.add_argument("--grid", default=None, help="smaller S grid n0,n1,n2 (profiling cases)")
    ap.add_argument("--sweep", default=None, help="speed sweep over atoms x reflections, e.g. 100,1000,10000")
    ap.add_argument("--row", default=None, help="run one row of the paths section alone (profiling), e.g. adjoint_cube")
    ap.add_argument("--reps", type=int, default=0,
                    help="paths rows: exactly this many timed calls per row (a fixed launch sequence for profiling)")
    ap.add_argument("--path", default="separable", choices=["generic", "separable"],
                    help="kernel family of the headline line (both meet the 1e-4 tolerance on this map)")
    args = ap.parse_args()
    if args.grid:
        global GRID
        GRID = tuple(int(v) for v in args.grid.split(","))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.sweep:
        return run_sweep(args)
    if args.row:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"row": args.row, **measure_paths(args, "cuda:0", None, only=args.row)}))
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
