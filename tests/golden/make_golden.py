"""Writes the stored expected values of the full-size parity tests.

Every value in the files this script writes comes from the FP64 CPU oracle
(``oracle/``) on the seeded synthetic inputs of
``paper_1010_2641_gb300.workloads``; nothing is taken from the GPU library.
Run it on the host (it takes hours of CPU time on a few cores):

    python tests/golden/make_golden.py [--only island|cube|batch|sphere] [--threads N]

Files (numpy ``.npz``; each holds a ``meta`` JSON string naming this script,
the workload, its seeds and the oracle calls):

  island_gid_subgrid.npz   the 1,013,496-atom truncated-pyramid island on
                           the 1/64 sub-grid of its 512 x 512 x 32
                           (h, k, alpha_f) map: every 8th h and every 8th k,
                           all 32 exit angles (131,072 points), four-beam
                           grazing-incidence sum (Section 4.3)
  strained_cube_128.npz    the 102,400-atom strained cube on the 128^3 grid
                           around (004): A of Eq. 2 at every point, I_obs of
                           the perturbed copy, the misfit L, the analytic
                           gradient and central differences for 50 seeded
                           atoms
  sphere_subgrid.npz       the 134,009-atom strained fcc sphere on the 1/16
                           sub-grid of its 256 x 256 x 64 map around (004):
                           every 4th h and every 4th k, all l (262,144
                           points), A of Eq. 2
  ewald_batch_sample.npz   the 64-crystal Ewald-slice batch: full maps of the
                           instances with N_b M_b <= 2e8 and a seeded 1 %
                           (at least 1024 points) of every other instance's
                           points
"""
from __future__ import annotations

import argparse
import json
import pathlib
import sys
import time

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
ROOT = HERE.parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1010_2641_gb300 import workloads as W  # noqa: E402

SCRIPT = "tests/golden/make_golden.py"
A_LAT = W.LATTICE_A

# island sub-grid: every 8th h and k of the 512 x 512 x 32 map
ISLAND_STRIDE = 8
# strained cube: 50 seeded atoms for the gradient checks
CUBE_SEL_SEED, CUBE_N_SEL, CUBE_FD_H = 4002, 50, 1e-5
CUBE_N, CUBE_STEP = 128, 0.005
# strained sphere: every 4th h and k of the 256 x 256 x 64 map, step 0.002
SPHERE_GRID, SPHERE_STEP, SPHERE_STRIDE = (256, 256, 64), 0.002, 4
# Ewald batch: full maps up to this many pairs, else a 1 % sample
BATCH_FULL_PAIRS, BATCH_FRACTION, BATCH_MIN_POINTS, BATCH_SAMPLE_SEED = 2e8, 0.01, 1024, 3100


def island_subgrid_axes():
    h, k, af = W.gid_axes()
    return h[::ISLAND_STRIDE], k[::ISLAND_STRIDE], af


def cube_axes():
    return [W.linspace_axis(0.0, CUBE_N, step=CUBE_STEP), W.linspace_axis(0.0, CUBE_N, step=CUBE_STEP),
            W.linspace_axis(4.0, CUBE_N, step=CUBE_STEP)]


def sphere_axes():
    n0, n1, n2 = SPHERE_GRID
    return [W.linspace_axis(0.0, n0, step=SPHERE_STEP), W.linspace_axis(0.0, n1, step=SPHERE_STEP),
            W.linspace_axis(4.0, n2, step=SPHERE_STEP)]


def sphere_subgrid_axes():
    h, k, l = sphere_axes()
    return h[::SPHERE_STRIDE], k[::SPHERE_STRIDE], l


def cube_selected_atoms(n_atoms: int) -> np.ndarray:
    return np.sort(np.random.default_rng(CUBE_SEL_SEED).choice(n_atoms, CUBE_N_SEL, replace=False))


def batch_sample(ao, so):
    """(global point indices, per-instance offsets into them, full flags)."""
    idx, off, full = [], [0], []
    for b in range(len(ao) - 1):
        n, m = int(ao[b + 1] - ao[b]), int(so[b + 1] - so[b])
        if n * m <= BATCH_FULL_PAIRS:
            loc = np.arange(m)
            full.append(True)
        else:
            k = min(m, max(BATCH_MIN_POINTS, int(np.ceil(BATCH_FRACTION * m))))
            loc = np.sort(np.random.default_rng(BATCH_SAMPLE_SEED + b).choice(m, k, replace=False))
            full.append(False)
        idx.append(so[b] + loc)
        off.append(off[-1] + len(loc))
    return np.concatenate(idx).astype(np.int32), np.array(off, np.int64), np.array(full)


def _meta(**kw) -> np.ndarray:
    kw.setdefault("script", SCRIPT)
    return np.array(json.dumps(kw, sort_keys=True))


def make_island(out: pathlib.Path) -> None:
    c = W.truncated_pyramid()
    h, k, af = island_subgrid_axes()
    pts = W.grid_points([h, k, af])
    t0 = time.time()
    A = oracle.dwba(c.xyz, pts, c.coef, A_LAT, W.WAVELENGTH_10KEV, W.GID_ALPHA_I, W.GID_DELTA, W.GID_BETA,
                    species=c.species)
    meta = _meta(workload="truncated_pyramid() on gid_axes(), every 8th h and k, all alpha_f",
                 seeds="none (deterministic geometry)", oracle="oracle.dwba", n_atoms=len(c.xyz),
                 shape=[len(h), len(k), len(af)], stride=ISLAND_STRIDE, seconds=round(time.time() - t0, 1),
                 threads=oracle.num_threads())
    np.savez(out, meta=meta, A=A.astype(np.complex64))


def make_cube(out: pathlib.Path) -> None:
    c = W.strained_cube()
    pert = W.perturbed_copy(c)
    S = W.grid_points(cube_axes())
    t0 = time.time()
    I_obs = (np.abs(oracle.amplitude(pert.xyz, S, c.coef, A_LAT, species=pert.species)) ** 2).astype(np.float32)
    A = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    sel = cube_selected_atoms(len(c.xyz))
    L, g = oracle.loss_grad_atoms(c.xyz, S, A, I_obs, c.coef, A_LAT, sel, species=c.species)
    fd = oracle.fd_grad(c.xyz, S, I_obs, c.coef, A_LAT, sel, h=CUBE_FD_H, species=c.species, A=A)
    meta = _meta(workload="strained_cube() (seed 4000), I_obs from perturbed_copy() (seed 4001), "
                          "128^3 grid step 0.005 around (0,0,4)",
                 seeds={"crystal": 4000, "perturbation": 4001, "atoms": CUBE_SEL_SEED},
                 oracle="oracle.amplitude, oracle.loss_grad_atoms, oracle.fd_grad(A=...)",
                 fd_h=CUBE_FD_H, n_atoms=len(c.xyz), seconds=round(time.time() - t0, 1),
                 threads=oracle.num_threads())
    np.savez(out, meta=meta, A=A.astype(np.complex64), I_obs=I_obs, loss=np.float64(L), atoms=sel, grad=g, fd=fd)


def make_sphere(out: pathlib.Path) -> None:
    c = W.fcc_sphere()
    h, k, l = sphere_subgrid_axes()
    pts = W.grid_points([h, k, l])
    t0 = time.time()
    A = oracle.amplitude(c.xyz, pts, c.coef, A_LAT, species=c.species)
    meta = _meta(workload="fcc_sphere() (radius 20 cells, 2 species, seed 2000) on the 256 x 256 x 64 grid "
                          "around (0,0,4), step 0.002, every 4th h and k, all l",
                 seeds={"crystal": 2000}, oracle="oracle.amplitude", n_atoms=len(c.xyz),
                 shape=[len(h), len(k), len(l)], stride=SPHERE_STRIDE, seconds=round(time.time() - t0, 1),
                 threads=oracle.num_threads())
    np.savez(out, meta=meta, A=A.astype(np.complex64))


def make_batch(out: pathlib.Path) -> None:
    xyz, sp, coef, S, ao, so = W.ewald_batch()
    idx, off, full = batch_sample(ao, so)
    t0 = time.time()
    vals = []
    for b in range(len(ao) - 1):
        a0, a1 = ao[b], ao[b + 1]
        vals.append(oracle.amplitude(xyz[a0:a1], S[idx[off[b]:off[b + 1]]], coef, A_LAT, species=sp[a0:a1]))
    meta = _meta(workload="ewald_batch() (seed 3000)", seeds={"batch": 3000, "samples": f"{BATCH_SAMPLE_SEED} + b"},
                 oracle="oracle.amplitude per instance", full_pairs=BATCH_FULL_PAIRS, fraction=BATCH_FRACTION,
                 min_points=BATCH_MIN_POINTS, n_full=int(full.sum()), seconds=round(time.time() - t0, 1),
                 threads=oracle.num_threads())
    np.savez(out, meta=meta, idx=idx, off=off, full=full, A=np.concatenate(vals).astype(np.complex64))


JOBS = {"batch": ("ewald_batch_sample.npz", make_batch), "island": ("island_gid_subgrid.npz", make_island),
        "cube": ("strained_cube_128.npz", make_cube), "sphere": ("sphere_subgrid.npz", make_sphere)}


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--only", choices=sorted(JOBS), action="append")
    ap.add_argument("--threads", type=int, default=0)
    args = ap.parse_args()
    oracle.set_threads(args.threads)
    for name in args.only or list(JOBS):
        fname, fn = JOBS[name]
        t0 = time.time()
        fn(HERE / fname)
        print(f"{fname}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
