"""scatter_amplitude_host: host positions in, host map out, through the C ABI.

On SEPARABLE grid plans the final reduction runs in row ranges and each
range is copied to the host on the plan's second stream while the next is
reduced; other plans copy the map after the forward.  Each case compares
the host map with the FP64 oracle (the path's own tolerance) and with the
device-buffer call on the same plan element by element (the same kernels on
the same inputs: bitwise equal).
"""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from closed_forms import rel_l2
from paper_1010_2641_gb300 import api
from paper_1010_2641_gb300 import binding as B
from paper_1010_2641_gb300 import workloads as W

pytestmark = pytest.mark.gpu
A_LAT = W.LATTICE_A


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _device_map(plan, xyz, occ=None):
    A = plan.amplitude(torch.tensor(xyz, dtype=torch.float64, device="cuda:0"),
                       None if occ is None else torch.tensor(occ, dtype=torch.float32, device="cuda:0"))
    plan.check()
    return A.cpu()


# n0 = 40 -> 80 map rows -> three 32-row blocks: three ragged copy ranges;
# n0 = 3 -> one block: one range; n0 = 128 -> eight blocks in eight ranges;
# n0 = 384 -> three M-tile pairs: the contraction's last pair runs on the
# plan's side stream beside the CTA-pair kernel, then the ranges are copied
@pytest.mark.parametrize("shape", [(40, 12, 20), (3, 33, 17), (128, 16, 8), (384, 4, 9)])
def test_separable_grid_ranges_copied_while_reducing(shape):
    c = W.fcc_sphere(radius_cells=4.5, seed=71)
    occ = np.random.default_rng(72).uniform(0.5, 1.0, len(c.xyz)).astype(np.float32)
    axes = [W.linspace_axis(0.0, shape[0], step=0.004), W.linspace_axis(0.0, shape[1], step=0.004),
            W.linspace_axis(4.0, shape[2], step=0.004)]
    S = W.grid_points(axes)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    xyz_h = torch.tensor(c.xyz, dtype=torch.float64).pin_memory()
    occ_h = torch.tensor(occ).pin_memory()
    out = plan.amplitude_host(xyz_h, occ_h)
    torch.cuda.synchronize()
    plan.check()
    assert out.device.type == "cpu" and out.is_pinned()
    dev = _device_map(plan, c.xyz, occ)
    assert torch.equal(out, dev)
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species, occ=occ)
    assert rel_l2(out.numpy().astype(np.complex128), ref) < 1e-3


def test_generic_list_with_pageable_buffers():
    c = W.fcc_sphere(radius_cells=3.5, seed=73)
    S = W.ewald_slice(3001, seed=74)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    out = torch.zeros(len(S), dtype=torch.complex64)  # pageable
    plan.amplitude_host(c.xyz, out=out)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, _device_map(plan, c.xyz))
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(out.numpy().astype(np.complex128), ref) < 1e-4
    # a second call into the same buffer (the plan's staging is reused)
    moved = c.xyz + np.array([0.25, -0.5, 1.0])
    plan.amplitude_host(moved, out=out)
    torch.cuda.synchronize()
    ref2 = oracle.amplitude(moved, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(out.numpy().astype(np.complex128), ref2) < 1e-4


def test_bench_map_sixteen_ranges_equal_the_device_call():
    c = W.fcc_sphere()
    axes = [W.linspace_axis(0.0, 256, step=0.002), W.linspace_axis(0.0, 256, step=0.002),
            W.linspace_axis(4.0, 64, step=0.002)]
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, path="separable")
    xyz_h = torch.tensor(c.xyz, dtype=torch.float64).pin_memory()
    out = plan.amplitude_host(xyz_h)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, _device_map(plan, c.xyz))
    # sampled points against the oracle (the map's 1e-4 metric tolerance)
    idx = np.sort(np.random.default_rng(75).choice(256 * 256 * 64, 2048, replace=False))
    S = W.grid_points(axes)[idx]
    ref = oracle.amplitude(c.xyz, S, c.coef, A_LAT, species=c.species)
    assert rel_l2(out.numpy()[idx].astype(np.complex128), ref) < 1e-4


def test_rejects_device_buffers():
    c = W.fcc_sphere(radius_cells=2.5, seed=76)
    S = W.ewald_slice(100, seed=77)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), s_list=S, atom_species=c.species)
    with pytest.raises(ValueError):
        plan.amplitude_host(torch.tensor(c.xyz, dtype=torch.float64, device="cuda:0"))
    # the C ABI itself: a device map pointer is INVALID_ARG
    xyz_h = torch.tensor(c.xyz, dtype=torch.float64)
    A_dev = torch.empty(len(S), dtype=torch.complex64, device="cuda:0")
    st = B.lib().scatter_amplitude_host(plan._h, ctypes.c_void_p(xyz_h.data_ptr()), None,
                                        ctypes.c_void_p(A_dev.data_ptr()), None)
    assert st == 1  # SCATTER_ERR_INVALID_ARG
    st = B.lib().scatter_amplitude_host(plan._h, None, None, ctypes.c_void_p(A_dev.data_ptr()), None)
    assert st == 1


@pytest.mark.parametrize("path,tol", [("separable", 1e-3), ("generic", 1e-4)])
def test_grazing_incidence_map(path, tol):
    """GID plans copy the map after the forward (the separable route's beams
    are combined after the reduction, so its map is not copied in ranges)."""
    c = W.truncated_pyramid(base_cells=12, height_cells=5, top_cells=4)
    axes = [np.linspace(3.8, 4.05, 24), np.linspace(-0.125, 0.125, 20), np.deg2rad((np.arange(32) + 1) / 32)]
    gid = dict(wavelength=W.WAVELENGTH_10KEV, alpha_i=W.GID_ALPHA_I, delta=W.GID_DELTA, beta=W.GID_BETA)
    plan = api.Plan(c.coef, A_LAT, len(c.xyz), axes=axes, atom_species=c.species, gid=gid, path=path)
    out = plan.amplitude_host(torch.tensor(c.xyz, dtype=torch.float64).pin_memory())
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, _device_map(plan, c.xyz))
    ref = oracle.dwba(c.xyz, W.grid_points(axes), c.coef, A_LAT, W.WAVELENGTH_10KEV, W.GID_ALPHA_I, W.GID_DELTA,
                      W.GID_BETA, species=c.species)
    assert rel_l2(out.numpy().astype(np.complex128), ref) < tol


def test_batch_of_uneven_instances():
    """A batch (persistent launch, per-instance offsets) through the host call;
    every instance against the oracle."""
    xyzs, sps, Ss = [], [], []
    for b, (r, m) in enumerate([(2.5, 700), (4.0, 1500), (1.5, 300)]):
        c = W.fcc_sphere(radius_cells=r, seed=80 + b)
        xyzs.append(c.xyz)
        sps.append(c.species)
        Ss.append(W.ewald_slice(m, seed=90 + b))
    coef = W.fcc_sphere(radius_cells=1.5, seed=80).coef
    ao = np.concatenate([[0], np.cumsum([len(x) for x in xyzs])]).astype(np.int64)
    so = np.concatenate([[0], np.cumsum([len(s) for s in Ss])]).astype(np.int64)
    xyz, sp, S = np.concatenate(xyzs), np.concatenate(sps), np.concatenate(Ss)
    plan = api.Plan(coef, A_LAT, len(xyz), s_list=S, atom_species=sp, atom_off=ao, s_off=so)
    out = plan.amplitude_host(xyz)
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(out, _device_map(plan, xyz))
    A = out.numpy().astype(np.complex128)
    for b in range(3):
        ref = oracle.amplitude(xyz[ao[b]:ao[b + 1]], S[so[b]:so[b + 1]], coef, A_LAT, species=sp[ao[b]:ao[b + 1]])
        assert rel_l2(A[so[b]:so[b + 1]], ref) < 1e-4, b
