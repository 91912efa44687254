"""PyTorch front end of libscatter: plans, calls on torch tensors, autograd.

torch provides device memory and streams only; every step of the
computation runs in libscatter's CUDA kernels (binding.py marshals the
arguments).  Tensors must be CUDA tensors on the plan's device:
positions float64 [N, 3] (lattice units), occupancies float32 [N].
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import binding as B

_PATHS = {"auto": B.SCATTER_PATH_AUTO, "generic": B.SCATTER_PATH_GENERIC,
          "separable": B.SCATTER_PATH_SEPARABLE, "fp64": B.SCATTER_PATH_FP64_REF}


def _species_array(coef) -> "ctypes.Array":
    coef = np.asarray(coef, dtype=np.float64).reshape(-1, 12)
    arr = (B.scatter_species * coef.shape[0])()
    for i, row in enumerate(coef):
        arr[i].a[:] = row[0:4]
        arr[i].b[:] = row[4:8]
        arr[i].c, arr[i].fp, arr[i].fpp, arr[i].b_dw = row[8], row[9], row[10], row[11]
    return arr


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Plan:
    """A planned scattering problem (scatter_plan).

    Parameters
    ----------
    coef : [n_species, 12] scattering-factor coefficients
        (a0..a3, b0..b3, c, f', f'', B_dw) per species.
    lattice_a : Angstrom.
    s_list : [M, 3] r.l.u. (list sampling), or
    axes : three 1-D arrays h, k, l (grid sampling; GID: h, k, alpha_f).
    atom_species : [N] int (or None: all species 0); n_atoms : N.
    center : reference reflection H (integers) or None (automatic).
    gid : dict(wavelength=, alpha_i=, delta=, beta=[, buried=True]) for grazing
        incidence; buried=True: the object lies in the substrate below the
        surface plane z = 0 (one transmitted beam), else on it (four beams).
    atom_off, s_off : batch CSR offsets (lists only).
    factor_table : [n_species, M] complex (Eq. 4, blocks of atoms): the
        "species" are block types with structure factors F_t(S_m) given per
        output point; positions are the displaced block origins.
    atoms_per_thread : generic path, one instance: 1/2/4/8/16 forces the
        atom-parallel form (for many atoms and few reflections), 0 lets the
        heuristic or autotuner choose, -1 keeps the S-parallel kernel.
    path : "auto" (default), "generic", "separable" or "fp64".  With "auto" a
        grid plan takes the separable tensor-core path when the grid is large
        enough and its error model (with a measured margin) meets `tolerance`
        (relative L2 of the map, 0 = 1e-4) for crystals of `radius_hint`
        lattice units around their centre (0 = compact); otherwise generic.
    """

    def __init__(self, coef, lattice_a: float, n_atoms: int, *, s_list=None, axes: Sequence | None = None,
                 atom_species=None, center=None, path: str = "auto", gid: dict | None = None,
                 atom_off=None, s_off=None, autotune: bool = False, tune_cache: str | None = None,
                 threads: int = 0, points_per_thread: int = 0, split_k: int = 0, use_graph: bool = True,
                 timing: bool = False, atoms_per_thread: int = 0, factor_table=None, tolerance: float = 0.0,
                 radius_hint: float = 0.0):
        L = B.lib()
        self._keep = []
        pr = B.scatter_problem()
        coef = np.asarray(coef, dtype=np.float64).reshape(-1, 12)
        sp = _species_array(coef)
        self._keep.append(sp)
        pr.n_atoms = int(n_atoms)
        pr.n_species = coef.shape[0]
        pr.species = sp
        if atom_species is not None:
            a = np.ascontiguousarray(np.asarray(atom_species, dtype=np.int32).reshape(-1))
            if a.shape[0] != n_atoms:
                raise ValueError("atom_species must have n_atoms entries")
            self._keep.append(a)
            pr.atom_species = a.ctypes.data
        pr.lattice_a = float(lattice_a)
        if s_list is not None:
            s = np.ascontiguousarray(np.asarray(s_list, dtype=np.float64).reshape(-1, 3))
            self._keep.append(s)
            pr.s_kind = B.SCATTER_S_LIST
            pr.n_s = s.shape[0]
            pr.s_list = s.ctypes.data if s.size else None
            self.shape = (s.shape[0],)
        elif axes is not None:
            pr.s_kind = B.SCATTER_S_GID_GRID if gid else B.SCATTER_S_GRID
            shape = []
            for d in range(3):
                ax = np.ascontiguousarray(np.asarray(axes[d], dtype=np.float64).reshape(-1))
                self._keep.append(ax)
                pr.axis[d] = ax.ctypes.data
                pr.n_axis[d] = ax.shape[0]
                shape.append(ax.shape[0])
            self.shape = tuple(shape)
        else:
            raise ValueError("give s_list or axes")
        if center is not None:
            pr.center_mode = 1
            pr.center_hkl[:] = [float(c) for c in center]
        if gid:
            pr.wavelength = float(gid["wavelength"])
            pr.alpha_i = float(gid["alpha_i"])
            pr.delta = float(gid.get("delta", 0.0))
            pr.beta = float(gid.get("beta", 0.0))
            pr.gid_mode = 1 if gid.get("buried", False) else 0
        pr.batch = 1
        if atom_off is not None:
            ao = np.ascontiguousarray(np.asarray(atom_off, dtype=np.int64))
            so = np.ascontiguousarray(np.asarray(s_off, dtype=np.int64))
            self._keep += [ao, so]
            pr.batch = ao.shape[0] - 1
            pr.atom_off = ao.ctypes.data
            pr.s_off = so.ctypes.data
        if factor_table is not None:
            m = int(np.prod(self.shape))
            ft = np.asarray(factor_table, dtype=np.complex128).reshape(coef.shape[0], m)
            ft2 = np.ascontiguousarray(np.stack([ft.real, ft.imag], -1))
            self._keep.append(ft2)
            pr.factor_table = ft2.ctypes.data
        op = B.scatter_options()
        op.path = _PATHS[path]
        op.autotune = int(bool(autotune))
        self._cache = tune_cache.encode() if tune_cache else None
        op.tune_cache = self._cache
        op.threads, op.points_per_thread, op.split_k = threads, points_per_thread, split_k
        op.use_graph = 0 if use_graph else -1
        op.timing = int(bool(timing))
        op.atoms_per_thread = int(atoms_per_thread)
        op.tolerance = float(tolerance)
        op.radius_hint = float(radius_hint)
        h = ctypes.c_void_p()
        B.check(L.scatter_plan(ctypes.byref(pr), ctypes.byref(op), ctypes.byref(h)), "scatter_plan")
        self._h = h
        self.n_atoms = int(n_atoms)
        self.n_s = int(np.prod(self.shape))
        self.device = torch.cuda.current_device()

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            B.lib().scatter_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- checks -----------------------------------------------------------
    def _xyz(self, xyz: torch.Tensor) -> torch.Tensor:
        if xyz.dtype != torch.float64 or not xyz.is_cuda or xyz.shape != (self.n_atoms, 3):
            raise ValueError(f"xyz must be a CUDA float64 tensor of shape ({self.n_atoms}, 3)")
        return xyz.contiguous()

    def _occ(self, occ):
        if occ is None:
            return None
        if occ.dtype != torch.float32 or not occ.is_cuda or occ.numel() != self.n_atoms:
            raise ValueError("occ must be a CUDA float32 tensor with n_atoms entries")
        return occ.contiguous()

    # -- calls -----------------------------------------------------------------
    def amplitude(self, xyz, occ=None, out=None, stream=None) -> torch.Tensor:
        xyz, occ = self._xyz(xyz), self._occ(occ)
        if out is None:
            out = torch.empty(self.n_s, dtype=torch.complex64, device=xyz.device)
        B.check(B.lib().scatter_amplitude(self._h, _ptr(xyz), _ptr(occ), _ptr(out), _stream(stream)),
                "scatter_amplitude")
        return out

    def amplitude_host(self, xyz, occ=None, out=None, stream=None) -> torch.Tensor:
        """A(S) from host positions into a host map (scatter_amplitude_host).

        `xyz` is a CPU float64 [N, 3] tensor or array (pinned for an
        asynchronous call), `out` a CPU complex64 [n_s] tensor (allocated
        pinned if not given).  The call enqueues on `stream`; synchronise it
        before reading `out`."""
        x = torch.as_tensor(xyz, dtype=torch.float64)
        if x.device.type != "cpu":
            raise ValueError("amplitude_host takes host positions; use amplitude for device tensors")
        x = x.contiguous()
        if x.shape != (self.n_atoms, 3):
            raise ValueError(f"xyz must be [{self.n_atoms}, 3]")
        o = None
        if occ is not None:
            o = torch.as_tensor(occ, dtype=torch.float32).contiguous()
            if o.device.type != "cpu" or o.shape != (self.n_atoms,):
                raise ValueError(f"occ must be a host [{self.n_atoms}] tensor")
        if out is None:
            out = torch.empty(self.n_s, dtype=torch.complex64).pin_memory()
        elif out.device.type != "cpu" or out.dtype != torch.complex64 or out.numel() != self.n_s \
                or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous host complex64 [{self.n_s}] tensor")
        B.check(B.lib().scatter_amplitude_host(self._h, _ptr(x), _ptr(o), _ptr(out), _stream(stream)),
                "scatter_amplitude_host")
        return out

    def intensity(self, xyz, occ=None, out=None, stream=None) -> torch.Tensor:
        xyz, occ = self._xyz(xyz), self._occ(occ)
        if out is None:
            out = torch.empty(self.n_s, dtype=torch.float32, device=xyz.device)
        B.check(B.lib().scatter_intensity(self._h, _ptr(xyz), _ptr(occ), _ptr(out), _stream(stream)),
                "scatter_intensity")
        return out

    def backward(self, xyz, A, I_obs, occ=None, want_grad=True, stream=None):
        """(loss [float64 scalar tensor], dL/dxyz [N,3] float32 or None)."""
        xyz, occ = self._xyz(xyz), self._occ(occ)
        loss = torch.empty((), dtype=torch.float64, device=xyz.device)
        grad = torch.empty(self.n_atoms, 3, dtype=torch.float32, device=xyz.device) if want_grad else None
        A = A.contiguous()
        I_obs = I_obs.contiguous()
        B.check(B.lib().scatter_backward(self._h, _ptr(xyz), _ptr(occ), _ptr(A), _ptr(I_obs), _ptr(loss),
                                         _ptr(grad), _stream(stream)), "scatter_backward")
        return loss, grad

    def vjp(self, xyz, G, occ=None, stream=None) -> torch.Tensor:
        xyz, occ = self._xyz(xyz), self._occ(occ)
        grad = torch.empty(self.n_atoms, 3, dtype=torch.float32, device=xyz.device)
        G = G.to(torch.complex64).contiguous()
        B.check(B.lib().scatter_vjp(self._h, _ptr(xyz), _ptr(occ), _ptr(G), _ptr(grad), _stream(stream)),
                "scatter_vjp")
        return grad

    def check(self, stream=None) -> None:
        B.check(B.lib().scatter_check(self._h, _stream(stream)), "scatter_check")

    def selftest_wait(self, stream=None) -> None:
        """Enqueue the device self-check of the bounded waits (the next check()
        raises SCATTER_ERR_TIMEOUT)."""
        B.check(B.lib().scatter_selftest_wait(self._h, _stream(stream)), "scatter_selftest_wait")

    def info(self) -> dict:
        inf = B.scatter_plan_info()
        B.check(B.lib().scatter_plan_get_info(self._h, ctypes.byref(inf)), "scatter_plan_get_info")
        return {k: (list(getattr(inf, k)) if k in ("center_hkl", "shift") else getattr(inf, k))
                for k, _ in B.scatter_plan_info._fields_}

    def timing(self):
        """(ms of the main kernel of the last call, kernels launched by it)."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        B.check(B.lib().scatter_plan_timing(self._h, ctypes.byref(ms), ctypes.byref(n)), "scatter_plan_timing")
        return ms.value, n.value

    def error_bound(self, radius: float):
        a, b = ctypes.c_double(), ctypes.c_double()
        B.check(B.lib().scatter_error_bound(self._h, float(radius), ctypes.byref(a), ctypes.byref(b)),
                "scatter_error_bound")
        return a.value, b.value


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class ScatterAmplitude(torch.autograd.Function):
    """A = amplitude(xyz); backward through scatter_vjp."""

    @staticmethod
    def forward(ctx, xyz, plan: Plan, occ=None):
        ctx.plan = plan
        ctx.save_for_backward(xyz, occ) if occ is not None else ctx.save_for_backward(xyz)
        return plan.amplitude(xyz.detach(), occ)

    @staticmethod
    def backward(ctx, G):
        saved = ctx.saved_tensors
        xyz = saved[0]
        occ = saved[1] if len(saved) > 1 else None
        grad = ctx.plan.vjp(xyz.detach(), G, occ)
        return grad.to(xyz.dtype), None, None


class ScatterLoss(torch.autograd.Function):
    """L = sum (|A|^2 - I_obs)^2 with the fused adjoint kernel."""

    @staticmethod
    def forward(ctx, xyz, plan: Plan, I_obs, occ=None):
        A = plan.amplitude(xyz.detach(), occ)
        loss, _ = plan.backward(xyz.detach(), A, I_obs, occ, want_grad=False)
        ctx.plan = plan
        ctx.save_for_backward(xyz, A, I_obs, *( [occ] if occ is not None else []))
        return loss

    @staticmethod
    def backward(ctx, gL):
        xyz, A, I_obs, *rest = ctx.saved_tensors
        occ = rest[0] if rest else None
        _, grad = ctx.plan.backward(xyz.detach(), A, I_obs, occ, want_grad=True)
        return (grad.to(xyz.dtype) * gL.to(xyz.dtype)), None, None, None


def amplitude(xyz, plan: Plan, occ=None):
    return ScatterAmplitude.apply(xyz, plan, occ)


def misfit(xyz, plan: Plan, I_obs, occ=None):
    return ScatterLoss.apply(xyz, plan, I_obs, occ)


def microbench(kind: int, iters: int = 20000) -> dict:
    r = B.scatter_microbench_result()
    B.check(B.lib().scatter_microbench(int(kind), int(iters), ctypes.byref(r)), "scatter_microbench")
    return {"ops_per_s": r.ops_per_s, "ops_per_clk_per_sm": r.ops_per_clk_per_sm, "sm_clock_hz": r.sm_clock_hz,
            "seconds": r.seconds, "n_sm": r.n_sm}


class FFTPlan:
    """Eq. 5/6: the FFT approximation (scatter_fft_*).

    Atoms go to the nearest node of a grid of `step` (lattice units) from
    `origin` with `n` nodes per axis; A is returned on the grid
    S = H + q, q_d = (i - n_d // 2) / (n_d step) (see axes()), valid while
    |(S - H).u| << 1 (Eq. 7: validity()).
    """

    def __init__(self, coef, lattice_a: float, n_atoms: int, *, center, step: float, origin, n):
        coef = np.asarray(coef, dtype=np.float64).reshape(-1, 12)
        self._species = _species_array(coef)
        pr = B.scatter_fft_problem()
        pr.n_atoms = int(n_atoms)
        pr.n_species = coef.shape[0]
        pr.species = ctypes.addressof(self._species)
        pr.lattice_a = float(lattice_a)
        pr.center_hkl[:] = [float(c) for c in center]
        pr.step = float(step)
        pr.origin[:] = [float(o) for o in origin]
        pr.n[:] = [int(k) for k in n]
        self.center = np.asarray(center, dtype=np.float64)
        self.step = float(step)
        self.n = tuple(int(k) for k in n)
        self.n_atoms = int(n_atoms)
        h = ctypes.c_void_p()
        B.check(B.lib().scatter_fft_plan(ctypes.byref(pr), ctypes.byref(h)), "scatter_fft_plan")
        self._h = h

    def axes(self):
        """The three S axes of the output grid (r.l.u.)."""
        return [self.center[d] + (np.arange(self.n[d]) - self.n[d] // 2) / (self.n[d] * self.step)
                for d in range(3)]

    def amplitude(self, xyz: torch.Tensor, atom_species: Optional[torch.Tensor] = None,
                  occ: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        assert xyz.dtype == torch.float64 and xyz.is_cuda and xyz.is_contiguous() and xyz.shape[0] == self.n_atoms
        sp = None if atom_species is None else atom_species.to(torch.int32).contiguous()
        w = None if occ is None else occ.to(torch.float32).contiguous()
        if out is None:
            out = torch.empty(self.n, dtype=torch.complex64, device=xyz.device)
        B.check(B.lib().scatter_fft_amplitude(self._h, _ptr(xyz), _ptr(sp), _ptr(w), out.data_ptr(),
                                              _stream(stream)), "scatter_fft_amplitude")
        return out

    def validity(self):
        """(max over atoms and grid of |(S - H).u|, atoms outside the grid) of the last call."""
        m, k = ctypes.c_double(), ctypes.c_int64()
        B.check(B.lib().scatter_fft_validity(self._h, ctypes.byref(m), ctypes.byref(k)), "scatter_fft_validity")
        return m.value, k.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            B.lib().scatter_fft_plan_destroy(h)
            self._h = None
