"""FP64 CPU oracle of the direct kinematic scattering sum.

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never imports it, and this package imports nothing from the library.

The arithmetic lives in ``scatter_oracle.c`` (plain loops in double precision,
OpenMP over reflections); this module compiles it with gcc into
``oracle/lib/liboracle.so`` and wraps it with ctypes and numpy.

Every function below follows the paper's definitions:
  amplitude    Eq. 2 with occupancies (Section 3) and per-species factors
               (Section 4.2)
  fresnel      substrate reflection/transmission (Section 3, pynx.gid)
  dwba         four-beam grazing-incidence sum (Section 4.3; the formula is a
               reading, the paper prints none)
  dwba_buried  the same geometry for an object inside the substrate: one
               transmitted beam, refracted and attenuated (a reading too)
  loss_grad    L = sum (|A|^2 - I_obs)^2 and its analytic gradient
  fd_grad      central finite differences of L (a second route to the gradient)
  loss_grad_table  L and the analytic gradient of Eq. 4 (block origins, F fixed)
  loss_grad_atoms  L and the analytic gradient of selected atoms from a map
               the caller already has (large maps summed once)
"""
from __future__ import annotations

import ctypes
import os
import pathlib
import subprocess

import numpy as np

HERE = pathlib.Path(__file__).resolve().parent
SRC = HERE / "scatter_oracle.c"
LIBDIR = HERE / "lib"
LIB = LIBDIR / "liboracle.so"

NCOEF = 12  # a0..a3, b0..b3, c, f', f'', B_dw

_lib = None


def build(force: bool = False) -> pathlib.Path:
    """Compile the oracle with gcc -O2 -fopenmp (no -ffast-math)."""
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        LIBDIR.mkdir(parents=True, exist_ok=True)
        tmp = LIBDIR / f"liboracle.{os.getpid()}.so"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(tmp), str(SRC), "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        lib.oracle_amplitude.argtypes = [i64, P, P, P, i32, P, f64, i64, P, P]
        lib.oracle_form_factor.argtypes = [P, f64, P, P]
        lib.oracle_amplitude_table.argtypes = [i64, P, P, P, i32, P, i64, P, P]
        lib.oracle_fft_approx.argtypes = [i64, P, P, P, i32, P, f64, P, f64, P, i64, P, P]
        lib.oracle_fresnel.argtypes = [f64, f64, f64, P, P]
        lib.oracle_dwba.argtypes = [i64, P, P, P, i32, P, f64, f64, f64, f64, f64, i64, P, P]
        lib.oracle_dwba_buried.argtypes = [i64, P, P, P, i32, P, f64, f64, f64, f64, f64, i64, P, P]
        lib.oracle_loss_grad.argtypes = [i64, P, P, P, i32, P, f64, i64, P, P, P, P]
        lib.oracle_fd_grad.argtypes = [i64, P, P, P, i32, P, f64, i64, P, P, i64, P, f64, P]
        lib.oracle_loss_grad_table.argtypes = [i64, P, P, P, i32, P, i64, P, P, P, P]
        lib.oracle_loss_grad_given_amplitude.argtypes = [i64, P, P, P, i32, P, f64, i64, P, P, P, i64, P, P, P]
        lib.oracle_fd_grad_given_amplitude.argtypes = [i64, P, P, P, i32, P, f64, i64, P, P, P, i64, P, f64, P]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_threads.restype = None
        _lib = lib
    return _lib


def _f64(a, shape_last=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_last is not None:
        a = a.reshape(-1, shape_last)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _atoms(xyz, species, occ, coef):
    xyz = _f64(xyz, 3)
    n = xyz.shape[0]
    sp = None if species is None else np.ascontiguousarray(np.asarray(species, dtype=np.int32).reshape(n))
    w = None if occ is None else _f64(occ).reshape(n)
    coef = _f64(coef, NCOEF)
    if sp is not None and n and (sp.min() < 0 or sp.max() >= coef.shape[0]):
        raise ValueError("species index out of range")
    return xyz, sp, w, coef


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> None:
    """Thread count of later oracle calls (n < 1: the OpenMP default)."""
    _load().oracle_set_threads(int(n))


def form_factor(coef, q_inv_angstrom: float) -> complex:
    """f(|S|) of one species; q = |S| in 1/Angstrom."""
    c = _f64(coef).reshape(NCOEF)
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().oracle_form_factor(_ptr(c), float(q_inv_angstrom), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def amplitude(xyz, S, coef, lattice_a, species=None, occ=None) -> np.ndarray:
    """A(S) of Eq. 2 for S [M,3] (r.l.u.), positions [N,3] (lattice units)."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    S = _f64(S, 3)
    out = np.zeros((S.shape[0], 2))
    _load().oracle_amplitude(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                             float(lattice_a), S.shape[0], _ptr(S), _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def amplitude_table(xyz, S, table, types=None, occ=None) -> np.ndarray:
    """Eq. 4: A(S) = sum_j w_j F_{t(j)}(S) exp(2 i pi S.r_j) with a complex
    factor table F [n_types, M] (block structure factors)."""
    xyz = _f64(xyz, 3)
    n = xyz.shape[0]
    t = None if types is None else np.ascontiguousarray(np.asarray(types, dtype=np.int32).reshape(n))
    w = None if occ is None else _f64(occ).reshape(n)
    S = _f64(S, 3)
    tab = np.asarray(table, dtype=np.complex128).reshape(-1, S.shape[0])
    if t is not None and n and (t.min() < 0 or t.max() >= tab.shape[0]):
        raise ValueError("type index out of range")
    tab2 = np.ascontiguousarray(np.stack([tab.real, tab.imag], -1))
    out = np.zeros((S.shape[0], 2))
    _load().oracle_amplitude_table(n, _ptr(xyz), _ptr(t), _ptr(w), tab.shape[0], _ptr(tab2), S.shape[0], _ptr(S),
                                   _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def fft_approx(xyz, S, coef, lattice_a, H, step, origin, species=None, occ=None) -> np.ndarray:
    """Eq. 5/6: atoms on the nearest node R_j of a grid of step `step` from
    `origin`, exp(2 i pi (S-H).u_j) dropped, as a direct sum at S [M, 3]."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    S = _f64(S, 3)
    Hv = _f64(np.asarray(H, dtype=np.float64), 3).reshape(3)
    ov = _f64(np.asarray(origin, dtype=np.float64), 3).reshape(3)
    out = np.zeros((S.shape[0], 2))
    _load().oracle_fft_approx(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                              float(lattice_a), _ptr(Hv), float(step), _ptr(ov), S.shape[0], _ptr(S), _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def fresnel(alpha: float, delta: float, beta: float) -> tuple[complex, complex]:
    R = np.zeros(2)
    T = np.zeros(2)
    _load().oracle_fresnel(float(alpha), float(delta), float(beta), _ptr(R), _ptr(T))
    return complex(R[0], R[1]), complex(T[0], T[1])


def dwba(xyz, pts, coef, lattice_a, wavelength, alpha_i, delta, beta, species=None, occ=None) -> np.ndarray:
    """Four-term DWBA amplitude at points (h, k, alpha_f) [M,3]."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    pts = _f64(pts, 3)
    out = np.zeros((pts.shape[0], 2))
    _load().oracle_dwba(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                        float(lattice_a), float(wavelength), float(alpha_i), float(delta), float(beta),
                        pts.shape[0], _ptr(pts), _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def dwba_buried(xyz, pts, coef, lattice_a, wavelength, alpha_i, delta, beta, species=None, occ=None) -> np.ndarray:
    """Grazing-incidence amplitude of an object buried in the substrate
    (z <= 0): one transmitted beam, T_i T_f, refracted and attenuated in the
    medium, at points (h, k, alpha_f) [M,3]."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    pts = _f64(pts, 3)
    out = np.zeros((pts.shape[0], 2))
    _load().oracle_dwba_buried(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                               float(lattice_a), float(wavelength), float(alpha_i), float(delta), float(beta),
                               pts.shape[0], _ptr(pts), _ptr(out))
    return out[:, 0] + 1j * out[:, 1]


def loss_grad(xyz, S, I_obs, coef, lattice_a, species=None, occ=None, grad=True):
    """(L, dL/dr [N,3] or None) for L = sum (|A|^2 - I_obs)^2."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    S = _f64(S, 3)
    I_obs = _f64(I_obs).reshape(S.shape[0])
    loss = ctypes.c_double()
    g = np.zeros((xyz.shape[0], 3)) if grad else None
    _load().oracle_loss_grad(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                             float(lattice_a), S.shape[0], _ptr(S), _ptr(I_obs), ctypes.byref(loss), _ptr(g))
    return loss.value, g


def _amp2(A, n_s):
    A = np.asarray(A, dtype=np.complex128).reshape(n_s)
    return np.ascontiguousarray(np.stack([A.real, A.imag], -1))


def fd_grad(xyz, S, I_obs, coef, lattice_a, atoms, h=1e-5, species=None, occ=None, A=None) -> np.ndarray:
    """Central-difference gradient of L for the selected atoms, [len(atoms),3].
    A: the unperturbed map from ``amplitude`` (computed here when None)."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    S = _f64(S, 3)
    I_obs = _f64(I_obs).reshape(S.shape[0])
    sel = np.ascontiguousarray(np.asarray(atoms, dtype=np.int64))
    out = np.zeros((sel.shape[0], 3))
    if A is None:
        _load().oracle_fd_grad(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                               float(lattice_a), S.shape[0], _ptr(S), _ptr(I_obs), sel.shape[0], _ptr(sel),
                               float(h), _ptr(out))
    else:
        A2 = _amp2(A, S.shape[0])
        _load().oracle_fd_grad_given_amplitude(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0],
                                               _ptr(coef), float(lattice_a), S.shape[0], _ptr(S), _ptr(A2),
                                               _ptr(I_obs), sel.shape[0], _ptr(sel), float(h), _ptr(out))
    return out


def loss_grad_table(xyz, S, I_obs, table, types=None, occ=None, grad=True):
    """(L, dL/dr [N,3] or None) of Eq. 4: blocks with the complex factor
    table F [n_types, M] held fixed, positions the block origins."""
    xyz = _f64(xyz, 3)
    n = xyz.shape[0]
    t = None if types is None else np.ascontiguousarray(np.asarray(types, dtype=np.int32).reshape(n))
    w = None if occ is None else _f64(occ).reshape(n)
    S = _f64(S, 3)
    I_obs = _f64(I_obs).reshape(S.shape[0])
    tab = np.asarray(table, dtype=np.complex128).reshape(-1, S.shape[0])
    tab2 = np.ascontiguousarray(np.stack([tab.real, tab.imag], -1))
    loss = ctypes.c_double()
    g = np.zeros((n, 3)) if grad else None
    _load().oracle_loss_grad_table(n, _ptr(xyz), _ptr(t), _ptr(w), tab.shape[0], _ptr(tab2), S.shape[0], _ptr(S),
                                   _ptr(I_obs), ctypes.byref(loss), _ptr(g))
    return loss.value, g


def loss_grad_atoms(xyz, S, A, I_obs, coef, lattice_a, atoms, species=None, occ=None):
    """(L, dL/dr [len(atoms),3]) from a map A the caller already has (the
    output of ``amplitude``): the formula of ``loss_grad`` for selected atoms."""
    xyz, sp, w, coef = _atoms(xyz, species, occ, coef)
    S = _f64(S, 3)
    I_obs = _f64(I_obs).reshape(S.shape[0])
    A2 = _amp2(A, S.shape[0])
    sel = np.ascontiguousarray(np.asarray(atoms, dtype=np.int64))
    loss = ctypes.c_double()
    g = np.zeros((sel.shape[0], 3))
    _load().oracle_loss_grad_given_amplitude(xyz.shape[0], _ptr(xyz), _ptr(sp), _ptr(w), coef.shape[0], _ptr(coef),
                                             float(lattice_a), S.shape[0], _ptr(S), _ptr(A2), _ptr(I_obs),
                                             sel.shape[0], _ptr(sel), ctypes.byref(loss), _ptr(g))
    return loss.value, g
