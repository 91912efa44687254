"""ctypes binding of libscatter.so — argument marshalling only.

Every entry point of include/scatter.h is exposed under the same name with
the same argument order; structs mirror the C layouts field by field.  The
library is loaded from ``paper_1010_2641_gb300/lib/libscatter.so`` (built in
tree by ``paper_1010_2641_gb300.build``).  If it is missing, ``lib()`` raises:
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import pathlib

_HERE = pathlib.Path(__file__).resolve().parent
LIB_PATH = _HERE / "lib" / "libscatter.so"

c_int32, c_int64, c_double, c_void_p, c_char_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_char_p)

# scatter_status
SCATTER_OK = 0
SCATTER_ERR_INVALID_ARG = 1
SCATTER_ERR_UNSUPPORTED = 2
SCATTER_ERR_OOM = 3
SCATTER_ERR_CUDA = 4
SCATTER_ERR_TIMEOUT = 5
SCATTER_ERR_NUMERIC = 6
SCATTER_ERR_NO_DEVICE = 7

# scatter_s_kind
SCATTER_S_LIST = 0
SCATTER_S_GRID = 1
SCATTER_S_GID_GRID = 2

# scatter_path
SCATTER_PATH_AUTO = 0
SCATTER_PATH_GENERIC = 1
SCATTER_PATH_SEPARABLE = 2
SCATTER_PATH_FP64_REF = 3


class scatter_species(ctypes.Structure):
    _fields_ = [("a", c_double * 4), ("b", c_double * 4), ("c", c_double), ("fp", c_double),
                ("fpp", c_double), ("b_dw", c_double)]


class scatter_problem(ctypes.Structure):
    _fields_ = [
        ("n_atoms", c_int64),
        ("n_species", c_int32),
        ("species", ctypes.POINTER(scatter_species)),
        ("atom_species", c_void_p),
        ("lattice_a", c_double),
        ("s_kind", c_int32),
        ("n_s", c_int64),
        ("s_list", c_void_p),
        ("axis", c_void_p * 3),
        ("n_axis", c_int64 * 3),
        ("center_mode", c_int32),
        ("center_hkl", c_double * 3),
        ("wavelength", c_double),
        ("alpha_i", c_double),
        ("delta", c_double),
        ("beta", c_double),
        ("batch", c_int32),
        ("atom_off", c_void_p),
        ("s_off", c_void_p),
        ("factor_table", c_void_p),
        ("gid_mode", c_int32),
    ]


class scatter_options(ctypes.Structure):
    _fields_ = [("path", c_int32), ("autotune", c_int32), ("tune_cache", c_char_p), ("threads", c_int32),
                ("points_per_thread", c_int32), ("split_k", c_int32), ("use_graph", c_int32), ("timing", c_int32),
                ("atoms_per_thread", c_int32), ("tolerance", c_double), ("radius_hint", c_double)]


class scatter_plan_info(ctypes.Structure):
    _fields_ = [("path", c_int32), ("threads", c_int32), ("points_per_thread", c_int32), ("split_k", c_int32),
                ("n_sm", c_int32), ("n_atoms_padded", c_int64), ("n_s", c_int64), ("workspace_bytes", c_int64),
                ("center_hkl", c_double * 3), ("shift", c_double * 3), ("atoms_per_thread", c_int32),
                ("adjoint_form", c_int32)]


class scatter_fft_problem(ctypes.Structure):
    _fields_ = [("n_atoms", c_int64), ("n_species", c_int32), ("species", c_void_p), ("lattice_a", c_double),
                ("center_hkl", c_double * 3), ("step", c_double), ("origin", c_double * 3), ("n", c_int64 * 3)]


class scatter_microbench_result(ctypes.Structure):
    _fields_ = [("ops_per_s", c_double), ("ops_per_clk_per_sm", c_double), ("sm_clock_hz", c_double),
                ("seconds", c_double), ("n_sm", c_int32)]


_PROTOTYPES = {
    "scatter_plan": (c_int32, [ctypes.POINTER(scatter_problem), ctypes.POINTER(scatter_options),
                               ctypes.POINTER(c_void_p)]),
    "scatter_amplitude": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scatter_amplitude_host": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scatter_intensity": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scatter_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "scatter_vjp": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scatter_check": (c_int32, [c_void_p, c_void_p]),
    "scatter_selftest_wait": (c_int32, [c_void_p, c_void_p]),
    "scatter_error_bound": (c_int32, [c_void_p, c_double, ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    "scatter_plan_get_info": (c_int32, [c_void_p, ctypes.POINTER(scatter_plan_info)]),
    "scatter_plan_timing": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int32)]),
    "scatter_plan_destroy": (None, [c_void_p]),
    "scatter_status_string": (c_char_p, [c_int32]),
    "scatter_last_error": (c_char_p, []),
    "scatter_microbench": (c_int32, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(scatter_microbench_result)]),
    "scatter_amplitude_noalloc": (c_int32, [c_int64, c_void_p, c_void_p, c_int64, c_void_p,
                                            ctypes.POINTER(c_double), c_void_p, c_void_p]),
    "scatter_fft_plan": (c_int32, [ctypes.POINTER(scatter_fft_problem), ctypes.POINTER(c_void_p)]),
    "scatter_fft_amplitude": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "scatter_fft_validity": (c_int32, [c_void_p, ctypes.POINTER(c_double), ctypes.POINTER(c_int64)]),
    "scatter_fft_plan_destroy": (None, [c_void_p]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libscatter.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"libscatter.so is not built ({LIB_PATH}); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = ctypes.CDLL(str(LIB_PATH))
        for name, (res, args) in _PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class ScatterError(RuntimeError):
    def __init__(self, status: int, where: str):
        L = lib()
        name = L.scatter_status_string(status).decode()
        msg = (L.scatter_last_error() or b"").decode()
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != SCATTER_OK:
        raise ScatterError(status, where)
