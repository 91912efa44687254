"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function include/scatter.h declares,
and reject bad arguments with SCATTER_ERR_INVALID_ARG before touching a
device.  On a machine without a GPU a valid problem gives
SCATTER_ERR_NO_DEVICE (never a crash).
"""
import ctypes
import pathlib
import re

import numpy as np
import pytest

from paper_1010_2641_gb300 import binding as B
from paper_1010_2641_gb300 import build as libbuild
from paper_1010_2641_gb300 import workloads as W

ROOT = pathlib.Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def L():
    libbuild.build()
    return B.lib()


def declared_functions():
    names = []
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        names += re.findall(r"^(?:scatter_status|void|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scatter_plan", "scatter_amplitude", "scatter_intensity", "scatter_backward",
                     "scatter_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert set(names) == set(B._PROTOTYPES), "binding and header disagree"


def test_status_strings(L):
    for code, name in [(0, "SCATTER_OK"), (1, "SCATTER_ERR_INVALID_ARG"), (5, "SCATTER_ERR_TIMEOUT"),
                       (7, "SCATTER_ERR_NO_DEVICE")]:
        assert L.scatter_status_string(code).decode() == name
    assert L.scatter_status_string(99).decode() == "SCATTER_ERR_UNKNOWN"


def test_struct_sizes_match_c_layout(tmp_path):
    """Every struct of the ABI: ctypes size and field offsets equal what the
    C compiler makes of include/scatter.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [B.scatter_species, B.scatter_problem, B.scatter_options, B.scatter_plan_info,
               B.scatter_microbench_result, B.scatter_fft_problem]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "scatter.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("%zu\\n", sizeof({st.__name__}));')
        for name, _ in st._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({st.__name__}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for st in structs:
        want.append(ctypes.sizeof(st))
        want += [getattr(st, name).offset for name, _ in st._fields_]
    assert got == want


def _problem(n_atoms=10, n_s=5, species_idx=None, coef=None):
    keep = []
    coef = W.si_ge_species() if coef is None else coef
    sp = (B.scatter_species * len(coef))()
    for i, row in enumerate(coef):
        sp[i].a[:] = row[0:4]
        sp[i].b[:] = row[4:8]
        sp[i].c, sp[i].fp, sp[i].fpp, sp[i].b_dw = row[8:12]
    S = np.zeros((n_s, 3)) + np.array([0, 0, 4.0])
    keep += [sp, S]
    pr = B.scatter_problem()
    pr.n_atoms = n_atoms
    pr.n_species = len(coef)
    pr.species = sp
    if species_idx is not None:
        a = np.asarray(species_idx, dtype=np.int32)
        keep.append(a)
        pr.atom_species = a.ctypes.data
    pr.lattice_a = W.LATTICE_A
    pr.s_kind = B.SCATTER_S_LIST
    pr.n_s = n_s
    pr.s_list = S.ctypes.data
    pr.batch = 1
    return pr, keep


def _plan(L, pr, op=None):
    h = ctypes.c_void_p()
    st = L.scatter_plan(ctypes.byref(pr) if pr is not None else None,
                        ctypes.byref(op) if op is not None else None, ctypes.byref(h))
    return st, h


def test_invalid_arguments_rejected_before_device(L):
    assert _plan(L, None)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.lattice_a = -1.0
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.n_species = 0
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem(n_atoms=4, species_idx=[0, 1, 2, 0])  # species 2 does not exist
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    assert b"species" in L.scatter_last_error()
    pr, keep = _problem()
    pr.s_list = None
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    keep[1][2, 1] = np.nan
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.s_kind = 7
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.center_mode = 1
    pr.center_hkl[:] = [0.0, 0.5, 4.0]  # H must be integer
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.batch = 2  # offsets missing
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    op = B.scatter_options()
    op.path = 9
    assert _plan(L, pr, op)[0] == B.SCATTER_ERR_INVALID_ARG
    pr, keep = _problem()
    pr.s_kind = B.SCATTER_S_GRID  # axes missing
    assert _plan(L, pr)[0] == B.SCATTER_ERR_INVALID_ARG
    st = L.scatter_plan(ctypes.byref(_problem()[0]), None, None)
    assert st == B.SCATTER_ERR_INVALID_ARG


def test_calls_on_null_plan(L):
    assert L.scatter_amplitude(None, None, None, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_intensity(None, None, None, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_backward(None, None, None, None, None, None, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_vjp(None, None, None, None, None, None) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_check(None, None) == B.SCATTER_ERR_INVALID_ARG
    a, b = ctypes.c_double(), ctypes.c_double()
    assert L.scatter_error_bound(None, 1.0, ctypes.byref(a), ctypes.byref(b)) == B.SCATTER_ERR_INVALID_ARG
    assert L.scatter_plan_get_info(None, None) == B.SCATTER_ERR_INVALID_ARG
    L.scatter_plan_destroy(None)  # NULL-safe


def test_valid_problem_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    pr, keep = _problem()
    st, h = _plan(L, pr)
    assert st == B.SCATTER_ERR_NO_DEVICE and not h.value
    r = B.scatter_microbench_result()
    assert L.scatter_microbench(0, 10, ctypes.byref(r)) == B.SCATTER_ERR_NO_DEVICE
    assert L.scatter_microbench(42, 10, ctypes.byref(r)) == B.SCATTER_ERR_INVALID_ARG
