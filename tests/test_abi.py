"""The C ABI library builds, loads, and exports every function include/aahrt.h
declares; host-side argument validation answers without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2505_00387_gb300 import _lib as L
from paper_2505_00387_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_ ]+\s*\**\s*(aahrt_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("aahrt_forward", "aahrt_adjoint", "aahrt_sparse_solve",
                 "aahrt_plan_create", "aahrt_plan_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(L._SIGS)


def test_binding_constants_match_header():
    """Every AAHRT_* integer the binding defines equals the header's #define
    or enumerator of the same name."""
    txt = re.sub(r"/\*.*?\*/", "", "".join(open(h).read() for h in HEADERS), flags=re.S)
    vals = {}
    for m in re.finditer(r"^#define\s+(AAHRT_\w+)\s+(\S[^\n]*?)\s*$", txt, re.M):
        expr = re.sub(r"(\d+)u\b", r"\1", m.group(2))
        if re.fullmatch(r"[-\d<>() ]+", expr):
            vals[m.group(1)] = int(eval(expr, {}, {}))
    names = [n for n in dir(L) if n.startswith("AAHRT_") and isinstance(getattr(L, n), int)]
    assert "AAHRT_NOALLOC_SCRATCH_BYTES" in names
    for n in names:
        assert n in vals, n
        assert getattr(L, n) == vals[n], n


def test_status_strings(lib):
    assert L.aahrt_status_string(0) == "success"
    assert L.aahrt_status_string(-1) == "invalid argument"
    assert L.aahrt_status_string(12345) == "unknown status"


def test_q_from_slowness(lib):
    q0, dq = L.aahrt_q_from_slowness(1 / 3500, 1 / 1500, 32)
    assert abs(q0 - (1 / 3500) ** 2) < 1e-22
    assert abs(q0 + 31 * dq - (1 / 1500) ** 2) < 1e-20
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_q_from_slowness(1 / 1500, 1 / 3500, 32)
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG


def _geom(nt=64, ntr=8, nq=4, ntheta=2, dt=0.004, dq=1e-8, keep=None):
    hx = np.linspace(100, 800, ntr)
    hy = np.linspace(-300, 300, ntr)
    keep.extend([hx, hy])
    dp = ctypes.POINTER(ctypes.c_double)
    return L.aahrt_geom(nt, dt, nt, nq, 1e-7, dq, ntheta, ntr, hx.ctypes.data_as(dp),
                        hy.ctypes.data_as(dp))


@pytest.mark.parametrize("field,value", [("nt", 2), ("ntr", 0), ("nq", 0), ("ntheta", 0),
                                         ("dt", 0.0), ("dq", -1e-8)])
def test_plan_create_rejects_bad_geometry(lib, field, value):
    keep = []
    g = _geom(keep=keep)
    setattr(g, field, value)
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_plan_create(g)
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [("spread_width", 3), ("spread_width", 13),
                                         ("interp_kind", 5), ("sigma_t", 0.5)])
def test_plan_create_rejects_bad_options(lib, field, value):
    keep = []
    g = _geom(keep=keep)
    o = L.aahrt_opts()
    setattr(o, field, value)
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_plan_create(g, o)
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG


def test_plan_create_rejects_nonfinite_offsets(lib):
    keep = []
    g = _geom(keep=keep)
    keep[0][3] = np.nan
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_plan_create(g)
    assert e.value.status == L.AAHRT_ERR_NONFINITE


def test_batched_rejects_mismatched_axes(lib):
    keep = []
    g1, g2 = _geom(keep=keep), _geom(keep=keep, nq=5)
    with pytest.raises(L.AahrtError) as e:
        L.aahrt_plan_create_batched([g1, g2])
    assert e.value.status == L.AAHRT_ERR_INVALID_ARG


def test_null_plan_calls(lib):
    bad = L.AAHRT_ERR_INVALID_ARG
    assert lib.aahrt_forward(None, None, None, None) == bad
    assert lib.aahrt_adjoint(None, None, None, None) == bad
    assert lib.aahrt_plan_query(None, None) == bad
    # every entry point that takes a plan refuses a NULL one before touching
    # a device
    assert lib.aahrt_sparse_solve(None, None, 0.0, 1, None, None, None, None) == bad
    assert lib.aahrt_apply_stage(None, 0, None, None, None) == bad
    assert lib.aahrt_fista_vjp(None, None, None, 0.0, 1.0, 1, 0, 0, None, None, None) == bad
    assert lib.aahrt_plan_set_wavelet(None, None, 0, 0) == bad
    assert lib.aahrt_pick_velocity(None, None, None, None, None) == bad
    assert lib.aahrt_velocity_scan_grid(None, None, None, None, None) == bad
    assert lib.aahrt_forward_noalloc(None, None, None, None) == bad
    assert lib.aahrt_partial_nmo(None, None, None, 1e-7, 0, None) == bad
    assert lib.aahrt_plan_test_stall(None, 1) == bad
    assert lib.aahrt_plan_set_profiling(None, 1) == bad
    assert lib.aahrt_plan_stage_times(None, None, None) == bad
    assert lib.aahrt_plan_status(None) == bad
    lib.aahrt_plan_destroy(None)


def test_package_import_does_not_load_cuda():
    import importlib
    import sys
    for k in [k for k in sys.modules if k.startswith("paper_2505_00387_gb300")]:
        if k.endswith("synthetic"):
            continue
    mod = importlib.import_module("paper_2505_00387_gb300.synthetic")
    assert hasattr(mod, "small_cube")


def test_ctypes_structs_match_the_header(tmp_path):
    """sizeof and every field offset of the ABI structs, as the C compiler
    lays them out from include/aahrt.h, equal the ctypes mirrors."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"aahrt_geom": L.aahrt_geom, "aahrt_opts": L.aahrt_opts,
               "aahrt_plan_info": L.aahrt_plan_info, "aahrt_solve_opts": L.aahrt_solve_opts,
               "aahrt_solve_info": L.aahrt_solve_info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "aahrt.h"',
             "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
