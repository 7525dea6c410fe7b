"""ctypes binding of libaahrt (include/aahrt.h): the same entry points under
the same names, argument marshalling only.  Every step of the transform runs
in the library's CUDA kernels; there is no Python or CPU fallback, and
loading fails loudly when the library is missing."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_float, c_int, c_longlong, c_void_p

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaahrt.so")

AAHRT_OK = 0
AAHRT_ERR_INVALID_ARG = -1
AAHRT_ERR_OOM = -2
AAHRT_ERR_CUDA = -3
AAHRT_ERR_UNSUPPORTED = -4
AAHRT_ERR_TIMEOUT = -5
AAHRT_ERR_NONFINITE = -6
AAHRT_INTERP_KEYS = 0
AAHRT_INTERP_LINEAR = 1
AAHRT_SLICE_SPREAD = 0
AAHRT_SLICE_LINEAR_K = 1
AAHRT_SLICE_DIRECT = 2
AAHRT_PRECISION_FP32 = 0
AAHRT_PRECISION_SPLIT_BF16 = 1
AAHRT_NSTAGES = 7
AAHRT_NOALLOC_SCRATCH_BYTES = 16 << 20
STAGE_NAMES = ("stretch_fft", "slice_fwd", "ifft_unstretch", "unstretchT_fft",
               "slice_adj", "ifft_stretchT", "solver_updates")


class aahrt_geom(ctypes.Structure):
    _fields_ = [("nt", c_int), ("dt", c_double), ("ntau", c_int), ("nq", c_int),
                ("q0", c_double), ("dq", c_double), ("ntheta", c_int), ("ntr", c_int),
                ("hx", POINTER(c_double)), ("hy", POINTER(c_double))]


class aahrt_opts(ctypes.Structure):
    _fields_ = [("interp_kind", c_int), ("spread_width", c_int), ("theta_group", c_int),
                ("ngather", c_int), ("sigma_t", c_double), ("fmax", c_double),
                ("time_pairs", c_int), ("autotune", c_int), ("precision", c_int),
                ("slice_interp", c_int), ("sigma_q", c_double),
                ("q_axis", POINTER(c_double)), ("r2max", c_double)]


class aahrt_plan_info(ctypes.Structure):
    _fields_ = [("nfft", c_int), ("ns", c_int), ("nbins", c_int), ("nq_os", c_int),
                ("spread_width", c_int), ("theta_group", c_int), ("ncube", c_int),
                ("ngather", c_int), ("ds", c_double), ("rho", c_double), ("beta", c_double),
                ("model_len", c_longlong), ("data_len", c_longlong),
                ("xspec_len", c_longlong), ("yspec_len", c_longlong),
                ("workspace_bytes", c_longlong), ("time_pairs", c_int), ("autotuned", c_int),
                ("tune_ms", c_double), ("precision", c_int), ("slice_interp", c_int)]


class aahrt_grid(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("x0", c_double), ("dx", c_double),
                ("y0", c_double), ("dy", c_double)]


class aahrt_solve_opts(ctypes.Structure):
    _fields_ = [("ista", c_int), ("warm_start", c_int), ("power_iters", c_int),
                ("use_graph", c_int), ("gamma", c_double), ("lambda_rel", c_double),
                ("per_cube", c_int), ("cube_gamma", POINTER(c_double)),
                ("cube_lambda", POINTER(c_double))]


class aahrt_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("gamma", c_double), ("lambda", c_double),
                ("resid_norm", c_double), ("l1_norm", c_double), ("objective", c_double)]


class AahrtError(RuntimeError):
    def __init__(self, status, where, text):
        super().__init__(f"{where}: status {status}: {text}")
        self.status = status


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "aahrt_plan_create": (c_int, [POINTER(c_void_p), POINTER(aahrt_geom), POINTER(aahrt_opts)]),
    "aahrt_plan_create_batched": (c_int, [POINTER(c_void_p), c_int, POINTER(aahrt_geom),
                                          POINTER(aahrt_opts)]),
    "aahrt_plan_destroy": (None, [c_void_p]),
    "aahrt_plan_query": (c_int, [c_void_p, POINTER(aahrt_plan_info)]),
    "aahrt_forward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "aahrt_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "aahrt_sparse_solve": (c_int, [c_void_p, c_void_p, c_float, c_int, c_void_p,
                                   POINTER(aahrt_solve_opts), POINTER(aahrt_solve_info),
                                   c_void_p]),
    "aahrt_apply_stage": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "aahrt_fista_vjp": (c_int, [c_void_p, c_void_p, c_void_p, c_float, c_float, c_int, c_int,
                                c_int, c_void_p, c_void_p, c_void_p]),
    "aahrt_plan_set_wavelet": (c_int, [c_void_p, c_void_p, c_int, c_int]),
    "aahrt_pick_velocity": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "aahrt_velocity_scan_grid": (c_int, [c_void_p, POINTER(aahrt_grid), c_void_p, c_void_p,
                                         c_void_p]),
    "aahrt_forward_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "aahrt_plan_test_stall": (c_int, [c_void_p, c_int]),
    "aahrt_q_axis_slowness": (c_int, [c_double, c_double, c_int, POINTER(c_double)]),
    "aahrt_nq_required": (c_int, [c_double, c_double, c_double, POINTER(c_int)]),
    "aahrt_partial_nmo": (c_int, [c_void_p, c_void_p, c_void_p, c_double, c_int, c_void_p]),
    "aahrt_q_from_slowness": (c_int, [c_double, c_double, c_int, POINTER(c_double),
                                      POINTER(c_double)]),
    "aahrt_plan_set_profiling": (c_int, [c_void_p, c_int]),
    "aahrt_plan_stage_times": (c_int, [c_void_p, POINTER(c_double), POINTER(c_longlong)]),
    "aahrt_plan_status": (c_int, [c_void_p]),
    "aahrt_status_string": (ctypes.c_char_p, [c_int]),
    "aahrt_last_error": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load libaahrt.so (built by paper_2505_00387_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libaahrt.so not found at {path}: build it with "
                      "`python -m paper_2505_00387_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != AAHRT_OK:
        lib = load()
        raise AahrtError(status, where, lib.aahrt_last_error().decode(errors="replace"))


# ------------------------------------------ entry points under their C names
def aahrt_plan_create(geom: aahrt_geom, opts: aahrt_opts | None = None) -> c_void_p:
    h = c_void_p()
    check(load().aahrt_plan_create(ctypes.byref(h), ctypes.byref(geom),
                                   ctypes.byref(opts) if opts is not None else None),
          "aahrt_plan_create")
    return h


def aahrt_plan_create_batched(geoms, opts: aahrt_opts | None = None) -> c_void_p:
    arr = (aahrt_geom * len(geoms))(*geoms)
    h = c_void_p()
    check(load().aahrt_plan_create_batched(ctypes.byref(h), len(geoms), arr,
                                           ctypes.byref(opts) if opts is not None else None),
          "aahrt_plan_create_batched")
    return h


def aahrt_plan_destroy(h):
    load().aahrt_plan_destroy(h)


def aahrt_plan_query(h) -> aahrt_plan_info:
    info = aahrt_plan_info()
    check(load().aahrt_plan_query(h, ctypes.byref(info)), "aahrt_plan_query")
    return info


def aahrt_forward(h, m_ptr: int, d_ptr: int, stream: int = 0):
    check(load().aahrt_forward(h, c_void_p(m_ptr), c_void_p(d_ptr), c_void_p(stream)),
          "aahrt_forward")


def aahrt_forward_noalloc(h, m_ptr: int, d_ptr: int, stream: int = 0):
    check(load().aahrt_forward_noalloc(h, c_void_p(m_ptr), c_void_p(d_ptr), c_void_p(stream)),
          "aahrt_forward_noalloc")


def aahrt_adjoint(h, d_ptr: int, m_ptr: int, stream: int = 0):
    check(load().aahrt_adjoint(h, c_void_p(d_ptr), c_void_p(m_ptr), c_void_p(stream)),
          "aahrt_adjoint")


def aahrt_sparse_solve(h, d_ptr: int, lam: float, iters: int, m_ptr: int,
                       opts: aahrt_solve_opts | None = None, want_info: bool = True,
                       stream: int = 0):
    info = aahrt_solve_info() if want_info else None
    check(load().aahrt_sparse_solve(h, c_void_p(d_ptr), c_float(lam), int(iters),
                                    c_void_p(m_ptr),
                                    ctypes.byref(opts) if opts is not None else None,
                                    ctypes.byref(info) if info is not None else None,
                                    c_void_p(stream)),
          "aahrt_sparse_solve")
    return info


def aahrt_fista_vjp(h, d_ptr: int, mbar_ptr: int, lam: float, gamma: float, iters: int,
                    ista: bool, checkpoint: int, mout_ptr, dbar_ptr: int, stream: int = 0):
    check(load().aahrt_fista_vjp(h, c_void_p(d_ptr), c_void_p(mbar_ptr), c_float(lam),
                                 c_float(gamma), int(iters), int(bool(ista)), int(checkpoint),
                                 c_void_p(mout_ptr) if mout_ptr else None, c_void_p(dbar_ptr),
                                 c_void_p(stream)), "aahrt_fista_vjp")


def aahrt_apply_stage(h, stage: int, in_ptr: int, out_ptr: int, stream: int = 0):
    check(load().aahrt_apply_stage(h, int(stage), c_void_p(in_ptr), c_void_p(out_ptr),
                                   c_void_p(stream)), "aahrt_apply_stage")


def aahrt_q_from_slowness(pmin: float, pmax: float, nq: int):
    q0, dq = c_double(), c_double()
    check(load().aahrt_q_from_slowness(pmin, pmax, nq, ctypes.byref(q0), ctypes.byref(dq)),
          "aahrt_q_from_slowness")
    return q0.value, dq.value


def aahrt_plan_test_stall(h, on: bool):
    check(load().aahrt_plan_test_stall(h, int(bool(on))), "aahrt_plan_test_stall")


def aahrt_q_axis_slowness(pmin: float, pmax: float, nq: int):
    q = (c_double * max(1, int(nq)))()
    check(load().aahrt_q_axis_slowness(pmin, pmax, int(nq), q), "aahrt_q_axis_slowness")
    return [q[i] for i in range(int(nq))]


def aahrt_nq_required(span: float, fmax: float, r2max: float) -> int:
    n = c_int()
    check(load().aahrt_nq_required(span, fmax, r2max, ctypes.byref(n)), "aahrt_nq_required")
    return n.value


def aahrt_partial_nmo(h, in_ptr: int, out_ptr: int, q_ref: float, transpose: bool = False,
                      stream: int = 0):
    check(load().aahrt_partial_nmo(h, c_void_p(in_ptr), c_void_p(out_ptr), c_double(q_ref),
                                   int(bool(transpose)), c_void_p(stream)), "aahrt_partial_nmo")


def aahrt_plan_set_profiling(h, on: bool):
    check(load().aahrt_plan_set_profiling(h, int(bool(on))), "aahrt_plan_set_profiling")


def aahrt_plan_stage_times(h):
    t = (c_double * AAHRT_NSTAGES)()
    n = (c_longlong * AAHRT_NSTAGES)()
    check(load().aahrt_plan_stage_times(h, t, n), "aahrt_plan_stage_times")
    return list(t), list(n)


def aahrt_plan_set_wavelet(h, w_ptr, nw: int, center: int):
    check(load().aahrt_plan_set_wavelet(h, c_void_p(w_ptr) if w_ptr else None, int(nw),
                                        int(center)), "aahrt_plan_set_wavelet")


def aahrt_pick_velocity(h, m_ptr: int, qhat_ptr: int, weight_ptr, stream: int = 0):
    check(load().aahrt_pick_velocity(h, c_void_p(m_ptr), c_void_p(qhat_ptr),
                                     c_void_p(weight_ptr) if weight_ptr else None,
                                     c_void_p(stream)), "aahrt_pick_velocity")


def aahrt_velocity_scan_grid(h, grid: aahrt_grid, d_ptr: int, m_ptr: int, stream: int = 0):
    check(load().aahrt_velocity_scan_grid(h, ctypes.byref(grid), c_void_p(d_ptr),
                                          c_void_p(m_ptr), c_void_p(stream)),
          "aahrt_velocity_scan_grid")


def aahrt_plan_status(h):
    check(load().aahrt_plan_status(h), "aahrt_plan_status")


def aahrt_status_string(status: int) -> str:
    return load().aahrt_status_string(status).decode()


def aahrt_last_error() -> str:
    return load().aahrt_last_error().decode(errors="replace")
