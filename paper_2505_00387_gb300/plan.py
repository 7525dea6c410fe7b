"""Convenience wrapper over the C ABI: owns a plan handle, checks tensor
shapes/devices, and passes torch's device pointers and current CUDA stream
to libaahrt.  PyTorch supplies device memory and streams only."""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _geom(nt, dt, ntau, nq, q0, dq, ntheta, hx, hy, keep):
    hx = np.ascontiguousarray(hx, dtype=np.float64)
    hy = np.ascontiguousarray(hy, dtype=np.float64)
    if hx.shape != hy.shape or hx.ndim != 1:
        raise ValueError("hx and hy must be 1-D arrays of equal length")
    keep.extend([hx, hy])
    dp = ctypes.POINTER(ctypes.c_double)
    return L.aahrt_geom(int(nt), float(dt), int(ntau), int(nq), float(q0), float(dq),
                        int(ntheta), int(hx.shape[0]), hx.ctypes.data_as(dp),
                        hy.ctypes.data_as(dp))


PRECISIONS = {"fp32": L.AAHRT_PRECISION_FP32, "split_bf16": L.AAHRT_PRECISION_SPLIT_BF16}


SLICE_INTERPS = {"spread": L.AAHRT_SLICE_SPREAD, "linear_k": L.AAHRT_SLICE_LINEAR_K,
                 "direct": L.AAHRT_SLICE_DIRECT}


def _opts(interp="keys", spread_width=0, theta_group=0, ngather=1, sigma_t=0.0, fmax=0.0,
          time_pairs=0, autotune=False, precision="fp32", slice_interp="spread",
          sigma_q=0.0, q_axis=None, keep=None, r2max=0.0):
    kind = {"keys": L.AAHRT_INTERP_KEYS, "linear": L.AAHRT_INTERP_LINEAR}[interp]
    qp = None
    if q_axis is not None:
        qa = np.ascontiguousarray(q_axis, dtype=np.float64)
        if qa.ndim != 1:
            raise ValueError("q_axis must be 1-D")
        if keep is not None:
            keep.append(qa)
        qp = qa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return L.aahrt_opts(kind, int(spread_width), int(theta_group), int(ngather),
                        float(sigma_t), float(fmax), int(time_pairs), int(bool(autotune)),
                        PRECISIONS[precision], SLICE_INTERPS[slice_interp], float(sigma_q),
                        qp, float(r2max))


def q_axis_slowness(pmin: float, pmax: float, nq: int) -> np.ndarray:
    """Uniform-slowness curvature axis q_l = p_l^2 (aahrt_q_axis_slowness)."""
    return np.array(L.aahrt_q_axis_slowness(pmin, pmax, nq), dtype=np.float64)


def nq_required(span: float, fmax: float, r2max: float) -> int:
    """Curvature samples for a range of width span (eq. q3; aahrt_nq_required)."""
    return L.aahrt_nq_required(span, fmax, r2max)


class AahrtPlan:
    """Plan of the AAHRT operator pair on the current CUDA device."""

    def __init__(self, nt, dt, ntau, nq, q0, dq, ntheta, hx, hy, *, interp="keys",
                 spread_width=0, theta_group=0, ngather=1, sigma_t=0.0, fmax=0.0,
                 time_pairs=0, autotune=False, precision="fp32", slice_interp="spread",
                 sigma_q=0.0, q_axis=None, r2max=0.0, _handle=None, _shapes=None):
        if _handle is not None:
            self.handle = _handle
        else:
            keep = []
            g = _geom(nt, dt, ntau, nq, q0, dq, ntheta, hx, hy, keep)
            self.handle = L.aahrt_plan_create(
                g, _opts(interp, spread_width, theta_group, ngather, sigma_t, fmax,
                         time_pairs, autotune, precision, slice_interp, sigma_q, q_axis,
                         keep, r2max))
        self.info = L.aahrt_plan_query(self.handle)
        self.nt, self.ntau, self.nq, self.ntheta = nt, ntau, nq, ntheta
        self.device = torch.device("cuda", torch.cuda.current_device())

    @classmethod
    def from_gather(cls, g, **kw):
        return cls(**g.geom_kwargs(), **kw)

    @classmethod
    def batched(cls, gathers: Sequence, interp="keys", spread_width=0, theta_group=0,
                sigma_t=0.0, fmax=0.0, time_pairs=0, autotune=False, slice_interp="spread",
                sigma_q=0.0, q_axis=None, r2max=0.0):
        keep = []
        geoms = [_geom(g.nt, g.dt, g.ntau, g.nq, g.q0, g.dq, g.ntheta, g.hx, g.hy, keep)
                 for g in gathers]
        h = L.aahrt_plan_create_batched(
            geoms, _opts(interp, spread_width, theta_group, 1, sigma_t, fmax, time_pairs,
                         autotune, "fp32", slice_interp, sigma_q, q_axis, keep, r2max))
        g0 = gathers[0]
        return cls(g0.nt, g0.dt, g0.ntau, g0.nq, g0.q0, g0.dq, g0.ntheta, None, None,
                   _handle=h)

    # ------------------------------------------------------------------
    @property
    def model_len(self) -> int:
        return int(self.info.model_len)

    @property
    def data_len(self) -> int:
        return int(self.info.data_len)

    def _check(self, t: torch.Tensor, n: int, name: str):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous float32")
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} elements, the plan needs {n}")

    def forward(self, m: torch.Tensor, d: Optional[torch.Tensor] = None, stream=None):
        """d = L m (Algorithm 1)."""
        self._check(m, self.model_len, "m")
        if d is None:
            d = torch.empty(self.data_len, device=m.device, dtype=torch.float32)
        self._check(d, self.data_len, "d")
        L.aahrt_forward(self.handle, m.data_ptr(), d.data_ptr(), _stream_ptr(stream))
        return d

    def adjoint(self, d: torch.Tensor, m: Optional[torch.Tensor] = None, stream=None):
        """m = L^T d (exact transpose)."""
        self._check(d, self.data_len, "d")
        if m is None:
            m = torch.empty(self.model_len, device=d.device, dtype=torch.float32)
        self._check(m, self.model_len, "m")
        L.aahrt_adjoint(self.handle, d.data_ptr(), m.data_ptr(), _stream_ptr(stream))
        return m

    def partial_nmo(self, d: torch.Tensor, q_ref: float, out: Optional[torch.Tensor] = None,
                    transpose: bool = False, stream=None):
        """Partial NMO of the data by q_ref (Sec. 3.5): curvature q -> q - q_ref
        (or the map's exact transpose)."""
        self._check(d, self.data_len, "d")
        if out is None:
            out = torch.empty(self.data_len, device=d.device, dtype=torch.float32)
        self._check(out, self.data_len, "out")
        L.aahrt_partial_nmo(self.handle, d.data_ptr(), out.data_ptr(), float(q_ref),
                            transpose, _stream_ptr(stream))
        return out

    def sparse_solve(self, d: torch.Tensor, lam: float, iters: int,
                     m: Optional[torch.Tensor] = None, *, ista=False, gamma=0.0,
                     lambda_rel=0.0, power_iters=0, warm_start=False, use_graph=True,
                     want_info=True, per_cube=False, cube_gamma=None, cube_lambda=None,
                     stream=None):
        """Sparse transform (eq. cost1) by ISTA/FISTA iterations (eq. ISTA).
        With per_cube, every cube (gather) is solved with its own step and
        threshold; cube_gamma / cube_lambda (float64 numpy arrays of ncube, or
        None) give them (entries <= 0 of cube_gamma are estimated) and
        receive the values used."""
        self._check(d, self.data_len, "d")
        if m is None:
            m = torch.zeros(self.model_len, device=d.device, dtype=torch.float32)
        self._check(m, self.model_len, "m")
        dp = ctypes.POINTER(ctypes.c_double)
        arrs = []
        for a in (cube_gamma, cube_lambda):
            if a is None:
                arrs.append(None)
                continue
            if (not isinstance(a, np.ndarray) or a.dtype != np.float64 or
                    a.shape != (int(self.info.ncube),) or not a.flags.c_contiguous):
                raise ValueError("cube_gamma / cube_lambda must be contiguous float64 arrays "
                                 "of ncube")
            arrs.append(a.ctypes.data_as(dp))
        o = L.aahrt_solve_opts(int(bool(ista)), int(bool(warm_start)), int(power_iters),
                               int(bool(use_graph)), float(gamma), float(lambda_rel),
                               int(bool(per_cube)), arrs[0], arrs[1])
        info = L.aahrt_sparse_solve(self.handle, d.data_ptr(), float(lam), int(iters),
                                    m.data_ptr(), o, want_info, _stream_ptr(stream))
        return m, info

    def fista_vjp(self, d: torch.Tensor, m_bar: torch.Tensor, lam: float, gamma: float,
                  iters: int, *, ista=False, checkpoint=0, want_m=True, stream=None):
        """(m^iters, d_bar) of the unrolled solve: d_bar = (dm/dd)^T m_bar
        (see aahrt_fista_vjp)."""
        self._check(d, self.data_len, "d")
        self._check(m_bar, self.model_len, "m_bar")
        d_bar = torch.empty(self.data_len, device=d.device, dtype=torch.float32)
        m_out = (torch.empty(self.model_len, device=d.device, dtype=torch.float32)
                 if want_m else None)
        L.aahrt_fista_vjp(self.handle, d.data_ptr(), m_bar.data_ptr(), float(lam),
                          float(gamma), int(iters), ista, int(checkpoint),
                          m_out.data_ptr() if m_out is not None else 0, d_bar.data_ptr(),
                          _stream_ptr(stream))
        return m_out, d_bar

    def apply_stage(self, stage: int, x: torch.Tensor, out: Optional[torch.Tensor] = None,
                    stream=None):
        """One operator stage (see aahrt_apply_stage); spectra are complex64."""
        xs, ys = int(self.info.xspec_len), int(self.info.yspec_len)
        n_in = [self.model_len, xs, ys, self.data_len, ys, xs][stage]
        n_out = [xs, ys, self.data_len, ys, xs, self.model_len][stage]
        cplx_in = stage in (1, 2, 4, 5)
        cplx_out = stage in (0, 1, 3, 4)
        want_in = torch.complex64 if cplx_in else torch.float32
        if x.dtype != want_in or x.numel() != n_in or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"stage {stage} needs a contiguous CUDA {want_in} input of {n_in}")
        if out is None:
            out = torch.empty(n_out, device=x.device,
                              dtype=torch.complex64 if cplx_out else torch.float32)
        L.aahrt_apply_stage(self.handle, stage, x.data_ptr(), out.data_ptr(),
                            _stream_ptr(stream))
        return out

    def velocity_scan_grid(self, d: torch.Tensor, grid, m: Optional[torch.Tensor] = None,
                           stream=None):
        """The paper's pull velocity scan (Algorithm 2) of data on a regular
        grid (nx, ny, x0, dx, y0, dy); see aahrt_velocity_scan_grid."""
        self._check(d, self.data_len, "d")
        if m is None:
            m = torch.empty(self.model_len, device=d.device, dtype=torch.float32)
        self._check(m, self.model_len, "m")
        nx, ny, x0, dx, y0, dy = grid
        g = L.aahrt_grid(int(nx), int(ny), float(x0), float(dx), float(y0), float(dy))
        L.aahrt_velocity_scan_grid(self.handle, g, d.data_ptr(), m.data_ptr(),
                                   _stream_ptr(stream))
        return m

    def pick_velocity(self, m: torch.Tensor, stream=None):
        """(q_hat, weight): the q-moment pick of eq. vel_est at every
        (tau, theta) (see aahrt_pick_velocity)."""
        self._check(m, self.model_len, "m")
        n = self.model_len // self.nq
        q_hat = torch.empty(n, device=m.device, dtype=torch.float32)
        weight = torch.empty(n, device=m.device, dtype=torch.float32)
        L.aahrt_pick_velocity(self.handle, m.data_ptr(), q_hat.data_ptr(), weight.data_ptr(),
                              _stream_ptr(stream))
        return q_hat, weight

    def set_wavelet(self, w, center: int):
        """Make the operator the deconvolutive W L (eq. DecRT): every trace
        convolved in time with w (sample `center` at lag 0); None clears."""
        if w is None:
            L.aahrt_plan_set_wavelet(self.handle, 0, 0, 0)
            return
        w = np.ascontiguousarray(w, dtype=np.float32)
        L.aahrt_plan_set_wavelet(self.handle, w.ctypes.data, int(w.size), int(center))

    def status(self):
        """Synchronise; raise AahrtError if a kernel reported a device-side
        timeout since the last check."""
        L.aahrt_plan_status(self.handle)

    def set_profiling(self, on: bool):
        L.aahrt_plan_set_profiling(self.handle, on)

    def stage_times(self):
        return L.aahrt_plan_stage_times(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            L.aahrt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
