"""Curvature-range tools of the oracle (Sec. 3.5, eqs. q1-q3): the sampling
bound on the number of curvatures, the uniform-slowness curvature axis, and
the partial NMO applied to the data before the transform.

* Eq. q3.  Along q the slice step is a DFT read at k_q = f' r^2, which is
  never negative, so a q step dq resolves k_q without aliasing over a whole
  period 1/dq: dq <= 1 / (f'max r^2max) (eqs. q1-q2).  A range of width
  `span` (2 q_max for the paper's symmetric axis [-q_max, q_max]) then needs
  N_q >= span f'max r^2max samples, eq. q3 with span = 2 q_max.
* Uniform slowness.  p_l = p_min + l (p_max - p_min)/(nq - 1), q_l = p_l^2:
  a non-uniform curvature axis (the slice step becomes a type-3 DFT).
* Partial NMO.  In stretched time s = t^2 a hyperbola t^2 = tau^2 + q r^2 is
  the line s = tau^2 + q r^2; shifting every stretched trace by -q_ref r^2
  (the paper's partial NMO of the time-stretched data) moves it to curvature
  q - q_ref, so a range [q_a, q_b] becomes one centred on zero when
  q_ref = (q_a + q_b)/2 and eq. q3 asks for (q_b - q_a) f'max r^2max samples
  instead of 2 max(|q_a|, |q_b|) f'max r^2max.  Here the shift is applied on
  the time axis in one resampling (reading of the paper: the stretch, shift
  and unstretch collapse into one interpolation):
      d_out(t_i, h) = sum_taps c(u - n) d(t_n, h),  u = sqrt(t_i^2 + q_ref r_h^2)/dt,
  zero where t_i^2 + q_ref r_h^2 < 0, with the plan's interpolation kernel c
  (Keys cubic or linear) and taps outside [0, nt) taken as zero.  Its
  inverse is the same map with -q_ref (up to interpolation and the muted
  zone); partial_nmo_T is its exact transpose.

TEST INFRASTRUCTURE (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import ops


def nq_required(span: float, fmax: float, r2max: float) -> int:
    """Smallest number of uniform curvature samples over a range of width
    `span` (s^2/m^2) that keeps k_q = f' r^2 <= fmax r2max unaliased (eq. q3
    with span = 2 q_max): ceil(span fmax r2max), at least 1."""
    if span < 0.0 or fmax < 0.0 or r2max < 0.0:
        raise ValueError("span, fmax and r2max must be >= 0")
    return max(1, int(math.ceil(span * fmax * r2max - 1e-12)))


def q_axis_slowness(pmin: float, pmax: float, nq: int) -> np.ndarray:
    """q_l = p_l^2 for slownesses p_l uniform on [pmin, pmax]."""
    if nq < 1:
        raise ValueError("nq must be >= 1")
    p = np.array([pmin], np.float64) if nq == 1 else np.linspace(pmin, pmax, nq)
    return p * p


def _positions(plan, q_ref):
    """Input sample positions u[i][h] and the mask of defined outputs."""
    t = np.arange(plan.nt) * plan.dt
    arg = t[:, None] ** 2 + q_ref * plan.r2[None, :]
    ok = arg >= 0.0
    u = np.sqrt(np.where(ok, arg, 0.0)) / plan.dt
    return u, ok


def partial_nmo(plan, d, q_ref: float) -> np.ndarray:
    """d_out[i][h] = sum_taps c(u - n) d[n][h] with u = sqrt(t_i^2 +
    q_ref r_h^2)/dt (zero where the root is imaginary)."""
    d = np.asarray(d, np.float64).reshape(plan.nt, plan.ntr)
    u, ok = _positions(plan, q_ref)
    out = np.zeros_like(d)
    for h in range(plan.ntr):
        idx, w = ops.taps(u[:, h], plan.nt, plan.interp)
        col = np.sum(w * d[idx, h], axis=1)
        out[:, h] = np.where(ok[:, h], col, 0.0)
    return out


def partial_nmo_T(plan, e, q_ref: float) -> np.ndarray:
    """Transpose of partial_nmo: every output sample's taps scatter back."""
    e = np.asarray(e, np.float64).reshape(plan.nt, plan.ntr)
    u, ok = _positions(plan, q_ref)
    out = np.zeros_like(e)
    for h in range(plan.ntr):
        idx, w = ops.taps(u[:, h], plan.nt, plan.interp)
        w = np.where(ok[:, h, None], w, 0.0)
        for c in range(idx.shape[1]):
            np.add.at(out[:, h], idx[:, c], w[:, c] * e[:, h])
    return out
