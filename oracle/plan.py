"""Sampling plan and trace geometry of the oracle (FP64, numpy).

Readings of the paper used here (each is listed with its reason in the
design notes of the repository):

* The curvature axis is uniform, q_l = q0 + l*dq (FFT along q, Sec. 3.4 and
  eq. q1-q3 need uniform q), unless explicit values q_axis are given (for
  instance a uniform slowness axis, q_l = p_l^2): the slice step is then the
  same sum over the non-uniform q_l (a type-3 DFT along q).
* The model intercept axis is tau_i = i*dt for i < ntau, the data axis is
  t_i = i*dt for i < nt.
* Stretched time s = t^2 (Sec. 3.1, eq. Inverse2) is sampled as
  s_n = n*ds, n < Ns, inside an FFT frame of Nfft samples.  Nfft is a power of
  two at least sigma_t*nt*(1+rho), rho = |q|_max r_max^2 / t_max^2, and
  Ns is the largest count with (Ns-1)(1+rho) <= Nfft-2, so that the largest
  moveout q r^2 never wraps stretched support back into [0, t_max^2].
* Frequency bins k = 0..K with K = Nfft/2 - 1: the Nyquist bin is excluded
  (its real-only constraint would break the exact transpose); an optional
  fmax (in 1/s^2) lowers K.
* Azimuth is axial, theta_h = atan2(hy, hx) mod pi (theta = 0 when r = 0), on
  the grid theta_j = j*pi/ntheta; the two neighbouring slices j_h and
  (j_h + 1) mod ntheta get the linear weights of the theta factors of the
  A-coefficients of eq. thli: w_{j_h} = (theta_{j_h+1} - theta_h)/dtheta and
  w_{j_h+1} = (theta_h - theta_{j_h})/dtheta.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np


def next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


@dataclass
class OraclePlan:
    nt: int
    dt: float
    ntau: int
    nq: int
    q0: float
    dq: float
    ntheta: int
    hx: np.ndarray
    hy: np.ndarray
    interp: str          # "keys" (cubic convolution, a = -1/2) or "linear"
    tmax: float
    rho: float
    nfft: int
    ns: int
    ds: float
    kmax: int            # K: bins 0..K are kept
    # per-trace geometry
    r2: np.ndarray
    theta: np.ndarray
    j0: np.ndarray
    j1: np.ndarray
    w0: np.ndarray
    w1: np.ndarray
    q_axis: np.ndarray | None = None   # explicit curvature values (non-uniform)

    @property
    def ntr(self) -> int:
        return int(self.hx.shape[0])

    @property
    def nbins(self) -> int:
        return self.kmax + 1

    @property
    def q(self) -> np.ndarray:
        """Curvature axis: q_l = q0 + l*dq, or the explicit values."""
        if self.q_axis is not None:
            return self.q_axis
        return self.q0 + self.dq * np.arange(self.nq)

    @property
    def freqs(self) -> np.ndarray:
        """Stretched-time frequencies f_k = k / (Nfft ds), k = 0..K."""
        return np.arange(self.kmax + 1) / (self.nfft * self.ds)

    def subset_traces(self, idx) -> "OraclePlan":
        """Same time sampling, only the traces idx (used to evaluate single
        output traces of the forward operator, or the traces that touch a
        few azimuth slices for the adjoint)."""
        idx = np.asarray(idx)
        return replace(self, hx=self.hx[idx], hy=self.hy[idx], r2=self.r2[idx],
                       theta=self.theta[idx], j0=self.j0[idx], j1=self.j1[idx],
                       w0=self.w0[idx], w1=self.w1[idx])


def azimuth_bins(hx, hy, ntheta):
    """Axial azimuth of every trace and its two-slice linear weights
    (theta factors of eq. thli, made periodic in theta with period pi)."""
    hx = np.asarray(hx, dtype=np.float64)
    hy = np.asarray(hy, dtype=np.float64)
    r2 = hx * hx + hy * hy
    th = np.mod(np.arctan2(hy, hx), np.pi)
    th = np.where(r2 > 0.0, th, 0.0)
    dth = np.pi / ntheta
    phi = th / dth
    j = np.floor(phi).astype(np.int64)
    frac = phi - j
    wrap = j >= ntheta             # theta rounded up to pi is azimuth 0
    j = np.where(wrap, j - ntheta, j)
    j = np.clip(j, 0, ntheta - 1)
    frac = np.where(wrap, 0.0, frac)
    w0 = 1.0 - frac
    w1 = frac
    j1 = (j + 1) % ntheta
    return r2, th, j, j1, w0, w1


def make_plan(nt, dt, ntau, nq, q0, dq, ntheta, hx, hy, *, sigma_t=2.0,
              fmax=0.0, interp="keys", r2max=None, q_axis=None) -> OraclePlan:
    """Stretched-time sampling plan (Sec. 3.4, step 1 and 2 of Algorithms 1
    and 2) and per-trace geometry.  r2max overrides the largest squared
    offset (a batch of cubes shares one time plan built from the batch-wide
    maximum).  q_axis: explicit curvature values (nq of them; q0 and dq are
    then ignored)."""
    if interp not in ("keys", "linear"):
        raise ValueError("interp must be 'keys' or 'linear'")
    r2, th, j0, j1, w0, w1 = azimuth_bins(hx, hy, ntheta)
    tmax = (nt - 1) * dt
    r2m = float(np.max(r2)) if r2max is None else float(r2max)
    if q_axis is not None:
        q_axis = np.array(q_axis, dtype=np.float64)
        if q_axis.ndim != 1 or q_axis.size != nq or not np.all(np.isfinite(q_axis)):
            raise ValueError("q_axis must hold nq finite values")
        qabs = float(np.max(np.abs(q_axis)))
    else:
        qabs = max(abs(q0), abs(q0 + (nq - 1) * dq))
    rho = qabs * r2m / (tmax * tmax)
    nfft = next_pow2(int(math.ceil(sigma_t * nt * (1.0 + rho))))
    ns = int(math.floor((nfft - 2) / (1.0 + rho))) + 1
    ds = tmax * tmax / (ns - 1)
    kmax = nfft // 2 - 1
    if fmax and fmax > 0.0:
        kmax = min(kmax, int(math.floor(fmax * nfft * ds)))
    return OraclePlan(nt=nt, dt=dt, ntau=ntau, nq=nq, q0=q0, dq=dq,
                      ntheta=ntheta, hx=np.asarray(hx, np.float64),
                      hy=np.asarray(hy, np.float64), interp=interp, tmax=tmax,
                      rho=rho, nfft=nfft, ns=ns, ds=ds, kmax=kmax, r2=r2,
                      theta=th, j0=j0, j1=j1, w0=w0, w1=w1, q_axis=q_axis)
