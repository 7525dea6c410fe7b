"""Paper-literal slice step of the oracle: linear interpolation in k
(the A-coefficients of eq. thli, Sec. 3.4 "Discrete Implementation").

The paper samples the q-spectrum of each azimuth slice on a uniform k grid
by an FFT along q and reads it at k_q = f' r^2 by linear interpolation
between the two neighbouring grid points (and linearly in theta, as the
exact operator does).  Discretely (readings of the paper):

* the q axis is centred on its middle sample l = cq = nq // 2 (the paper's
  q range is symmetric about zero); the centred column is zero-padded to
  nos = max(16, next_pow2(ceil(sigma_q * nq))) points, and
      G[u] = sum_l X[l] exp(-2 pi i u (l - cq) / nos),   u = 0..nos-1,
  is its spectrum at k = u / (nos dq) (period nos);
* trace h at bin k sits at grid position x = f_k r_h^2 dq nos; with
  i = floor(x), a = x - i, the slice value is (1 - a) G[i] + a G[i+1]
  (indices mod nos), times exp(-2 pi i f_k (q0 + cq dq) r_h^2) to undo the
  centring;
* sigma_q = 1 is the unpadded FFT of the paper's own sampling (eq. q1-q3);
  larger sigma_q refines the k grid.

The adjoint is the exact transpose.  TEST INFRASTRUCTURE (see the package
docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import ops


def grid_size(nq: int, sigma_q: float) -> int:
    n = 16
    while n < math.ceil(sigma_q * nq):
        n *= 2
    return n


def _geometry(plan, sigma_q):
    if plan.q_axis is not None:
        raise ValueError("the k-interpolation needs a uniform q axis (FFT along q)")
    nos = grid_size(plan.nq, sigma_q)
    cq = plan.nq // 2
    n_l = (np.arange(plan.nq) - cq) % nos                 # padded index of sample l
    x = plan.freqs[:, None] * plan.r2[None, :] * plan.dq * nos     # (K+1, ntr)
    i0 = np.floor(x)
    a = x - i0
    i0 = i0.astype(np.int64) % nos
    i1 = (i0 + 1) % nos
    ph = np.exp(-2j * np.pi * plan.freqs[:, None] * (plan.q0 + cq * plan.dq)
                * plan.r2[None, :])
    return nos, n_l, i0, i1, a, ph


def slice_forward(plan, X, sigma_q: float = 2.0):
    """Y[K+1][ntr] from X[K+1][nq][ntheta] by linear interpolation in k."""
    X = np.asarray(X, np.complex128)
    nos, n_l, i0, i1, a, ph = _geometry(plan, sigma_q)
    Y = np.zeros((plan.nbins, plan.ntr), np.complex128)
    h = np.arange(plan.ntr)
    for k in range(plan.nbins):
        pad = np.zeros((nos, plan.ntheta), np.complex128)
        pad[n_l] = X[k]
        G = np.fft.fft(pad, axis=0)                       # G[u, j]
        v = ((1.0 - a[k])[:, None] * G[i0[k]] + a[k][:, None] * G[i1[k]])   # (ntr, ntheta)
        s = plan.w0 * v[h, plan.j0] + plan.w1 * v[h, plan.j1]
        Y[k] = ph[k] * s
    return Y


def slice_adjoint(plan, Y, sigma_q: float = 2.0):
    """The exact transpose of slice_forward."""
    Y = np.asarray(Y, np.complex128)
    nos, n_l, i0, i1, a, ph = _geometry(plan, sigma_q)
    X = np.zeros((plan.nbins, plan.nq, plan.ntheta), np.complex128)
    for k in range(plan.nbins):
        z = np.conj(ph[k]) * Y[k]
        V = np.zeros((nos, plan.ntheta), np.complex128)
        for w, j in ((plan.w0, plan.j0), (plan.w1, plan.j1)):
            np.add.at(V, (i0[k], j), (1.0 - a[k]) * w * z)
            np.add.at(V, (i1[k], j), a[k] * w * z)
        # sum_u V[u] exp(+2 pi i u n / nos) = nos * ifft(V)[n]
        X[k] = nos * np.fft.ifft(V, axis=0)[n_l]
    return X


def forward(plan, m, sigma_q: float = 2.0):
    """d = U F1inv P_lin F S m (Algorithm 1 with the paper's interpolation)."""
    C = plan.nq * plan.ntheta
    ms = ops.stretch(plan, np.asarray(m, np.float64).reshape(plan.ntau, C))
    X = ops.rfft_bins(plan, ms).reshape(plan.nbins, plan.nq, plan.ntheta)
    return ops.unstretch(plan, ops.irfft_bins(plan, slice_forward(plan, X, sigma_q)))


def adjoint(plan, d, sigma_q: float = 2.0):
    """m = forward^T d."""
    R = ops.irfft_bins_T(plan, ops.unstretch_T(plan, np.asarray(d, np.float64)))
    Xa = slice_adjoint(plan, R, sigma_q)
    gs = ops.rfft_bins_T(plan, Xa.reshape(plan.nbins, plan.nq * plan.ntheta))
    return ops.stretch_T(plan, gs).reshape(plan.ntau, plan.nq, plan.ntheta)
