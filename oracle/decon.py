"""Deconvolutive AAHRT of the oracle (Sec. 4, eq. DecRT): R_w^{-1} = W R^{-1}.

W convolves every trace in time with a band-limited wavelet w (it replaces
the Dirac pulse of the basis functions).  Discretely, with the wavelet given
as samples w[s], s = 0..nw-1, whose sample `center` sits at lag zero,

    (W x)[i]   = sum_s w[s] x[i - s + center],     i = 0..nt-1,
    (W^T y)[n] = sum_s w[s] y[n + s - center],     n = 0..nt-1,

with x and y zero outside [0, nt): a linear convolution truncated to the
trace length, and its exact transpose (a correlation).

TEST INFRASTRUCTURE (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import ops


def conv_t(x, w, center):
    """W x for x[nt][ntr] (every column convolved)."""
    x = np.asarray(x, np.float64)
    nt = x.shape[0]
    out = np.zeros_like(x)
    for s, ws in enumerate(np.asarray(w, np.float64)):
        lag = s - center                 # out[i] += w[s] x[i - lag]
        if lag >= 0:
            if lag < nt:
                out[lag:] += ws * x[:nt - lag]
        elif -lag < nt:
            out[:nt + lag] += ws * x[-lag:]
    return out


def corr_t(y, w, center):
    """W^T y (the transpose of conv_t)."""
    y = np.asarray(y, np.float64)
    nt = y.shape[0]
    out = np.zeros_like(y)
    for s, ws in enumerate(np.asarray(w, np.float64)):
        lag = s - center                 # out[n] += w[s] y[n + lag]
        if lag >= 0:
            if lag < nt:
                out[:nt - lag] += ws * y[lag:]
        elif -lag < nt:
            out[-lag:] += ws * y[:nt + lag]
    return out


def forward(plan, m, w, center, impl: str = "c"):
    """d = W L m (eq. DecRT)."""
    return conv_t(ops.forward(plan, m, impl), w, center)


def adjoint(plan, d, w, center, impl: str = "c"):
    """m = L^T W^T d."""
    return ops.adjoint(plan, corr_t(d, w, center), impl)
