"""Independent evaluations that pin the oracle (test infrastructure).

None of these is used by ``ops``; each evaluates a quantity the paper or the
mathematics fixes by a different route, so a dropped term, wrong sign or
transposed operand in the oracle shows up as a mismatch.
"""
from __future__ import annotations

import numpy as np


def ricker(t, f):
    a = (np.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def riemann_sum_forward(nt, dt, traces_r2, traces_w, events):
    """Physical-domain evaluation of eq. Inverse for a model made of
    Ricker wavelets on single (q, azimuth-slice) cells: with the time-stretch
    convention of eq. Inverse2 (no Jacobian factor), a model column
    M(tau) = a * ricker(tau - tau_e) at curvature q produces on a trace of
    squared offset r^2 and slice weight w the signal
        w * a * ricker(sqrt(t^2 - q r^2) - tau_e)   for t^2 >= q r^2, else 0.
    events: list of (a, tau_e, f, q, slice) and traces_w[h][slice] the
    azimuth weight of slice `slice` for trace h."""
    t = np.arange(nt) * dt
    d = np.zeros((nt, len(traces_r2)))
    for (a, tau_e, f, q, sl) in events:
        for h, r2 in enumerate(traces_r2):
            w = traces_w[h].get(sl, 0.0)
            if w == 0.0:
                continue
            arg = t * t - q * r2
            ok = arg >= 0.0
            tau = np.sqrt(np.where(ok, arg, 0.0))
            d[:, h] += np.where(ok, w * a * ricker(tau - tau_e, f), 0.0)
    return d


def dirichlet(x, nfft, kmax):
    """Periodic band-limited interpolation kernel of the kept bins:
    D(x) = (1/N) [1 + 2 sum_{k=1..K} cos(2 pi k x / N)]."""
    k = np.arange(1, kmax + 1)
    return (1.0 + 2.0 * np.cos(2.0 * np.pi * np.outer(x, k) / nfft).sum(axis=1)) / nfft


def time_domain_shift(xs, shift, nfft, kmax, ns):
    """Delay of a stretched-time column xs[n] (n < len(xs), zero beyond) by a
    fractional number of samples `shift`, evaluated directly in the time
    domain with the Dirichlet kernel: out[n] = sum_m xs[m] D(n - m - shift),
    n < ns.  By the shift theorem this is what F1inv P F computes for a
    single curvature and azimuth (eq. Inv_op)."""
    n = np.arange(ns)
    out = np.zeros(ns)
    for mi, v in enumerate(xs):
        if v != 0.0:
            out += v * dirichlet(n - mi - shift, nfft, kmax)
    return out


def explicit_dft(x, nfft, nbins):
    """X_k = sum_n x_n exp(-i 2 pi k n / N) by explicit summation."""
    n = np.arange(len(x))
    return np.array([np.sum(x * np.exp(-2j * np.pi * k * n / nfft))
                     for k in range(nbins)])


def soft_piecewise(x, t):
    """Soft threshold written piecewise: x - t for x > t, x + t for x < -t,
    0 otherwise (equal to eq. soft for t >= 0)."""
    return np.where(x > t, x - t, np.where(x < -t, x + t, 0.0))
