"""The oracle's discrete AAHRT operator and its exact transpose (FP64).

    L  = U . F1inv . P . F . S            (eq. axb2, Algorithm 1)
    L^T = S^T . F^T . P^H . F1inv^T . U^T  (transpose of every factor; the
                                            paper's adjoint, Sec. 3.2)

S     time stretch tau -> s = tau^2 (Algorithm 1 step 1, Sec. 3.4): the model
      column is resampled at tau = sqrt(s_n) by a local interpolation kernel.
U     the stretch undone (step 5, the paper's S^{-1}): the stretched-time data
      are resampled at s = t_i^2.  Both use Keys' cubic convolution
      (a = -1/2, four taps; "spline" interpolation, which the paper requires
      only to be local) or, optionally, linear interpolation.  Taps outside
      the input axis contribute zero.
F     DFT along stretched time, X_k = sum_n x_n exp(-i 2 pi k n / Nfft),
      k = 0..K (step 2; sign as in eq. Inv_op).
P     Fourier slice (step 3, eqs. Inv_op and inv_GFST) -- see nudft.c.
F1inv band-limited synthesis (step 4):
      x_n = (1/Nfft) [Re Y_0 + 2 Re sum_{k=1..K} Y_k exp(+i 2 pi k n / Nfft)].

Arrays: model m[ntau][nq][ntheta], data d[nt][ntr], spectra X[K+1][nq][ntheta]
and Y[K+1][ntr] (complex128).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .plan import OraclePlan

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_nudft.so")
_lib = None


# --------------------------------------------------------------- C direct sum
def build_nudft(force: bool = False) -> str:
    """Compile nudft.c with gcc (OpenMP when available)."""
    src = os.path.join(_HERE, "nudft.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", src, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_nudft())
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_longlong)
        for name in ("oracle_slice_forward", "oracle_slice_adjoint"):
            fn = getattr(lib, name)
            fn.argtypes = [ctypes.c_int] * 4 + [dp] * 3 + [lp] * 2 + [dp] * 4
            fn.restype = None
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the direct sum runs on."""
    return int(_load().oracle_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))


def _geom_args(plan: OraclePlan):
    f = np.ascontiguousarray(plan.freqs, np.float64)
    q = np.ascontiguousarray(plan.q, np.float64)
    r2 = np.ascontiguousarray(plan.r2, np.float64)
    j0 = np.ascontiguousarray(plan.j0, np.int64)
    j1 = np.ascontiguousarray(plan.j1, np.int64)
    w0 = np.ascontiguousarray(plan.w0, np.float64)
    w1 = np.ascontiguousarray(plan.w1, np.float64)
    return f, q, r2, j0, j1, w0, w1


def slice_forward(plan: OraclePlan, X: np.ndarray, impl: str = "c") -> np.ndarray:
    """P: X[K+1][nq][ntheta] -> Y[K+1][ntr] (Algorithm 1 step 3)."""
    X = np.ascontiguousarray(X, np.complex128)
    assert X.shape == (plan.nbins, plan.nq, plan.ntheta)
    if impl == "numpy":
        return slice_forward_numpy(plan, X)
    f, q, r2, j0, j1, w0, w1 = _geom_args(plan)
    Y = np.zeros((plan.nbins, plan.ntr), np.complex128)
    _load().oracle_slice_forward(plan.nbins, plan.nq, plan.ntheta, plan.ntr,
                                 _dp(f), _dp(q), _dp(r2), _lp(j0), _lp(j1),
                                 _dp(w0), _dp(w1), _dp(X.view(np.float64)),
                                 _dp(Y.view(np.float64)))
    return Y


def slice_adjoint(plan: OraclePlan, Y: np.ndarray, impl: str = "c") -> np.ndarray:
    """P^H: Y[K+1][ntr] -> X[K+1][nq][ntheta] (transpose of step 3)."""
    Y = np.ascontiguousarray(Y, np.complex128)
    assert Y.shape == (plan.nbins, plan.ntr)
    if impl == "numpy":
        return slice_adjoint_numpy(plan, Y)
    f, q, r2, j0, j1, w0, w1 = _geom_args(plan)
    X = np.zeros((plan.nbins, plan.nq, plan.ntheta), np.complex128)
    _load().oracle_slice_adjoint(plan.nbins, plan.nq, plan.ntheta, plan.ntr,
                                 _dp(f), _dp(q), _dp(r2), _lp(j0), _lp(j1),
                                 _dp(w0), _dp(w1), _dp(Y.view(np.float64)),
                                 _dp(X.view(np.float64)))
    return X


def slice_forward_numpy(plan: OraclePlan, X: np.ndarray) -> np.ndarray:
    """Same sum as oracle_slice_forward, as one broadcast expression (small
    cases only: it holds a (K+1) x nq x ntr phase array)."""
    E = np.exp(-2j * np.pi * plan.freqs[:, None, None] * plan.q[None, :, None]
               * plan.r2[None, None, :])
    Xa = X[:, :, plan.j0] * plan.w0 + X[:, :, plan.j1] * plan.w1
    return np.sum(E * Xa, axis=1)


def slice_adjoint_numpy(plan: OraclePlan, Y: np.ndarray) -> np.ndarray:
    E = np.exp(2j * np.pi * plan.freqs[:, None, None] * plan.q[None, :, None]
               * plan.r2[None, None, :])
    V = E * Y[:, None, :]                       # (K+1, nq, ntr)
    X = np.zeros((plan.nbins, plan.nq, plan.ntheta), np.complex128)
    for h in range(plan.ntr):
        X[:, :, plan.j0[h]] += plan.w0[h] * V[:, :, h]
        X[:, :, plan.j1[h]] += plan.w1[h] * V[:, :, h]
    return X


# ------------------------------------------------------------- resampling
def keys_kernel(x):
    """Keys' cubic convolution kernel with a = -1/2."""
    a = -0.5
    ax = np.abs(x)
    inner = (a + 2.0) * ax**3 - (a + 3.0) * ax**2 + 1.0
    outer = a * ax**3 - 5.0 * a * ax**2 + 8.0 * a * ax - 4.0 * a
    return np.where(ax <= 1.0, inner, np.where(ax < 2.0, outer, 0.0))


def linear_kernel(x):
    return np.maximum(0.0, 1.0 - np.abs(x))


def taps(pos: np.ndarray, n_in: int, interp: str):
    """Input indices and weights of the interpolation at fractional sample
    positions pos of an input axis of n_in samples; taps outside [0, n_in)
    get weight zero."""
    base = np.floor(pos).astype(np.int64)
    if interp == "keys":
        offs, ker = np.arange(-1, 3), keys_kernel
    else:
        offs, ker = np.arange(0, 2), linear_kernel
    idx = base[:, None] + offs[None, :]
    w = ker(pos[:, None] - idx)
    ok = (idx >= 0) & (idx < n_in)
    return np.clip(idx, 0, n_in - 1), np.where(ok, w, 0.0)


def stretch_positions(plan: OraclePlan) -> np.ndarray:
    """Model sample positions read by the stretch: tau = sqrt(n ds) in units
    of dt, n < Ns."""
    return np.sqrt(np.arange(plan.ns) * plan.ds) / plan.dt


def unstretch_positions(plan: OraclePlan) -> np.ndarray:
    """Stretched sample positions read when undoing it: s = (i dt)^2 in units
    of ds, i < nt."""
    return (np.arange(plan.nt) * plan.dt) ** 2 / plan.ds


def stretch(plan, m2):
    """S: m[ntau][C] -> m'[Ns][C]."""
    idx, w = taps(stretch_positions(plan), plan.ntau, plan.interp)
    return np.einsum("nt,ntc->nc", w, m2[idx])


def stretch_T(plan, g2):
    """S^T: [Ns][C] -> [ntau][C]."""
    idx, w = taps(stretch_positions(plan), plan.ntau, plan.interp)
    out = np.zeros((plan.ntau, g2.shape[1]))
    for t in range(idx.shape[1]):
        np.add.at(out, idx[:, t], w[:, t, None] * g2)
    return out


def unstretch(plan, dp):
    """U: d'[Ns][C] -> d[nt][C]."""
    idx, w = taps(unstretch_positions(plan), plan.ns, plan.interp)
    return np.einsum("it,itc->ic", w, dp[idx])


def unstretch_T(plan, d):
    """U^T: d[nt][C] -> [Ns][C]."""
    idx, w = taps(unstretch_positions(plan), plan.ns, plan.interp)
    out = np.zeros((plan.ns, d.shape[1]))
    for t in range(idx.shape[1]):
        np.add.at(out, idx[:, t], w[:, t, None] * d)
    return out


# ----------------------------------------------------------- time-axis DFT
def rfft_bins(plan, x):
    """F: x[Ns][C] (zero beyond Ns) -> X[K+1][C]."""
    return np.fft.rfft(x, n=plan.nfft, axis=0)[: plan.nbins]


def irfft_bins(plan, Y):
    """F1inv: Y[K+1][C] -> x[Ns][C], band-limited synthesis with the DC bin's
    real part and no Nyquist term."""
    spec = np.zeros((plan.nfft // 2 + 1, Y.shape[1]), np.complex128)
    spec[: plan.nbins] = Y
    spec[0] = spec[0].real
    return np.fft.irfft(spec, n=plan.nfft, axis=0)[: plan.ns]


def rfft_bins_T(plan, Y):
    """F^T: x_n = Re Y_0 + sum_{k=1..K} Re(Y_k exp(+i 2 pi k n/Nfft)), n < Ns
    (written through irfft: Nfft * irfft of [Re Y_0, Y_1/2, ..., Y_K/2])."""
    spec = np.zeros((plan.nfft // 2 + 1, Y.shape[1]), np.complex128)
    spec[: plan.nbins] = 0.5 * Y
    spec[0] = Y[0].real
    return plan.nfft * np.fft.irfft(spec, n=plan.nfft, axis=0)[: plan.ns]


def irfft_bins_T(plan, x):
    """F1inv^T: x[Ns][C] -> (c_k/Nfft) sum_n x_n exp(-i 2 pi k n/Nfft) with
    c_0 = 1 and c_k = 2 for k >= 1."""
    X = np.fft.rfft(x, n=plan.nfft, axis=0)[: plan.nbins] / plan.nfft
    X[1:] *= 2.0
    return X


# --------------------------------------------------------------- operators
def forward_stages(plan: OraclePlan, m: np.ndarray, impl: str = "c") -> dict:
    """L m with every intermediate: m' = S m, X = F m', Y = P X,
    d' = F1inv Y, d = U d'."""
    C = plan.nq * plan.ntheta
    ms = stretch(plan, np.asarray(m, np.float64).reshape(plan.ntau, C))
    X = rfft_bins(plan, ms).reshape(plan.nbins, plan.nq, plan.ntheta)
    Y = slice_forward(plan, X, impl)
    dp = irfft_bins(plan, Y)
    d = unstretch(plan, dp)
    return dict(ms=ms, X=X, Y=Y, dp=dp, d=d)


def forward(plan: OraclePlan, m: np.ndarray, impl: str = "c") -> np.ndarray:
    """d = L m (Algorithm 1, eq. axb2)."""
    return forward_stages(plan, m, impl)["d"]


def adjoint_stages(plan: OraclePlan, d: np.ndarray, impl: str = "c") -> dict:
    """L^T d with every intermediate."""
    r = unstretch_T(plan, np.asarray(d, np.float64))
    R = irfft_bins_T(plan, r)
    Xa = slice_adjoint(plan, R, impl)
    gs = rfft_bins_T(plan, Xa.reshape(plan.nbins, plan.nq * plan.ntheta))
    g = stretch_T(plan, gs).reshape(plan.ntau, plan.nq, plan.ntheta)
    return dict(r=r, R=R, Xa=Xa, gs=gs, g=g)


def adjoint(plan: OraclePlan, d: np.ndarray, impl: str = "c") -> np.ndarray:
    """m = L^T d (exact transpose of L; Sec. 3.2)."""
    return adjoint_stages(plan, d, impl)["g"]


def forward_traces(plan: OraclePlan, m: np.ndarray, traces) -> np.ndarray:
    """Columns d[:, traces] of L m, computed on those traces alone."""
    return forward(plan.subset_traces(traces), m)


def adjoint_slices(plan: OraclePlan, d: np.ndarray, slices) -> np.ndarray:
    """(L^T d)[:, :, slices]: only traces whose two azimuth weights touch
    one of the slices contribute to them, so the adjoint is evaluated on
    those traces alone."""
    slices = np.atleast_1d(slices)
    touch = np.isin(plan.j0, slices) | np.isin(plan.j1, slices)
    idx = np.nonzero(touch)[0]
    g = adjoint(plan.subset_traces(idx), np.asarray(d)[:, idx])
    return g[:, :, slices]
