"""The paper's own velocity scan (Algorithm 2 with the B-coefficients of
Sec. 3.4): data on a regular offset grid are pulled, not spread.

Steps (eq. Fwd_op, frwrd and the B-coefficient form of eq. thli):

1. stretch the data time axis by interpolation, D(t') = D(t^2) -- the same
   resampler S that stretches the model (needs ntau = nt);
2. FFT along t' (bins k = 0..K, f' = f_k);
3. for every azimuth slice theta_j and every q-grid wavenumber
   k_u = u / (nos dq), u = 0..nos-1, read D^(f', x, y) at the two points
   (x, y) = +-sqrt(k/f') (cos theta_j, sin theta_j) by bilinear interpolation
   on the regular grid (zero outside it), for k = k_u + n/dq, n = 0, 1, ...
   while the ring stays inside the grid (the q-DFT is periodic in k with
   period 1/dq, so every alias ring lands on the same grid sample), with the
   phase exp(+2 pi i k q_c) of the centred q axis (q_c = q0 + cq dq);
4. inverse DFT along u onto the q axis, M^(f', q_l) = sum_u G[u]
   exp(+2 pi i u (l - cq)/nos), and the Hermitian synthesis along f';
5. undo the stretch with the resampler U (model rows = nt).

Readings: the delta of theta = arctan(y/x) (period pi) selects both antipodal
points; the paper's relation carries no Jacobian factor and none is applied;
bin 0 (f' = 0) has no finite ring and is set to zero.  The scan is the
paper's approximation of the velocity stack, not the transpose of the
forward operator.

TEST INFRASTRUCTURE (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lineark, ops


@dataclass
class Grid:
    """Regular offsets: trace ix * ny + iy sits at (x0 + ix dx, y0 + iy dy)."""
    nx: int
    ny: int
    x0: float
    dx: float
    y0: float
    dy: float

    def r2max(self) -> float:
        xs = (self.x0, self.x0 + (self.nx - 1) * self.dx)
        ys = (self.y0, self.y0 + (self.ny - 1) * self.dy)
        return max(x * x for x in xs) + max(y * y for y in ys)


def bilinear(Dk, grid: Grid, x, y):
    """B-coefficient interpolation of Dk[nx*ny] at points (x, y)."""
    fx = (np.asarray(x) - grid.x0) / grid.dx
    fy = (np.asarray(y) - grid.y0) / grid.dy
    ix = np.floor(fx).astype(np.int64)
    iy = np.floor(fy).astype(np.int64)
    ax, ay = fx - ix, fy - iy
    out = np.zeros(np.shape(fx), np.complex128)
    for cx, wx in ((0, 1.0 - ax), (1, ax)):
        for cy, wy in ((0, 1.0 - ay), (1, ay)):
            jx, jy = ix + cx, iy + cy
            ok = (jx >= 0) & (jx < grid.nx) & (jy >= 0) & (jy < grid.ny)
            v = np.where(ok, Dk[np.clip(jx, 0, grid.nx - 1) * grid.ny
                                + np.clip(jy, 0, grid.ny - 1)], 0.0)
            out += wx * wy * v
    return out


def pull_grid(plan, grid: Grid, Dk, k: int, sigma_q: float = 2.0):
    """G[u][j] of step 3 at bin k."""
    if plan.q_axis is not None:
        raise ValueError("the pull scan needs a uniform q axis (FFT along q)")
    nos = lineark.grid_size(plan.nq, sigma_q)
    cq = plan.nq // 2
    qc = plan.q0 + cq * plan.dq
    G = np.zeros((nos, plan.ntheta), np.complex128)
    f = plan.freqs[k]
    if k == 0:
        return G
    r2max = grid.r2max()
    th = np.arange(plan.ntheta) * np.pi / plan.ntheta
    c, s = np.cos(th), np.sin(th)
    for u in range(nos):
        n = 0
        while True:
            kap = (u + n * nos) / (nos * plan.dq)
            r2 = kap / f
            if r2 > r2max:
                break
            r = np.sqrt(r2)
            ph = np.exp(2j * np.pi * kap * qc)
            G[u] += ph * (bilinear(Dk, grid, r * c, r * s) + bilinear(Dk, grid, -r * c, -r * s))
            n += 1
    return G


def scan(plan, grid: Grid, d, sigma_q: float = 2.0):
    """M[ntau][nq][ntheta] of Algorithm 2 from d[nt][nx*ny]."""
    assert plan.ntau == plan.nt and plan.ntr == grid.nx * grid.ny
    nos = lineark.grid_size(plan.nq, sigma_q)
    n_l = (np.arange(plan.nq) - plan.nq // 2) % nos
    ds_ = ops.stretch(plan, np.asarray(d, np.float64))
    D = ops.rfft_bins(plan, ds_)                                   # (K+1, ntr)
    X = np.zeros((plan.nbins, plan.nq, plan.ntheta), np.complex128)
    for k in range(plan.nbins):
        G = pull_grid(plan, grid, D[k], k, sigma_q)
        X[k] = nos * np.fft.ifft(G, axis=0)[n_l]
    # Hermitian synthesis along f', then the stretch undone (U) on model rows
    Xd = X.reshape(plan.nbins, plan.nq * plan.ntheta)
    return ops.unstretch(plan, ops.irfft_bins(plan, Xd)).reshape(plan.ntau, plan.nq,
                                                                  plan.ntheta)
