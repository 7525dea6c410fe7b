"""Pins of the oracle's pull velocity scan (Algorithm 2, B-coefficients).

* The B-coefficient interpolation reproduces functions bilinear in (x, y)
  exactly inside the grid and reads zero outside it.
* The ring sum of step 3 visits exactly the aliases k_u + n/dq whose radius
  stays inside the grid (counted independently).
* The scan focuses a single hyperbolic event (generated by the exact
  operator) on its own (tau, q, theta) cell, as the exact adjoint does, and
  correlates with the adjoint (the paper drops the Jacobian 1/(2 f'), so the
  two differ in frequency weighting only).
"""
import numpy as np

import oracle
from oracle import bpull, lineark, ops
from paper_2505_00387_gb300 import synthetic as syn


def grid_case(nx=16, ny=16, d=80.0, nt=128, nq=24, ntheta=6):
    grid = bpull.Grid(nx, ny, -(nx - 1) / 2 * d, d, -(ny - 1) / 2 * d, d)
    x = grid.x0 + np.arange(nx) * d
    y = grid.y0 + np.arange(ny) * d
    hx, hy = np.meshgrid(x, y, indexing="ij")
    q0, dq = syn.q_axis(nq)
    p = oracle.make_plan(nt, 0.008, nt, nq, q0, dq, ntheta, hx.ravel(), hy.ravel())
    return p, grid


def test_bilinear_is_exact_for_bilinear_functions():
    p, grid = grid_case()
    x = grid.x0 + np.arange(grid.nx) * grid.dx
    y = grid.y0 + np.arange(grid.ny) * grid.dy
    X, Y = np.meshgrid(x, y, indexing="ij")
    f = lambda a, b: (1.5 - 0.3j) + 2e-3 * a - 1e-3j * b + 4e-6 * a * b
    D = f(X, Y).ravel()
    rng = np.random.default_rng(1)
    px = rng.uniform(x[0], x[-1], 50)
    py = rng.uniform(y[0], y[-1], 50)
    np.testing.assert_allclose(bpull.bilinear(D, grid, px, py), f(px, py), rtol=0, atol=1e-12)
    out = bpull.bilinear(D, grid, np.array([x[-1] + 2 * grid.dx]), np.array([0.0]))
    assert out[0] == 0.0


def test_pull_grid_sums_every_alias_ring():
    """G[u][j] against an independent evaluation: scipy's linear grid
    interpolator on the zero-bordered grid (samples outside the grid are
    zero), summed over both antipodes of every ring k_u + n/dq inside the
    grid's corner radius (ring count in closed form) with the centring
    phase."""
    from scipy.interpolate import RegularGridInterpolator
    p, grid = grid_case()
    x = grid.x0 + np.arange(grid.nx) * grid.dx
    y = grid.y0 + np.arange(grid.ny) * grid.dy
    X, Y = np.meshgrid(x, y, indexing="ij")
    f = lambda a, b: (0.7 + 0.2j) + 1e-3 * a + 2e-3j * b + 3e-6 * a * b
    D = f(X, Y).ravel()
    k = p.nbins // 3
    nos = lineark.grid_size(p.nq, 2.0)
    qc = p.q0 + (p.nq // 2) * p.dq
    G = bpull.pull_grid(p, grid, D, k)
    fk = p.freqs[k]
    span = fk * grid.r2max() * nos * p.dq          # largest ring index u + n nos
    th = np.arange(p.ntheta) * np.pi / p.ntheta
    xp = np.concatenate([[x[0] - grid.dx], x, [x[-1] + grid.dx]])
    yp = np.concatenate([[y[0] - grid.dy], y, [y[-1] + grid.dy]])
    Fp = np.zeros((xp.size, yp.size), complex)
    Fp[1:-1, 1:-1] = f(X, Y)
    ire = RegularGridInterpolator((xp, yp), Fp.real, bounds_error=False, fill_value=0.0)
    iim = RegularGridInterpolator((xp, yp), Fp.imag, bounds_error=False, fill_value=0.0)
    interp = lambda a, b: (ire(np.stack([a, b], -1)) + 1j * iim(np.stack([a, b], -1)))
    for u in (0, 3, nos // 2, nos - 1):
        nring = int(np.floor((span - u) / nos)) + 1 if u <= span else 0
        ref = np.zeros(p.ntheta, complex)
        for n in range(nring):
            kap = (u + n * nos) / (nos * p.dq)
            r = np.sqrt(kap / fk)
            for sgn in (1.0, -1.0):
                a, b = sgn * r * np.cos(th), sgn * r * np.sin(th)
                ref += np.exp(2j * np.pi * kap * qc) * interp(a, b)
        np.testing.assert_allclose(G[u], ref, rtol=0, atol=1e-9 * max(1.0, np.abs(ref).max()))


def test_scan_focuses_single_events():
    # 40 m spacing (the paper's): at 80 m the steepest of these events is
    # spatially aliased for the interpolation and the scan smears it
    p, grid = grid_case(nx=24, ny=24, d=40.0)
    for (tau_i, l, j) in ((50, 12, 2), (80, 5, 4), (35, 18, 0)):
        m = np.zeros((p.ntau, p.nq, p.ntheta))
        m[:, l, j] = syn.ricker((np.arange(p.ntau) - tau_i) * p.dt, 20.0)
        d = ops.forward(p, m)
        M = bpull.scan(p, grid, d)
        i, lh, jh = np.unravel_index(np.argmax(np.abs(M)), M.shape)
        assert abs(i - tau_i) <= 1 and abs(lh - l) <= 1 and jh == j
        A = ops.adjoint(p, d)
        cos = float(np.sum(M * A) / np.linalg.norm(M) / np.linalg.norm(A))
        assert cos > 0.85
