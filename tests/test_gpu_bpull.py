"""GPU: the paper's pull velocity scan on a regular offset grid (Algorithm 2,
B-coefficients) through the C ABI against the oracle's scan, its focusing of
a single event, and its argument checks."""
import numpy as np
import pytest

import oracle
from oracle import bpull, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, host, rel

pytestmark = pytest.mark.gpu


def case(nx=24, ny=24, d=40.0, nt=128, nq=24, ntheta=6):
    grid = bpull.Grid(nx, ny, -(nx - 1) / 2 * d, d, -(ny - 1) / 2 * d, d)
    x = grid.x0 + np.arange(nx) * d
    y = grid.y0 + np.arange(ny) * d
    hx, hy = np.meshgrid(x, y, indexing="ij")
    q0, dq = syn.q_axis(nq)
    g = syn.Gather(nt, 0.008, nt, nq, q0, dq, ntheta, hx.ravel(), hy.ravel())
    return g, grid


def gpu(g, **kw):
    from paper_2505_00387_gb300.plan import AahrtPlan
    return AahrtPlan(**g.geom_kwargs(), **kw)


def as_tuple(grid):
    return (grid.nx, grid.ny, grid.x0, grid.dx, grid.y0, grid.dy)


@pytest.mark.parametrize("sigma_q", [0.0, 4.0])
def test_scan_matches_oracle(sigma_q):
    g, grid = case()
    op = oracle.make_plan(**g.geom_kwargs())
    gp = gpu(g, sigma_q=sigma_q)
    rng = np.random.default_rng(120)
    d = rng.standard_normal((g.nt, g.ntr))
    mg = host(gp.velocity_scan_grid(dev(d), as_tuple(grid)), (g.ntau, g.nq, g.ntheta))
    mo = bpull.scan(op, grid, d, sigma_q if sigma_q > 0 else 2.0)
    assert rel(mg, mo) < 1e-4


def test_scan_focuses_event():
    g, grid = case()
    op = oracle.make_plan(**g.geom_kwargs())
    gp = gpu(g)
    m = np.zeros((g.ntau, g.nq, g.ntheta))
    m[:, 18, 0] = syn.ricker((np.arange(g.ntau) - 35) * g.dt, 20.0)
    d = ops.forward(op, m)
    mg = host(gp.velocity_scan_grid(dev(d), as_tuple(grid)), m.shape)
    assert np.unravel_index(np.argmax(np.abs(mg)), mg.shape) == (35, 18, 0)


def test_scan_checks_arguments():
    from paper_2505_00387_gb300._lib import AahrtError
    g, grid = case()
    gp = gpu(g)
    d = dev(np.zeros((g.nt, g.ntr)))
    bad = (grid.nx + 1, grid.ny, grid.x0, grid.dx, grid.y0, grid.dy)
    with pytest.raises(AahrtError):
        gp.velocity_scan_grid(d, bad)
    g2 = syn.Gather(g.nt, g.dt, g.nt - 8, g.nq, g.q0, g.dq, g.ntheta, g.hx, g.hy)
    with pytest.raises(AahrtError):
        gpu(g2).velocity_scan_grid(d, as_tuple(grid))
