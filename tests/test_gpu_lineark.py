"""GPU: the paper-literal slice step (linear interpolation in k, the
A-coefficients of eq. thli) through the C ABI against the oracle's own
linear-k operator, and its error against the exact operator."""
import numpy as np
import pytest

from oracle import fista, lineark, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, gpu_plan, host, oracle_plan, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4
TOL_SOLVE = 1e-3


def ragged():
    rng = np.random.default_rng(110)
    hx, hy = syn.disc_offsets(rng, 333, 1800.0)
    q0, dq = syn.q_axis(37)
    return syn.Gather(300, 0.004, 280, 37, q0, dq, 5, hx, hy)


@pytest.mark.parametrize("case", ["small_cube", "ragged"])
@pytest.mark.parametrize("sigma_q", [1.0, 2.0])
def test_lineark_matches_oracle(case, sigma_q):
    g = syn.small_cube() if case == "small_cube" else ragged()
    op = oracle_plan(g)
    gp = gpu_plan(g, slice_interp="linear_k", sigma_q=sigma_q)
    assert gp.info.spread_width == 2
    assert gp.info.nq_os == lineark.grid_size(g.nq, sigma_q)
    rng = np.random.default_rng(111)
    m = rng.standard_normal((g.ntau, g.nq, g.ntheta))
    d = rng.standard_normal((g.nt, g.ntr))
    dg = host(gp.forward(dev(m)), d.shape)
    mg = host(gp.adjoint(dev(d)), m.shape)
    assert rel(dg, lineark.forward(op, m, sigma_q)) < TOL_OP
    assert rel(mg, lineark.adjoint(op, d, sigma_q)) < TOL_OP
    # dot test on a well-conditioned pair of FP32 inputs: d2 = L m by the
    # oracle plus as much noise, so <L m, d2> is about |L m|^2
    m32 = m.astype(np.float32).astype(np.float64)
    lm = lineark.forward(op, m32, sigma_q)
    d2 = lm + np.sqrt(np.mean(lm * lm)) * rng.standard_normal(lm.shape)
    d2 = d2.astype(np.float32).astype(np.float64)
    lhs = float(np.sum(host(gp.forward(dev(m32)), d.shape) * d2))
    rhs = float(np.sum(host(gp.adjoint(dev(d2)), m.shape) * m32))
    print(f"{case} sigma_q={sigma_q}: fwd {rel(dg, lineark.forward(op, m, sigma_q)):.2e} "
          f"dot {abs(lhs - rhs) / abs(lhs):.2e}")
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def test_lineark_error_against_exact_operator():
    """The GPU reproduces the method's own error (not FP32 noise): on the
    small-cube model, linear k-interpolation at sigma_q = 1, 2, 4."""
    g = syn.small_cube()
    op = oracle_plan(g)
    exact = ops.forward(op, g.m)
    errs = {}
    for s in (1.0, 2.0, 4.0):
        gp = gpu_plan(g, slice_interp="linear_k", sigma_q=s)
        eg = rel(host(gp.forward(dev(g.m)), exact.shape), exact)
        eo = rel(lineark.forward(op, g.m, s), exact)
        errs[s] = eg
        assert abs(eg - eo) <= 1e-3 * eo
    assert errs[1.0] > errs[2.0] > errs[4.0]
    print("linear-k relative L2 error vs the exact operator:", errs)


def test_lineark_sparse_solve():
    g = syn.small_cube()
    op = oracle_plan(g)
    s = 2.0
    gp = gpu_plan(g, slice_interp="linear_k", sigma_q=s)
    pair = (lambda m: lineark.forward(op, m, s), lambda r: lineark.adjoint(op, r, s))
    d = ops.forward(op, g.m)
    gamma = float(np.float32(0.95 / fista.power_sigma2(op, d, iters=10, op=pair)))
    lam = float(np.float32(0.05 * np.abs(pair[1](d)).max()))
    ref = fista.solve(op, d, lam, 10, gamma, op=pair)
    m, _ = gp.sparse_solve(dev(d), lam, 10, gamma=gamma, want_info=False)
    assert rel(host(m, ref.shape), ref) <= TOL_SOLVE


def test_lineark_options_checked():
    from paper_2505_00387_gb300._lib import AahrtError
    g = syn.small_cube()
    with pytest.raises(AahrtError):
        gpu_plan(g, slice_interp="linear_k", spread_width=6)
    with pytest.raises(AahrtError):
        gpu_plan(g, slice_interp="linear_k", ngather=2, precision="split_bf16")
    with pytest.raises(AahrtError):
        gpu_plan(g, sigma_q=1.0)          # the spreading kernel needs >= 1.25 nq
