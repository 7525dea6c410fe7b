"""GPU: autograd of L and the unrolled sparse solve through the C ABI.

* backward of d = L m is the oracle's L^T (and vice versa), <= 1e-4;
* aahrt_fista_vjp against the oracle's reverse-mode derivative of the same
  unrolled solve (small_cube cube, FISTA and ISTA, several checkpoint spacings);
* at the paper-scale geometry, where the FP64 oracle is too slow for
  central differences, GPU FP32 central differences of <m_bar, m^n(d)> along
  64 random directions against <d_bar, v> (loose tolerance, FP32; steps and
  iteration counts where the differences stay on one linear piece).
"""
import numpy as np
import pytest
import torch

from oracle import fista, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, gpu_plan, host, oracle_plan, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case0():
    g = syn.small_cube()
    op = oracle_plan(g)
    gp = gpu_plan(g)
    d = ops.forward(op, g.m)
    rng = np.random.default_rng(20)
    d = d + 0.05 * np.sqrt(np.mean(d * d)) * rng.standard_normal(d.shape)
    gamma = 0.95 / fista.power_sigma2(op, d)
    lam = 0.05 * float(np.abs(ops.adjoint(op, d)).max())
    return g, op, gp, d, float(np.float32(gamma)), float(np.float32(lam)), rng


def test_radon_backward_is_oracle_adjoint(case0):
    from paper_2505_00387_gb300.autograd import radon, radon_adjoint
    g, op, gp, d, _, _, rng = case0
    m = dev(rng.standard_normal(g.m.shape)).requires_grad_(True)
    w = rng.standard_normal(d.shape)
    out = radon(gp, m)
    (out * dev(w)).sum().backward()
    assert rel(host(m.grad, g.m.shape), ops.adjoint(op, w)) <= 1e-4
    # the adjoint's backward is L
    dd = dev(rng.standard_normal(d.shape)).requires_grad_(True)
    v = rng.standard_normal(g.m.shape)
    (radon_adjoint(gp, dd) * dev(v)).sum().backward()
    assert rel(host(dd.grad, d.shape), ops.forward(op, v)) <= 1e-4


@pytest.mark.parametrize("ista,iters,ck", [(False, 20, 5), (False, 20, 7), (False, 12, 0),
                                           (True, 15, 4), (False, 6, 50)])
def test_fista_vjp_matches_oracle(case0, ista, iters, ck):
    g, op, gp, d, gamma, lam, rng = case0
    m_bar = rng.standard_normal(g.m.shape)
    m_ref, db_ref = fista.unrolled_vjp(op, d, m_bar, lam, gamma, iters, momentum=not ista)
    m_n, d_bar = gp.fista_vjp(dev(d), dev(m_bar), lam, gamma, iters, ista=ista, checkpoint=ck)
    torch.cuda.synchronize()
    assert rel(host(m_n, g.m.shape), m_ref) <= 1e-3
    assert rel(host(d_bar, d.shape), db_ref) <= 1e-3


def test_fista_vjp_linear_case(case0):
    g, op, gp, d, gamma, _, rng = case0
    m_bar = rng.standard_normal(g.m.shape)
    m_ref, db_ref = fista.unrolled_vjp(op, d, m_bar, 0.0, gamma, 10)
    m_n, d_bar = gp.fista_vjp(dev(d), dev(m_bar), 0.0, gamma, 10, checkpoint=3)
    assert rel(host(d_bar, d.shape), db_ref) <= 1e-4
    assert rel(host(m_n, g.m.shape), m_ref) <= 1e-4


def test_fista_vjp_result_is_the_solvers(case0):
    g, op, gp, d, gamma, lam, rng = case0
    dd = dev(d)
    m_bar = dev(rng.standard_normal(g.m.shape))
    m_n, _ = gp.fista_vjp(dd, m_bar, lam, gamma, 20, checkpoint=6)
    m_s, _ = gp.sparse_solve(dd, lam, 20, gamma=gamma, want_info=False)
    torch.cuda.synchronize()
    a, b = host(m_n), host(m_s)
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))


def test_fista_vjp_zero_iterations(case0):
    g, op, gp, d, gamma, lam, rng = case0
    m_n, d_bar = gp.fista_vjp(dev(d), dev(rng.standard_normal(g.m.shape)), lam, gamma, 0)
    assert float(m_n.abs().max()) == 0.0 and float(d_bar.abs().max()) == 0.0


def test_fista_vjp_rejects_bad_arguments(case0):
    from paper_2505_00387_gb300._lib import AahrtError
    g, op, gp, d, gamma, lam, rng = case0
    dd, mb = dev(d), dev(rng.standard_normal(g.m.shape))
    with pytest.raises(AahrtError):
        gp.fista_vjp(dd, mb, lam, 0.0, 5)
    with pytest.raises(AahrtError):
        gp.fista_vjp(dd, mb, -1.0, gamma, 5)
    with pytest.raises(AahrtError):
        gp.fista_vjp(dd, mb, lam, gamma, -1)


def test_autograd_fista_layer_backward(case0):
    from paper_2505_00387_gb300.autograd import fista as fista_layer
    g, op, gp, d, gamma, lam, rng = case0
    m_bar = rng.standard_normal(g.m.shape)
    dd = dev(d).requires_grad_(True)
    m = fista_layer(gp, dd, lam, gamma, 12, checkpoint=4)
    (m * dev(m_bar)).sum().backward()
    _, db_ref = fista.unrolled_vjp(op, d, m_bar, lam, gamma, 12)
    assert rel(host(dd.grad, d.shape), db_ref) <= 1e-3


@pytest.mark.slow
def test_fista_vjp_matches_oracle_50_iterations(case0):
    g, op, gp, d, gamma, lam, rng = case0
    m_bar = rng.standard_normal(g.m.shape)
    m_ref, db_ref = fista.unrolled_vjp(op, d, m_bar, lam, gamma, 50)
    m_n, d_bar = gp.fista_vjp(dev(d), dev(m_bar), lam, gamma, 50, checkpoint=10)
    assert rel(host(m_n, g.m.shape), m_ref) <= 1e-3
    assert rel(host(d_bar, d.shape), db_ref) <= 1e-3


@pytest.fixture(scope="module")
def case1():
    g = syn.paper_gather()
    gp = gpu_plan(g)
    d = dev(g.d)
    _, info = gp.sparse_solve(d, 0.0, 0, lambda_rel=0.05)   # gamma and lambda of the data
    return gp, d, float(np.float32(info.gamma)), float(np.float32(getattr(info, "lambda")))


# The unrolled map is piecewise linear in d; with the threshold on, a
# perturbation of relative size eps moves some pre-shrinkage values across
# gamma*lambda, and the central difference then averages slopes of several
# pieces.  Measured at this gather (6 directions): 50 FISTA iterations give
# 25-50 % disagreement for eps >= 3e-4 and 7 % at 1e-4, where FP32 noise
# takes over; 50 ISTA iterations and 10 FISTA iterations give about 1 % at
# eps = 1e-4.  The threshold-free (linear) map is checked at eps = 1e-3.
@pytest.mark.slow
@pytest.mark.parametrize("ista,thresholded,iters,eps,tol", [
    (False, False, 50, 1e-3, 1e-2),
    (True, True, 50, 1e-4, 3e-2),
    (False, True, 10, 1e-4, 3e-2)])
def test_fista_vjp_central_differences_paper_scale(case1, ista, thresholded, iters, eps, tol):
    """64 directions at the paper-scale gather: FP32 central differences of
    <m_bar, m^n(d)> (step eps |d|) against <d_bar, v>."""
    gp, d, gamma, lam = case1
    lam = lam if thresholded else 0.0
    rng = np.random.default_rng(2)
    m_bar = dev(rng.standard_normal(gp.model_len))
    _, d_bar = gp.fista_vjp(d, m_bar, lam, gamma, iters, ista=ista, checkpoint=10)
    dn = float(torch.linalg.norm(d.double()))
    fd, an = [], []
    for _ in range(64):
        v = dev(rng.standard_normal(gp.data_len))
        v *= dn / float(torch.linalg.norm(v.double()))
        mp, _ = gp.sparse_solve(d + eps * v, lam, iters, gamma=gamma, ista=ista,
                                want_info=False)
        mm, _ = gp.sparse_solve(d - eps * v, lam, iters, gamma=gamma, ista=ista,
                                want_info=False)
        fd.append(float(torch.dot(m_bar.double(), (mp.double() - mm.double()))) / (2 * eps))
        an.append(float(torch.dot(d_bar.double(), v.double())))
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= tol * np.linalg.norm(an)
