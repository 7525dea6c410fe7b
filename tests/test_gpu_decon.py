"""GPU: the deconvolutive operator W L (eq. DecRT) through the C ABI against
the oracle: forward, adjoint, dot test, sparse solve (graph and eager), the
derivative of the unrolled solve, the allocation-free forward, the
tensor-core plan, and clearing the wavelet."""
import numpy as np
import pytest
import torch

from oracle import decon, fista, ops
from paper_2505_00387_gb300 import synthetic as syn

from gpu_util import dev, gpu_plan, host, oracle_plan, rel

pytestmark = pytest.mark.gpu

TOL_OP = 1e-4
TOL_SOLVE = 1e-3


def wavelet(dt, center=15, n=31, f=25.0, shift=0):
    t = (np.arange(n) - center - shift) * dt
    return syn.ricker(t, f)


@pytest.fixture(scope="module")
def case():
    g = syn.small_cube()
    op = oracle_plan(g)
    gp = gpu_plan(g)
    return g, op, gp


@pytest.mark.parametrize("center,shift", [(15, 0), (0, 0), (30, 0), (12, 3)])
def test_forward_adjoint_dot(case, center, shift):
    g, op, gp = case
    w = wavelet(g.dt, center=center, shift=shift)
    gp.set_wavelet(w, center)
    rng = np.random.default_rng(90)
    m = rng.standard_normal(g.m.shape)
    d = rng.standard_normal((g.nt, g.ntr))
    dg = host(gp.forward(dev(m)), d.shape)
    mg = host(gp.adjoint(dev(d)), m.shape)
    wf = w.astype(np.float32).astype(np.float64)
    assert rel(dg, decon.forward(op, m, wf, center)) < TOL_OP
    assert rel(mg, decon.adjoint(op, d, wf, center)) < TOL_OP
    # dot test on a well-conditioned pair: d2 = W L m by the oracle plus as
    # much noise, so <W L m, d2> is about |W L m|^2 (for two independent
    # random vectors the inner product is itself often near zero)
    m32 = m.astype(np.float32).astype(np.float64)
    lm = decon.forward(op, m32, wf, center)
    d2 = lm + np.sqrt(np.mean(lm * lm)) * rng.standard_normal(lm.shape)
    d2 = d2.astype(np.float32).astype(np.float64)
    lhs = float(np.sum(host(gp.forward(dev(m32)), d.shape) * d2))
    rhs = float(np.sum(host(gp.adjoint(dev(d2)), m.shape) * m32))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    gp.set_wavelet(None, 0)


def test_sparse_solve_and_vjp(case):
    g, op, gp = case
    w = wavelet(g.dt).astype(np.float32)
    wf = w.astype(np.float64)
    gp.set_wavelet(w, 15)
    pair = (lambda m: decon.forward(op, m, wf, 15), lambda r: decon.adjoint(op, r, wf, 15))
    d = decon.forward(op, g.m, wf, 15)
    gamma = float(np.float32(0.95 / fista.power_sigma2(op, d, op=pair)))
    lam = float(np.float32(0.05 * np.abs(pair[1](d)).max()))
    ref = fista.solve(op, d, lam, 20, gamma, op=pair)
    for graph in (True, False):
        m, _ = gp.sparse_solve(dev(d), lam, 20, gamma=gamma, use_graph=graph, want_info=False)
        assert rel(host(m, ref.shape), ref) <= TOL_SOLVE
    # derivative of the unrolled deconvolutive solve, linear case: transpose identity
    rng = np.random.default_rng(91)
    m_bar = rng.standard_normal(g.m.shape)
    m_n, d_bar = gp.fista_vjp(dev(d), dev(m_bar), 0.0, gamma, 8, checkpoint=3)
    lhs = float(np.sum(host(m_n) * m_bar.ravel()))
    rhs = float(np.sum(host(d_bar) * d.ravel()))
    assert abs(lhs - rhs) <= 1e-4 * (abs(lhs) + abs(rhs))
    gp.set_wavelet(None, 0)


def test_noalloc_and_clearing(case):
    from paper_2505_00387_gb300 import _lib as L
    g, op, gp = case
    rng = np.random.default_rng(92)
    m = dev(rng.standard_normal(g.m.shape))
    plain = gp.forward(m).clone()
    w = wavelet(g.dt).astype(np.float32)
    gp.set_wavelet(w, 15)
    dw = gp.forward(m).clone()
    d_na = torch.empty_like(dw)
    L.aahrt_forward_noalloc(gp.handle, m.data_ptr(), d_na.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(dw, d_na)
    gp.set_wavelet(None, 0)
    assert torch.equal(gp.forward(m), plain)


def test_rejects_bad_wavelet(case):
    from paper_2505_00387_gb300._lib import AahrtError
    g, op, gp = case
    with pytest.raises(AahrtError):
        gp.set_wavelet(np.ones(5, np.float32), 5)
    with pytest.raises(AahrtError):
        gp.set_wavelet(np.array([1.0, np.nan], np.float32), 0)


def test_tensorcore_plan_with_wavelet():
    g = syn.small_cube()
    op = oracle_plan(g)
    G = 3
    gp = gpu_plan(g, ngather=G, precision="split_bf16")
    w = wavelet(g.dt).astype(np.float32)
    gp.set_wavelet(w, 15)
    rng = np.random.default_rng(93)
    ms = [rng.standard_normal(g.m.shape) for _ in range(G)]
    dg = host(gp.forward(dev(np.stack(ms, axis=-1)))).reshape(g.nt, g.ntr, G)
    gp.status()
    for i in range(G):
        assert rel(dg[..., i], decon.forward(op, ms[i], w.astype(np.float64), 15)) < TOL_OP
