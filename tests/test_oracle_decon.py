"""Pins of the oracle's deconvolutive operator W L (eq. DecRT).

W is fixed by numpy's full linear convolution (an independent routine), its
transpose by inner products, the composite by the plain operator it reduces
to for a unit pulse, and the purpose of the construction -- time resolution
of the sparse transform -- by recovering isolated spikes from band-limited
data at their own intercept times.
"""
import numpy as np
import pytest

import oracle
from oracle import decon, fista, ops
from paper_2505_00387_gb300 import synthetic as syn


def small_plan(nt=96, ntr=36, nq=8, ntheta=4):
    hx, hy = syn.grid_offsets(6, 700.0)
    q0, dq = syn.q_axis(nq)
    return oracle.make_plan(nt, 0.004, nt, nq, q0, dq, ntheta, hx[:ntr], hy[:ntr])


@pytest.mark.parametrize("center", [0, 7, 12, 30])
def test_conv_matches_numpy_full_convolution(center):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((50, 3))
    w = rng.standard_normal(13)
    out = decon.conv_t(x, w, center)
    for h in range(3):
        full = np.convolve(x[:, h], w)               # full[i] = sum_s w[s] x[i - s]
        ref = np.zeros(50)
        lo, hi = center, min(center + 50, full.size)
        if lo < full.size:
            ref[:hi - lo] = full[lo:hi]
        np.testing.assert_allclose(out[:, h], ref, rtol=0, atol=1e-13)


def test_corr_is_the_transpose():
    rng = np.random.default_rng(2)
    nt, w, c = 40, rng.standard_normal(9), 4
    Wm = np.stack([decon.conv_t(np.eye(nt)[:, [i]], w, c)[:, 0] for i in range(nt)], axis=1)
    y = rng.standard_normal((nt, 2))
    np.testing.assert_allclose(decon.corr_t(y, w, c), Wm.T @ y, rtol=0, atol=1e-13)


def test_unit_pulse_reduces_to_plain_operator_and_dot_test():
    p = small_plan()
    rng = np.random.default_rng(3)
    m = rng.standard_normal((p.ntau, p.nq, p.ntheta))
    d = rng.standard_normal((p.nt, p.ntr))
    np.testing.assert_allclose(decon.forward(p, m, [1.0], 0), ops.forward(p, m), rtol=0,
                               atol=1e-14)
    w = syn.ricker((np.arange(21) - 10) * p.dt, 30.0)
    lhs = np.vdot(decon.forward(p, m, w, 10), d)
    rhs = np.vdot(m, decon.adjoint(p, d, w, 10))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_sparse_deconvolutive_transform_resolves_spikes():
    """Band-limited events d = W L m from three isolated cells: the sparse
    solve with W L puts its largest coefficients on those cells, the solve
    with L alone smears them over the wavelet's length in tau."""
    p = small_plan(nt=128)
    w = syn.ricker((np.arange(31) - 15) * p.dt, 30.0)
    m_true = np.zeros((p.ntau, p.nq, p.ntheta))
    cells = [(30, 2, 1), (64, 5, 2), (95, 3, 3)]
    for (i, l, j) in cells:
        m_true[i, l, j] = 1.0
    d = decon.forward(p, m_true, w, 15)
    op_w = (lambda m: decon.forward(p, m, w, 15), lambda r: decon.adjoint(p, r, w, 15))
    res = {}
    for name, op in (("decon", op_w), ("plain", None)):
        fwd_adj = op if op is not None else (lambda m: ops.forward(p, m),
                                             lambda r: ops.adjoint(p, r))
        gamma = 0.95 / fista.power_sigma2(p, d, op=fwd_adj)
        lam = 0.02 * np.abs(fwd_adj[1](d)).max()
        m = fista.solve(p, d, lam, 200, gamma, op=fwd_adj)
        near = np.zeros_like(m, bool)
        for (i, l, j) in cells:
            near[max(i - 1, 0):i + 2, max(l - 1, 0):l + 2, j] = True
        res[name] = float(np.sum(m[near] ** 2) / np.sum(m ** 2))
        if name == "decon":
            for (i, l, j) in cells:
                col = np.abs(m[:, l, j])
                assert abs(int(np.argmax(col)) - i) <= 1
    assert res["decon"] > 0.8
    assert res["decon"] > res["plain"] + 0.2
