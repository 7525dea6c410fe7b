"""Pins of the oracle's reverse-mode derivative of the unrolled solve.

The map d -> m^n of n ISTA/FISTA iterations (fixed step and threshold, start
0) is evaluated by `fista.solve`, which the pins of test_oracle_pins.py fix.
Its derivative from `fista.unrolled_vjp` is checked against that map alone:

* lambda = 0 makes the shrinkage the identity and the map linear, so
  <m_bar, m^n(d)> = <J^T m_bar, d> holds to rounding;
* lambda > 0: FP64 central differences of <m_bar, m^n(d)> along 64 random
  directions agree with <J^T m_bar, v> (the step is far below the distance
  of any pre-shrinkage value to the threshold).
"""
import numpy as np
import pytest

import oracle
from oracle import fista, ops
from paper_2505_00387_gb300 import synthetic as syn


def small_case(seed=5):
    rng = np.random.default_rng(seed)
    hx, hy = syn.grid_offsets(6, 800.0)
    q0, dq = syn.q_axis(8)
    p = oracle.make_plan(64, 0.008, 64, 8, q0, dq, 4, hx, hy)
    m_true, _ = syn.spike_model(rng, 64, 0.008, 8, q0, dq, 4, nspike=3, tau_rng=(0.1, 0.4))
    d = ops.forward(p, m_true) + 0.05 * rng.standard_normal((p.nt, p.ntr))
    gamma = 0.95 / fista.power_sigma2(p, d)
    lam = 0.05 * float(np.abs(ops.adjoint(p, d)).max())
    m_bar = rng.standard_normal(m_true.shape)
    return p, d, gamma, lam, m_bar, rng


@pytest.mark.parametrize("momentum", [True, False])
def test_vjp_linear_case_is_exact_transpose(momentum):
    p, d, gamma, _, m_bar, _ = small_case()
    m_n, d_bar = fista.unrolled_vjp(p, d, m_bar, 0.0, gamma, 12, momentum)
    # the returned iterate is the solver's
    ref = fista.solve(p, d, 0.0, 12, gamma, momentum=momentum)
    assert np.max(np.abs(m_n - ref)) <= 1e-13 * np.max(np.abs(ref))
    lhs = float(np.vdot(m_bar, m_n))
    rhs = float(np.vdot(d_bar, d))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs))


@pytest.mark.parametrize("momentum,ndir", [(True, 64), (False, 16)])
def test_vjp_matches_central_differences(momentum, ndir):
    p, d, gamma, lam, m_bar, rng = small_case()
    iters = 10
    m_n, d_bar = fista.unrolled_vjp(p, d, m_bar, lam, gamma, iters, momentum)
    # the threshold is active: some entries shrink to zero, some survive
    frac = float(np.mean(m_n != 0.0))
    assert 0.01 < frac < 0.9
    eps = 1e-6 * np.linalg.norm(d)
    fd, an = [], []
    for _ in range(ndir):
        v = rng.standard_normal(d.shape)
        v /= np.linalg.norm(v)
        jp = np.vdot(m_bar, fista.solve(p, d + eps * v, lam, iters, gamma, momentum=momentum))
        jm = np.vdot(m_bar, fista.solve(p, d - eps * v, lam, iters, gamma, momentum=momentum))
        fd.append((jp - jm) / (2.0 * eps))
        an.append(np.vdot(d_bar, v))
    fd, an = np.array(fd), np.array(an)
    assert np.linalg.norm(fd - an) <= 1e-6 * np.linalg.norm(an)
