"""Pins of the oracle's paper-literal slice step (linear interpolation in k,
the A-coefficients of eq. thli).

* Traces whose k_q falls on the k grid at every bin read grid values only:
  the linear interpolation is then exact and equals the exact non-uniform
  DFT of the slice step (the C direct sum).
* Linear interpolation of a smooth spectrum converges at second order:
  doubling the q oversampling divides the error against the exact operator
  by about four.
* The adjoint is the transpose (complex inner products, FP64), also through
  the full operator.
"""
from dataclasses import replace

import numpy as np

import oracle
from oracle import lineark, ops
from paper_2505_00387_gb300 import synthetic as syn


def base_plan(ntr=20, nq=12, ntheta=4, seed=0):
    rng = np.random.default_rng(seed)
    hx, hy = syn.disc_offsets(rng, ntr, 1200.0)
    q0, dq = syn.q_axis(nq)
    return oracle.make_plan(96, 0.008, 96, nq, q0, dq, ntheta, hx, hy)


def test_grid_aligned_traces_are_exact():
    p = base_plan()
    sigma = 2.0
    nos = lineark.grid_size(p.nq, sigma)
    # r^2 = m N ds / (dq nos) puts trace h on grid point k*m at every bin k
    mlist = np.arange(1, p.ntr + 1) % 5 + 1
    r2 = mlist * p.nfft * p.ds / (p.dq * nos)
    pa = replace(p, r2=r2)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((p.nbins, p.nq, p.ntheta)) + 1j * rng.standard_normal(
        (p.nbins, p.nq, p.ntheta))
    Yl = lineark.slice_forward(pa, X, sigma)
    Ye = ops.slice_forward(pa, X)
    assert np.max(np.abs(Yl - Ye)) <= 1e-10 * np.max(np.abs(Ye))


def test_second_order_convergence_in_oversampling():
    p = base_plan(ntr=30, nq=16)
    g = syn.Gather(p.nt, p.dt, p.ntau, p.nq, p.q0, p.dq, p.ntheta, p.hx, p.hy)
    rng = np.random.default_rng(2)
    m, _ = syn.spike_model(rng, p.ntau, p.dt, p.nq, p.q0, p.dq, p.ntheta, nspike=3,
                           tau_rng=(0.1, 0.5))
    assert g.ntr == p.ntr
    exact = ops.forward(p, m)
    errs = [np.linalg.norm(lineark.forward(p, m, s) - exact) / np.linalg.norm(exact)
            for s in (2.0, 4.0, 8.0, 16.0)]
    assert errs[0] > errs[1] > errs[2] > errs[3]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.0 < r < 5.0 for r in ratios[1:]), (errs, ratios)


def test_transposes():
    p = base_plan()
    rng = np.random.default_rng(3)
    X = rng.standard_normal((p.nbins, p.nq, p.ntheta)) + 1j * rng.standard_normal(
        (p.nbins, p.nq, p.ntheta))
    Y = rng.standard_normal((p.nbins, p.ntr)) + 1j * rng.standard_normal((p.nbins, p.ntr))
    for s in (1.0, 2.0):
        lhs = np.vdot(Y, lineark.slice_forward(p, X, s))
        rhs = np.vdot(lineark.slice_adjoint(p, Y, s), X)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    m = rng.standard_normal((p.ntau, p.nq, p.ntheta))
    d = rng.standard_normal((p.nt, p.ntr))
    lhs = np.vdot(lineark.forward(p, m), d)
    rhs = np.vdot(m, lineark.adjoint(p, d))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
