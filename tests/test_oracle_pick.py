"""Pins of the oracle's velocity pick (eq. vel_est).

A single cell gives its own q; two equal cells their midpoint; the linear
split between neighbouring q cells that the spike generator uses returns the
elliptical curvature the generator put there (so the pick of the exact model
is the generator's ellipse); and after a sparse solve of the data the pick at
each event's intercept time lies within half a q cell of that ellipse.
"""
import numpy as np

import oracle
from oracle import fista, ops, pick
from paper_2505_00387_gb300 import synthetic as syn


def test_single_and_double_cells():
    g = syn.small_cube()
    p = oracle.make_plan(**g.geom_kwargs())
    m = np.zeros((g.ntau, g.nq, g.ntheta))
    m[10, 7, 2] = -3.0
    m[20, 4, 5] = 1.5
    m[20, 9, 5] = -1.5
    q_hat, w = pick.pick(p, m)
    assert q_hat[10, 2] == p.q[7] and w[10, 2] == 3.0
    assert abs(q_hat[20, 5] - 0.5 * (p.q[4] + p.q[9])) < 1e-15
    assert q_hat[0, 0] == 0.0 and w[0, 0] == 0.0


def test_pick_of_generated_model_is_the_ellipse():
    g = syn.small_cube()
    p = oracle.make_plan(**g.geom_kwargs())
    th = np.arange(g.ntheta) * np.pi / g.ntheta
    q_hat, _ = pick.pick(p, g.m)
    for sp in g.info["spikes"]:
        i = int(round(sp["tau"] / g.dt))
        # the spike's Ricker peak (positive) sits on the sample nearest tau;
        # skip samples where another spike overlaps
        if any(abs(o["tau"] - sp["tau"]) < 0.06 for o in g.info["spikes"] if o is not sp):
            continue
        qe = np.clip(syn.ellipse_q(th, sp["v"], sp["v"] / 1.1, sp["axis"]), p.q[0], p.q[-1])
        np.testing.assert_allclose(q_hat[i], qe, rtol=0, atol=1e-6 * g.dq + 1e-3 * g.dq)


def test_pick_after_sparse_solve_tracks_the_ellipse():
    g = syn.small_cube()
    p = oracle.make_plan(**g.geom_kwargs())
    d = ops.forward(p, g.m)
    gamma = 0.95 / fista.power_sigma2(p, d)
    lam = 0.05 * np.abs(ops.adjoint(p, d)).max()
    m = fista.solve(p, d, lam, 60, gamma)
    q_hat, w = pick.pick(p, m)
    th = np.arange(g.ntheta) * np.pi / g.ntheta
    checked = 0
    for sp in g.info["spikes"]:
        if any(abs(o["tau"] - sp["tau"]) < 0.06 for o in g.info["spikes"] if o is not sp):
            continue
        i = int(round(sp["tau"] / g.dt))
        qe = np.clip(syn.ellipse_q(th, sp["v"], sp["v"] / 1.1, sp["axis"]), p.q[0], p.q[-1])
        assert np.max(np.abs(q_hat[i] - qe)) <= 0.5 * g.dq
        checked += 1
    assert checked >= 2
