"""Pins of the oracle's curvature-range tools (Sec. 3.5, eqs. q1-q3) and of
its operator on a non-uniform (uniform-slowness) curvature axis.

* non-uniform q: the slice step on cell l equals the band-limited time-domain
  delay by q_l r^2/ds samples, an exact circular delay when that is an
  integer, and the operator matches the physical-domain Riemann sum along
  the hyperbolae of eq. Inverse at uniform-slowness curvatures;
* partial NMO: identity at q_ref = 0, exact transpose, events moved from q
  to q - q_ref (Riemann sum at both curvatures), inverse by -q_ref;
* eq. q3: the sample count is the smallest whose step keeps the largest
  k_q = f' r^2 inside one period of the DFT along q;
* end to end: data with events in [q_a, q_b], partially NMO'd by the range
  centre, are inverted on a centred axis of eq. q3's (smaller) sample count
  and the events land at q - q_ref.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import checks, fista, ops, pnmo
from paper_2505_00387_gb300 import synthetic as syn


def slowness_axis(nq):
    return pnmo.q_axis_slowness(syn.P_MIN, syn.P_MAX, nq)


# ------------------------------------------------------- uniform slowness axis
def test_slowness_axis_closed_form():
    q = slowness_axis(9)
    p = np.sqrt(q)
    np.testing.assert_allclose(np.diff(p), (syn.P_MAX - syn.P_MIN) / 8, rtol=1e-12)
    assert q[0] == pytest.approx(syn.P_MIN ** 2, rel=1e-15)
    assert q[-1] == pytest.approx(syn.P_MAX ** 2, rel=1e-15)
    # non-uniform in q: the steps grow linearly with p
    assert np.all(np.diff(np.diff(q)) > 0)


def test_plan_with_q_axis_no_wrap():
    """rho uses max |q_l| of the explicit axis; a centred axis with negative
    curvatures keeps the no-wrap frame."""
    hx, hy = syn.grid_offsets(8, 1500.0)
    for qa in (slowness_axis(7), np.linspace(-1.5e-7, 1.0e-7, 6)):
        p = oracle.make_plan(128, 0.008, 128, len(qa), 0.0, 0.0, 4, hx, hy, q_axis=qa)
        rho = np.abs(qa).max() * p.r2.max() / p.tmax ** 2
        assert p.rho == pytest.approx(rho, rel=1e-14)
        assert (p.ns - 1) * (1.0 + p.rho) <= p.nfft - 2
        np.testing.assert_array_equal(p.q, qa)
    with pytest.raises(ValueError):
        oracle.make_plan(128, 0.008, 128, 3, 0.0, 0.0, 4, hx, hy, q_axis=[1e-7, np.nan, 2e-7])


def test_nonuniform_slice_matches_time_domain_shift():
    """Each cell l of a uniform-slowness axis is delayed by q_l r^2/ds."""
    rng = np.random.default_rng(31)
    nq, nth = 5, 4
    ang = 2 * np.pi / nth                       # exactly on slice 2
    hx = np.array([800.0 * np.cos(ang), 1500.0 * np.cos(ang)])
    hy = np.array([800.0 * np.sin(ang), 1500.0 * np.sin(ang)])
    p = oracle.make_plan(80, 0.008, 80, nq, 0.0, 0.0, nth, hx, hy, q_axis=slowness_axis(nq))
    xs = np.zeros(p.ns)
    xs[4:50] = rng.standard_normal(46)
    for l in (0, 2, 4):
        X = np.zeros((p.nbins, nq, nth), complex)
        X[:, l, 2] = ops.rfft_bins(p, xs[:, None])[:, 0]
        dp = ops.irfft_bins(p, ops.slice_forward(p, X))
        for h in range(2):
            want = checks.time_domain_shift(xs, p.q[l] * p.r2[h] / p.ds, p.nfft, p.kmax, p.ns)
            np.testing.assert_allclose(dp[:, h], want, atol=1e-12 * np.abs(want).max())


def test_nonuniform_integer_shift_is_exact_delay():
    rng = np.random.default_rng(32)
    nq, nth = 4, 2
    base = oracle.make_plan(64, 0.008, 64, nq, 0.0, 0.0, nth, np.array([1500.0]),
                            np.array([0.0]), q_axis=slowness_axis(nq))
    l, s0 = 1, 7                               # below the largest q: ds unchanged
    qa = base.q.copy()
    qa[l] = s0 * base.ds / base.r2[0]
    assert qa[l] < qa[-1]
    p = replace(base, q_axis=qa)
    xs = np.zeros(p.ns)
    xs[2:30] = rng.standard_normal(28)
    X = np.zeros((p.nbins, nq, nth), complex)
    X[:, l, 0] = ops.rfft_bins(p, xs[:, None])[:, 0]
    dp = ops.irfft_bins(p, ops.slice_forward(p, X))[:, 0]
    full = np.zeros(p.nfft)
    full[: p.ns] = xs
    alt = (-1.0) ** np.arange(p.nfft)
    proj = full - np.dot(full, alt) / p.nfft * alt
    np.testing.assert_allclose(dp, np.roll(proj, s0)[: p.ns], atol=1e-13)


def test_nonuniform_riemann_sum_brute_force():
    nt, dt, nq, nth = 500, 0.004, 12, 4
    r = np.linspace(100.0, 1600.0, 8)
    hx = np.concatenate([r * np.cos(j * np.pi / nth) for j in range(nth)])
    hy = np.concatenate([r * np.sin(j * np.pi / nth) for j in range(nth)])
    p = oracle.make_plan(nt, dt, nt, nq, 0.0, 0.0, nth, hx, hy, q_axis=slowness_axis(nq))
    events = [(1.0, 0.8, 15.0, 2, 0), (-0.7, 1.2, 12.0, 9, 1), (0.6, 1.5, 16.0, 11, 3)]
    m = np.zeros((nt, nq, nth))
    tau = np.arange(nt) * dt
    ev = []
    for a, te, f, l, j in events:
        m[:, l, j] += a * checks.ricker(tau - te, f)
        ev.append((a, te, f, p.q[l], j))
    d = ops.forward(p, m)
    wmaps = [{int(p.j0[h]): p.w0[h]} for h in range(p.ntr)]
    for h in range(p.ntr):
        wmaps[h][int(p.j1[h])] = wmaps[h].get(int(p.j1[h]), 0.0) + p.w1[h]
    want = checks.riemann_sum_forward(nt, dt, p.r2, wmaps, ev)
    assert np.linalg.norm(d - want) / np.linalg.norm(want) < 2e-2


@pytest.mark.parametrize("qa", [slowness_axis(7), np.array([-1.2e-7, -3e-8, 0.0, 4e-8, 1.1e-7])])
def test_nonuniform_dot_product(qa):
    rng = np.random.default_rng(33)
    hx, hy = syn.disc_offsets(rng, 14, 1300.0)
    p = oracle.make_plan(96, 0.008, 96, len(qa), 0.0, 0.0, 5, hx, hy, q_axis=qa)
    m = rng.standard_normal((p.ntau, p.nq, p.ntheta))
    d = rng.standard_normal((p.nt, p.ntr))
    lhs = np.sum(ops.forward(p, m) * d)
    assert abs(lhs - np.sum(m * ops.adjoint(p, d))) <= 1e-12 * abs(lhs)


def test_explicit_uniform_axis_is_the_uniform_plan():
    rng = np.random.default_rng(34)
    hx, hy = syn.disc_offsets(rng, 10, 1200.0)
    q0, dq = syn.q_axis(6)
    a = oracle.make_plan(80, 0.008, 80, 6, q0, dq, 4, hx, hy)
    b = oracle.make_plan(80, 0.008, 80, 6, 0.0, 0.0, 4, hx, hy, q_axis=q0 + dq * np.arange(6))
    assert (a.nfft, a.ns, a.ds) == (b.nfft, b.ns, b.ds)
    m = rng.standard_normal((80, 6, 4))
    np.testing.assert_allclose(ops.forward(b, m), ops.forward(a, m), atol=1e-12)


# ------------------------------------------------------------- partial NMO
def pnmo_plan(interp="keys", nt=400, dt=0.004):
    r = np.linspace(150.0, 1800.0, 12)
    return oracle.make_plan(nt, dt, nt, 2, 0.0, 1e-8, 4, r, np.zeros_like(r), interp=interp)


def test_partial_nmo_zero_is_identity():
    p = pnmo_plan()
    d = np.random.default_rng(35).standard_normal((p.nt, p.ntr))
    np.testing.assert_allclose(pnmo.partial_nmo(p, d, 0.0), d, atol=1e-12)


@pytest.mark.parametrize("interp", ["keys", "linear"])
@pytest.mark.parametrize("q_ref", [2.1e-7, -1.3e-7])
def test_partial_nmo_transpose(interp, q_ref):
    p = pnmo_plan(interp)
    rng = np.random.default_rng(36)
    d = rng.standard_normal((p.nt, p.ntr))
    e = rng.standard_normal((p.nt, p.ntr))
    lhs = np.sum(pnmo.partial_nmo(p, d, q_ref) * e)
    rhs = np.sum(d * pnmo.partial_nmo_T(p, e, q_ref))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("q_ref", [2.0e-7, -1.0e-7])
def test_partial_nmo_moves_events_to_q_minus_qref(q_ref):
    """eq. Inverse's hyperbola at q, partially NMO'd by q_ref, is the one at
    q - q_ref (Riemann sums on both sides; interpolation-limited)."""
    p = pnmo_plan()
    w = [{0: 1.0} for _ in range(p.ntr)]
    ev = [(1.0, 0.5, 14.0, 3.0e-7, 0), (-0.8, 0.9, 11.0, 1.5e-7, 0), (0.6, 1.2, 15.0, 2.4e-7, 0)]
    d = checks.riemann_sum_forward(p.nt, p.dt, p.r2, w, ev)
    want = checks.riemann_sum_forward(p.nt, p.dt, p.r2, w,
                                      [(a, te, f, q - q_ref, s) for a, te, f, q, s in ev])
    got = pnmo.partial_nmo(p, d, q_ref)
    t = np.arange(p.nt) * p.dt
    u = np.sqrt(np.maximum(t[:, None] ** 2 + q_ref * p.r2[None, :], 0.0)) / p.dt
    inside = u <= p.nt - 3                     # every tap reads the input axis
    err = np.linalg.norm((got - want)[inside]) / np.linalg.norm(want[inside])
    assert err < 1e-2, err
    # inverse: the same map with -q_ref takes the data back
    back = pnmo.partial_nmo(p, got, -q_ref)
    v = np.sqrt(np.maximum(t[:, None] ** 2 - q_ref * p.r2[None, :], 0.0)) / p.dt
    ok = inside & (u <= p.nt - 6) & (v <= p.nt - 3) & (t[:, None] ** 2 - q_ref * p.r2[None, :] > 0.0)
    assert np.linalg.norm((back - d)[ok]) / np.linalg.norm(d[ok]) < 2e-2


# --------------------------------------------------------------- eq. q3
@pytest.mark.parametrize("span,fmax,r2max", [(6.2e-7, 60.0, 4.5e6), (1.98e-7, 60.0, 4.5e6),
                                             (3e-8, 250.0, 9e6), (1e-9, 1.0, 1.0)])
def test_nq_required_is_the_tight_eq_q3_bound(span, fmax, r2max):
    n = pnmo.nq_required(span, fmax, r2max)
    # the step span/n keeps the largest k_q = fmax r2max within one period
    # 1/dq of the DFT along q; one sample fewer does not
    assert (span / n) * fmax * r2max <= 1.0 + 1e-12
    if n > 1:
        assert (span / (n - 1)) * fmax * r2max > 1.0
    # the paper's symmetric axis [-q_max, q_max]: N_q >= 2 q_max f'max r^2max
    qmax = span / 2
    assert n >= 2 * qmax * fmax * r2max - 1e-9


def test_partial_nmo_shrinks_eq_q3():
    qa, qb = (1 / 3000.0) ** 2, (1 / 1800.0) ** 2
    full = pnmo.nq_required(2 * max(abs(qa), abs(qb)), 60.0, 4.5e6)
    centred = pnmo.nq_required(qb - qa, 60.0, 4.5e6)
    assert centred < full
    assert centred / full == pytest.approx((qb - qa) / (2 * qb), abs=2.0 / full)


def test_centred_axis_after_partial_nmo_recovers_curvature():
    """Events with curvatures in [q_a, q_b] (Riemann sum of eq. Inverse),
    partially NMO'd by q_ref = (q_a + q_b)/2, inverted on a centred axis of
    eq. q3's sample count: each event's energy peaks at q_e - q_ref."""
    nt, dt, nth = 160, 0.008, 2
    hx, hy = syn.grid_offsets(8, 1400.0)
    qa, qb = (1 / 3000.0) ** 2, (1 / 2000.0) ** 2
    q_ref = 0.5 * (qa + qb)
    fmax = 12.0                                 # stretched frequency band kept, 1/s^2
    r2max = float(np.max(hx * hx + hy * hy))
    nq = pnmo.nq_required(qb - qa, fmax, r2max) + 2
    half = 0.5 * (qb - qa) * nq / (nq - 2)
    qc = np.linspace(-half, half, nq)
    p = oracle.make_plan(nt, dt, nt, nq, 0.0, 0.0, nth, hx, hy, q_axis=qc, fmax=fmax)
    p0 = oracle.make_plan(nt, dt, nt, 2, 0.0, 1e-8, nth, hx, hy)
    w = [{int(p0.j0[h]): p0.w0[h]} for h in range(p0.ntr)]
    for h in range(p0.ntr):
        w[h][int(p0.j1[h])] = w[h].get(int(p0.j1[h]), 0.0) + p0.w1[h]
    qe = [qa + 0.2 * (qb - qa), qa + 0.8 * (qb - qa)]
    ev = [(1.0, 0.35, 6.0, qe[0], 0), (1.0, 0.75, 6.0, qe[1], 0)]
    d = checks.riemann_sum_forward(nt, dt, p0.r2, w, ev)
    dn = pnmo.partial_nmo(p, d, q_ref)
    gamma = 0.95 / fista.power_sigma2(p, dn, iters=30)
    lam = 0.05 * np.abs(ops.adjoint(p, dn)).max()
    m = fista.solve(p, dn, lam, 60, gamma)
    for (a, te, f, q, _) in ev:
        i = int(round(te / dt))
        prof = np.sum(np.abs(m[i - 4:i + 5, :, :]), axis=(0, 2))
        l_hat = int(np.argmax(prof))
        l_true = int(np.argmin(np.abs(qc - (q - q_ref))))
        assert abs(l_hat - l_true) <= 1, (l_hat, l_true)
