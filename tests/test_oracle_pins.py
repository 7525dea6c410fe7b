"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test evaluates a quantity by a route independent of the oracle's own
code (explicit sums, closed forms, invariants, brute force), so that a
dropped term, a wrong sign or index, or a transposed operand fails one.
"""
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle
from oracle import checks, fista, ops
from paper_2505_00387_gb300 import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_plan(ntr=12, nt=96, dt=0.008, nq=6, ntheta=4, seed=0, **kw):
    rng = np.random.default_rng(seed)
    hx, hy = syn.disc_offsets(rng, ntr, 1200.0)
    q0, dq = syn.q_axis(nq)
    return oracle.make_plan(nt, dt, nt, nq, q0, dq, ntheta, hx, hy, **kw)


# ------------------------------------------------------------ plan (eq. q3)
@pytest.mark.parametrize("cfg", [0, 1])
def test_plan_sampling_no_wrap(cfg):
    g = syn.small_cube() if cfg == 0 else syn.paper_gather()
    p = oracle.make_plan(**g.geom_kwargs())
    assert p.nfft & (p.nfft - 1) == 0
    assert p.nfft >= 2.0 * p.nt * (1.0 + p.rho)
    assert p.nfft // 2 < 2.0 * p.nt * (1.0 + p.rho)
    # largest moveout stays inside the frame, and Ns is the largest such count
    assert (p.ns - 1) * (1.0 + p.rho) <= p.nfft - 2
    assert p.ns * (1.0 + p.rho) > p.nfft - 2
    assert abs((p.ns - 1) * p.ds - p.tmax ** 2) < 1e-12 * p.tmax ** 2
    assert p.kmax == p.nfft // 2 - 1
    expect = {0: (1024, 512), 1: (4096, 2048)}[cfg]
    assert (p.nfft, p.nbins) == expect


def test_plan_fmax_limits_bins():
    p = tiny_plan()
    f_lim = 0.3 / (2.0 * p.ds)
    p2 = tiny_plan(fmax=f_lim)
    assert p2.kmax == int(np.floor(f_lim * p.nfft * p.ds)) < p.kmax
    assert p2.freqs[-1] <= f_lim < p2.freqs[-1] + 1.0 / (p.nfft * p.ds)


# -------------------------------------------------- azimuth weights (thli)
def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "azimuth_weights.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                a = line.split()
                rows.append((int(a[0]), float(a[1]), int(a[2]), int(a[3]),
                             float(a[4]), float(a[5])))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_azimuth_weights_golden(row):
    nth, deg, j0, j1, w0, w1 = row
    ang = np.deg2rad(deg)
    r2, th, jj0, jj1, ww0, ww1 = oracle.plan.azimuth_bins(
        np.array([1000.0 * np.cos(ang)]), np.array([1000.0 * np.sin(ang)]), nth)

    def as_map(a, b, wa, wb):
        out = {}
        for j, w in ((a, wa), (b, wb)):
            out[int(j)] = out.get(int(j), 0.0) + float(w)
        return {j: w for j, w in out.items() if abs(w) > 1e-12}

    got = as_map(jj0[0], jj1[0], ww0[0], ww1[0])
    want = as_map(j0, j1, w0, w1)
    assert got.keys() == want.keys()
    for j in want:
        assert abs(got[j] - want[j]) < 1e-12


def test_azimuth_weights_invariants():
    rng = np.random.default_rng(3)
    hx, hy = syn.disc_offsets(rng, 5000, 3000.0)
    for nth in (1, 3, 8, 36):
        r2, th, j0, j1, w0, w1 = oracle.plan.azimuth_bins(hx, hy, nth)
        dth = np.pi / nth
        assert np.all((th >= 0) & (th < np.pi))
        assert np.all((w0 >= 0) & (w1 >= 0))
        np.testing.assert_allclose(w0 + w1, 1.0, atol=1e-15)
        # linear interpolation reproduces theta itself (periodic extension)
        thj0 = j0 * dth
        thj1 = thj0 + dth
        np.testing.assert_allclose(w0 * thj0 + w1 * thj1, th, atol=1e-12)
        assert np.all(j1 == (j0 + 1) % nth)


# ----------------------------------------------- Keys / linear resampling
@pytest.mark.parametrize("interp", ["keys", "linear"])
def test_stretch_reproduces_polynomials(interp):
    """Keys' kernel reproduces quadratics exactly, the linear kernel linears:
    so S applied to m(tau) = a + b tau (+ c tau^2) must return m(sqrt(s))
    at s_n = n ds away from the ends (fixes u = sqrt(s)/dt and the taps)."""
    p = tiny_plan(interp=interp)
    tau = np.arange(p.ntau) * p.dt
    a, b, c = 0.3, -1.7, (2.1 if interp == "keys" else 0.0)
    m = (a + b * tau + c * tau ** 2)[:, None]
    ms = ops.stretch(p, m)[:, 0]
    s = np.arange(p.ns) * p.ds
    u = np.sqrt(s) / p.dt
    inner = (u >= 1.0) & (u <= p.ntau - 3.0)
    np.testing.assert_allclose(ms[inner], (a + b * np.sqrt(s) + c * s)[inner],
                               atol=1e-12)


@pytest.mark.parametrize("interp", ["keys", "linear"])
def test_unstretch_reproduces_polynomials(interp):
    p = tiny_plan(interp=interp)
    s = np.arange(p.ns) * p.ds
    a, b, c = -0.4, 0.9, (0.35 if interp == "keys" else 0.0)
    dp = (a + b * s + c * s * s)[:, None]
    d = ops.unstretch(p, dp)[:, 0]
    t = np.arange(p.nt) * p.dt
    v = t * t / p.ds
    inner = (v >= 1.0) & (v <= p.ns - 3.0)
    np.testing.assert_allclose(d[inner], (a + b * t ** 2 + c * t ** 4)[inner],
                               atol=1e-12)


def test_resampler_transposes():
    p = tiny_plan()
    rng = np.random.default_rng(1)
    x = rng.standard_normal((p.ntau, 3))
    y = rng.standard_normal((p.ns, 3))
    assert abs(np.sum(ops.stretch(p, x) * y) - np.sum(x * ops.stretch_T(p, y))) < 1e-12
    x = rng.standard_normal((p.ns, 3))
    y = rng.standard_normal((p.nt, 3))
    assert abs(np.sum(ops.unstretch(p, x) * y) - np.sum(x * ops.unstretch_T(p, y))) < 1e-12


# -------------------------------------------------------------- DFT (O1)
def test_rfft_bins_explicit_sum():
    p = tiny_plan()
    rng = np.random.default_rng(2)
    x = rng.standard_normal(p.ns)
    X = ops.rfft_bins(p, x[:, None])[:, 0]
    np.testing.assert_allclose(X, checks.explicit_dft(x, p.nfft, p.nbins),
                               rtol=0, atol=1e-11)


def test_band_limited_round_trip():
    """F1inv F x = x for a frame-length x without Nyquist content."""
    p = tiny_plan()
    pf = replace(p, ns=p.nfft)             # whole frame
    rng = np.random.default_rng(4)
    Y = rng.standard_normal((pf.nbins, 2)) + 1j * rng.standard_normal((pf.nbins, 2))
    x = ops.irfft_bins(pf, Y)
    Y[0] = Y[0].real
    np.testing.assert_allclose(ops.rfft_bins(pf, x), Y, atol=1e-12)
    np.testing.assert_allclose(ops.irfft_bins(pf, ops.rfft_bins(pf, x)), x, atol=1e-13)


def test_dft_transposes_explicit():
    p = tiny_plan()
    rng = np.random.default_rng(5)
    Y = rng.standard_normal(p.nbins) + 1j * rng.standard_normal(p.nbins)
    n = np.arange(p.ns)
    k = np.arange(1, p.nbins)
    want = Y[0].real + np.sum((Y[1:, None] * np.exp(2j * np.pi * np.outer(k, n) / p.nfft)).real, axis=0)
    np.testing.assert_allclose(ops.rfft_bins_T(p, Y[:, None])[:, 0], want, atol=1e-11)
    x = rng.standard_normal((p.ns, 2))
    Z = rng.standard_normal((p.nbins, 2)) + 1j * rng.standard_normal((p.nbins, 2))
    lhs = np.sum((ops.rfft_bins(p, x) * np.conj(Z)).real)
    assert abs(lhs - np.sum(x * ops.rfft_bins_T(p, Z))) < 1e-11
    lhs = np.sum(ops.irfft_bins(p, Z) * x)
    assert abs(lhs - np.sum((Z * np.conj(ops.irfft_bins_T(p, x))).real)) < 1e-12


# ------------------------------------------------- Fourier slice (O2, O3)
def test_slice_matches_time_domain_shift():
    """F1inv P F on one curvature/azimuth cell equals the band-limited
    time-domain delay by q r^2 / ds samples (shift theorem, eq. Inv_op)."""
    rng = np.random.default_rng(6)
    nq, nth = 5, 4
    q0, dq = syn.q_axis(nq)
    ang = 2 * np.pi / nth          # exactly on slice 2 -> weight 1
    hx = np.array([900.0 * np.cos(ang), 1400.0 * np.cos(ang)])
    hy = np.array([900.0 * np.sin(ang), 1400.0 * np.sin(ang)])
    p = oracle.make_plan(80, 0.008, 80, nq, q0, dq, nth, hx, hy)
    l = 3
    xs = np.zeros(p.ns)
    xs[5:60] = rng.standard_normal(55)
    X = np.zeros((p.nbins, nq, nth), complex)
    X[:, l, 2] = ops.rfft_bins(p, xs[:, None])[:, 0]
    dp = ops.irfft_bins(p, ops.slice_forward(p, X))
    for h in range(2):
        shift = p.q[l] * p.r2[h] / p.ds
        want = checks.time_domain_shift(xs, shift, p.nfft, p.kmax, p.ns)
        np.testing.assert_allclose(dp[:, h], want, atol=1e-12 * np.abs(want).max())


def test_integer_shift_is_exact_delay():
    """When q r^2 / ds is an integer s0 the slice is an exact circular delay
    by s0 samples of the Nyquist-free part of the stretched column; a positive
    curvature delays (t^2 = tau^2 + q r^2)."""
    rng = np.random.default_rng(7)
    nq, nth = 4, 2
    q0, dq = syn.q_axis(nq)
    base = oracle.make_plan(64, 0.008, 64, nq, q0, dq, nth,
                            np.array([1500.0]), np.array([0.0]))
    l, s0 = 2, 9
    r2 = s0 * base.ds / base.q[l]
    p = replace(base, hx=np.array([np.sqrt(r2)]), hy=np.array([0.0]),
                r2=np.array([r2]))
    xs = np.zeros(p.ns)
    xs[3:40] = rng.standard_normal(37)
    X = np.zeros((p.nbins, nq, nth), complex)
    X[:, l, 0] = ops.rfft_bins(p, xs[:, None])[:, 0]
    dp = ops.irfft_bins(p, ops.slice_forward(p, X))[:, 0]
    full = np.zeros(p.nfft)
    full[: p.ns] = xs
    alt = (-1.0) ** np.arange(p.nfft)
    proj = full - np.dot(full, alt) / p.nfft * alt          # remove Nyquist
    want = np.roll(proj, s0)[: p.ns]
    np.testing.assert_allclose(dp, want, atol=1e-13)


def test_slice_c_matches_numpy_sum():
    p = tiny_plan(ntr=9, nq=5, ntheta=3)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((p.nbins, p.nq, p.ntheta)) + 1j * rng.standard_normal((p.nbins, p.nq, p.ntheta))
    Y = rng.standard_normal((p.nbins, p.ntr)) + 1j * rng.standard_normal((p.nbins, p.ntr))
    np.testing.assert_allclose(ops.slice_forward(p, X), ops.slice_forward(p, X, "numpy"), atol=1e-11)
    np.testing.assert_allclose(ops.slice_adjoint(p, Y), ops.slice_adjoint(p, Y, "numpy"), atol=1e-11)


def test_slice_single_term_explicit():
    """One nonzero X entry and one trace: Y_k = w * X * exp(-i 2 pi f_k q r^2)."""
    p = tiny_plan(ntr=3, nq=4, ntheta=4)
    X = np.zeros((p.nbins, p.nq, p.ntheta), complex)
    l, j = 2, int(p.j1[1])
    X[:, l, j] = 1.0 + 0.5j
    Y = ops.slice_forward(p, X)[:, 1]
    w = (p.w1[1] if p.j1[1] == j else 0.0) + (p.w0[1] if p.j0[1] == j else 0.0)
    want = w * (1.0 + 0.5j) * np.exp(-2j * np.pi * p.freqs * (p.q0 + l * p.dq) * p.r2[1])
    np.testing.assert_allclose(Y, want, atol=1e-13)


# ------------------------------------------------ physical domain (O4, O7)
def test_riemann_sum_brute_force():
    """L m against eq. Inverse evaluated directly along the hyperbolae for
    Ricker events on single cells, traces on azimuth slices (weight 1);
    the gap is the interpolation error of S and U (bounded, reported)."""
    nt, dt, nq, nth = 500, 0.004, 16, 4
    q0, dq = syn.q_axis(nq)
    r = np.linspace(100.0, 1600.0, 8)
    hx = np.concatenate([r * np.cos(j * np.pi / nth) for j in range(nth)])
    hy = np.concatenate([r * np.sin(j * np.pi / nth) for j in range(nth)])
    p = oracle.make_plan(nt, dt, nt, nq, q0, dq, nth, hx, hy)
    events = [(1.0, 0.8, 15.0, 3, 0), (-0.7, 1.2, 12.0, 11, 1),
              (0.5, 1.5, 18.0, 7, 2), (0.9, 1.0, 14.0, 14, 3)]
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
    err = np.linalg.norm(d - want) / np.linalg.norm(want)
    assert err < 2e-2, err
    # the event sits at t = sqrt(tau^2 + q r^2): check the peak of one trace
    h = 7
    t_peak = np.argmax(d[:, h]) * dt
    assert abs(t_peak - np.sqrt(0.8 ** 2 + p.q[3] * p.r2[h])) <= 1.5 * dt


def test_zero_curvature_and_single_slice():
    """q = 0 removes all moveout, and a trace on slice j reads slice j only."""
    nt, dt, nth = 120, 0.008, 4
    hx = np.array([800.0, 0.0])
    hy = np.array([0.0, 800.0])           # slices 0 and 2
    p = oracle.make_plan(nt, dt, nt, 2, 0.0, 1e-7, nth, hx, hy)
    rng = np.random.default_rng(9)
    m = rng.standard_normal((nt, 2, nth))
    m[:, 1, :] = 0.0                      # only the q = 0 plane
    d = ops.forward(p, m)
    # no moveout: every trace sees U F1inv F S of its own slice's column
    for h, j in ((0, 0), (1, 2)):
        solo = np.zeros_like(m)
        solo[:, 0, j] = m[:, 0, j]
        d_solo = ops.forward(p, solo)
        np.testing.assert_allclose(d[:, h], d_solo[:, h], atol=1e-12)
        d_other = ops.forward(p, m - solo)
        assert np.abs(d_other[:, h]).max() < 1e-12
    # and that column is the band-limited stretch round trip of the model
    full = np.zeros(p.nfft)
    full[: p.ns] = ops.stretch(p, m[:, 0, 0][:, None])[:, 0]
    alt = (-1.0) ** np.arange(p.nfft)
    proj = (full - np.dot(full, alt) / p.nfft * alt)[: p.ns]
    np.testing.assert_allclose(d[:, 0], ops.unstretch(p, proj[:, None])[:, 0], atol=1e-12)


# ------------------------------------------------------------ adjoint (O5)
def test_dot_product_fp64_small_cube():
    g = syn.small_cube()
    p = oracle.make_plan(**g.geom_kwargs())
    m, d = syn.random_pair(11, g)
    lhs = np.sum(ops.forward(p, m) * d)
    rhs = np.sum(m * ops.adjoint(p, d))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("interp", ["keys", "linear"])
def test_dot_product_fp64_tiny(interp):
    p = tiny_plan(interp=interp, ntheta=5, nq=7)
    rng = np.random.default_rng(12)
    m = rng.standard_normal((p.ntau, p.nq, p.ntheta))
    d = rng.standard_normal((p.nt, p.ntr))
    lhs = np.sum(ops.forward(p, m) * d)
    assert abs(lhs - np.sum(m * ops.adjoint(p, d))) <= 1e-12 * abs(lhs)


def test_sampled_outputs_match_full():
    p = tiny_plan(ntr=15, ntheta=4)
    rng = np.random.default_rng(13)
    m = rng.standard_normal((p.ntau, p.nq, p.ntheta))
    d = rng.standard_normal((p.nt, p.ntr))
    full = ops.forward(p, m)
    np.testing.assert_allclose(ops.forward_traces(p, m, [2, 7]), full[:, [2, 7]], atol=1e-12)
    g = ops.adjoint(p, d)
    np.testing.assert_allclose(ops.adjoint_slices(p, d, [1, 3]), g[:, :, [1, 3]], atol=1e-12)


# -------------------------------------------------------------- FISTA (O6)
def test_soft_threshold_piecewise():
    x = np.linspace(-3, 3, 1201)
    for t in (0.0, 0.37, 1.0, 2.5):
        np.testing.assert_allclose(fista.soft(x, t), checks.soft_piecewise(x, t), atol=1e-15)


class _Diag:
    """A diagonal operator on a 1 x 1 x n model, recording the points the
    solver evaluates L at (the extrapolated iterates z^k)."""

    def __init__(self, a):
        self.a = np.asarray(a, np.float64)
        self.ntau, self.nq, self.ntheta = 1, 1, len(a)
        self.seen = []

    def fwd(self, m):
        self.seen.append(np.array(m, np.float64).ravel())
        return self.a * m.ravel()

    def adj(self, r):
        return (self.a * r).reshape(1, 1, -1)


def _golden_fista():
    rows = []
    with open(os.path.join(GOLDEN, "fista_diagonal.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v = [float(x) for x in line.split()]
                rows.append((int(v[0]), v[1], np.array(v[2:6]), np.array(v[6:10])))
    return rows


def test_fista_iterates_hand_worked():
    """The first four FISTA iterates m^k and extrapolated points z^k of a
    decoupled problem, worked by hand from Beck and Teboulle's recursion
    (tests/golden/fista_diagonal.txt): pins the weight (t_k - 1)/t_{k+1}, the
    index of t, the extrapolation from m^k, the step and the threshold."""
    rows = _golden_fista()
    d = np.array([3.0, 4.0, -4.8, -0.4])
    for k, _, m_want, _ in rows:
        op = _Diag([2.0, 1.0, 1.0, 1.0])
        m = fista.solve(op, d, 2.0, k, 0.25, op=(op.fwd, op.adj))
        np.testing.assert_allclose(m.ravel(), m_want, rtol=0, atol=1e-14)
    # the solver evaluates the gradient at z^0 .. z^3
    op = _Diag([2.0, 1.0, 1.0, 1.0])
    fista.solve(op, d, 2.0, 4, 0.25, op=(op.fwd, op.adj))
    np.testing.assert_allclose(op.seen[0], 0.0, atol=0)
    for (k, _, _, z_want), z_got in zip(rows[:3], op.seen[1:]):
        np.testing.assert_allclose(z_got, z_want, rtol=0, atol=1e-14)
    # ISTA on the same problem: z^k = m^k, so m^{k+1} = 3 m^k / 4 + 1/2 in
    # coordinate 1 (1/2, 7/8, 37/32, ...)
    op = _Diag([2.0, 1.0, 1.0, 1.0])
    m = fista.solve(op, d, 2.0, 3, 0.25, momentum=False, op=(op.fwd, op.adj))
    np.testing.assert_allclose(m.ravel(), [1.0, 37 / 32, -1.4 * 37 / 32, 0.0], atol=1e-15)


def test_momentum_schedule_quadratic_identity():
    """t_{k+1} is the positive root of t^2 - t - t_k^2 = 0 and t_0 = 1, so
    beta_0 = 0, t_1 is the golden ratio and, recovering t_{k+1} = (t_k - 1) /
    beta_k, every later pair satisfies t_{k+1}^2 - t_{k+1} = t_k^2; Beck and
    Teboulle's bound t_k >= (k + 2)/2 holds (their Lemma 4.3)."""
    b = fista.momentum_schedule(40)
    assert b[0] == 0.0
    t = [1.0, (1.0 + np.sqrt(5.0)) / 2.0]
    for k in range(1, 40):
        t.append((t[k] - 1.0) / b[k])
    t = np.array(t)
    np.testing.assert_allclose(t[1:] ** 2 - t[1:], t[:-1] ** 2, rtol=1e-12)
    assert np.all(t >= (np.arange(len(t)) + 2) / 2.0 - 1e-12)
    rows = _golden_fista()
    np.testing.assert_allclose(t[1:5], [r[1] for r in rows], rtol=1e-15)


def test_fista_rate_bound():
    """Beck and Teboulle's Theorem 4.4 on a small AAHRT problem: with a step
    gamma <= 1/||L||^2, F(m^k) - F* <= 2 ||m^0 - m*||^2 / (gamma (k + 1)^2)
    for every k, F of eq. cost1.  F* and m* come from a long run (F* from a
    run is an upper bound of the minimum, so the check is, if anything,
    looser than the theorem)."""
    p = tiny_plan(ntr=10, nt=64, nq=5, ntheta=3, seed=5)
    rng = np.random.default_rng(21)
    d = rng.standard_normal((p.nt, p.ntr))
    sig2 = fista.power_sigma2(p, d, iters=200)
    gamma = 0.9 / sig2
    lam = 0.1 * np.abs(ops.adjoint(p, d)).max()
    m_star, hist_long = fista.solve(p, d, lam, 1500, gamma, history=True)
    f_star = min(hist_long)
    _, hist = fista.solve(p, d, lam, 60, gamma, history=True)
    k = np.arange(1, 61)
    bound = 2.0 * float(np.sum(m_star ** 2)) / (gamma * (k + 1) ** 2)
    gap = np.array(hist) - f_star
    assert np.all(gap <= bound * 1.001 + 1e-12 * abs(f_star))
    # and the momentum is doing something: FISTA is ahead of ISTA at k = 60
    _, hist_ista = fista.solve(p, d, lam, 60, gamma, momentum=False, history=True)
    assert hist[-1] - f_star < hist_ista[-1] - f_star


def _sparse_case(seed=14):
    """Isolated single-cell spikes seen by a small regular offset grid."""
    nt, dt, nq, nth = 96, 0.008, 10, 4
    q0, dq = syn.q_axis(nq)
    hx, hy = syn.grid_offsets(8, 1500.0)
    p = oracle.make_plan(nt, dt, nt, nq, q0, dq, nth, hx, hy)
    m = np.zeros((nt, nq, nth))
    cells = [(30, 2, 0), (55, 7, 1), (70, 4, 2), (45, 8, 3)]
    for i, l, j in cells:
        m[i, l, j] = 1.0
    return p, m, cells


def test_ista_monotone_and_kkt():
    p, m_true, _ = _sparse_case()
    d = ops.forward(p, m_true)
    sig2 = fista.power_sigma2(p, d, iters=60)
    gamma = 0.95 / sig2
    lam = 0.05 * np.abs(ops.adjoint(p, d)).max()
    m, hist = fista.solve(p, d, lam, 40, gamma, momentum=False, history=True)
    assert np.all(np.diff(hist) <= 1e-9 * abs(hist[0]))
    m = fista.solve(p, d, lam, 800, gamma, momentum=True, m0=m)
    g = ops.adjoint(p, d - ops.forward(p, m))
    on = np.abs(m) > 1e-8
    assert np.abs(g[~on]).max() <= lam * 1.02
    np.testing.assert_allclose(g[on], lam * np.sign(m[on]), atol=0.05 * lam)


def test_spike_recovery_at_prescribed_moveout():
    p, m_true, cells = _sparse_case()
    d = ops.forward(p, m_true)
    gamma = 0.95 / fista.power_sigma2(p, d, iters=60)
    lam = 0.02 * np.abs(ops.adjoint(p, d)).max()
    m = fista.solve(p, d, lam, 300, gamma, momentum=True)
    for (i, l, j) in cells:
        win = np.abs(m[i - 3:i + 4, :, j])
        di, dl = np.unravel_index(np.argmax(win), win.shape)
        assert abs(di - 3) <= 1 and abs(dl - l) <= 1
    r = np.linalg.norm(d - ops.forward(p, m)) / np.linalg.norm(d)
    assert r < 0.1
