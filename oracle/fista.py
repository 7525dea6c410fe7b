"""Sparse AAHRT solve of the oracle (Sec. 4, eqs. cost1, ISTA and soft).

    minimise  1/2 ||d - L m||_2^2 + lambda ||m||_1                 (eq. cost1)

by forward-backward splitting (eq. ISTA)

    m^{k+1} = soft(m^k + gamma L^T (d - L m^k), gamma*lambda)

with the soft shrinkage of eq. soft, soft(x, t) = x * max(1 - t/|x|, 0).
With momentum on, the gradient step is taken at the extrapolated point z^k
of Beck and Teboulle's FISTA:

    m^{k+1} = soft(z^k + gamma L^T (d - L z^k), gamma*lambda)
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
    z^{k+1} = m^{k+1} + ((t_k - 1)/t_{k+1}) (m^{k+1} - m^k)

starting from m^0 = z^0 = 0 (or a given m^0 = z^0) and t_0 = 1.  The paper
does not give gamma; gamma = 0.95 / sigma^2 with sigma^2 estimated by power
iteration on L^T L started from L^T d.
"""
from __future__ import annotations

import numpy as np

from . import ops


def soft(x, t):
    """Soft shrinkage of eq. soft: x * max(1 - t/|x|, 0) (0 at x = 0)."""
    ax = np.abs(x)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(ax > 0.0, np.maximum(1.0 - t / ax, 0.0), 0.0)
    return x * scale


def momentum_schedule(iters: int):
    """FISTA extrapolation weights beta_k = (t_k - 1)/t_{k+1}, k < iters."""
    t = 1.0
    out = []
    for _ in range(iters):
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        out.append((t - 1.0) / tn)
        t = tn
    return np.array(out)


def _pair(plan, impl, op):
    """(forward, adjoint) callables: L and L^T, or the given pair."""
    if op is not None:
        return op
    return (lambda m: ops.forward(plan, m, impl)), (lambda d: ops.adjoint(plan, d, impl))


def power_sigma2(plan, d, iters: int = 30, impl: str = "c", op=None) -> float:
    """Estimate of the largest eigenvalue of L^T L by power iteration from
    L^T d / ||L^T d|| (Rayleigh quotient of the last iterate).  `op` may give
    another (forward, adjoint) pair, e.g. the deconvolutive operator."""
    fwd, adj = _pair(plan, impl, op)
    v = adj(d)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = adj(fwd(v))
        lam = float(np.vdot(v, w).real)
        v = w / np.linalg.norm(w)
    return lam


def objective(plan, d, m, lam, impl: str = "c", op=None) -> float:
    fwd, _ = _pair(plan, impl, op)
    r = d - fwd(m)
    return 0.5 * float(np.sum(r * r)) + lam * float(np.sum(np.abs(m)))


def solve(plan, d, lam, iters, gamma, momentum: bool = True, m0=None,
          impl: str = "c", history: bool = False, op=None):
    """Run `iters` iterations of ISTA (momentum off) or FISTA (on); `op`
    replaces (L, L^T) by another pair (the deconvolutive W L, L^T W^T)."""
    fwd, adj = _pair(plan, impl, op)
    d = np.asarray(d, np.float64)
    shape = (plan.ntau, plan.nq, plan.ntheta)
    m = np.zeros(shape) if m0 is None else np.array(m0, np.float64)
    z = m.copy()
    t = 1.0
    hist = []
    for _ in range(iters):
        g = adj(d - fwd(z))
        m_new = soft(z + gamma * g, gamma * lam)
        if momentum:
            tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            z = m_new + ((t - 1.0) / tn) * (m_new - m)
            t = tn
        else:
            z = m_new
        m = m_new
        if history:
            hist.append(objective(plan, d, m, lam, impl, op))
    return (m, hist) if history else m


def unrolled_states(plan, d, lam, gamma, iters, momentum: bool = True, impl: str = "c"):
    """The iterations of `solve` from m^0 = z^0 = 0 with every intermediate
    kept: lists z[k] (k <= iters), m[k] (k <= iters) and the pre-shrinkage
    points u[k] = z^k + gamma L^T (d - L z^k) (k < iters), and the
    extrapolation weights beta_k (zeros for ISTA)."""
    d = np.asarray(d, np.float64)
    shape = (plan.ntau, plan.nq, plan.ntheta)
    betas = momentum_schedule(iters) if momentum else np.zeros(iters)
    m = [np.zeros(shape)]
    z = [np.zeros(shape)]
    u = []
    for k in range(iters):
        g = ops.adjoint(plan, d - ops.forward(plan, z[k], impl), impl)
        u.append(z[k] + gamma * g)
        m.append(soft(u[k], gamma * lam))
        z.append(m[k + 1] + betas[k] * (m[k + 1] - m[k]))
    return z, m, u, betas


def unrolled_vjp(plan, d, m_bar, lam, gamma, iters, momentum: bool = True,
                 impl: str = "c"):
    """Reverse-mode derivative of the unrolled solve d -> m^iters (fixed
    gamma and lambda, start 0): returns (m^iters, d_bar) with
    d_bar = (d m^iters / d d)^T m_bar.

    Each iteration is u = z + gamma L^T (d - L z), m+ = soft(u, t),
    z+ = (1 + beta) m+ - beta m, with t = gamma*lambda.  Going backwards with
    the cotangents a_m of m+ and a_z of z+:
        total cotangent of m+     c = a_m + (1 + beta) a_z
        through the shrinkage     u_bar = c * [|u| > t]
        data                      d_bar += gamma L u_bar
        the iterate z             z_bar = u_bar - gamma L^T L u_bar
        the previous m            m_bar_prev = -beta a_z
    The shrinkage has slope 1 where |u| > t and 0 where |u| < t; at |u| = t
    it has no derivative and the slope 0 is taken."""
    z, m, u, betas = unrolled_states(plan, d, lam, gamma, iters, momentum, impl)
    t = gamma * lam
    a_m = np.array(m_bar, np.float64).reshape(m[0].shape)
    a_z = np.zeros_like(a_m)
    d_bar = np.zeros((plan.nt, plan.ntr))
    for k in range(iters - 1, -1, -1):
        c = a_m + (1.0 + betas[k]) * a_z
        u_bar = np.where(np.abs(u[k]) > t, c, 0.0)
        s = ops.forward(plan, u_bar, impl)
        d_bar += gamma * s
        a_z_new = u_bar - gamma * ops.adjoint(plan, s, impl)
        a_m = -betas[k] * a_z
        a_z = a_z_new
    return m[iters], d_bar
