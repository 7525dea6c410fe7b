"""Helpers of the GPU parity tests (test infrastructure)."""
import numpy as np
import torch

import oracle
from oracle import ops


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32).ravel()).cuda()


def host(t, shape=None):
    a = t.detach().cpu().numpy().astype(np.float64 if t.dtype == torch.float32 else np.complex128)
    return a.reshape(shape) if shape is not None else a


def oracle_plan(g, **kw):
    return oracle.make_plan(**g.geom_kwargs(), **kw)


def gpu_plan(g, **kw):
    from paper_2505_00387_gb300.plan import AahrtPlan
    return AahrtPlan(**g.geom_kwargs(), **kw)


def oracle_H(p, X):
    """H(X) = Re X_0 + 2 Re sum_k X_k e^{+...} written through the oracle's F^T."""
    Xd = X.copy()
    Xd[1:] *= 2.0
    return ops.rfft_bins_T(p, Xd)


def dot_rel_conditioned(gp, oracle_fwd, seed):
    """FP32 dot test of the GPU pair on a well-conditioned pair of vectors:
    m random and d = L m (by the oracle, `oracle_fwd` maps the flat model to
    the flat data) plus as much independent noise, so <L m, d> is about
    |L m|^2.  For two independent random vectors <L m, d> is itself a random
    projection, often near zero, and the relative error of the test would
    measure that cancellation rather than the adjointness."""
    rng = np.random.default_rng(seed)
    m = rng.standard_normal(gp.model_len).astype(np.float32).astype(np.float64)
    lm = np.asarray(oracle_fwd(m), np.float64).ravel()
    d = lm + np.sqrt(np.mean(lm * lm)) * rng.standard_normal(lm.shape)
    d = d.astype(np.float32).astype(np.float64)
    lhs = float(np.dot(host(gp.forward(dev(m))), d))
    rhs = float(np.dot(host(gp.adjoint(dev(d))), m))
    return abs(lhs - rhs) / abs(lhs)
