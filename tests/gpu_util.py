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
