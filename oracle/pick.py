"""Automatic anisotropic velocity picking of the oracle (Sec. 3.3, eq.
vel_est): the squared slowness at each (tau, theta) is the first moment of
the Radon cube along q,

    v^{-2}(tau, theta) = sum_l q_l |M(tau, l, theta)| / sum_l |M(tau, l, theta)|.

Reading: the weights are |M| (the paper writes M; a sparse cube's band-
limited events carry negative side lobes, which would pull the signed ratio
outside the q axis).  Where the weight is zero the pick is 0.

TEST INFRASTRUCTURE (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def pick(plan, m):
    """(q_hat[tau][theta], weight[tau][theta]) of m[tau][q][theta]."""
    a = np.abs(np.asarray(m, np.float64))
    wsum = a.sum(axis=1)
    num = np.einsum("l,ilj->ij", plan.q, a)
    with np.errstate(divide="ignore", invalid="ignore"):
        q_hat = np.where(wsum > 0.0, num / wsum, 0.0)
    return q_hat, wsum
