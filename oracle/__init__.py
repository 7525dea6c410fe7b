"""FP64 CPU oracle of the fast azimuthally anisotropic hyperbolic Radon
transform (AAHRT), its exact adjoint and the forward-backward splitting solve.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import, call, link or run anything in this
package.  The CUDA library never uses it and shares no code with it.

What it computes (paper sections and equations):

* ``plan``      sampling of the stretched time axis (Sec. 3.4 step 1, Sec. 3.5 eq. q3)
                and the azimuth binning of every trace (eq. thli, theta part).
* ``ops``       the discrete operator R^{-1} = S^{-1} F1^{-1} P F2 S of
                eq. axb2 (Algorithm 1) and its exact transpose (the adjoint of
                Sec. 3.2 / Algorithm 2, built as a true transpose).
                The q-part of F2 followed by the k-interpolation of P
                (eq. Inv_op, inv_GFST) is evaluated exactly as the
                non-uniform DFT along q at k_q = f' r^2, which is what the
                paper's linear interpolation in k approximates.
* ``nudft.c``   the direct sum of that slice step (FP64, OpenMP over bins).
* ``fista``     soft shrinkage (eq. soft), ISTA (eq. ISTA) and its FISTA
                momentum variant, power iteration for the step length.
* ``decon``     the deconvolutive operator W L of eq. DecRT (time convolution
                with a wavelet) and its transpose.
* ``pick``      the q-moment velocity pick of eq. vel_est.
* ``lineark``   the paper-literal slice step: linear interpolation in k of
                the FFT'd q columns (A-coefficients of eq. thli).
* ``bpull``     the paper's velocity scan (Algorithm 2): data on a regular
                offset grid pulled at the rings k = f' r^2 (B-coefficients).
* ``pnmo``      the curvature range of Sec. 3.5: the sample count of eq. q3,
                the uniform-slowness (non-uniform q) axis, and the partial
                NMO of the data with its transpose.
* ``checks``    independent evaluations used only to pin the oracle: the
                physical-domain Riemann sum along the azimuth-dependent
                hyperbolae (eq. Inverse, Sec. 5.1) and the time-domain
                band-limited shift that the Fourier slice step must equal
                (the shift theorem behind eq. Inv_op).

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``): the DFT against an
explicit sum, the Fourier slice against the time-domain shift, integer
shifts, the physical-domain brute force, the dot-product adjoint test, the
Keys kernel's reproduction of quadratics, the azimuth weights' invariants,
the soft threshold's piecewise form, ISTA monotonicity, KKT optimality and
spike recovery.  Every function in this package is covered by at least one.
"""
from .plan import OraclePlan, make_plan            # noqa: F401
from . import ops, fista, checks, decon, pick, lineark, bpull, pnmo   # noqa: F401
