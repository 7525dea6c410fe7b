"""CPU tests of host-side logic: the shared-memory FFT groups and the
per-trace slice arithmetic compiled for the host from the same headers the
CUDA kernels use."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = "/usr/local/cuda/include"


def _compile(src, out):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or CUDA headers not available")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I" + CUDA_INC, src, "-o", out],
                   check=True, capture_output=True)


def test_fft_groups_match_dft(tmp_path):
    exe = str(tmp_path / "fft_harness")
    _compile(os.path.join(HERE, "host", "fft_harness.cpp"), exe)
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    worst = float(r.stdout.strip().splitlines()[-1].split()[-1])
    assert worst < 1e-6


def test_trace_taps_exact(tmp_path):
    """Phase and tap position from the 64-bit fixed-point products agree with
    exact integer arithmetic; the Horner weights agree with the kernel."""
    exe = str(tmp_path / "slice_harness")
    _compile(os.path.join(HERE, "host", "slice_math_harness.cpp"), exe)
    rng = np.random.default_rng(0)
    cases = []
    for _ in range(400):
        A = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        B = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        k = int(rng.integers(0, 8192))
        Lq = int(rng.integers(4, 10))
        W = int(rng.integers(4, 13))
        sig = 2.0 ** (Lq) / max(1, int(rng.integers(2 ** (Lq - 2), 2 ** (Lq - 1) + 1)))
        beta = 0.97 * np.pi * W * (1 - 1 / (2 * sig))
        cases.append((A, B, k, Lq, W, beta))
    inp = "\n".join("%d %d %d %d %d %.17g" % c for c in cases) + "\n"
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True)
    for (A, B, k, Lq, W, beta), line in zip(cases, r.stdout.strip().splitlines()):
        vals = line.split()
        u0, g, ph = int(vals[0]), float(vals[1]), float(vals[2])
        phi = np.array([float(v) for v in vals[3:]])
        pa = (k * A) % 2**64
        ph_exact = (pa >> 32) / 2**32
        if ph_exact >= 0.5:
            ph_exact -= 1.0
        assert abs(ph - ph_exact) < 2e-7
        y = ((k * B) % 2**64 >> 32) / 2**32 * 2**Lq
        assert -0.5 <= g < 0.5
        # tap i sits at distance z_i = g + (W-1)/2 - i = y - (u0 + i)
        assert abs((y - u0) - (g + (W - 1) / 2)) < 2e-6 * 2**Lq
        z = g + (W - 1) / 2 - np.arange(W)
        t = 2 * z / W
        want = np.exp(beta * (np.sqrt(np.clip(1 - t * t, 0, None)) - 1))
        # polynomial fit + float rounding; the edge discontinuity e^-beta bounds it
        np.testing.assert_allclose(phi, want, rtol=0, atol=2e-6 + 4 * np.exp(-beta))


def test_curvature_axis_helpers_match_oracle():
    """aahrt_q_axis_slowness and aahrt_nq_required (host functions of the
    library, no device work) against the oracle's uniform-slowness axis and
    eq. q3 count."""
    from oracle import pnmo
    from paper_2505_00387_gb300 import _lib as L
    for pmin, pmax, nq in ((1 / 3500.0, 1 / 1500.0, 100), (1 / 3000.0, 1 / 2000.0, 1),
                           (2e-4, 6e-4, 7)):
        q = np.array(L.aahrt_q_axis_slowness(pmin, pmax, nq))
        np.testing.assert_allclose(q, pnmo.q_axis_slowness(pmin, pmax, nq), rtol=1e-15)
    for span, fmax, r2max in ((6.2e-7, 60.0, 4.5e6), (0.0, 10.0, 1e6), (1.98e-7, 12.0, 3.9e6)):
        assert L.aahrt_nq_required(span, fmax, r2max) == pnmo.nq_required(span, fmax, r2max)
    with pytest.raises(L.AahrtError):
        L.aahrt_nq_required(-1.0, 1.0, 1.0)
    with pytest.raises(L.AahrtError):
        L.aahrt_q_axis_slowness(1e-4, float("nan"), 4)


def test_direct_sum_phase_top_word(tmp_path):
    """The direct sum's phase from 32-bit multiplies (offset curvature index,
    dropped low-word carry) equals the exact top word of k A + n k B
    (mod 2^64) or falls short of it by one unit (2^-32 cycle), for curvature
    indices up to the axis quantisation's 2^30."""
    exe = str(tmp_path / "phase32_harness")
    _compile(os.path.join(HERE, "host", "phase32_harness.cpp"), exe)
    rng = np.random.default_rng(5)
    cases = []
    for _ in range(2000):
        kA = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        kB = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        n = int(rng.integers(-2**30, 2**30 + 1))
        cases.append((kA, kB, n))
    cases += [(0, 0, 0), (2**64 - 1, 2**64 - 1, 2**30), (2**63, 1, -2**30), (12345, 2**32, -1)]
    inp = "\n".join("%d %d %d" % c for c in cases) + "\n"
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True)
    for (kA, kB, n), line in zip(cases, r.stdout.strip().splitlines()):
        top, exact = (int(v) for v in line.split())
        assert exact == ((kA + n * kB) % 2**64) >> 32
        assert (exact - top) % 2**32 in (0, 1)
