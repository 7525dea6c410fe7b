"""Seeded synthetic CMP inputs shaped like the paper's numerical tests.

This module holds input generation only: offsets, a Ricker wavelet, hyperbolic
events with elliptical azimuthal anisotropy (the model of Sec. 2.1, eq. ellip1)
and Gaussian noise.  It contains none of the fast transform's arithmetic (no
time stretch, no Fourier slice, no azimuth binning); both the CUDA path and the
CPU checker consume the arrays it returns, so either side can be fed the same
seeded input.

The paper's own synthetic CMP (Sec. 5.1: dt = 4 ms, hyperbolic events with
anisotropic velocities) exists only as a figure, so these generators stand in
for it with the same sampling and event structure.

Axes:
  model m[tau][q][theta]    float, theta fastest, q_l = q0 + l*dq (squared slowness)
  data  d[t][trace]         float, trace fastest, trace h at offset (hx[h], hy[h])
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Slowness range of the configurations: 1/3500 .. 1/1500 s/m.  The model axis
# is the curvature q = p^2 (Sec. 2, eq. RT_basis), sampled uniformly in q.
P_MIN = 1.0 / 3500.0
P_MAX = 1.0 / 1500.0


def q_axis(nq: int, pmin: float = P_MIN, pmax: float = P_MAX):
    """Uniform curvature axis spanning [pmin^2, pmax^2]; returns (q0, dq)."""
    q0 = pmin * pmin
    q1 = pmax * pmax
    dq = (q1 - q0) / (nq - 1) if nq > 1 else 0.0
    return q0, dq


def ricker(t, f):
    """Ricker wavelet of peak frequency f (Hz) at times t (s)."""
    a = (np.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ellipse_q(theta, v_a, v_b, axis):
    """Elliptical azimuthal curvature (eq. ellip1) rotated by `axis`:
    q(theta) = cos^2(theta-axis)/v_a^2 + sin^2(theta-axis)/v_b^2."""
    c = np.cos(theta - axis)
    s = np.sin(theta - axis)
    return c * c / (v_a * v_a) + s * s / (v_b * v_b)


@dataclass
class Gather:
    """One CMP cube: axes, offsets and (optionally) data and/or model."""
    nt: int
    dt: float
    ntau: int
    nq: int
    q0: float
    dq: float
    ntheta: int
    hx: np.ndarray
    hy: np.ndarray
    d: Optional[np.ndarray] = None      # [nt][ntr] float64
    m: Optional[np.ndarray] = None      # [ntau][nq][ntheta] float64
    info: dict = field(default_factory=dict)

    @property
    def ntr(self) -> int:
        return int(self.hx.shape[0])

    def geom_kwargs(self) -> dict:
        return dict(nt=self.nt, dt=self.dt, ntau=self.ntau, nq=self.nq,
                    q0=self.q0, dq=self.dq, ntheta=self.ntheta,
                    hx=self.hx, hy=self.hy)


# ----------------------------------------------------------------- offsets
def grid_offsets(n: int = 16, half: float = 1000.0):
    """Regular n x n offset grid on [-half, half]^2; trace index = ix*n + iy."""
    x = np.linspace(-half, half, n)
    hx, hy = np.meshgrid(x, x, indexing="ij")
    return hx.ravel().copy(), hy.ravel().copy()


def disc_offsets(rng, ntr: int, radius: float, az_start: float = 0.0,
                 az_width: float = 2.0 * np.pi):
    """ntr offsets uniform in a disc (or a sector of it) of the given radius."""
    r = radius * np.sqrt(rng.random(ntr))
    az = az_start + az_width * rng.random(ntr)
    return r * np.cos(az), r * np.sin(az)


# ------------------------------------------------------------- data domain
def hyperbolic_events(rng, nt, dt, hx, hy, nev, tau_rng, v_rng, aniso_rng,
                      f_rng, window=1.6):
    """Data-domain CMP: nev Ricker events on azimuth-dependent hyperbolae
    t = sqrt(tau^2 + q_e(theta_h) r^2) with q_e an elliptical curvature
    (eq. ellip1) of random strength and axis.  Each wavelet is evaluated on
    the samples within window/f of its centre (the rest is below 1e-10)."""
    ntr = hx.shape[0]
    d = np.zeros(nt * ntr)
    r2 = hx * hx + hy * hy
    az = np.arctan2(hy, hx)
    events = []
    cols = np.arange(ntr)
    for _ in range(nev):
        tau = rng.uniform(*tau_rng)
        v = rng.uniform(*v_rng)
        an = rng.uniform(*aniso_rng)
        axis = rng.uniform(0.0, np.pi)
        f = rng.uniform(*f_rng)
        amp = rng.uniform(0.5, 1.0) * (1.0 if rng.random() < 0.8 else -1.0)
        events.append(dict(tau=tau, v=v, aniso=an, axis=axis, f=f, amp=amp))
        q = ellipse_q(az, v, v * (1.0 + an), axis)
        te = np.sqrt(tau * tau + q * r2)
        half = int(np.ceil(window / f / dt)) + 1
        off = np.arange(-half, half + 1)
        i = np.rint(te / dt).astype(np.int64)[:, None] + off[None, :]
        ok = (i >= 0) & (i < nt)
        vals = amp * ricker(i * dt - te[:, None], f)
        flat = (i * ntr + cols[:, None])[ok]
        d += np.bincount(flat, weights=vals[ok], minlength=nt * ntr)
    return d.reshape(nt, ntr), events


def add_noise(rng, d, level):
    """Gaussian noise with standard deviation level * rms(d)."""
    rms = float(np.sqrt(np.mean(d * d)))
    return d + level * rms * rng.standard_normal(d.shape)


# ------------------------------------------------------------ model domain
def spike_model(rng, ntau, dt, nq, q0, dq, ntheta, nspike=5, f=25.0,
                tau_rng=(0.15, 0.9), v_rng=(1650.0, 3300.0), aniso=0.10):
    """Radon-domain model of isolated events: each spike follows an
    elliptical q(theta) (eq. ellip1) with fast velocity v and slow velocity
    v/(1+aniso) about a random axis; at each azimuth theta_j = j*pi/ntheta it
    is split linearly between the two neighbouring q cells, then convolved
    along tau with a Ricker wavelet of peak frequency f."""
    m = np.zeros((ntau, nq, ntheta))
    tau_ax = np.arange(ntau) * dt
    th = np.arange(ntheta) * np.pi / ntheta
    spikes = []
    for _ in range(nspike):
        tau = rng.uniform(*tau_rng)
        v = rng.uniform(*v_rng)
        axis = rng.uniform(0.0, np.pi)
        amp = rng.uniform(0.6, 1.0)
        spikes.append(dict(tau=tau, v=v, axis=axis, amp=amp))
        w = amp * ricker(tau_ax - tau, f)
        qj = ellipse_q(th, v, v / (1.0 + aniso), axis)
        pos = np.clip((qj - q0) / dq, 0.0, nq - 1.0)
        for j in range(ntheta):
            l = min(int(np.floor(pos[j])), nq - 2)
            fr = pos[j] - l
            m[:, l, j] += (1.0 - fr) * w
            m[:, l + 1, j] += fr * w
    return m, spikes


# ----------------------------------------------------------- configurations
def small_cube(seed: int = 0) -> Gather:
    """Single CMP cube: nt=256 at 4 ms, 16x16 offset grid on [-1000,1000]^2 m,
    model 256 x 32 q x 8 azimuths holding 5 Ricker (25 Hz) spikes with 10%
    elliptical anisotropy.  The data of this case are the forward transform of
    the model, computed by the caller."""
    rng = np.random.default_rng(seed)
    nt, dt, nq, nth = 256, 0.004, 32, 8
    q0, dq = q_axis(nq)
    hx, hy = grid_offsets(16, 1000.0)
    m, spikes = spike_model(rng, nt, dt, nq, q0, dq, nth)
    return Gather(nt, dt, nt, nq, q0, dq, nth, hx, hy, m=m,
                  info=dict(name="cmp-256t-16x16-32q-8az", spikes=spikes))


def paper_gather(seed: int = 1, ntr: int = 2000) -> Gather:
    """Paper-scale gather: nt=1001 at 4 ms, 2000 traces uniform in a 3 km
    disc, model 100 q x 36 azimuths, data = 30 Ricker events (15-40 Hz) with
    0-20% elliptical anisotropy plus 10% Gaussian noise."""
    rng = np.random.default_rng(seed)
    nt, dt, nq, nth = 1001, 0.004, 100, 36
    q0, dq = q_axis(nq)
    hx, hy = disc_offsets(rng, ntr, 3000.0)
    d, ev = hyperbolic_events(rng, nt, dt, hx, hy, 30, (0.2, 3.8),
                              (1600.0, 3300.0), (0.0, 0.2), (15.0, 40.0))
    d = add_noise(rng, d, 0.10)
    return Gather(nt, dt, nt, nq, q0, dq, nth, hx, hy, d=d,
                  info=dict(name="cmp-1001t-2000tr-100q-36az", events=ev))


def cube_batch(seed: int = 3, ncube: int = 512, cubes: Optional[List[int]] = None,
               with_data: bool = True):
    """Batch of CMP cubes: nt=1001 at 4 ms, fold uniform in [200, 3000],
    offsets in a 3 km disc restricted to a random azimuth sector 90-360
    degrees wide, model 64 q x 24 azimuths, events as in paper_gather.  Each cube
    draws from its own seed so any subset can be regenerated alone; with
    with_data=False only the geometry is drawn (the same offsets, no data)."""
    out = []
    idx = range(ncube) if cubes is None else cubes
    nt, dt, nq, nth = 1001, 0.004, 64, 24
    q0, dq = q_axis(nq)
    for c in idx:
        rng = np.random.default_rng([seed, c])
        fold = int(rng.integers(200, 3001))
        width = np.deg2rad(rng.uniform(90.0, 360.0))
        start = rng.uniform(0.0, 2.0 * np.pi)
        hx, hy = disc_offsets(rng, fold, 3000.0, start, width)
        d = None
        if with_data:
            d, ev = hyperbolic_events(rng, nt, dt, hx, hy, 30, (0.2, 3.8),
                                      (1600.0, 3300.0), (0.0, 0.2), (15.0, 40.0))
            d = add_noise(rng, d, 0.10)
        out.append(Gather(nt, dt, nt, nq, q0, dq, nth, hx, hy, d=d,
                          info=dict(name=f"cube{c}", fold=fold)))
    return out


def shared_batch(seed: int = 4, ngather: int = 64, ntr: int = 8000,
            gathers: Optional[List[int]] = None):
    """Shared-geometry batch: ngather gathers on one geometry of 8000 traces
    in a 4 km disc, nt=2048 at 2 ms, model 200 q x 72 azimuths.  Returns
    (geometry Gather without data, list of data arrays)."""
    rng = np.random.default_rng([seed, 10**6])
    nt, dt, nq, nth = 2048, 0.002, 200, 72
    q0, dq = q_axis(nq)
    hx, hy = disc_offsets(rng, ntr, 4000.0)
    geo = Gather(nt, dt, nt, nq, q0, dq, nth, hx, hy,
                 info=dict(name="shared-8000tr-2048t-200q-72az"))
    ds = []
    for g in (range(ngather) if gathers is None else gathers):
        r = np.random.default_rng([seed, g])
        d, _ = hyperbolic_events(r, nt, dt, hx, hy, 30, (0.2, 3.8),
                                 (1600.0, 3300.0), (0.0, 0.2), (15.0, 40.0))
        ds.append(add_noise(r, d, 0.10))
    return geo, ds


def random_pair(seed: int, g: Gather):
    """Standard-normal model and data arrays of the gather's shapes."""
    rng = np.random.default_rng(seed)
    m = rng.standard_normal((g.ntau, g.nq, g.ntheta))
    d = rng.standard_normal((g.nt, g.ntr))
    return m, d
