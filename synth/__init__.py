"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds none of the method's arithmetic: it only draws velocity
models, acquisition geometry, frequency lists, source wavelets and
band-limited noise traces from seeded PCG64 generators.  Both the FP64 CPU
oracle and the CUDA path consume what it returns, and neither imports the
other.

Workload shapes follow the paper's two benchmark classes (a layered and
faulted Marmousi-like model, a salt-body BP-like model) with surface
acquisition and receivers denser than sources (the paper's Marmousi II and
2004 BP sections); the models themselves are not available, so these seeded
stand-ins take their place.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Case",
    "ricker",
    "bandlimited_noise",
    "linear_gradient_model",
    "layered_faulted_model",
    "salt_model",
    "case_small",
    "case_layered",
    "case_salt_patches",
    "case_tiny",
    "slice_case",
]


class Case(dict):
    """A workload description: a plain dict with attribute access."""

    __getattr__ = dict.__getitem__


def ricker(nt: int, dt: float, f_peak: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet samples r(n dt), n = 0..nt-1, peak frequency f_peak, delay t0 (default 1/f_peak)."""
    if t0 is None:
        t0 = 1.0 / f_peak
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (np.pi * f_peak * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def bandlimited_noise(rng: np.random.Generator, shape, dt: float, fmin: float, fmax: float,
                      taper_hz: float = 0.5) -> np.ndarray:
    """Gaussian noise along the last axis, band-passed to [fmin, fmax] Hz with cosine tapers."""
    x = rng.standard_normal(shape)
    n = x.shape[-1]
    f = np.fft.rfftfreq(n, dt)
    w = np.zeros_like(f)
    inside = (f >= fmin) & (f <= fmax)
    w[inside] = 1.0
    lo = (f >= fmin - taper_hz) & (f < fmin)
    w[lo] = 0.5 - 0.5 * np.cos(np.pi * (f[lo] - (fmin - taper_hz)) / taper_hz)
    hi = (f > fmax) & (f <= fmax + taper_hz)
    w[hi] = 0.5 + 0.5 * np.cos(np.pi * (f[hi] - fmax) / taper_hz)
    y = np.fft.irfft(np.fft.rfft(x, axis=-1) * w, n=n, axis=-1)
    y /= max(np.sqrt(np.mean(y * y)), 1e-30)
    return y


def linear_gradient_model(nz: int, nx: int, v_top: float, v_bottom: float) -> np.ndarray:
    """Velocity increasing linearly with depth from v_top (row 0) to v_bottom (row nz-1)."""
    vz = v_top + (v_bottom - v_top) * np.arange(nz) / max(nz - 1, 1)
    return np.repeat(vz[:, None], nx, axis=1).astype(np.float64)


def _gaussian_anomaly(nz, nx, cz, cx, sigma, amp):
    z = np.arange(nz)[:, None]
    x = np.arange(nx)[None, :]
    return 1.0 + amp * np.exp(-((z - cz) ** 2 + (x - cx) ** 2) / (2.0 * sigma ** 2))


def layered_faulted_model(rng: np.random.Generator, nz: int, nx: int, nlayers: int = 30,
                          vmin: float = 1500.0, vmax: float = 4700.0, nfaults: int = 3) -> np.ndarray:
    """Layered model (monotone velocities vmin..vmax with jitter) cut by random normal faults."""
    min_t = 3.0
    thick = min_t + rng.dirichlet(np.full(nlayers, 4.0)) * (nz - min_t * nlayers)
    bounds = np.cumsum(thick)[:-1]
    base = np.linspace(vmin, vmax, nlayers)
    vel_l = np.sort(np.clip(base + rng.uniform(-60.0, 60.0, nlayers), vmin, vmax))
    vel_l[0], vel_l[-1] = vmin, vmax
    z = np.arange(nz, dtype=np.float64)[:, None] * np.ones((1, nx))
    x = np.ones((nz, 1)) * np.arange(nx, dtype=np.float64)[None, :]
    depth = z.copy()
    for _ in range(nfaults):
        x0 = rng.uniform(0.15, 0.85) * nx
        dip = np.deg2rad(rng.uniform(50.0, 70.0))
        side = rng.choice([-1.0, 1.0])
        throw = rng.uniform(5.0, 20.0)
        xf = x0 + side * z / np.tan(dip)
        hanging = (x - xf) * side > 0.0
        depth = depth - throw * hanging
    idx = np.searchsorted(bounds, np.maximum(depth, 0.0), side="right")
    return vel_l[np.clip(idx, 0, nlayers - 1)].astype(np.float64)


def salt_model(rng: np.random.Generator, nz: int, nx: int, vsed=(1500.0, 4000.0),
               vsalt: float = 4500.0) -> np.ndarray:
    """Sediments with a depth gradient plus a salt body whose boundary is a smooth random curve."""
    v = linear_gradient_model(nz, nx, vsed[0], vsed[1])
    cx = rng.uniform(0.35, 0.65) * nx
    half_w = rng.uniform(0.15, 0.25) * nx
    top0 = rng.uniform(0.25, 0.4) * nz
    bot0 = rng.uniform(0.6, 0.75) * nz
    xs = np.arange(nx)
    k = np.arange(1, 6)
    ph = rng.uniform(0, 2 * np.pi, (2, 5))
    am = rng.uniform(0.0, 0.04 * nz, (2, 5)) / k
    s = (xs[:, None] - cx) / half_w
    top = top0 + (am[0] * np.sin(np.pi * k * s + ph[0])).sum(1)
    bot = bot0 + (am[1] * np.sin(np.pi * k * s + ph[1])).sum(1)
    inside_x = np.abs(s[:, 0]) < 1.0
    shape = np.sqrt(np.clip(1.0 - s[:, 0] ** 2, 0.0, 1.0))
    top = top + (1.0 - shape) * (bot - top) * 0.5
    bot = bot - (1.0 - shape) * (bot - top) * 0.5
    z = np.arange(nz)[:, None]
    mask = inside_x[None, :] & (z >= top[None, :]) & (z <= bot[None, :])
    v[mask] = vsalt
    return v


def _smooth(v: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(v, sigma, mode="nearest")


def case_small(seed: int = 1) -> Case:
    """101x101 model, dx 10 m, 1500->2500 m/s gradient, +10 % Gaussian anomaly (sigma 8 pts)
    at a seeded centre in the middle third; 21 receivers and 11 Ricker 10 Hz sources on the
    surface row; dt 1 ms, 1000 steps, 20-point sponge, frequencies 3-7 Hz, mu = 1e-2 x mean diag."""
    rng = np.random.default_rng(seed)
    nz = nx = 101
    v_start = linear_gradient_model(nz, nx, 1500.0, 2500.0)
    cz, cx = rng.uniform(nz / 3, 2 * nz / 3, 2)
    v_true = v_start * _gaussian_anomaly(nz, nx, cz, cx, 8.0, 0.10)
    return Case(
        name="small-101x101-nr21-nf5-nt1000",
        nz=nz, nx=nx, dz=10.0, dx=10.0, dt=1e-3, nt=1000, nsponge=20, sponge_R=1e-3,
        vel_true=v_true, vel_start=v_start,
        rec_iz=np.zeros(21, np.int32), rec_ix=np.arange(0, 101, 5, dtype=np.int32),
        src_iz=np.zeros(11, np.int32), src_ix=np.arange(0, 101, 10, dtype=np.int32),
        freqs=np.array([3.0, 4.0, 5.0, 6.0, 7.0]), ricker_hz=10.0, mu_alpha=1e-2,
    )


def case_layered(seed: int = 2) -> Case:
    """921x301 layered-and-faulted model (30 layers, 1500-4700 m/s, 3 normal faults), dx 10 m;
    231 receivers (every 4th column) and 115 Ricker 8 Hz sources (every 8th column from 4) on the
    surface row; dt 1 ms, 4000 steps, 26 frequencies 3.0:0.2:8.0 Hz; the start model is the true
    model smoothed by a Gaussian of 30 points."""
    rng = np.random.default_rng(seed)
    nz, nx = 301, 921
    v_true = layered_faulted_model(rng, nz, nx)
    v_start = _smooth(v_true, 30.0)
    return Case(
        name="layered-921x301-nr231-nf26-nt4000-ns115",
        nz=nz, nx=nx, dz=10.0, dx=10.0, dt=1e-3, nt=4000, nsponge=20, sponge_R=1e-3,
        vel_true=v_true, vel_start=v_start,
        rec_iz=np.zeros(231, np.int32), rec_ix=(4 * np.arange(231)).astype(np.int32),
        src_iz=np.zeros(115, np.int32), src_ix=(4 + 8 * np.arange(115)).astype(np.int32),
        freqs=3.0 + 0.2 * np.arange(26), ricker_hz=8.0, mu_alpha=1e-2,
    )


def case_salt_patches(seed: int = 4) -> Case:
    """1701x351 salt model (4500 m/s body over 1500-4000 m/s sediments), nt 6000, three
    surface patches of 161, 257 and 341 receivers, 40 frequencies 2-10 Hz each."""
    rng = np.random.default_rng(seed)
    nz, nx = 351, 1701
    v = salt_model(rng, nz, nx)
    patches = [
        (100 + 5 * np.arange(161)).astype(np.int32),
        (400 + 4 * np.arange(257)).astype(np.int32),
        (300 + 3 * np.arange(341)).astype(np.int32),
    ]
    return Case(
        name="salt-1701x351-patches-161-257-341-nf40-nt6000",
        nz=nz, nx=nx, dz=10.0, dx=10.0, dt=1e-3, nt=6000, nsponge=20, sponge_R=1e-3,
        vel_true=v, patches=patches, freqs=np.linspace(2.0, 10.0, 40), mu_alpha=1e-2,
    )


def case_tiny(seed: int = 7, nz: int = 10, nx: int = 12, nsponge: int = 4, nrec: int = 5,
              nt: int = 48, dt: float = 1e-3, dx: float = 10.0) -> Case:
    """Tiny heterogeneous model for brute-force checks: smooth random velocity 1800-2600 m/s,
    receivers spread along the top physical row."""
    rng = np.random.default_rng(seed)
    v = 2200.0 + 400.0 * np.tanh(_smooth(rng.standard_normal((nz, nx)), 2.0) * 3.0)
    rix = np.linspace(0, nx - 1, nrec).round().astype(np.int32)
    return Case(
        name=f"tiny-{nx}x{nz}-nr{nrec}-nt{nt}",
        nz=nz, nx=nx, dz=dx, dx=dx, dt=dt, nt=nt, nsponge=nsponge, sponge_R=1e-3,
        vel_true=v, vel_start=v, rec_iz=np.zeros(nrec, np.int32), rec_ix=rix,
        freqs=np.array([15.0, 30.0, 45.0]), mu_alpha=1e-2,
    )


def slice_case(c: Case, nrec: int, nt: int, nsrc: int = 8) -> Case:
    """The same model and grid with fewer receivers (evenly spread), fewer sources and a shorter
    record: a bounded case for profiling captures."""
    d = Case(c)
    sel = np.linspace(0, c.rec_ix.size - 1, nrec).round().astype(int)
    ssel = np.linspace(0, c.src_ix.size - 1, nsrc).round().astype(int)
    d.update(name=f"{c.name}-slice-nr{nrec}-nt{nt}", nt=nt, rec_iz=c.rec_iz[sel], rec_ix=c.rec_ix[sel],
             src_iz=c.src_iz[ssel], src_ix=c.src_ix[ssel])
    return d
