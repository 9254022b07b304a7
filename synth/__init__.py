"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the FWIME method itself: it only draws
velocity models, acquisition geometries, source wavelets and random
perturbations, shaped like the paper's workloads (Marmousi2, BP-2004 North Sea,
salt examples; Barnier et al., Marmousi2, North Sea and Salt sections and the
computational-time table).  The public benchmark models themselves are not
available here; these seeded stand-ins reproduce their sizes, velocity ranges
and acquisition structure, never their content.

Seeds: ``SEED0 + config index`` with ``numpy.random.default_rng``.
Units: metres, seconds, m/s.  Arrays are float32 unless noted; indices are on
the physical grid (row-major ``[nz][nx]``, x fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED0 = 2206_02362


# ------------------------------------------------------------------ wavelets

def ricker(nt: int, dt: float, f0: float, delay: float | None = None) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - delay.

    The default delay 1.5/f0 makes |w(0)| < 1e-9 relative to the peak.
    Returned in float64 (callers cast).
    """
    if delay is None:
        delay = 1.5 / f0
    t = np.arange(nt) * dt - delay
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def ricker_at(t, f0: float, delay: float | None = None):
    """The same Ricker wavelet evaluated at arbitrary times t (float64)."""
    if delay is None:
        delay = 1.5 / f0
    a = (math.pi * f0 * (np.asarray(t, dtype=np.float64) - delay)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def lowcut(w: np.ndarray, dt: float, f_stop: float, f_pass: float) -> np.ndarray:
    """Zero-phase low-cut: spectrum x 0 below f_stop, cos^2 ramp to 1 at f_pass (float64)."""
    n = len(w)
    nfft = 1 << int(math.ceil(math.log2(2 * n)))
    W = np.fft.rfft(np.asarray(w, dtype=np.float64), nfft)
    f = np.fft.rfftfreq(nfft, dt)
    h = np.ones_like(f)
    h[f <= f_stop] = 0.0
    ramp = (f > f_stop) & (f < f_pass)
    h[ramp] = np.sin(0.5 * math.pi * (f[ramp] - f_stop) / (f_pass - f_stop)) ** 2
    return np.fft.irfft(W * h, nfft)[:n]


# ------------------------------------------------------------------- models

def _smooth1d(x: np.ndarray, width: int) -> np.ndarray:
    if width <= 1:
        return x
    k = np.hanning(width + 2)[1:-1]
    k /= k.sum()
    return np.convolve(np.pad(x, width, mode="edge"), k, mode="same")[width:-width]


def tiny_model(nz=100, nx=200, dx=10.0, seed=SEED0 + 0) -> np.ndarray:
    """1.5 km/s at the top, linear to 3.0 km/s at the bottom, times (1 +/- 10 % Gaussian, sigma 150 m)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None] * dx
    x = np.arange(nx)[None, :] * dx
    v = 1500.0 + 1500.0 * z / ((nz - 1) * dx)
    zc = rng.uniform(0.35, 0.65) * (nz - 1) * dx
    xc = rng.uniform(0.35, 0.65) * (nx - 1) * dx
    sign = 1.0 if rng.uniform() < 0.5 else -1.0
    v = v * (1.0 + sign * 0.1 * np.exp(-((z - zc) ** 2 + (x - xc) ** 2) / (2.0 * 150.0 ** 2)))
    return v.astype(np.float32)


def marmousi_like(nz=350, nx=1700, dx=10.0, water=450.0, vmax=4700.0, seed=SEED0 + 1) -> np.ndarray:
    """Folded and faulted layers under a water layer (Marmousi2-shaped stand-in)."""
    rng = np.random.default_rng(seed)
    v = np.full((nz, nx), 1500.0)
    x = np.arange(nx) * dx
    iw = int(round(water / dx))
    nlay = int(rng.integers(10, 15))
    depth = nz * dx
    # layer base depths (flat reference), folded by a sum of sinusoids
    bases = np.sort(rng.uniform(water + 50.0, depth, nlay - 1))
    bases = np.concatenate([bases, [depth + 1e3]])
    amp = rng.uniform(50.0, 300.0)
    fold = amp * np.sin(2 * math.pi * x / rng.uniform(3000, 8000) + rng.uniform(0, 6.28)) \
        + 0.4 * amp * np.sin(2 * math.pi * x / rng.uniform(1200, 2500) + rng.uniform(0, 6.28))
    # normal faults: throw applied to the right of each fault trace
    nf = int(rng.integers(3, 6))
    shift = np.zeros(nx)
    for _ in range(nf):
        xf = rng.uniform(0.1, 0.9) * nx * dx
        throw = rng.uniform(20.0, 80.0)
        shift[x > xf] += throw
    vel = np.linspace(1700.0, vmax, nlay) * (1.0 + rng.uniform(-0.05, 0.05, nlay))
    vel = np.minimum(vel, vmax)
    zz = np.arange(nz)[:, None] * dx
    for j in range(nx):
        top = water
        for k in range(nlay):
            base = bases[k] + fold[j] + shift[j]
            sel = (zz[:, 0] >= top) & (zz[:, 0] < base) & (zz[:, 0] >= water)
            v[sel, j] = vel[k]
            top = base
    v[:iw, :] = 1500.0
    return v.astype(np.float32)


def north_sea_like(nz=400, nx=1600, dx=12.5, seed=SEED0 + 2):
    """Flat layered sediments with a high-velocity chalk layer; returns (true, initial 1-D trend)."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz) * dx
    depth = nz * dx
    nlay = int(rng.integers(8, 14))
    bases = np.sort(rng.uniform(200.0, depth, nlay - 1))
    prof = np.full(nz, 1500.0)
    vel = np.linspace(1600.0, 4200.0, nlay)
    top = 0.0
    for k, base in enumerate(np.concatenate([bases, [depth + 1.0]])):
        prof[(z >= top) & (z < base)] = vel[k]
        top = base
    ctop = rng.uniform(0.3, 0.5) * depth
    cthk = rng.uniform(100.0, 200.0)
    prof[(z >= ctop) & (z < ctop + cthk)] = 4500.0
    prof[z < 100.0] = 1500.0
    v = np.repeat(prof[:, None], nx, axis=1)
    v0 = np.repeat(np.linspace(1500.0, 4000.0, nz)[:, None], nx, axis=1)
    return v.astype(np.float32), v0.astype(np.float32)


def salt_like(nz=1200, nx=5000, dx=6.25, seed=SEED0 + 4) -> np.ndarray:
    """Sediments 1.5-3.5 km/s, a 4.5 km/s salt body with a rugose top and a feeder stem."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz)[:, None] * dx
    x = np.arange(nx)[None, :] * dx
    depth, width = nz * dx, nx * dx
    v = 1500.0 + 2000.0 * np.clip((z - 300.0) / (depth - 300.0), 0.0, 1.0) * np.ones_like(x)
    v[(z < 300.0)[:, 0], :] = 1500.0
    rough = _smooth1d(rng.normal(0.0, 1.0, nx), 40)
    rough = rough / (np.abs(rough).max() + 1e-12) * rng.uniform(30.0, 60.0)
    xc = rng.uniform(0.4, 0.6) * width
    half = 0.22 * width
    top = 0.35 * depth + 0.12 * depth * ((x[0] - xc) / half) ** 2 + rough
    base = 0.62 * depth - 0.06 * depth * ((x[0] - xc) / half) ** 2
    inside = (np.abs(x - xc) < half) & (z >= top[None, :]) & (z <= base[None, :])
    stem = (np.abs(x - xc) < 150.0) & (z >= 0.4 * depth)
    v = np.where(inside | stem, 4500.0, v)
    return v.astype(np.float32)


def layered(nz, nx, dx, seed, vmin=1500.0, vmax=4500.0) -> np.ndarray:
    """Seeded flat-ish layered model (serving-mix requests)."""
    rng = np.random.default_rng(seed)
    nlay = int(rng.integers(4, 10))
    z = np.arange(nz) * dx
    bases = np.sort(rng.uniform(0.1, 1.0, nlay - 1)) * nz * dx
    vel = np.sort(rng.uniform(vmin, vmax, nlay))
    vel[0] = vmin
    prof = np.empty(nz)
    top = -1.0
    for k, base in enumerate(np.concatenate([bases, [nz * dx + 1.0]])):
        prof[(z >= top) & (z < base)] = vel[k]
        top = base
    return np.repeat(prof[:, None], nx, axis=1).astype(np.float32)


# ------------------------------------------------------------- perturbations

def gaussian_blobs(nz, nx, rng, nblob=4, amp=1.0, sigma_pts=6.0, ring=2) -> np.ndarray:
    """Smooth random perturbation, exactly zero on the outer `ring` points (float64)."""
    z = np.arange(nz)[:, None]
    x = np.arange(nx)[None, :]
    out = np.zeros((nz, nx))
    for _ in range(nblob):
        zc = rng.uniform(0.2, 0.8) * nz
        xc = rng.uniform(0.2, 0.8) * nx
        out += rng.normal() * np.exp(-((z - zc) ** 2 + (x - xc) ** 2) / (2 * sigma_pts ** 2))
    out *= amp / (np.abs(out).max() + 1e-300)
    out[:ring, :] = 0.0; out[-ring:, :] = 0.0; out[:, :ring] = 0.0; out[:, -ring:] = 0.0
    return out


def random_ptilde(nh, nz, nx, rng) -> np.ndarray:
    """Extended perturbation p~ ~ N(0, 1), [nh][nz][nx] (float64)."""
    return rng.standard_normal((nh, nz, nx))


# ------------------------------------------------------------------ configs

@dataclass
class Workload:
    """One seeded synthetic workload: grid, acquisition, wavelet and model."""
    name: str
    nz: int
    nx: int
    dx: float
    dt: float
    nt: int
    W: int
    nh: int
    f0: float
    src_iz: np.ndarray
    src_ix: np.ndarray
    rec_iz: np.ndarray
    rec_ix: np.ndarray
    v: np.ndarray = field(repr=False)
    w: np.ndarray = field(repr=False)   # [nt] float64, shared by all shots
    seed: int = SEED0

    @property
    def nshot(self) -> int:
        return len(self.src_iz)

    @property
    def nrec(self) -> int:
        return len(self.rec_iz)

    @property
    def padded(self) -> tuple[int, int]:
        return self.nz + 2 * (self.W + 4), self.nx + 2 * (self.W + 4)

    def updates_per_propagation(self) -> int:
        """Padded grid points x time steps of one propagation of one shot."""
        NZ, NX = self.padded
        return NZ * NX * (self.nt - 1)


def tiny(nt: int = 1000) -> Workload:
    """100 x 200 at 10 m, nt=1000, dt=1 ms, 15 Hz Ricker at (20 m, 1000 m), 200 receivers at 20 m, W=30, nh=5."""
    nz, nx, dx = 100, 200, 10.0
    v = tiny_model(nz, nx, dx)
    return Workload("tiny-100x200-nt1000-nh5", nz, nx, dx, 1e-3, nt, 30, 5, 15.0,
                    np.array([2]), np.array([100]),
                    np.full(nx, 2), np.arange(nx), v, ricker(nt, 1e-3, 15.0), SEED0 + 0)


def marmousi2(nshot: int = 100, nt: int = 4000) -> Workload:
    """350 x 1700 at 10 m, 100 shots every 170 m, 850 receivers every 20 m at 20 m depth,
    nt=4000, dt=0.8 ms, 8 Hz Ricker low-cut below 4 Hz, nh=21, W=50."""
    nz, nx, dx, dt = 350, 1700, 10.0, 8e-4
    v = marmousi_like(nz, nx, dx)
    w = lowcut(ricker(nt, dt, 8.0), dt, 2.0, 4.0)
    src_ix = (8 + 17 * np.arange(100))[:nshot]
    return Workload(f"marmousi2-like-350x1700-nt{nt}-nh21", nz, nx, dx, dt, nt, 50, 21, 8.0,
                    np.full(len(src_ix), 2), src_ix, np.full(850, 2), 2 * np.arange(850), v, w,
                    SEED0 + 1)


def north_sea(nshot: int = 120, nt: int = 5000):
    """400 x 1600 at 12.5 m, 120 shots, 800 receivers every 2 points, nt=5000, dt=1 ms, nh=31.
    Returns (workload with the true model, initial 1-D trend model)."""
    nz, nx, dx, dt = 400, 1600, 12.5, 1e-3
    v, v0 = north_sea_like(nz, nx, dx)
    src_ix = np.round(np.linspace(6, nx - 7, 120)).astype(int)[:nshot]
    wl = Workload(f"north-sea-like-400x1600-nt{nt}-nh31", nz, nx, dx, dt, nt, 50, 31, 8.0,
                  np.full(len(src_ix), 2), src_ix, np.full(800, 2), 2 * np.arange(800), v,
                  ricker(nt, dt, 8.0), SEED0 + 2)
    return wl, v0


def salt(nshot: int = 400, nt: int = 8000) -> Workload:
    """1200 x 5000 at 6.25 m, 400 shots, 2500 receivers every 2 points, nt=8000, dt=0.5 ms, 10 Hz, nh=41."""
    nz, nx, dx, dt = 1200, 5000, 6.25, 5e-4
    v = salt_like(nz, nx, dx)
    src_ix = np.round(np.linspace(6, nx - 7, 400)).astype(int)[:nshot]
    return Workload(f"salt-like-1200x5000-nt{nt}-nh41", nz, nx, dx, dt, nt, 50, 41, 10.0,
                    np.full(len(src_ix), 4), src_ix, np.full(2500, 4), 2 * np.arange(2500), v,
                    ricker(nt, dt, 10.0), SEED0 + 4)


@dataclass
class Request:
    """One serving request: a forward-modelling or a gradient shot on its own grid."""
    rid: int
    arrival: float
    kind: str            # "forward" | "gradient"
    workload: Workload


def serving_mix(nreq: int = 2000, rate: float = 200.0, seed: int = SEED0 + 3,
                nz_range=(200, 600), nx_range=(400, 2000), nt_range=(2000, 6000),
                nh_choices=(1, 11, 31)) -> list[Request]:
    """Poisson arrivals (mean `rate`/s); grids, nt and nh drawn uniformly; forward:gradient 1:1."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(nreq):
        t += rng.exponential(1.0 / rate)
        nz = int(rng.integers(nz_range[0], nz_range[1] + 1))
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1)) // 4 * 4
        nt = int(rng.integers(nt_range[0], nt_range[1] + 1))
        nh = int(rng.choice(nh_choices))
        v = layered(nz, nx, 10.0, seed * 7919 + i)
        ix = int(rng.integers(nx // 4, 3 * nx // 4))
        nrec = nx // 2
        wl = Workload(f"req{i}", nz, nx, 10.0, 1e-3, nt, 50, nh, 10.0, np.array([2]), np.array([ix]),
                      np.full(nrec, 2), 2 * np.arange(nrec), v, ricker(nt, 1e-3, 10.0), seed * 7919 + i)
        out.append(Request(i, t, "forward" if rng.uniform() < 0.5 else "gradient", wl))
    return out
