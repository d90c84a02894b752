"""Seeded synthetic interferometer inputs (array geometry, uvw tracks, sky, visibilities).

This module is the one piece shared by the FP64 oracle and the CUDA path. It holds
input synthesis only (antenna layout, the textbook baseline -> uvw rotation, a point
source sky, the measurement equation used to make visibility values, noise) and none
of the W-projection arithmetic: no coordinate quantisation, no kernels, no gridding,
no FFT.

The paper's workload is a JVLA L-band D-array Measurement Set of G55.7+3.4
(Sec. 3.1: 8 h, 1-2 GHz, 1024^2 pixels of 8 arcsec, 23 w-planes, full support 9).
That dataset is not available, so these generators stand in for it with arrays of the
same kind (antennas uniform in a disk with small height scatter, Earth-rotation tracks
over hours, point sources in the field, Gaussian noise).

Visibility convention (measurement equation, used only to synthesise values):
    V(u, v, w) = sum_s F_s exp(-2 pi i (u l_s + v m_s + w (n_s - 1))),  n = sqrt(1 - l^2 - m^2)
with u, v, w in wavelengths. Rows are ordered (time, baseline) as a Measurement Set
stores them (Fig. 1 caption: rows x channels x polarisations, one correlation here).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0
ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0
# Site latitude of the stand-in array (a JVLA-like site; the paper's data is JVLA).
SITE_LAT = 34.08 * DEG


@dataclass
class ArrayConfig:
    """One synthetic observation plus the imaging parameters it is imaged with."""
    name: str
    n_ant: int
    radius_m: float
    height_m: float
    dec: float                      # phase-centre declination (rad)
    n_time: int
    duration_h: float
    freqs: np.ndarray               # channel frequencies (Hz)
    n_src: int
    src_field: float                # sources uniform in |l|,|m| < src_field/2 (rad)
    flux: str                       # "loguniform" (0.01-1 Jy) or "powerlaw" (dN/dS ~ S^-1.5 on [0.01, 1])
    noise_sigma: float
    n: int                          # grid / image size (pixels per side)
    cell: float                     # cell size (rad)
    n_w: int
    s_min: int
    s_max: int
    oversample: int
    hermitian_pairs: bool = False   # grid each sample and its conjugate at -uvw
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_baselines(self) -> int:
        return self.n_ant * (self.n_ant - 1) // 2

    @property
    def n_rows(self) -> int:
        return self.n_baselines * self.n_time

    @property
    def n_vis(self) -> int:
        return self.n_rows * len(self.freqs)

    @property
    def n_gridded(self) -> int:
        return self.n_vis * (2 if self.hermitian_pairs else 1)


def config(name: str) -> ArrayConfig:
    """The workloads used by the tests and the benchmark.

    parity    : 27 antennas, 2 km disk, +-20 m, dec +45, 60 hour angles over 2 h, 1 channel
                at 1.4 GHz -> 21,060 visibilities from 10 sources; 256^2 grid, 10" cells,
                16 w-planes, support 7, oversampling 8.
    fp32      : 128 antennas, 5 km disk, +-50 m, 4 channels 1.0-1.4 GHz, 480 samples over
                8 h -> 15.6M samples gridded with their Hermitian conjugates (31.2M
                gridded visibilities); 200 power-law sources; 2048^2 grid, 1" cells,
                32 w-planes, support 8-16, oversampling 8.
    mixed     : 256 antennas, 10 km disk, 16 channels 1.0-1.4 GHz, 720 samples over 8 h
                -> 376M visibilities; 4096^2 grid, 0.5" cells, 64 w-planes, support 8-32.
    diff      : 64 antennas, 2016 baselines x 496 samples ~ 1.0M visibilities; 2048^2,
                32 w-planes, support 12, oversampling 8.
    """
    if name == "parity":
        return ArrayConfig(name, n_ant=27, radius_m=2000.0, height_m=20.0, dec=45 * DEG,
                           n_time=60, duration_h=2.0, freqs=np.array([1.4e9]),
                           n_src=10, src_field=1.0 * DEG, flux="loguniform", noise_sigma=0.01,
                           n=256, cell=10 * ARCSEC, n_w=16, s_min=7, s_max=7, oversample=8,
                           seed=1001)
    if name == "fp32":
        return ArrayConfig(name, n_ant=128, radius_m=5000.0, height_m=50.0, dec=45 * DEG,
                           n_time=480, duration_h=8.0, freqs=np.linspace(1.0e9, 1.4e9, 4),
                           n_src=200, src_field=0.9 * 2048 * ARCSEC, flux="powerlaw",
                           noise_sigma=0.01, n=2048, cell=1.0 * ARCSEC, n_w=32, s_min=8,
                           s_max=16, oversample=8, hermitian_pairs=True, seed=1002)
    if name == "mixed":
        return ArrayConfig(name, n_ant=256, radius_m=10000.0, height_m=50.0, dec=45 * DEG,
                           n_time=720, duration_h=8.0, freqs=np.linspace(1.0e9, 1.4e9, 16),
                           n_src=200, src_field=0.9 * 4096 * 0.5 * ARCSEC, flux="powerlaw",
                           noise_sigma=0.01, n=4096, cell=0.5 * ARCSEC, n_w=64, s_min=8,
                           s_max=32, oversample=8, seed=1003)
    if name == "diff":
        return ArrayConfig(name, n_ant=64, radius_m=5000.0, height_m=50.0, dec=45 * DEG,
                           n_time=496, duration_h=8.0, freqs=np.array([1.4e9]),
                           n_src=50, src_field=0.9 * 2048 * ARCSEC, flux="powerlaw",
                           noise_sigma=0.01, n=2048, cell=1.0 * ARCSEC, n_w=32, s_min=12,
                           s_max=12, oversample=8, seed=1005)
    raise KeyError(name)


def antenna_enu(n_ant: int, radius_m: float, height_m: float, rng: np.random.Generator) -> np.ndarray:
    """Antennas uniform in a disk (r = R sqrt(U), theta uniform), heights uniform in +-h. [n_ant, 3] (E, N, U) m."""
    r = radius_m * np.sqrt(rng.random(n_ant))
    th = 2 * np.pi * rng.random(n_ant)
    up = height_m * (2 * rng.random(n_ant) - 1)
    return np.stack([r * np.cos(th), r * np.sin(th), up], axis=1)


def baseline_pairs(n_ant: int) -> tuple[np.ndarray, np.ndarray]:
    """Unordered antenna pairs (i < j), no autocorrelations."""
    a1, a2 = np.triu_indices(n_ant, k=1)
    return a1.astype(np.int64), a2.astype(np.int64)


def row_antennas(n_ant: int, n_time: int) -> tuple[np.ndarray, np.ndarray]:
    """Antenna IDs (ant1, ant2) int32 of every row in uvw_metres' time-major row order."""
    a1, a2 = baseline_pairs(n_ant)
    return np.tile(a1, n_time).astype(np.int32), np.tile(a2, n_time).astype(np.int32)


def hour_angles(n_time: int, duration_h: float) -> np.ndarray:
    """Sample centres H_k = -T/2 + (k + 1/2) T / n, centred on transit (rad)."""
    t = -duration_h / 2 + (np.arange(n_time) + 0.5) * duration_h / n_time
    return t * (2 * np.pi / 24.0)


def uvw_metres(enu: np.ndarray, lat: float, dec: float, ha: np.ndarray) -> np.ndarray:
    """Baseline uvw in metres for every (time, baseline) row, the textbook equatorial rotation.

    Local (E, N, U) -> equatorial (X, Y, Z): X = -N sin(lat) + U cos(lat), Y = E,
    Z = N cos(lat) + U sin(lat). Then for hour angle H and declination d:
        u =  sin H X + cos H Y
        v = -sin d cos H X + sin d sin H Y + cos d Z
        w =  cos d cos H X - cos d sin H Y + sin d Z
    Returns [n_time * n_baselines, 3], rows ordered time-major.
    """
    e, n, up = enu[:, 0], enu[:, 1], enu[:, 2]
    x = -n * math.sin(lat) + up * math.cos(lat)
    y = e
    z = n * math.cos(lat) + up * math.sin(lat)
    a1, a2 = baseline_pairs(len(enu))
    bx, by, bz = x[a2] - x[a1], y[a2] - y[a1], z[a2] - z[a1]
    sh, ch = np.sin(ha)[:, None], np.cos(ha)[:, None]
    sd, cd = math.sin(dec), math.cos(dec)
    u = sh * bx + ch * by
    v = -sd * ch * bx + sd * sh * by + cd * bz
    w = cd * ch * bx - cd * sh * by + sd * bz
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


def sky(n_src: int, field: float, flux: str, rng: np.random.Generator) -> np.ndarray:
    """Point sources [n_src, 3] = (l, m, flux Jy), uniform in |l|, |m| < field/2."""
    lm = (rng.random((n_src, 2)) - 0.5) * field
    if flux == "loguniform":
        f = 10 ** rng.uniform(-2, 0, n_src)
    elif flux == "powerlaw":
        # dN/dS ~ S^-1.5 on [a, b]: inverse CDF of S^-0.5
        a, b = 0.01, 1.0
        q = rng.random(n_src)
        f = (a ** -0.5 - q * (a ** -0.5 - b ** -0.5)) ** -2.0
    else:
        raise ValueError(flux)
    return np.concatenate([lm, f[:, None]], axis=1)


def predict_numpy(uvw_m: np.ndarray, freqs: np.ndarray, src: np.ndarray) -> np.ndarray:
    """Measurement equation on the host, complex128 [nrow, nchan] (small inputs only)."""
    l, m, f = src[:, 0], src[:, 1], src[:, 2]
    nm1 = np.sqrt(1 - l * l - m * m) - 1
    out = np.zeros((uvw_m.shape[0], len(freqs)), np.complex128)
    for c, fr in enumerate(freqs):
        s = fr / C_LIGHT
        ph = (uvw_m[:, 0:1] * l + uvw_m[:, 1:2] * m + uvw_m[:, 2:3] * nm1) * s
        out[:, c] = (f * np.exp(-2j * np.pi * ph)).sum(1)
    return out


def predict_torch(uvw_m, freqs: np.ndarray, src: np.ndarray, chunk: int = 1 << 20):
    """Measurement equation with torch on uvw_m's device (any size), complex64 [nrow, nchan].

    Phases are formed in float64 (source by source) and exponentiated in float32; these
    are input values only, so their own rounding is irrelevant to any parity check,
    which always compares two computations on the same stored values.
    """
    import torch
    dev = uvw_m.device
    nrow = uvw_m.shape[0]
    out = torch.zeros((nrow, len(freqs)), dtype=torch.complex64, device=dev)
    srct = torch.as_tensor(src, dtype=torch.float64, device=dev)
    l, m, f = srct[:, 0], srct[:, 1], srct[:, 2]
    nm1 = torch.sqrt(1 - l * l - m * m) - 1
    for r0 in range(0, nrow, chunk):
        u = uvw_m[r0:r0 + chunk]
        base = u[:, 0:1] * l + u[:, 1:2] * m + u[:, 2:3] * nm1          # [rows, nsrc] metres
        for c, fr in enumerate(freqs):
            ph = torch.remainder(base * (fr / C_LIGHT), 1.0).to(torch.float32)
            val = torch.polar(f.to(torch.float32).expand_as(ph), -2 * math.pi * ph)
            out[r0:r0 + chunk, c] = val.sum(1)
    return out


def predict_torch_f32(uvw_m, freqs: np.ndarray, src: np.ndarray, chunk: int = 1 << 19):
    """The measurement equation with every phase in float32, for workloads too large for the
    float64 route on a GPU whose float64 rate is a small fraction of its float32 rate (the
    376M-visibility workload with 200 sources is 75G source terms).

    Phases of these arrays stay below ~1e3 turns, so float32 keeps them to ~1e-4 turn: the
    values are a point-source sky plus noise either way, and parity checks always compare two
    computations on the same stored values.
    """
    import torch
    dev = uvw_m.device
    nrow = uvw_m.shape[0]
    out = torch.zeros((nrow, len(freqs)), dtype=torch.complex64, device=dev)
    srct = torch.as_tensor(src, dtype=torch.float64, device=dev)
    lmn = torch.stack([srct[:, 0], srct[:, 1], torch.sqrt(1 - srct[:, 0] ** 2 - srct[:, 1] ** 2) - 1]).to(torch.float32)
    flux = srct[:, 2].to(torch.complex64)
    for r0 in range(0, nrow, chunk):
        base = uvw_m[r0:r0 + chunk].to(torch.float32) @ lmn                 # [rows, nsrc] metres
        for c, fr in enumerate(freqs):
            ph = torch.frac(base * float(fr / C_LIGHT))
            out[r0:r0 + chunk, c] = torch.polar(torch.ones_like(ph), -2 * math.pi * ph) @ flux
    return out


@dataclass
class Observation:
    cfg: ArrayConfig
    uvw: object        # [nrow, 3] float64 metres (numpy or torch)
    freqs: np.ndarray  # [nchan] float64 Hz
    vis: object        # [nrow, nchan] complex64
    weight: object     # [nrow, nchan] float32
    sources: np.ndarray
    w_max: float       # max |w| in wavelengths over all rows and channels


def observe(cfg: ArrayConfig, device: str = "cpu", rows: int | None = None) -> Observation:
    """Build the observation for `cfg` (optionally only the first `rows` rows).

    Seeds: geometry cfg.seed, sources cfg.seed + 1000, noise cfg.seed + 2000.
    Small inputs are made with numpy on the host; with device="cuda" the uvw, values and
    weights are made as torch tensors on the GPU (the values need the measurement
    equation over every source and sample, which is too slow on the host at scale), with
    float64 phases, or float32 phases beyond 4e9 source terms (predict_torch_f32).
    """
    rng = np.random.default_rng(cfg.seed)
    enu = antenna_enu(cfg.n_ant, cfg.radius_m, cfg.height_m, rng)
    ha = hour_angles(cfg.n_time, cfg.duration_h)
    uvw = uvw_metres(enu, SITE_LAT, cfg.dec, ha)
    if rows is not None:
        uvw = uvw[:rows]
    src = sky(cfg.n_src, cfg.src_field, cfg.flux, np.random.default_rng(cfg.seed + 1000))
    freqs = np.asarray(cfg.freqs, dtype=np.float64)
    w_max = float(np.max(np.abs(uvw[:, 2])) * freqs.max() / C_LIGHT)
    nrow, nchan = uvw.shape[0], len(freqs)
    if device == "cpu":
        vis = predict_numpy(uvw, freqs, src)
        nrng = np.random.default_rng(cfg.seed + 2000)
        vis = vis + cfg.noise_sigma * (nrng.standard_normal(vis.shape) + 1j * nrng.standard_normal(vis.shape))
        vis = vis.astype(np.complex64)
        weight = np.ones((nrow, nchan), np.float32)
        return Observation(cfg, uvw, freqs, vis, weight, src, w_max)
    import torch
    uvw_t = torch.as_tensor(uvw, dtype=torch.float64, device=device)
    big = nrow * nchan * cfg.n_src > 4_000_000_000
    vis = predict_torch_f32(uvw_t, freqs, src) if big else predict_torch(uvw_t, freqs, src)
    g = torch.Generator(device=device)
    g.manual_seed(cfg.seed + 2000)
    noise = torch.randn((nrow, nchan, 2), generator=g, device=device, dtype=torch.float32) * cfg.noise_sigma
    vis = vis + torch.view_as_complex(noise)
    weight = torch.ones((nrow, nchan), dtype=torch.float32, device=device)
    return Observation(cfg, uvw_t, freqs, vis, weight, src, w_max)


def random_visibilities(nrow: int, nchan: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit-variance complex64 values and weights in [0.5, 1.5) (for parity cases)."""
    rng = np.random.default_rng(seed)
    vis = (rng.standard_normal((nrow, nchan)) + 1j * rng.standard_normal((nrow, nchan))).astype(np.complex64)
    wt = (0.5 + rng.random((nrow, nchan))).astype(np.float32)
    return vis, wt


def random_grid(n: int, seed: int) -> np.ndarray:
    """Unit-variance complex64 [n, n] grid (degridding parity input)."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)


# ---------------------------------------------------------------- batched imaging jobs

@dataclass
class JobSpec:
    """One imaging job of the batched workload: its array, grid and kernel geometry."""
    n: int
    n_w: int
    s_min: int
    s_max: int
    oversample: int
    n_ant: int
    n_time: int
    freqs: np.ndarray
    cell: float
    radius_m: float
    seed: int


def batch_jobs(n_jobs: int = 64, seed: int = 1004, nvis_min: float = 1e4, nvis_max: float = 2e7,
               scale: float = 1.0) -> list[JobSpec]:
    """Channel / snapshot imaging jobs of uneven sizes: grid sizes from {512, 1024, 2048, 4096},
    visibility counts log-uniform in [nvis_min, nvis_max] (times `scale`), supports 7-31,
    oversampling 4, 6 or 8 and 8-64 w-planes. Snapshot jobs have many baselines and few samples,
    channel jobs one channel and long tracks; the cell size makes the longest baseline fill the
    grid to 95%."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        n = int(rng.choice([512, 1024, 2048, 4096]))
        nvis = float(np.exp(rng.uniform(np.log(nvis_min), np.log(nvis_max)))) * scale
        s_min = int(rng.integers(7, 32))
        s_max = int(rng.integers(s_min, 32))
        os_ = int(rng.choice([4, 6, 8]))                    # even, as the kernel tables need
        n_w = int(rng.integers(8, 65))
        nchan = int(rng.choice([1, 2, 4]))
        n_ant = int(rng.integers(16, 129))
        nbl = n_ant * (n_ant - 1) // 2
        n_time = max(1, int(round(nvis / (nbl * nchan))))
        radius = float(rng.uniform(1000.0, 8000.0))
        freqs = np.linspace(1.0e9, 1.4e9, nchan) if nchan > 1 else np.array([1.2e9])
        umax = 2.0 * radius * freqs.max() / C_LIGHT           # longest baseline in wavelengths
        cell = 1.0 / (2.0 * umax / 0.95)
        jobs.append(JobSpec(n, n_w, s_min, s_max, os_, n_ant, n_time, freqs, cell, radius, seed * 100 + j))
    return jobs


def job_uvw(spec: JobSpec) -> np.ndarray:
    """uvw [n_baselines * n_time, 3] (m) of a job's array over 6 h at declination +40 deg."""
    rng = np.random.default_rng(spec.seed)
    enu = antenna_enu(spec.n_ant, spec.radius_m, 20.0, rng)
    return uvw_metres(enu, SITE_LAT, 40 * DEG, hour_angles(spec.n_time, 6.0))
