"""Seeded synthetic workloads for direct inverse ray-shooting.

This module is the one piece that both the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1406_0559_b300``) are fed from.  It holds only parameter
sets and seeded draws of those parameters; it performs none of the method's
arithmetic (no lens placement, no deflection, no binning).  Lens fields are
drawn by each side from the same counter-based generator definition, given the
``seed`` recorded here.

Units: lengths in Einstein radii of the mean microlens mass (Eq. 5), masses in
units of that mean mass.  A ray grid is ``n1 x n2`` cell-centred rays over the
rectangle ``[c1-half1, c1+half1] x [c2-half2, c2+half2]``; a map is ``npix^2``
pixels over the square of side ``width`` centred on ``(mc1, mc2)``.

The shapes follow the GERLUMPH survey (Sec. 3.1, Table 3: 4096^2 maps over
24 R_E, 10000^2 over 25 R_E, N_* ~ 1e3-1e5 (Sec. 2.1), ~1e9 rays).  The
survey's maps and lens files are not used; these synthetic fields stand in
for them.
"""
from __future__ import annotations

from dataclasses import dataclass, replace, asdict
import math

import numpy as np

MASS_UNIT = 0
MASS_SALPETER = 1


@dataclass(frozen=True)
class MapJob:
    """One magnification-map job: macromodel, lens field, ray grid, map."""

    name: str
    kappa_star: float          # compact-object convergence (Eq. 2)
    kappa_s: float             # smooth-matter convergence (Eq. 1)
    gamma: float               # external shear (Eq. 1)
    n_lens: int                # explicit N_*; 0 means "from Eq. 3"
    lens_radius: float         # radius of the lens disk (area A = pi R^2)
    mass_model: int = MASS_UNIT
    m_lo: float = 0.1
    m_hi: float = 1.0
    slope: float = 2.35        # dN/dm ~ m^-slope for the Salpeter model
    seed: int = 1
    n1: int = 2048             # rays along x1
    n2: int = 2048             # rays along x2
    c1: float = 0.0
    c2: float = 0.0
    half1: float = 7.5         # half-width of the ray rectangle along x1
    half2: float = 7.5
    mc1: float = 0.0           # map centre
    mc2: float = 0.0
    width: float = 10.0        # map side
    npix: int = 256

    @property
    def kappa(self) -> float:
        return self.kappa_star + self.kappa_s

    @property
    def n_rays(self) -> int:
        return self.n1 * self.n2

    def with_(self, **kw) -> "MapJob":
        return replace(self, **kw)

    def to_dict(self) -> dict:
        return asdict(self)


# Plain single map, small enough for the oracle to finish in seconds:
# 150 unit lenses in a disk of radius 11, map 256^2 over 10 R_E, rays
# 2048^2 over a 15 R_E square (about 6.3e8 ray-lens interactions).
PARITY = MapJob(name="parity-256", kappa_star=0.4, kappa_s=0.0, gamma=0.3,
                n_lens=150, lens_radius=11.0, seed=1,
                n1=2048, n2=2048, half1=7.5, half2=7.5, width=10.0, npix=256)

# GERLUMPH-scale plain map: 24,000 unit lenses (kappa_* R^2 = 0.6 * 200^2,
# i.e. Eq. 3), map 4096^2 over 25 R_E, rays 16384^2 over a 60 R_E square.
GERLUMPH = MapJob(name="gerlumph-4096", kappa_star=0.6, kappa_s=0.0, gamma=0.3,
                  n_lens=24000, lens_radius=200.0, seed=2,
                  n1=16384, n2=16384, half1=30.0, half2=30.0, width=25.0, npix=4096)

# Precision-form map: kappa = 0.8 split 0.4/0.4, gamma 0.2, 50,000 Salpeter
# lenses (0.1-1.0, slope 2.35, mean-normalised) in a disk of radius 280.
PRECISION = MapJob(name="precision-4096", kappa_star=0.4, kappa_s=0.4, gamma=0.2,
                   n_lens=50000, lens_radius=280.0, mass_model=MASS_SALPETER,
                   seed=3, n1=16384, n2=16384, half1=30.0, half2=30.0,
                   width=25.0, npix=4096)
PRECISION_WINDOW = 512       # central sub-window compared against the oracle

# The GERLUMPH-scale map with 2048^2 rays (same lenses, map and ray square):
# the profiling case, small enough for a multi-pass hardware-counter capture.
GERLUMPH_SMALL = GERLUMPH.with_(name="gerlumph-4096/rays2048", n1=2048, n2=2048)

# Few lenses (N = 200, the low end of the serving range) on the benchmark's
# geometry with 4096^2 rays: per-ray work (FP64 ray positions, Eq. 1
# combine, binning) weighs as much as the deflection sum here.
GERLUMPH_N200 = GERLUMPH.with_(name="gerlumph-4096/n200", n_lens=200,
                               lens_radius=math.sqrt(200 / 0.6), n1=4096, n2=4096)

CONFIGS = {j.name: j for j in (PARITY, GERLUMPH, PRECISION, GERLUMPH_SMALL, GERLUMPH_N200)}


def scaled(job: MapJob, ray_scale: int = 1, map_scale: int = 1,
           lens_scale: int = 1, name: str | None = None) -> MapJob:
    """Shrink a job by integer factors (rays per side, pixels per side, lens
    count and disk area) while keeping its geometry and lens density."""
    n_lens = max(1, job.n_lens // lens_scale) if job.n_lens else 0
    radius = job.lens_radius / math.sqrt(lens_scale)
    return job.with_(name=name or f"{job.name}/r{ray_scale}m{map_scale}l{lens_scale}",
                     n1=job.n1 // ray_scale, n2=job.n2 // ray_scale,
                     npix=job.npix // map_scale, n_lens=n_lens, lens_radius=radius)


def batch_grid(n_maps: int = 64, seed: int = 4, n_lo: int = 500, n_hi: int = 50000,
               map_sides=(1024, 2048, 4096), ray_factor: int = 4,
               ray_width: float = 60.0, map_width: float = 25.0,
               smooth_fracs=(0.0, 0.3, 0.6, 0.9), crit_gap: float = 0.05) -> list[MapJob]:
    """Seeded draw of a (kappa, gamma) survey grid of uneven map jobs.

    kappa ~ U[0.1, 1.2], gamma ~ U[0, 1.0], rejecting points with
    |(1-kappa)^2 - gamma^2| < crit_gap (too close to the critical line);
    smooth fraction s from ``smooth_fracs``; N log-uniform in [n_lo, n_hi];
    map side from ``map_sides``; ray side = ray_factor x map side.  The disk
    radius is chosen so that N lenses of unit mean mass give kappa_* over the
    disk area.
    """
    rng = np.random.default_rng(seed)
    jobs: list[MapJob] = []
    while len(jobs) < n_maps:
        kappa = float(rng.uniform(0.1, 1.2))
        gamma = float(rng.uniform(0.0, 1.0))
        if abs((1.0 - kappa) ** 2 - gamma ** 2) < crit_gap:
            continue
        s = float(rng.choice(np.asarray(smooth_fracs)))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        side = int(rng.choice(np.asarray(map_sides)))
        lseed = int(rng.integers(1, 2**62))
        kstar = kappa * (1.0 - s)
        radius = math.sqrt(n / kstar)
        k = len(jobs)
        jobs.append(MapJob(name=f"batch{k:03d}", kappa_star=kstar, kappa_s=kappa * s,
                           gamma=gamma, n_lens=n, lens_radius=radius, seed=lseed,
                           n1=side * ray_factor, n2=side * ray_factor,
                           half1=ray_width / 2, half2=ray_width / 2,
                           width=map_width, npix=side))
    return jobs


@dataclass(frozen=True)
class Request:
    """One map request of the serving stream."""
    rid: int
    arrival_s: float
    job: MapJob


def serve_stream(n_req: int = 1000, seed: int = 5, rate_hz: float = 1.0,
                 n_lo: int = 200, n_hi: int = 80000,
                 map_sides=(512, 1024, 2048, 4096, 8192), **grid_kw) -> list[Request]:
    """Seeded Poisson stream of map requests drawn from the batch grid's
    parameter ranges (kappa, gamma, smooth fraction), with N and map side
    from the serving ranges.  ``rate_hz`` is the mean arrival rate."""
    rng = np.random.default_rng(seed)
    jobs = batch_grid(n_maps=n_req, seed=seed + 1000, n_lo=n_lo, n_hi=n_hi,
                      map_sides=map_sides, **grid_kw)
    gaps = rng.exponential(1.0 / rate_hz, size=n_req)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(rid=k, arrival_s=float(t[k]), job=j.with_(name=f"req{k:04d}"))
            for k, j in enumerate(jobs)]


def sample_tiles(n_tiles_total: int, k: int, seed: int) -> np.ndarray:
    """Seeded choice of ``k`` distinct tile indices out of ``n_tiles_total``
    (used to sample rays of a full-size map for per-ray comparison)."""
    rng = np.random.default_rng(seed)
    k = min(k, n_tiles_total)
    return np.sort(rng.choice(n_tiles_total, size=k, replace=False)).astype(np.int64)


def sample_rays(n1: int, n2: int, k: int, seed: int) -> np.ndarray:
    """Seeded choice of ``k`` ray indices (i, j) of an n1 x n2 grid, as an
    int64 array of shape (k, 2)."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, n1, size=k, dtype=np.int64)
    j = rng.integers(0, n2, size=k, dtype=np.int64)
    return np.stack([i, j], axis=1)


# --------------------------------------------------------------------------
# finite-source convolution inputs (Sec. 2.4, Sec. 2.5 item 3)
# --------------------------------------------------------------------------

PROFILE_UNIFORM = 0
PROFILE_GAUSSIAN = 1
PROFILE_POWER_LAW = 2
PROFILE_THIN_DISC = 3

# A typical Einstein radius of the lensed-quasar samples the survey draws on
# (Sec. 2.5 item 3: ~5e16 cm for <M> = 1 solar mass); source sizes of
# 5e14-5e16 cm are then 0.01-1 R_E.
R_EIN_CM = 5.0e16


@dataclass(frozen=True)
class Profile:
    """Source brightness profile, lengths in Einstein radii (see the oracle
    header for the formulas).  ``r_out`` is the size (where the brightness
    drops to zero), ``r_in`` a central hole."""
    name: str = "gaussian"
    type: int = PROFILE_GAUSSIAN
    supersample: int = 8
    r_out: float = 0.2
    r_in: float = 0.0
    sigma1: float = 0.05
    sigma2: float = 0.05
    r_scale: float = 0.0
    index: float = 0.0

    def with_(self, **kw) -> "Profile":
        return replace(self, **kw)

    def as_dict(self) -> dict:
        return asdict(self)


def profile_from_cm(kind: str, size_cm: float, r_ein_cm: float = R_EIN_CM,
                    supersample: int = 8) -> Profile:
    """One of the survey's simple profile families with the given size."""
    r = size_cm / r_ein_cm
    if kind == "uniform":
        return Profile(name=kind, type=PROFILE_UNIFORM, supersample=supersample, r_out=r)
    if kind == "gaussian":
        return Profile(name=kind, type=PROFILE_GAUSSIAN, supersample=supersample, r_out=r,
                       sigma1=r / 4, sigma2=r / 4)
    if kind == "gaussian+hole":
        return Profile(name=kind, type=PROFILE_GAUSSIAN, supersample=supersample, r_out=r,
                       r_in=r / 10, sigma1=r / 4, sigma2=r / 4)
    if kind == "power-law":
        return Profile(name=kind, type=PROFILE_POWER_LAW, supersample=supersample, r_out=r,
                       r_in=r / 50, r_scale=r / 10, index=1.5)
    if kind == "thin-disc":
        return Profile(name=kind, type=PROFILE_THIN_DISC, supersample=supersample, r_out=r,
                       r_in=r / 100, r_scale=r / 10)
    raise ValueError(kind)


PROFILE_KINDS = ("uniform", "gaussian", "gaussian+hole", "power-law", "thin-disc")


@dataclass(frozen=True)
class ConvJob:
    """A count map to convolve: npix^2 pixels over ``width`` R_E with mean
    count ``mean_count`` (N_avg times the mean magnification)."""
    name: str
    npix: int
    width: float
    mean_count: float
    seed: int
    profile: Profile

    @property
    def pixel(self) -> float:
        return self.width / self.npix

    def with_(self, **kw) -> "ConvJob":
        return replace(self, **kw)


# GD1-GD3 resolution (Table 3): 10000^2 pixels over 25 R_E; a Gaussian source
# of size 1e16 cm (0.2 R_E, 80 pixels).
CONV_GD1 = ConvJob(name="conv-10000", npix=10000, width=25.0, mean_count=300.0, seed=6,
                   profile=profile_from_cm("gaussian", 1.0e16))
# GD0 resolution: 4096^2 over 24 R_E.
CONV_GD0 = ConvJob(name="conv-4096", npix=4096, width=24.0, mean_count=300.0, seed=7,
                   profile=profile_from_cm("gaussian", 1.0e16))
# small maps the oracle convolves directly in seconds (ragged sizes)
CONV_SMALL = ConvJob(name="conv-200", npix=200, width=0.5, mean_count=300.0, seed=8,
                     profile=profile_from_cm("gaussian", 1.0e15))


def count_map(job: ConvJob, sigma: float = 0.6, rows_per_chunk: int = 512) -> np.ndarray:
    """Seeded synthetic count map (npix, npix) int32: lognormal magnification
    with unit mean times ``mean_count``, stochastically rounded to integers.
    White noise, the hardest case for the round-off of an FFT convolution."""
    n = job.npix
    rng = np.random.default_rng(job.seed)
    out = np.empty((n, n), dtype=np.int32)
    for r0 in range(0, n, rows_per_chunk):
        r1 = min(n, r0 + rows_per_chunk)
        z = rng.standard_normal((r1 - r0, n))
        u = rng.random((r1 - r0, n))
        out[r0:r1] = np.floor(job.mean_count * np.exp(sigma * z - 0.5 * sigma * sigma) + u)
    return out


def log_edges(lo: float, hi: float, n_bins: int) -> np.ndarray:
    """n_bins + 1 float32 edges evenly spaced in log10 between 10^lo and 10^hi."""
    return (10.0 ** np.linspace(lo, hi, n_bins + 1)).astype(np.float32)
