"""Seeded synthetic inputs shaped like the paper's ptychography workloads.

This module only draws inputs: textured complex objects, disk probes with a defocus
phase, jittered raster scans, Poisson counts from given expected intensities, and random
test vectors.  It contains none of the reconstruction method's arithmetic (no Fourier
propagation, no error metric, no derivative), so both the CUDA path and the CPU oracle can
take their inputs from it.

Workload recipe (matching the paper's far-field simulations of Sec. 5 in structure):
  * object: amplitude in [0.8, 1] and phase in [-pi/4, pi/4], each an independent
    N(0,1) field smoothed by a periodic Gaussian filter (sigma = 3 px) and min-max mapped;
  * probe: hard-edged disk of radius R centred at ((m-1)/2, (m-1)/2) with a quadratic
    phase reaching pi at the edge (a defocused aperture);
  * positions: a raster of integer shifts, step s, optional seeded +-J jitter, clamped so
    every patch lies inside the object (a requested step that overflows is reduced);
  * measurements: Poisson counts drawn from the noiseless expected intensities that the
    caller computes with its own forward model.
Seeds: object 0, probe/jitter 1, noise 2, initial guess / test vectors 3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    n: int          # object side (pixels)
    m: int          # probe / detector side (pixels)
    grid: int       # raster points per side
    step: int       # requested raster step
    jitter: int     # +- integer jitter (px)
    radius: float   # probe disk radius (px)
    loss: int       # 0 Gaussian (amplitude), 1 Poisson
    peak: float     # peak expected photons per pattern (0 = noiseless, unscaled probe)
    joint: bool     # object + probe problem

    @property
    def K(self):
        return self.grid * self.grid


# The three single-reconstruction workloads.
SMALL = Workload("obj128_probe32_pos64_amplitude_noiseless", 128, 32, 8, 8, 0, 10.0, 0, 0.0, False)
MEDIUM = Workload("obj256_probe64_pos400_poisson_1e4", 256, 64, 20, 10, 2, 20.0, 1, 1e4, True)
LARGE = Workload("obj1024_probe128_pos3600_poisson_1e3", 1024, 128, 60, 16, 2, 40.0, 1, 1e3, False)
WORKLOADS = {w.name: w for w in (SMALL, MEDIUM, LARGE)}


def _smooth_periodic(field: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(field, sigma=sigma, mode="wrap")


def _minmax(a: np.ndarray, lo: float, hi: float) -> np.ndarray:
    a = a - a.min()
    a = a / a.max()
    return lo + (hi - lo) * a


def object_texture(n: int, seed: int = 0, sigma: float = 3.0) -> np.ndarray:
    """Complex object [n, n] (complex128): amp in [0.8, 1], phase in [-pi/4, pi/4]."""
    rng = np.random.default_rng(seed)
    amp = _minmax(_smooth_periodic(rng.standard_normal((n, n)), sigma), 0.8, 1.0)
    ph = _minmax(_smooth_periodic(rng.standard_normal((n, n)), sigma), -math.pi / 4, math.pi / 4)
    return amp * np.exp(1j * ph)


def probe_disk_defocus(m: int, radius: float, amplitude: float = 1.0, phased: bool = True) -> np.ndarray:
    """Disk of ``radius`` px with a quadratic phase of pi at the edge (complex128 [m, m])."""
    c = (m - 1) / 2.0
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64)
    r = np.hypot(yy - c, xx - c)
    disk = (r <= radius).astype(np.float64)
    phase = math.pi * (r / radius) ** 2 if phased else 0.0 * r
    return amplitude * disk * np.exp(1j * phase)


def raster_positions(n: int, m: int, grid: int, step: int, jitter: int = 0, seed: int = 1):
    """int32 [grid*grid, 2] top-left (row, col) corners of a centred, jittered raster.

    The step is reduced to floor((n - m - 2 J) / (grid - 1)) when the requested one would
    carry patches outside the object; positions are clamped to [0, n - m].
    Returns (positions, step_used).
    """
    span = n - m
    if span < 0:
        raise ValueError("probe larger than object")
    s = step
    if grid > 1:
        s = min(step, max((span - 2 * jitter) // (grid - 1), 0))
    extent = s * (grid - 1)
    off = (span - extent) // 2
    rng = np.random.default_rng(seed)
    pos = np.empty((grid * grid, 2), np.int64)
    k = 0
    for i in range(grid):
        for j in range(grid):
            pos[k] = (off + i * s, off + j * s)
            k += 1
    if jitter:
        pos += rng.integers(-jitter, jitter + 1, size=pos.shape)
    pos = np.clip(pos, 0, span)
    return pos.astype(np.int32), s


def poisson_counts(h: np.ndarray, seed: int = 2) -> np.ndarray:
    """Photon counts y ~ Poisson(h) as float64 (same shape as h)."""
    rng = np.random.default_rng(seed)
    return rng.poisson(np.asarray(h, dtype=np.float64)).astype(np.float64)


def flat_object(n: int) -> np.ndarray:
    return np.ones((n, n), np.complex128)


def random_complex(shape, seed: int = 3, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def random_real(shape, seed: int = 3, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def to_c64(a: np.ndarray) -> np.ndarray:
    """Round to complex64 (what the CUDA path stores) and back to complex128, so that both
    sides of a comparison see identical inputs."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def to_f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a).astype(np.float32).astype(np.float64)


def illumination_mask(n: int, probe: np.ndarray, positions: np.ndarray, frac: float = 0.1):
    """Boolean [n, n] mask of pixels whose summed probe intensity >= frac * max.
    (A bookkeeping aid for error metrics; it sums |P|^2 over patch footprints.)"""
    acc = np.zeros((n, n))
    p2 = np.abs(probe) ** 2
    m0, m1 = probe.shape
    for r, c in positions:
        acc[r:r + m0, c:c + m1] += p2
    return acc >= frac * acc.max()


# ---------------------------------------------------------------------------------------
# Batches of independent reconstructions of uneven sizes
# ---------------------------------------------------------------------------------------
@dataclass(frozen=True)
class BatchMember:
    n: int          # object side
    m: int          # probe side (32, 64 or 128)
    K: int          # scan positions
    loss: int       # 0 Gaussian (noiseless data), 1 Poisson (counts at `peak`)
    peak: float
    seed: int

    @property
    def radius(self):
        return 0.3125 * self.m


def batch_members(B: int = 64, seed: int = 7, n_range=(128, 512), K_range=(64, 1024)):
    """B problems drawn uniformly: probe side from {32, 64, 128}, object side from
    [max(n_lo, 2 m), n_hi] (so N >= 2 x probe), K from K_range, loss Gaussian or Poisson
    (peak 1e3 photons)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(B):
        m = int(rng.choice([32, 64, 128]))
        n = int(rng.integers(max(n_range[0], 2 * m), n_range[1] + 1))
        K = int(rng.integers(K_range[0], K_range[1] + 1))
        loss = int(rng.integers(0, 2))
        out.append(BatchMember(n, m, K, loss, 1e3 if loss else 0.0, 1000 * seed + b))
    return out


def batch_positions(mem: BatchMember, jitter: int = 2):
    """The first K points of a ceil(sqrt K)^2 jittered raster with step m / 4 (reduced to
    fit the object)."""
    g = int(math.ceil(math.sqrt(mem.K)))
    pos, _ = raster_positions(mem.n, mem.m, g, max(1, mem.m // 4), jitter, seed=mem.seed + 1)
    return np.ascontiguousarray(pos[:mem.K])


BATCH64 = "batch64_obj128-512_probe32-128_pos64-1024_mixed"
