"""Shared test problems: seeded synthetic inputs (paper_2103_01767_gb300.synth) with
measurements computed by the FP64 oracle, rounded to the FP32/complex64 precision the CUDA
path stores so that both sides see identical inputs."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle
from paper_2103_01767_gb300 import synth


@dataclass
class Case:
    n: int
    m: int
    pos: np.ndarray          # int32 [K, 2]
    O_true: np.ndarray       # complex128 (complex64-rounded)
    P: np.ndarray            # complex128 (complex64-rounded)
    y: np.ndarray            # float64 (float32-rounded) [K, m, m]
    loss: int
    b: float

    @property
    def K(self):
        return self.pos.shape[0]

    def problem(self):
        return oracle.Problem((self.n, self.n), self.P, self.pos, self.y, self.loss, self.b)


def random_positions(n, m, K, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n - m + 1, size=(K, 2)).astype(np.int32)


def make_case(n, m, K=None, loss=0, peak=0.0, seed=0, grid=None, step=None, jitter=0, radius=None,
              b=1e-8, noisy=True):
    """A problem on an n^2 object with an m^2 probe.  Positions come from a jittered raster
    (grid/step given) or are uniform random (K given).  peak > 0 scales the probe so the
    brightest noiseless pixel holds `peak` photons; then y are Poisson counts (noisy) or the
    expected counts themselves (noisy=False)."""
    O_true = synth.to_c64(synth.object_texture(n, seed=seed))
    P = synth.probe_disk_defocus(m, radius if radius is not None else 0.3125 * m)
    if grid is not None:
        pos, _ = synth.raster_positions(n, m, grid, step, jitter, seed=seed + 1)
    else:
        pos = random_positions(n, m, K, seed + 1)
    P = synth.to_c64(P)
    pb = oracle.Problem((n, n), P, pos, None, loss, b)
    h = oracle.intensity(pb, O_true)
    if peak > 0:
        P = synth.to_c64(P * np.sqrt(peak / h.max()))
        pb = oracle.Problem((n, n), P, pos, None, loss, b)
        h = oracle.intensity(pb, O_true)
        y = synth.poisson_counts(h, seed=seed + 2) if noisy else h
    else:
        y = h
    return Case(n, m, pos, O_true, P, synth.to_f32(y), loss, b)


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
