"""Seeded synthetic catalogues (log-normal mocks) shared by the tests, the
benchmark and the smoke check.

This module holds none of the 3PCF method's arithmetic: it only draws inputs.
The recipe stands in for the N-body snapshot the paper measures on (MDPL2,
Sec. 3): a Gaussian random field with a power-law spectrum P(k) = A k^-1.5
scaled to unit variance, a log-normal density rho = exp(G - 1/2), and exactly
N_p particles drawn cell by cell in proportion to rho, uniform inside their
cell, all of weight 1.  Every array is produced by numpy's PCG64 from an
explicit seed, so the CUDA path and the FP64 oracle see bit-identical inputs.

Array conventions used throughout the project:
  * grids are indexed [z][y][x] (x fastest), side n, cell size H = box / n;
  * a particle is a float32 quadruple (x, y, z, w) in box units, with every
    coordinate in [0, box).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_field",
    "lognormal_density",
    "sample_particles",
    "uniform_particles",
    "lognormal_catalogue",
    "batch_sizes",
    "loss_weights",
]


def gaussian_field(n: int, seed: int, slope: float = -1.5) -> np.ndarray:
    """Unit-variance Gaussian random field on an n^3 grid, P(k) ~ k^slope, k=0 removed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    del white
    iz = np.fft.fftfreq(n, 1.0 / n)
    ix = np.fft.rfftfreq(n, 1.0 / n)
    k2 = iz[:, None, None] ** 2 + iz[None, :, None] ** 2 + ix[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)  # sqrt(P) with P ~ |k|^slope
    amp[0, 0, 0] = 0.0
    wk *= amp
    del amp, k2
    g = np.fft.irfftn(wk, s=(n, n, n), axes=(0, 1, 2))
    del wk
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_density(n: int, seed: int) -> np.ndarray:
    """rho = exp(G - 1/2) with G the unit-variance field above (mean of rho is ~1)."""
    g = gaussian_field(n, seed)
    np.subtract(g, 0.5, out=g)
    np.exp(g, out=g)
    return g


def _to_float32_positions(pos: np.ndarray, box: float) -> np.ndarray:
    p = pos.astype(np.float32)
    # float32 rounding can push a coordinate onto the upper face; wrap it back.
    p[p >= np.float32(box)] -= np.float32(box)
    p[p < 0] += np.float32(box)
    p[p >= np.float32(box)] = 0.0
    return p


def sample_particles(rho: np.ndarray, n_p: int, box: float, seed: int) -> np.ndarray:
    """Draw exactly n_p particles: cells categorically in proportion to rho, uniform inside.

    Returns float32 array (n_p, 4) of (x, y, z, w=1).
    """
    n = rho.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    cdf = np.cumsum(rho.ravel(), dtype=np.float64)
    u = rng.random(n_p) * cdf[-1]
    cells = np.searchsorted(cdf, u, side="right")
    del cdf, u
    cells = np.minimum(cells, n ** 3 - 1)
    iz, rem = np.divmod(cells, n * n)
    iy, ix = np.divmod(rem, n)
    off = rng.random((n_p, 3))
    h = box / n
    out = np.empty((n_p, 4), np.float32)
    out[:, 0] = _to_float32_positions((ix + off[:, 0]) * h, box)
    out[:, 1] = _to_float32_positions((iy + off[:, 1]) * h, box)
    out[:, 2] = _to_float32_positions((iz + off[:, 2]) * h, box)
    out[:, 3] = 1.0
    return out


def uniform_particles(n_p: int, box: float, seed: int) -> np.ndarray:
    """Poisson (uniform) catalogue of n_p unit-weight particles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n_p, 4), np.float32)
    out[:, :3] = _to_float32_positions(rng.random((n_p, 3)) * box, box)
    out[:, 3] = 1.0
    return out


def lognormal_catalogue(n: int, n_p: int, box: float, field_seed: int, sample_seed: int) -> np.ndarray:
    """Log-normal mock catalogue on an n^3 density grid (float32 (n_p, 4))."""
    rho = lognormal_density(n, field_seed)
    return sample_particles(rho, n_p, box, sample_seed)


def loss_weights(lmax: int, nbins: int, seed: int) -> np.ndarray:
    """Gaussian weights w[l, i, j] of the scalar loss L = sum w * zeta_l(r_i, r_j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((lmax + 1, nbins, nbins))


def batch_sizes(n_cat: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Per-catalogue particle counts drawn uniformly from the integers [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_cat, dtype=np.int64)
