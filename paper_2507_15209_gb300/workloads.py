"""Named workloads: grid, catalogue and binning parameters plus the seeds that
make each one reproducible.  Pure data; no arithmetic of the method.

Bins are linear in r between r_lo and r_hi (nbins of them, edges inclusive of
r_lo, exclusive of r_hi).  `dsup` is the support D of the centred B-spline
scaling function (2: linear hat, 4: cubic).
"""
from __future__ import annotations

import numpy as np

WORKLOADS = {
    # small plain-method case: every summation form, plus a uniform null catalogue
    "box500_n64_np20k": dict(
        box=500.0, n=64, n_p=20_000, lmax=4, nbins=8, r_lo=10.0, r_hi=90.0, dsup=2,
        field_seed=1001, sample_seed=1002, null_seed=1003,
        summation=("gamma", "particle", "node"),
    ),
    # FP32 GPU path, particle summation
    "box1000_n256_np2m": dict(
        box=1000.0, n=256, n_p=2_000_000, lmax=10, nbins=15, r_lo=5.0, r_hi=150.0, dsup=4,
        field_seed=2001, sample_seed=2002, summation=("particle",),
    ),
    # 512^3 precision study; the headline timing workload
    "box2000_n512_np16m": dict(
        box=2000.0, n=512, n_p=16_000_000, lmax=10, nbins=20, r_lo=5.0, r_hi=200.0, dsup=4,
        field_seed=3001, sample_seed=3002, summation=("particle", "node"),
    ),
    # 64 catalogues of uneven size in one batched call
    "batch64_n256": dict(
        box=1000.0, n=256, n_cat=64, n_p_lo=500_000, n_p_hi=4_000_000, lmax=8, nbins=12,
        r_lo=10.0, r_hi=130.0, dsup=4, size_seed=4999, summation=("particle",),
    ),
    # adjoint workload: density grid + particles, Gaussian loss weights
    "adjoint_n256_np1m": dict(
        box=1000.0, n=256, n_p=1_000_000, lmax=6, nbins=10, r_lo=10.0, r_hi=110.0, dsup=4,
        field_seed=5001, sample_seed=5002, loss_seed=5003, summation=("node", "particle"),
    ),
}


def edges(w: dict) -> np.ndarray:
    """Bin edges (nbins+1,) in box units."""
    return np.linspace(w["r_lo"], w["r_hi"], w["nbins"] + 1)


def batch_seeds(i: int) -> tuple[int, int]:
    """(field seed, sampling seed) of catalogue i of the batched workload."""
    return 4000 + 2 * i, 4001 + 2 * i
