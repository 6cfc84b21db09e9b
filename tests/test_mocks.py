"""The seeded input recipe (it stands in for the paper's N-body snapshot): the properties the
design states for the mock generators and the named workloads.  CPU only."""
import math

import numpy as np

from paper_2507_15209_gb300 import mocks
from paper_2507_15209_gb300.workloads import WORKLOADS, batch_seeds, edges


def test_gaussian_field_is_unit_variance_with_the_stated_slope():
    n = 32
    g = mocks.gaussian_field(n, 7)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    np.testing.assert_array_equal(g, mocks.gaussian_field(n, 7))
    assert not np.array_equal(g, mocks.gaussian_field(n, 8))
    # shell-averaged power against |k| on a 64^3 field: log-log slope of P(k) ~ k^-1.5
    m = 64
    pk = np.abs(np.fft.fftn(mocks.gaussian_field(m, 7))) ** 2
    f = np.fft.fftfreq(m, 1.0 / m)
    kk = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    shells = np.arange(4, 25)
    p = np.array([pk[(kk >= s - 0.5) & (kk < s + 0.5)].mean() for s in shells])
    slope = np.polyfit(np.log(shells), np.log(p), 1)[0]
    assert abs(slope + 1.5) < 0.08, slope
    assert pk[0, 0, 0] < 1e-20 * pk.sum()  # k = 0 removed


def test_lognormal_density_is_positive_with_unit_mean():
    rho = mocks.lognormal_density(32, 11)
    assert np.all(rho > 0)
    assert abs(rho.mean() - 1.0) < 0.1
    np.testing.assert_allclose(np.log(rho), mocks.gaussian_field(32, 11) - 0.5, rtol=0, atol=1e-12)


def test_sampled_particles_follow_the_density():
    n, n_p, box = 16, 200_000, 100.0
    rho = mocks.lognormal_density(n, 21)
    p = mocks.sample_particles(rho, n_p, box, 22)
    assert p.dtype == np.float32 and p.shape == (n_p, 4)
    assert np.all(p[:, :3] >= 0) and np.all(p[:, :3] < np.float32(box))
    assert np.all(p[:, 3] == 1.0)
    cell = np.floor(p[:, :3].astype(np.float64) * (n / box)).astype(np.int64) % n
    counts = np.bincount((cell[:, 2] * n + cell[:, 1]) * n + cell[:, 0], minlength=n ** 3)
    expect = rho.ravel() / rho.sum() * n_p
    assert np.corrcoef(counts, expect)[0, 1] > 0.95
    np.testing.assert_array_equal(p, mocks.sample_particles(rho, n_p, box, 22))


def test_uniform_particles_and_batch_sizes():
    p = mocks.uniform_particles(50_000, 80.0, 3)
    assert p.dtype == np.float32 and np.all(p[:, :3] >= 0) and np.all(p[:, :3] < np.float32(80.0))
    assert np.all(p[:, 3] == 1.0)
    assert abs(p[:, :3].astype(np.float64).mean() - 40.0) < 0.5
    s = mocks.batch_sizes(64, 500_000, 4_000_000, 4999)
    assert s.dtype == np.int64 and s.min() >= 500_000 and s.max() <= 4_000_000
    assert len({batch_seeds(i) for i in range(64)}) == 64


def test_named_workloads_are_consistent():
    for name, w in WORKLOADS.items():
        e = edges(w)
        assert len(e) == w["nbins"] + 1 and np.all(np.diff(e) > 0) and e[0] > 0
        assert e[-1] < w["box"] / 2, name  # the library requires r_hi < L/2
        assert w["n"] & (w["n"] - 1) == 0 and w["dsup"] in (2, 4) and w["lmax"] <= 14
    big = WORKLOADS["box2000_n512_np16m"]
    np.testing.assert_allclose(np.diff(edges(big)), 9.75)
    assert (big["n"], big["n_p"], big["lmax"], big["nbins"], big["dsup"]) == (512, 16_000_000, 10, 20, 4)
    # particles per grid cell across the workloads: 0.03 (smallest batched catalogue) to 0.24
    ratios = [w["n_p"] / w["n"] ** 3 for w in WORKLOADS.values() if "n_p" in w]
    b = WORKLOADS["batch64_n256"]
    ratios += [b["n_p_lo"] / b["n"] ** 3, b["n_p_hi"] / b["n"] ** 3]
    assert math.isclose(min(ratios), 0.0298, abs_tol=1e-3) and math.isclose(max(ratios), 0.238, abs_tol=1e-3)
