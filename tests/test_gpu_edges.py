"""Edge cases of the CUDA path against the FP64 oracle (GPU).

Bin counts at the group boundaries (1, 3, 4 and the maximum 32 bins), the smallest grid with
the highest multipole, a one-particle catalogue, and particles on or outside the box faces
(periodic wrap).  Same tolerances as the parity tests: 1e-5 relative for the float32 path.
"""
import numpy as np
import pytest

from oracle import zeta_oracle as O
from paper_2507_15209_gb300 import mocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    return zeta


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _sorted_sum(Z, ctx, parts, a, wsum):
    srt, start = ctx.sort_particles(_dev(parts))
    return ctx.sum_particles(srt, start, torch.tensor([wsum], dtype=torch.float64, device="cuda"),
                             _dev(Z.interleave(a))).cpu().numpy()


@pytest.mark.parametrize("staging", [0, 257])
@pytest.mark.parametrize("nb,dsup", [(1, 4), (3, 4), (4, 2), (32, 4)])
def test_particle_sum_bin_counts(Z, nb, dsup, staging):
    # 1-4 bins: one bin group (the copy ring then loads each batch's particles itself);
    # 32 bins: the largest Gram (8 x 8 blocks of 4)
    n, box = 32, 150.0
    edges = np.linspace(4.0, 60.0, nb + 1)
    rng = np.random.default_rng(100 + nb)
    parts = np.empty((4000, 4), np.float32)
    parts[:, :3] = rng.uniform(0, box, (4000, 3))
    parts[:, 3] = rng.uniform(0.5, 2.0, 4000)
    ctx = Z.Context(n, box, dsup, 1, edges, np_max=len(parts), forms=("particle",))
    ctx.set_staging(staging)
    a = rng.standard_normal((nb, n, n, n)).astype(np.float32)
    w = float(parts[:, 3].astype(np.float64).sum())
    got = _sorted_sum(Z, ctx, parts, a, w)
    want = O.sum_particles(a.astype(np.float64), parts[:, :3], parts[:, 3], n, box, dsup)
    assert _rel(got, want) < 1e-5


@pytest.mark.parametrize("nb", [1, 32])
def test_grid_sums_bin_counts(Z, nb):
    n, box, dsup = 16, 100.0, 4
    edges = np.linspace(5.0, 45.0, nb + 1)
    rng = np.random.default_rng(200 + nb)
    ctx = Z.Context(n, box, dsup, 1, edges)
    d = rng.standard_normal((n, n, n)).astype(np.float32)
    a = rng.standard_normal((nb, n, n, n)).astype(np.float32)
    ai = _dev(Z.interleave(a))
    got = ctx.sum_grid(_dev(d), ai, "node").cpu().numpy()
    assert _rel(got, O.sum_node(d.astype(np.float64), a.astype(np.float64))) < 1e-5
    got_g = ctx.sum_grid(_dev(d), ai, "gamma").cpu().numpy()
    assert _rel(got_g, O.sum_gamma(d.astype(np.float64), a.astype(np.float64), dsup)) < 1e-5


def test_smallest_grid_highest_multipole(Z):
    # n = 16 and lmax = 14 (the largest l the library accepts), one radial bin
    n, box, lmax, dsup = 16, 120.0, 14, 4
    edges = np.array([15.0, 45.0])
    parts = mocks.lognormal_catalogue(n, 3000, box, 301, 302)
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=len(parts), forms=("node", "particle"))
    got = ctx.zeta_ell(particles=_dev(parts), forms=("node", "particle"))
    assert ctx.get_status() == 0
    want, _ = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, dsup, forms=("node", "particle"))
    for f in ("node", "particle"):
        g = got[f].cpu().numpy()
        scale = max(np.abs(want[f]).max(), 1e-300)
        for l in range(lmax + 1):
            # odd l vanish up to rounding; compare against the largest multipole
            assert np.abs(g[l] - want[f][l]).max() / scale < 1e-5, (f, l)


def test_one_particle_catalogue(Z):
    n, box, lmax, dsup = 16, 80.0, 2, 4
    edges = np.array([5.0, 15.0, 30.0])
    parts = np.array([[12.3, 40.1, 71.9, 1.5]], np.float32)
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=1, forms=("node", "particle"))
    got = ctx.zeta_ell(particles=_dev(parts), forms=("node", "particle"))
    assert ctx.get_status() == 0
    want, _ = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, dsup, forms=("node", "particle"))
    for f in ("node", "particle"):
        g = got[f].cpu().numpy()
        for l in range(lmax + 1):
            assert _rel(g[l], want[f][l]) < 1e-5, (f, l)


@pytest.mark.parametrize("dsup", [2, 4])
def test_particles_on_and_outside_the_faces(Z, dsup):
    # coordinates exactly on the upper face, just below zero and beyond the box wrap
    # periodically: assignment and interpolation agree with the oracle's modular indices
    n, box, nb = 32, 64.0, 5
    edges = np.linspace(3.0, 25.0, nb + 1)
    rng = np.random.default_rng(7 + dsup)
    parts = np.empty((3000, 4), np.float32)
    parts[:, :3] = rng.uniform(0, box, (3000, 3))
    parts[:, 3] = 1.0
    parts[:100, 0] = box                      # on the face
    parts[100:200, 1] = -1e-3                 # just outside, below
    parts[200:300, 2] = box + 0.37            # beyond the face
    parts[300:400, :3] = 0.0                  # the origin
    ctx = Z.Context(n, box, dsup, 1, edges, np_max=len(parts), forms=("node", "particle"))
    d, wsum = ctx.assign(_dev(parts))
    eps, w = O.assign(parts[:, :3], parts[:, 3], n, box, dsup)
    want_d = eps / (w / n ** 3) - 1.0
    got_d = d.cpu().numpy()
    assert np.abs(got_d - want_d).max() / np.abs(want_d).max() < 1e-5
    a = rng.standard_normal((nb, n, n, n)).astype(np.float32)
    got = _sorted_sum(Z, ctx, parts, a, float(parts[:, 3].astype(np.float64).sum()))
    want = O.sum_particles(a.astype(np.float64), parts[:, :3], parts[:, 3], n, box, dsup)
    assert _rel(got, want) < 1e-5
