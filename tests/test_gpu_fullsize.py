"""Parity at full workload sizes, in the launch configuration the benchmark times.

256^3 (2M log-normal particles, lmax 10, 15 bins, cubic B-spline): the assignment on every
cell, the fields of one (l, m) on every cell for three bins, zeta_0 of the node form from the
whole measurement, and the particle sum of l = 0 (without its mass term, which the small
cases pin), all against the FP64 oracle.
512^3 (16M particles, lmax 10, 20 bins): the assignment at sampled cells (the oracle sums the
particles near each sampled cell), and properties that hold at any size: finiteness,
symmetry in (b1, b2), and invariance under a whole-cell translation of the catalogue.
"""
import numpy as np
import pytest

from oracle import zeta_oracle as O
from paper_2507_15209_gb300 import mocks
from paper_2507_15209_gb300.workloads import WORKLOADS, edges as wl_edges

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_fullsize_256(Z):
    w = WORKLOADS["box1000_n256_np2m"]
    n, box, lmax, dsup = w["n"], w["box"], w["lmax"], w["dsup"]
    e = wl_edges(w)
    nb = len(e) - 1
    parts = mocks.lognormal_catalogue(n, w["n_p"], box, w["field_seed"], w["sample_seed"])
    ctx = Z.Context(n, box, dsup, lmax, e, np_max=len(parts), forms=("particle", "node"))
    pd = torch.from_numpy(parts).cuda()
    # assignment, every cell
    delta, wsum = ctx.assign(pd)
    eps, wtot = O.assign(parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64), n, box, dsup)
    d64 = O.contrast(eps, wtot)
    assert np.abs(delta.cpu().numpy() - d64).max() < 2e-6 * np.abs(d64).max()
    # one (l, m): every cell of three bins
    dh = np.fft.fftn(d64)
    dhat = ctx.fft_r2c(delta)
    l, m, bins = 7, -3, [0, 7, 14]
    got = Z.deinterleave(ctx.reconstruct_alm(dhat, l, m).cpu().numpy(), nb)
    want = O.multipole_fields(dh, l, m, n, box, e, bins=bins)
    for i, b in enumerate(bins):
        err = np.abs(got[b] - want[i]).max() / np.abs(want[i]).max()
        assert err < 2e-5, (b, err)
    # zeta_0 of the node form from the whole measurement; the l = 0 particle sum
    z = ctx.zeta_ell(particles=pd, forms=("particle", "node"))
    assert ctx.get_status() == 0
    a0 = O.multipole_fields(dh, 0, 0, n, box, e)
    zn = O.sum_node(d64, a0)
    assert _rel(z["node"][0].cpu().numpy(), 0.5 * (zn + zn.T)) < 1e-5
    srt, start = ctx.sort_particles(pd)
    a0_gpu = ctx.reconstruct_alm(dhat, 0, 0)
    pg = ctx.sum_particles(srt, start, wsum, a0_gpu).cpu().numpy()
    pos, ww = parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64)
    assert _rel(pg, O.sum_particles(a0, pos, ww, n, box, dsup)) < 1e-5


def test_fullsize_512_sampled_and_properties(Z):
    w = WORKLOADS["box2000_n512_np16m"]
    n, box, lmax, dsup = w["n"], w["box"], w["lmax"], w["dsup"]
    e = wl_edges(w)
    parts = mocks.lognormal_catalogue(n, w["n_p"], box, w["field_seed"], w["sample_seed"])
    ctx = Z.Context(n, box, dsup, lmax, e, np_max=len(parts), forms=("particle", "node"))
    pd = torch.from_numpy(parts).cuda()
    delta, wsum = ctx.assign(pd)
    dgpu = delta.cpu().numpy()
    # sampled cells: the oracle's B-spline sum over the particles within the stencil reach
    rng = np.random.default_rng(5)
    cells = rng.integers(0, n, (24, 3))
    u = parts[:, :3].astype(np.float64) * (n / box)
    wtot = float(parts[:, 3].astype(np.float64).sum())
    for cz, cy, cx in cells:
        dd = (u - np.array([cx, cy, cz]) + n / 2) % n - n / 2  # periodic offset in cells
        near = np.all(np.abs(dd) < 2.0, axis=1)
        eps = float(np.sum(parts[near, 3] * np.prod(O.bspline(dd[near], dsup), axis=1)))
        want = eps / (wtot / n ** 3) - 1.0
        assert abs(dgpu[cz, cy, cx] - want) < 2e-6 * max(1.0, abs(want)), (cz, cy, cx)
    z = ctx.zeta_ell(particles=pd, forms=("particle", "node"))
    assert ctx.get_status() == 0
    zz = {f: v.cpu().numpy() for f, v in z.items()}
    for f, v in zz.items():
        assert np.all(np.isfinite(v))
        np.testing.assert_array_equal(v, np.swapaxes(v, 1, 2))
    # translate every particle by whole cells: zeta is invariant (float32 rounding differs)
    shifted = parts.copy()
    h = box / n
    shifted[:, :3] = ((parts[:, :3].astype(np.float64) + h * np.array([37, 5, 300])) % box).astype(np.float32)
    shifted[:, :3][shifted[:, :3] >= np.float32(box)] -= np.float32(box)
    z2 = ctx.zeta_ell(particles=torch.from_numpy(shifted).cuda(), forms=("particle", "node"))
    for f in zz:
        v2 = z2[f].cpu().numpy()
        for l in range(lmax + 1):
            assert _rel(v2[l], zz[f][l]) < 1e-4, (f, l)
