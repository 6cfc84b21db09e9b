"""Parity at full workload sizes, in the launch configuration the benchmark times.

256^3 (2M log-normal particles, lmax 10, 15 bins, cubic B-spline): the assignment on every
cell, the fields of one (l, m) on every cell for three bins, zeta_0 of the node form from the
whole measurement, and the particle sum of l = 0, all against the FP64 oracle.
512^3 (16M particles, lmax 10, 20 bins; the benchmark's workload):
  * the assignment at sampled cells (the oracle sums the particles near each sampled cell);
  * the fields of two (l, m), one with odd l, on every cell of three bins;
  * for one (l, m): the node-form Gram over all 20 bins, the particle sum over the particles of
    a 32-cell slab (about 1M particles at the workload's density, so tile batches are as full
    as in the benchmark), and the uniform term of that l;
  * properties that hold at any size: finiteness, symmetry in (b1, b2), and invariance under a
    whole-cell translation of the catalogue.
Stage inputs are the library's own float32 outputs of the previous stage (widened to float64),
so each comparison measures one stage's arithmetic.  Field tolerance: max |a_gpu - a_oracle| <=
1e-5 max |a_oracle| per bin; sums: relative Frobenius 1e-5.
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
    # one (l, m): every cell of three bins, from the library's own delta (stage parity)
    dh = np.fft.fftn(d64)
    dhat = ctx.fft_r2c(delta)
    l, m, bins = 7, -3, [0, 7, 14]
    got = Z.deinterleave(ctx.reconstruct_alm(dhat, l, m).cpu().numpy(), nb)
    want = O.multipole_fields(np.fft.fftn(delta.cpu().numpy().astype(np.float64)), l, m, n, box, e, bins=bins)
    for i, b in enumerate(bins):
        err = np.abs(got[b] - want[i]).max() / np.abs(want[i]).max()
        print(f"256^3 field (l={l}, m={m}, b={b}): max-relative error {err:.2e}")
        assert err < 1e-5, (b, err)
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


@pytest.fixture(scope="module")
def big(Z):
    """The 512^3 workload: context, catalogue, delta and delta_hat on the device."""
    w = WORKLOADS["box2000_n512_np16m"]
    e = wl_edges(w)
    parts = mocks.lognormal_catalogue(w["n"], w["n_p"], w["box"], w["field_seed"], w["sample_seed"])
    ctx = Z.Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=len(parts), forms=("particle", "node"))
    pd = torch.from_numpy(parts).cuda()
    delta, wsum = ctx.assign(pd)
    dhat = ctx.fft_r2c(delta)
    d64 = delta.cpu().numpy().astype(np.float64)
    yield dict(w=w, e=e, parts=parts, ctx=ctx, pd=pd, delta=delta, wsum=wsum, dhat=dhat, d64=d64,
               dh64=np.fft.fftn(d64))
    ctx.close()


@pytest.mark.parametrize("l,m", [(4, 3), (7, -5)])
def test_fullsize_512_fields(Z, big, l, m):
    w, e, ctx = big["w"], big["e"], big["ctx"]
    nb = len(e) - 1
    bins = [0, 9, 19]
    got = Z.deinterleave(ctx.reconstruct_alm(big["dhat"], l, m).cpu().numpy(), nb)
    wants = O.multipole_fields(big["dh64"], l, m, w["n"], w["box"], e, bins=bins)
    for b, want in zip(bins, wants):
        err = np.abs(got[b] - want).max() / np.abs(want).max()
        print(f"512^3 field (l={l}, m={m}, b={b}): max-relative error {err:.2e}")
        assert err < 1e-5, (l, m, b, err)


def test_fullsize_512_sums_one_lm(Z, big):
    w, e, ctx = big["w"], big["e"], big["ctx"]
    n, box, dsup = w["n"], w["box"], w["dsup"]
    nb = len(e) - 1
    l, m = 7, -5
    alm = ctx.reconstruct_alm(big["dhat"], l, m)
    a64 = Z.deinterleave(alm.cpu().numpy(), nb).astype(np.float64)
    # node form, all 20 bins
    got = ctx.sum_grid(big["delta"], alm, "node").cpu().numpy()
    want = O.sum_node(big["d64"], a64)
    want = 0.5 * (want + want.T)
    print(f"512^3 node Gram (l={l}, m={m}): rel {_rel(got, want):.2e}")
    assert _rel(got, want) < 1e-5
    # particle form over a 32-cell slab of the catalogue (the workload's density and tile fill)
    parts = big["parts"]
    slab = parts[parts[:, 2] < np.float32(32 * box / n)]
    sd = torch.from_numpy(np.ascontiguousarray(slab)).cuda()
    srt, start = ctx.sort_particles(sd)
    wsum = torch.tensor([float(slab[:, 3].astype(np.float64).sum())], dtype=torch.float64, device="cuda")
    got = ctx.sum_particles(srt, start, wsum, alm).cpu().numpy()
    want = O.sum_particles(a64, slab[:, :3].astype(np.float64), slab[:, 3].astype(np.float64), n, box, dsup)
    want = 0.5 * (want + want.T)
    print(f"512^3 particle sum (l={l}, m={m}, {len(slab)} particles): rel {_rel(got, want):.2e}")
    assert _rel(got, want) < 1e-5
    # the uniform term of this l, three bins
    bins = [0, 9, 19]
    got = ctx.mass_term(big["dhat"], l).cpu().numpy()[np.ix_(bins, bins)]
    want = O.mass_term_fourier(big["dh64"], l, n, box, e, dsup, bins=bins)
    print(f"512^3 uniform term (l={l}): rel {_rel(got, want):.2e}")
    assert _rel(got, want) < 1e-5


def test_fullsize_512_sampled_and_properties(Z, big):
    w = big["w"]
    n, box, lmax, dsup = w["n"], w["box"], w["lmax"], w["dsup"]
    parts, ctx, pd = big["parts"], big["ctx"], big["pd"]
    dgpu = big["delta"].cpu().numpy()
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
