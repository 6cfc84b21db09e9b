"""Batched measurement (zeta_batch, one CUDA-graph launch for many catalogues of uneven
size) and the persistent-grid autotuner, on the GPU."""
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


def _cats(n, box, sizes, seed0):
    return [mocks.lognormal_catalogue(n, int(s), box, seed0 + 2 * i, seed0 + 2 * i + 1) for i, s in enumerate(sizes)]


def test_batch_equals_one_by_one_and_replays(Z):
    n, box, lmax, dsup = 32, 200.0, 3, 4
    edges = np.linspace(10.0, 70.0, 6)
    sizes = mocks.batch_sizes(5, 800, 9000, 77)
    cats = _cats(n, box, sizes, 500)
    allp = np.concatenate(cats)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    forms = ("node", "particle")
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=int(sizes.max()), forms=forms)
    dev = torch.from_numpy(allp).to("cuda")
    out = ctx.batch(dev, offs, forms=forms)
    again = ctx.batch(dev, offs, forms=forms, out=out.clone())  # new output pointer: re-captured
    replay = ctx.batch(dev, offs, forms=forms, out=out)          # same key: cached graph relaunched
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    for i, p in enumerate(cats):
        one = ctx.zeta_ell(particles=torch.from_numpy(p).to("cuda"), forms=forms)
        for k, f in enumerate(("node", "particle")):
            np.testing.assert_array_equal(out[i, k].cpu().numpy(), one[f].cpu().numpy())
            np.testing.assert_array_equal(again[i, k].cpu().numpy(), one[f].cpu().numpy())
    # the first catalogue against the FP64 oracle
    want, _ = O.zeta_multipoles(cats[0].astype(np.float64), n, box, edges, lmax, dsup, forms=forms)
    for k, f in enumerate(("node", "particle")):
        got = replay[0, k].cpu().numpy()
        for l in range(lmax + 1):
            err = np.linalg.norm(got[l] - want[f][l]) / np.linalg.norm(want[f][l])
            assert err < 1e-5, (f, l, err)


@pytest.mark.parametrize("copies", [2, 3])
def test_concurrent_batch_equals_one_by_one(Z, copies):
    """With room for several per-catalogue workspaces the batch graph runs catalogues on forked
    streams; every catalogue's result is still bit-identical to zeta_ell's."""
    n, box, lmax, dsup = 32, 200.0, 3, 4
    edges = np.linspace(10.0, 70.0, 6)
    sizes = mocks.batch_sizes(7, 800, 9000, 78)
    cats = _cats(n, box, sizes, 700)
    allp = torch.from_numpy(np.concatenate(cats)).to("cuda")
    offs = np.concatenate([[0], np.cumsum(sizes)])
    forms = ("node", "particle")
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=int(sizes.max()), forms=forms, ws_copies=copies)
    out = ctx.batch(allp, offs, forms=forms)
    replay = ctx.batch(allp, offs, forms=forms, out=out.clone())
    torch.cuda.synchronize()
    assert ctx.get_status() == 0
    for i, p in enumerate(cats):
        one = ctx.zeta_ell(particles=torch.from_numpy(p).to("cuda"), forms=forms)
        for k, f in enumerate(forms):
            np.testing.assert_array_equal(out[i, k].cpu().numpy(), one[f].cpu().numpy())
            np.testing.assert_array_equal(replay[i, k].cpu().numpy(), one[f].cpu().numpy())
    ctx.close()


def test_autotune_keeps_results(Z):
    n, box, lmax, dsup = 32, 200.0, 2, 4
    edges = np.linspace(10.0, 70.0, 5)
    p = torch.from_numpy(mocks.lognormal_catalogue(n, 20000, box, 91, 92)).to("cuda")
    forms = ("node", "particle")
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=20000, forms=forms)
    before = {f: v.cpu().numpy() for f, v in ctx.zeta_ell(particles=p, forms=forms).items()}
    tune = ctx.autotune(p, forms=forms)
    assert len(tune) == 5 and all(1 <= t <= 8 for t in tune)
    after = {f: v.cpu().numpy() for f, v in ctx.zeta_ell(particles=p, forms=forms).items()}
    # the grid partition among CTAs and, for the particle form, the staging threshold (which
    # kernel interpolates each batch, so the float32 summation order) changed: rounding-level
    # differences only
    for f in forms:
        np.testing.assert_allclose(after[f], before[f], rtol=1e-6, atol=1e-9 * np.abs(before[f]).max())


def test_tuning_roundtrip_and_validation(Z):
    ctx = Z.Context(32, 200.0, 4, 1, np.linspace(10.0, 70.0, 5), np_max=1000, forms=("particle",))
    ctx.set_tuning([3, 2, 5, 1, 7])
    assert ctx.tuning() == [3, 2, 5, 1, 7]
    lib = Z.lib()
    bad = np.array([1, 0, 1, 1, 1], np.int32)
    assert lib.zeta_set_tuning(ctx._h, bad.ctypes.data, 5) == -1
    assert lib.zeta_set_tuning(ctx._h, bad.ctypes.data, 6) == -1
    assert ctx.tuning() == [3, 2, 5, 1, 7]  # unchanged after a rejected call
    assert lib.zeta_set_staging(ctx._h, -1) == -1
    ctx.set_staging(40)
    assert ctx.staging() == 40


@pytest.mark.parametrize("n", [16, 64])
def test_every_tile_shape_gives_the_fields_and_zeta(Z, n):
    """The tile shapes of the three reconstruction passes (zeta_set_shapes) only move columns
    between threads: every combination gives the oracle's fields of one (l, m) and zeta_l within
    the float32 bound, and the same zeta_l as the default shapes to float32 rounding."""
    box, lmax, dsup = 4.0 * n, 2, 4
    edges = np.linspace(2.5 * box / n, 0.4 * box, 5)
    parts = mocks.lognormal_catalogue(n, 3 * n ** 3 // 16, box, 90 + n, 91 + n)
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=len(parts), forms=("node", "particle"))
    pd = torch.from_numpy(parts).cuda()
    d, _ = ctx.assign(pd)
    dh = ctx.fft_r2c(d)
    dh64 = np.fft.fftn(d.cpu().numpy().astype(np.float64))
    ref = O.multipole_fields(dh64, 2, -1, n, box, edges)
    base = None
    for sz in (0, 1):
        for sy in (0, 1):
            for sx in (0, 1):
                ctx.set_shapes([sz, sy, sx])
                assert ctx.shapes() == [sz, sy, sx]
                got = Z.deinterleave(ctx.reconstruct_alm(dh, 2, -1).cpu().numpy(), ctx.nbins)
                for b in range(ctx.nbins):
                    assert np.abs(got[b] - ref[b]).max() <= 1e-5 * np.abs(ref[b]).max(), (sz, sy, sx, b)
                z = ctx.zeta_ell(particles=pd, forms=("node", "particle"))
                zz = {f: z[f].cpu().numpy() for f in z}
                if base is None:
                    base = zz
                for f in zz:
                    rel = np.abs(zz[f] - base[f]).max() / np.abs(base[f]).max()
                    assert rel < 1e-5, (sz, sy, sx, f, rel)
    with pytest.raises(Z.ZetaError):
        ctx.set_shapes([2, 0, 0])
    tuned = ctx.autotune(pd, forms=("node", "particle"))
    assert len(tuned) == 5 and all(s in (0, 1) for s in ctx.shapes())
    ctx.close()
