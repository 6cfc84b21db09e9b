"""Parity of every C-ABI call with the FP64 oracle on the same seeded inputs (GPU).

Sizes span several 8^3 tiles, several FFT tiles and ragged bin / particle-batch tails.
Tolerances: float32 path within 1e-5 relative (Frobenius per l, or max-abs relative for
grids); integer/index work (particle tiling) bit-exact.
"""
import math

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


def _maxrel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _rand_grid(n, seed, scale=1.0):
    return (np.random.default_rng(seed).standard_normal((n, n, n)) * scale).astype(np.float32)


@pytest.mark.parametrize("n", [16, 32, 64])
def test_fft_r2c_matches_dft(Z, n):
    ctx = Z.Context(n, 100.0, 4, 2, [5.0, 10.0])
    d = _rand_grid(n, n)
    got = ctx.fft_r2c(_dev(d)).cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    want = np.fft.fftn(d.astype(np.float64))[:, :, : n // 2]
    assert _maxrel(got, want) < 2e-6


@pytest.mark.parametrize("n,box", [(32, 200.0), (64, 500.0)])
def test_reconstruct_alm_matches_oracle(Z, n, box):
    edges = np.array([9.0, 21.0, 33.0, 47.0, 60.0, 88.0])
    ctx = Z.Context(n, box, 4, 5, edges)
    d = _rand_grid(n, 3 + n)
    dh = ctx.fft_r2c(_dev(d))
    dh64 = np.fft.fftn(d.astype(np.float64))
    nb = len(edges) - 1
    for l, m in [(0, 0), (1, -1), (1, 1), (2, 0), (3, 2), (4, -4), (5, 3)]:
        raw = ctx.reconstruct_alm(dh, l, m).cpu().numpy()
        assert raw.shape == (2, n, n, n, 4)
        np.testing.assert_array_equal(raw[1, ..., 1:], 0.0)  # zero padding lanes of the last group
        got = Z.deinterleave(raw, nb)
        want = O.multipole_fields(dh64, l, m, n, box, edges)
        for b in range(nb):
            assert _maxrel(got[b], want[b]) < 1e-5, (l, m, b, _maxrel(got[b], want[b]))
        sub = Z.deinterleave(ctx.reconstruct_alm(dh, l, m, 4, 5).cpu().numpy(), 1)
        np.testing.assert_array_equal(sub, got[4:5])


@pytest.mark.parametrize("n,dsup", [(16, 2), (32, 4), (32, 2)])
def test_assign_matches_oracle(Z, n, dsup):
    box = 150.0
    parts = mocks.lognormal_catalogue(n, 7000, box, 21, 22)
    parts[0, :3] = 0.0                              # on a corner node
    parts[1, :3] = np.float32(box) - np.float32(1e-3)  # just inside the upper faces
    parts[2, 3] = 2.5                               # a non-unit weight
    ctx = Z.Context(n, box, dsup, 0, [5.0, 10.0])
    delta, wsum = ctx.assign(_dev(parts))
    eps, w = O.assign(parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64), n, box, dsup)
    want = O.contrast(eps, w)
    assert abs(float(wsum.item()) - w) < 1e-12 * w
    assert np.abs(delta.cpu().numpy() - want).max() < 2e-6 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n,dsup,nb", [(16, 2, 5), (32, 4, 5), (32, 4, 12), (16, 4, 20)])
def test_sum_grid_matches_oracle(Z, n, dsup, nb):
    edges = np.linspace(5.0, 30.0, nb + 1)
    ctx = Z.Context(n, 80.0, dsup, 1, edges)
    d = _rand_grid(n, 5)
    a = np.random.default_rng(6).standard_normal((nb, n, n, n)).astype(np.float32)
    ai = _dev(Z.interleave(a))
    got = ctx.sum_grid(_dev(d), ai, "node").cpu().numpy()
    want = O.sum_node(d.astype(np.float64), a.astype(np.float64))
    assert _rel(got, want) < 1e-5
    if n == 16:
        got_g = ctx.sum_grid(_dev(d), ai, "gamma").cpu().numpy()
        want_g = O.sum_gamma(d.astype(np.float64), a.astype(np.float64), dsup)
        assert _rel(got_g, want_g) < 1e-5
        # accumulation semantics: a second call adds
        g2 = ctx.sum_grid(_dev(d), ai, "node", gram=torch.from_numpy(got).to("cuda")).cpu().numpy()
        assert _rel(g2, 2 * want) < 1e-5


def _clustered(n_p, box, seed):
    rng = np.random.default_rng(seed)
    p = np.empty((n_p, 4), np.float32)
    p[:, :3] = rng.uniform(0, box, (n_p, 3))
    k = n_p // 3  # a dense clump: one tile gets far more than one 256-point batch
    p[:k, :3] = (np.array([0.3, 0.6, 0.2]) * box + rng.normal(0, box / 200, (k, 3))) % box
    p[:, 3] = rng.uniform(0.5, 1.5, n_p)
    return p


@pytest.mark.parametrize("staging", [0, 16, 257])
@pytest.mark.parametrize("n,dsup,nb", [(32, 4, 5), (32, 2, 12), (16, 4, 9)])
def test_sort_and_particle_sum_match_oracle(Z, n, dsup, nb, staging):
    # staging 0: every tile batch interpolates from its shared-memory halo; 257: every one
    # from global memory; 16: both kinds in one launch (sparse and dense tiles)
    box = 120.0
    edges = np.linspace(5.0, 40.0, nb + 1)
    parts = _clustered(3001, box, 9)
    ctx = Z.Context(n, box, dsup, 1, edges, np_max=len(parts), forms=("particle",))
    ctx.set_staging(staging)
    assert ctx.staging() == staging
    pd = _dev(parts)
    srt, start = ctx.sort_particles(pd)
    srt, start = srt.cpu().numpy(), start.cpu().numpy()
    # tiling is exact: tile index of every particle, original order inside a tile
    cell = np.floor(parts[:, :3].astype(np.float64) * (n / box)).astype(np.int64) % n
    nt = n // 8
    tile = (cell[:, 2] // 8 * nt + cell[:, 1] // 8) * nt + cell[:, 0] // 8
    order = np.argsort(tile, kind="stable")
    np.testing.assert_array_equal(srt, parts[order])
    np.testing.assert_array_equal(start, np.concatenate([[0], np.cumsum(np.bincount(tile, minlength=nt ** 3))]))
    a = np.random.default_rng(10).standard_normal((nb, n, n, n)).astype(np.float32)
    w = float(parts[:, 3].astype(np.float64).sum())
    wsum = torch.tensor([w], dtype=torch.float64, device="cuda")
    got = ctx.sum_particles(_dev(srt), _dev(start), wsum, _dev(Z.interleave(a))).cpu().numpy()
    want = O.sum_particles(a.astype(np.float64), parts[:, :3], parts[:, 3], n, box, dsup)
    assert _rel(got, want) < 1e-5
    # a particle listed under the wrong tile is still interpolated at its own position
    moved = srt.copy()
    moved[5, 0] = (moved[5, 0] + 8.5 * box / n) % box
    got_m = ctx.sum_particles(_dev(moved), _dev(start), wsum, _dev(Z.interleave(a))).cpu().numpy()
    want_m = O.sum_particles(a.astype(np.float64), moved[:, :3], moved[:, 3], n, box, dsup)
    assert _rel(got_m, want_m) < 1e-5


@pytest.mark.parametrize("dsup", [2, 4])
def test_mass_term_matches_oracle(Z, dsup):
    n, box, lmax = 16, 90.0, 3
    edges = np.array([6.0, 14.0, 25.0, 31.0])
    ctx = Z.Context(n, box, dsup, lmax, edges)
    d = _rand_grid(n, 12)
    dh = ctx.fft_r2c(_dev(d))
    dh64 = np.fft.fftn(d.astype(np.float64))
    for l in range(lmax + 1):
        got = ctx.mass_term(dh, l).cpu().numpy()
        want = sum(O.mass_term(O.multipole_fields(dh64, l, m, n, box, edges), dsup) for m in range(-l, l + 1))
        assert _rel(got, want) < 1e-5, l


def _zeta_case(Z, n, box, lmax, edges, dsup, n_p, forms, seed):
    parts = mocks.lognormal_catalogue(n, n_p, box, seed, seed + 1)
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=n_p, forms=forms)
    got = ctx.zeta_ell(particles=_dev(parts), forms=forms)
    assert ctx.get_status() == 0
    want, cond = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, dsup, forms=forms)
    return {f: got[f].cpu().numpy() for f in got}, want, cond, ctx, parts


@pytest.mark.parametrize("dsup,forms", [(4, ("node", "particle")), (2, ("node", "gamma", "particle"))])
def test_zeta_ell_matches_oracle(Z, dsup, forms):
    n, box, lmax = 32, 240.0, 4
    edges = np.linspace(10.0, 85.0, 6)
    got, want, cond, ctx, parts = _zeta_case(Z, n, box, lmax, edges, dsup, 12000, forms, 31 + dsup)
    for f in forms:
        for l in range(lmax + 1):
            err = _rel(got[f][l], want[f][l])
            assert err < 1e-5, (f, l, err)
            # the error against the condition sum (sum of |terms|): what float32 can reach
            # whatever the cancellation in zeta_l (the oracle forms the sum for node and particle)
            if cond[f][l].max() > 0:
                err_c = float(np.abs(got[f][l] - want[f][l]).max() / cond[f][l].max())
                assert err_c < 2e-6, (f, l, err_c)
        np.testing.assert_array_equal(got[f], np.swapaxes(got[f], 1, 2))
    # bitwise reproducible
    again = ctx.zeta_ell(particles=_dev(parts), forms=forms)
    for f in forms:
        np.testing.assert_array_equal(again[f].cpu().numpy(), got[f])


def test_zeta_ell_from_delta_grid(Z):
    n, box, lmax, dsup = 32, 300.0, 3, 4
    edges = np.array([12.0, 30.0, 51.0, 77.0, 100.0])
    delta = (mocks.lognormal_density(n, 41) - 1.0).astype(np.float32)
    ctx = Z.Context(n, box, dsup, lmax, edges)
    got = ctx.zeta_ell(delta=_dev(delta), forms=("node",))["node"].cpu().numpy()
    want, _ = O.zeta_from_delta(delta.astype(np.float64), n, box, edges, lmax, dsup, forms=("node",))
    for l in range(lmax + 1):
        assert _rel(got[l], want["node"][l]) < 1e-5, l


def test_bounded_device_wait_reports_timeout_and_context_survives(Z):
    ctx = Z.Context(16, 100.0, 4, 1, [10.0, 20.0], np_max=500, forms=("particle",))
    ctx.selftest_wait(2000)
    assert ctx.get_status() == -4  # ZETA_ETIMEOUT, then cleared
    parts = torch.from_numpy(mocks.uniform_particles(500, 100.0, 4)).cuda()
    z = ctx.zeta_ell(particles=parts, forms=("particle",))["particle"]
    assert ctx.get_status() == 0 and bool(torch.isfinite(z).all())


def test_nonfinite_particle_is_reported_and_workspace_checked(Z):
    n, box = 16, 100.0
    parts = mocks.uniform_particles(500, box, 3)
    parts[7, 1] = np.nan
    ctx = Z.Context(n, box, 4, 1, [10.0, 20.0], np_max=500, forms=("particle",))
    ctx.zeta_ell(particles=_dev(parts), forms=("particle",))
    assert ctx.get_status() == -7
    assert ctx.get_status() == 0  # cleared
    lib = Z.lib()
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    assert lib.zeta_set_workspace(ctx._h, small.data_ptr(), 1024) == 0
    with pytest.raises(Z.ZetaError) as e:
        ctx.zeta_ell(particles=_dev(parts), forms=("particle",))
    assert e.value.code == -6


# --- node-form Gram on the tensor cores (tcgen05): per-arithmetic error bounds -------------
@pytest.mark.parametrize("gram,tol", [("tf32", 5e-3), ("bf16", 3e-2), ("bf16x3", 1e-4)])
@pytest.mark.parametrize("nb", [5, 20, 32])
def test_tensor_core_node_gram(Z, gram, tol, nb):
    n = 32
    edges = np.linspace(5.0, 30.0, nb + 1)
    ctx = Z.Context(n, 80.0, 4, 1, edges, gram=gram)
    d = _rand_grid(n, 15)
    a = np.random.default_rng(16).standard_normal((nb, n, n, n)).astype(np.float32)
    got = ctx.sum_grid(_dev(d), _dev(Z.interleave(a)), "node").cpu().numpy()
    assert ctx.get_status() == 0
    want = O.sum_node(d.astype(np.float64), a.astype(np.float64))
    err = _rel(got, want)
    assert err < tol, (gram, nb, err)


def test_tensor_core_zeta_ell_node_form(Z):
    n, box, lmax = 32, 240.0, 3
    edges = np.linspace(10.0, 85.0, 6)
    parts = mocks.lognormal_catalogue(n, 12000, box, 51, 52)
    want, _ = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, 4, forms=("node",))
    for gram, tol in (("bf16x3", 1e-4), ("tf32", 5e-3)):
        ctx = Z.Context(n, box, 4, lmax, edges, gram=gram, np_max=len(parts), forms=("node",))
        got = ctx.zeta_ell(particles=_dev(parts), forms=("node",))["node"].cpu().numpy()
        assert ctx.get_status() == 0
        for l in range(lmax + 1):
            assert _rel(got[l], want["node"][l]) < tol, (gram, l)


@pytest.mark.parametrize("nb", [6, 27])
def test_bfloat16_fields_node_form_on_the_tensor_cores(Z, nb):
    """Fields stored as bfloat16 by the last inverse pass, contracted on the tensor cores (any bin
    count up to 32): zeta_l of the node form against the oracle.  Bound: the fields carry a
    relative rounding of 2^-9 and so does delta a; 5e-3 of |zeta_l| per l (or 5e-4 of the condition
    sum where that exceeds 100 |zeta_l|)."""
    n, box, lmax = 32, 240.0, 2
    edges = np.linspace(8.0, 100.0, nb + 1)
    parts = mocks.lognormal_catalogue(n, 12000, box, 57, 58)
    want, cond = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, 4, forms=("node",))
    ctx = Z.Context(n, box, 4, lmax, edges, gram="bf16_fields", np_max=len(parts), forms=("node",))
    got = ctx.zeta_ell(particles=_dev(parts), forms=("node",))["node"].cpu().numpy()
    assert ctx.get_status() == 0
    for l in range(lmax + 1):
        err = float(np.linalg.norm(got[l] - want["node"][l]))
        zn, cn = float(np.linalg.norm(want["node"][l])), float(np.linalg.norm(cond["node"][l]))
        print(nb, l, f"{err / zn:.1e}", f"{err / cn:.1e}")
        assert err <= (5e-4 * cn if cn > 100 * zn else 5e-3 * zn), (nb, l, err / zn)
