"""The Daubechies basis (dsup = 3: the genus-4 scaling function of Sec. 2.2, D_sup = 3) through
the C ABI against the FP64 oracle on the same seeded catalogues (GPU).

Checked: the assignment on every node (64^3, and the 256^3 grid with the 2M-particle
catalogue); zeta_l of the node and particle forms on the 64^3 / 20k-particle catalogue
(lmax 4, 8 bins 10-90) and on its uniform null catalogue; the Gamma form (the exact connection
coefficients applied through their eigen-split) on a 16^3 grid, inside zeta_ell and as the
grid sum alone at 3 and 29 bins; the 2PCF in both forms; the
fields of one (l, m) with the basis's own Phi-hat window; the node gradient; and that the
particle gradient refuses this basis.

Tolerances: the library reads phi from float32 dyadic values joined linearly, at an in-cell
offset t rounded to float32; phi's slope between dyadic points reaches about 2^(0.45 * 10),
so a weight can differ from the oracle's by about 1e-6.  Assignment: max |delta_gpu -
delta_oracle| <= 1e-5 max(1, |delta|).  zeta_l: per l, relative Frobenius 1e-5, or 1e-6 of the
condition sum where that is more than 100 times |zeta_l| (as for the B-splines).
"""
import numpy as np
import pytest

from oracle import zeta_oracle as O
from paper_2507_15209_gb300 import mocks
from paper_2507_15209_gb300.workloads import WORKLOADS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, BOX, LMAX = 64, 500.0, 4
EDGES = np.linspace(10.0, 90.0, 9)


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    return zeta


def _check(got, want, cond, label):
    errs = []
    for ell in range(want.shape[0]):
        err = float(np.linalg.norm(got[ell] - want[ell]))
        zn = float(np.linalg.norm(want[ell]))
        cn = float(np.linalg.norm(cond[ell])) if cond is not None else 0.0
        errs.append(err / zn)
        if cond is not None and cn > 100.0 * zn:
            assert err <= 1e-6 * cn, (label, ell, err / zn, err / cn)
        else:
            assert err <= 1e-5 * zn, (label, ell, err / zn)
    print(label, [f"{e:.1e}" for e in errs])


def _assign_check(Z, n, box, parts):
    ctx = Z.Context(n, box, 3, 0, [5.0, 10.0])
    d, wsum = ctx.assign(torch.from_numpy(parts).cuda())
    got = d.cpu().numpy()
    eps, wtot = O.assign(parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64), n, box, 3)
    want = O.contrast(eps, wtot)
    err = float(np.abs(got - want).max())
    print(f"assign {n}^3: max error {err:.2e}, max |delta| {np.abs(want).max():.2f}")
    assert err <= 1e-5 * max(1.0, float(np.abs(want).max()))
    assert abs(float(wsum.item()) - wtot) <= 1e-9 * wtot
    ctx.close()


def test_assignment_64_and_256(Z):
    w = WORKLOADS["box500_n64_np20k"]
    _assign_check(Z, 64, w["box"], mocks.lognormal_catalogue(64, w["n_p"], w["box"], w["field_seed"],
                                                             w["sample_seed"]))
    w = WORKLOADS["box1000_n256_np2m"]
    _assign_check(Z, 256, w["box"], mocks.lognormal_catalogue(256, w["n_p"], w["box"], w["field_seed"],
                                                              w["sample_seed"]))


@pytest.mark.parametrize("null", [False, True])
def test_node_and_particle_forms_64(Z, null):
    w = WORKLOADS["box500_n64_np20k"]
    if null:
        parts = mocks.uniform_particles(w["n_p"], w["box"], w["null_seed"])
    else:
        parts = mocks.lognormal_catalogue(N, w["n_p"], w["box"], w["field_seed"], w["sample_seed"])
    forms = ("node", "particle")
    ctx = Z.Context(N, BOX, 3, LMAX, EDGES, np_max=len(parts), forms=forms)
    z = ctx.zeta_ell(particles=torch.from_numpy(parts).cuda(), forms=forms)
    assert ctx.get_status() == 0
    want, cond = O.zeta_multipoles(parts.astype(np.float64), N, BOX, EDGES, LMAX, 3, forms=forms)
    for f in forms:
        got = z[f].cpu().numpy()
        np.testing.assert_array_equal(got, np.swapaxes(got, 1, 2))
        _check(got, want[f], cond[f], ("null" if null else "data", f))
    ctx.close()


def test_gamma_form_16(Z):
    n, box, lmax = 16, 120.0, 2
    edges = np.array([8.0, 16.0, 26.0, 38.0, 50.0])
    parts = mocks.lognormal_catalogue(n, 6000, box, 351, 352)
    forms = ("node", "gamma")
    ctx = Z.Context(n, box, 3, lmax, edges, np_max=len(parts), forms=forms)
    z = ctx.zeta_ell(particles=torch.from_numpy(parts).cuda(), forms=forms)
    assert ctx.get_status() == 0
    want, cond = O.zeta_multipoles(parts.astype(np.float64), n, box, edges, lmax, 3, forms=forms)
    _check(z["node"].cpu().numpy(), want["node"], cond["node"], "node 16")
    _check(z["gamma"].cpu().numpy(), want["gamma"], cond["node"], "gamma 16")
    ctx.close()


@pytest.mark.parametrize("nb", [3, 29])
def test_gamma_grid_sum_with_the_eigen_split(Z, nb):
    """The Gamma form's grid sum alone on random fields: 3 bins (one padded group) and 29 (the
    largest padded bin count, 32, whose per-batch buffers are the largest)."""
    n = 16
    edges = np.linspace(5.0, 40.0, nb + 1)
    rng = np.random.default_rng(700 + nb)
    d = rng.standard_normal((n, n, n)).astype(np.float32)
    a = rng.standard_normal((nb, n, n, n)).astype(np.float32)
    ctx = Z.Context(n, 100.0, 3, 1, edges)
    got = ctx.sum_grid(torch.from_numpy(d).cuda(), torch.from_numpy(Z.interleave(a)).cuda(), "gamma").cpu().numpy()
    want = O.sum_gamma(d.astype(np.float64), a.astype(np.float64), 3)
    err = float(np.linalg.norm(got - want)) / float(np.linalg.norm(want))
    print(f"gamma grid sum, {nb} bins: relative error {err:.1e}")
    assert err < 1e-5
    ctx.close()


def test_xi_both_forms_and_phi_hat_fields(Z):
    w = WORKLOADS["box500_n64_np20k"]
    parts = mocks.lognormal_catalogue(N, w["n_p"], w["box"], w["field_seed"], w["sample_seed"])
    pd = torch.from_numpy(parts).cuda()
    ctx = Z.Context(N, BOX, 3, LMAX, EDGES, np_max=len(parts), forms=("node", "particle"), phi_hat=True)
    xi = ctx.xi(particles=pd, forms=("node", "particle"))
    eps, wtot = O.assign(parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64), N, BOX, 3)
    delta = O.contrast(eps, wtot)
    vertex = {"phi_dsup": 3}
    want_node = O.xi_node(delta, N, BOX, EDGES, vertex=vertex)
    want_part = O.xi_particle(parts.astype(np.float64), N, BOX, EDGES, 3, vertex=vertex)
    for got, want, f in ((xi["node"], want_node, "node"), (xi["particle"], want_part, "particle")):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max(), (f, got, want)
    d, _ = ctx.assign(pd)
    dh = ctx.fft_r2c(d)
    dh64 = np.fft.fftn(d.cpu().numpy().astype(np.float64))
    got = Z.deinterleave(ctx.reconstruct_alm(dh, 3, -2).cpu().numpy(), ctx.nbins)
    ref = O.multipole_fields(dh64, 3, -2, N, BOX, EDGES, vertex=vertex)
    for b in range(ctx.nbins):
        assert np.abs(got[b] - ref[b]).max() <= 1e-5 * np.abs(ref[b]).max(), b
    ctx.close()


def test_gradients_with_the_daubechies_basis(Z):
    n, box, lmax = 16, 120.0, 2
    edges = np.array([9.0, 20.0, 31.0])
    rng = np.random.default_rng(53)
    delta = rng.standard_normal((n, n, n)).astype(np.float32)
    wts = rng.standard_normal((lmax + 1, 2, 2))
    ctx = Z.Context(n, box, 3, lmax, edges, np_max=100, forms=("node", "backward"))
    got = ctx.backward_node(torch.from_numpy(delta).cuda(), wts).cpu().numpy()
    want = O.grad_node_delta(delta.astype(np.float64), wts, n, box, edges, lmax)
    assert np.abs(got - want).max() <= 2e-5 * np.abs(want).max()
    parts = torch.from_numpy(mocks.uniform_particles(100, box, 54)).cuda()
    with pytest.raises(Z.ZetaError) as e:
        ctx.backward_particles(parts, wts)
    assert e.value.code == -5
    ctx.close()
