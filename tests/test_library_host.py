"""CPU-side checks of libzeta: it builds, loads, exports every declared symbol, and its
host float64 table code agrees with the oracle.  No kernel is launched here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import zeta_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zmod():
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    zeta.lib()
    return zeta


def _declared():
    text = open(os.path.join(ROOT, "include", "zeta.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(zeta_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(zmod):
    names = _declared()
    assert len(names) >= 15
    lib = zmod.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(zmod.declared_symbols()) == names


def test_version_and_errors(zmod):
    lib = zmod.lib()
    assert lib.zeta_version() >= 10000
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.zeta_strerror(code)
    assert lib.zeta_strerror(-99) == b"unknown error"


def test_create_rejects_bad_parameters_without_touching_the_device(zmod):
    lib = zmod.lib()
    edges = np.array([5.0, 10.0, 20.0])
    good = dict(n=32, box=100.0, dsup=4, lmax=4, nbins=2, gram=0)
    bad = [dict(n=48), dict(n=8), dict(n=1024), dict(box=-1.0), dict(dsup=1), dict(dsup=5), dict(lmax=15),
           dict(nbins=0),
           dict(nbins=40), dict(gram=7), dict(box=30.0)]
    for change in bad:
        kw = {**good, **change}
        e = edges if kw["nbins"] <= 2 else np.linspace(5, 20, kw["nbins"] + 1)
        p = zmod._Params(kw["n"], kw["box"], kw["dsup"], kw["lmax"], kw["nbins"],
                         e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), kw["gram"])
        h = ctypes.c_void_p()
        assert lib.zeta_create(ctypes.byref(p), ctypes.byref(h)) == -1, change
        assert not h.value
    for e in (np.array([0.0, 5.0, 10.0]), np.array([5.0, 4.0, 10.0])):
        p = zmod._Params(32, 100.0, 4, 4, 2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
        h = ctypes.c_void_p()
        assert lib.zeta_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert lib.zeta_destroy(None) == 0
    assert lib.zeta_workspace_bytes(None, 0, 1) == 0


@pytest.mark.parametrize("box,r_lo,r_hi", [(500.0, 10.0, 20.0), (2000.0, 190.25, 200.0), (1000.0, 5.0, 14.6667)])
def test_host_jbar_matches_oracle(zmod, box, r_lo, r_hi):
    n = 512
    h = n // 2 - 1
    rng = np.random.default_rng(0)
    n2 = np.unique(np.concatenate([np.arange(0, 40), rng.integers(0, 3 * h * h + 1, 400), [3 * h * h]]))
    k = 2 * math.pi / box * np.sqrt(n2.astype(float))
    for ell in (0, 1, 2, 5, 10, 14):
        got = zmod.host_jbar(ell, box, r_lo, r_hi, n2)
        want = O.jbar(ell, k, r_lo, r_hi)
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-13)


def test_host_ylm_matches_oracle(zmod):
    rng = np.random.default_rng(1)
    v = rng.integers(-255, 256, (200, 3)).astype(float)
    v[0] = (0, 0, 7)
    v[1] = (3, 0, 0)
    for ell in range(15):
        for m in range(-ell, ell + 1):
            got = np.array([zmod.host_ylm(ell, m, *row) for row in v])
            want = O.real_ylm(ell, m, v[:, 0], v[:, 1], v[:, 2])
            np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)
    assert zmod.host_ylm(0, 0, 0.0, 0.0, 0.0) == pytest.approx(1 / math.sqrt(4 * math.pi), rel=1e-15)
    assert zmod.host_ylm(3, 1, 0.0, 0.0, 0.0) == 0.0


@pytest.mark.parametrize("n,dsup", [(16, 2), (16, 4), (512, 4), (32, 3)])
def test_host_mass_hat_matches_oracle(zmod, n, dsup):
    got = zmod.host_mass_hat(n, dsup)
    m = O.mass_1d(dsup)
    k = np.arange(n)
    want = sum(m[a] * np.cos(2 * math.pi * k * a / n) for a in m)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert got[0] == pytest.approx(1.0, abs=1e-14)  # sum_a M(a) = (int beta)^2 = 1
    np.testing.assert_allclose(got[1:], got[1:][::-1], rtol=0, atol=1e-15)  # Mhat(k) = Mhat(n - k)
    assert np.all(got > 0)  # the sampled B-spline autocorrelation has a positive DFT


@pytest.mark.parametrize("q,dsup", [(2, 2), (5, 4), (12, 4)])
def test_host_cell_quadrature_matches_oracle(zmod, q, dsup):
    t, wq, beta = zmod.host_cell_quadrature(q, dsup)
    x, w = np.polynomial.legendre.leggauss(q)
    np.testing.assert_allclose(t, 0.5 * (x + 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(wq, 0.5 * w, rtol=0, atol=1e-15)
    for o in range(dsup):
        np.testing.assert_allclose(beta[:, o], O.bspline(t + dsup // 2 - 1 - o, dsup), rtol=0, atol=4e-15)
    np.testing.assert_allclose(beta.sum(1), 1.0, rtol=0, atol=1e-15)  # partition of unity
    # exact for polynomials of degree 2q - 1 on the cell
    for p in range(2 * q):
        assert float(np.sum(wq * t ** p)) == pytest.approx(1.0 / (p + 1), abs=1e-14)


def test_host_table_helpers_reject_bad_arguments(zmod):
    lib = zmod.lib()
    out = np.empty(64, np.float64)
    assert lib.zeta_host_mass_hat(16, 5, out.ctypes.data) == -1
    assert lib.zeta_host_cell_quadrature(5, 3, out.ctypes.data, out.ctypes.data, out.ctypes.data) == -1
    assert lib.zeta_host_daub4_dyadic(-1, out.ctypes.data) == -1 and lib.zeta_host_daub4_dyadic(21, out.ctypes.data) == -1
    assert lib.zeta_host_daub4_gamma(None, None, None) == -1
    shape = np.zeros(3, np.int32)
    assert lib.zeta_set_shapes(None, shape.ctypes.data, 3) == -1
    assert lib.zeta_get_shapes(None, shape.ctypes.data, 3) == -1
    assert lib.zeta_host_mass_hat(1, 4, out.ctypes.data) == -1
    assert lib.zeta_host_cell_quadrature(0, 4, out.ctypes.data, out.ctypes.data, out.ctypes.data) == -1
    assert lib.zeta_host_cell_quadrature(5, 4, None, out.ctypes.data, out.ctypes.data) == -1


@pytest.mark.parametrize("n,box,lmax,edges", [
    (16, 120.0, 14, [10.0, 20.0, 32.0, 45.0, 50.0, 55.0]),
    (64, 500.0, 6, [10.0, 20.0, 30.0, 40.0, 50.0, 60.0, 70.0, 80.0, 90.0]),
])
def test_host_window_table_matches_oracle(zmod, n, box, lmax, edges):
    # the exact float32 table a context uploads: layout [l][|n|^2][bin], bins padded to 4 with zeros
    tab = zmod.host_jbar_table(n, box, lmax, edges)
    nb = len(edges) - 1
    h = n // 2 - 1
    assert tab.shape == (lmax + 1, 3 * h * h + 1, 4 * ((nb + 3) // 4))
    assert not np.any(tab[:, :, nb:])
    k = 2 * math.pi / box * np.sqrt(np.arange(3 * h * h + 1, dtype=np.float64))
    pref = math.sqrt(4 * math.pi) / n ** 3
    for ell in range(lmax + 1):
        for b in range(nb):
            want = pref * O.jbar(ell, k, edges[b], edges[b + 1])
            np.testing.assert_allclose(tab[ell, :, b], want, rtol=1e-6, atol=1e-9 * pref)


@pytest.mark.parametrize("vertex", [
    {"radial": "shell", "tophat": 12.0},
    {"radial": "point", "radii": [7.5, 19.0, 41.0]},
    {"radial": "point", "radii": [7.5, 19.0, 41.0], "tophat": 5.0},
])
def test_window_table_with_vertex_windows_matches_oracle(zmod, vertex):
    """The table a context uploads with the vertex windows of Sec. 3 on, every entry against the
    oracle's radial window: sqrt(4 pi) W_l,b(k) / N_g."""
    n, box, lmax = 32, 200.0, 6
    edges = np.array([6.0, 13.0, 22.0, 35.0])
    p, keep = zmod.make_params(n, box, 4, lmax, edges if vertex["radial"] == "shell" else None,
                               radial=vertex["radial"], radii=vertex.get("radii"), tophat=vertex.get("tophat", 0.0))
    nb = p.nbins
    nbp = 4 * ((nb + 3) // 4)
    n2max = 3 * (n // 2 - 1) ** 2 + 1
    out = np.zeros((lmax + 1) * n2max * nbp, np.float32)
    assert zmod.lib().zeta_host_window_table(ctypes.byref(p), out.ctypes.data_as(ctypes.c_void_p)) == 0
    out = out.reshape(lmax + 1, n2max, nbp)
    k = 2 * math.pi / box * np.sqrt(np.arange(n2max, dtype=np.float64))
    for ell in range(lmax + 1):
        for b in range(nb):
            want = math.sqrt(4 * math.pi) * O.radial_window(ell, k, b, edges, vertex) / n ** 3
            np.testing.assert_allclose(out[ell, :, b], want, rtol=2e-6, atol=1e-7 * np.abs(want).max())
        np.testing.assert_array_equal(out[ell, :, nb:], 0.0)
    bad, keep2 = zmod.make_params(n, box, 4, lmax, None, radial="point", radii=[7.5, -1.0])
    assert zmod.lib().zeta_host_window_table(ctypes.byref(bad), out.ctypes.data_as(ctypes.c_void_p)) == -1


@pytest.mark.parametrize("dsup", [2, 3, 4])
def test_phi_hat_per_axis_matches_oracle(zmod, dsup):
    n = 24
    out = np.zeros(n)
    assert zmod.lib().zeta_host_phi_hat(n, dsup, out.ctypes.data_as(ctypes.c_void_p)) == 0
    full = O.phi_hat(n, dsup)
    # the Daubechies product takes about 25 factors, each rounded
    np.testing.assert_allclose(out, full[0, 0, :], rtol=1e-14 if dsup != 3 else 1e-13)
    np.testing.assert_allclose(np.multiply.outer(np.multiply.outer(out, out), out), full, rtol=1e-13)


def test_create_rejects_bad_vertex_windows(zmod):
    lib = zmod.lib()
    edges = np.array([5.0, 10.0, 20.0])
    for kw in (dict(radial="point", radii=[5.0, 60.0]), dict(radial="point", radii=[0.0, 10.0]),
               dict(tophat=-1.0), dict(tophat_primary=float("nan"))):
        p, keep = zmod.make_params(32, 100.0, 4, 2, None if kw.get("radial") == "point" else edges, **kw)
        h = ctypes.c_void_p()
        assert lib.zeta_create(ctypes.byref(p), ctypes.byref(h)) == -1, kw


def test_legendre_sum_and_reduced_q_match_oracle(zmod):
    rng = np.random.default_rng(17)
    zl = rng.standard_normal((9, 3, 3))
    mu = np.linspace(-1.0, 1.0, 13)
    np.testing.assert_allclose(zmod.legendre_sum(zl, mu), O.legendre_sum(zl, mu), rtol=1e-13, atol=1e-13)
    z, x1, x2, x3 = (rng.uniform(0.2, 2.0, 7) for _ in range(4))
    np.testing.assert_allclose(zmod.reduced_q(z, x1, x2, x3), O.reduced_q(z, x1, x2, x3), rtol=1e-15)
    # the generating function of the Legendre polynomials, through the library
    t = 0.45
    gl = zmod.legendre_sum((t ** np.arange(61))[:, None, None] * np.ones((1, 1, 1)), mu)
    np.testing.assert_allclose(gl[:, 0, 0], (1 - 2 * mu * t + t * t) ** -0.5, rtol=1e-14)
    with pytest.raises(zmod.ZetaError):
        zmod.legendre_sum(zl, [1.5])


@pytest.mark.parametrize("level", [0, 3, 10])
def test_daub4_dyadic_table_matches_oracle(zmod, level):
    got = zmod.host_daub4_dyadic(level)
    np.testing.assert_allclose(got, O.daub4_dyadic(level), rtol=0, atol=2e-15)


def test_daub4_connection_coefficients_and_split_match_oracle(zmod):
    g, lam, u = zmod.host_daub4_gamma()
    want = O.daub4_gamma()
    for a in range(-2, 3):
        for b in range(-2, 3):
            assert abs(g[a + 2, b + 2] - want.get((a, b), 0.0)) < 1e-14, (a, b)
    np.testing.assert_allclose(u @ u.T, np.eye(5), atol=1e-14)       # orthonormal eigenvectors
    np.testing.assert_allclose(u @ np.diag(lam) @ u.T, g, atol=1e-14)  # the split the Gamma form applies
