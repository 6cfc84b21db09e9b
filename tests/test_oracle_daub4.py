"""Pins of the oracle's Daubechies basis (dsup = 3: the genus-4 scaling function of the paper's
Sec. 2.2, support D_sup = 3) against facts fixed by the mathematics of the two-scale relation:
the filter's orthogonality and vanishing moments, the closed-form values of phi at the
integers, polynomial reproduction, orthonormality (in space and in Fourier space), brute-force
quadrature of the connection coefficients, and the triple integral the Gamma form stands for.
CPU only.
"""
import math

import numpy as np
import pytest

from oracle import zeta_oracle as O

S3 = math.sqrt(3.0)
MU1 = (3.0 - S3) / 2.0  # int x phi(x) dx = sum_k k h_k / sqrt2 for this filter


def _table(level):
    t = O.daub4_dyadic(level)
    return np.arange(t.size) / 2.0 ** level, t


def test_filter_orthogonality_and_vanishing_moments():
    h = O.daub4_filter()
    assert abs(h.sum() - math.sqrt(2.0)) < 1e-15
    assert abs((h * h).sum() - 1.0) < 1e-15
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-16          # double shifts orthogonal
    k = np.arange(4)
    alt = (-1.0) ** k
    assert abs((alt * h).sum()) < 1e-15 and abs((alt * k * h).sum()) < 1e-15  # two vanishing moments
    assert abs((k * h).sum() / math.sqrt(2.0) - MU1) < 1e-15


def test_integer_values_and_polynomial_reproduction():
    x, t = _table(10)
    assert t[0] == 0.0 and t[-1] == 0.0
    assert abs(t[1024] - (1.0 + S3) / 2.0) < 1e-14 and abs(t[2048] - (1.0 - S3) / 2.0) < 1e-14
    assert abs(O.daub4_phi(0.5) - (2.0 + S3) / 4.0) < 1e-14  # phi(1/2) = sqrt2 h0 phi(1)
    rng = np.random.default_rng(31)
    u = rng.uniform(-4.0, 4.0, 500)
    ls = range(-10, 11)
    np.testing.assert_allclose(sum(O.daub4_phi(u - l) for l in ls), 1.0, atol=1e-14)
    np.testing.assert_allclose(sum(l * O.daub4_phi(u - l) for l in ls), u - MU1, atol=1e-13)
    assert np.all(O.daub4_phi(np.array([-0.3, 3.0, 3.2])) == 0.0)


def test_table_is_the_fixed_point_of_the_refinement():
    """At every point of level 10 (not only the odd ones the construction computes),
    phi(x) = sqrt2 sum_i h_i phi(2x - i), and level 9 is level 10 at the even points."""
    h = O.daub4_filter()
    _, t10 = _table(10)
    _, t9 = _table(9)
    np.testing.assert_array_equal(t10[0::2], t9)
    k = np.arange(t10.size)
    rhs = np.zeros(t10.size)
    for i, hi in enumerate(h):
        src = k - i * 2 ** 9  # level-9 index of 2 (k / 2^10) - i
        ok = (src >= 0) & (src < t9.size)
        rhs[ok] += math.sqrt(2.0) * hi * t9[src[ok]]
    np.testing.assert_allclose(rhs, t10, atol=1e-14)


def test_mass_is_orthonormal_and_gamma_is_the_triple_integral():
    m = O.daub4_mass()
    for a, v in m.items():
        assert abs(v - (1.0 if a == 0 else 0.0)) < 1e-14, (a, v)
    assert O.mass_1d(3) == m
    g = O.daub4_gamma()
    assert len(g) == 19 and O.gamma_1d(3) == g
    assert abs(sum(g.values()) - 1.0) < 1e-13
    for (a, b), v in g.items():
        assert abs(v - g[(b, a)]) < 1e-15                     # symmetric
        assert abs(v - g[(-a, b - a)]) < 1e-14                # x -> x + a (not imposed by the solve)
    for a in range(-2, 3):
        assert abs(sum(v for (p, _), v in g.items() if p == a) - m[a]) < 1e-14
    # brute force: trapezoid on the level-13 dyadic values (the integrand vanishes at both ends)
    x, t = _table(13)
    for (a, b), v in g.items():
        num = np.trapezoid(t * O.daub4_phi(x - a, 13) * O.daub4_phi(x - b, 13), x)
        assert abs(num - v) < 1e-6, (a, b, num, v)
    # first moment: sum_b b Gamma(0, b) = int phi^2 (x - mu1) dx (linear reproduction)
    want = np.trapezoid(t * t * (x - MU1), x)
    assert abs(sum(b * v for (p, b), v in g.items() if p == 0) - want) < 1e-6


def test_power_spectrum_orthonormality_closed_form_and_transform():
    w = np.linspace(-3.1, 3.1, 9)
    tot = sum(O.daub4_power(w + 2.0 * math.pi * k) for k in range(-3000, 3001))
    np.testing.assert_allclose(tot, 1.0, atol=2e-7)           # sum_k |phi-hat(w + 2 pi k)|^2 = 1
    # |m0(w)|^2 = cos^4(w/2) (1 + 2 sin^2(w/2)) and prod_j cos(w/2^(j+1)) = sin(w/2) / (w/2)
    om = np.array([0.2, 0.9, 1.7, 2.9, 5.0])
    closed = np.sinc(om / (2.0 * math.pi)) ** 4
    for j in range(1, 60):
        closed = closed * (1.0 + 2.0 * np.sin(om / 2.0 ** (j + 1)) ** 2)
    np.testing.assert_allclose(O.daub4_power(om), closed, rtol=1e-13)
    x, t = _table(13)
    for o in om[:4]:
        ft = np.trapezoid(t * np.exp(-1j * o * x), x)
        assert abs(abs(ft) ** 2 - O.daub4_power(np.array([o]))[0]) < 1e-7
    n = 16
    p1 = O.daub4_power(2.0 * math.pi * O.fft_integers(n) / n)
    np.testing.assert_allclose(O.phi_hat(n, 3), p1[:, None, None] * p1[None, :, None] * p1[None, None, :],
                               rtol=1e-15)


def test_assign_and_interpolate_moments_and_adjoint():
    n, box = 16, 80.0
    rng = np.random.default_rng(32)
    pos = rng.uniform(20.0, 60.0, (60, 3))
    w = rng.uniform(0.5, 2.0, 60)
    eps, wsum = O.assign(pos, w, n, box, 3)
    assert abs(eps.sum() - w.sum()) < 1e-12 and abs(wsum - w.sum()) < 1e-12
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = pos / (box / n)
    assert abs((eps * lx).sum() - (w * (u[:, 0] - MU1)).sum()) < 1e-10
    assert abs((eps * lz).sum() - (w * (u[:, 2] - MU1)).sum()) < 1e-10
    a = np.stack([1.5 * lx - 0.25 * ly + 2.0 * lz + 0.5, np.ones((n, n, n))]).astype(float)
    f = O.interpolate(a, pos, n, box, 3)
    np.testing.assert_allclose(f[0], 1.5 * (u[:, 0] - MU1) - 0.25 * (u[:, 1] - MU1) + 2.0 * (u[:, 2] - MU1) + 0.5,
                               atol=1e-12)
    np.testing.assert_allclose(f[1], 1.0, atol=1e-14)
    g = rng.standard_normal((1, n, n, n))
    lhs = float((eps * g[0]).sum())
    rhs = float((w * O.interpolate(g, pos, n, box, 3)[0]).sum())
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))
    # every particle's stencil is the three nodes floor(u) - 2 .. floor(u)
    one, _ = O.assign(np.array([[10.3, 20.7, 33.1]]), np.array([1.0]), n, box, 3)
    nz = np.argwhere(one != 0.0)
    assert sorted(set(nz[:, 2])) == [0, 1, 2] and sorted(set(nz[:, 1])) == [2, 3, 4]


def test_gamma_form_is_the_triple_integral_of_the_expansions():
    """(1/N_g) sum_l delta_l sum Gamma a_b1 a_b2 = (1/N_g) int n f_b1 f_b2 over the periodic box
    (grid units), n and f the expansions in the periodised basis.  The basis is separable, so the
    integral is sum delta_l a_b1(m) a_b2(k) prod_d T(l_d, m_d, k_d) with the 1-D integrals
    T(l, m, k) = int phi(s - l) phi(s - m) phi(s - k) ds over the period, taken here by the
    trapezoid rule on the level-13 dyadic values (error about 1e-7); no connection coefficient
    or offset convention of the oracle enters.  An offset of the wrong sign changes the sum by
    far more."""
    n, lev = 4, 13
    rng = np.random.default_rng(33)
    delta = rng.standard_normal((n, n, n))
    a = rng.standard_normal((2, n, n, n))
    got = O.sum_gamma(delta, a, 3)
    s = np.arange(n * 2 ** lev) / 2.0 ** lev
    bmat = np.zeros((n, s.size))  # periodic 1-D basis phi(s - l)
    for l in range(n):
        for k in range(-2, 3):
            bmat[l] += O.daub4_phi(s - l - k * n, lev)
    t3 = np.einsum("ls,ms,ks->lmk", bmat, bmat, bmat) / 2.0 ** lev  # periodic: every sample once
    want = np.array([[np.einsum("zyx,ZYX,ABC,zZA,yYB,xXC->", delta, a[i], a[j], t3, t3, t3, optimize=True)
                      for j in range(2)] for i in range(2)]) / n ** 3
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max(), (got, want)
    # the same sum with Gamma(a, b) replaced by Gamma(-a, -b) is far off
    g = O.gamma_1d(3)
    bad = np.zeros((2, 2))
    for (pz, qz), vz in g.items():
        for (py, qy), vy in g.items():
            for (px, qx), vx in g.items():
                a1 = np.roll(a, (pz, py, px), axis=(1, 2, 3)).reshape(2, -1) * delta.reshape(1, -1)
                a2 = np.roll(a, (qz, qy, qx), axis=(1, 2, 3)).reshape(2, -1)
                bad += vz * vy * vx * (a1 @ a2.T)
    bad /= n ** 3
    assert np.abs(bad - want).max() > 20 * np.abs(got - want).max()


def test_mass_term_matches_fourier_space_form():
    n, box, lmax = 12, 60.0, 2
    edges = np.array([7.0, 15.0, 24.0])
    rng = np.random.default_rng(34)
    dh = np.fft.fftn(rng.standard_normal((n, n, n)))
    for ell in range(lmax + 1):
        u = np.zeros((2, 2))
        for m in range(-ell, ell + 1):
            a = O.multipole_fields(dh, ell, m, n, box, edges)
            u += O.mass_term(a, 3)
            np.testing.assert_allclose(O.mass_term(a, 3), O.sum_node(np.ones((n, n, n)), a), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(O.mass_term_fourier(dh, ell, n, box, edges, 3), u, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("forms", [("node", "particle", "gamma")])
def test_zeta_invariances(forms):
    """Translation by whole cells, axis permutation and a global weight scale leave zeta_l
    unchanged (reflection does not: the Daubechies function is not symmetric)."""
    n, box, lmax = 8, 40.0, 2
    edges = np.array([6.0, 12.0, 18.0])
    rng = np.random.default_rng(35)
    p = np.empty((300, 4))
    p[:, :3] = rng.uniform(0, box, (300, 3))
    p[:, 3] = rng.uniform(0.5, 1.5, 300)
    z0, _ = O.zeta_multipoles(p, n, box, edges, lmax, 3, forms=forms)
    h = box / n
    moved = p.copy()
    moved[:, :3] = (moved[:, :3] + h * np.array([3, 5, 7])) % box
    perm = p.copy()
    perm[:, [0, 1, 2]] = p[:, [2, 0, 1]]
    scaled = p.copy()
    scaled[:, 3] *= 2.5
    for q in (moved, perm, scaled):
        z1, _ = O.zeta_multipoles(q, n, box, edges, lmax, 3, forms=forms)
        for f in forms:
            np.testing.assert_allclose(z1[f], z0[f], rtol=1e-10, atol=1e-12 * np.abs(z0[f]).max())
    refl = p.copy()
    refl[:, 1] = (box - p[:, 1]) % box
    z1, _ = O.zeta_multipoles(refl, n, box, edges, lmax, 3, forms=("node",))
    assert np.abs(z1["node"] - z0["node"]).max() > 1e-6 * np.abs(z0["node"]).max()
