"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics:
closed forms, textbook values, invariants, library special cases and brute
force.  Each test names the oracle function(s) it pins.  CPU only.
"""
import math
import os
import warnings

import numpy as np
import pytest
from scipy import integrate, special

from oracle import zeta_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_mass():
    out = {}
    with open(os.path.join(GOLDEN, "bspline_mass.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            d, a, num, den = (int(t) for t in line.split())
            out[(d, a)] = num / den
    return out


# --- bspline, mass_1d, gamma_1d --------------------------------------------------------
@pytest.mark.parametrize("dsup", [2, 4])
def test_bspline_partition_of_unity_and_integral(dsup):
    rng = np.random.default_rng(1)
    u = rng.uniform(-3, 3, 200)
    s = sum(O.bspline(u - l, dsup) for l in range(-8, 9))
    np.testing.assert_allclose(s, 1.0, atol=1e-14)
    val, _ = integrate.quad(lambda x: float(O.bspline(x, dsup)), -dsup / 2, dsup / 2, points=[0.0, -1.0, 1.0])
    assert abs(val - 1.0) < 1e-12
    # knot values of the order-D cardinal spline
    if dsup == 2:
        assert O.bspline(0.0, 2) == 1.0 and O.bspline(0.5, 2) == 0.5
    else:
        assert abs(O.bspline(0.0, 4) - 2 / 3) < 1e-15 and abs(O.bspline(1.0, 4) - 1 / 6) < 1e-15
        assert O.bspline(2.0, 4) == 0.0


@pytest.mark.parametrize("dsup", [2, 4])
def test_mass_matches_textbook_and_gamma_sums(dsup):
    gold = _golden_mass()
    m1 = O.mass_1d(dsup)
    for a, v in m1.items():
        assert abs(v - gold.get((dsup, abs(a)), 0.0)) < 1e-14, (a, v)
    g = O.gamma_1d(dsup)
    assert abs(sum(g.values()) - 1.0) < 1e-13            # sum Gamma = int phi = 1
    for a in range(-(dsup - 1), dsup):                   # sum_b gamma(a, b) = M(a)
        s = sum(v for (p, q), v in g.items() if p == a)
        assert abs(s - m1[a]) < 1e-14
    for (p, q), v in g.items():                          # symmetries of the triple integral
        assert abs(v - g[(q, p)]) < 1e-15 and abs(v - g[(-p, -q)]) < 1e-15
    assert len(g) == {2: 7, 4: 37}[dsup]


# --- assign / interpolate ---------------------------------------------------------------
@pytest.mark.parametrize("dsup", [2, 4])
def test_assign_partition_and_linear_moment(dsup):
    n, box = 16, 80.0
    rng = np.random.default_rng(2)
    pos = rng.uniform(20.0, 60.0, (50, 3))  # far from the periodic wrap
    w = rng.uniform(0.5, 2.0, 50)
    eps, wsum = O.assign(pos, w, n, box, dsup)
    assert abs(eps.sum() - w.sum()) < 1e-12 and abs(wsum - w.sum()) < 1e-12
    # centred B-splines reproduce linear functions: sum_l l beta(u - l) = u
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    u = pos / (box / n)
    assert abs((eps * lx).sum() - (w * u[:, 0]).sum()) < 1e-10
    assert abs((eps * lz).sum() - (w * u[:, 2]).sum()) < 1e-10


def test_assign_hat_at_nodes_is_identity():
    n, box = 8, 8.0
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    pos = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], 1).astype(float)
    w = np.arange(n ** 3, dtype=float) + 1.0
    eps, _ = O.assign(pos, w, n, box, 2)
    np.testing.assert_array_equal(eps.ravel(), w)


@pytest.mark.parametrize("dsup", [2, 4])
def test_interpolate_linear_reproduction_and_adjoint(dsup):
    n, box = 16, 32.0
    rng = np.random.default_rng(3)
    pos = rng.uniform(8.0, 24.0, (40, 3))
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a = np.stack([1.5 * lx - 0.25 * ly + 2.0 * lz + 0.5, np.ones((n, n, n))]).astype(float)
    f = O.interpolate(a, pos, n, box, dsup)
    u = pos / (box / n)
    np.testing.assert_allclose(f[0], 1.5 * u[:, 0] - 0.25 * u[:, 1] + 2.0 * u[:, 2] + 0.5, atol=1e-12)
    np.testing.assert_allclose(f[1], 1.0, atol=1e-14)
    # assignment is the transpose of interpolation: <assign(w), g> = sum_p w_p g(x_p)
    g = rng.standard_normal((1, n, n, n))
    w = rng.uniform(0.5, 2.0, 40)
    eps, _ = O.assign(pos, w, n, box, dsup)
    lhs = float((eps * g[0]).sum())
    rhs = float((w * O.interpolate(g, pos, n, box, dsup)[0]).sum())
    assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(lhs))


# --- jbar -----------------------------------------------------------------------------
def test_jbar_l0_closed_form_and_k0():
    r_lo, r_hi = 10.0, 20.0
    k = np.linspace(0.0, 2.0, 401)[1:]
    x_hi, x_lo = k * r_hi, k * r_lo
    closed = 3.0 * ((np.sin(x_hi) - x_hi * np.cos(x_hi)) - (np.sin(x_lo) - x_lo * np.cos(x_lo))) / (
        k ** 3 * (r_hi ** 3 - r_lo ** 3))
    np.testing.assert_allclose(O.jbar(0, k, r_lo, r_hi), closed, rtol=0, atol=1e-13)
    for ell in range(0, 11):
        assert abs(O.jbar(ell, np.array([0.0]), r_lo, r_hi)[0] - (1.0 if ell == 0 else 0.0)) < 1e-15


def test_jbar_against_adaptive_quadrature_and_small_k():
    r_lo, r_hi = 5.0, 14.75
    den = (r_hi ** 3 - r_lo ** 3) / 3.0
    for ell in range(0, 15, 3):
        for kk in (0.01, 0.3, 1.1, 2.4):
            # for high l at small k the integrand is ~1e-30 and quad warns that it cannot reach
            # epsabs; the comparison below holds with the absolute floor all the same
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", integrate.IntegrationWarning)
                ref, _ = integrate.quad(lambda r: r * r * special.spherical_jn(ell, kk * r), r_lo, r_hi,
                                        epsabs=1e-15, epsrel=1e-13, limit=200)
            got = O.jbar(ell, np.array([kk]), r_lo, r_hi)[0]
            assert abs(got - ref / den) < 1e-12 * max(1.0, abs(ref / den)) + 1e-16
    # small-k limit: j_l(x) ~ x^l / (2l+1)!!
    kk = 1e-4
    for ell in range(1, 6):
        dfact = float(np.prod(np.arange(1, 2 * ell + 2, 2)))
        lim = kk ** ell / dfact * (r_hi ** (ell + 3) - r_lo ** (ell + 3)) / (ell + 3) / den
        got = O.jbar(ell, np.array([kk]), r_lo, r_hi)[0]
        assert abs(got / lim - 1.0) < 1e-6


# --- real_ylm ---------------------------------------------------------------------------
def test_real_ylm_l1_explicit_and_north_pole():
    rng = np.random.default_rng(4)
    v = rng.standard_normal((100, 3))
    r = np.linalg.norm(v, axis=1)
    c = math.sqrt(3.0 / (4.0 * math.pi))
    np.testing.assert_allclose(O.real_ylm(1, 1, *v.T), c * v[:, 0] / r, atol=1e-14)
    np.testing.assert_allclose(O.real_ylm(1, -1, *v.T), c * v[:, 1] / r, atol=1e-14)
    np.testing.assert_allclose(O.real_ylm(1, 0, *v.T), c * v[:, 2] / r, atol=1e-14)
    for ell in range(15):
        for m in range(-ell, ell + 1):
            val = O.real_ylm(ell, m, 0.0, 0.0, 2.0)
            want = math.sqrt((2 * ell + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert abs(val - want) < 1e-12
            assert O.real_ylm(ell, m, 0.0, 0.0, 0.0) == ((1 / math.sqrt(4 * math.pi)) if ell == 0 else 0.0)


def test_real_ylm_addition_theorem_and_orthonormality():
    rng = np.random.default_rng(5)
    v = rng.standard_normal((300, 3))
    for ell in range(15):
        s = sum(O.real_ylm(ell, m, *v.T) ** 2 for m in range(-ell, ell + 1))
        np.testing.assert_allclose(s, (2 * ell + 1) / (4 * math.pi), rtol=1e-12)
    # orthonormality by Gauss-Legendre in cos(theta) x uniform phi (exact for l <= 6)
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = 2 * math.pi * np.arange(nphi) / nphi
    ct = np.repeat(xg, nphi)
    st = np.sqrt(1 - ct ** 2)
    ph = np.tile(phi, len(xg))
    wt = np.repeat(wg, nphi) * (2 * math.pi / nphi)
    vx, vy, vz = st * np.cos(ph), st * np.sin(ph), ct
    ylist = [(l, m) for l in range(7) for m in range(-l, l + 1)]
    Y = np.array([O.real_ylm(l, m, vx, vy, vz) for l, m in ylist])
    gram = (Y * wt) @ Y.T
    np.testing.assert_allclose(gram, np.eye(len(ylist)), atol=1e-13)


def test_rotation_average_identity_monte_carlo():
    """Eq. (double-e-expansion): the rotation average of exp(i k1.r1) exp(i k2.r2) equals
    sum_l [sum_m W_lm(k1) W_lm(k2)] P_l(r1.r2) with W_lm = sqrt(4pi) i^l j_l R_lm (reading R1)."""
    from scipy.spatial.transform import Rotation
    k1, k2 = np.array([0.9, 0.3, -0.4]), np.array([0.7, 0.5, -0.1])
    r1, r2 = np.array([1.0, 1.5, 0.5]), np.array([0.8, 1.9, 0.9])
    rots = Rotation.random(400_000, random_state=6).as_matrix()
    q1 = np.einsum("nij,j->ni", rots, r1)
    q2 = np.einsum("nij,j->ni", rots, r2)
    samples = np.exp(1j * (q1 @ k1 + q2 @ k2))
    mc = samples.mean()
    sem = math.sqrt(samples.real.var() / len(samples))
    series = 0.0
    mu_r = r1 @ r2 / (np.linalg.norm(r1) * np.linalg.norm(r2))
    for ell in range(30):
        w1 = math.sqrt(4 * math.pi) * (1j ** ell) * special.spherical_jn(ell, np.linalg.norm(k1) * np.linalg.norm(r1))
        w2 = math.sqrt(4 * math.pi) * (1j ** ell) * special.spherical_jn(ell, np.linalg.norm(k2) * np.linalg.norm(r2))
        pair = sum(w1 * O.real_ylm(ell, m, *k1) * w2 * O.real_ylm(ell, m, *k2) for m in range(-ell, ell + 1))
        series += pair * special.eval_legendre(ell, mu_r)
    assert abs(series.imag) < 1e-14
    assert abs(mc.real - series.real) < 5 * sem
    assert abs(mc.imag) < 5 * sem
    # the odd multipoles matter here: flipping their sign moves the series well outside the noise
    odd = 0.0
    for ell in range(1, 30, 2):
        j1 = special.spherical_jn(ell, np.linalg.norm(k1) * np.linalg.norm(r1))
        j2 = special.spherical_jn(ell, np.linalg.norm(k2) * np.linalg.norm(r2))
        mu_k = k1 @ k2 / (np.linalg.norm(k1) * np.linalg.norm(k2))
        odd += -(2 * ell + 1) * special.eval_legendre(ell, mu_k) * special.eval_legendre(ell, mu_r) * j1 * j2
    assert abs(2 * odd) > 10 * sem


# --- window_kernel / multipole_fields / sum_node: Fourier triad closed form --------------
def _triad_delta(n, modes, amps, phases):
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    d = np.zeros((n, n, n))
    for (mx, my, mz), A, ph in zip(modes, amps, phases):
        d += 2 * A * np.cos(2 * math.pi * (mx * lx + my * ly + mz * lz) / n + ph)
    return d


def test_triad_closed_form_node_sum():
    n, box, lmax = 16, 100.0, 3
    edges = np.array([8.0, 20.0, 37.0])
    modes = [(1, 2, 0), (-3, 1, 2)]
    modes.append(tuple(-(a + b) for a, b in zip(*modes)))
    amps, phases = (0.7, 1.1, 0.9), (0.3, -1.2, 2.0)
    # no other zero-sum triple of the six modes (mod n)
    allm = [np.array(m) for m in modes] + [-np.array(m) for m in modes]
    zero_sum = 0
    for i in range(6):
        for j in range(6):
            for k in range(6):
                if not np.any((allm[i] + allm[j] + allm[k]) % n):
                    zero_sum += 1
    assert zero_sum == 12  # the 3! orderings of (k1, k2, k3) and of their negatives
    delta = _triad_delta(n, modes, amps, phases)
    zeta, _ = O.zeta_from_delta(delta, n, box, edges, lmax, 2, forms=("node",))
    kv = [2 * math.pi / box * np.array(m, float) for m in modes]
    pref = 2 * np.prod(amps) * math.cos(sum(phases))
    for ell in range(lmax + 1):
        want = np.zeros((2, 2))
        for b1 in range(2):
            for b2 in range(2):
                s = 0.0
                for a1 in range(3):
                    for a2 in range(3):
                        if a1 == a2:
                            continue
                        j1 = O.jbar(ell, np.array([np.linalg.norm(kv[a1])]), edges[b1], edges[b1 + 1])[0]
                        j2 = O.jbar(ell, np.array([np.linalg.norm(kv[a2])]), edges[b2], edges[b2 + 1])[0]
                        mu = kv[a1] @ kv[a2] / (np.linalg.norm(kv[a1]) * np.linalg.norm(kv[a2]))
                        s += j1 * j2 * special.eval_legendre(ell, mu)
                want[b1, b2] = pref * (-1) ** ell * (2 * ell + 1) * s
        np.testing.assert_allclose(zeta["node"][ell], want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))


# --- vertex windows: tophat, point radius, basis power spectrum, primary tophat ---------------
def test_tophat_window_is_the_average_over_a_ball():
    """W_TH(kR) is the mean of exp(i k.x) over the uniform ball of radius R (Monte Carlo)."""
    rng = np.random.default_rng(31)
    npts = 400_000
    v = rng.standard_normal((npts, 3))
    v *= (rng.random(npts) ** (1.0 / 3.0) / np.linalg.norm(v, axis=1))[:, None]  # uniform in the unit ball
    for kr in (0.3, 2.0, 4.4934, 7.0):
        kvec = np.array([0.3, -0.5, 0.8])
        kvec *= kr / np.linalg.norm(kvec)
        samples = np.cos(v @ kvec)
        sem = samples.std() / math.sqrt(npts)
        assert abs(samples.mean() - float(O.tophat_window(kr))) < 5 * sem + 1e-12, kr
    assert float(O.tophat_window(0.0)) == 1.0
    np.testing.assert_allclose(O.tophat_window(np.array([1e-3, 5e-3])),
                               3 * (np.sin([1e-3, 5e-3]) - np.array([1e-3, 5e-3]) * np.cos([1e-3, 5e-3]))
                               / np.array([1e-3, 5e-3]) ** 3, rtol=1e-6)


def test_point_radius_is_the_thin_shell_limit():
    """The point-radius window j_l(k r) is the limit of the shell average over [r - e, r + e):
    the difference falls as e^2."""
    k = np.array([0.05, 0.31, 0.9])
    r = 23.0
    for ell in (0, 1, 4):
        want = O.radial_window(ell, k, 0, None, {"radial": "point", "radii": [r]})
        np.testing.assert_allclose(want, special.spherical_jn(ell, k * r), rtol=1e-14)
        errs = [np.abs(O.jbar(ell, k, r - e, r + e) - want).max() for e in (1.0, 0.5, 0.25)]
        assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, (ell, errs)


@pytest.mark.parametrize("dsup", [2, 4])
def test_phi_hat_is_the_bspline_power_spectrum(dsup):
    """Phi-hat(n) = prod_d |beta-hat(2 pi n_d / n)|^2 with beta-hat the continuous Fourier transform of
    the B-spline (exact Gauss-Legendre quadrature per unit interval)."""
    n = 16
    half = dsup // 2

    def bhat(q):
        return O._unit_interval_quadrature(lambda u: O.bspline(u, dsup) * np.cos(q * u), -half, half, nq=16)

    iv = O.fft_integers(n)
    one = np.array([bhat(2 * math.pi * f / n) ** 2 for f in iv])
    want = one[:, None, None] * one[None, :, None] * one[None, None, :]
    np.testing.assert_allclose(O.phi_hat(n, dsup), want, rtol=1e-12, atol=1e-15)


def test_triad_closed_form_with_vertex_windows():
    """The Fourier-triad closed form with every vertex window on: point radii, a secondary-vertex
    tophat, Phi-hat and a primary-vertex tophat, node and Gamma forms' primary."""
    n, box, lmax, dsup = 16, 100.0, 3, 2
    radii = [13.0, 29.0]
    rt, rp = 9.0, 6.0
    vertex = {"radial": "point", "radii": radii, "tophat": rt, "phi_dsup": dsup}
    modes = [(1, 2, 0), (-3, 1, 2)]
    modes.append(tuple(-(a + b) for a, b in zip(*modes)))
    amps, phases = (0.7, 1.1, 0.9), (0.3, -1.2, 2.0)
    delta = _triad_delta(n, modes, amps, phases)
    zeta, _ = O.zeta_from_delta(delta, n, box, None, lmax, dsup, forms=("node",), vertex=vertex,
                                primary_tophat=rp)
    kv = [2 * math.pi / box * np.array(m, float) for m in modes]
    s1 = {f: np.sinc(f / n) ** (2 * dsup) for f in range(-n, n)}
    phi = [s1[m[0]] * s1[m[1]] * s1[m[2]] for m in modes]
    pref = 2 * np.prod(amps) * math.cos(sum(phases))
    for ell in range(lmax + 1):
        want = np.zeros((2, 2))
        for b1 in range(2):
            for b2 in range(2):
                tot = 0.0
                for a1 in range(3):
                    for a2 in range(3):
                        if a1 == a2:
                            continue
                        a3 = 3 - a1 - a2
                        k1, k2, k3 = (np.linalg.norm(kv[a]) for a in (a1, a2, a3))
                        v1 = special.spherical_jn(ell, k1 * radii[b1]) * O.tophat_window(k1 * rt) * phi[a1]
                        v2 = special.spherical_jn(ell, k2 * radii[b2]) * O.tophat_window(k2 * rt) * phi[a2]
                        mu = kv[a1] @ kv[a2] / (k1 * k2)
                        tot += v1 * v2 * float(O.tophat_window(k3 * rp)) * special.eval_legendre(ell, mu)
                want[b1, b2] = pref * (-1) ** ell * (2 * ell + 1) * tot
        np.testing.assert_allclose(zeta["node"][ell], want, rtol=0, atol=1e-12 * max(1.0, np.abs(want).max()))


# --- 2PCF, angular 3PCF and reduced 3PCF -------------------------------------------------
def test_xi_of_a_single_mode_is_the_shell_average_of_its_cosine():
    """For delta = 2A cos(k.x + phi) on the lattice, the node-form 2PCF of bin b is
    2A^2 jbar_0(|k|; b) (shell average of cos(k.r)); with a point radius 2A^2 j_0(|k| r); a primary
    and a secondary tophat each multiply by W_TH(|k| R)."""
    n, box = 16, 80.0
    edges = np.array([5.0, 11.0, 19.0])
    mode, amp, ph = (2, -1, 3), 0.8, 0.4
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    delta = 2 * amp * np.cos(2 * math.pi * (mode[0] * lx + mode[1] * ly + mode[2] * lz) / n + ph)
    k = 2 * math.pi / box * np.linalg.norm(mode)
    want = 2 * amp ** 2 * np.array([O.jbar(0, np.array([k]), edges[b], edges[b + 1])[0] for b in range(2)])
    np.testing.assert_allclose(O.xi_node(delta, n, box, edges), want, rtol=1e-12)
    v = {"radial": "point", "radii": [7.0, 15.0], "tophat": 4.0}
    want = 2 * amp ** 2 * special.spherical_jn(0, k * np.array([7.0, 15.0])) * O.tophat_window(k * 4.0) \
        * O.tophat_window(k * 3.0)
    np.testing.assert_allclose(O.xi_node(delta, n, box, None, vertex=v, primary_tophat=3.0), want, rtol=1e-12)


def test_xi_particle_form_on_nodes_reduces_to_the_node_form():
    """Hat basis with a particle of weight 1 + delta_l on every node: the particle-form 2PCF is the
    node-form one plus the mean of the field, which is zero."""
    n, box = 8, 64.0
    edges = np.array([9.0, 17.0, 27.0])
    rng = np.random.default_rng(12)
    d0 = rng.uniform(-0.7, 0.7, (n, n, n))
    d0 -= d0.mean()
    h = box / n
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    parts = np.stack([lx.ravel() * h, ly.ravel() * h, lz.ravel() * h, (1 + d0).ravel()], 1)
    np.testing.assert_allclose(O.xi_particle(parts, n, box, edges, 2), O.xi_node(d0, n, box, edges),
                               rtol=1e-11, atol=1e-14)


def test_legendre_sum_generating_function():
    """sum_l t^l P_l(mu) = (1 - 2 mu t + t^2)^(-1/2): with zeta_l = t^l the resummation is closed."""
    t, lmax = 0.45, 60
    mu = np.linspace(-1, 1, 41)
    zl = (t ** np.arange(lmax + 1))[:, None, None] * np.ones((1, 2, 2))
    got = O.legendre_sum(zl, mu)
    want = (1 - 2 * mu * t + t * t) ** -0.5
    np.testing.assert_allclose(got[:, 0, 1], want, rtol=1e-14)


def test_reduced_q_of_a_hierarchical_3pcf():
    xi1, xi2, xi3 = np.array([0.8]), np.array([0.3]), np.array([1.7])
    zeta = 1.3 * (xi1 * xi2 + xi2 * xi3 + xi3 * xi1)
    np.testing.assert_allclose(O.reduced_q(zeta, xi1, xi2, xi3), 1.3, rtol=1e-15)


def test_szapudi_szalay_with_lattice_randoms_reduces_to_the_plain_estimator():
    """Randoms on every node of the lattice (hat basis) have delta_R = 0 exactly, so the numerator
    is the plain measurement of delta_D and the denominator that of the constant 1 (1 for l = 0, 0
    above)."""
    n, box, lmax = 8, 64.0, 2
    edges = np.array([9.0, 17.0, 27.0])
    h = box / n
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    lattice = np.stack([lx.ravel() * h, ly.ravel() * h, lz.ravel() * h, np.full(n ** 3, 2.5)], 1)
    data = _small_catalogue(21, n_p=900, box=box)
    num, den = O.zeta_szapudi_szalay(data, lattice, n, box, edges, lmax, 2, forms=("node", "gamma"))
    plain, _ = O.zeta_multipoles(data, n, box, edges, lmax, 2, forms=("node", "gamma"))
    for f in ("node", "gamma"):
        np.testing.assert_allclose(num[f], plain[f], rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(den[f][0], 1.0, rtol=1e-13)
        np.testing.assert_allclose(den[f][1:], 0.0, atol=1e-13)


def test_constant_field_gives_c_cubed():
    n, box = 8, 50.0
    edges = np.array([6.0, 12.0, 20.0])
    c = 1.7
    delta = np.full((n, n, n), c)
    zeta, _ = O.zeta_from_delta(delta, n, box, edges, 2, 2, forms=("node", "gamma"))
    for f in ("node", "gamma"):
        np.testing.assert_allclose(zeta[f][0], c ** 3, rtol=1e-13)
        np.testing.assert_allclose(zeta[f][1:], 0.0, atol=1e-13)


# --- sum_gamma: exact per-cell Gauss-Legendre quadrature of (1/V) int n_rec f1 f2 ----------
@pytest.mark.parametrize("dsup,q", [(2, 2), (4, 5)])
def test_sum_gamma_equals_cell_quadrature(dsup, q):
    n = 8
    rng = np.random.default_rng(7)
    delta = rng.standard_normal((n, n, n))
    a = rng.standard_normal((2, n, n, n))
    got = O.sum_gamma(delta, a, dsup)
    xg, wg = np.polynomial.legendre.leggauss(q)
    t = 0.5 + 0.5 * xg  # nodes inside a unit cell
    wq = 0.5 * wg
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cells = np.stack([lx.ravel(), ly.ravel(), lz.ravel()], 1).astype(float)
    want = np.zeros((2, 2))
    fields = np.concatenate([delta[None], a])
    for iz in range(q):
        for iy in range(q):
            for ix in range(q):
                pts = cells + np.array([t[ix], t[iy], t[iz]])  # grid units, box = n
                vals = O.interpolate(fields, pts, n, float(n), dsup)
                wgt = wq[ix] * wq[iy] * wq[iz] * vals[0]
                want += (vals[1:] * wgt) @ vals[1:].T
    want /= n ** 3
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)


# --- sum_particles / interpolate / assign: hat basis with a particle on every node ---------
def test_particle_form_on_nodes_reduces_to_node_form():
    n, box, lmax = 8, 64.0, 2
    edges = np.array([10.0, 18.0, 28.0])
    rng = np.random.default_rng(8)
    d0 = rng.uniform(-0.8, 0.8, (n, n, n))
    d0 -= d0.mean()
    h = box / n
    lz, ly, lx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    parts = np.stack([lx.ravel() * h, ly.ravel() * h, lz.ravel() * h, (1 + d0).ravel()], 1)
    eps, wsum = O.assign(parts[:, :3], parts[:, 3], n, box, 2)
    np.testing.assert_allclose(O.contrast(eps, wsum), d0, atol=1e-13)
    zeta, _ = O.zeta_multipoles(parts, n, box, edges, lmax, 2, forms=("particle", "node"))
    dh = np.fft.fftn(d0)
    for ell in range(lmax + 1):
        extra = np.zeros((2, 2))
        for m in range(-ell, ell + 1):
            a = O.multipole_fields(dh, ell, m, n, box, edges)
            extra += O.sum_node(np.ones((n, n, n)), a) - O.mass_term(a, 2)
        np.testing.assert_allclose(zeta["particle"][ell], zeta["node"][ell] + 0.5 * (extra + extra.T),
                                   rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("dsup", [2, 4])
def test_mass_term_matches_fourier_space_form(dsup):
    """U summed over m equals (2l+1)/N_g^2 sum_n |delta_hat|^2 jbar_b1 jbar_b2 Mhat(n) (addition theorem)."""
    n, box, lmax = 12, 60.0, 3
    edges = np.array([7.0, 15.0, 24.0])
    rng = np.random.default_rng(9)
    delta = rng.standard_normal((n, n, n))
    dh = np.fft.fftn(delta)
    gold = _golden_mass()
    iv = O.fft_integers(n)
    mhat1 = np.array([gold[(dsup, 0)] + 2 * sum(gold[(dsup, a)] * math.cos(2 * math.pi * k * a / n)
                                                 for a in range(1, dsup)) for k in iv])
    nz, ny, nx = np.meshgrid(iv, iv, iv, indexing="ij")
    kmag = 2 * math.pi / box * np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
    keep = ~O.nyquist_mask(n)
    mh = mhat1[:, None, None] * mhat1[None, :, None] * mhat1[None, None, :]
    for ell in range(lmax + 1):
        u = np.zeros((2, 2))
        for m in range(-ell, ell + 1):
            u += O.mass_term(O.multipole_fields(dh, ell, m, n, box, edges), dsup)
        j = [O.jbar(ell, kmag, edges[b], edges[b + 1]) for b in range(2)]
        want = np.array([[(2 * ell + 1) * np.sum((np.abs(dh) ** 2 * j[b1] * j[b2] * mh)[keep])
                          for b2 in range(2)] for b1 in range(2)]) / n ** 6
        np.testing.assert_allclose(u, want, rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(O.mass_term_fourier(dh, ell, n, box, edges, dsup), u, rtol=1e-11, atol=1e-14)


# --- whole pipeline: symmetries and invariances ---------------------------------------------
def _small_catalogue(seed, n_p=600, box=60.0):
    rng = np.random.default_rng(seed)
    p = np.empty((n_p, 4))
    p[:, :3] = rng.uniform(0, box, (n_p, 3))
    p[:, 3] = rng.uniform(0.5, 1.5, n_p)
    return p


def test_zeta_symmetries_and_invariances():
    n, box, lmax, dsup = 12, 60.0, 2, 4
    edges = np.array([6.0, 14.0, 22.0, 29.0])
    p = _small_catalogue(10)
    forms = ("node", "particle")
    z0, _ = O.zeta_multipoles(p, n, box, edges, lmax, dsup, forms=forms)
    h = box / n
    moved = p.copy()
    moved[:, :3] = (moved[:, :3] + h * np.array([3, 5, 7])) % box
    perm = p.copy()
    perm[:, [0, 1, 2]] = p[:, [2, 0, 1]]
    refl = p.copy()
    refl[:, 1] = (box - p[:, 1]) % box
    scaled = p.copy()
    scaled[:, 3] *= 3.7
    for q in (moved, perm, refl, scaled):
        z1, _ = O.zeta_multipoles(q, n, box, edges, lmax, dsup, forms=forms)
        for f in forms:
            np.testing.assert_allclose(z1[f], z0[f], rtol=1e-10, atol=1e-12 * np.abs(z0[f]).max())
    for f in forms:
        np.testing.assert_allclose(z0[f], np.swapaxes(z0[f], 1, 2), atol=0)


@pytest.mark.slow
def test_poisson_null_is_consistent_with_zero():
    n, box, lmax, dsup = 12, 60.0, 2, 2
    edges = np.array([8.0, 16.0, 26.0])
    runs = []
    for s in range(32):
        rng = np.random.default_rng(1000 + s)
        p = np.empty((3000, 4))
        p[:, :3] = rng.uniform(0, box, (3000, 3))
        p[:, 3] = 1.0
        z, _ = O.zeta_multipoles(p, n, box, edges, lmax, dsup, forms=("particle", "node"))
        runs.append(np.concatenate([z["particle"].ravel(), z["node"].ravel()]))
    runs = np.array(runs)
    mean = runs.mean(0)
    sem = runs.std(0, ddof=1) / math.sqrt(len(runs))
    assert np.all(np.abs(mean) < 4.0 * sem + 1e-15)


# --- brute-force enumeration: three-point closed form, and convergence of the raw reading ----
def test_brute_force_three_points_closed_form():
    box = 100.0
    edges = np.array([5.0, 12.0, 20.0])
    pts = np.array([[50.0, 50.0, 50.0], [58.0, 50.0, 50.0], [50.0, 56.0, 57.0]])
    p = np.concatenate([pts, np.ones((3, 1))], 1)
    got = O.brute_force_raw(p, box, edges, 4)
    vb = 4 * math.pi / 3 * (edges[1:] ** 3 - edges[:-1] ** 3)
    want = np.zeros_like(got)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                if i in (j, k):
                    continue
                dj, dk = pts[j] - pts[i], pts[k] - pts[i]
                bj = np.searchsorted(edges, np.linalg.norm(dj), "right") - 1
                bk = np.searchsorted(edges, np.linalg.norm(dk), "right") - 1
                mu = dj @ dk / (np.linalg.norm(dj) * np.linalg.norm(dk))
                for ell in range(5):
                    want[ell, bj, bk] += (2 * ell + 1) * special.eval_legendre(ell, mu)
    want *= box ** 6 / (27.0 * np.outer(vb, vb))[None]
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)


@pytest.mark.slow
def test_raw_reading_converges_to_brute_force():
    box, lmax = 200.0, 2
    edges = np.array([12.0, 44.0, 84.0])
    base = np.array([100.0, 100.0, 100.0])
    offs = np.array([[0, 0, 0], [28, 0, 0], [14, 24.25, 0], [10, 8, 62], [-40, 30, 20]], float)
    p = np.concatenate([base + offs, np.ones((len(offs), 1))], 1)
    ref = O.brute_force_raw(p, box, edges, lmax)
    errs = []
    for n in (32, 64, 128):
        z, _ = O.zeta_multipoles(p, n, box, edges, lmax, 2, forms=("particle",), raw=True)
        errs.append(np.abs(z["particle"] - ref).max() / np.abs(ref).max())
    assert errs[2] < errs[1] < errs[0]
    assert errs[0] / errs[2] > 2.5


# --- gradients: central finite differences of the FP64 loss --------------------------------
def test_bspline_derivative_matches_finite_difference():
    u = np.linspace(-2.3, 2.3, 97) + 1e-3
    for dsup in (2, 4):
        fd = (O.bspline(u + 1e-6, dsup) - O.bspline(u - 1e-6, dsup)) / 2e-6
        np.testing.assert_allclose(O.bspline_deriv(u, dsup), fd, atol=1e-6)


def test_node_gradient_matches_finite_differences():
    n, box, lmax = 8, 60.0, 2
    edges = np.array([7.0, 14.0, 22.0])
    rng = np.random.default_rng(21)
    delta = rng.standard_normal((n, n, n))
    wts = rng.standard_normal((lmax + 1, 2, 2))

    def lossf(d):
        z, _ = O.zeta_from_delta(d, n, box, edges, lmax, 2, forms=("node",))
        return O.loss(z["node"], wts)

    g = O.grad_node_delta(delta, wts, n, box, edges, lmax)
    for k in range(3):
        v = rng.standard_normal((n, n, n))
        e = 1e-4
        fd = (lossf(delta + e * v) - lossf(delta - e * v)) / (2 * e)
        assert abs(fd - float((g * v).sum())) < 1e-7 * max(1.0, abs(fd)), (fd, float((g * v).sum()))


def test_particle_position_gradient_matches_finite_differences():
    n, box, lmax, dsup = 8, 40.0, 2, 4
    edges = np.array([5.0, 10.0, 17.0])
    rng = np.random.default_rng(22)
    parts = np.empty((150, 4))
    parts[:, :3] = rng.uniform(0, box, (150, 3))
    parts[:, 3] = rng.uniform(0.5, 1.5, 150)
    wts = rng.standard_normal((lmax + 1, 2, 2))

    def lossf(p):
        z, _ = O.zeta_multipoles(p, n, box, edges, lmax, dsup, forms=("particle",))
        return O.loss(z["particle"], wts)

    g = O.grad_particle_positions(parts, wts, n, box, edges, lmax, dsup)
    for pi, d in [(0, 0), (3, 1), (17, 2), (88, 0), (149, 2)]:
        e = 1e-4
        pp, pm = parts.copy(), parts.copy()
        pp[pi, d] += e
        pm[pi, d] -= e
        fd = (lossf(pp) - lossf(pm)) / (2 * e)
        assert abs(fd - g[pi, d]) < 1e-6 * max(1.0, np.abs(g).max()), (pi, d, fd, g[pi, d])
