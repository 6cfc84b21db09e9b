"""Plain FP64 CPU oracle for the in-situ multipole 3PCF of Ju et al. (2025),
"An Optimal In-Situ Multipole Algorithm for the Isotropic Three-Point
Correlation Function" (arXiv:2507.15209).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls, links
or executes this module: only the test-suite, the smoke check and the
benchmark's CPU-baseline leg do.  It shares no code with the CUDA library and
takes every input (particles, grids, bin edges) as plain arrays.

Each function restates one step of the method in the order of the paper's
Sec. 2 and Fig. 1, with numpy / scipy library primitives (FFT, special
functions, matmul, bincount) as the only building blocks.  Everything is
float64.

Readings taken where the paper is silent, ambiguous or garbled (each is also
listed in the design notes):
  R1  Eq. (double-e-expansion) drops a conjugate; we use real orthonormal
      spherical harmonics R_lm with i^l in both vertex windows, so the pair
      product is sum_m a_lm,b1 a_lm,b2 of real fields.
  R2  DFT conventions: forward unnormalised e^{-2 pi i n.l/N}; inverse carries
      1/N_g; k_n = 2 pi n / L_box with n_d in (-N/2, N/2).
  R3  The basis window Phi-hat of Eq. (SFC-3PCF-vertex) is 1 (the translation
      kernel is the lattice-sampled shell harmonic only).
  R4  Radial binning: the vertex window is the r^2-weighted shell average
      jbar_l(k; b) = int r^2 j_l(kr) dr / int r^2 dr over [r_lo, r_hi).
  R5  Every Nyquist plane (any n_d = N/2) of the kernel is zero; at k = 0,
      R_00 = 1/sqrt(4 pi) and R_{l>0} = 0.
  R6  The SFCs are B-spline expansion coefficients assigned from the points,
      eps_l = sum_p w_p beta(x_p/H - l); contrast delta = eps/eps_bar - 1 with
      eps_bar = W/N_g (Sec. 3 uses the contrast in a periodic box).
  R7  Particle form, Eq. (DDD-sum-privertex) with the primary vertex carried
      by delta = n/n_bar - 1: zeta = (1/W) sum_p w_p sum_m f_b1 f_b2 - U, where
      U = (1/V) int sum_m f_b1 f_b2 dx is the "-1" (uniform) term.
  R8  No self-triplet or shot-noise subtraction (the paper's formulas have none).
  R9  dsup = 3 selects the Daubechies scaling function of genus 4 (four filter taps,
      support [0, 3]; Sec. 2.2 and the runtime benchmark of Sec. 3).  It is known only
      through its two-scale relation phi(x) = sqrt2 sum_k h_k phi(2x - k): its point values
      are the exact dyadic values of level DAUB_LEVEL = 10 joined linearly (what a cascade
      table of that level holds), while its mass and connection coefficients and its
      Fourier transform are those of phi itself, solved from the same relation.

Parity pins of each function live in tests/test_oracle_pins.py; none of the
functions below is unpinned.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

__all__ = [
    "bspline", "daub4_filter", "daub4_dyadic", "daub4_phi", "daub4_power", "daub4_mass", "daub4_gamma",
    "basis", "stencil_base", "assign", "contrast", "fft_integers", "nyquist_mask",
    "jbar", "real_ylm", "tophat_window", "phi_hat", "radial_window", "primary_filter", "window_kernel", "multipole_fields", "sum_node",
    "gamma_1d", "mass_1d", "sum_gamma", "interpolate", "sum_particles",
    "mass_term", "mass_term_fourier", "zeta_multipoles", "xi_node", "xi_particle", "legendre_sum", "reduced_q",
    "zeta_szapudi_szalay", "zeta_from_delta", "brute_force_raw",
    "bspline_deriv", "interpolate_grad", "loss", "grad_node_delta", "grad_particle_positions",
]

FOUR_PI = 4.0 * math.pi


# ---------------------------------------------------------------------------
# Sec. 2.1: multiresolution basis.  The scaling function is the centred
# cardinal B-spline of order D (support D cells): D=2 linear hat, D=4 cubic.
# ---------------------------------------------------------------------------
def bspline(u, dsup: int):
    """beta_D(u), the centred B-spline of order dsup (dsup in {2, 4})."""
    a = np.abs(np.asarray(u, dtype=np.float64))
    if dsup == 2:
        return np.where(a < 1.0, 1.0 - a, 0.0)
    if dsup == 4:
        inner = 2.0 / 3.0 - a * a + 0.5 * a ** 3
        outer = (2.0 - a) ** 3 / 6.0
        return np.where(a < 1.0, inner, np.where(a < 2.0, outer, 0.0))
    raise ValueError("dsup must be 2 or 4")


# ---------------------------------------------------------------------------
# The Daubechies scaling function of genus D_g = 4 (Sec. 2.2: support D_sup = D_g - 1 = 3;
# the basis of the paper's runs), selected by dsup = 3 (reading R9).
# ---------------------------------------------------------------------------
DAUB_LEVEL = 10
_SQRT2 = math.sqrt(2.0)
_DYADIC = {}


def daub4_filter():
    """Low-pass taps h_0..h_3 of the genus-4 Daubechies filter: (1+s, 3+s, 3-s, 1-s) / (4 sqrt2), s = sqrt3."""
    s3 = math.sqrt(3.0)
    return np.array([1.0 + s3, 3.0 + s3, 3.0 - s3, 1.0 - s3]) / (4.0 * _SQRT2)


def daub4_dyadic(level: int = DAUB_LEVEL):
    """phi(k / 2^level) for k = 0 .. 3 * 2^level, from the two-scale relation.

    Level 0: phi(0) = phi(3) = 0, and (phi(1), phi(2)) is the eigenvector of eigenvalue 1 of the
    relation restricted to the integers, scaled to sum 1 (partition of unity).  Level j+1: the
    even points are those of level j; an odd point k / 2^(j+1) takes
    phi = sqrt2 sum_i h_i phi(k / 2^j - i), whose arguments are points of level j.
    """
    if level not in _DYADIC:
        h = daub4_filter()
        t = _SQRT2 * np.array([[h[1], h[0]], [h[3], h[2]]])
        ev, vec = np.linalg.eig(t)
        v = vec[:, int(np.argmin(np.abs(ev - 1.0)))].real
        v = v / v.sum()
        vals = np.array([0.0, v[0], v[1], 0.0])
        for j in range(level):
            m = 3 * 2 ** (j + 1)
            new = np.zeros(m + 1)
            new[0::2] = vals
            odd = np.arange(1, m, 2)
            for i, hi in enumerate(h):
                src = odd - i * 2 ** j  # level-j index of k / 2^j - i
                ok = (src >= 0) & (src <= 3 * 2 ** j)
                new[odd[ok]] += _SQRT2 * hi * vals[src[ok]]
            vals = new
        _DYADIC[level] = vals
    return _DYADIC[level]


def daub4_phi(u, level: int = DAUB_LEVEL):
    """phi(u): the dyadic values of the given level joined linearly, zero outside [0, 3] (R9)."""
    tab = daub4_dyadic(level)
    x = np.arange(tab.size, dtype=np.float64) / 2.0 ** level
    return np.interp(np.asarray(u, np.float64), x, tab, left=0.0, right=0.0)


def daub4_power(omega):
    """|phi-hat(omega)|^2 = prod_{j >= 1} |m0(omega / 2^j)|^2 with m0(w) = (1/sqrt2) sum_k h_k e^{-i k w}
    (the Fourier transform of the two-scale relation); the factors left once |omega| / 2^j < 1e-6
    differ from 1 by less than 1e-22 (m0 has two vanishing moments)."""
    h = daub4_filter()
    w = np.asarray(omega, np.float64) / 2.0
    out = np.ones_like(w)
    while w.size and np.max(np.abs(w)) > 1e-6:
        m0 = sum(hk * np.exp(-1j * k * w) for k, hk in enumerate(h)) / _SQRT2
        out = out * np.abs(m0) ** 2
        w = w / 2.0
    return out


def _two_scale_solve(offsets, rows, norm_rows, norm_rhs):
    """Least-squares solution of (T - I) x = 0 stacked with the normalisation rows."""
    idx = {o: i for i, o in enumerate(offsets)}
    a = np.zeros((len(offsets), len(offsets)))
    for o in offsets:
        for o2, c in rows(o):
            if o2 in idx:
                a[idx[o], idx[o2]] += c
        a[idx[o], idx[o]] -= 1.0
    lhs = np.vstack([a, norm_rows(idx)])
    rhs = np.concatenate([np.zeros(len(offsets)), norm_rhs])
    x, *_ = np.linalg.lstsq(lhs, rhs, rcond=None)
    return {o: float(x[idx[o]]) for o in offsets}


def daub4_mass():
    """M(a) = int phi(x) phi(x - a) dx for |a| <= 2, from M(a) = sum_{i,j} h_i h_j M(2a + j - i)
    (substitute the two-scale relation twice) and sum_a M(a) = int phi = 1."""
    h = daub4_filter()
    offs = list(range(-2, 3))

    def rows(a):
        return [(2 * a + j - i, h[i] * h[j]) for i in range(4) for j in range(4)]

    return _two_scale_solve(offs, rows, lambda idx: np.ones((1, len(offs))), np.array([1.0]))


def daub4_gamma():
    """Gamma(a, b) = int phi(x) phi(x - a) phi(x - b) dx (Eq. con-coeff in 1-D) for the 23 pairs
    whose supports overlap, from Gamma(a, b) = sqrt2 sum_{i,j,k} h_i h_j h_k
    Gamma(2a + j - i, 2b + k - i) and sum_b Gamma(a, b) = M(a) (partition of unity)."""
    h = daub4_filter()
    offs = [(a, b) for a in range(-2, 3) for b in range(-2, 3) if abs(a - b) < 3]
    mass = daub4_mass()

    def rows(ab):
        a, b = ab
        return [((2 * a + j - i, 2 * b + k - i), _SQRT2 * h[i] * h[j] * h[k])
                for i in range(4) for j in range(4) for k in range(4)]

    def norm_rows(idx):
        out = np.zeros((5, len(offs)))
        for (a, b), i in idx.items():
            out[a + 2, i] = 1.0
        return out

    return _two_scale_solve(offs, rows, norm_rows, np.array([mass[a] for a in range(-2, 3)]))


def basis(u, dsup: int):
    """The scaling function of the basis: beta_D for dsup 2 or 4, the Daubechies phi for dsup 3."""
    if dsup == 3:
        return daub4_phi(u)
    return bspline(u, dsup)


def stencil_base(u, dsup: int):
    """First node of the stencil of grid coordinate u: the dsup nodes l with basis(u - l) != 0
    (centred B-splines: floor(u) - (dsup/2 - 1); Daubechies, support [0, 3]: floor(u) - 2)."""
    if dsup == 3:
        return np.floor(u).astype(np.int64) - 2
    return np.floor(u).astype(np.int64) - (dsup // 2 - 1)


def assign(pos, w, n: int, box: float, dsup: int):
    """SFCs of the point process, Sec. 2.1 and Fig. 1 step (2) (reading R6).

    eps_l = sum_p w_p prod_d phi(u_pd - l_d), periodic in l; u = x / H; phi the basis function.
    Returns (eps[z, y, x], W = sum_p w_p).
    """
    pos = np.asarray(pos, np.float64)
    w = np.asarray(w, np.float64)
    u = pos / (box / n)
    base = stencil_base(u, dsup)
    eps = np.zeros(n ** 3)
    for oz in range(dsup):
        lz = base[:, 2] + oz
        bz = basis(u[:, 2] - lz, dsup)
        for oy in range(dsup):
            ly = base[:, 1] + oy
            by = basis(u[:, 1] - ly, dsup)
            for ox in range(dsup):
                lx = base[:, 0] + ox
                bx = basis(u[:, 0] - lx, dsup)
                idx = ((lz % n) * n + (ly % n)) * n + (lx % n)
                eps += np.bincount(idx, weights=w * bx * by * bz, minlength=n ** 3)
    return eps.reshape(n, n, n), float(w.sum())


def contrast(eps, wsum: float):
    """delta = eps / eps_bar - 1 with eps_bar = W / N_g (Sec. 3, periodic box)."""
    return eps / (wsum / eps.size) - 1.0


# ---------------------------------------------------------------------------
# Sec. 2.1-2.2: DFT wavevectors and the multipole window of
# Eq. (3PCF-multipole-window) with radial binning (Sec. 2.2, binning windows).
# ---------------------------------------------------------------------------
def fft_integers(n: int):
    """Integer wavenumber of each DFT index: i for i < n/2, i - n otherwise."""
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n)


def nyquist_mask(n: int):
    """True on every plane where some axis index equals n/2 (reading R5)."""
    i = np.arange(n) == n // 2
    return i[:, None, None] | i[None, :, None] | i[None, None, :]


def jbar(ell: int, k, r_lo: float, r_hi: float, nq: int = 32):
    """r^2-weighted shell average of j_l(k r) over [r_lo, r_hi) (reading R4).

    Gauss-Legendre quadrature on sub-intervals short enough that the
    integrand is resolved at the largest k supplied.
    """
    k = np.asarray(k, np.float64)
    kmax = float(k.max()) if k.size else 0.0
    nsub = max(1, int(math.ceil(kmax * (r_hi - r_lo) / 2.0)))
    xg, wg = np.polynomial.legendre.leggauss(nq)
    edges = np.linspace(r_lo, r_hi, nsub + 1)
    num = np.zeros_like(k)
    for a, b in zip(edges[:-1], edges[1:]):
        half = 0.5 * (b - a)
        r = 0.5 * (a + b) + half * xg
        jl = special.spherical_jn(ell, k[..., None] * r)
        num += half * np.sum(wg * r * r * jl, axis=-1)
    den = (r_hi ** 3 - r_lo ** 3) / 3.0
    return num / den


def _sph_harm_complex(ell: int, m: int, theta, phi):
    if hasattr(special, "sph_harm_y"):
        return special.sph_harm_y(ell, m, theta, phi)
    return special.sph_harm(m, ell, phi, theta)  # older scipy: (order, degree, azimuth, polar)


def real_ylm(ell: int, m: int, vx, vy, vz):
    """Real orthonormal spherical harmonic R_lm of the direction of (vx, vy, vz).

    R_l0 = Y_l^0;  R_lm = sqrt2 (-1)^m Re Y_l^m (m > 0);  R_lm = sqrt2 (-1)^m Im Y_l^|m| (m < 0),
    i.e. sqrt2 N_lm P_l^|m|(cos theta) {cos, sin}(|m| phi) without the Condon-Shortley
    phase.  The zero vector gets R_00 = 1/sqrt(4 pi) and 0 otherwise (reading R5).
    """
    vx = np.asarray(vx, np.float64)
    vy = np.asarray(vy, np.float64)
    vz = np.asarray(vz, np.float64)
    r = np.sqrt(vx * vx + vy * vy + vz * vz)
    safe = np.where(r > 0, r, 1.0)
    theta = np.arccos(np.clip(vz / safe, -1.0, 1.0))
    phi = np.arctan2(vy, vx)
    y = _sph_harm_complex(ell, abs(m), theta, phi)
    if m > 0:
        out = math.sqrt(2.0) * (-1.0) ** m * y.real
    elif m < 0:
        out = math.sqrt(2.0) * (-1.0) ** (-m) * y.imag
    else:
        out = y.real
    zero_val = 1.0 / math.sqrt(FOUR_PI) if ell == 0 else 0.0
    return np.where(r > 0, out, zero_val)


def _grid_integers(n: int):
    iv = fft_integers(n)
    nz, ny, nx = np.meshgrid(iv, iv, iv, indexing="ij")
    return nx, ny, nz


def tophat_window(x):
    """W_TH(x) = 3 (sin x - x cos x) / x^3, x = k R: the Fourier transform of the uniform ball of
    radius R (unit volume integral), the vertex binning window of Sec. 3 (spherical tophat)."""
    x = np.asarray(x, np.float64)
    small = np.abs(x) < 1e-2
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    x2 = x * x
    return np.where(small, 1.0 - x2 / 10.0 + x2 * x2 / 280.0, w)


def phi_hat(n: int, dsup: int):
    """Phi-hat(n) = prod_d sinc^{2 dsup}(pi n_d / n), the power spectrum |beta-hat|^2 of the
    B-spline basis at the lattice wavevectors, without the aliasing sum (Fig. 1 step (3) and
    Eq. SFC-3PCF-vertex; reading: the aliasing images are dropped as the paper's delta_{m,n}
    does).  Full DFT grid [z, y, x].  dsup = 3: |phi-hat|^2 of the Daubechies function
    (daub4_power at 2 pi n_d / n)."""
    if dsup == 3:
        s1 = daub4_power(2.0 * math.pi * fft_integers(n) / n)
    else:
        s1 = np.sinc(fft_integers(n) / n) ** (2 * dsup)
    return s1[:, None, None] * s1[None, :, None] * s1[None, None, :]


def radial_window(ell: int, k, b: int, edges, vertex=None):
    """The radial factor of the vertex window of bin b at wavenumbers k.

    vertex["radial"] == "shell" (default): jbar_l(k; [edges[b], edges[b+1])) (reading R4);
    "point": j_l(k r_b) with r_b = vertex["radii"][b], the spherical shell of Eq.
    (3PCF-multipole-window) itself (the paper's triangle sides R_A, R_B).  A vertex["tophat"]
    radius R > 0 multiplies by the spherical tophat W_TH(k R) (Sec. 3 binning)."""
    vertex = vertex or {}
    k = np.asarray(k, np.float64)
    if vertex.get("radial", "shell") == "point":
        out = special.spherical_jn(ell, k * float(vertex["radii"][b]))
    else:
        out = jbar(ell, k, edges[b], edges[b + 1])
    if vertex.get("tophat", 0.0) > 0.0:
        out = out * tophat_window(k * float(vertex["tophat"]))
    return out


def window_kernel(ell: int, m: int, n: int, box: float, edges, bins=None, vertex=None):
    """K_lm,b(n) = sqrt(4 pi) i^l W_l,b(|k_n|) R_lm(k_n-hat) [Phi-hat(n)], Nyquist planes zero.

    Eq. (3PCF-multipole-window) with the radial factor of radial_window (the bin average of
    reading R4 by default) and, when vertex["phi_dsup"] = D > 0, the basis power spectrum
    Phi-hat of Eq. (SFC-3PCF-vertex).  Returns complex array (len(bins), n, n, n) over the full
    DFT grid [z, y, x]; bins defaults to every bin.
    """
    vertex = vertex or {}
    nx, ny, nz = _grid_integers(n)
    n2 = nx * nx + ny * ny + nz * nz
    uniq, inv = np.unique(n2, return_inverse=True)
    kmag = 2.0 * math.pi / box * np.sqrt(uniq.astype(np.float64))
    ang = real_ylm(ell, m, nx, ny, nz)
    if vertex.get("phi_dsup", 0):
        ang = ang * phi_hat(n, vertex["phi_dsup"])
    ny_mask = nyquist_mask(n)
    nbins = len(vertex["radii"]) if vertex.get("radial") == "point" else len(edges) - 1
    bins = list(range(nbins)) if bins is None else list(bins)
    out = np.empty((len(bins), n, n, n), np.complex128)
    for i, b in enumerate(bins):
        jb = radial_window(ell, kmag, b, edges, vertex)[inv].reshape(n2.shape)
        kern = math.sqrt(FOUR_PI) * (1j ** ell) * jb * ang
        kern[ny_mask] = 0.0
        out[i] = kern
    return out


def primary_filter(delta, n: int, box: float, radius: float):
    """The primary vertex smoothed by the spherical tophat of the given radius:
    IDFT[DFT(delta) W_TH(|k| R)] (the binning function W_p of Fig. 1 step (3)), with the
    Nyquist planes zero like every kernel of the method (reading R5)."""
    nx, ny, nz = _grid_integers(n)
    kmag = 2.0 * math.pi / box * np.sqrt((nx * nx + ny * ny + nz * nz).astype(np.float64))
    kern = tophat_window(kmag * radius)
    kern[nyquist_mask(n)] = 0.0
    return np.fft.ifftn(np.fft.fftn(delta) * kern).real


def multipole_fields(delta_hat, ell: int, m: int, n: int, box: float, edges, bins=None, vertex=None):
    """a_lm,b(l) = IDFT[delta_hat * K_lm,b], Eq. (SFC-3PCF-vertex), Fig. 1 step (5).

    The fields are real (readings R1, R5); returns float64 (len(bins), n, n, n).
    """
    kern = window_kernel(ell, m, n, box, edges, bins, vertex)
    out = np.empty(kern.shape, np.float64)
    for b in range(kern.shape[0]):
        a = np.fft.ifftn(delta_hat * kern[b])
        scale = max(1e-300, float(np.abs(a.real).max()))
        if float(np.abs(a.imag).max()) > 1e-9 * scale:
            raise AssertionError("multipole field is not real")
        out[b] = a.real
    return out


# ---------------------------------------------------------------------------
# Sec. 2.2: grid-based summation.
# ---------------------------------------------------------------------------
def sum_node(delta, a):
    """Node form: (1/N_g) sum_l delta_l a_b1(l) a_b2(l), Eq. (3PCF-multipole-sum) at one m."""
    nb = a.shape[0]
    af = a.reshape(nb, -1)
    return (af * delta.reshape(1, -1)) @ af.T / delta.size


def _unit_interval_quadrature(func, lo: int, hi: int, nq: int = 8):
    """int_lo^hi func(u) du for a function that is a polynomial on every unit interval."""
    xg, wg = np.polynomial.legendre.leggauss(nq)
    total = 0.0
    for k in range(lo, hi):
        u = k + 0.5 + 0.5 * xg
        total += 0.5 * float(np.sum(wg * func(u)))
    return total


def gamma_1d(dsup: int):
    """1-D connection coefficients gamma(a, b) = int phi(u) phi(u-a) phi(u-b) du.

    Eq. (con-coeff) factorises over axes: Gamma_{l1,l2} = prod_d gamma(l1_d, l2_d).
    Returns {(a, b): value} for |a|, |b| < dsup with a nonzero value (B-splines: exact
    piecewise-polynomial quadrature; Daubechies: the two-scale solution, daub4_gamma).
    """
    if dsup == 3:
        return daub4_gamma()
    half = dsup // 2
    out = {}
    for a in range(-(dsup - 1), dsup):
        for b in range(-(dsup - 1), dsup):
            v = _unit_interval_quadrature(
                lambda u: bspline(u, dsup) * bspline(u - a, dsup) * bspline(u - b, dsup), -half, half)
            if v != 0.0:
                out[(a, b)] = v
    return out


def mass_1d(dsup: int):
    """M(a) = int phi(u) phi(u - a) du for |a| < dsup (Daubechies: daub4_mass)."""
    if dsup == 3:
        return daub4_mass()
    half = dsup // 2
    return {a: _unit_interval_quadrature(lambda u: bspline(u, dsup) * bspline(u - a, dsup), -half, half)
            for a in range(-(dsup - 1), dsup)}


def _shift(a, off):
    """Periodic shift: out[..., l] = a[..., l + off], off given as (z, y, x)."""
    return np.roll(a, shift=(-off[0], -off[1], -off[2]), axis=(-3, -2, -1))


def sum_gamma(delta, a, dsup: int):
    """Connection-coefficient form, Eqs. (SFC-3PCF) and (3PCF-multipole-sum) at one m:

    (1/N_g) sum_l delta_l sum_{l1, l2} Gamma_{l1,l2} a_b1(l + l1) a_b2(l + l2).
    """
    g1 = gamma_1d(dsup)
    nb = a.shape[0]
    ng = delta.size
    cache = {}

    def shifted(off):
        if off not in cache:
            cache[off] = _shift(a, off).reshape(nb, -1)
        return cache[off]

    dflat = delta.reshape(1, -1)
    out = np.zeros((nb, nb))
    items = list(g1.items())
    for (pz, qz), vz in items:
        for (py, qy), vy in items:
            for (px, qx), vx in items:
                a1 = shifted((pz, py, px)) * dflat
                a2 = shifted((qz, qy, qx))
                out += (vz * vy * vx) * (a1 @ a2.T)
    return out / ng


# ---------------------------------------------------------------------------
# Sec. 2.2: particle-based summation, Eq. (DDD-sum-privertex) and the
# per-(L, M) densities n^LM(x, r) = sum_l eps~^LM_l phi_l(x).
# ---------------------------------------------------------------------------
def interpolate(a, pos, n: int, box: float, dsup: int):
    """f_b(x_p) = sum_l phi(u_p - l) a_b(l) (the basis expansion at each point)."""
    pos = np.asarray(pos, np.float64)
    u = pos / (box / n)
    base = stencil_base(u, dsup)
    nb = a.shape[0]
    af = a.reshape(nb, -1)
    f = np.zeros((nb, pos.shape[0]))
    for oz in range(dsup):
        lz = base[:, 2] + oz
        bz = basis(u[:, 2] - lz, dsup)
        for oy in range(dsup):
            ly = base[:, 1] + oy
            by = basis(u[:, 1] - ly, dsup)
            for ox in range(dsup):
                lx = base[:, 0] + ox
                bx = basis(u[:, 0] - lx, dsup)
                idx = ((lz % n) * n + (ly % n)) * n + (lx % n)
                f += (bx * by * bz)[None, :] * af[:, idx]
    return f


def sum_particles(a, pos, w, n: int, box: float, dsup: int):
    """(1/W) sum_p w_p f_b1(x_p) f_b2(x_p) at one (l, m) (reading R7, first term)."""
    w = np.asarray(w, np.float64)
    f = interpolate(a, pos, n, box, dsup)
    return (f * w[None, :]) @ f.T / float(w.sum())


def mass_term(a, dsup: int):
    """U = (1/V) int f_b1 f_b2 dx = (1/N_g) sum_{l,l'} a_b1(l) M3(l - l') a_b2(l') (reading R7)."""
    m1 = mass_1d(dsup)
    nb = a.shape[0]
    ng = a[0].size
    af = a.reshape(nb, -1)
    out = np.zeros((nb, nb))
    for dz, mz in m1.items():
        for dy, my in m1.items():
            for dx, mx in m1.items():
                out += (mz * my * mx) * (af @ _shift(a, (dz, dy, dx)).reshape(nb, -1).T)
    return out / ng


def mass_term_fourier(delta_hat, ell: int, n: int, box: float, edges, dsup: int, bins=None, vertex=None):
    """U summed over m for one l, in Fourier space (reading R7 with the addition theorem).

    The real-space form above is (1/N_g) a_b1^T M3 a_b2 with a_b = IDFT(delta_hat K_b); by
    Parseval it is (1/N_g^2) sum_n conj(K_b1) K_b2 |delta_hat|^2 Mhat(n), Mhat the DFT of the
    separable mass sequence M(a).  Summing R_lm R_lm over m gives (2l+1)/(4 pi) (the addition
    theorem, Eq. double-e-expansion-sep of the appendix), so
      U_l[b1][b2] = (2l+1)/N_g^2 sum_{n not Nyquist} |delta_hat(n)|^2 Mhat(n) jbar_l(k_n;b1) jbar_l(k_n;b2).
    Returns (len(bins), len(bins)).
    """
    m1 = mass_1d(dsup)
    iv = fft_integers(n)
    mhat1 = np.array([sum(v * math.cos(2.0 * math.pi * k * a / n) for a, v in m1.items()) for k in iv])
    nx, ny, nz = _grid_integers(n)
    n2 = nx * nx + ny * ny + nz * nz
    keep = ~nyquist_mask(n)
    vertex = vertex or {}
    p = np.abs(delta_hat) ** 2 * (mhat1[:, None, None] * mhat1[None, :, None] * mhat1[None, None, :])
    if vertex.get("phi_dsup", 0):
        p = p * phi_hat(n, vertex["phi_dsup"]) ** 2
    p = p[keep]
    n2k = n2[keep]
    uniq, inv = np.unique(n2k, return_inverse=True)
    psum = np.bincount(inv.ravel(), weights=p, minlength=len(uniq))  # |delta_hat|^2 Mhat per |n|^2
    kmag = 2.0 * math.pi / box * np.sqrt(uniq.astype(np.float64))
    nbins = len(vertex["radii"]) if vertex.get("radial") == "point" else len(edges) - 1
    bins = list(range(nbins)) if bins is None else list(bins)
    jb = np.stack([radial_window(ell, kmag, b, edges, vertex) for b in bins])
    return (2 * ell + 1) * (jb * psum[None, :]) @ jb.T / float(n) ** 6


# ---------------------------------------------------------------------------
# Fig. 1 steps (2)-(7): the whole multipole measurement.
# ---------------------------------------------------------------------------
def _symmetrise(x):
    return 0.5 * (x + np.swapaxes(x, -1, -2))


def zeta_from_delta(delta, n: int, box: float, edges, lmax: int, dsup: int,
                    forms=("node",), particles=None, raw_particle=False, vertex=None, primary_tophat=0.0):
    """zeta_l(b1, b2) for l <= lmax from a contrast grid (and particles for that form).

    forms: any of "node", "gamma", "particle".  Returns (zeta, cond) dicts of
    float64 arrays (lmax+1, nb, nb); cond holds the sum of absolute values of
    the summed terms (the condition sum used to judge FP32 attainable error).
    raw_particle drops the U term (the raw-DDD reading used against brute force).
    vertex sets the secondary-vertex windows (see window_kernel); primary_tophat > 0 smooths
    the primary vertex of the grid forms with the spherical tophat of that radius (the
    particle form's primary vertex is the particles themselves, unfiltered).
    """
    vertex = vertex or {}
    nb = len(vertex["radii"]) if vertex.get("radial") == "point" else len(edges) - 1
    delta = np.asarray(delta, np.float64)
    delta_hat = np.fft.fftn(delta)
    prim = primary_filter(delta, n, box, primary_tophat) if primary_tophat > 0.0 else delta
    zeta = {f: np.zeros((lmax + 1, nb, nb)) for f in forms}
    cond = {f: np.zeros((lmax + 1, nb, nb)) for f in forms}
    if "particle" in forms:
        pos = np.asarray(particles[:, :3], np.float64)
        w = np.asarray(particles[:, 3], np.float64)
    for ell in range(lmax + 1):
        for m in range(-ell, ell + 1):
            a = multipole_fields(delta_hat, ell, m, n, box, edges, vertex=vertex)
            if "node" in forms:
                zeta["node"][ell] += sum_node(prim, a)
                cond["node"][ell] += sum_node(np.abs(prim), np.abs(a))
            if "gamma" in forms:
                zeta["gamma"][ell] += sum_gamma(prim, a, dsup)
            if "particle" in forms:
                f = interpolate(a, pos, n, box, dsup)
                wsum = float(w.sum())
                part = (f * w[None, :]) @ f.T / wsum
                cond["particle"][ell] += (np.abs(f) * np.abs(w)[None, :]) @ np.abs(f).T / wsum
                if not raw_particle:
                    u = mass_term(a, dsup)
                    part = part - u
                    cond["particle"][ell] += np.abs(u)
                zeta["particle"][ell] += part
    return ({f: _symmetrise(v) for f, v in zeta.items()}, cond)


def zeta_multipoles(particles, n: int, box: float, edges, lmax: int, dsup: int,
                    forms=("node",), raw=False, vertex=None, primary_tophat=0.0):
    """Full pipeline from a catalogue: assign -> contrast -> DFT -> fields -> sums.

    raw=True keeps the primary and the fields on n/n_bar (no -1) and drops U,
    the reading compared with brute-force triplet enumeration.
    """
    particles = np.asarray(particles)
    eps, wsum = assign(particles[:, :3], particles[:, 3], n, box, dsup)
    delta = eps / (wsum / eps.size) if raw else contrast(eps, wsum)
    return zeta_from_delta(delta, n, box, edges, lmax, dsup, forms=forms,
                           particles=particles, raw_particle=raw, vertex=vertex, primary_tophat=primary_tophat)


# ---------------------------------------------------------------------------
# Sec. 2.1 and Sec. 3: the 2PCF from the same machinery, the 3PCF in angle, and the
# reduced 3PCF.
# ---------------------------------------------------------------------------
def xi_node(delta, n: int, box: float, edges, vertex=None, primary_tophat=0.0):
    """2PCF of the grid (Eq. pair-counting with the translated field of Eq. trans-field-FT):
    xi_b = (1/N_g) sum_l delta_p(l) a_00,b(l), a_00,b the l = 0 field of bin b (whose window is
    sqrt(4 pi) Y_00 W_0,b = W_0,b, the isotropic shell filter of Eq. DD-windowfunction) and
    delta_p the primary vertex (smoothed when primary_tophat > 0).  Returns (nbins,)."""
    delta = np.asarray(delta, np.float64)
    prim = primary_filter(delta, n, box, primary_tophat) if primary_tophat > 0.0 else delta
    a = multipole_fields(np.fft.fftn(delta), 0, 0, n, box, edges, vertex=vertex)
    return (a.reshape(a.shape[0], -1) @ prim.ravel()) / delta.size


def xi_particle(particles, n: int, box: float, edges, dsup: int, vertex=None):
    """2PCF in the particle form: xi_b = (1/W) sum_p w_p f_b(x_p), f_b the B-spline expansion of
    the l = 0 field of bin b from the particles' own contrast (the primary vertex is the
    catalogue; the uniform term vanishes because the fields have zero mean).  Returns (nbins,)."""
    p = np.asarray(particles, np.float64)
    eps, wsum = assign(p[:, :3], p[:, 3], n, box, dsup)
    delta = contrast(eps, wsum)
    a = multipole_fields(np.fft.fftn(delta), 0, 0, n, box, edges, vertex=vertex)
    f = interpolate(a, p[:, :3], n, box, dsup)
    return f @ p[:, 3] / wsum


def legendre_sum(zeta_l, mu):
    """zeta(b1, b2, mu) = sum_l zeta_l(b1, b2) P_l(mu), Eq. (triplet-counting); zeta_l of shape
    (lmax+1, nb, nb), mu a 1-D array -> (len(mu), nb, nb).  P_l by the three-term recurrence."""
    zeta_l = np.asarray(zeta_l, np.float64)
    mu = np.asarray(mu, np.float64)
    out = np.zeros((len(mu),) + zeta_l.shape[1:])
    p0, p1 = np.ones_like(mu), mu.copy()
    for ell in range(zeta_l.shape[0]):
        pl = p0 if ell == 0 else p1
        out += pl[:, None, None] * zeta_l[ell][None]
        if ell >= 1:
            p0, p1 = p1, ((2 * ell + 1) * mu * p1 - ell * p0) / (ell + 1)
    return out


def reduced_q(zeta, xi1, xi2, xi3):
    """Q = zeta / (xi(r1) xi(r2) + xi(r2) xi(r3) + xi(r3) xi(r1)), Eq. (Q-factor)."""
    return zeta / (xi1 * xi2 + xi2 * xi3 + xi3 * xi1)


def zeta_szapudi_szalay(data, randoms, n: int, box: float, edges, lmax: int, dsup: int, forms=("node",),
                        vertex=None):
    """Eq. (SSestimator) in multipoles: the numerator <(D - R)^3> and the denominator <R^3> with D and
    R each normalised to unit mean density, Delta = delta_D - delta_R and R~ = 1 + delta_R (the SFC
    difference of Sec. 3), each measured like zeta_from_delta (grid forms).  The estimator is
    zeta(theta) = sum_l num_l P_l(cos theta) / sum_l den_l P_l(cos theta).  Returns (num, den) dicts."""
    d = np.asarray(data, np.float64)
    r = np.asarray(randoms, np.float64)
    eps_d, w_d = assign(d[:, :3], d[:, 3], n, box, dsup)
    eps_r, w_r = assign(r[:, :3], r[:, 3], n, box, dsup)
    dd, dr = contrast(eps_d, w_d), contrast(eps_r, w_r)
    num, _ = zeta_from_delta(dd - dr, n, box, edges, lmax, dsup, forms=forms, vertex=vertex)
    den, _ = zeta_from_delta(1.0 + dr, n, box, edges, lmax, dsup, forms=forms, vertex=vertex)
    return num, den


# ---------------------------------------------------------------------------
# Continuum target of the raw-DDD reading: explicit pair/harmonic enumeration.
# ---------------------------------------------------------------------------
def brute_force_raw(particles, box: float, edges, lmax: int):
    """D_l(b1,b2) = (4 pi / W) sum_i w_i sum_m Abar_lm(i;b1) Abar_lm(i;b2) with
    Abar_lm(i;b) = V / (W V_b) sum_{j != i, r_ij in b} w_j R_lm(r_ij-hat), minimum image.

    Loops over primaries in Python; meant for a few thousand points at most.
    """
    p = np.asarray(particles, np.float64)
    pos, w = p[:, :3], p[:, 3]
    wsum = float(w.sum())
    vol = box ** 3
    edges = np.asarray(edges, np.float64)
    nb = len(edges) - 1
    vb = 4.0 * math.pi / 3.0 * (edges[1:] ** 3 - edges[:-1] ** 3)
    out = np.zeros((lmax + 1, nb, nb))
    for i in range(len(p)):
        d = pos - pos[i]
        d -= box * np.round(d / box)
        r = np.sqrt(np.sum(d * d, axis=1))
        sel = np.arange(len(p)) != i
        bidx = np.searchsorted(edges, r, side="right") - 1
        ok = sel & (bidx >= 0) & (bidx < nb) & (r < edges[-1])
        if not np.any(ok):
            continue
        dd, ww, bb = d[ok], w[ok], bidx[ok]
        for ell in range(lmax + 1):
            for m in range(-ell, ell + 1):
                rl = real_ylm(ell, m, dd[:, 0], dd[:, 1], dd[:, 2])
                abar = np.zeros(nb)
                np.add.at(abar, bb, ww * rl)
                abar *= vol / (wsum * vb)
                out[ell] += w[i] * np.outer(abar, abar)
    return out * FOUR_PI / wsum


# ---------------------------------------------------------------------------
# Gradients of a scalar loss L = sum_l sum_ij W_l[i, j] zeta_l[i, j] (field-level
# inference), by the transpose of every linear step of the measurement above.
# With S_l = (W_l + W_l^T) / 2 (zeta is symmetric), and A_lm,b the map delta -> a_lm,b:
#   A^T h = (-1)^l IDFT[K_lm,b DFT(h)]   (the window is i^l times a real function).
# ---------------------------------------------------------------------------
def bspline_deriv(u, dsup: int):
    """d beta_D / du."""
    u = np.asarray(u, dtype=np.float64)
    a = np.abs(u)
    sg = np.sign(u)
    if dsup == 2:
        return np.where(a < 1.0, -sg, 0.0)
    if dsup == 4:
        inner = -2.0 * u + 1.5 * u * a
        outer = -0.5 * sg * (2.0 - a) ** 2
        return np.where(a < 1.0, inner, np.where(a < 2.0, outer, 0.0))
    raise ValueError("dsup must be 2 or 4")


def interpolate_grad(a, pos, n: int, box: float, dsup: int):
    """Gradient with respect to the point of f_b(x) = sum_l beta(x/H - l) a_b(l): (nb, N_p, 3)."""
    pos = np.asarray(pos, np.float64)
    h = box / n
    u = pos / h
    base = stencil_base(u, dsup)
    nb = a.shape[0]
    af = a.reshape(nb, -1)
    g = np.zeros((nb, pos.shape[0], 3))
    for oz in range(dsup):
        lz = base[:, 2] + oz
        bz, dz = bspline(u[:, 2] - lz, dsup), bspline_deriv(u[:, 2] - lz, dsup)
        for oy in range(dsup):
            ly = base[:, 1] + oy
            by, dy = bspline(u[:, 1] - ly, dsup), bspline_deriv(u[:, 1] - ly, dsup)
            for ox in range(dsup):
                lx = base[:, 0] + ox
                bx, dx = bspline(u[:, 0] - lx, dsup), bspline_deriv(u[:, 0] - lx, dsup)
                idx = ((lz % n) * n + (ly % n)) * n + (lx % n)
                v = af[:, idx]
                g[:, :, 0] += (dx * by * bz)[None, :] * v
                g[:, :, 1] += (bx * dy * bz)[None, :] * v
                g[:, :, 2] += (bx * by * dz)[None, :] * v
    return g / h


def loss(zeta_l, weights):
    """L = sum_l sum_ij W_l[i, j] zeta_l[i, j]."""
    return float(np.sum(np.asarray(weights) * np.asarray(zeta_l)))


def grad_node_delta(delta, weights, n: int, box: float, edges, lmax: int, vertex=None):
    """dL/d delta for the node form: (1/N_g) [sum_lm sum S a a + IDFT(sum_lm (-1)^l sum_b K_b DFT(h_b))],
    h_b = 2 delta sum_b' S[b, b'] a_b'."""
    delta = np.asarray(delta, np.float64)
    ng = delta.size
    dh = np.fft.fftn(delta)
    q = np.zeros(delta.shape)
    gk = np.zeros(delta.shape, np.complex128)
    for ell in range(lmax + 1):
        s = 0.5 * (weights[ell] + weights[ell].T)
        for m in range(-ell, ell + 1):
            kern = window_kernel(ell, m, n, box, edges, vertex=vertex)
            a = np.stack([np.fft.ifftn(dh * kern[b]).real for b in range(kern.shape[0])])
            q += np.einsum("ij,ixyz,jxyz->xyz", s, a, a)
            hb = 2.0 * delta[None] * np.einsum("ij,jxyz->ixyz", s, a)
            gk += (-1.0) ** ell * sum(kern[b] * np.fft.fftn(hb[b]) for b in range(kern.shape[0]))
    return (q + np.fft.ifftn(gk).real) / ng


def grad_particle_positions(particles, weights, n: int, box: float, edges, lmax: int, dsup: int, vertex=None):
    """dL/dx_p (N_p, 3) for the particle form, with the fields built from the particles' own
    assignment: the direct term through f_b(x_p), plus the term through delta (assignment),
    where dL/d delta = IDFT(sum_lm (-1)^l sum_b K_b DFT(h_b - u_b)), h_b the assignment of
    (2 w_p / W) (S f)_b, u_b = dU/da_b = (2/N_g) sum_b' S[b, b'] (M3 * a_b')."""
    p = np.asarray(particles, np.float64)
    pos, w = p[:, :3], p[:, 3]
    wsum = float(w.sum())
    ng = n ** 3
    eps, _ = assign(pos, w, n, box, dsup)
    delta = contrast(eps, wsum)
    dh = np.fft.fftn(delta)
    m1 = mass_1d(dsup)
    direct = np.zeros((len(p), 3))
    gk = np.zeros((n, n, n), np.complex128)
    for ell in range(lmax + 1):
        s = 0.5 * (weights[ell] + weights[ell].T)
        for m in range(-ell, ell + 1):
            kern = window_kernel(ell, m, n, box, edges, vertex=vertex)
            nb = kern.shape[0]
            a = np.stack([np.fft.ifftn(dh * kern[b]).real for b in range(nb)])
            f = interpolate(a, pos, n, box, dsup)
            df = interpolate_grad(a, pos, n, box, dsup)
            c = (2.0 * w / wsum)[None, :] * (s @ f)
            direct += np.einsum("bp,bpd->pd", c, df)
            for b in range(nb):
                hb, _ = assign(pos, c[b], n, box, dsup)
                mb = np.zeros((n, n, n))
                for dz, mz in m1.items():
                    for dy, my in m1.items():
                        for dx, mx in m1.items():
                            mb += mz * my * mx * _shift(np.einsum("j,jxyz->xyz", s[b], a), (dz, dy, dx))
                ub = 2.0 / ng * mb
                gk += (-1.0) ** ell * kern[b] * np.fft.fftn(hb - ub)
    gdelta = np.fft.ifftn(gk).real
    via = (ng / wsum) * w[:, None] * interpolate_grad(gdelta[None], pos, n, box, dsup)[0]
    return direct + via
