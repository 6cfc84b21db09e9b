"""The Gamma (connection-coefficient) form as the library's kernel evaluates it, replayed in
float64 on the CPU from the library's own host tables, against the oracle's literal double sum
of Eqs. (con-coeff), (SFC-3PCF) (no GPU).

The kernel never forms Gamma_{l1,l2}.  For the B-splines (dsup 2, 4) it integrates
n_rec f_b1 f_b2 over every cell with the K^3 Gauss-Legendre points of zeta_host_cell_quadrature
(K = 2, 5: exact, the integrand being a polynomial of degree 3 (D - 1) per axis); for the
Daubechies basis (dsup 3) it applies the per-axis 5 x 5 connection matrix through its eigen-split
gamma = U diag(lam) U^T of zeta_host_daub4_gamma, A_k(l) = sum_o U[o][k] a(l + o - 2) with weight
lam_kx lam_ky lam_kz delta_l.  Either way a point value is a tensor-product filter of the
D^3 stencil, which is what the kernel's x, y and z passes compute one axis at a time.  Agreement
to 1e-12 pins the host tables and the algebra the kernel relies on; a wrong stencil offset, a
transposed filter or a dropped eigenvalue fails it."""
import numpy as np
import pytest

from oracle import zeta_oracle as O


@pytest.fixture(scope="module")
def zmod():
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    zeta.lib()
    return zeta


def _stencils(f, off, d):
    """S[..., z, y, x, oz, oy, ox] = f[..., z - off + oz, y - off + oy, x - off + ox] (periodic)."""
    n = f.shape[-1]
    idx = (np.arange(n)[:, None] - off + np.arange(d)[None, :]) % n  # [cell][o]
    return f[..., idx[:, None, None, :, None, None], idx[None, :, None, None, :, None],
             idx[None, None, :, None, None, :]]


def _filtered(f, filt, off):
    """Point values P[..., z, y, x, kz, ky, kx] = sum_o F[oz][kz] F[oy][ky] F[ox][kx] f(stencil)."""
    s = _stencils(f, off, filt.shape[0])
    return np.einsum("...zyxabc,ak,bl,cm->...zyxklm", s, filt, filt, filt, optimize=True)


def kernel_form(zmod, delta, a, dsup):
    n = delta.shape[0]
    if dsup == 3:
        _, lam, u = zmod.host_daub4_gamma()
        pts = _filtered(a, u, 2)                                   # [b][cell][k]
        w = np.einsum("k,l,m->klm", lam, lam, lam)[None, None, None] * delta[..., None, None, None]
    else:
        q = 2 if dsup == 2 else 5
        _, wq, beta = zmod.host_cell_quadrature(q, dsup)
        filt = beta.T                                              # F[o][k] = beta[k][o]
        off = dsup // 2 - 1
        pts = _filtered(a, filt, off)
        w = np.einsum("k,l,m->klm", wq, wq, wq)[None, None, None] * _filtered(delta, filt, off)
    nb = a.shape[0]
    p = pts.reshape(nb, -1)
    return (p * w.reshape(1, -1)) @ p.T / n ** 3


@pytest.mark.parametrize("dsup", [2, 4, 3])
def test_kernel_reformulation_equals_the_double_sum(zmod, dsup):
    n, nb = 8, 3
    rng = np.random.default_rng(90 + dsup)
    delta = rng.standard_normal((n, n, n))
    a = rng.standard_normal((nb, n, n, n))
    got = kernel_form(zmod, delta, a, dsup)
    want = O.sum_gamma(delta, a, dsup)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (dsup, got, want)


def test_a_dropped_eigenvalue_or_shifted_stencil_is_caught(zmod):
    """The check above has teeth: dropping an eigenvalue of the Daubechies split, or shifting the
    fields' stencil against delta's by one cell (a common shift of all three is a translation,
    which the periodic sum does not see), moves the result far outside its tolerance."""
    n, nb = 8, 2
    rng = np.random.default_rng(97)
    delta = rng.standard_normal((n, n, n))
    a = rng.standard_normal((nb, n, n, n))
    want = O.sum_gamma(delta, a, 3)
    _, lam, u = zmod.host_daub4_gamma()
    lam2 = lam.copy()
    lam2[np.argmin(np.abs(lam))] = 0.0
    pts = _filtered(a, u, 2)
    w = np.einsum("k,l,m->klm", lam2, lam2, lam2)[None, None, None] * delta[..., None, None, None]
    p = pts.reshape(nb, -1)
    bad = (p * w.reshape(1, -1)) @ p.T / n ** 3
    assert np.abs(bad - want).max() > 1e-6 * np.abs(want).max()
    want4 = O.sum_gamma(delta, a, 4)
    _, wq, beta = zmod.host_cell_quadrature(5, 4)
    pts = _filtered(a, beta.T, 0)  # the fields' stencil one cell off
    w = np.einsum("k,l,m->klm", wq, wq, wq)[None, None, None] * _filtered(delta, beta.T, 1)
    p = pts.reshape(nb, -1)
    bad4 = (p * w.reshape(1, -1)) @ p.T / n ** 3
    assert np.abs(bad4 - want4).max() > 1e-3 * np.abs(want4).max()
