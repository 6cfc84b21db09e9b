"""The Szapudi-Szalay estimator with a random catalogue (Eq. SSestimator) through the C ABI against
the FP64 oracle (GPU): numerator <(D - R)^3> and denominator <R^3> multipoles of a log-normal data
catalogue and a uniform random catalogue three times as large, node and Gamma forms, and the
estimator in angle from them.  Tolerance: per l, 1e-5 relative Frobenius, or 1e-6 of the condition
sum where that exceeds 100 |zeta_l| (the denominator's l > 0 multipoles are noise about zero).
"""
import numpy as np
import pytest

from oracle import zeta_oracle as O
from paper_2507_15209_gb300 import mocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, BOX, LMAX, DSUP = 32, 250.0, 3, 2
EDGES = np.array([12.0, 25.0, 37.0, 52.0])


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    return zeta


def _check(got, want, cond, label):
    for ell in range(want.shape[0]):
        err = float(np.linalg.norm(got[ell] - want[ell]))
        zn, cn = float(np.linalg.norm(want[ell])), float(np.linalg.norm(cond[ell]))
        if cn > 100.0 * zn:
            assert err <= 1e-6 * cn, (label, ell, err / zn, err / cn)
        else:
            assert err <= 1e-5 * zn, (label, ell, err / zn)


def test_szapudi_szalay_numerator_and_denominator(Z):
    data = mocks.lognormal_catalogue(N, 10000, BOX, 501, 502)
    rand = mocks.uniform_particles(30000, BOX, 503)
    forms = ("node", "gamma")
    ctx = Z.Context(N, BOX, DSUP, LMAX, EDGES, forms=forms + ("ss",))
    num, den = ctx.zeta_ell_ss(torch.from_numpy(data).cuda(), torch.from_numpy(rand).cuda(), forms=forms)
    assert ctx.get_status() == 0
    d64, r64 = data.astype(np.float64), rand.astype(np.float64)
    eps_d, w_d = O.assign(d64[:, :3], d64[:, 3], N, BOX, DSUP)
    eps_r, w_r = O.assign(r64[:, :3], r64[:, 3], N, BOX, DSUP)
    dd, dr = O.contrast(eps_d, w_d), O.contrast(eps_r, w_r)
    want_n, cond_n = O.zeta_from_delta(dd - dr, N, BOX, EDGES, LMAX, DSUP, forms=forms)
    want_d, cond_d = O.zeta_from_delta(1.0 + dr, N, BOX, EDGES, LMAX, DSUP, forms=forms)
    ref_n, ref_d = O.zeta_szapudi_szalay(d64, r64, N, BOX, EDGES, LMAX, DSUP, forms=forms)
    for f in forms:
        np.testing.assert_allclose(ref_n[f], want_n[f], rtol=1e-12, atol=1e-15)
        _check(num[f].cpu().numpy(), want_n[f], cond_n["node"], ("num", f))
        _check(den[f].cpu().numpy(), want_d[f], cond_d["node"], ("den", f))
    mu = np.linspace(-0.95, 0.95, 9)
    est = Z.legendre_sum(num["node"].cpu().numpy(), mu) / Z.legendre_sum(den["node"].cpu().numpy(), mu)
    ref = O.legendre_sum(want_n["node"], mu) / O.legendre_sum(want_d["node"], mu)
    assert np.abs(est - ref).max() <= 1e-4 * np.abs(ref).max()
    ctx.close()
