"""The 2PCF, the 3PCF in angle and the reduced 3PCF through the C ABI against the FP64 oracle (GPU).

xi_b in the node form (evaluated by the library in Fourier space from per-|n|^2 sums) and the
particle form, with and without vertex windows; xi(r) at arbitrary radii; and Q(r1, r2, theta)
assembled from zeta_l, xi(r1), xi(r2), xi(r3) as a user of the library would.  Tolerance: 1e-5
relative (max over bins, against the largest |xi_b|).
"""
import math

import numpy as np
import pytest

from oracle import zeta_oracle as O
from paper_2507_15209_gb300 import mocks

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N, BOX, LMAX = 32, 250.0, 4
EDGES = np.array([12.0, 25.0, 37.0, 52.0, 66.0])


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    return zeta


def _close(got, want, tol=1e-5):
    return np.abs(np.asarray(got) - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("dsup,win", [(4, {}), (2, {"tophat": 7.0, "phi_hat": True, "tophat_primary": 5.0})])
def test_xi_node_and_particle_forms(Z, dsup, win):
    parts = mocks.lognormal_catalogue(N, 15000, BOX, 401, 402)
    p64 = parts.astype(np.float64)
    ctx = Z.Context(N, BOX, dsup, LMAX, EDGES, np_max=len(parts), forms=("node", "particle"), **win)
    xi = ctx.xi(particles=torch.from_numpy(parts).cuda(), forms=("node", "particle"))
    assert ctx.get_status() == 0
    vertex = {"tophat": win.get("tophat", 0.0), "phi_dsup": dsup if win.get("phi_hat") else 0}
    eps, wsum = O.assign(p64[:, :3], p64[:, 3], N, BOX, dsup)
    delta = O.contrast(eps, wsum)
    want_n = O.xi_node(delta, N, BOX, EDGES, vertex=vertex, primary_tophat=win.get("tophat_primary", 0.0))
    assert _close(xi["node"].cpu().numpy(), want_n), (xi["node"].cpu().numpy(), want_n)
    want_p = O.xi_particle(p64, N, BOX, EDGES, dsup, vertex=vertex)
    assert _close(xi["particle"].cpu().numpy(), want_p), (xi["particle"].cpu().numpy(), want_p)
    ctx.close()


def test_xi_at_radii_and_reduced_q(Z):
    parts = mocks.lognormal_catalogue(N, 20000, BOX, 403, 404)
    p64 = parts.astype(np.float64)
    radii = [15.0, 30.0]
    ctx = Z.Context(N, BOX, 4, LMAX, None, np_max=len(parts), forms=("node",), radial="point", radii=radii)
    pd = torch.from_numpy(parts).cuda()
    zeta_l = ctx.zeta_ell(particles=pd, forms=("node",))["node"].cpu().numpy()
    delta, _ = ctx.assign(pd)
    dh = ctx.fft_r2c(delta)
    mu = np.array([-0.9, -0.3, 0.2, 0.7])
    r3 = np.sqrt(radii[0] ** 2 + radii[1] ** 2 - 2 * radii[0] * radii[1] * mu)
    xi_r = ctx.xi_radii(dh, list(radii) + list(r3)).cpu().numpy()
    d64 = delta.cpu().numpy().astype(np.float64)
    want_xi = O.xi_node(d64, N, BOX, None, vertex={"radial": "point", "radii": list(radii) + list(r3)})
    assert _close(xi_r, want_xi), (xi_r, want_xi)
    zt = Z.legendre_sum(zeta_l, mu)[:, 0, 1]
    q = Z.reduced_q(zt, np.full(len(mu), xi_r[0]), np.full(len(mu), xi_r[1]), xi_r[2:])
    zo, _ = O.zeta_from_delta(d64, N, BOX, None, LMAX, 4, forms=("node",), vertex={"radial": "point", "radii": radii})
    qo = O.reduced_q(O.legendre_sum(zo["node"], mu)[:, 0, 1], want_xi[0], want_xi[1], want_xi[2:])
    assert np.abs(q - qo).max() <= 1e-4 * np.abs(qo).max(), (q, qo)
    assert np.all(np.isfinite(q))
    ctx.close()
