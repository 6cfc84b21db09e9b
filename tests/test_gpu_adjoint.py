"""Gradients on the GPU (zeta_backward_node / zeta_backward_particles and the
torch.autograd.Function wrappers) against the FP64 oracle gradient and FP64 finite
differences of the oracle loss."""
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
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nb", [4, 10])
def test_node_gradient_matches_oracle(Z, nb):
    n, box, lmax = 16, 96.0, 3
    edges = np.linspace(8.0, 40.0, nb + 1)
    delta = (mocks.lognormal_density(n, 71) - 1.0).astype(np.float32)
    wts = mocks.loss_weights(lmax, nb, 72)
    ctx = Z.Context(n, box, 4, lmax, edges, forms=("node", "backward"))
    got = ctx.backward_node(torch.from_numpy(delta).cuda(), wts).cpu().numpy()
    assert ctx.get_status() == 0
    want = O.grad_node_delta(delta.astype(np.float64), wts, n, box, edges, lmax)
    assert _rel(got, want) < 2e-5


@pytest.mark.parametrize("dsup", [4, 2])
def test_particle_gradient_matches_oracle(Z, dsup):
    n, box, lmax, nb = 16, 80.0, 2, 3
    edges = np.linspace(6.0, 30.0, nb + 1)
    parts = mocks.lognormal_catalogue(n, 1500, box, 73, 74)
    parts[:, 3] = np.random.default_rng(75).uniform(0.5, 1.5, len(parts)).astype(np.float32)
    wts = mocks.loss_weights(lmax, nb, 76)
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=len(parts), forms=("particle", "backward"))
    got = ctx.backward_particles(torch.from_numpy(parts).cuda(), wts).cpu().numpy()
    assert ctx.get_status() == 0
    want = O.grad_particle_positions(parts.astype(np.float64), wts, n, box, edges, lmax, dsup)
    assert _rel(got, want) < 1e-4


def test_autograd_node_against_fp64_finite_differences_32(Z):
    n, box, lmax, nb = 32, 250.0, 2, 3
    edges = np.linspace(10.0, 50.0, nb + 1)
    delta = (mocks.lognormal_density(n, 81) - 1.0).astype(np.float32)
    wts = mocks.loss_weights(lmax, nb, 82)
    ctx = Z.Context(n, box, 4, lmax, edges, forms=("node", "backward"))
    d = torch.from_numpy(delta).cuda().requires_grad_(True)
    z = Z.zeta_node(d, ctx)
    loss = (z * torch.from_numpy(wts).cuda()).sum()
    loss.backward()
    g = d.grad.cpu().numpy().astype(np.float64)
    v = np.random.default_rng(83).standard_normal((n, n, n))
    eps = 1e-3

    def lossf(x):
        zz, _ = O.zeta_from_delta(x, n, box, edges, lmax, 4, forms=("node",))
        return O.loss(zz["node"], wts)

    d64 = delta.astype(np.float64)
    fd = (lossf(d64 + eps * v) - lossf(d64 - eps * v)) / (2 * eps)
    assert abs(float((g * v).sum()) - fd) < 1e-4 * abs(fd)


def test_autograd_particles_against_fp64_finite_differences_32(Z):
    n, box, lmax, nb = 32, 250.0, 2, 3
    edges = np.linspace(10.0, 50.0, nb + 1)
    parts = mocks.lognormal_catalogue(n, 4000, box, 85, 86)
    wts = mocks.loss_weights(lmax, nb, 87)
    ctx = Z.Context(n, box, 4, lmax, edges, np_max=len(parts), forms=("particle", "backward"))
    pos = torch.from_numpy(parts[:, :3].copy()).cuda().requires_grad_(True)
    w = torch.from_numpy(parts[:, 3].copy()).cuda()
    z = Z.zeta_particles(pos, w, ctx)
    (z * torch.from_numpy(wts).cuda()).sum().backward()
    g = pos.grad.cpu().numpy().astype(np.float64)
    v = np.random.default_rng(88).standard_normal((len(parts), 3))
    eps = 1e-3

    def lossf(p):
        zz, _ = O.zeta_multipoles(p, n, box, edges, lmax, 4, forms=("particle",))
        return O.loss(zz["particle"], wts)

    p64 = parts.astype(np.float64)
    pp, pm = p64.copy(), p64.copy()
    pp[:, :3] += eps * v
    pm[:, :3] -= eps * v
    fd = (lossf(pp) - lossf(pm)) / (2 * eps)
    assert abs(float((g * v).sum()) - fd) < 1e-3 * abs(fd)
