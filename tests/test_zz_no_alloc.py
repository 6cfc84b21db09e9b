"""The allocation-free assignment (zeta_assign_noalloc) against the regular one and the oracle.

zeta_assign_noalloc serves callers that cannot allocate device memory at call time (a host
framework whose pool owns the GPU, latency-critical loops, services that must not run out of
memory); it keeps its scratch in a fixed array inside the library.  Two calls in a row with
different catalogues and grid sizes must each match zeta_assign and the FP64 oracle's
assignment, which also shows that the shared scratch is cleared between calls.  A catalogue
with a non-finite particle must come back as an all-NaN result (this call has no context to
report through), and the call after it must be clean again.  This file is collected last on
purpose.
"""
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


def _noalloc(Z, n, box, dsup, parts):
    got = torch.full((n, n, n), 7.0, dtype=torch.float32, device="cuda")
    wsum = torch.zeros(1, dtype=torch.float64, device="cuda")
    Z.assign_noalloc(n, box, dsup, parts, delta=got, wsum=wsum)
    torch.cuda.synchronize()
    return got.cpu().numpy(), float(wsum.item())


def test_noalloc_assign_matches_regular_assign_and_oracle_twice(Z):
    cases = [(64, 400.0, 4, 30000, 61), (32, 150.0, 2, 9000, 63)]
    for n, box, dsup, n_p, seed in cases:
        host = mocks.lognormal_catalogue(n, n_p, box, seed, seed + 1)
        parts = torch.from_numpy(host).to("cuda")
        ctx = Z.Context(n, box, dsup, 0, [5.0, 10.0])
        want, wsum_want = ctx.assign(parts)
        g, wsum = _noalloc(Z, n, box, dsup, parts)
        w = want.cpu().numpy()
        assert np.abs(g - w).max() <= 2e-6 * max(1.0, np.abs(w).max())
        assert abs(wsum - float(wsum_want.item())) <= 1e-12 * abs(float(wsum_want.item()))
        eps, wtot = O.assign(host[:, :3].astype(np.float64), host[:, 3].astype(np.float64), n, box, dsup)
        d64 = O.contrast(eps, wtot)
        assert np.abs(g - d64).max() <= 2e-6 * max(1.0, np.abs(d64).max())
        assert abs(wsum - wtot) <= 1e-9 * wtot
        ctx.close()


def test_noalloc_reports_a_non_finite_particle_in_its_result(Z):
    n, box, dsup = 32, 150.0, 4
    host = mocks.lognormal_catalogue(n, 5000, box, 71, 72)
    bad = host.copy()
    bad[17, 1] = np.nan
    g, wsum = _noalloc(Z, n, box, dsup, torch.from_numpy(bad).to("cuda"))
    assert np.all(np.isnan(g)) and np.isnan(wsum)
    # the next call starts from a clean status
    g, wsum = _noalloc(Z, n, box, dsup, torch.from_numpy(host).to("cuda"))
    eps, wtot = O.assign(host[:, :3].astype(np.float64), host[:, 3].astype(np.float64), n, box, dsup)
    assert np.abs(g - O.contrast(eps, wtot)).max() <= 2e-6 * max(1.0, np.abs(O.contrast(eps, wtot)).max())


def test_noalloc_rejects_grid_beyond_its_fixed_scratch(Z):
    parts = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(Z.ZetaError) as e:
        Z.assign_noalloc(256, 100.0, 4, parts)
    assert e.value.code == -1
