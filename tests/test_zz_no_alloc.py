"""The allocation-free assignment (zeta_assign_noalloc) against the regular one.

zeta_assign_noalloc serves callers that cannot allocate device memory at call time (a host
framework whose pool owns the GPU, latency-critical loops, services that must not run out of
memory); it keeps its scratch in a fixed array inside the library.  Two calls in a row with
different catalogues and grid sizes must each match zeta_assign, which also shows that the
shared scratch is cleared between calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def test_noalloc_assign_matches_regular_assign_twice(Z):
    cases = [(64, 400.0, 4, 30000, 61), (32, 150.0, 2, 9000, 63)]
    for n, box, dsup, n_p, seed in cases:
        parts = torch.from_numpy(mocks.lognormal_catalogue(n, n_p, box, seed, seed + 1)).to("cuda")
        ctx = Z.Context(n, box, dsup, 0, [5.0, 10.0])
        want, wsum_want = ctx.assign(parts)
        got = torch.full((n, n, n), float("nan"), dtype=torch.float32, device="cuda")
        wsum = torch.zeros(1, dtype=torch.float64, device="cuda")
        Z.assign_noalloc(n, box, dsup, parts, delta=got, wsum=wsum)
        torch.cuda.synchronize()
        w = want.cpu().numpy()
        g = got.cpu().numpy()
        assert np.abs(g - w).max() <= 2e-6 * max(1.0, np.abs(w).max())
        assert abs(float(wsum.item()) - float(wsum_want.item())) <= 1e-12 * abs(float(wsum_want.item()))
        ctx.close()


def test_noalloc_rejects_grid_beyond_its_fixed_scratch(Z):
    parts = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(Z.ZetaError) as e:
        Z.assign_noalloc(256, 100.0, 4, parts)
    assert e.value.code == -1
