"""The measurement split over (l, m) pairs (zeta_zeta_lm + zeta_reduce_lm) on one GPU.

P "ranks" run one after another on this GPU, each with its own subset of the (l, m) pairs
(index l^2 + l + m mod P); their slot arrays are summed element-wise in float64 (exact: every
slot has one non-zero contributor) and reduced.  The result must equal zeta_zeta_ell bit for
bit, for every form, and each rank's non-zero slots must be exactly the pairs lm_pairs assigns
it (plus the uniform terms of the l whose (l, -l) it owns).
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


@pytest.mark.parametrize("forms", [("node", "gamma", "particle"), ("particle",)])
def test_lm_split_sums_to_the_full_measurement_bit_for_bit(Z, forms):
    n, box, lmax, dsup = 32, 250.0, 4, 4
    edges = np.array([12.0, 25.0, 37.0, 52.0, 66.0, 80.0])
    nb = len(edges) - 1
    parts = torch.from_numpy(mocks.lognormal_catalogue(n, 9000, box, 91, 92)).cuda()
    ctx = Z.Context(n, box, dsup, lmax, edges, np_max=parts.shape[0], forms=forms)
    full = ctx.zeta_ell(particles=parts, forms=forms)
    full = {f: v.clone() for f, v in full.items()}
    nf = len(full)
    nslot = (lmax + 1) ** 2 + lmax + 1
    for P in (1, 2, 3, 7):
        total = torch.zeros(ctx.lm_slots(forms), dtype=torch.float64, device="cuda")
        for r in range(P):
            s = ctx.zeta_lm(r, P, particles=parts, forms=forms).clone()
            sv = s.view(nf, nslot, nb, nb).abs().sum(dim=(2, 3)).cpu().numpy()
            owned = {Z.lm_slot(l, m) for l, m in Z.lm_pairs(r, P, lmax)}
            for fi, f in enumerate([f for f in ("node", "gamma", "particle") if f in forms]):
                nz = {int(i) for i in np.nonzero(sv[fi])[0]}
                want = set(owned)
                if f == "particle":
                    want |= {(lmax + 1) ** 2 + l for l in range(lmax + 1) if (l * l) % P == r}
                assert nz == want, (P, r, f)
            total += s
        got = ctx.reduce_lm(total, forms=forms)
        assert ctx.get_status() == 0
        for f in full:
            assert torch.equal(got[f], full[f]), (P, f)
    ctx.close()


def test_lm_split_rejects_a_bad_rank(Z):
    ctx = Z.Context(16, 100.0, 2, 1, [5.0, 10.0])
    d = torch.zeros((16, 16, 16), dtype=torch.float32, device="cuda")
    for r, P in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(Z.ZetaError):
            ctx.zeta_lm(r, P, delta=d, forms=("node",))
    ctx.close()
