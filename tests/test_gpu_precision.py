"""Reduced-precision node-form Gram contractions (tcgen05 tensor cores) against the FP64 oracle (GPU).

zeta_l of the 256^3 / 2M-particle workload (lmax 10, 15 bins) with the node-form Gram in TF32,
BF16 and split BF16 (hi*hi + hi*lo + lo*hi) on the tensor cores, and with the fields stored as
bfloat16 by the last inverse pass (float32 Gram of bfloat16 inputs), each compared per l with the
oracle's result cached
in tests/golden/zeta_box1000_n256_np2m.json.  The bounds are per arithmetic: the relative
Frobenius error of zeta_l, or, where the condition sum C_l exceeds 100 |zeta_l|, the error over
C_l (float32 inputs rounded to 8 or 11 significant bits cannot do better than that there).
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2507_15209_gb300 import mocks
from paper_2507_15209_gb300.workloads import WORKLOADS, edges as wl_edges

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "zeta_box1000_n256_np2m.json")
# (relative bound, bound over the condition sum)
# (measured on this workload: fp32 <= 6.5e-6, bf16x3 <= 8.3e-6, tf32 <= 9.6e-6, bf16 <= 3.7e-5; the
# rounding errors of 16.7M products largely cancel in each sum)
BOUNDS = {"fp32": (1e-5, 1e-6), "bf16x3": (2e-5, 1e-6), "tf32": (3e-5, 2e-6), "bf16": (1e-4, 1e-5),
          "bf16_fields": (1e-4, 1e-5)}


@pytest.fixture(scope="module")
def Z():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_15209_gb300 import build
    build.build()
    from paper_2507_15209_gb300 import zeta
    return zeta


def test_node_gram_precision_variants_per_l(Z):
    w = WORKLOADS["box1000_n256_np2m"]
    with open(GOLDEN) as fh:
        gold = json.load(fh)["data"]
    parts = mocks.lognormal_catalogue(w["n"], w["n_p"], w["box"], w["field_seed"], w["sample_seed"])
    assert hashlib.sha256(parts.tobytes()).hexdigest() == gold["catalogue_sha256"]
    want = np.array(gold["zeta"]["node"])
    cond = np.array(gold["cond"]["node"])
    ctx = Z.Context(w["n"], w["box"], w["dsup"], w["lmax"], wl_edges(w), np_max=len(parts), forms=("node",))
    pd = torch.from_numpy(parts).cuda()
    report = {}
    for g, (rel_b, cond_b) in BOUNDS.items():
        ctx.set_gram(g)
        got = ctx.zeta_ell(particles=pd, forms=("node",))["node"].cpu().numpy()
        assert ctx.get_status() == 0
        rels = []
        for ell in range(want.shape[0]):
            err = float(np.linalg.norm(got[ell] - want[ell]))
            zn, cn = float(np.linalg.norm(want[ell])), float(np.linalg.norm(cond[ell]))
            rels.append(err / zn)
            if cn > 100 * zn:
                assert err <= cond_b * cn, (g, ell, err / zn, err / cn)
            else:
                assert err <= rel_b * zn, (g, ell, err / zn)
        report[g] = [f"{r:.1e}" for r in rels]
    print("per-l relative error against the FP64 oracle:", report)
    ctx.close()
