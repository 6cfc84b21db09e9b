"""Host-side bookkeeping of bench.py (no GPU): every stage that the stage timers report with
algorithmic bytes can be named as the roofline's dominant stage, so each needs a source-file
entry; the stored counter capture must name existing sources; the algorithmic bytes follow
their stated formulas."""
import os

import bench

STAGES = ["assign", "sort", "r2c", "alm_z", "alm_y", "alm_x", "gram_node", "gram_gamma", "gram_particles", "mass",
          "reduce"]


def test_every_stage_with_bytes_has_sources():
    w = bench.WORKLOADS["box2000_n512_np16m"]
    for st in STAGES:
        if bench._alg_bytes(st, w, 20) is not None:
            assert st in bench.STAGE_SOURCES, st
            for f in bench.STAGE_SOURCES[st]:
                assert os.path.exists(os.path.join(bench.ROOT, "paper_2507_15209_gb300", "csrc", f)), f


def test_stored_traffic_names_a_stage_with_sources():
    for st, tr in bench.NCU_TRAFFIC.items():
        assert st in bench.STAGE_SOURCES
        assert len(tr["sha"]) == len(bench.STAGE_SOURCES[st])
        assert tr["bytes"] > bench._alg_bytes(st, bench.WORKLOADS["box2000_n512_np16m"], 20)


def test_algorithmic_bytes_of_the_512_workload():
    w = bench.WORKLOADS["box2000_n512_np16m"]
    g = 4.0 * 512 ** 3
    assert bench._alg_bytes("alm_z", w, 20) == 21 * g
    assert bench._alg_bytes("alm_y", w, 20) == bench._alg_bytes("alm_x", w, 20) == 40 * g
    assert bench._alg_bytes("gram_node", w, 20) == 21 * g
    assert bench._alg_bytes("gram_particles", w, 20) == 20 * g + 16.0 * 16_000_000
    assert bench._alg_bytes("assign", w, 20) == 16.0 * 16_000_000 + g
    assert bench._alg_bytes("gram_gamma", w, 20) is None
