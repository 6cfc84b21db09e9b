"""The multi-rank path of bench.py on CPU: two gloo ranks (no GPU).

One catalogue per rank (weak scaling): every rank draws its own seeded catalogue, the timings
are reduced with a max over ranks, and the whole-job value divides the slowest rank's time by
all ranks' catalogues.  The reference arm runs on rank 0 only.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_dev, ms_e2e = 1000.0 * (rank + 1), 1500.0 * (rank + 1)
        v, e, md, me = bench.reduce_timings(ms_dev, ms_e2e, steps=4, world=world, dist=dist, device="cpu")
        parts = bench._make_inputs(bench.WORKLOADS["box500_n64_np20k"], rank)
        out.put((rank, v, e, md, me, float(parts[:, :3].sum()), parts.shape[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_draw_distinct_catalogues():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, v, e, md, me, _, n in res:
        assert md == 2000.0 and me == 3000.0          # the slowest rank's times on every rank
        assert v == pytest.approx(2000.0 / 1e3 / (4 * world))
        assert e == pytest.approx(3000.0 / 1e3 / (4 * world))
        assert n == 20000
    assert res[0][5] != res[1][5]                      # each rank has its own catalogue


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import bench
    args = bench.argparse.Namespace(steps=1, warmup=3, workload="box500_n64_np20k")
    assert bench.run_reference(args, bench.WORKLOADS["box500_n64_np20k"], rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


def test_algorithmic_byte_counts_of_the_headline_workload():
    # the per-call and per-catalogue minimum bytes the roofline figures divide by
    import bench
    w = bench.WORKLOADS["box2000_n512_np16m"]
    g = 4.0 * 512 ** 3
    assert bench._alg_bytes("gram_particles", w, 20) == pytest.approx(20 * g + 16 * 16e6)   # 10.99 GB
    assert bench._alg_bytes("gram_particles", w, 20) == pytest.approx(10.993418240e9)
    assert bench._alg_bytes("alm_y", w, 20) == 2 * g * 20
    assert bench._alg_bytes("gram_node", w, 20) == g * 21
    assert bench._alg_bytes("no_such_stage", w, 20) is None
    cat = bench._catalogue_bytes(w, 20, ("particle", "node"))
    assert cat == pytest.approx(6.659977150464e12)                                       # 6.66 TB
