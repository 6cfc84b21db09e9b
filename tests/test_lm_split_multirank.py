"""The (l, m) split of one catalogue over ranks, on CPU: two gloo ranks, oracle partials (no GPU).

Each rank takes the (l, m) pairs the library's rule gives it (index l^2 + l + m mod P, the rule
of zeta_zeta_lm, exposed as zeta.lm_pairs), computes their node-form contributions with the FP64
oracle standing in for the GPU, writes them into its slot array (zero elsewhere), and the ranks
sum the slot arrays with bench.allreduce_slots (a float64 SUM all-reduce).  Checked: the pairs
of the ranks are disjoint and cover every (l, m); after the all-reduce every slot equals its
owner's value exactly; and summing the slots in the order of the library's zeta_reduce_lm
(0, then m = -l .. l) reproduces the oracle's own whole measurement bit for bit.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N, BOX, LMAX = 10, 50.0, 3
EDGES = np.array([6.0, 13.0, 21.0])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _delta():
    d = np.random.default_rng(77).standard_normal((N, N, N))
    return d - d.mean()


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    from oracle import zeta_oracle as O
    from paper_2507_15209_gb300.zeta import lm_pairs, lm_slot
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nb = len(EDGES) - 1
        delta = _delta()
        dh = np.fft.fftn(delta)
        slots = torch.zeros(((LMAX + 1) ** 2 + LMAX + 1, nb, nb), dtype=torch.float64)
        mine = lm_pairs(rank, world, LMAX)
        for l, m in mine:
            a = O.multipole_fields(dh, l, m, N, BOX, EDGES)
            slots[lm_slot(l, m)] = torch.from_numpy(O.sum_node(delta, a))
        own = slots.clone()
        bench.allreduce_slots(slots, dist)
        out.put((rank, mine, own.numpy(), slots.numpy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_lm_and_reduce_exactly():
    from oracle import zeta_oracle as O
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    pairs = [set(r[1]) for r in res]
    assert not (pairs[0] & pairs[1])
    assert pairs[0] | pairs[1] == {(l, m) for l in range(LMAX + 1) for m in range(-l, l + 1)}
    assert abs(len(pairs[0]) - len(pairs[1])) <= 1
    summed = res[0][3]
    np.testing.assert_array_equal(res[1][3], summed)                  # every rank holds the same sum
    for rank, mine, own, _ in res:
        for l, m in mine:
            np.testing.assert_array_equal(summed[l * l + l + m], own[l * l + l + m])   # exact
    zeta = np.zeros((LMAX + 1, len(EDGES) - 1, len(EDGES) - 1))
    for l in range(LMAX + 1):
        for m in range(-l, l + 1):
            zeta[l] += summed[l * l + l + m]
    zeta = 0.5 * (zeta + np.swapaxes(zeta, -1, -2))
    want, _ = O.zeta_from_delta(_delta(), N, BOX, EDGES, LMAX, 2, forms=("node",))
    np.testing.assert_array_equal(zeta, want["node"])


def test_lm_pairs_balance_and_cover():
    from paper_2507_15209_gb300.zeta import lm_pairs
    for lmax in (0, 4, 10):
        for size in (1, 2, 3, 8):
            got = [lm_pairs(r, size, lmax) for r in range(size)]
            flat = [p for g in got for p in g]
            assert len(flat) == len(set(flat)) == (lmax + 1) ** 2
            assert max(map(len, got)) - min(map(len, got)) <= 1
