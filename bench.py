#!/usr/bin/env python
"""Benchmark of the in-situ multipole 3PCF measurement: seconds per catalogue.

One step = one full measurement of zeta_l(r1, r2), l <= lmax, for one log-normal
catalogue through libzeta's zeta_ell: B-spline assignment, R2C, the per-(l, m)
windowed C2R of every radial bin, the particle-form and node-form summations, the
mass term and the float64 reduction.  Default workload: 512^3 grid, 2000 Mpc/h box,
16M particles, lmax 10, 20 bins, cubic B-spline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one catalogue per rank (weak scaling, no collective on
the data path; only a barrier and a max-reduce of the timings), or with --partition lm
one catalogue whose (l, m) pairs are split round robin over the ranks, the per-pair
float64 slots summed by one NCCL all-reduce (strong scaling).  --impl reference
times the FP64 CPU oracle on a bounded sample of the same workload and scales it
to one catalogue.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2507_15209_gb300 import mocks  # noqa: E402
from paper_2507_15209_gb300.workloads import WORKLOADS, edges as wl_edges  # noqa: E402

METRIC = "zeta_l(r1,r2) s/catalog at Ng=512^3"
UNIT = "s/catalog"
FALLBACK_HBM_GBS = 6800.0

# dram bytes (read + write) per call of a stage, from one ncu capture of its kernels on a small
# case scaled to the 512^3 / 16M-particle / 20-bin workload by the ratio of the algorithmic bytes
# per call, and the shas of the source files they were built from (the entry is ignored once a
# source changes).  gram_particles: k_interp_part (1.446297 + 0.121082 GB) + k_gram_node_rb<16, 2>
# (0.160077 + 0.000138 GB) on the 256^3 / 2M-particle / 15-bin case, 1.727594 GB against
# 1.038633 GB algorithmic (1.663x), times 10.993418 GB.  The fields' re-read share grows with the
# grid (L2 holds a smaller part of a field), so at 512^3 this is a lower bound.
NCU_TRAFFIC = {"gram_particles": {"bytes": 18285736709,
                                  "sha": ["50434d7e3b4e428b", "c0ee103de8e92020", "4de64bc1cb299339"]}}


# the source files (under paper_2507_15209_gb300/csrc) of every stage that has algorithmic bytes,
# for matching a stored counter capture against the current sources
STAGE_SOURCES = {"assign": ["assign.cu"], "alm_z": ["fft.cu"], "alm_y": ["fft.cu"], "alm_x": ["fft.cu"],
                 "r2c": ["fft.cu"], "gram_particles": ["particles.cu", "sums.cu", "gram.cuh"],
                 "gram_node": ["sums.cu"], "mass": ["sums.cu"]}


def _sha(path):
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_timings(ms_dev, ms_e2e, steps, world, dist=None, device="cuda", shared=False):
    """Whole-job seconds per catalogue: the slowest rank's time (max over ranks) divided by all
    ranks' catalogues (steps per rank x world; steps alone when the ranks share one catalogue per
    step, as in the (l, m) split).  Returns (value, e2e value, max device ms, max end-to-end ms)."""
    import torch
    t = torch.tensor([ms_dev, ms_e2e], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    cats = steps if shared else steps * world
    return float(t[0]) / 1e3 / cats, float(t[1]) / 1e3 / cats, float(t[0]), float(t[1])


def allreduce_slots(slots, dist):
    """Sum the ranks' per-(l, m) slot arrays (float64).  Every slot has one non-zero contributor
    (its owner), so the sum is exact and the reduced zeta equals the one-GPU result bit for bit."""
    if dist is not None:
        dist.all_reduce(slots, op=dist.ReduceOp.SUM)
    return slots


def _make_inputs(w, rank):
    rho = mocks.lognormal_density(w["n"], w["field_seed"] + 100 * rank)
    parts = mocks.sample_particles(rho, w["n_p"], w["box"], w["sample_seed"] + 100 * rank)
    return parts


def _alg_bytes(stage, w, nb):
    """Algorithmic HBM bytes of one launch of a stage (minimum traffic of what it computes);
    for the assignment and the uniform term, of one catalogue."""
    ng = w["n"] ** 3
    g = 4.0 * ng  # one float grid == one half spectrum without the x-Nyquist column
    n_p = w["n_p"]
    return {
        "assign": 16.0 * n_p + g,       # per catalogue: read the particles once, write delta
        "alm_z": g * (1 + nb),          # read delta_hat once, write nb z-transformed spectra
        "alm_y": 2 * g * nb,            # read + write nb spectra
        "alm_x": 2 * g * nb,            # read nb half spectra, write nb real fields
        "gram_particles": g * nb + 16.0 * n_p,  # read nb fields once and the particles
        "gram_node": g * (nb + 1),      # read nb fields and delta
        # per catalogue, not per launch: the |n|^2 sums read delta_hat once, then each l reads
        # the table of its windows and the sums over the 3 (n/2 - 1)^2 + 1 values of |n|^2
        "mass": g + (w["lmax"] + 1) * (3 * (w["n"] // 2 - 1) ** 2 + 1) * (4.0 * 4 * ((nb + 3) // 4) + 8),
        "r2c": 2 * g,                   # per pass: read + write one grid
    }.get(stage)


SUB = 16  # fraction of a grid or a catalogue one sampled oracle step runs on


def _cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _avail_gb():
    try:
        with open("/proc/meminfo") as fh:
            for line in fh:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 16.0


def _timed(fn, *a, **k):
    t0 = time.perf_counter()
    r = fn(*a, **k)
    return r, time.perf_counter() - t0


def _oracle_prepare(w, parts, cache):
    """The per-catalogue steps of the FP64 oracle, run whole once: the assignment of the whole
    catalogue, the forward DFT (whose cost also stands for one inverse DFT of a field: the same
    transform size) and the sort of the integer |n|^2 that every window build does.  The grid,
    its DFT and the particles go to `cache` for the sample workers."""
    from oracle import zeta_oracle as O
    n = w["n"]
    p64 = parts.astype(np.float64)
    (eps, wsum), t_assign = _timed(O.assign, p64[:, :3], p64[:, 3], n, w["box"], w["dsup"])
    delta = O.contrast(eps, wsum)
    del eps
    dh, t_fft = _timed(np.fft.fftn, delta)
    iv = O.fft_integers(n)
    n2 = iv[:, None, None] ** 2 + iv[None, :, None] ** 2 + iv[None, None, :] ** 2
    (uniq, _), t_uniq = _timed(np.unique, n2, return_inverse=True)
    del n2, dh
    paths = {"delta": os.path.join(cache, "delta.npy"), "parts": os.path.join(cache, "parts.npy"),
             "kmag": os.path.join(cache, "kmag.npy")}
    np.save(paths["delta"], delta)
    np.save(paths["parts"], p64[::SUB])
    np.save(paths["kmag"], 2.0 * np.pi / w["box"] * np.sqrt(uniq.astype(np.float64)))
    return {"assign": t_assign, "fft": t_fft, "uniq": t_uniq, "paths": paths}


def _oracle_unit(job):
    """Sampled per-(l, m, b) steps of the oracle (run in a worker process), each on 1/SUB of its
    input: R_lm and the window assembly on a slab of n/SUB z-planes, jbar of the bin on every
    |n|^2, the B-spline interpolation and weighted Gram at every SUB-th particle, and the node
    Gram over a slab of the grid for all bins.  Returns the measured seconds of each step."""
    from oracle import zeta_oracle as O
    w, l, m, b, paths = job
    n, box, dsup = w["n"], w["box"], w["dsup"]
    e = wl_edges(w)
    nb = len(e) - 1
    delta = np.load(paths["delta"], mmap_mode="r")
    ps = np.load(paths["parts"])
    kmag = np.load(paths["kmag"])
    iv = O.fft_integers(n)
    nz, ny, nx = np.meshgrid(iv[: n // SUB], iv, iv, indexing="ij")
    t = {}
    ang, t["ylm"] = _timed(O.real_ylm, l, m, nx, ny, nz)
    n2 = nx * nx + ny * ny + nz * nz
    del nx, ny, nz
    jb, t["jbar"] = _timed(O.jbar, l, kmag, e[b], e[b + 1])
    t0 = time.perf_counter()
    idx = np.searchsorted((kmag * box / (2.0 * np.pi)) ** 2, n2.astype(np.float64) - 0.5)
    kern = np.sqrt(4.0 * np.pi) * (1j ** l) * jb[np.minimum(idx, len(jb) - 1)] * ang
    t["kern"] = time.perf_counter() - t0
    del kern, ang, n2, idx
    slab = np.asarray(delta[: n // SUB])
    field = np.asarray(delta)[None]
    f, t["interp"] = _timed(O.interpolate, field, ps[:, :3], n, box, dsup)
    t0 = time.perf_counter()
    _ = (f * ps[:, 3][None, :]) @ f.T
    t["interp"] += time.perf_counter() - t0
    a = np.broadcast_to(slab, (nb,) + slab.shape)
    _, t["node"] = _timed(O.sum_node, slab, np.ascontiguousarray(a))
    return t


def _oracle_sample(w, prep, cores):
    """The FP64 oracle's time per catalogue from a bounded sample (a model with stated scale
    factors), run on `cores` worker processes at once.

    Whole once per catalogue: assignment (all particles), forward DFT, |n|^2 sort.  Sampled:
    one unit per worker, each a different (l, m, b), see _oracle_unit.  Per catalogue:
      assign + DFT + (L+1)^2 [SUB ylm + uniq + SUB node + nb (jbar + SUB kern + DFT + SUB interp)]
      + (L+1) [uniq + nb jbar]           (the uniform term: one |n|^2 sort and nb jbar per l)
    with every sampled step's mean over the units; the parallel part is divided by the pool's
    measured concurrency (sum of the units' times / the pool's wall time), so the value is the
    wall time `cores` processes would take.
    """
    import multiprocessing as mp
    L1 = w["lmax"] + 1
    nb = w["nbins"]
    jobs = []
    for i in range(cores):
        l = (2 + i) % L1
        jobs.append((w, l, (i % (2 * l + 1)) - l, (3 * i + 1) % nb, prep["paths"]))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_unit, jobs)
    wall = time.perf_counter() - t0
    mean = {k: statistics.mean(r[k] for r in res) for k in res[0]}
    busy = sum(sum(r.values()) for r in res)
    conc = max(1.0, busy / wall)
    per_lm = SUB * mean["ylm"] + prep["uniq"] + SUB * mean["node"] + nb * (
        mean["jbar"] + SUB * mean["kern"] + prep["fft"] + SUB * mean["interp"])
    parallel = L1 * L1 * per_lm + L1 * (prep["uniq"] + nb * mean["jbar"])
    total = prep["assign"] + prep["fft"] + parallel / conc
    sample = (f"scaled sample of the FP64 oracle on {cores} processes: assignment of all particles, forward DFT and "
              f"the |n|^2 sort timed whole; {cores} (l,m,b) units timed on 1/{SUB} of their inputs (R_lm and the "
              f"window on n/{SUB} z-planes x{SUB}, jbar of the bin, interpolation+Gram at every {SUB}th particle "
              f"x{SUB}, node Gram on n/{SUB} z-planes x{SUB}); inverse DFT = the forward DFT's time; scaled by "
              f"(lmax+1)^2={L1 * L1} (l,m) x {nb} bins, uniform term (lmax+1)={L1} x (|n|^2 sort + {nb} jbar); "
              f"parallel part / measured concurrency {conc:.1f}")
    return total, sample


def _cpu_baseline(w, parts, reps=1):
    """Time the oracle's scaled sample `reps` times (after one preparation); returns
    (values, sample text, cores used)."""
    import tempfile
    cores = max(1, min(_cpu_cores(), int(_avail_gb() // 14)))
    with tempfile.TemporaryDirectory(prefix="zeta_cpu_") as cache:
        prep = _oracle_prepare(w, parts, cache)
        vals, sample = [], ""
        for _ in range(reps):
            v, sample = _oracle_sample(w, prep, cores)
            vals.append(v)
    return vals, sample, cores


def _gen_catalogue(args):
    n, n_p, box, fs, ss = args
    return mocks.lognormal_catalogue(n, n_p, box, fs, ss)


def _events_ms(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _gram_variants(ctx, dev, w, stream):
    """Node-form Gram per arithmetic.  On this workload: ms per launch on the fields of one (l, m)
    and speedup over float32 (tensor-core variants), and the node-form measurement alone in
    float32 against bfloat16 field storage (seconds per catalogue, relative Frobenius difference).
    On the 256^3 / 2M-particle workload: each variant's per-l relative error against the FP64
    oracle's cached result (tests/golden/zeta_box1000_n256_np2m.json)."""
    import torch
    from paper_2507_15209_gb300.zeta import Context
    nb = ctx.nbins
    delta, _ = ctx.assign(dev)
    dhat = ctx.fft_r2c(delta)
    alm = ctx.reconstruct_alm(dhat, 2, 1)
    out = {}
    for g in ("fp32", "tf32", "bf16", "bf16x3"):
        ctx.set_gram(g)
        gram = torch.zeros((nb, nb), dtype=torch.float64, device="cuda")
        ms = _events_ms(lambda: ctx.sum_grid(delta, alm, "node", gram=gram), 5, stream)
        out[g] = {"ms_per_launch": round(ms, 4)}
    del alm
    for g in out:
        out[g]["speedup_vs_fp32"] = round(out["fp32"]["ms_per_launch"] / out[g]["ms_per_launch"], 3)
    node = {}
    res = {}
    stage_ms = {}
    for g in ("fp32", "bf16_fields"):
        ctx.set_gram(g)
        node[g] = _events_ms(lambda: ctx.zeta_ell(particles=dev, forms=("node",)), 1, stream) / 1e3
        ctx.profile_enable(True)
        res[g] = ctx.zeta_ell(particles=dev, forms=("node",))["node"].cpu().numpy()
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        stage_ms[g] = {k: round(v[0] / max(v[2], 1), 4) for k, v in prof.items()
                       if k in ("alm_x", "gram_node") and v[1]}
    ctx.set_gram("fp32")
    out["node_form_s_per_catalog"] = {g: round(v, 4) for g, v in node.items()}
    out["node_form_ms_per_call"] = stage_ms
    out["node_gram_bf16_fields_speedup"] = round(stage_ms["fp32"]["gram_node"] / stage_ms["bf16_fields"]["gram_node"],
                                                 3)
    out["node_form_bf16_fields_speedup"] = round(node["fp32"] / node["bf16_fields"], 3)
    out["node_form_bf16_fields_rel_diff"] = float(np.linalg.norm(res["bf16_fields"] - res["fp32"])
                                                  / np.linalg.norm(res["fp32"]))
    gpath = os.path.join(ROOT, "tests", "golden", "zeta_box1000_n256_np2m.json")
    if os.path.exists(gpath):
        with open(gpath) as fh:
            gold = json.load(fh)["data"]
        w2 = WORKLOADS["box1000_n256_np2m"]
        parts = mocks.lognormal_catalogue(w2["n"], w2["n_p"], w2["box"], w2["field_seed"], w2["sample_seed"])
        want = np.array(gold["zeta"]["node"])
        c2 = Context(w2["n"], w2["box"], w2["dsup"], w2["lmax"], wl_edges(w2), np_max=len(parts), forms=("node",))
        p2 = torch.from_numpy(parts).cuda()
        errs = {}
        for g in ("fp32", "tf32", "bf16", "bf16x3", "bf16_fields"):
            c2.set_gram(g)
            got = c2.zeta_ell(particles=p2, forms=("node",))["node"].cpu().numpy()
            errs[g] = [float(f"{np.linalg.norm(got[l] - want[l]) / np.linalg.norm(want[l]):.2e}")
                       for l in range(want.shape[0])]
        c2.close()
        out["per_l_rel_err_vs_fp64_oracle_box1000_n256"] = errs
    return out


def _batch_sample(ncat, stream):
    """Batched (one CUDA-graph launch) against one-by-one zeta_ell on ncat catalogues of the
    batched workload (256^3, lmax 8, 12 bins, sizes drawn uniformly in 0.5M-4M)."""
    import multiprocessing as mp
    import torch
    from paper_2507_15209_gb300.workloads import batch_seeds
    from paper_2507_15209_gb300.zeta import Context
    w = WORKLOADS["batch64_n256"]
    sizes = mocks.batch_sizes(w["n_cat"], w["n_p_lo"], w["n_p_hi"], w["size_seed"])[:ncat]
    jobs = [(w["n"], int(sizes[i]), w["box"], *batch_seeds(i)) for i in range(ncat)]
    with mp.get_context("spawn").Pool(min(ncat, 8)) as pool:
        cats = pool.map(_gen_catalogue, jobs)
    allp = torch.from_numpy(np.concatenate(cats)).cuda()
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    e = wl_edges(w)
    views = [allp[int(offs[i]):int(offs[i + 1])] for i in range(ncat)]
    out = torch.empty((ncat, 1, w["lmax"] + 1, len(e) - 1, len(e) - 1), dtype=torch.float64, device="cuda")
    res = {"workload": "batch64_n256", "catalogues": ncat, "particles": int(sizes.sum())}
    for copies in (1, 2, 3):
        ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=int(sizes.max()), forms=("particle",),
                      ws_copies=copies)
        if copies == 1:
            res["tuned_ctas_per_sm"] = ctx.autotune(allp[: int(sizes[0])], forms=("particle",))
            tuned, staging = res["tuned_ctas_per_sm"], ctx.staging()

            def one_by_one():
                for i in range(ncat):
                    ctx.zeta_ell(particles=views[i], forms=("particle",), out=out[i])

            ms_seq = _events_ms(one_by_one, 2, stream)
            res["s_per_catalog_one_by_one"] = ms_seq / 1e3 / ncat
        else:
            ctx.set_tuning(tuned)
            ctx.set_staging(staging)
        ms_batch = _events_ms(lambda: ctx.batch(allp, offs, forms=("particle",), out=out), 2, stream)
        res[f"s_per_catalog_batched_{copies}_in_flight"] = ms_batch / 1e3 / ncat
        res[f"speedup_{copies}_in_flight"] = round(ms_seq / ms_batch, 4)
        ctx.close()
    return res


def _cufft_reference(w, nb, stages, stream):
    """cuFFT (torch.fft, a library) on the inverse transforms of one (l, m) beside this
    library's own passes, for reference only: batched irfftn of nb half spectra of the workload
    grid.  Our side is the window pass + y-pass + x-pass time per (l, m) from the stage timers
    (which also applies the window and writes bin-interleaved fields)."""
    import torch
    n = w["n"]
    spec = torch.complex(torch.randn((nb, n, n, n // 2 + 1), device="cuda"),
                         torch.randn((nb, n, n, n // 2 + 1), device="cuda"))
    ms = _events_ms(lambda: torch.fft.irfftn(spec, s=(n, n, n), dim=(1, 2, 3)), 3, stream)
    del spec
    torch.cuda.empty_cache()
    ours = sum(stages[k]["ms"] / stages[k]["launches"] for k in ("alm_z", "alm_y", "alm_x") if k in stages)
    return {"fields": nb, "grid": n, "cufft_irfftn_ms": round(ms, 3), "ours_window_plus_c2r_ms": round(ours, 3)}


def _catalogue_bytes(w, nb, forms):
    """One-pass algorithmic HBM bytes of one catalogue (the minimum traffic of the whole path):
    assignment 16 N_p + 4 N_g, R2C 16 N_g, and per (l, m) the delta_hat read, each field written
    once and read once after a single transpose round trip (16 N_g per field), the particles
    (particle form) and the delta re-read plus a second field read (node form)."""
    ng = w["n"] ** 3
    n_p = w["n_p"]
    per_lm = 4 * ng * (1 + 4 * nb)
    if "particle" in forms:
        per_lm += 16 * n_p
    if "node" in forms:
        per_lm += 4 * ng * (nb + 1)
    return 16 * n_p + 4 * ng + 16 * ng + (w["lmax"] + 1) ** 2 * per_lm


def _adjoint_ratio(stream):
    """Gradient cost on the adjoint workload (256^3 grid and 1M particles, lmax 6, 10 bins):
    backward / forward time of the node form (dL/d delta) and the particle form (dL/dx)."""
    import torch
    from paper_2507_15209_gb300.zeta import Context
    w = WORKLOADS["adjoint_n256_np1m"]
    rho = mocks.lognormal_density(w["n"], w["field_seed"])
    delta = torch.from_numpy((rho - 1.0).astype(np.float32)).cuda()
    parts = torch.from_numpy(mocks.sample_particles(rho, w["n_p"], w["box"], w["sample_seed"])).cuda()
    wts = mocks.loss_weights(w["lmax"], w["nbins"], w["loss_seed"])
    e = wl_edges(w)
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=("node", "particle", "backward"))
    f_node = _events_ms(lambda: ctx.zeta_ell(delta=delta, forms=("node",)), 2, stream)
    b_node = _events_ms(lambda: ctx.backward_node(delta, wts), 2, stream)
    f_part = _events_ms(lambda: ctx.zeta_ell(particles=parts, forms=("particle",)), 2, stream)
    b_part = _events_ms(lambda: ctx.backward_particles(parts, wts), 2, stream)
    ctx.close()
    return {"workload": "adjoint_n256_np1m", "node_forward_ms": f_node, "node_backward_ms": b_node,
            "node_backward_over_forward": round(b_node / f_node, 3), "particle_forward_ms": f_part,
            "particle_backward_ms": b_part, "particle_backward_over_forward": round(b_part / f_part, 3)}


def _extension_rows(stream):
    """The extension rows on the 256^3 / 2M-particle workload (lmax 10, 15 bins, cubic B-spline
    unless stated), seconds per catalogue (CUDA events, 2 repetitions after a warm-up) and the
    ratio to the plain measurement of the same forms:
      plain      zeta_ell, particle + node forms
      windows    the same with point radii (the bin centres), a secondary tophat of one cell,
                 Phi-hat and a primary tophat of one cell (Fig. 1 steps (3)-(4), Sec. 3)
      daub4      the same forms on the Daubechies basis (dsup 3)
      ss         the Szapudi-Szalay numerator and denominator (node form) with a uniform random
                 catalogue of 2M points (Eq. SSestimator); ratio to the plain node form
      xi         the 2PCF of every bin in both forms (Eq. pair-counting); ratio to the plain
                 particle + node measurement
      gamma      the connection-coefficient form of the grid sum (Eqs. con-coeff, SFC-3PCF) with
                 each basis, ms per (l, m) beside the node form's Gram on the same fields"""
    import torch
    from paper_2507_15209_gb300.zeta import Context
    w = WORKLOADS["box1000_n256_np2m"]
    e = wl_edges(w)
    nb = len(e) - 1
    parts = torch.from_numpy(mocks.lognormal_catalogue(w["n"], w["n_p"], w["box"], w["field_seed"],
                                                       w["sample_seed"])).cuda()
    rand = torch.from_numpy(mocks.uniform_particles(w["n_p"], w["box"], 7001)).cuda()
    h = w["box"] / w["n"]
    both = ("particle", "node")
    res = {"workload": "box1000_n256_np2m", "unit": "s/catalog"}

    def run(key, fn, ctx):
        ms = _events_ms(fn, 2, stream)
        assert ctx.get_status() == 0
        ctx.close()
        res[key] = round(ms / 1e3, 5)

    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=both)
    run("plain", lambda: ctx.zeta_ell(particles=parts, forms=both), ctx)
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=("node",))
    run("plain_node", lambda: ctx.zeta_ell(particles=parts, forms=("node",)), ctx)
    radii = 0.5 * (e[:-1] + e[1:])
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], None, np_max=w["n_p"], forms=both, radial="point",
                  radii=radii, tophat=h, phi_hat=True, tophat_primary=h)
    run("windows", lambda: ctx.zeta_ell(particles=parts, forms=both), ctx)
    ctx = Context(w["n"], w["box"], 3, w["lmax"], e, np_max=w["n_p"], forms=both)
    run("daub4", lambda: ctx.zeta_ell(particles=parts, forms=both), ctx)
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=("node", "ss"))
    run("ss", lambda: ctx.zeta_ell_ss(parts, rand, forms=("node",)), ctx)
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=both)
    run("xi", lambda: ctx.xi(particles=parts, forms=both), ctx)
    for k in ("windows", "daub4", "xi"):
        res[k + "_over_plain"] = round(res[k] / res["plain"], 4)
    res["ss_over_plain_node"] = round(res["ss"] / res["plain_node"], 4)
    # the connection-coefficient (Gamma) form of the grid sum, per (l, m) of lmax 1 on the same grid
    # (its cost grows as the cube of the cell's quadrature points times the stencil: D^6)
    delta = None  # the catalogue's contrast (linear assignment) serves every basis as input data
    gam = {}
    for dsup, name in ((2, "linear"), (4, "cubic"), (3, "daub4")):
        ctx = Context(w["n"], w["box"], dsup, 1, e, np_max=w["n_p"], forms=("gamma", "node"))
        if delta is None:
            delta, _ = ctx.assign(parts)
        ctx.zeta_ell(delta=delta, forms=("gamma", "node"))
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        ctx.zeta_ell(delta=delta, forms=("gamma", "node"))
        torch.cuda.synchronize()
        p = ctx.profile_read()
        ctx.profile_enable(False)
        ctx.close()
        gam[name] = {"gamma_ms_per_lm": round(p["gram_gamma"][0] / p["gram_gamma"][2], 3),
                     "node_ms_per_lm": round(p["gram_node"][0] / p["gram_node"][2], 3)}
    res["gamma_form_per_lm"] = gam
    del parts, rand
    torch.cuda.empty_cache()
    return res


def _emit(d):
    print(json.dumps(d), flush=True)


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    parts = _make_inputs(w, 0)
    vals, sample, cpu_threads = _cpu_baseline(w, parts, reps=args.warmup + args.steps)
    v = statistics.median(vals[args.warmup:])
    _emit({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic log-normal mock (seeded)",
        "config": {"workload": args.workload, "n": w["n"], "box": w["box"], "n_p": w["n_p"], "lmax": w["lmax"],
                   "nbins": w["nbins"], "dsup": w["dsup"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_threads, "kind": "oracle, scaled sample",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })
    return 0


def run_ours(args, w, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_2507_15209_gb300 import build as zbuild
    zbuild.build()
    from paper_2507_15209_gb300.zeta import Context

    forms = tuple(args.forms.split(","))
    lm_split = args.partition == "lm" and world > 1
    parts = _make_inputs(w, 0 if lm_split else rank)
    e = wl_edges(w)
    nb = len(e) - 1
    ctx = Context(w["n"], w["box"], w["dsup"], w["lmax"], e, np_max=w["n_p"], forms=forms)
    host = torch.from_numpy(parts).pin_memory()
    dev = host.to("cuda", non_blocking=True)
    nforms = len(forms)
    out = torch.empty((nforms, w["lmax"] + 1, nb, nb), dtype=torch.float64, device="cuda")
    out_host = torch.empty(out.shape, dtype=torch.float64).pin_memory()
    stream = torch.cuda.current_stream()
    if lm_split:  # this rank's (l, m) pairs, an FP64 all-reduce of the slots, the fixed-order sum
        slots = torch.empty(ctx.lm_slots(forms), dtype=torch.float64, device="cuda")

        def measure():
            ctx.zeta_lm(rank, world, particles=dev, forms=forms, out=slots)
            allreduce_slots(slots, dist)
            ctx.reduce_lm(slots, forms=forms, out=out)
    else:
        def measure():
            ctx.zeta_ell(particles=dev, forms=forms, out=out)

    for _ in range(args.warmup):
        measure()
    torch.cuda.synchronize()
    if ctx.get_status() != 0:
        raise RuntimeError("device status error during warm-up")

    props = torch.cuda.get_device_properties(local_rank)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local_rank)
    clocks = ClockSampler(gpu_id)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # device-timed region: inputs resident in HBM
    clocks.start()
    ctx.profile_enable(True)
    barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        measure()
    t1.record(stream)
    barrier()
    ms_dev = t0.elapsed_time(t1)
    prof = ctx.profile_read()
    ctx.profile_enable(False)

    # end-to-end region: host particles -> device, measurement, result -> host, every step
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dev.copy_(host, non_blocking=True)
        measure()
        out_host.copy_(out, non_blocking=True)
    e1.record(stream)
    barrier()
    ms_e2e = e0.elapsed_time(e1)
    ck = clocks.stop()
    if ctx.get_status() != 0:
        raise RuntimeError("device status error in the timed region")

    value, e2e_value, ms_dev, ms_e2e = reduce_timings(ms_dev, ms_e2e, args.steps, world, dist, shared=lm_split)

    if rank == 0:
        peak, peak_src = _peaks()
        # dominant memory-bound kernel
        rows = {k: v for k, v in prof.items() if v[1] > 0 and k != "mass" and _alg_bytes(k, w, nb) is not None}
        dom = max(rows, key=lambda k: rows[k][0])
        # per call of the stage (a stage is one kernel launch per call, except the particle
        # form when its threshold splits tile batches between the staged and the L1 kernel)
        ms_k, launches_k, calls_k = rows[dom]
        bytes_launch = _alg_bytes(dom, w, nb)
        achieved = bytes_launch * calls_k / (ms_k / 1e3) / 1e9
        src = STAGE_SOURCES[dom]
        tr = NCU_TRAFFIC.get(dom)
        traffic = None
        if tr and tr["sha"] == [_sha(os.path.join(ROOT, "paper_2507_15209_gb300", "csrc", f)) for f in src]:
            traffic = tr["bytes"]
        gpu_launches = sum(v[1] for v in prof.values())
        stages = {k: {"ms": round(v[0] / args.steps, 3), "launches": v[1] // args.steps}
                  for k, v in prof.items() if v[1]}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_dev / args.steps, "higher_is_better": False,
            "scaling": "strong" if lm_split else "weak", "vs_baseline": None, "dtype": "f32",
            "data": ("synthetic log-normal mock (seeded), one catalogue shared by all ranks" if lm_split
                     else "synthetic log-normal mock (seeded), one catalogue per rank"),
            "config": {"workload": args.workload, "n": w["n"], "box": w["box"], "n_p": w["n_p"],
                       "lmax": w["lmax"], "nbins": nb, "dsup": w["dsup"], "forms": list(forms),
                       "gram": "fp32", "l2": "inputs larger than L2 (fields 20 x 512 MB, particles 256 MB)",
                       "parallelism": f"lm-split x{world}" if lm_split else f"catalogue-per-gpu x{world}"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                         "alg_bytes_per_call": bytes_launch, "calls": calls_k, "launches": launches_k,
                         "avg_call_ms": ms_k / calls_k},
            "stages_ms_per_step": stages,
            "clocks": ck,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(parts.nbytes),
                    "d2h_bytes_per_step": int(out.numel() * 8)},
            "gpu_launches": int(gpu_launches),
        }
        cat_bytes = _catalogue_bytes(w, nb, forms)
        line["catalogue_roofline"] = {"alg_bytes": cat_bytes, "achieved_gbs": cat_bytes / value / 1e9,
                                      "peak_gbs": peak, "frac": cat_bytes / value / 1e9 / peak}
        units = lambda k, v: {"r2c": v[1], "mass": args.steps}.get(k, v[2])  # noqa: E731
        line["stage_gbs"] = {k: round(_alg_bytes(k, w, nb) * units(k, v) / (v[0] / 1e3) / 1e9, 1)
                             for k, v in prof.items() if v[1] > 0 and _alg_bytes(k, w, nb) is not None}
        extras = set() if args.no_extras else set(args.extras.split(","))
        if "variants" in extras:
            line["gram_variants"] = _gram_variants(ctx, dev, w, stream)
        if "batch" in extras:
            line["batch_sample"] = _batch_sample(8, stream)
        if "adjoint" in extras:
            line["adjoint"] = _adjoint_ratio(stream)
        if "cufft" in extras:
            line["cufft_reference"] = _cufft_reference(w, nb, stages, stream)
        if "rows" in extras:
            line["extension_rows"] = _extension_rows(stream)
        if world == 1 and not args.no_cpu_baseline:
            vals, sample, cores = _cpu_baseline(w, parts)
            line["cpu_baseline"] = {"value": vals[0], "unit": UNIT, "cores": cores, "kind": "oracle, scaled sample",
                                    "sample": sample}
        _emit(line)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="box2000_n512_np16m")
    ap.add_argument("--forms", default="particle,node")
    ap.add_argument("--partition", default="catalogue", choices=["catalogue", "lm"],
                    help="N > 1: one catalogue per rank (weak scaling, no collective) or one catalogue split "
                         "over (l, m) pairs with an FP64 all-reduce of the per-pair slots (strong scaling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the Gram-variant, batch and adjoint extras")
    ap.add_argument("--extras", default="variants,batch,adjoint,cufft,rows", help="comma list of extras to measure")
    ap.add_argument("--lmax", type=int, default=None, help="override lmax (small profiling runs only)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = dict(WORKLOADS[args.workload])
    if args.lmax is not None:
        w["lmax"] = args.lmax
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    return run_ours(args, w, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
