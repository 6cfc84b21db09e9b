#!/usr/bin/env python
"""Write the FP64 oracle's zeta_l of a named workload to tests/golden/ (test infrastructure).

Only the FP64 oracle (oracle/zeta_oracle.py) computes anything here; the seeded catalogue comes
from the input generator (paper_2507_15209_gb300.mocks), which holds none of the method's
arithmetic.  The steps are the oracle's own, in the order of the paper's Fig. 1:
  (2) assign + contrast + DFT                      O.assign, O.contrast, numpy fftn
  (3)-(5) per (l, m): the fields of every bin      O.multipole_fields
  (6) per (l, m): node form, Gamma form and the    O.sum_node, O.sum_gamma, O.interpolate
      particle form                                (the sums of O.sum_particles)
      per l: the uniform term U_l summed over m    O.mass_term_fourier
  (7) zeta_l = sum_m ..., symmetrised
The (l, m) pairs run in a process pool and are checkpointed one file each in --cache, so an
interrupted run resumes.  The output JSON holds, per form, zeta[l][b1][b2] and the condition
sum (sum of absolute values of the summed terms), the SHA-256 of the catalogue it was computed
on, and the command.

  python tests/golden/make_zeta_golden.py box1000_n256_np2m --forms particle,node --procs 4
  python tests/golden/make_zeta_golden.py box500_n64_np20k --forms node,gamma,particle --null
  python tests/golden/make_zeta_golden.py batch64_n256 --catalogue 3 --forms particle --procs 6

For the batched workload (uneven catalogue sizes) --catalogue picks catalogue i of the batch
(its size from the workload's size draw, its seeds from batch_seeds(i)); the output is then
tests/golden/zeta_<workload>_cat<i>.json.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import zeta_oracle as O  # noqa: E402
from paper_2507_15209_gb300 import mocks  # noqa: E402
from paper_2507_15209_gb300.workloads import WORKLOADS, batch_seeds, edges as wl_edges  # noqa: E402

BIN_GROUP = 5  # fields built per oracle call (bounds the memory of one worker)


def catalogue(w: dict, null: bool, cat: int = -1) -> np.ndarray:
    if "n_cat" in w:  # one catalogue of a batched workload
        sizes = mocks.batch_sizes(w["n_cat"], w["n_p_lo"], w["n_p_hi"], w["size_seed"])
        return mocks.lognormal_catalogue(w["n"], int(sizes[cat]), w["box"], *batch_seeds(cat))
    if null:
        return mocks.uniform_particles(w["n_p"], w["box"], w["null_seed"])
    return mocks.lognormal_catalogue(w["n"], w["n_p"], w["box"], w["field_seed"], w["sample_seed"])


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _one_lm(job):
    """Per-(l, m) sums of one catalogue, written to the cache (skipped when already there)."""
    ell, m, cfg = job
    out = os.path.join(cfg["cache"], f"lm_{ell}_{m}.npz")
    if os.path.exists(out):
        return out
    w, forms = cfg["w"], cfg["forms"]
    n, box, dsup = w["n"], w["box"], w["dsup"]
    e = wl_edges(w)
    nb = len(e) - 1
    dh = np.load(cfg["dh"], mmap_mode="r")
    delta = np.load(cfg["delta"], mmap_mode="r")
    parts = np.load(cfg["parts"], mmap_mode="r").astype(np.float64)
    a = np.empty((nb, n, n, n))
    for b0 in range(0, nb, BIN_GROUP):
        bins = list(range(b0, min(nb, b0 + BIN_GROUP)))
        a[bins] = O.multipole_fields(np.asarray(dh), ell, m, n, box, e, bins=bins)
    res = {}
    d = np.asarray(delta)
    if "node" in forms:
        res["node"] = O.sum_node(d, a)
        res["node_cond"] = O.sum_node(np.abs(d), np.abs(a))
    if "gamma" in forms:
        res["gamma"] = O.sum_gamma(d, a, dsup)
    if "particle" in forms:
        pos, wt = parts[:, :3], parts[:, 3]
        f = O.interpolate(a, pos, n, box, dsup)
        wsum = float(wt.sum())
        res["particle"] = (f * wt[None, :]) @ f.T / wsum
        res["particle_cond"] = (np.abs(f) * np.abs(wt)[None, :]) @ np.abs(f).T / wsum
    tmp = out + ".tmp.npz"
    np.savez(tmp, **res)
    os.replace(tmp, out)
    return out


def run(name: str, forms, null: bool, procs: int, cache: str, cat: int = -1) -> dict:
    w = dict(WORKLOADS[name])
    n, box, lmax, dsup = w["n"], w["box"], w["lmax"], w["dsup"]
    e = wl_edges(w)
    nb = len(e) - 1
    parts = catalogue(w, null, cat)
    os.makedirs(cache, exist_ok=True)
    eps, wsum = O.assign(parts[:, :3].astype(np.float64), parts[:, 3].astype(np.float64), n, box, dsup)
    delta = O.contrast(eps, wsum)
    dh = np.fft.fftn(delta)
    paths = {k: os.path.join(cache, k + ".npy") for k in ("dh", "delta", "parts")}
    np.save(paths["dh"], dh)
    np.save(paths["delta"], delta)
    np.save(paths["parts"], parts)
    cfg = {"w": w, "forms": list(forms), "cache": cache, **paths}
    jobs = [(ell, m, cfg) for ell in range(lmax, -1, -1) for m in range(-ell, ell + 1)]
    t0 = time.time()
    with mp.get_context("spawn").Pool(procs) as pool:
        for i, _ in enumerate(pool.imap_unordered(_one_lm, jobs)):
            print(f"  {name}{' (null)' if null else ''}: {i + 1}/{len(jobs)} (l, m) done, {time.time() - t0:.0f} s",
                  flush=True)
    zeta = {f: np.zeros((lmax + 1, nb, nb)) for f in forms}
    cond = {f: np.zeros((lmax + 1, nb, nb)) for f in forms if f != "gamma"}
    for ell in range(lmax + 1):
        for m in range(-ell, ell + 1):
            r = np.load(os.path.join(cache, f"lm_{ell}_{m}.npz"))
            for f in forms:
                zeta[f][ell] += r[f]
                if f in cond:
                    cond[f][ell] += r[f + "_cond"]
        if "particle" in forms:
            u = O.mass_term_fourier(dh, ell, n, box, e, dsup)
            zeta["particle"][ell] -= u
            cond["particle"][ell] += np.abs(u)
    sym = lambda x: 0.5 * (x + np.swapaxes(x, -1, -2))  # noqa: E731
    return {
        "workload": name, "catalogue": "uniform null" if null else "log-normal",
        "batch_index": cat if "n_cat" in w else None,
        "catalogue_sha256": sha(parts), "n": n, "box": box, "lmax": lmax, "dsup": dsup, "edges": e.tolist(),
        "n_p": int(len(parts)), "wsum": wsum,
        "zeta": {f: sym(v).tolist() for f, v in zeta.items()},
        "cond": {f: sym(v).tolist() for f, v in cond.items()},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--forms", default="particle,node")
    ap.add_argument("--null", action="store_true", help="also the uniform null catalogue of the workload")
    ap.add_argument("--procs", type=int, default=max(1, min(8, (os.cpu_count() or 2) // 2)))
    ap.add_argument("--cache", default=None, help="checkpoint directory (default: a temporary one)")
    ap.add_argument("--catalogue", type=int, default=-1, help="catalogue index of a batched workload")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    if ("n_cat" in WORKLOADS[args.workload]) != (args.catalogue >= 0):
        ap.error("--catalogue is required for a batched workload and only there")
    forms = tuple(args.forms.split(","))
    cache = args.cache or tempfile.mkdtemp(prefix="zeta_golden_")
    argv = []
    skip = False
    for a in sys.argv[1:]:  # the checkpoint directory is not part of the result's recipe
        if skip or a == "--cache" or a.startswith("--cache="):
            skip = a == "--cache"
            continue
        argv.append(a)
    res = {"command": "python tests/golden/make_zeta_golden.py " + " ".join(argv),
           "oracle": "oracle/zeta_oracle.py (FP64)", "data": run(args.workload, forms, False, args.procs,
                                                                  os.path.join(cache, "data"), args.catalogue)}
    if args.null:
        res["null"] = run(args.workload, forms, True, args.procs, os.path.join(cache, "null"))
    tag = f"_cat{args.catalogue}" if args.catalogue >= 0 else ""
    out = args.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"zeta_{args.workload}{tag}.json")
    with open(out, "w") as fh:
        json.dump(res, fh, indent=None, separators=(",", ":"))
        fh.write("\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
