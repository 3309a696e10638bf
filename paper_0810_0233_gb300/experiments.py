"""Scaling experiments of Sec. IV redone on the GPU (synthetic lattices).

* scaling():  time of the fast method against system size for random
  dipoles on an n^3 simple cubic lattice, with the brute-force sum beside it
  (the paper's Fig. 1: linear complexity, crossover with the O(N^2) sum);
* leaf_sweep(): time against the leaf occupancy s for the 32^3 lattice at
  (p, alpha) = (3, 0.54) (the paper's Table I, whose optimum is s = 8);
* optimal_leaf(): the best occupancy s_o(p), averaged over lattices 30^3 ..
  59^3 as in Fig. 2, to set beside the rule of thumb of Eq. so.

Times are CUDA-event times of the library's own call sequence (tree, lists
and D tables, then the field) on the current device, best of `repeats`.  The
brute force is the library's FP64 direct sum.  Nothing here computes the
method: every step runs in libccfmm.

Run on a GPU:  python -m paper_0810_0233_gb300.experiments [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import ccfmm as C
from . import workloads as W


def _timer():
    import torch
    stream = torch.cuda.current_stream()

    def run(fn, repeats):
        best = float("inf")
        for _ in range(repeats):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best  # ms

    return run, stream


def _lattice(n, seed):
    pos, mom, box = W.lattice(n, seed=seed)
    return pos, mom, box


def fmm_ms(pos, mom, box, p, theta, leaf, repeats=3, precision="mixed"):
    """Best time (ms) of set_positions + field for one configuration."""
    import torch
    run, stream = _timer()
    pd = torch.from_numpy(pos).cuda()
    md = torch.from_numpy(mom).cuda()
    H = torch.zeros((len(pos), 3), dtype=torch.float64, device="cuda")
    with C.FMM(pd, md, p, theta, leaf, box=box, precision=precision, stream=stream) as f:
        f.field(H)

        def step():
            f.set_positions(pd, md)
            f.field(H)

        ms = run(step, repeats)
        depth = f.stats()["depth"]
    return ms, depth


def direct_ms(pos, mom, repeats=2):
    import torch
    run, stream = _timer()
    pd = torch.from_numpy(pos).cuda()
    md = torch.from_numpy(mom).cuda()
    out = torch.zeros((len(pos), 3), dtype=torch.float64, device="cuda")
    return run(lambda: C.direct_field(pd, md, out=out, stream=stream), repeats)


def scaling(sizes=(8, 10, 13, 16, 20, 25, 32, 40, 50, 63, 79, 100),
            params=((4, 0.5), (5, 0.71)), direct_max=200_000, seed=1):
    """Fig. 1: time against N; the direct sum up to direct_max points."""
    rows = []
    for n in sizes:
        pos, mom, box = _lattice(n, seed + n)
        row = {"n": n, "N": len(pos)}
        for p, th in params:
            ms, L = fmm_ms(pos, mom, box, p, th, 0.0)
            row["fmm_p%d_a%.2f_ms" % (p, th)] = ms
            row["depth_p%d" % p] = L
        if len(pos) <= direct_max:
            row["direct_ms"] = direct_ms(pos, mom)
        rows.append(row)
    return rows


def leaf_sweep(n=32, p=3, theta=0.54, leaves=(1, 2, 4, 8, 16, 32, 64), seed=2):
    """Table I: time against the leaf occupancy s."""
    pos, mom, box = _lattice(n, seed)
    out = []
    for s in leaves:
        ms, L = fmm_ms(pos, mom, box, p, theta, float(s))
        out.append({"s": s, "depth": L, "ms": ms})
    return out


def optimal_leaf(ps=(2, 3, 4, 5, 6, 7, 8), sizes=range(30, 60), theta=0.54, seed=3):
    """Fig. 2: for each p and lattice size, the occupancy N / 2^L of the
    fastest depth L; s_o(p) is its mean over the sizes."""
    res = {}
    for p in ps:
        best_s = []
        for n in sizes:
            pos, mom, box = _lattice(n, seed + n)
            N = len(pos)
            times = {}
            # every depth whose mean occupancy lies in [1, 512]
            for L in range(max(1, int(math.log2(N / 512.0))), int(math.log2(N)) + 1):
                ms, depth = fmm_ms(pos, mom, box, p, theta, N / 2.0 ** L, repeats=2)
                times[depth] = min(ms, times.get(depth, float("inf")))
            Lb = min(times, key=times.get)
            best_s.append(N / 2.0 ** Lb)
        res[p] = {"s_o": float(np.mean(best_s)), "s_per_size": best_s,
                  "rule": C.leaf_size_rule(p)}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer sizes (smoke run)")
    ap.add_argument("--out", default="experiments.json")
    args = ap.parse_args()
    t0 = time.time()
    res = {}
    if args.quick:
        res["scaling"] = scaling(sizes=(8, 16, 32), params=((4, 0.5),))
        res["leaf_sweep"] = leaf_sweep(leaves=(4, 8, 16))
        res["optimal_leaf"] = optimal_leaf(ps=(3, 5), sizes=(30, 31))
    else:
        res["scaling"] = scaling()
        print(json.dumps(res["scaling"]), flush=True)
        res["leaf_sweep"] = leaf_sweep()
        print(json.dumps(res["leaf_sweep"]), flush=True)
        res["optimal_leaf"] = optimal_leaf()
    res["seconds"] = time.time() - t0
    json.dump(res, open(args.out, "w"), indent=1)
    print(json.dumps({k: v for k, v in res.items() if k != "optimal_leaf"}), flush=True)
    print(json.dumps({p: {"s_o": v["s_o"], "rule": v["rule"]}
                      for p, v in res["optimal_leaf"].items()}), flush=True)


if __name__ == "__main__":
    main()
