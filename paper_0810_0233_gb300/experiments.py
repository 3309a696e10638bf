"""Scaling experiments of Sec. IV redone on the GPU (synthetic lattices).

* scaling():  time of the fast method against system size for random
  dipoles on an n^3 simple cubic lattice, with the brute-force sum beside it
  (the paper's Fig. 1: linear complexity, crossover with the O(N^2) sum);
* leaf_sweep(): time against the leaf occupancy s for the 32^3 lattice at
  (p, alpha) = (3, 0.54) (the paper's Table I, whose optimum is s = 8);
* optimal_leaf(): the best occupancy s_o(p), averaged over lattices 30^3 ..
  59^3 as in Fig. 2, to set beside the rule of thumb of Eq. so;
* error_budget(): for error estimates e = [alpha/(2 - alpha)]^p (Sec. IV),
  every order p with the alpha that meets e, timed on the 32^3 lattice with
  the measured field and energy errors against the direct sum (Table II and
  the optimal-time-versus-accuracy curve of Fig. 3).
* fft_comparator(): the FFT lattice convolution (the comparator of Sec. V)
  against the fast method on n^3 lattices: time per evaluation of each (FFT
  in FP64 and FP32; the fast method at the paper's (5, 0.71) and at
  (6, 0.5), tree included) and each one's error against the direct sum.
* truncation(): the square truncation of Eq. taylorcalc against the
  total-degree one (terms |n|+|k| <= p+1) on the ferrofluid workload: field
  error against the direct sum, evaluation time, and the M2L stage time of
  the tensor-core and the FP32 FMA engines.

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


def alpha_for(e, p):
    """The opening angle whose error estimate [alpha/(2-alpha)]^p equals e."""
    r = e ** (1.0 / p)
    return 2.0 * r / (1.0 + r)


def error_budget(n=32, es=(0.05, 0.01, 1e-3, 2e-4), ps=(2, 3, 4, 5, 6, 7, 8), seed=4):
    """Table II / Fig. 3: time per (e, p) and the errors actually reached."""
    import torch
    run, stream = _timer()
    pos, mom, box = _lattice(n, seed)
    pd = torch.from_numpy(pos).cuda()
    md = torch.from_numpy(mom).cuda()
    Hd = C.direct_field(pd, md, stream=stream)
    Ed = -0.5 * float((mom * Hd).sum())
    H = torch.zeros((len(pos), 3), dtype=torch.float64, device="cuda")
    rows = []
    for e in es:
        for p in ps:
            a = alpha_for(e, p)
            with C.FMM(pd, md, p, a, 0.0, box=box, stream=stream) as f:
                _, E = f.field_energy(H)

                def step():
                    f.set_positions(pd, md)
                    f.field(H)

                ms = run(step, 3)
                Hf = H.cpu().numpy()
            err = float(np.sqrt(((Hf - Hd) ** 2).sum() / (Hd ** 2).sum()))
            rows.append({"e": e, "p": p, "alpha": a, "ms": ms, "rms_field_error": err,
                         "energy_error": abs(E - Ed) / abs(Ed)})
    best = {}
    for e in es:
        cand = [r for r in rows if r["e"] == e]
        b = min(cand, key=lambda r: r["ms"])
        best[e] = {"p": b["p"], "alpha": b["alpha"], "ms": b["ms"]}
    return {"rows": rows, "fastest": best}


def truncation(n=1_000_000, ps=(4, 5, 6, 7), theta=0.5, nsub=10_000, evals=10, seed=5):
    """Square against total-degree truncation on the ferrofluid (one dipole
    per unit volume, minimum separation 0.5), mixed precision."""
    import os
    import torch
    pos, mom = W.ferrofluid(n, side=n ** (1.0 / 3.0), seed=810233 + 50 + seed)
    stream = torch.cuda.current_stream()
    pd = torch.from_numpy(pos).cuda()
    md = torch.from_numpy(mom).cuda()
    sub = np.random.default_rng(seed).choice(n, min(nsub, n), replace=False)
    Hd = C.direct_field(pd, md, targets=torch.from_numpy(sub).cuda(), stream=stream)
    H = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    saved = os.environ.get("CCFMM_M2L")
    rows = []
    try:
        for p in ps:
            for bound in (None, p + 1):
                row = {"p": p, "max_degree": 2 * p if bound is None else bound,
                       "truncation": "square" if bound is None else "total degree"}
                for eng in ("tc", "fma"):
                    os.environ["CCFMM_M2L"] = eng
                    with C.FMM(pd, md, p, theta, stream=stream) as f:
                        f.set_truncation(bound)
                        f.field(H)
                        if eng == "tc":
                            Hf = H.cpu().numpy()[sub]
                            row["rms_field_error"] = float(
                                np.sqrt(((Hf - Hd) ** 2).sum() / (Hd ** 2).sum()))
                        f.reset_stats()
                        for _ in range(evals):
                            f.evaluate()
                        torch.cuda.synchronize()
                        st = f.stats()
                    row["%s_eval_ms" % eng] = st["ms_eval"]
                    row["%s_m2l_ms" % eng] = st["ms_stage"][2]
                rows.append(row)
    finally:
        if saved is None:
            os.environ.pop("CCFMM_M2L", None)
        else:
            os.environ["CCFMM_M2L"] = saved
    return rows


def fft_comparator(sizes=(16, 32, 64, 100, 128), repeats=5, nsub=2000, seed=6):
    """FFT convolution and the fast method on random-moment n^3 lattices."""
    import torch
    run, stream = _timer()
    rows = []
    for n in sizes:
        pos, mom, box = W.lattice(n, seed=810233 + 60 + seed)
        N = len(pos)
        pd = torch.from_numpy(pos).cuda()
        md = torch.from_numpy(mom).cuda()
        sub = np.random.default_rng(seed).choice(N, min(nsub, N), replace=False)
        Hd = C.direct_field(pd, md, targets=torch.from_numpy(sub).cuda(), stream=stream)
        H = torch.zeros((N, 3), dtype=torch.float64, device="cuda")
        row = {"n": n, "N": N}

        def err():
            Hs = H.cpu().numpy()[sub]
            return float(np.sqrt(((Hs - Hd) ** 2).sum() / (Hd ** 2).sum()))

        for prec in ("fp64", "mixed"):
            with C.Lattice(n, precision=prec, stream=stream) as lat:
                lat.field_energy(md, out=H)
                row["fft_%s_ms" % prec] = run(lambda: lat.field_energy(md, out=H), repeats)
                row["fft_%s_error" % prec] = err()
        for p, th in ((5, 0.71), (6, 0.5)):
            with C.FMM(pd, md, p, th, box=box, precision="mixed", stream=stream) as f:
                f.field(H)

                def step():
                    f.set_positions(pd, md)
                    f.field(H)

                row["fmm_p%d_ms" % p] = run(step, repeats)
                row["fmm_p%d_error" % p] = err()
        rows.append(row)
        print(json.dumps(row), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="fewer sizes (smoke run)")
    ap.add_argument("--part", default="all",
                    choices=["all", "scaling", "leaf_sweep", "optimal_leaf", "error_budget",
                             "truncation", "fft"])
    ap.add_argument("--out", default="experiments.json")
    args = ap.parse_args()
    t0 = time.time()
    quick = {"scaling": dict(sizes=(8, 16, 32), params=((4, 0.5),)),
             "leaf_sweep": dict(leaves=(4, 8, 16)),
             "optimal_leaf": dict(ps=(3, 5), sizes=(30, 31)),
             "error_budget": dict(n=16, es=(0.05,), ps=(3, 5)),
             "truncation": dict(n=100_000, ps=(4, 6), evals=3),
             "fft": dict(sizes=(16, 32), repeats=2)}
    parts = {"scaling": scaling, "leaf_sweep": leaf_sweep, "optimal_leaf": optimal_leaf,
             "error_budget": error_budget, "truncation": truncation, "fft": fft_comparator}
    res = {}
    for name, fn in parts.items():
        if args.part not in ("all", name):
            continue
        res[name] = fn(**quick[name]) if args.quick else fn()
        show = res[name]
        if name == "optimal_leaf":
            show = {p: {"s_o": v["s_o"], "rule": v["rule"]} for p, v in show.items()}
        elif name == "error_budget":
            show = show["fastest"]
        print(json.dumps({name: show}), flush=True)
    res["seconds"] = time.time() - t0
    json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
