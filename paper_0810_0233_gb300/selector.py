"""Parameter selector driver: sweep, training, evaluation (project addition).

The paper chooses the leaf occupancy by Eq. so and (p_m, alpha_m) by hand
from Table II / Fig. 3 (Sec. IV).  Here the FMM itself generates training
data: problem instances drawn from the lattice, ferrofluid, ring and
clustered generators are run (library kernels, FP32 mixed precision) over
(p, theta, leaf) grid cells, and each run records the time per dipole (tree +
lists + evaluation, CUDA events) and the relative RMS field error against the
FP64 GPU direct sum on a subset.  The network (library kernels) is trained on
these runs; ``fmm_select`` then picks the fastest configuration predicted to
meet a target.  This module only schedules runs and moves arrays: every
arithmetic step runs in libccfmm.

Run on a GPU:  python -m paper_0810_0233_gb300.selector --runs 20000 --eval
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import ccfmm as C
from . import workloads as W

GRID_P = (2, 3, 4, 5, 6, 7, 8)
GRID_THETA = (0.3, 0.4, 0.5, 0.6, 0.7)
GRID_LEAF = (4, 8, 16, 32, 64)
KINDS = ("uniform", "lattice", "ring", "clustered")


def instance(kind: str, n: int, seed: int):
    """A dipole set of about n points from one of the generators."""
    if kind == "uniform":
        return W.ferrofluid(n, side=n ** (1.0 / 3.0), seed=seed)
    if kind == "lattice":
        m = max(2, int(round(n ** (1.0 / 3.0))))
        pos, mom, _ = W.lattice(m, seed=seed)
        return pos, mom
    if kind == "ring":
        # three layers, inner radius a third of the outer one
        ro = math.sqrt(n / (3.0 * math.pi * (1.0 - 1.0 / 9.0)))
        return W.ring(r_out=ro, r_in=ro / 3.0, seed=seed)
    if kind == "clustered":
        return W.clustered(n, seed=seed)
    raise ValueError(kind)


class Runner:
    """Times FMM runs of one instance on the current CUDA device."""

    def __init__(self, pos, mom, n_err=512, seed=0):
        import torch
        self.torch = torch
        self.stream = torch.cuda.current_stream()
        self.n = len(pos)
        self.pos = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
        self.mom = torch.from_numpy(np.ascontiguousarray(mom)).cuda()
        self.H = torch.zeros((self.n, 3), dtype=torch.float64, device="cuda")
        self.sub = W.subset(self.n, n_err, seed)
        self.Hd = C.direct_field(self.pos, self.mom, targets=torch.from_numpy(self.sub).cuda(),
                                 stream=self.stream)
        self.feat = C.features(self.pos)

    def run(self, p, theta, leaf, repeats=1):
        torch = self.torch
        with C.FMM(self.pos, self.mom, p, theta, leaf, precision="mixed", stream=self.stream) as f:
            f.field(self.H)
            best = float("inf")
            for _ in range(repeats):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(self.stream)
                f.set_positions(self.pos, self.mom)
                f.field(self.H)
                b.record(self.stream)
                b.synchronize()
                best = min(best, a.elapsed_time(b))
        H = self.H.cpu().numpy()[self.sub]
        err = float(np.sqrt(((H - self.Hd) ** 2).sum() / (self.Hd ** 2).sum()))
        return best * 1e6 / self.n, err  # ns per dipole


def row(feat, p, theta, leaf):
    return np.concatenate([feat, [p, theta, math.log2(leaf)]]).astype(np.float32)


def sweep(n_runs=20000, per_instance=50, n_lo=2000, n_hi=2_000_000, seed=2024, log=None):
    """Run random (p, theta, leaf) cells on random instances.  Returns
    X (runs x 12), T (runs x 2) = (log10 ns per dipole, log10 error)."""
    rng = np.random.default_rng(seed)
    grid = [(p, t, l) for p in GRID_P for t in GRID_THETA for l in GRID_LEAF]
    X, T = [], []
    inst = 0
    t0 = time.time()
    while len(X) < n_runs:
        kind = KINDS[inst % len(KINDS)]
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        pos, mom = instance(kind, n, seed=int(rng.integers(1 << 30)))
        r = Runner(pos, mom, seed=inst)
        for k in rng.choice(len(grid), size=min(per_instance, len(grid)), replace=False):
            p, th, lf = grid[k]
            try:
                ns, err = r.run(p, th, lf)
            except C.CCFMMError as e:
                # a configuration the library refuses (lists beyond 32-bit
                # offsets for very small leaves and angles): no run
                if e.status != C.ERR_ARG:
                    raise
                continue
            X.append(row(r.feat, p, th, lf))
            T.append([math.log10(ns), math.log10(max(err, 1e-12))])
            if len(X) >= n_runs:
                break
        inst += 1
        if log and inst % 20 == 0:
            log("sweep: %d runs, %d instances, %.0f s" % (len(X), inst, time.time() - t0))
    return np.array(X, np.float32), np.array(T, np.float32)


def train(X, T, epochs=200, batch=256, lr=2e-3, seed=7):
    """Initialise (He, seeded) and train the network on the GPU."""
    rng = np.random.default_rng(seed)
    mlp = C.MLP()
    sizes = (12, 64, 64, 64, 2)
    theta = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        theta.append((rng.standard_normal((a, b)) * math.sqrt(2.0 / a)).ravel())
        theta.append(np.zeros(b))
    mlp.set_params(np.concatenate(theta).astype(np.float32))
    mask = np.ones_like(T)
    mlp.fit_norm(X, T, mask)
    perm = rng.permutation(len(X))
    Xs, Ts = X[perm], T[perm]
    loss = None
    for ep in range(epochs):
        loss = mlp.train(Xs, Ts, mask, batch=batch, epochs=1, lr=lr * (0.5 ** (ep / (epochs / 3))))
    return mlp, loss


TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "selector_params.npz")


def load_trained(path=TRAINED):
    """The network trained by ``main(--save)`` on the GPU (parameters and
    input/target normalisation), or None when the file is absent."""
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return C.MLP(z["params"], z["norm"])


def rule_of_thumb(target):
    """Sec. IV: Eq. so leaves; (5, 0.71) for ~1 % error, else (6, 0.48)."""
    p, th = (5, 0.71) if target >= 1e-2 else (6, 0.48)
    return p, th, C.leaf_size_rule(p)


def evaluate(mlp, pos, mom, target=1e-4, autotune_leaves=(8, 16, 26.64, 32, 48, 64)):
    """Selector pick vs the rule of thumb vs an autotuner over leaf sizes for
    the rule's (p, theta); each configuration measured (time, error)."""
    r = Runner(pos, mom, n_err=2000, seed=99)
    out = {"n": len(pos), "target": target}
    p, th, lf, fb = C.select(mlp, r.pos, target)
    ns, err = r.run(p, th, lf, repeats=3)
    out["selector"] = {"p": p, "theta": th, "leaf": lf, "fallback": fb, "ns_per_dipole": ns,
                       "error": err}
    p, th, lf = rule_of_thumb(target)
    ns, err = r.run(p, th, lf, repeats=3)
    out["rule_of_thumb"] = {"p": p, "theta": th, "leaf": lf, "ns_per_dipole": ns, "error": err}
    best = None
    for l in autotune_leaves:
        ns_l, err_l = r.run(p, th, l, repeats=3)
        if best is None or ns_l < best[1]:
            best = (l, ns_l, err_l)
    out["autotuner"] = {"p": p, "theta": th, "leaf": best[0], "ns_per_dipole": best[1],
                        "error": best[2]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--runs", type=int, default=20000)
    ap.add_argument("--per-instance", type=int, default=50)
    ap.add_argument("--n-hi", type=int, default=2_000_000, help="largest training instance")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--eval", action="store_true")
    ap.add_argument("--eval-n", type=int, default=10_000_000)
    ap.add_argument("--out", default="selector_run.json")
    ap.add_argument("--save", default="")
    args = ap.parse_args()
    log = lambda s: print(s, flush=True)
    t = time.time()
    X, T = sweep(args.runs, args.per_instance, n_hi=args.n_hi, log=log)
    log("sweep done: %d runs in %.0f s" % (len(X), time.time() - t))
    n_hold = len(X) // 10
    mlp, loss = train(X[n_hold:], T[n_hold:], epochs=args.epochs)
    Y = mlp.predict(X[:n_hold])
    res = {"runs": len(X), "train_loss": loss,
           "holdout_rmse_log10_time": float(np.sqrt(((Y[:, 0] - T[:n_hold, 0]) ** 2).mean())),
           "holdout_rmse_log10_error": float(np.sqrt(((Y[:, 1] - T[:n_hold, 1]) ** 2).mean()))}
    log(json.dumps(res))
    if args.save:
        p, q = mlp.get_params()
        np.savez(args.save, params=p, norm=q)
    if args.eval:
        res["eval"] = []
        for kind in ("uniform", "clustered"):
            pos, mom = instance(kind, args.eval_n, seed=123456)
            e = evaluate(mlp, pos, mom)
            e["kind"] = kind
            res["eval"].append(e)
            log(json.dumps(e))
    json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
