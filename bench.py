"""Benchmark: dipole fields per second of the Cartesian FMM on one GB300.

Workload (one step = the whole hot path over one input): the 10^6-dipole
ferrofluid (uniform in a 100^3 box, minimum separation 0.5, unit moments),
p = 6, theta = 0.5, leaf occupancy from Eq. so; tree, lists and D tables
rebuilt every step (fmm_set_positions), then the field evaluation
(fmm_field), FP32 bulk with FP64 derivative tensors and FP64 local
accumulation.  Inputs are resident on the device; L2 is flushed (256 MB
write) between timed steps.  Also reported: the evaluation alone (tree
reused), the end-to-end call with host buffers, the roofline of the
dominant kernel, the accuracy gate, the SM clocks during timing and the CPU
oracle on a bounded sample.

--impl reference times the CPU oracle (FP64, all host cores) on the same
workload instead.  Multi-GPU (torchrun): independent replicas, one per rank.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dipole fields/s at RMS err ≤1e-4 (FP32 vs FP64 FMM, 1 GB300); % roofline"
FP32_LANES_PER_SM, SMS = 128, 152
# dram read+write bytes per launch of the 10^6-dipole workload from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum), with the hash of the
# kernel source they were taken on; reported only while it is unchanged
NCU_TRAFFIC = {"p2p": {"bytes": 112552064, "src": "3a4619a873c7"},
               "m2l": {"bytes": 142318848, "src": "523b27571533"}}
# dense TF32 tensor peak = measured bf16 peak x nominal 1.1 / 2.25
TF32_PER_BF16 = 1.1 / 2.25


def _src_hash(names):
    """Hash of the kernel's source files (a name or a list of names)."""
    h = hashlib.sha1()
    for name in ([names] if isinstance(names, str) else names):
        with open(os.path.join(ROOT, "paper_0810_0233_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the first sample marks a running sampler; it predates the timed
            # region, so it is dropped
            t0 = time.time()
            while not self.samples and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.samples.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# (p, theta) per workload
WORKLOADS = {"ferrofluid": (6, 0.5), "ring": (6, 0.4), "ring-stated": (6, 0.4),
             "ensemble": (5, 0.5)}


def workload(name="ferrofluid", n=1_000_000):
    """Positions and moments of a single-system workload.  The ferrofluid at
    n < 10^6 keeps the density (box side scaled) and is used only for small
    profiling cases."""
    from paper_0810_0233_gb300 import workloads as W
    if name == "ring":
        return W.ring()
    if name == "ring-stated":
        return W.ring(r_out=1200.0, r_in=400.0)
    if n == 1_000_000:
        return W.ferrofluid()
    return W.ferrofluid(n, side=100.0 * (n / 1e6) ** (1.0 / 3.0))


def describe(name, n, leaf, p, theta, precision=None, step=None):
    text = {
        "ferrofluid": "ferrofluid: N=%d uniform in [0,100]^3, min separation 0.5, unit moments "
                      "uniform on the sphere (seed 810235)" % n,
        "ring": "ring: N=%d, 3 layers at spacing 1, radii 707.58/235.86 (the stated ring scaled "
                "to 2^22 points), tilted vortex moments (seed 810236)" % n,
        "ring-stated": "ring: N=%d, 3 layers at spacing 1, radii 1200/400 as stated, tilted "
                       "vortex moments (seed 810236)" % n,
    }[name]
    return {"workload": text, "N": n, "p": p, "theta": theta, "leaf_size": leaf,
            "precision": precision or "FP32 bulk; FP64 D tensors and FP64 local-expansion "
                                      "accumulation",
            "step": step or "tree + lists + D tables + field evaluation (P2M..P2P, unpermute)",
            "l2": "flushed between timed steps by a 256 MB write"}


def selector_line(C, torch, pos_d, mom_d, H_d, stream, timed, steps, warm, sub, Hd,
                  headline_s):
    """FP32 + selector on the same workload: the learned selector's pick for
    a 1e-4 target (the network trained by the library's kernels, parameters
    shipped with the package), timed like the headline step, with its error
    against the FP64 direct sum on the same 10k subset; the rule of thumb
    (Eq. so with (6, 0.48), Sec. IV) beside it."""
    from paper_0810_0233_gb300 import selector as S
    mlp = S.load_trained()
    if mlp is None:
        return {"unavailable": "no trained selector parameters in the package"}
    n = pos_d.shape[0]
    target = 1e-4

    def measure(p, th, lf):
        with C.FMM(pos_d, mom_d, p, th, lf, precision="mixed", stream=stream) as g:
            def step():
                g.set_positions(pos_d, mom_d)
                g.field(H_d)
            t = timed(step, steps, warm)
            H = H_d.cpu().numpy()
        err = float(np.sqrt(((H[sub] - Hd) ** 2).sum() / (Hd ** 2).sum()))
        return {"p": p, "theta": th, "leaf": lf, "value": n * steps / t, "unit": "fields/s",
                "ms_per_step": 1e3 * t / steps, "rms_vs_direct_10k": err}

    p, th, lf, fb = C.select(mlp, pos_d, target)
    out = dict(measure(p, th, lf), target=target, fallback=fb)
    rp, rth = (5, 0.71) if target >= 1e-2 else (6, 0.48)
    out["rule_of_thumb"] = measure(rp, rth, C.leaf_size_rule(rp))
    out["speedup_vs_rule"] = out["rule_of_thumb"]["ms_per_step"] / out["ms_per_step"]
    out["speedup_vs_headline"] = 1e3 * headline_s / out["ms_per_step"]
    out["note"] = ("selector: the library's MLP (fmm_select) on the library's features; the "
                   "headline line keeps p = 6, theta = 0.5 and Eq. so leaves")
    return out


def cpu_oracle_sample(pos, mom, p, theta, nleaves=4096, seed=11):
    """The CPU oracle on a bounded sample of the workload: tree, lists and
    upward pass over every dipole, then the downward pass and near field for
    `nleaves` random occupied leaves.  Fields/s is extrapolated to the full
    evaluation: N / (t_setup + t_sample * occupied_leaves / nleaves)."""
    import oracle as O
    t0 = time.perf_counter()
    f = O.OracleFMM(pos, mom, p, theta, 0.0)
    f.upward()
    t_setup = time.perf_counter() - t0
    leaf_of = f.leaf_of()
    occ = np.unique(leaf_of)
    rng = np.random.default_rng(seed)
    pick = rng.choice(occ, size=min(nleaves, len(occ)), replace=False)
    mask = np.zeros(1 << f.depth, np.uint8)
    mask[pick] = 1
    t1 = time.perf_counter()
    f.downward(mask)
    t_sample = time.perf_counter() - t1
    t_full = t_setup + t_sample * len(occ) / len(pick)
    value = len(pos) / t_full
    return {"value": value, "unit": "fields/s", "cores": O.threads(), "kind": "oracle",
            "sample": "FP64 CPU oracle: tree, lists and upward pass over all %d dipoles (%.1f s), "
                      "downward pass + near field for %d random occupied leaves of %d (%.1f s, "
                      "%d fields); fields/s extrapolated to all leaves"
                      % (len(pos), t_setup, len(pick), len(occ), t_sample,
                         int(np.isin(leaf_of, pick).sum())),
            "seconds": t_setup + t_sample}


def oracle_ensemble_sample(pos, mom, off, p, theta, budget_s=15.0, seed=12, tree="adaptive"):
    """The CPU oracle over whole samples of the ensemble, drawn at random
    until about budget_s seconds of work; fields/s over those samples.  With
    the adaptive tree the oracle's adaptive mode runs at s = 2 x Eq. so (the
    middle of the autotuner's candidates)."""
    import oracle as O
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(off) - 1)
    t0 = time.perf_counter()
    done = fields = 0
    for i in order:
        sl = slice(int(off[i]), int(off[i + 1]))
        if tree == "adaptive":
            O.afmm_field(pos[sl], mom[sl], p, theta, 2.0 * O.leaf_size_rule(p))
        else:
            O.fmm_field(pos[sl], mom[sl], p, theta)
        done += 1
        fields += sl.stop - sl.start
        if time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return {"value": fields / t, "unit": "fields/s", "cores": O.threads(), "kind": "oracle",
            "sample": "FP64 CPU oracle (%s tree), full FMM (tree, lists, all passes) of %d "
                      "random samples of the ensemble, %d fields in %.1f s"
                      % (tree, done, fields, t),
            "seconds": t}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, theta = WORKLOADS[args.workload]
    times = []
    res = None
    if args.workload == "ensemble":
        from paper_0810_0233_gb300 import workloads as W
        pos, mom, off = W.ensemble()
        for it in range(args.warmup + args.steps):
            res = oracle_ensemble_sample(pos, mom, off, p, theta, budget_s=5.0, seed=100 + it,
                                         tree=args.tree)
            if it >= args.warmup:
                times.append(len(pos) / res["value"])
        config = describe_ensemble(len(off) - 1, len(pos), p, theta, args.tree)
        config["precision"] = "FP64 throughout (the CPU oracle)"
        config["step"] = ("FP64 CPU oracle: whole FMM of random samples for about 5 s per step, "
                          "fields/s over those samples (no rotation)")
        config["l2"] = "not applicable (CPU)"
    else:
        pos, mom = workload(args.workload, args.n)
        for it in range(args.warmup + args.steps):
            res = cpu_oracle_sample(pos, mom, p, theta, nleaves=256, seed=100 + it)
            if it >= args.warmup:
                times.append(len(pos) / res["value"])
        config = describe(args.workload, len(pos), 0.74 * p * p, p, theta,
                          precision="FP64 throughout (the CPU oracle)",
                          step="FP64 CPU oracle: tree, lists and upward pass over all dipoles, "
                               "then the downward pass and near field of 256 random occupied "
                               "leaves; the step time is extrapolated from those leaves to all "
                               "occupied leaves (not a measured full evaluation)")
        config["l2"] = "not applicable (CPU)"
    t = float(np.mean(times))
    value = len(pos) / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "fields/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "extrapolated": args.workload != "ensemble",
            "cpu_baseline": {"value": value, "unit": "fields/s", "cores": res["cores"],
                             "kind": "oracle", "sample": res["sample"]},
            "e2e": {"value": value, "unit": "fields/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def describe_ensemble(ns, total, p, theta, tree="adaptive", astep="graph"):
    if tree == "adaptive" and astep == "persistent":
        how = ("adaptive-depth trees (a cell splits while it holds more than s dipoles, s per "
               "size class by the library's autotuner); one CUDA graph launch holding one "
               "persistent kernel whose blocks take every stage's tiles of all samples from "
               "one task queue (bounded waits between the stages)")
        prec = ("FP32 bulk, M2L on 3xTF32 warp-level MMA; FP64 D tensors; per-cell M2L sums "
                "in FP32, L2L in FP64")
    elif tree == "adaptive":
        how = ("adaptive-depth trees (a cell splits while it holds more than s dipoles, s per "
               "size class by the library's autotuner); one CUDA graph launch, one kernel per "
               "stage over all samples (per level for M2M and L2L)")
        prec = ("FP32 bulk, M2L on 3xTF32 warp-level MMA; FP64 D tensors; per-cell M2L sums "
                "in FP32, L2L in FP64")
    else:
        how = ("complete trees at the Eq. so depth; one CUDA graph launch of batched stages "
               "(one kernel per stage over all samples)")
        prec = "FP32 bulk; FP64 D tensors and FP64 local-expansion accumulation"
    return {"workload": "ensemble: %d clustered samples (80%% Gaussian blobs sigma 3 of 500, 20%% "
                        "chains of 20), N log-uniform in [1e3, 2e5], sum N = %d (seed 810237)"
                        % (ns, total),
            "N": total, "samples": ns, "p": p, "theta": theta, "tree": tree,
            "precision": prec,
            "step": "rotate every moment (Philox4x64-10, angle U[0, 0.05]) + field and energy "
                    "of every sample; trees fixed; " + how,
            "l2": "inputs (%.0f MB of moments) larger than L2" % (total * 24 / 1e6)}


def run_ensemble(args, torch, dist, C, world, rank, dev, stream):
    """The ensemble step: every rank steps all samples of its share
    (samples dealt round-robin over ranks, no collective in the step)."""
    from paper_0810_0233_gb300 import ranks as R
    from paper_0810_0233_gb300 import workloads as W
    p, theta = WORKLOADS["ensemble"]
    pos, mom, off = W.ensemble()
    ns = len(off) - 1
    mine, o, rows = R.shard(off, rank, world)
    P_, M_ = R.gather_rows(pos, rows), R.gather_rows(mom, rows)
    total = int(o[-1])
    t0 = time.perf_counter()
    adaptive = args.tree == "adaptive"
    if adaptive:
        b = C.Adaptive(torch.from_numpy(P_).to(dev), torch.from_numpy(M_).to(dev), p, theta,
                       offsets=o, precision=args.precision, stream=stream,
                       autotune=not args.no_autotune, persistent=args.astep == "persistent")
    else:
        b = C.Batch(torch.from_numpy(P_).to(dev), torch.from_numpy(M_).to(dev), o, p, theta,
                    precision=args.precision, stream=stream, autotune=not args.no_autotune)
    t_create = time.perf_counter() - t0
    E_d = torch.zeros(len(mine), dtype=torch.float64, device=dev)
    counter = [0]

    def step():
        b.step(seed=810237, step=counter[0], max_angle=0.05, E_out=E_d)
        counter[0] += 1

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        z.record(stream)
        z.synchronize()
        total_t = a.elapsed_time(z) / 1e3
        barrier()
        return R.max_over_ranks(total_t, dist if world > 1 else None, dev)

    launches0 = C.kernel_launches()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t_step = timed(step, args.steps, args.warmup)
    launches = (C.kernel_launches() - launches0) // (args.steps + args.warmup)
    H_h = torch.zeros((total, 3), dtype=torch.float64).pin_memory()
    E_h = torch.zeros(len(mine), dtype=torch.float64).pin_memory()

    def step_e2e():
        b.step(seed=810237, step=counter[0], max_angle=0.05, H_out=H_h, E_out=E_h)
        counter[0] += 1

    t_e2e = timed(step_e2e, args.steps, 1)
    all_total = int(R.sum_over_ranks(total, dist if world > 1 else None, dev))
    # algorithmic work of one step, summed over this rank's samples
    K = (p + 1) * (p + 2) * (p + 3) // 6 - 1
    pairs = far = 0
    if adaptive:
        ast = b.stats()
        pairs, far = ast["near_pairs"], ast["far_pairs"]
    else:
        for i in range(len(mine)):
            st = b.sample(i).stats()
            pairs += st["p2p_pairs"]
            far += st["far_pairs"]
    peaks = _peaks()
    clock = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * clock * 1e6 / 1e12
    # the FP32 M2L engines (tensor cores) contract the harmonic reduction
    KM = (p + 1) * (p + 1) - 1 if args.precision == "mixed" else K
    flops = 30.0 * pairs + 2.0 * KM * KM * far
    ach = flops / (t_step / args.steps) / 1e12
    line = {"metric": METRIC, "value": all_total * args.steps / t_step, "unit": "fields/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": describe_ensemble(ns, len(pos), p, theta, args.tree, args.astep),
            "e2e": {"value": all_total * args.steps / t_e2e, "unit": "fields/s",
                    "ms_per_step": 1e3 * t_e2e / args.steps, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(total * 24 + len(mine) * 8),
                    "note": "the step's fields and energies read back to pinned host memory"},
            "gpu_launches": int(launches) * args.steps,
            "gpu_launches_per_step": int(launches),
            "roofline": {"kernel": "whole step (graph)", "bound": "alu", "achieved": ach,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                         "traffic": None,
                         "algorithmic": {"p2p_pairs": pairs, "far_pairs": far,
                                         "flop": flops},
                         "note": "all near-pair and M2L flops of the step over the step time; "
                                 "M2L on the tensor cores"},
            "clocks": clk.summary(),
            "samples_per_rank": len(mine)}
    if adaptive:
        ast = b.stats()
        line["kernels_per_step"] = int(ast["kernels_per_eval"]) + 1
        line["adaptive_tree"] = {k: ast[k] for k in ("ncells", "nleaves", "max_level",
                                                     "far_pairs", "near_pairs", "d_rows",
                                                     "m2l_items", "ms_build")}
        line["autotune"] = {"classes": [{"n_min": c[0], "split": c[1]} for c in b.tuning()],
                            "create_s": t_create,
                            "note": "per size class (octave of N) the split threshold of the "
                                    "fastest timed trial evaluation (library autotuner, at "
                                    "creation, outside the timed steps)"}
    else:
        line["kernels_per_step"] = b.kernels_per_step()
        line["autotune"] = {"classes": [{"n_min": c[0], "leaf": c[1], "m2l_item_len": c[2]}
                                        for c in b.tuning()],
                            "create_s": t_create,
                            "note": "per size class (octave of N) the leaf occupancy and M2L "
                                    "item length of the fastest timed trial evaluation (library "
                                    "autotuner, at creation, outside the timed steps)"}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = oracle_ensemble_sample(pos, mom, off, p, theta, tree=args.tree)
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="ensemble: Eq. so leaves (splits) for every sample instead of the "
                         "autotuner")
    ap.add_argument("--tree", default="adaptive", choices=["adaptive", "uniform"],
                    help="ensemble: adaptive-depth trees (default) or complete trees")
    ap.add_argument("--astep", default="graph", choices=["graph", "persistent"],
                    help="ensemble on adaptive trees: the stages as kernels of one graph "
                         "(default) or one persistent kernel over a task queue")
    ap.add_argument("--no-selector", action="store_true",
                    help="skip the selector object (learned (p, theta, leaf) at 1e-4)")
    ap.add_argument("--profile", action="store_true",
                    help="one warm-up and two steps only (for ncu launch lists and captures)")
    ap.add_argument("--n", type=int, default=1_000_000,
                    help="ferrofluid dipoles; below 10^6 only for small profiling cases")
    ap.add_argument("--workload", default="ferrofluid", choices=sorted(WORKLOADS),
                    help="ferrofluid (the default line), ring (4.19e6), ring-stated (1.2e7), "
                         "ensemble (512 samples)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_0810_0233_gb300 import ccfmm as C
    from paper_0810_0233_gb300 import ranks as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    if args.workload == "ensemble":
        return run_ensemble(args, torch, dist, C, world, rank, dev, stream)

    P, THETA = WORKLOADS[args.workload]
    pos, mom = workload(args.workload, args.n)
    n = len(pos)
    pos_d = torch.from_numpy(pos).to(dev)
    mom_d = torch.from_numpy(mom).to(dev)
    H_d = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    f = C.FMM(pos_d, mom_d, P, THETA, 0.0, precision=args.precision, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(step, k, w):
        for _ in range(w):
            step()
        barrier()
        total = 0.0
        for _ in range(k):
            flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b) / 1e3
        barrier()
        return R.max_over_ranks(total, dist if world > 1 else None, dev)

    def step_full():
        f.set_positions(pos_d, mom_d)
        f.field(H_d)

    def step_eval():
        f.field(H_d)

    steps = 2 if args.profile else args.steps
    warm = 1 if args.profile else args.warmup
    if args.profile:
        t_full = timed(step_full, steps, warm)
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": 1e3 * t_full / steps}))
        return
    # end to end through the C-ABI with host buffers: H2D of positions and
    # moments and D2H of the field inside every step
    pos_h = torch.from_numpy(pos).pin_memory()
    mom_h = torch.from_numpy(mom).pin_memory()
    H_h = torch.zeros((n, 3), dtype=torch.float64).pin_memory()

    def step_e2e():
        f.set_positions(pos_h, mom_h)
        f.field(H_h)

    # clocks are sampled over the three timed regions
    with ClockSampler(local) as clk:
        launches0 = C.kernel_launches()
        t_full = timed(step_full, steps, warm)
        launches = (C.kernel_launches() - launches0) // (steps + warm)
        f.reset_stats()
        t_eval = timed(step_eval, steps, 0)
        st = f.stats()
        t_e2e = timed(step_e2e, steps, 1)

    value = world * n * steps / t_full
    line = {"metric": METRIC, "value": value, "unit": "fields/s", "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * t_full / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": describe(args.workload, n, st["leaf_target"], P, THETA),
            "eval": {"value": world * n * steps / t_eval, "unit": "fields/s",
                     "ms_per_step": 1e3 * t_eval / steps, "note": "tree and lists reused"},
            "e2e": {"value": world * n * steps / t_e2e, "unit": "fields/s",
                    "ms_per_step": 1e3 * t_e2e / steps,
                    "h2d_bytes_per_step": int(pos.nbytes + mom.nbytes),
                    "d2h_bytes_per_step": int(n * 3 * 8)},
            "gpu_launches": int(launches) * steps,
            "gpu_launches_per_step": int(launches)}

    # roofline of the dominant kernel, from the library's stage events of the
    # timed evaluations (same stream)
    K = (P + 1) * (P + 2) * (P + 3) // 6 - 1
    ms = st["ms_stage"]
    stages = {"p2p": ms[5], "m2l": ms[2], "p2m": ms[0], "m2m": ms[1], "l2l": ms[3], "l2p": ms[4],
              "finish": ms[6]}
    peaks = _peaks()
    clock = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES_PER_SM * 2 * clock * 1e6 / 1e12  # TFLOP/s
    tc = args.precision == "mixed" and os.environ.get("CCFMM_M2L", "tc") != "fma"
    # the tensor-core path contracts the harmonic reduction: (p+1)^2 - 1
    # coefficients on either side (the Laplace identity of the D tensors)
    KM = (P + 1) * (P + 1) - 1 if tc else K
    flops = {"p2p": 30.0 * st["p2p_pairs"], "m2l": 2.0 * KM * KM * st["far_pairs"]}
    tf32_peak = peaks.get("bf16_tflops", 1900.0) * TF32_PER_BF16
    src = {"p2p": ["p2p.cu", "stages.cuh"], "m2l": "m2l_tc.cu" if tc else "m2l.cu"}

    def traffic(k):
        # the capture is of the 10^6-dipole ferrofluid: other workloads have none
        if getattr(args, "workload", "ferrofluid") != "ferrofluid" or args.n != 1_000_000:
            return None
        tr = NCU_TRAFFIC.get(k)
        return tr["bytes"] if tr and tr.get("src") == _src_hash(src[k]) else None

    def roof(k):
        ach = flops[k] / (stages[k] * 1e-3) / 1e12
        if k == "m2l" and tc:
            return {"kernel": "m2l", "bound": "tensor", "achieved": ach, "peak": tf32_peak,
                    "unit": "TFLOP/s", "frac": ach / tf32_peak, "traffic": traffic(k),
                    "peak_note": "dense TF32 tensor peak = measured bf16 %.0f TFLOP/s x 1.1/2.25; "
                                 "3xTF32 issues 3 MMAs per product, so 1/3 of it is the ceiling for "
                                 "FP32-accurate results" % peaks.get("bf16_tflops", 1900.0),
                    "frac_of_3xtf32": 3 * ach / tf32_peak,
                    "full_tensor_equivalent_tflops": ach * (K * K) / (KM * KM),
                    "stage": "moment fold and split + tcgen05 contraction over the harmonic "
                             "reduction ((p+1)^2 - 1 = %d coefficients) + FP64 reduce and "
                             "completion of V" % KM}
        return {"kernel": k, "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": traffic(k),
                "peak_note": "FP32 FMA peak 152 SMs x 128 lanes x 2 flop x %.0f MHz" % clock}

    dom = max(("p2p", "m2l"), key=lambda k: stages[k])
    line["roofline"] = dict(roof(dom), **{
        "algorithmic": {"p2p_flop_per_pair": 30, "p2p_pairs": st["p2p_pairs"],
                        "m2l_flop_per_far_pair": 2 * KM * KM, "far_pairs": st["far_pairs"]},
        "stage_ms": stages,
        "other": {k: roof(k) for k in flops if k != dom}})
    # the same kernels timed alone (near/far overlap off, a few untimed-step
    # evaluations outside the timed regions)
    prev = os.environ.get("CCFMM_OVERLAP")
    os.environ["CCFMM_OVERLAP"] = "0"
    f.reset_stats()
    timed(step_eval, min(steps, 10), 1)
    st_iso = f.stats()
    if prev is None:
        del os.environ["CCFMM_OVERLAP"]
    else:
        os.environ["CCFMM_OVERLAP"] = prev
    ms_iso = st_iso["ms_stage"]
    iso = {"p2p": ms_iso[5], "m2l": ms_iso[2]}
    line["roofline"]["isolated"] = {
        k: {"ms": iso[k], "achieved": flops[k] / (iso[k] * 1e-3) / 1e12,
            "frac": flops[k] / (iso[k] * 1e-3) / 1e12 /
            (tf32_peak if (k == "m2l" and tc) else fp32_peak)}
        for k in iso}
    line["roofline"]["note"] = ("stage times of the timed evaluations, where P2P runs concurrently "
                                "with P2M..L2L on a second stream; 'isolated': the same kernels "
                                "timed with the overlap off")
    line["clocks"] = clk.summary()
    line["build_ms"] = st["ms_build"]
    line["build_stages_ms"] = dict(zip(
        ("upload_box_keys_sort", "depth_leaves_points_counts", "lists_tiles",
         "items_upload", "tile_fill_dtables", "plan_host"), st["ms_build_stage"]))

    if not args.no_accuracy:
        from paper_0810_0233_gb300 import workloads as W
        sub = W.subset(n, 10000, 77)
        sub_d = torch.from_numpy(sub).to(dev)
        t0 = time.perf_counter()
        Hd = C.direct_field(pos_d, mom_d, targets=sub_d, stream=stream)
        t_direct = time.perf_counter() - t0
        H = H_d.cpu().numpy()
        err_direct = float(np.sqrt(((H[sub] - Hd) ** 2).sum() / (Hd ** 2).sum()))
        acc = {"rms_vs_direct_10k": err_direct,
               "direct_sum_10k_ms": 1e3 * t_direct,
               "direct_sum_note": "FP64 GPU direct sum at the 10k subset over all N sources "
                                  "(wall time of the call)"}
        if args.precision == "mixed":
            with C.FMM(pos_d, mom_d, P, THETA, 0.0, precision="fp64", stream=stream) as g:
                H64 = torch.zeros_like(H_d)
                g.field(H64)
                torch.cuda.synchronize()
                acc["rms_vs_fp64_fmm"] = float(torch.sqrt(((H_d - H64) ** 2).sum() /
                                                          (H64 ** 2).sum()).item())
        line["accuracy"] = acc
        if (args.workload == "ferrofluid" and args.precision == "mixed" and n == 1_000_000
                and not args.no_selector):
            line["selector"] = selector_line(C, torch, pos_d, mom_d, H_d, stream, timed,
                                             min(steps, 20), warm, sub, Hd, t_full / steps)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample(pos, mom, P, THETA)
        # the same oracle on one host thread, on a smaller sample
        import oracle as O
        nthr = O.threads()
        O.set_threads(1)
        try:
            one = cpu_oracle_sample(pos, mom, P, THETA, nleaves=128, seed=12)
        finally:
            O.set_threads(nthr)
        line["cpu_baseline"]["single_thread"] = {k: one[k] for k in ("value", "cores", "sample")}
    f.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
