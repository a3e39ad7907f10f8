"""Autotuner: the fastest treecode parameters that meet an error budget.

For each (MAC mode, degree n, leaf size N0) it walks theta downward from the
largest candidate and keeps the first theta whose relative L2 error against the
FP64 direct sum (on sampled targets, computed on the GPU) is within the budget;
since the error grows with theta and the work falls with it, that theta is the
fastest feasible one for that (mode, n, N0).  The step time (tree, modified
weights, lists, evaluation) is measured with CUDA events after a warm-up run.

    python -m paper_1902_02250_gb300.tune [--n 1000000] [--budget 8e-7]
"""
import argparse
import itertools
import json
import math

import numpy as np

from . import kitc as K
from . import workloads as wl

THETAS = (0.8, 0.75, 0.7, 0.65, 0.6, 0.55, 0.5)
DEGREES = (6, 7, 8, 9, 10)
LEAVES = (1000, 2000, 4000)
MACS = (K.MAC_PARTICLE, K.MAC_BATCH, K.MAC_ALL)


def _rel(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((a ** 2).sum()))


def time_step(xd, fd, p, out, reps=2):
    """Milliseconds of one build + weights + evaluate (best of reps after a warm-up)."""
    import torch
    stream = torch.cuda.current_stream()
    best = float("inf")
    st = None
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = K.kitc_build_tree(xd, p)
        try:
            K.kitc_modified_weights(t, fd)
            K.kitc_evaluate(t, xd, out)
            st = t.stats()
        finally:
            t.free()
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            best = min(best, e0.elapsed_time(e1))
    return best, st


def tune(xd, fd, base, budget, idx, ref, thetas=THETAS, degrees=DEGREES, leaves=LEAVES, macs=MACS,
         log=None):
    """Returns (best Params, best record, all records)."""
    import torch
    out = torch.empty((xd.shape[0], K.kernel_wout(base.kernel)), dtype=torch.float64, device=xd.device)
    records = []
    best = None
    for mac, n, leaf in itertools.product(macs, degrees, leaves):
        for th in thetas:
            p = K.Params(theta=th, degree=n, leaf_size=leaf, eps=base.eps, kernel=base.kernel,
                         precision=base.precision, mac=mac, target_batch=base.target_batch,
                         weights=base.weights)
            ms, st = time_step(xd, fd, p, out)
            E = _rel(ref, out.cpu().numpy()[idx])
            rec = dict(mac=mac, degree=n, leaf_size=leaf, theta=th, ms=ms, E=E,
                       near=st["near_pairs"], far=st["far_points"])
            records.append(rec)
            if log:
                log(rec)
            if E <= budget:
                if best is None or ms < best[1]["ms"]:
                    best = (p, rec)
                break
    return best, records


def time_forest(xd, fd, counts, p, out, reps=2):
    """Milliseconds of one forest build + weights + evaluate (best of reps after a warm-up)."""
    import torch
    stream = torch.cuda.current_stream()
    best = float("inf")
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = K.kitc_build_forest(xd, counts, p)
        try:
            K.kitc_modified_weights(t, fd)
            K.kitc_evaluate_forest(t, xd, counts, out)
        finally:
            t.free()
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            best = min(best, e0.elapsed_time(e1))
    return best


def tune_forest(xd, fd, counts, base, leaves=(250, 500, 1000, 2000), batches=(32, 64), macs=None,
                log=None):
    """Fastest leaf size N0, target-batch size and MAC mode (of macs, default
    base's) for a forest at fixed theta, n."""
    import torch
    out = torch.empty((xd.shape[0], K.kernel_wout(base.kernel)), dtype=torch.float64, device=xd.device)
    best = None
    for leaf, b, mac in itertools.product(leaves, batches, macs or (base.mac,)):
        p = K.Params(theta=base.theta, degree=base.degree, leaf_size=leaf, eps=base.eps,
                     kernel=base.kernel, precision=base.precision, mac=mac, target_batch=b,
                     weights=base.weights)
        ms = time_forest(xd, fd, counts, p, out)
        if log:
            log(dict(leaf_size=leaf, target_batch=b, mac=mac, ms=ms))
        if best is None or ms < best[1]:
            best = (p, ms)
    return best


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--budget", type=float, default=8e-7)
    ap.add_argument("--samples", type=int, default=4000)
    ap.add_argument("--out", default=None)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_leaf", "fp64"],
                    help="mixed_leaf: near-field differences from leaf offsets")
    args = ap.parse_args()
    x, f = wl.uniform_cube(args.n, args.seed)
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(f).cuda()
    idx = wl.sample_indices(args.n, args.samples, 101)
    base = K.Params(eps=args.eps, precision={"mixed": K.MIXED, "mixed_leaf": K.MIXED_LEAF,
                                             "fp64": K.FP64}[args.precision])
    ref = K.kitc_direct(xd[torch.from_numpy(idx).cuda()].contiguous(), xd, fd,
                        K.Params(eps=args.eps, precision=K.FP64)).cpu().numpy()
    best, recs = tune(xd, fd, base, args.budget, idx, ref, log=lambda r: print(json.dumps(r), flush=True))
    res = {"budget": args.budget, "best": best[1] if best else None, "records": recs}
    print(json.dumps({"best": res["best"]}))
    if args.out:
        json.dump(res, open(args.out, "w"), indent=1)


if __name__ == "__main__":
    main()
