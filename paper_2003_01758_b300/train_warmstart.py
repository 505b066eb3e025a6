"""Trains the warm-start network on libpcba's own certified solutions and
writes its parameters (run on a GPU machine):

    python -m paper_2003_01758_b300.train_warmstart [--n-train 100000] [--epochs 30]

Training problems are rtd problems with obstacle counts log-uniform in
[64, 1024] and seeds warmstart.TRAIN_SEED0 + k; each is solved by libpcba in
FP32 (opt_tol 1e-3) and its certified minimiser, in normalised coordinates,
is the target.  A held-out set (seeds warmstart.EVAL_SEED0 + k) gives the
validation loss and an A/B comparison of cold and guided batch solves.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import pcba, warmstart
from . import workloads as W

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_rtd.npz")


def held_out(n, lo=64, hi=1024):
    counts = W.batch_obstacle_counts(n, warmstart.EVAL_SEED0, lo, hi)
    return [W.rtd(warmstart.EVAL_SEED0 + k, n_obstacles=int(c)) for k, c in enumerate(counts)]


def ab_compare(mlp, probs, mem_cap_total=64 << 30, repeats=3, maker=None):
    """One batch solved three ways: cold (the plain solver), learned (network
    guess + default stencil, then the refinement stencil around the seed;
    device time includes the feature kernel and the network's forward pass) and
    grid (a fixed 25 x 25 grid of candidates, then the same refinement, no
    network: what the learned arm must beat to be worth its training)."""
    maker = maker or pcba.solver_from_problem
    b = pcba.Batch([maker(p, pcba.FP32) for p in probs], mem_cap_total)
    stream = torch.cuda.Stream()
    refine = warmstart.refine_stencil()
    b.set_stream(stream.cuda_stream)
    pk = warmstart.Packed(*warmstart.host_inputs(probs))
    zero = torch.zeros((len(probs), 2), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    out = {}
    for arm in ("cold", "learned", "grid"):
        times = []
        for _ in range(repeats + 1):
            with torch.cuda.stream(stream):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if arm == "cold":
                    res = b.solve(opt_tol=1e-3)
                elif arm == "learned":
                    b.set_refine_stencil(refine)
                    b.cost_grid(warmstart.GRID, pk.glob.data_ptr(), warmstart.GLOBAL_DIM,
                                warmstart.HOST_DIM)
                    y = warmstart.predict(mlp, pk, stream=stream.cuda_stream)
                    res = b.solve_guided(y.data_ptr(), 2, warmstart.default_stencil(), opt_tol=1e-3)
                else:
                    b.set_refine_stencil(refine)
                    res = b.solve_guided(zero.data_ptr(), 2, warmstart.grid_stencil(), opt_tol=1e-3)
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = float(np.median(times[1:]))
        t = np.array([r["time_ms"] for r in res])
        cert = sum(r["status"] in (pcba.OPTIMAL, pcba.INFEASIBLE) for r in res)
        seeds = [b.warm_point(k, with_cost=True) for k in range(len(probs))] if arm != "cold" else []
        gaps = [s[1] - r["lower"] for s, r in zip(seeds, res) if s is not None]
        out[arm] = {"ms": ms, "solves_per_s": cert / (ms * 1e-3), "certified": cert,
                    "p50_ms": float(np.percentile(t, 50)), "p99_ms": float(np.percentile(t, 99)),
                    "mean_steps": float(np.mean([r["steps"] for r in res])),
                    "seeded": len(gaps),
                    "median_seed_gap": float(np.median(gaps)) if gaps else None}
    b.close()
    out["speedup_learned"] = out["cold"]["ms"] / out["learned"]["ms"]
    out["speedup_grid"] = out["cold"]["ms"] / out["grid"]["ms"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=100_000)
    ap.add_argument("--n-eval", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch-sets", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--eval-only", default=None,
                    help="skip training: load these parameters and run the comparison")
    a = ap.parse_args()
    log = lambda s: print(s, flush=True)  # noqa: E731
    if a.eval_only:
        theta, meta = warmstart.load_params(a.eval_only)
        mlp = pcba.Mlp(warmstart.POINT_DIM, warmstart.GLOBAL_DIM, meta["hidden"], pcba.Mlp.BF16)
        mlp.set_params(theta)
        log(json.dumps(ab_compare(mlp, held_out(a.n_eval))))
        return
    t0 = time.time()
    data = warmstart.make_dataset(a.n_train, chunk=2048, mem_cap_total=128 << 30, log=log)
    t_data = time.time() - t0
    mlp = pcba.Mlp(warmstart.POINT_DIM, warmstart.GLOBAL_DIM, warmstart.HIDDEN, pcba.Mlp.BF16,
                   a.seed)
    tr = warmstart.Trainer(mlp, data, a.batch_sets)
    torch.cuda.synchronize()
    t1 = time.time()
    losses = tr.train(a.epochs, lr=a.lr, seed=a.seed, log=log)
    t_train = time.time() - t1
    # validation
    probs = held_out(a.n_eval)
    cold = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32) for p in probs], 64 << 30)
    res = cold.solve(opt_tol=1e-3)
    cold.close()
    keep = [k for k, r in enumerate(res) if r["status"] == pcba.OPTIMAL]
    tgt = np.stack([warmstart.normalise(res[k]["x"], probs[k]) for k in keep]).astype(np.float32)
    kb = pcba.Batch([pcba.solver_from_problem(probs[k], pcba.FP32) for k in keep], 8 << 30)
    pk = warmstart.pack_batch([probs[k] for k in keep], kb, tgt)
    kb.close()
    _, val_loss = mlp.gradient(*pk.args(), pk.target.data_ptr())
    y = warmstart.predict(mlp, pk).cpu().numpy()
    dist = np.linalg.norm(y - tgt, axis=1)
    ab = ab_compare(mlp, probs)
    summary = {"n_train": int(len(data["target"])), "epochs": a.epochs, "lr": a.lr,
               "batch_sets": a.batch_sets, "dataset_s": t_data, "train_s": t_train,
               "train_steps": a.epochs * tr.n_batches,
               "final_train_loss": losses[-1][1], "val_loss": val_loss,
               "val_median_dist": float(np.median(dist)), "val_p90_dist": float(np.percentile(dist, 90)),
               "ab": ab}
    np.savez(a.out, theta=mlp.get_params(), hidden=warmstart.HIDDEN,
             summary=json.dumps(summary))
    log(json.dumps(summary))


if __name__ == "__main__":
    main()
