"""Learned warm start for rtd problems (not part of the paper).

A set-encoder network (libpcba's ``pcba_mlp_*`` kernels: BF16 tensor-core
GEMMs with FP32 accumulation, Adam on FP32 master weights) maps one planning
problem - its obstacle points and a global vector holding the goal, the
coefficients of the map F and the cost on a coarse grid of the box (computed
by the library on the device) - to a guess of the minimiser in the box's
normalised coordinates.  ``pcba_batch_solve_guided`` then evaluates a stencil
of candidate points around every guess in FP64 with rounding-error bounds and
seeds p_up (Def. 4) with the best certified-feasible one.  The guess affects
only how early suboptimal boxes are cut off (Alg. 4); every certified bound
holds whatever the network predicts.

This module marshals arrays and device pointers (torch supplies the device
memory); every forward, backward, optimiser and candidate-evaluation step runs
in libpcba's kernels.
"""
from __future__ import annotations

import math
import os
import time

import numpy as np
import torch

from . import pcba
from . import workloads as W

POINT_DIM = 2
HOST_DIM = 34             # goal (2) + F_1, F_2 coefficients (2 x 16) of rtd(f_degree=3)
GRID = 9                  # cost landscape on a GRID x GRID grid (pcba_batch_cost_grid)
GLOBAL_DIM = HOST_DIM + GRID * GRID
HIDDEN = 128
TRAIN_SEED0 = 5_000_000   # training problems use seeds TRAIN_SEED0 + k
EVAL_SEED0 = 6000         # held-out problems use seeds EVAL_SEED0 + k


def features(prob):
    """(points [n][2], host part of glob [34]) float32 of one rtd problem:
    obstacles / 2, goal / 2 and the coefficients of F divided by their
    standard deviation 0.5.  The rest of glob is the cost landscape that
    ``pack_batch`` has the library compute on the device."""
    m = prob.meta
    pts = (np.asarray(m["obstacles"], dtype=np.float64) / 2.0).astype(np.float32)
    glob = np.concatenate([np.asarray(m["goal"]) / 2.0, np.ravel(m["F"][0]) / 0.5,
                           np.ravel(m["F"][1]) / 0.5]).astype(np.float32)
    assert glob.size == HOST_DIM, "features expect rtd problems with f_degree=3"
    return pts, glob


def normalise(x, prob):
    """Point of the box -> normalised coordinates in [-1, 1]^l."""
    return 2.0 * (np.asarray(x)[:prob.l] - prob.lo) / (prob.hi - prob.lo) - 1.0


def default_stencil(half=8, step=0.02, radii=(0.25, 0.35, 0.5, 0.7), n_dir=16):
    """Stencil rows (normalised offsets): a (2 half + 1)^2 square of spacing
    step centred on the guess (the guess itself included), then n_dir points
    on each circle of the given radii."""
    k = np.arange(-half, half + 1) * step
    a, b = np.meshgrid(k, k, indexing="ij")
    rows = [np.stack([a.ravel(), b.ravel()], axis=1)]
    for r in radii:
        t = 2.0 * math.pi * np.arange(n_dir) / n_dir
        rows.append(np.stack([r * np.cos(t), r * np.sin(t)], axis=1))
    return np.concatenate(rows).astype(np.float64)


def refine_stencil(half=8, step=0.005):
    """Second-round stencil (pcba_batch_set_refine_stencil): a (2 half + 1)^2
    square of spacing step around the first seed, the seed itself included."""
    k = np.arange(-half, half + 1) * step
    a, b = np.meshgrid(k, k, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


def grid_stencil(n=25):
    """Guess-free candidates: an n x n grid over the whole normalised box
    (used with a zero guess; the non-learned arm of the comparison)."""
    k = np.linspace(-1.0, 1.0, n)
    a, b = np.meshgrid(k, k, indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1)


class Packed:
    """Device copies of a batch of sets: points [P][2], offsets [B+1] int32,
    glob [B][dg] and optionally targets [B][2], all float32 except offsets."""

    def __init__(self, points, offsets, glob, target=None, device="cuda"):
        self.points = torch.as_tensor(np.ascontiguousarray(points, np.float32), device=device)
        self.offsets = torch.as_tensor(np.ascontiguousarray(offsets, np.int32), device=device)
        self.glob = torch.as_tensor(np.ascontiguousarray(glob, np.float32), device=device)
        self.target = None if target is None else torch.as_tensor(
            np.ascontiguousarray(target, np.float32), device=device)
        self.n_sets = int(self.glob.shape[0])
        self.n_points = int(self.points.shape[0])

    def args(self):
        return (self.points.data_ptr(), self.offsets.data_ptr(), self.n_sets, self.n_points,
                self.glob.data_ptr())


def pack_batch(problems, batch, targets=None, device="cuda"):
    """Packed network inputs of the problems of a pcba.Batch (same order): the
    host features plus the cost landscape, computed by the library on the
    device into the last GRID^2 columns of glob."""
    points, offsets, glob = host_inputs(problems)
    pk = Packed(points, offsets, glob, targets, device)
    torch.cuda.synchronize()
    batch.cost_grid(GRID, pk.glob.data_ptr(), GLOBAL_DIM, HOST_DIM)
    torch.cuda.synchronize()
    return pk


def make_dataset(n, seed0=TRAIN_SEED0, lo=64, hi=1024, chunk=512, mem_cap_total=64 << 30,
                 opt_tol=1e-3, log=None):
    """Solves n rtd problems (obstacle counts log-uniform in [lo, hi], seeds
    seed0 + k) with libpcba in FP32 and returns the certified ones as host
    arrays: points, offsets (int64), glob, target (normalised minimisers)."""
    counts = W.batch_obstacle_counts(n, seed0, lo, hi)
    pts, gl, tg, sizes = [], [], [], []
    t0 = time.time()
    for c0 in range(0, n, chunk):
        probs = [W.rtd(seed0 + k, n_obstacles=int(counts[k])) for k in range(c0, min(n, c0 + chunk))]
        b = pcba.Batch([pcba.solver_from_problem(p, pcba.FP32) for p in probs], mem_cap_total)
        res = b.solve(opt_tol=opt_tol)
        glob = pack_batch(probs, b).glob.cpu().numpy()
        b.close()
        for k, (p, r) in enumerate(zip(probs, res)):
            if r["status"] != pcba.OPTIMAL or not np.all(np.isfinite(r["x"])):
                continue
            f = features(p)
            pts.append(f[0])
            gl.append(glob[k])
            tg.append(normalise(r["x"], p).astype(np.float32))
            sizes.append(f[0].shape[0])
        if log:
            log("dataset %d/%d problems, %d kept, %.1f s" % (min(n, c0 + chunk), n, len(tg),
                                                           time.time() - t0))
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return {"points": np.concatenate(pts), "offsets": offsets, "glob": np.stack(gl),
            "target": np.stack(tg)}


class Trainer:
    """Mini-batch training of a ``pcba.Mlp`` on a device-resident dataset.

    The dataset's sets are cut once into consecutive mini-batches of
    ``batch_sets`` sets (the sets are in random order already); every epoch
    visits the mini-batches in a new random order."""

    def __init__(self, mlp, data, batch_sets=256, device="cuda"):
        self.mlp = mlp
        off = np.asarray(data["offsets"], dtype=np.int64)
        n = len(off) - 1
        self.n_batches = n // batch_sets
        self.B = batch_sets
        self.points = torch.as_tensor(np.ascontiguousarray(data["points"], np.float32),
                                      device=device)
        self.glob = torch.as_tensor(np.ascontiguousarray(data["glob"], np.float32), device=device)
        self.target = torch.as_tensor(np.ascontiguousarray(data["target"], np.float32),
                                      device=device)
        rel = np.empty((self.n_batches, batch_sets + 1), dtype=np.int32)
        self.first_point = np.empty(self.n_batches, dtype=np.int64)
        self.n_points = np.empty(self.n_batches, dtype=np.int64)
        for b in range(self.n_batches):
            o = off[b * batch_sets:(b + 1) * batch_sets + 1]
            rel[b] = (o - o[0]).astype(np.int32)
            self.first_point[b] = o[0]
            self.n_points[b] = o[-1] - o[0]
        self.rel = torch.as_tensor(rel, device=device)

    def batch_args(self, b):
        s0 = b * self.B
        return (self.points.data_ptr() + 4 * POINT_DIM * int(self.first_point[b]),
                self.rel.data_ptr() + 4 * (self.B + 1) * b, self.B, int(self.n_points[b]),
                self.glob.data_ptr() + 4 * GLOBAL_DIM * s0,
                self.target.data_ptr() + 4 * 2 * s0)

    def train(self, epochs, lr=1e-3, seed=0, log=None, loss_every=50):
        rng = np.random.default_rng(seed)
        total = epochs * self.n_batches
        step = 0
        losses = []
        for ep in range(epochs):
            for b in rng.permutation(self.n_batches):
                lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
                want = (step % loss_every) == 0
                loss = self.mlp.train_step(*self.batch_args(int(b)), lr_t, want_loss=want)
                if want:
                    losses.append((step, loss))
                step += 1
            if log:
                log("epoch %d: last sampled loss %.5f" % (ep, losses[-1][1]))
        torch.cuda.synchronize()
        return losses


def predict(mlp, packed, stream=0):
    """Network outputs [B][2] (a float32 CUDA tensor) for a Packed batch."""
    y = torch.empty((packed.n_sets, 2), dtype=torch.float32, device=packed.glob.device)
    mlp.forward(*packed.args(), y.data_ptr(), stream=stream)
    return y


def load_params(path):
    z = np.load(path)
    return z["theta"].astype(np.float32), dict(hidden=int(z["hidden"]))


DEFAULT_PARAMS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warmstart_rtd.npz")


def load_model(path=DEFAULT_PARAMS):
    """The trained network (BF16) with the parameters stored at path."""
    theta, meta = load_params(path)
    m = pcba.Mlp(POINT_DIM, GLOBAL_DIM, meta["hidden"], pcba.Mlp.BF16)
    m.set_params(theta)
    return m


def host_inputs(problems):
    """Host arrays of the network inputs of a batch: points [P][2], offsets
    [B+1] int32 and glob [B][GLOBAL_DIM] whose cost-landscape columns are zero
    (pcba_batch_cost_grid fills them on the device)."""
    feats = [features(p) for p in problems]
    sizes = [f[0].shape[0] for f in feats]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    glob = np.zeros((len(problems), GLOBAL_DIM), dtype=np.float32)
    glob[:, :HOST_DIM] = np.stack([f[1] for f in feats])
    return np.concatenate([f[0] for f in feats]), offsets, glob
