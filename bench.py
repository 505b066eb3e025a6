"""Benchmark: certified-optimal PCBA solves per second and time-to-certify.

One step = one batched solve, through the C ABI, of the uneven 256-problem
workload per GPU with the whole path of Alg. 1: the FP64 monomial-to-Bernstein
conversion, the branch and bound loop of subdivide / bound / incumbent /
cut-off / compaction, and the FP64 check of the returned points, until every
problem is certified or stops.  Only certified solves (OPTIMAL or INFEASIBLE)
count.  The incumbent also takes certified box corners (vertex incumbents,
batch flag 8: a corner coefficient is the polynomial's value at the corner,
Sec. II-D); the plain Alg. 1-5 run is the no_vertex leg.  On this workload the learned warm start (cost-landscape features, the
set-encoder network's forward pass, FP32-certified candidates seeding the
incumbent) costs more per step than it saves, so it is a leg beside the
headline, not the headline.

  python bench.py [--gpus N --steps K --warmup W]      the CUDA library
  python bench.py --impl reference [...]               the CPU oracle on host cores

Workload: 256 rtd problems per GPU (rank k: seeds 4000 + 256 k + j), obstacle
counts floor(exp U(ln 16, ln 4096)); each is l = 2 on [-1,1]^2, a degree-(3,3)
map F with N(0, 0.5^2) coefficients, obstacle constraints r^2 - ||F(q) - o_i||^2
<= 0 (degree (6,6), r = 0.15, o_i ~ U([-2,2]^2)), cost ||F(q) - goal||^2.  The
library receives the constraints as a linear family in (||F||^2, F_1, F_2)
(pcba_create_linear); patches are FP32 with directed-rounding error bounds.
Inputs are resident in HBM when the timed region starts; L2 is flushed
between timed steps by writing a 256 MiB buffer.  Legs beside the headline:
the same workload with the learned warm start, in FP64 and with dense
constraints; the 64-problem 512-obstacle batch (linear, dense, dense FP64);
the tiny problems one at a time; the 4-D problems with equalities; the
warm-start A/B; the RTD* planning POPs (Sec. VI-A); the increasing-constraints
problems (Sec. V-C).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "certified-optimal solves/sec and p50/p99 time-to-certify (opt_tol 1e-3), 1 B300"
UNIT = "solves/s"
BATCH = 256
BASE_SEED = 4000
OBS_LO, OBS_HI = 16, 4096
OPT_TOL = 1e-3
EQ_TOL = 1e-4
RELAX_OPT_TOL, RELAX_EQ_TOL = 3e-2, 1e-1   # first solve of the polished pipeline (equalities)
MAX_ITERS = 28
MEM_CAP = 64 << 30        # list memory of the linear-family batch
DENSE_MEM = 200 << 30     # list memory of the dense-constraint batch (same problems)
WORKLOAD = ("uneven batch of %d rtd-shaped POPs per GPU (rank k: seeds %d+%d*k+j): l=2 on "
            "[-1,1]^2, F degree (3,3) N(0,0.5^2), obstacles floor(exp U(ln %d, ln %d)) "
            "U([-2,2]^2) r=0.15, constraints degree (6,6) given as a linear family in "
            "(||F||^2, F_1, F_2), cost ||F-goal||^2; FP32 patches with directed-rounding error "
            "bounds; vertex incumbents (corner coefficients, Sec. II-D); no warm start; "
            "opt_tol %g"
            % (BATCH, BASE_SEED, BATCH, OBS_LO, OBS_HI, OPT_TOL))


def shard_seeds(rank: int, batch: int = BATCH, base: int = BASE_SEED):
    """Seeds of the problems one rank solves (independent problems, no exchange)."""
    return [base + batch * rank + j for j in range(batch)]


def shard_problems(rank: int, batch: int = BATCH):
    """The rank's problems: obstacle counts drawn from the rank's first seed."""
    from paper_2003_01758_b300 import workloads as W
    seeds = shard_seeds(rank, batch)
    counts = W.batch_obstacle_counts(batch, seeds[0], OBS_LO, OBS_HI)
    return [W.rtd(s, n_obstacles=int(c)) for s, c in zip(seeds, counts)]


def reduce_max(value: float, world: int) -> float:
    """Max over ranks of a host scalar (gloo, CPU tensors)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def kernel_code_hash(path):
    """sha256 (first 16 hex) of a CUDA source with comments and whitespace
    removed, so that the hash changes only when the code does."""
    import hashlib
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    text = " ".join(text.split())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def profiled_traffic(src_name, prof_name):
    """DRAM bytes per subdivision step from a committed ncu summary, or None
    when the kernel code changed since that capture."""
    import re
    src = os.path.join(ROOT, "paper_2003_01758_b300", "csrc", src_name)
    prof = os.path.join(ROOT, "profiles", prof_name)
    try:
        text = open(prof).read()
        if "`%s`" % kernel_code_hash(src) not in text:
            return None
        m = re.search(r"TRAFFIC_BYTES_PER_LAUNCH = ([0-9.e+]+)", text)
        return float(m.group(1)) if m else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------

def _oracle_one(k):
    """The oracle on problem k of the rank-0 workload (its dense constraints)."""
    import oracle
    from paper_2003_01758_b300 import workloads as W
    count = W.batch_obstacle_counts(BATCH, BASE_SEED, OBS_LO, OBS_HI)[k]
    p = W.rtd(BASE_SEED + k, n_obstacles=int(count))
    t = time.perf_counter()
    r = oracle.solve(p.cost, p.ineq, p.eq, p.lo, p.hi, opt_tol=OPT_TOL, eq_tol=EQ_TOL,
                     max_iters=MAX_ITERS)
    return r["status"], time.perf_counter() - t


def oracle_pool(procs):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn"))


def run_oracle(pool, ks):
    t = time.perf_counter()
    out = list(pool.map(_oracle_one, ks))
    return out, time.perf_counter() - t


def cpu_procs():
    return max(1, min(os.cpu_count() or 1, 32))


# every 8th problem of the 256: the same spread of obstacle counts
ORACLE_SAMPLE = list(range(0, BATCH, 8))


def cpu_baseline(pool, procs):
    run_oracle(pool, [0] * procs)  # start-up of the workers
    out, dt = run_oracle(pool, ORACLE_SAMPLE)
    ok = sum(1 for s, _ in out if s in (0, 1))
    return {"value": ok / dt, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": "%d of the 256 problems (every 8th), FP64 oracle with the dense "
                      "constraints, one problem per process, %d processes, %.1f s wall"
                      % (len(ORACLE_SAMPLE), procs, dt),
            "p50_ms": 1e3 * float(np.median([t for _, t in out])),
            "p99_ms": 1e3 * float(np.percentile([t for _, t in out], 99))}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    procs = cpu_procs()
    pool = oracle_pool(procs)
    per_step = procs
    ks = lambda s: [(s * per_step + j) % BATCH for j in range(per_step)]
    for s in range(args.warmup):
        run_oracle(pool, ks(s))
    total, solved, lat = 0.0, 0, []
    for s in range(args.steps):
        out, dt = run_oracle(pool, ks(args.warmup + s))
        total += dt
        solved += sum(1 for st, _ in out if st in (0, 1))
        lat += [t for _, t in out]
    pool.shutdown()
    value = solved / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.split("; FP32")[0] + "; FP64 CPU oracle with the "
                   "dense constraints", "problems_per_step": per_step},
        "p50_ms": 1e3 * float(np.median(lat)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": "%d problems of the workload per step, one per process"
                                   % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_batch(probs, precision, linear=True, flags=0, mem_cap=MEM_CAP):
    from paper_2003_01758_b300 import pcba
    mk = pcba.linear_solver_from_problem if linear else pcba.solver_from_problem
    return pcba.Batch([mk(p, precision) for p in probs], mem_cap, flags=flags)


def host_coeffs(probs, linear=True):
    """The monomial coefficients of a batch as the library lays them out: per
    problem the cost, then the shared polynomials (linear) or every constraint."""
    parts = []
    for p in probs:
        parts.append(p.cost.ravel())
        parts.append(p.meta["linear"][0].ravel() if linear else p.ineq.ravel())
        if not linear:
            parts.append(p.eq.ravel())
    return np.concatenate(parts)


class Learned:
    """The learned-warm-start step on one batch: features, forward pass and
    guided solve, all queued on one stream."""

    def __init__(self, batch, probs):
        import torch
        from paper_2003_01758_b300 import warmstart
        self.ws = warmstart
        self.batch = batch
        self.model = warmstart.load_model()
        self.stream = torch.cuda.Stream()
        batch.set_stream(self.stream.cuda_stream)
        self.points, self.offsets, self.glob = warmstart.host_inputs(probs)
        self.pk = warmstart.Packed(self.points, self.offsets, self.glob)
        self.y = torch.empty((len(probs), 2), dtype=torch.float32, device="cuda")
        self.stencil = warmstart.default_stencil()
        batch.set_refine_stencil(warmstart.refine_stencil())
        torch.cuda.synchronize()

    def step(self, raw=True):
        ws, b = self.ws, self.batch
        b.cost_grid(ws.GRID, self.pk.glob.data_ptr(), ws.GLOBAL_DIM, ws.HOST_DIM)
        self.model.forward(*self.pk.args(), self.y.data_ptr(), stream=self.stream.cuda_stream)
        return b.solve_guided(self.y.data_ptr(), 2, self.stencil, OPT_TOL, EQ_TOL, MAX_ITERS,
                              raw=raw)

    def launches_per_step(self):
        # the solve's kernels, the cost grid and the network's forward pass
        before = self.model.kernel_launches()
        self.step()
        net = self.model.kernel_launches() - before
        return self.batch.stats()["kernel_launches"] + 1 + net

    def timed(self, steps, flush):
        """K learned steps; device time from CUDA events on the step's stream."""
        import torch
        ms, times, status, steps_ = [], [], [], []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            res = self.step()
            e1.record(self.stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            times += [r.time_ms for r in res]
            status += [r.status for r in res]
            steps_ += [r.steps for r in res]
        return ms, times, status, steps_


def timed_steps(batch, steps, flush, polished=False):
    """K solves; per-step device time from the library's CUDA events on its stream.
    polished: pcba_batch_solve_polished (relaxed solve, polish, certified solve)."""
    import torch
    ms, times, status = [], [], []
    res = None
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        if polished:
            res = batch.solve_polished(OPT_TOL, EQ_TOL, RELAX_OPT_TOL, RELAX_EQ_TOL, MAX_ITERS)
        else:
            res = batch.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
        ms.append(batch.timing()["total_ms"])
        times += [r["time_ms"] for r in res]
        status += [r["status"] for r in res]
    return ms, times, status, res


def certified(status):
    return sum(1 for s in status if s in (0, 1))


def leg_summary(ms, times, status, n_problems):
    """Certified solves/s and latency of a timed leg."""
    return {"value": certified(status) / (sum(ms) / 1e3), "unit": UNIT,
            "ms_per_step": float(np.mean(ms)), "certified": certified(status),
            "infeasible": sum(1 for s in status if s == 1), "solves": len(status),
            "p50_ms": float(np.median(times)), "p99_ms": float(np.percentile(times, 99)),
            "problems_per_step": n_problems}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="device loop in a conditional CUDA graph, or driven from the host")
    ap.add_argument("--no-extras", action="store_true",
                    help="timed headline steps only (no e2e, roofline or side legs)")
    ap.add_argument("--problems", type=int, default=0,
                    help="profiling: only the first N problems of the workload (0: all)")
    ap.add_argument("--mem-gb", type=int, default=MEM_CAP >> 30,
                    help="list memory of the headline batch in GiB")
    ap.add_argument("--launch-bytes", action="store_true",
                    help="with --no-extras: also an instrumented host-loop solve, printing "
                         "the algorithmic bytes of each subdivision step")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and "MASTER_ADDR" in os.environ:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    else:
        world = 1
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        return rc
    args.warmup = max(args.warmup, 3)

    # the oracle pool starts before the first CUDA call (spawned workers)
    pool = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pool = oracle_pool(cpu_procs())

    import torch
    from paper_2003_01758_b300 import build, pcba
    build.build()
    torch.cuda.set_device(local)
    probs = shard_problems(rank)
    if args.problems > 0:
        probs = probs[:args.problems]
    loop_flag = 0 if args.loop == "graph" else pcba.Batch.HOST_LOOP
    batch = make_batch(probs, pcba.FP32, linear=True, flags=loop_flag | pcba.Batch.VERTEX,
                       mem_cap=args.mem_gb << 30)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    learned = Learned(batch, probs)

    for _ in range(args.warmup):
        batch.solve(OPT_TOL, EQ_TOL, MAX_ITERS)

    # ---- timed region: K batched solves (Alg. 1, no warm start), inputs
    # resident in HBM ----
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, times, status, last = timed_steps(batch, args.steps, flush)
    clk = clocks.stop()
    nsteps = [r["steps"] for r in last]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = reduce_max(float(sum(ms)), world)
    cert_all = reduce_sum(float(certified(status)), world)
    value = cert_all / (total_ms / 1e3)
    optimal = sum(1 for s in status if s == pcba.OPTIMAL)
    infeasible = sum(1 for s in status if s == pcba.INFEASIBLE)
    launches = batch.stats()["kernel_launches"] * args.steps
    if args.no_extras:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "ms_per_step": total_ms / args.steps,
               "problems_per_step": len(probs), "loop": args.loop,
               "certified": optimal + infeasible, "clocks": clk}
        if args.launch_bytes:
            # after the timed solves: one instrumented host-loop solve
            ib = make_batch(probs, pcba.FP32, linear=True,
                            flags=pcba.Batch.INSTRUMENT | pcba.Batch.VERTEX,
                            mem_cap=args.mem_gb << 30)
            ib.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
            out["launch_bytes"] = [float(x) for x in ib.launch_bytes()]
            ib.close()
        if rank == 0:
            print(json.dumps(out))
        return 0

    from paper_2003_01758_b300 import warmstart
    # ---- the same solves without vertex incumbents (Alg. 1-5 as printed) ----
    nb = make_batch(probs, pcba.FP32, linear=True, mem_cap=args.mem_gb << 30)
    nb.set_stream(learned.stream.cuda_stream)
    nb.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
    nms, ntimes, nstatus, nres = timed_steps(nb, args.steps, flush)
    no_vertex = leg_summary(nms, ntimes, nstatus, len(probs))
    no_vertex["mean_bisection_steps"] = float(np.mean([r["steps"] for r in nres]))
    no_vertex["value"] = reduce_sum(float(certified(nstatus)), world) / (
        reduce_max(float(sum(nms)), world) / 1e3)
    nb.close()

    # ---- the same solves with the learned warm start (network forward pass,
    # candidates certified, guided solve; all in the step) ----
    learned.step()
    lms, ltimes, lstatus, lsteps = learned.timed(args.steps, flush)
    learned_leg = leg_summary(lms, ltimes, lstatus, len(probs))
    learned_leg["mean_bisection_steps"] = float(np.mean(lsteps))
    learned_leg["value"] = reduce_sum(float(certified(lstatus)), world) / (
        reduce_max(float(sum(lms)), world) / 1e3)
    learned_leg["gpu_launches_per_step"] = learned.launches_per_step()
    learned_leg["warm_start"] = ("set-encoder network, BF16 on tcgen05; %d-candidate stencil, "
                                 "then %d around the seed, certified in FP32"
                                 % (len(learned.stencil), len(warmstart.refine_stencil())))

    # ---- end to end: host inputs in (monomial coefficients and constraint
    # rows), solve, results out; wall clock ----
    # (page-locked by the library with cudaHostAlloc: torch's pinned buffers
    # measured ~10 GB/s for these copies, the library's ~50 GB/s)
    # the rows are sent without their padding (1 + K doubles per constraint)
    hc, hr = host_coeffs(probs), pcba.linear_rows_packed(probs)
    h_coeffs = pcba.host_empty(hc.size)
    h_coeffs[:] = hc.ravel()
    h_rows = pcba.host_empty(hr.size)
    h_rows[:] = hr.ravel()
    assert h_coeffs.size == batch.input_doubles() and h_rows.size == batch.rows_packed_doubles()

    def e2e_step():
        batch.upload(h_coeffs)
        batch.upload_rows_packed(h_rows)
        return batch.solve(OPT_TOL, EQ_TOL, MAX_ITERS, raw=True)

    e2e_step()
    e2e_s, e2e_status = 0.0, []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        res = e2e_step()
        e2e_s += time.perf_counter() - t
        e2e_status += [r.status for r in res]
    e2e_stats = batch.stats()
    e2e_value = reduce_sum(float(certified(e2e_status)), world) / reduce_max(e2e_s, world)

    # ---- roofline of the subdivision step (split + bound kernels): CUDA
    # events around each launch pair in a host-driven loop ----
    ibatch = make_batch(probs, pcba.FP32, linear=True,
                        flags=pcba.Batch.INSTRUMENT | pcba.Batch.VERTEX)
    ibatch.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
    ibatch.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
    it = ibatch.timing()
    lin = ibatch.linear_stats()
    ibatch.close()
    peak, peak_kind = load_peaks()
    achieved = it["subdiv_bytes"] / (it["subdiv_ms"] * 1e-3) / 1e9 if it["subdiv_ms"] > 0 else 0.0

    # ---- FP64 (plain arithmetic, no warm start), same problems: the FP32
    # bounds against the FP64 ones, per result ----
    fp32_res = [dict(lower=r["lower"], upper=r["upper"], status=r["status"],
                     upper_err=r["upper_err"]) for r in batch.solve(OPT_TOL, EQ_TOL, MAX_ITERS)]
    b64 = make_batch(probs, pcba.FP64, linear=True, flags=pcba.Batch.VERTEX)
    b64.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
    ms64, t64, st64, res64 = timed_steps(b64, 2, flush)
    b64.close()
    both = [(a, b) for a, b in zip(fp32_res, res64)
            if a["status"] == 0 and b["status"] == 0]
    dlo = np.array([abs(a["lower"] - b["lower"]) for a, b in both])
    dup = np.array([abs(a["upper"] - b["upper"]) for a, b in both])
    uerr = np.array([a["upper_err"] for a, _ in both])
    fp32_vs_fp64 = {
        "problems_compared": len(both),
        "status_equal": sum(1 for a, b in zip(fp32_res, res64) if a["status"] == b["status"]),
        "abs_lower_diff": {"max": float(dlo.max()), "median": float(np.median(dlo))},
        "abs_upper_diff": {"max": float(dup.max()), "median": float(np.median(dup))},
        "fp32_upper_err": {"max": float(uerr.max()), "median": float(np.median(uerr))},
        "fp64": leg_summary(ms64, t64, st64, len(probs)),
    }

    # the main batch's memory is not needed any more
    batch.close()
    torch.cuda.synchronize()

    side = {}
    if rank == 0 and world == 1:
        from paper_2003_01758_b300 import train_warmstart
        from paper_2003_01758_b300 import workloads as W
        # ---- the same 256 problems with dense constraints (a patch per
        # obstacle), learned warm start, autotuned subdivision kernel ----
        db = make_batch(probs, pcba.FP32, linear=False, mem_cap=DENSE_MEM)
        tune = db.autotune(OPT_TOL, EQ_TOL, MAX_ITERS)
        dl = Learned(db, probs)
        dl.step()
        dms, dtimes, dstatus, _ = dl.timed(2, flush)
        side["dense_constraints"] = leg_summary(dms, dtimes, dstatus, len(probs))
        side["dense_constraints"]["autotune"] = tune
        db.close()
        torch.cuda.synchronize()

        # ---- 64 problems with 512 obstacles: linear and dense constraints
        # (learned warm start) and the paper's plain FP64 method (dense, no
        # warm start) ----
        c2 = [W.rtd(2000 + j) for j in range(64)]
        for name, linear, prec, warm in (("linear_fp32_learned", True, pcba.FP32, True),
                                         ("dense_fp32_learned", False, pcba.FP32, True),
                                         ("dense_fp64_plain", False, pcba.FP64, False)):
            b2 = make_batch(c2, prec, linear=linear, mem_cap=64 << 30)
            if warm:
                l2 = Learned(b2, c2)
                l2.step()
                m2, t2, s2, _ = l2.timed(3, flush)
            else:
                b2.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
                m2, t2, s2, _ = timed_steps(b2, 2, flush)
            side.setdefault("batch64_obstacles512", {})[name] = leg_summary(m2, t2, s2, 64)
            b2.close()

        # ---- the tiny problems (degree 4, 10 constraints, FP64), one at a time ----
        tiny_ms, tiny_status = [], []
        for j in range(32):
            q = W.tiny(1000 + j)
            sb = pcba.Batch([pcba.solver_from_problem(q, pcba.FP64)], 1 << 28)
            sb.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
            r = sb.solve(OPT_TOL, EQ_TOL, MAX_ITERS)[0]
            tiny_ms.append(sb.timing()["total_ms"])
            tiny_status.append(r["status"])
            sb.close()
        side["tiny_one_at_a_time"] = {
            "p50_ms": float(np.median(tiny_ms)), "p99_ms": float(np.percentile(tiny_ms, 99)),
            "certified": certified(tiny_status), "solves": len(tiny_status),
            "workload": "32 tiny POPs (seeds 1000+k): l=2, cost and 10 constraints of degree "
                        "(4,4), FP64, each solved alone"}

        # ---- one problem of the workload at a time (linear, FP32, no warm start) ----
        single = []
        for q in probs[:16]:
            sb = make_batch([q], pcba.FP32, linear=True, mem_cap=4 << 30)
            sb.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
            sb.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
            single.append(sb.timing()["total_ms"])
            sb.close()
        side["single_problem_ms"] = {"p50": float(np.median(single)),
                                     "p99": float(np.percentile(single, 99))}

        # ---- learned warm start A/B: 256 held-out problems, obstacles
        # log-uniform in [64, 1024] (the training range), seeds 6000+k ----
        ab = train_warmstart.ab_compare(learned.model, train_warmstart.held_out(256),
                                        maker=pcba.linear_solver_from_problem)
        ab["workload"] = ("256 held-out rtd problems, obstacles floor(exp U(ln 64, ln 1024)), "
                          "seeds 6000+k, linear families in FP32, one batched solve per arm and "
                          "repeat; network trained on 100k solutions of seeds 5000000+k")
        side["learned_warm_start_ab"] = ab

        # ---- 4-D problems: 64 inequalities of degree 3, 2 equalities of
        # degree 2, eq_tol 1e-4, 8 GiB list cap per problem ----
        d4 = [W.dim4(3000 + k) for k in range(8)]
        dim4 = {"workload": "8 problems l=4, cost degree 4, 64 g_i degree 3, 2 h_j degree 2, "
                            "seeds 3000+k, eq_tol 1e-4, 8 GiB per problem",
                "polished": "pcba_batch_solve_polished: solve at opt_tol %g, eq_tol %g, "
                            "barrier-Newton polish of its points, certified solve at opt_tol "
                            "1e-3, eq_tol 1e-4 seeded with them; time and launches of all "
                            "three phases" % (RELAX_OPT_TOL, RELAX_EQ_TOL)}
        for prec, name in ((pcba.FP32, "fp32_polished"), (pcba.FP64, "fp64_polished")):
            dbt = pcba.Batch([pcba.solver_from_problem(q, prec) for q in d4], 8 * (8 << 30))
            dbt.solve_polished(OPT_TOL, EQ_TOL, RELAX_OPT_TOL, RELAX_EQ_TOL, MAX_ITERS)
            dms4, dt4, ds4, dres = timed_steps(dbt, 5, flush, polished=True)
            dim4[name] = leg_summary(dms4, dt4, ds4, len(d4))
            dim4[name]["max_width"] = float(max(r["upper"] - r["lower"] for r in dres))
            dim4[name]["max_abs_h"] = float(max(r["verify_max_abs_h"] for r in dres))
            dbt.close()
        side["dim4"] = dim4

        # ---- RTD* planning POPs (Sec. VI-A): 64 problems, 30..300 degree-12
        # obstacle constraints (log-uniform), one or two waypoints ----
        rng = np.random.default_rng(9)
        counts = np.floor(np.exp(rng.uniform(np.log(30), np.log(300), 64))).astype(int)
        rs = [W.rtd_star(7000 + k, n_ineq=int(c), n_wp=1 + k % 2) for k, c in enumerate(counts)]
        star = {"workload": "64 RTD* POPs (seeds 7000+k): Q = [0,1] x [-1,1], waypoint-product "
                            "cost (degree 10 with one waypoint, 16 with two), 30..300 "
                            "degree-12 obstacle constraints, no warm start"}
        for name, linear, prec in (("linear_fp32", True, pcba.FP32),
                                   ("dense_fp64_plain", False, pcba.FP64)):
            bs = make_batch(rs, prec, linear=linear, mem_cap=32 << 30)
            bs.solve(OPT_TOL, EQ_TOL, MAX_ITERS)
            sm, st, ss, _ = timed_steps(bs, 3, flush)
            star[name] = leg_summary(sm, st, ss, len(rs))
            bs.close()
        side["rtd_star"] = star

        # ---- increasing constraints (Sec. V-C): per objective the paper's 20
        # trials, 10, 20, ..., 200 random degree-2 constraints, one batch ----
        from tests import benchmarks
        inc = {"workload": "per appendix objective, the problems with 10, 20, .., 200 random constraints "
                           "of total degree <= 2 (coefficients U[-5, 5], the optimizer kept "
                           "feasible with margin 1), seeds 11+n; dense FP32; opt_tol 1e-3 "
                           "max(1, |optimum|)"}
        # list memory per problem: 1 GiB, Powell 5 GiB; Wood keeps ~1.9M boxes
        # of dense patches (9.5 GB at 10 constraints, > 40 GB from 50 on), so
        # only its trials with 10..40 constraints run, one at a time at 40 GiB
        for name in ("EVD", "Powell", "Wood", "DixonPrice2", "DixonPrice3", "DixonPrice4",
                     "Beale", "Bukin02", "DeckkersAarts"):
            bm = benchmarks.load(name)
            trials = range(10, 41, 10) if name == "Wood" else range(10, 201, 10)
            per = {"Powell": 5 << 30, "Wood": 40 << 30}.get(name, 1 << 30)
            ps = [W.increasing_constraints(bm["cost"], bm["lo"], bm["hi"], bm["x_opt"], n,
                                           seed=11 + n) for n in trials]
            tol = 1e-3 * max(1.0, abs(bm["optimum"]))
            groups = [[q] for q in ps] if name == "Wood" else [ps]
            ims, itimes, ist, ipeak = [0.0] * 3, [], [], 0
            for grp in groups:
                bi = pcba.Batch([pcba.solver_from_problem(q, pcba.FP32) for q in grp],
                                len(grp) * per)
                bi.solve(tol, EQ_TOL, MAX_ITERS)
                for rep in range(3):
                    flush.zero_()
                    torch.cuda.synchronize()
                    ires = bi.solve(tol, EQ_TOL, MAX_ITERS)
                    ims[rep] += bi.timing()["total_ms"]
                    itimes += [r["time_ms"] for r in ires]
                    ist += [r["status"] for r in ires]
                    ipeak = max(ipeak, max(r["peak_items"] for r in ires))
                bi.close()
            inc[name] = leg_summary(ims, itimes, ist, len(ps))
            inc[name]["peak_items"] = int(ipeak)
        side["increasing_constraints"] = inc

    base = None
    if pool is not None:
        base = cpu_baseline(pool, cpu_procs())
        pool.shutdown()

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "problems_per_step": len(probs),
                   "warm_start": "none (Alg. 1 from the root box; the learned warm start is "
                                 "the learned_warm_start leg)",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "independent problems per GPU (dp%d)" % world,
                   "device_loop": args.loop},
        "p50_ms": float(np.median(times)), "p99_ms": float(np.percentile(times, 99)),
        "certified": {"optimal": optimal, "infeasible": infeasible,
                      "failed": len(status) - optimal - infeasible},
        "mean_bisection_steps": float(np.mean(nsteps)),
        "no_vertex": no_vertex,
        "learned_warm_start": learned_leg,
        "fp32_vs_fp64": fp32_vs_fp64,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_traffic("pcba_linear.cuh", "k2_lin_uneven256_fp32.md"),
                     "kernel": "k2_lin_split + k2_lin_bound (one subdivision step)",
                     "peak_kind": peak_kind, "launches": it["subdiv_launches"],
                     "algorithmic_bytes_per_launch":
                         it["subdiv_bytes"] / max(1, it["subdiv_launches"]),
                     "avg_launch_ms": it["subdiv_ms"] / max(1, it["subdiv_launches"]),
                     "constraint_bounds": lin["pairs"], "coefficient_ranges": lin["full"]},
        "cpu_baseline": base,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": e2e_stats["h2d_bytes"],
                "d2h_bytes_per_step": e2e_stats["d2h_bytes"]},
        "gpu_launches": launches,
        "clocks": clk,
    }
    line.update(side)
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
