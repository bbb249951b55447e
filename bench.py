"""Benchmark of the PDNQP rAPDHG hot path on one GB300 (or N replicas).

Workload: the 1M-variable synthetic nonconvex QP (n = 1,000,000, m = 500,000,
Q ~ 5M nnz banded + random, A ~ 4M nnz, box [-1, 1], two-sided rows).

A step is one pass of the whole hot path: pdnqp_solve from the start point
with a fixed budget of accepted inner iterations (setup of each inner solve,
trial/accept/average/check/restart iterations, outer multiplier and penalty
updates).  `value` is accepted rAPDHG inner iterations per second over the
timed steps, all ranks (replicas only: each rank solves its own seeded
instance, no data-path collective).  Inputs are larger than L2 (129 MB), so
no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       [--precision 32|64] [--budget B] [--ttk SECONDS]

Other legs, each printing its own JSON line instead of the one above:
  --batch K [--batch-threads T] [--batch-time-limit S]
      the batched form: K independent problems of uneven sizes solved
      concurrently (sharded by problem across ranks under torchrun);
  --solve-times [--no-cpu]
      end-to-end solve times of the GPU forms and the oracle on the n = 200
      and n = 50,000 workloads, to rel-KKT 1e-4 and 1e-6.
"""
from __future__ import annotations

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

METRIC = "rAPDHG iters/s & time-to-1e-4 KKT (1M-var QP), %HBM peak, vs plain FP64 form"
WORKLOAD = "synthetic nonconvex QP n=1e6 m=5e5 (Q 5M nnz band+random, A 4M nnz, box [-1,1])"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="native", choices=["native", "reference"])
    p.add_argument("--precision", type=int, default=32, choices=[32, 64])
    p.add_argument("--budget", type=int, default=2000, help="accepted inner iterations per step")
    p.add_argument("--ttk", type=float, default=90.0,
                   help="also time solves to rel-KKT 1e-4, each capped at this many seconds (0: skip)")
    p.add_argument("--no-compare", action="store_true", help="skip the plain FP64 comparison leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU (oracle) baseline leg")
    p.add_argument("--loop", default="persistent", choices=["persistent", "cond", "unrolled"],
                   help="inner loop: one persistent cooperative launch per check period (default), or a CUDA graph "
                        "with conditional WHILE/IF nodes, or unrolled graph slots")
    p.add_argument("--batch", type=int, default=0,
                   help="batched form instead: solve this many problems of uneven sizes concurrently")
    p.add_argument("--batch-threads", type=int, default=16)
    p.add_argument("--batch-time-limit", type=float, default=5.0, help="seconds per problem")
    p.add_argument("--batch-median", type=float, default=1e4, help="median n of the batch's log-normal sizes")
    p.add_argument("--batch-sigma", type=float, default=1.0, help="log-std of the batch's sizes")
    p.add_argument("--batch-procs", type=int, default=min(16, os.cpu_count() or 1),
                   help="processes that build the batch's problems")
    p.add_argument("--batch-mix", default="alternate", choices=["alternate", "small"],
                   help="alternate: half small generator, half Motzkin-Straus; small: small generator only")
    p.add_argument("--batch-compare", action="store_true",
                   help="also solve the whole batch in the thread-pool form (fresh handles) and report both walls")
    p.add_argument("--solve-times", action="store_true",
                   help="instead: end-to-end solve times of the GPU forms and the oracle on the n=200 and "
                        "n=50,000 workloads")
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--m", type=int, default=500_000)
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def captured_traffic(precision, trials_per_launch):
    """DRAM bytes (read + write) per launch of the trial loop from the committed
    ncu capture (profiles/traffic_trials_fp{32,64}.json) scaled to the launch's
    trials, or None when the kernel sources changed since the capture."""
    tr_path = os.path.join(ROOT, "profiles", f"traffic_trials_fp{precision}.json")
    if not os.path.exists(tr_path):
        return None
    tj = json.load(open(tr_path))
    hsh = hashlib.sha256()
    for f in tj.get("source_files", []):
        hsh.update(open(os.path.join(ROOT, f), "rb").read())
    if tj.get("source_sha256") != hsh.hexdigest() or not tj.get("dram_bytes_per_trial"):
        return None
    return tj["dram_bytes_per_trial"] * trials_per_launch


def trial_bytes(inst, v):
    """Algorithmic bytes of one accepted trial of the inner iteration with each
    array read or written once (value size v, int32 indices): the matrices Q
    (with its diagonal), A and A^T with their row pointers, 14 touches of an
    n-vector (x, xbar, Hx, Hxbar, A'y read and written; q, tau, l, u read),
    20 of an inequality-row vector (s, r, sbar, rbar, y, ybar, Bw read and
    written; tau_s, tau_r, l_s, u_s, q_r, eta read) and 12 of an equality-row
    vector."""
    Q, A = inst["Q"], inst["A"]
    n, m = Q.shape[0], A.shape[0]
    nnz_h = Q.nnz + int((Q.diagonal() == 0).sum())
    m_e = int((inst["l_c"] == inst["u_c"]).sum())
    mats = (v + 4) * (nnz_h + 2 * A.nnz) + 4 * (2 * n + m + 2)
    return float(mats + 14 * v * n + 20 * v * (m - m_e) + 12 * v * m_e)


def make_instance(args, seed):
    from paper_2609_19557_gb300 import instances as I
    return I.large_qp(seed, n=args.n, m=args.m)


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def set_loop(P, h, loop):
    P.pdnqp_set_param(h, "persistent", 1 if loop == "persistent" else 0)
    P.pdnqp_set_param(h, "cond_graph", 1 if loop == "cond" else 0)


def aggregate(ws, dt, iters, device):
    """Whole-job figures of a timed region: the slowest rank's time and the sum
    of the units all ranks processed (replicas: no data-path collective; this
    is the only exchange, after the timed region)."""
    if ws <= 1:
        return dt, iters
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(dt)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def run_native(args):
    import torch

    from paper_2609_19557_gb300 import build as B
    from paper_2609_19557_gb300 import pdnqp as P

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    P.load()
    inst = make_instance(args, seed=rank)
    stream = torch.cuda.current_stream()
    h = P.create_from_instance(inst, precision=args.precision, stream=stream.cuda_stream)
    P.pdnqp_set_param(h, "iter_budget", args.budget)
    set_loop(P, h, args.loop)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        P.pdnqp_solve(h, 1e-4, 1e-4)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = 0
    launches = 0
    loop_s, loop_trials, loop_launches, blocks = 0.0, 0, 0, 0
    barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        P.pdnqp_solve(h, 1e-4, 1e-4)
        _, _, r = P.pdnqp_get(h)
        iters += r["inner_iters"]
        launches += r["kernel_launches"]
        loop_s += r["loop_seconds"]
        loop_trials += r["loop_trials"]
        loop_launches += r["loop_launches"]
        blocks = r["loop_blocks"]
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    dt = ev0.elapsed_time(ev1) / 1e3
    t_max, it_all = aggregate(ws, dt, iters, "cuda")
    value = it_all / t_max

    # Dominant kernel: the persistent trial loop (k_trials), timed live inside
    # the timed region by CUDA events around each of its launches on this
    # stream; algorithmic bytes per trial from the library (every array once
    # per pass, gathers served from L2).
    peak, peak_src = measured_peaks()
    roof = None
    if loop_trials > 0 and loop_s > 0:
        # Algorithmic bytes of one trial with every array read or written once
        # per trial (matrices, x-state, row state); the library's per-pass
        # count (arrays touched by several passes counted once per pass) is
        # reported beside it.
        bpt_pass = P.pdnqp_kernel_bytes(h, 5)
        bpt = trial_bytes(inst, 4 if args.precision == 32 else 8)
        achieved = bpt * loop_trials / loop_s / 1e9
        per_launch = loop_trials / max(1, loop_launches)
        traffic = captured_traffic(args.precision, per_launch)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "k_trials (persistent trial loop: primal, row and column passes, "
                "acceptance decision)", "peak_source": peak_src,
                "algorithmic_bytes_per_trial": bpt, "per_pass_bytes_per_trial": bpt_pass,
                "frac_per_pass": bpt_pass * loop_trials / loop_s / 1e9 / peak, "trials_per_launch": per_launch,
                "us_per_trial": 1e6 * loop_s / loop_trials, "blocks": blocks}

    # End to end through the public API with host buffers: create (H2D of the
    # problem) + solve + get (D2H of x, y) inside the timed region.
    h2d = sum(a.nbytes for a in (inst["Q"].data, inst["Q"].indices, inst["Q"].indptr, inst["A"].data,
                                 inst["A"].indices, inst["A"].indptr, inst["c"], inst["l_c"], inst["u_c"],
                                 inst["l_x"], inst["u_x"]))
    d2h = 8 * (inst["Q"].shape[0] + inst["A"].shape[0])
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(e2e_steps):
        h2 = P.create_from_instance(inst, precision=args.precision, stream=stream.cuda_stream)
        P.pdnqp_set_param(h2, "iter_budget", args.budget)
        set_loop(P, h2, args.loop)
        P.pdnqp_solve(h2, 1e-4, 1e-4)
        x, y, r2 = P.pdnqp_get(h2)
        e2e_iters += r2["inner_iters"]
        h2.close()
    barrier()
    e2e_dt = time.perf_counter() - t0
    e2e_dt, e2e_iters = aggregate(ws, e2e_dt, e2e_iters, "cuda")

    # Plain FP64 form on the same GPU (the comparison the metric names).
    compare = None
    if not args.no_compare and args.precision != 64:
        h64 = P.create_from_instance(inst, precision=64, stream=stream.cuda_stream)
        P.pdnqp_set_param(h64, "iter_budget", args.budget)
        set_loop(P, h64, args.loop)
        P.pdnqp_solve(h64, 1e-4, 1e-4)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        it64, ls64, lt64, ll64 = 0, 0.0, 0, 0
        for _ in range(max(1, args.steps // 2)):
            P.pdnqp_solve(h64, 1e-4, 1e-4)
            r64 = P.pdnqp_get(h64)[2]
            it64 += r64["inner_iters"]
            ls64 += r64["loop_seconds"]
            lt64 += r64["loop_trials"]
            ll64 += r64["loop_launches"]
        a1.record(stream)
        torch.cuda.synchronize()
        compare = {"fp64_iters_per_s": it64 / (a0.elapsed_time(a1) / 1e3)}
        if lt64 > 0 and ls64 > 0:
            # The plain FP64 form's trial loop against the same HBM roofline
            # (one count per array per trial, 8-byte values).
            b64 = trial_bytes(inst, 8)
            ach64 = b64 * lt64 / ls64 / 1e9
            compare["roofline"] = {"bound": "hbm", "achieved": ach64, "peak": peak, "unit": "GB/s",
                                   "frac": ach64 / peak, "kernel": "k_trials<double>",
                                   "traffic": captured_traffic(64, lt64 / max(1, ll64)),
                                   "algorithmic_bytes_per_trial": b64, "us_per_trial": 1e6 * ls64 / lt64,
                                   "trials_per_launch": lt64 / max(1, ll64),
                                   "fp64_pipe": "the FP64 pipe is 67 % busy in this kernel (ncu, "
                                                "profiles/k_trials_n1e6_fp64.md): it binds before HBM"}
        h64.close()

    ttk = None
    if args.ttk > 0 and rank == 0:
        # Time to relative KKT 1e-4 (capped at --ttk seconds each): the FP32-bulk
        # form with the trained controller (when its weights are present) and
        # the plain FP64 form with the paper's rules.
        ttk = {}
        wpath = os.path.join(ROOT, "paper_2609_19557_gb300", "controller_weights.npy")
        legs = [("fp32_controller" if os.path.exists(wpath) else "fp32", 32, os.path.exists(wpath)),
                ("fp64_plain", 64, False)]
        for name, prec, use_ctrl in legs:
            h3 = P.create_from_instance(inst, precision=prec, stream=stream.cuda_stream)
            P.pdnqp_set_param(h3, "time_limit", args.ttk)
            if use_ctrl:
                P.pdnqp_set_controller(h3, np.load(wpath))
                P.pdnqp_set_param(h3, "controller", 1)
            st = P.pdnqp_solve(h3, 1e-4, 1e-4)
            _, _, r3 = P.pdnqp_get(h3)
            ttk[name] = {"status": P.STATUS_NAMES[st], "seconds": r3["solve_seconds"], "rel_kkt": r3["rel_kkt"],
                         "outer_iters": r3["outer_iters"], "inner_iters": r3["inner_iters"], "cap_s": args.ttk,
                         "time_to_1e-4_s": r3["solve_seconds"] if P.STATUS_NAMES[st] == "SOLVED" else None}
            h3.close()

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(inst)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == 32 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "m": args.m, "step": f"pdnqp_solve with {args.budget} "
                       "accepted inner iterations", "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU", "loop": args.loop,
                       "precision": "FP32-bulk" if args.precision == 32 else "plain FP64"},
            "e2e": {"value": e2e_iters / e2e_dt, "unit": "iters/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        if compare:
            out["vs_plain_fp64"] = {"fp64_iters_per_s": compare["fp64_iters_per_s"],
                                    "speedup": value / ws / compare["fp64_iters_per_s"],
                                    "roofline": compare.get("roofline")}
        if ttk:
            out["time_to_1e-4"] = ttk
        print(json.dumps(out), flush=True)
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def host_cpu():
    """The host's processor and core count (stated beside every CPU timing)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and not model:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return {"nproc": os.cpu_count(), "cpu": model or platform.processor() or "unknown", "arch": platform.machine()}


def cpu_baseline(inst, first=2, last=6):
    """The oracle as it stands, single-threaded, on a bounded sample of the same
    workload: accepted inner iterations per second between two checkpoints of
    the first inner solve."""
    from oracle import oracle as O
    O.build()
    times, setup = O.debug_inner_timed(inst, [first, last])
    if len(times) < 2:
        return None
    rate = (last - first) / (times[1] - times[0])
    return {"value": rate, "unit": "iters/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"accepted inner iterations {first}..{last} of the first inner solve (setup {setup:.1f} s excluded)"}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload and metric."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    inst = make_instance(args, seed=0)
    per_step = 1  # accepted inner iterations per step (the oracle needs ~seconds per iteration here)
    ck = [per_step * (k + 1) for k in range(args.warmup + args.steps)]
    times, setup = O.debug_inner_timed(inst, ck)
    t_w = times[args.warmup - 1] if args.warmup > 0 else 0.0
    dt = times[-1] - t_w
    value = per_step * args.steps / dt
    out = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "n": args.n, "m": args.m,
                      "step": f"{per_step} accepted inner iteration(s) of the FP64 oracle"},
           "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                            "sample": f"{args.steps} timed steps after {args.warmup} warm-up steps; setup "
                                      f"{setup:.1f} s excluded"},
           "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batch_shard(count, ws, rank):
    """Problems of a batch that one rank solves: positions rank, rank + ws, ...
    (the batch shards by problem; sizes interleave, so the ranks get similar
    mixes)."""
    return list(range(rank, count, ws))


def batch_totals(ws, wall, solved, inner, device):
    """Whole-job batch figures: the slowest rank's wall time and the sums of
    solved problems and inner iterations (the only exchange, after the solves)."""
    if ws <= 1:
        return wall, solved, inner
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(wall)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(solved), float(inner)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c[0].item())), int(round(c[1].item()))


def _batch_one(a):
    from paper_2609_19557_gb300 import instances as I
    count, k, med, sig, mix, shift = a
    return I.batched_set(0, count=count, only=[k], n_median=med, sigma=sig, mix=mix, shift=shift)[0]


def spawn_pool(procs):
    """A pool of `procs` spawned processes whose numeric libraries run one
    thread each (the variables are read when a child imports them; with one
    BLAS thread pool per child the children oversubscribe the cores)."""
    import multiprocessing as mp
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        return mp.get_context("spawn").Pool(procs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def batch_instances(count, positions, median, sigma, procs, mix="alternate"):
    """The batch's problems at `positions`, built in `procs` spawned processes
    (each problem has its own seed and the shift is computed once, so the
    result does not depend on procs)."""
    from paper_2609_19557_gb300 import instances as I
    shift = I.batched_shift(0)
    if procs <= 1:
        return I.batched_set(0, count=count, only=positions, n_median=median, sigma=sigma, mix=mix, shift=shift)
    with spawn_pool(procs) as pool:
        return pool.map(_batch_one, [(count, k, median, sigma, mix, shift) for k in positions], chunksize=1)


def run_batch(args):
    """Batched form: `args.batch` independent problems (sizes lognormal in
    [1e3, 1e5] with median --batch-median and log-std --batch-sigma; half from
    the small generator with m = n / 2, half Motzkin-Straus on G(n, 0.01))
    solved to rel-KKT 1e-4, each with its own termination and a per-problem
    time limit, in the fused form (all inner iterations in one captured graph,
    one launch per phase for the whole batch); plus the first 8 problems
    solved one after another, in the fused form and in the thread-pool form."""
    import torch
    from paper_2609_19557_gb300 import instances as I
    from paper_2609_19557_gb300 import pdnqp as P
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.load()
    t = time.perf_counter()
    insts = batch_instances(args.batch, batch_shard(args.batch, ws, rank), args.batch_median, args.batch_sigma,
                            args.batch_procs, args.batch_mix)
    gen_s = time.perf_counter() - t
    t = time.perf_counter()
    hs = []
    for inst in insts:
        h = P.create_from_instance(inst, precision=args.precision)
        P.pdnqp_set_param(h, "time_limit", args.batch_time_limit)
        hs.append(h)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t

    def solve_all(sub, fused, threads=16):
        P.pdnqp_set_param(sub[0], "batch_fused", fused)
        t0 = time.perf_counter()
        sts = P.pdnqp_solve_batch(sub, 1e-4, 1e-4, threads=threads)
        return sts, time.perf_counter() - t0

    if ws > 1:
        torch.distributed.barrier()
    sts, wall = solve_all(hs, 1)
    res = [P.pdnqp_get(h)[2] for h in hs]
    names = [P.STATUS_NAMES[s] for s in sts]
    solved = names.count("SOLVED")
    inner = sum(r["inner_iters"] for r in res)
    # HBM roofline of the batched graph: algorithmic bytes of every trial of
    # every problem (one count per array per trial) over the device time of
    # the graph launches (CUDA events on the batch's stream).
    vb = 4 if args.precision == 32 else 8
    trial_b = sum(r["trials"] * trial_bytes(inst, vb) for r, inst in zip(res, insts))
    gsec = P.pdnqp_get_param(hs[0], "batch_graph_seconds")
    peak, peak_src = measured_peaks()
    roof = None
    if gsec > 0:
        ach = trial_b / gsec / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "kernel": "batched graph (kb_primal, kb_rows, kb_cols, kb_check_*), all problems",
                "peak_source": peak_src, "graph_seconds": gsec,
                "graph_launches": int(P.pdnqp_get_param(hs[0], "batch_graph_launches")),
                "algorithmic_bytes": trial_b}
    wall, solved_all, inner_all = batch_totals(ws, wall, solved, inner, torch.device("cuda", local))
    if rank != 0:
        for h in hs:
            h.close()
        torch.distributed.destroy_process_group()
        return
    whole_pool = None
    if args.batch_compare and ws == 1:
        hp = []
        for inst in insts:
            h = P.create_from_instance(inst, precision=args.precision)
            P.pdnqp_set_param(h, "time_limit", args.batch_time_limit)
            hp.append(h)
        sts_p, wall_p = solve_all(hp, 0, args.batch_threads)
        rp = [P.pdnqp_get(h)[2] for h in hp]
        whole_pool = {"wall_s": wall_p, "solved": [P.STATUS_NAMES[x] for x in sts_p].count("SOLVED"),
                      "inner_iters_total": int(sum(r["inner_iters"] for r in rp)),
                      "same_iterates_as_fused": all(np.array_equal(P.pdnqp_get(a)[0], P.pdnqp_get(b)[0])
                                                    for a, b in zip(hs, hp)),
                      "fused_speedup": wall_p / wall}
        for h in hp:
            h.close()
    sub = hs[:8]
    t0 = time.perf_counter()
    for h in sub:
        P.pdnqp_set_param(h, "persistent", 0)
        P.pdnqp_solve(h, 1e-4, 1e-4)
    seq_s = time.perf_counter() - t0
    _, fused_s = solve_all(sub, 1)
    _, pool_s = solve_all(sub, 0, args.batch_threads)
    ns = [h.n for h in hs]
    out = {"metric": "batched solves to rel-KKT 1e-4", "value": solved_all / wall, "unit": "solved instances/s",
           "leg": "batched", "n_gpus": ws, "higher_is_better": True,
           "scaling": "strong (the batch is split by problem)" if ws > 1 else None,
           "dtype": "f32+f64" if args.precision == 32 else "f64",
           "data": "synthetic", "instances": args.batch, "solved": solved_all,
           "instances_per_s": args.batch / wall,
           "statuses_rank0": {k: names.count(k) for k in sorted(set(names))},
           "wall_s": wall, "inner_iters_total": inner_all, "inner_iters_per_s": inner_all / wall,
           "roofline": roof, "time_limit_per_problem_s": args.batch_time_limit,
           "generate_s": gen_s, "create_s": create_s,
           "first8": {"sequential_s": seq_s, "fused_s": fused_s, "thread_pool_s": pool_s,
                      "speedup_fused": seq_s / fused_s},
           "whole_batch_thread_pool": whole_pool,
           "config": {"workload": f"{args.batch} independent nonconvex QPs: n lognormal (median {args.batch_median:g}, "
                                  f"log-std {args.batch_sigma:g}) clipped to [1e3, 1e5]; "
                                  + ("half small generator (m = n/2), half Motzkin-Straus G(n, 0.01)"
                                     if args.batch_mix == "alternate" else "small generator (m = n/2)"),
                      "n_total": int(sum(ns)), "n_min": int(min(ns)), "n_max": int(max(ns)),
                      "n_scope": "rank 0 share" if ws > 1 else "whole batch",
                      "form": "fused: one captured graph, one launch per phase over all problems"}}
    for h in hs:
        h.close()
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_solve_times(args):
    """Wall time of pdnqp_solve (FP64 and FP32-bulk, persistent loop, 120 s cap) and, unless
    --no-cpu, of the FP64 oracle (one host core, 300 s cap) to rel-KKT 1e-4 and 1e-6 on the
    n=200 (m=100) and n=50,000 (m=25,000) workloads; every final point is
    judged by the oracle's external KKT test."""
    from oracle import oracle as O
    from paper_2609_19557_gb300 import instances as I
    from paper_2609_19557_gb300 import pdnqp as P
    O.build()
    P.load()
    rows = []
    for name, inst in (("n=200 m=100", I.small_qp(0)), ("n=50000 m=25000", I.mid_qp(0))):
        for eps in (1e-4, 1e-6):
            row = {"workload": name, "eps": eps}
            for prec in (64, 32):
                h = P.create_from_instance(inst, precision=prec)
                P.pdnqp_set_param(h, "time_limit", 120.0)
                t0 = time.perf_counter()
                st = P.pdnqp_solve(h, eps, eps)
                dt = time.perf_counter() - t0
                x, y, r = P.pdnqp_get(h)
                h.close()
                row[f"gpu_fp{prec}"] = {"status": P.STATUS_NAMES[st], "seconds": dt, "outer": r["outer_iters"],
                                        "inner": r["inner_iters"], "kkt_pass": bool(O.kkt_pass(inst, x, y, eps, eps))}
            if not args.no_cpu:
                t0 = time.perf_counter()
                x, y, info = O.solve(inst, eps_abs=eps, eps_rel=eps, time_limit=300.0)
                dt = time.perf_counter() - t0
                row["oracle"] = {"status": info["status_name"], "seconds": dt, "outer": info["outer_iters"],
                                 "inner": info["inner_iters"], "kkt_pass": bool(O.kkt_pass(inst, x, y, eps, eps))}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print(json.dumps({"leg": "solve_times", "cores": 1, "host": host_cpu(), "rows": len(rows)}), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.solve_times and a.impl != "reference":
        run_solve_times(a)
    elif a.batch > 0 and a.impl != "reference":
        run_batch(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_native(a)
