"""Benchmark: PDLP solve of the set-cover LP relaxation to relative KKT <= 1e-4 on GB300.

Workload (one "step" = one whole solve, rows A0-A11 of the hot path: device
setup, scaling, iterations, KKT checks, output): the covering LP with
m = 50,000 >=-rows (b = 1), n = 200,000 columns in [0, 1], each covering 3-10
uniformly chosen rows (1,296,541 nonzeros, all 1), integer costs U[1,100],
seed 2025; synthetic, generated by ``lpgen.set_cover``.  The main arm runs the
float32 path (matrix stored as a bare pattern, every value being 1), next to
the plain float64 path on the same instance.

Printed: one JSON line (rank 0).  ``value`` = accepted PDHG iterations per
second over the whole job (all ranks), ``ms_per_step`` = time to tolerance.
With N > 1 processes (torchrun) every rank solves its own replica: a single LP
does not shard without an exchange per half step, so this is replicas only.

``--impl reference`` times the float64 CPU oracle (the reference arm) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to rel. KKT≤1e-4 and PDHG iters/s vs plain FP64 PDLP, 1×GB300"
UNIT = "PDHG iters/s"
WORKLOAD = "set_cover m=50000 n=200000 nnz=1296541 seed=2025 tol=1e-4"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave out the energy, batch and 200 x 400 workloads of the default line")
    ap.add_argument("--cpu-sample-iters", type=int, default=400)
    ap.add_argument("--kernels-only", action="store_true",
                    help="only time the fused kernels (pdlp_time_kernels) and print them")
    ap.add_argument("--reps", type=int, default=200)
    ap.add_argument("--workload", default="set_cover",
                    choices=["set_cover", "batch", "energy", "fp", "c1", "variants", "warmstart"],
                    help="batch: 256 uneven covering sub-LPs (m in [2000, 40000], n = 4m, "
                         "10-50 %% of the columns fixed), solved together by pdlp_solve_batch; "
                         "c1 (with --kernels-only): the 200 x 400 MIP relaxation")
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--persistent", type=int, default=0, choices=[0, 1, 2],
                    help="1: one cooperative step kernel per check period; 2: one block per check "
                         "period (the LP in shared memory when it fits); 0: two launches per attempt")
    ap.add_argument("--tiles", type=int, default=0, choices=[0, 1, 2],
                    help="float32 steps: 0 lanes-per-row kernels; 1 staged block tiles (bulk "
                         "copies into shared memory); 2 warp tiles")
    ap.add_argument("--halpern", type=int, default=0, choices=[0, 1],
                    help="1: the reflected restarted Halpern PDHG variant (single LPs)")
    ap.add_argument("--restart-metric", type=int, default=0, choices=[0, 1],
                    help="1: normalized-duality-gap restarts (single LPs)")
    for k in ("lanes-a", "lanes-at", "lanes-kkt-a", "lanes-kkt-at"):
        ap.add_argument("--" + k, type=int, default=0, help="SpMV lanes per row (0 = automatic)")
    return ap.parse_args()


def lane_params(args) -> dict:
    return {"lanes_A": args.lanes_a, "lanes_AT": args.lanes_at, "lanes_kkt_A": args.lanes_kkt_a,
            "lanes_kkt_AT": args.lanes_kkt_at, "persistent": args.persistent, "tiles": args.tiles,
            "halpern": args.halpern, "restart_metric": args.restart_metric}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def combine_ranks(total_s: float, iters: int, ws: int, device="cpu"):
    """Whole-job figures of a replicas-only run: the timed region's MAX over the
    ranks and the accepted iterations SUMMED over them (one all-reduce each; the
    process group is the caller's).  With one rank, the rank's own figures."""
    if ws == 1:
        return total_s, float(iters)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_s, float(iters)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def shard_by_nnz(sizes, ws: int):
    """Split independent LPs across ranks by a greedy balance of their nonzeros:
    largest first, each onto the least loaded rank (ties: the lower rank).  Every
    rank computes the same split from the sizes alone, so no exchange is needed.
    Returns one sorted index list per rank."""
    load = [0] * ws
    parts = [[] for _ in range(ws)]
    for i in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(ws), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += sizes[i]
    return [sorted(p) for p in parts]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in self.out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows]
        mx = [float(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(rows),
                "reasons": reasons}


def ncu_traffic(kernel: str, precision: str, workload: str = "set_cover"):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu capture, if
    one exists for this kernel version and precision (profiles/dram_traffic.txt), else
    None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if (len(f) == 4 and not line.startswith("#") and f[0] == workload and f[1] == kernel
                and f[2] == precision):
            return float(f[3])
    return None


# ------------------------------------------------------------------ CPU oracle
CPU_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import lpgen
from oracle import pdlp_oracle as O
lp = lpgen.set_cover(2025)
start_at = {start_at!r}
while start_at is not None and time.time() < start_at:  # replicas start together
    time.sleep(0.001)
w0 = time.time()
t = time.perf_counter()
r = O.solve(lp, O.Params(iter_limit={iters}, terminate={terminate}, check_period=64, tol=1e-4))
dt = time.perf_counter() - t
print(json.dumps({{"iters": r.iters, "seconds": dt, "status": r.status, "rel_kkt": r.kkt.rel_kkt,
                  "wall0": w0, "wall1": time.time()}}))
"""


CPU_WORKLOAD_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import lpgen
from oracle import pdlp_oracle as O
lps = {maker}
setup = total = 0.0
its = 0
for lp in lps:
    t = time.perf_counter()
    O.solve(lp, O.Params(iter_limit=0, terminate=False))
    setup += time.perf_counter() - t
    t = time.perf_counter()
    r = O.solve(lp, O.Params(iter_limit={iters}, terminate=False))
    total += time.perf_counter() - t
    its += r.iters
print(json.dumps({{"iters": its, "setup_s": setup, "total_s": total, "lps": len(lps)}}))
"""


def cpu_oracle_workload(maker: str, iters: int, what: str) -> dict:
    """The float64 oracle, as it stands, on a bounded sample of another workload, one core:
    each LP of `maker` solved once with no iteration (its setup: canonical form, scaling,
    the check at the start) and once for `iters` iterations; iterations per second of the
    difference."""
    code = CPU_WORKLOAD_SNIPPET.format(root=ROOT, maker=maker, iters=iters)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         env=_oracle_env(), check=True)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    run_s = d["total_s"] - d["setup_s"]
    return {"value": d["iters"] / run_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "setup_s": d["setup_s"] / d["lps"],
            "sample": f"{iters} iterations of the float64 oracle on {what} "
                      f"({d['iters']} in all, {run_s:.1f} s after {d['setup_s']:.1f} s of setup)"}


def _oracle_env():
    return dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def cpu_oracle_sample(iters: int) -> dict:
    """The float64 oracle, as it stands, on the full workload for a bounded number of
    iterations, single-threaded (numpy/scipy with one BLAS thread)."""
    code = CPU_SNIPPET.format(root=ROOT, iters=iters, terminate=False, start_at=None)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         env=_oracle_env(), check=True)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{d['iters']} accepted iterations of the float64 oracle (scaling included) "
                      f"on the full workload, {d['seconds']:.1f} s"}


def cpu_oracle_to_tolerance() -> dict:
    """The float64 oracle, as it stands, solving the full workload to rel. KKT 1e-4 on one
    core: its iterations per second and its time to tolerance (scaling included)."""
    code = CPU_SNIPPET.format(root=ROOT, iters=100_000, terminate=True, start_at=None)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                         env=_oracle_env(), check=True)
    d = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": d["iters"] / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
            "time_to_tol_s": d["seconds"], "iters": d["iters"], "status": d["status"],
            "rel_kkt": d["rel_kkt"],
            "sample": f"one solve of the full workload to rel. KKT 1e-4 by the float64 oracle "
                      f"(scaling included): {d['iters']} iterations in {d['seconds']:.1f} s"}


def cpu_oracle_all_cores(iters: int, procs: int | None = None) -> dict:
    """The same oracle sample in one single-threaded process per host core, started
    together (each builds the LP, then waits for a common wall-clock start): the host's
    aggregate oracle throughput = all accepted iterations / (latest end - earliest start)."""
    if procs is None:  # the cores this process may run on, at most 32 replicas
        procs = min(32, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                    else (os.cpu_count() or 1))
    start_at = time.time() + 8.0 + 0.05 * procs  # time for the imports and the LP build
    code = CPU_SNIPPET.format(root=ROOT, iters=iters, terminate=False, start_at=start_at)
    runs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                             stderr=subprocess.PIPE, text=True, env=_oracle_env()) for _ in range(procs)]
    outs = []
    for r in runs:
        out, err = r.communicate()
        if r.returncode != 0:
            raise RuntimeError(f"oracle replica failed: {err.strip()[-200:]}")
        outs.append(json.loads(out.strip().splitlines()[-1]))
    t0 = min(d["wall0"] for d in outs)
    t1 = max(d["wall1"] for d in outs)
    late = max(d["wall0"] for d in outs) - t0
    rate = sum(d["iters"] for d in outs) / (t1 - t0)
    return {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{procs} single-threaded replicas started together, {iters} accepted "
                      f"iterations each on the full workload; all iterations / "
                      f"(latest end - earliest start) = {t1 - t0:.1f} s "
                      f"(starts spread over {late:.2f} s)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        s = cpu_oracle_sample(args.cpu_sample_iters)
        if i >= args.warmup:
            steps.append(s)
    it_s = statistics.mean(s["value"] for s in steps)
    line = {"impl": "reference", "metric": METRIC, "value": it_s, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * args.cpu_sample_iters / it_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64 oracle (numpy/scipy)",
                       "sample": f"{args.cpu_sample_iters} iterations per step"},
            "cpu_baseline": {"value": it_s, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": steps[-1]["sample"]},
            "e2e": {"value": it_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    lp = lpgen.set_cover(2025)
    d = P.DeviceLP(lp, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    def timed_solves(prm, steps, warmup):
        wsz = P.workspace_size(lp.m, lp.n, lp.nnz, prm)
        wbuf = torch.empty(wsz + 256, dtype=torch.uint8, device=dev)
        xo = torch.empty(lp.n, dtype=torch.float64, device=dev)
        yo = torch.empty(lp.m, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            P.pdlp_solve_device(d, prm, x_out=xo, y_out=yo, workspace=wbuf, stream=stream)
        ms, iters, launches, res = [], 0, 0, None
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        barrier()
        for k in range(steps):
            flush.fill_(float(k))  # L2 flush between timed solves, outside the events
            ev[k][0].record(stream)
            _, _, res = P.pdlp_solve_device(d, prm, x_out=xo, y_out=yo, workspace=wbuf, stream=stream)
            ev[k][1].record(stream)
            iters += res["iters"]
            launches += res["kernel_launches"]
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, iters, launches, res, (xo, yo)

    prm = P.default_params(tol=1e-4, precision=args.precision, **lane_params(args))
    with ClockSampler(dev.index) as clk:
        ms, iters, launches, res, (xo, yo) = timed_solves(prm, args.steps, args.warmup)
    clocks = clk.summary()
    total_s = sum(ms) / 1e3
    # max over ranks of the timed region, units summed over ranks
    total_s, all_iters = combine_ranks(total_s, iters, ws, dev)
    value = all_iters / total_s

    # plain float64 PDLP on the same instance (the comparison line)
    ms64, it64, l64, res64, _ = timed_solves(P.default_params(tol=1e-4, precision="fp64"),
                                             max(1, min(args.steps, 3)), 1)
    # end to end through the host C ABI: host buffers, copies inside the timed region
    e2e_t, e2e_it = 0.0, 0
    for k in range(args.steps + 1):
        t0 = time.perf_counter()
        _, _, r = P.pdlp_solve(lp, prm)
        dt = time.perf_counter() - t0
        if k > 0:  # first call warms the host path
            e2e_t += dt
            e2e_it += r["iters"]
    e2e_t, e2e_it = combine_ranks(e2e_t, e2e_it, ws, dev)
    h2d = 8 * (lp.m + 1) + 12 * lp.nnz + 9 * lp.m + 24 * lp.n
    d2h = 8 * (lp.n + lp.m)
    # roofline of the dominant kernel, timed live with CUDA events on this stream
    kt = P.time_kernels(d, prm, reps=200, stream=stream)
    import json as _j
    peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    # the persistent kernel (persistent = 1, not the default) runs every step attempt of a
    # check period in one launch; the two-launch form times its primal and dual kernels apart
    if prm.persistent and kt["persistent_attempt"]["ms"] > 0:
        dom = "persistent_attempt"
    else:
        dom = max(("primal_step", "dual_step"), key=lambda k: kt[k]["ms"])
    ach = kt[dom]["bytes"] / (kt[dom]["ms"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "traffic": ncu_traffic(dom, args.precision),
            "peak_source": "measured" if peaks else "fallback",
            "kernels": {k: {"us": 1e3 * v["ms"], "bytes": v["bytes"],
                            "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
                        for k, v in kt.items() if v["ms"] > 0}}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_oracle_to_tolerance()
        except Exception as e:  # reported, never silently replaced
            cpu = {"error": str(e)[:200]}
        try:
            cpu["all_cores"] = cpu_oracle_all_cores(args.cpu_sample_iters)
        except Exception as e:
            cpu["all_cores"] = {"error": str(e)[:200]}
    extra = {}
    if rank == 0 and ws == 1 and not args.no_extra:
        # the other workloads, one GPU each (replicas only under torchrun: rank 0 alone)
        for key, fn in (("c1", c1_section), ("energy", energy_section), ("batch", batch_section),
                        ("c5", c5_section)):
            try:
                extra[key] = fn(args, dev, stream, peak)
            except Exception as e:  # reported, never silently replaced
                extra[key] = {"error": str(e)[:300]}
        if not args.no_cpu_baseline:
            # the oracle beside the two workloads that stream from HBM, on bounded samples
            for key, maker, iters, what in (
                    ("energy", "[lpgen.energy_system()]", 16, "the energy system"),
                    ("batch", "lpgen.set_cover_batch(count=8)", 64,
                     "each of the first 8 sub-LPs of the batch")):
                if key in extra and "error" not in extra[key]:
                    try:
                        extra[key]["cpu_baseline"] = cpu_oracle_workload(maker, iters, what)
                    except Exception as e:
                        extra[key]["cpu_baseline"] = {"error": str(e)[:200]}
    if rank == 0:
        prec_used = {0: "fp64", 1: "fp32", 2: "fp32 iterates, bf16 matrix",
                     3: "fp32 iterates, pattern matrix"}[res["precision_used"]]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": prec_used, "l2_flush": True,
                       "parallelism": f"replicas{ws}" if ws > 1 else "single",
                       "lanes": lane_params(args)},
            "time_to_tol_s": total_s / args.steps,
            "iters_per_solve": iters / args.steps,
            "setup_ms": 1e3 * res["setup_s"], "iteration_phase_ms": 1e3 * res["solve_s"],
            "status": res["status"], "rel_kkt": res["rel_kkt"], "primal_obj": res["primal_obj"],
            "fp64_baseline": {"time_to_tol_s": sum(ms64) / 1e3 / len(ms64),
                              "iters_per_s": it64 / (sum(ms64) / 1e3),
                              "iters_per_solve": it64 / len(ms64), "rel_kkt": res64["rel_kkt"],
                              "primal_obj": res64["primal_obj"]},
            "speedup_vs_fp64_time_to_tol": (sum(ms64) / len(ms64)) / (sum(ms) / len(ms)),
            "e2e": {"value": e2e_it / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------ other workloads
def kernel_roofline(kt, peak, peak_source, workload=None, precision=None):
    """Roofline of the step kernels from pdlp_time_kernels: the dominant of the primal
    step and the dual half-step, with every timed kernel's bytes, time and GB/s; the
    dominant kernel's DRAM bytes per launch from the committed ncu capture of `workload`
    (None where there is none)."""
    kern = {k: {"us": 1e3 * v["ms"], "bytes": v["bytes"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                "frac": v["bytes"] / (v["ms"] * 1e-3) / 1e9 / peak}
            for k, v in kt.items() if v["ms"] > 0}
    dom = max(("primal_step", "dual_step"), key=lambda k: kt[k]["ms"])
    traffic = ncu_traffic(dom, precision, workload) if workload else None
    return {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
            "frac": kern[dom]["frac"], "traffic": traffic, "peak_source": peak_source, "kernels": kern}


def _peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path))["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def energy_section(args, dev, stream, peak):
    """The energy-system LP (8760 h x 20 regions x 6 technologies: 2.10M rows, 2.45M
    columns, 7.88M nonzeros, coefficients in [0.1, 10]) to rel. KKT 1e-4 with float32
    iterates, next to plain float64 PDLP on the same instance; inputs resident, CUDA
    events on the stream; its step data (~0.3 GB per attempt) streams from HBM."""
    import torch

    import lpgen
    import paper_2503_10344_gb300 as P

    lp = lpgen.energy_system()
    d = P.DeviceLP(lp, device=dev)

    def solves(prm, steps, warmup):
        wbuf = torch.empty(P.workspace_size(lp.m, lp.n, lp.nnz, prm) + 256, dtype=torch.uint8,
                           device=dev)
        for _ in range(warmup):
            P.pdlp_solve_device(d, prm, workspace=wbuf, stream=stream)
        ms, res = [], None
        for _ in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            a.record(stream)
            _, _, res = P.pdlp_solve_device(d, prm, workspace=wbuf, stream=stream)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(b))
        return statistics.median(ms), res

    prm = P.default_params(tol=1e-4, precision="fp32", iter_limit=200_000, tiles=args.tiles)
    with ClockSampler(dev.index) as clk:
        ms, res = solves(prm, 2, 1)
    ms64, res64 = solves(P.default_params(tol=1e-4, precision="fp64", iter_limit=200_000), 1, 0)
    # the bound-objective rescaling variant on the same instance (not the default iteration)
    msr, resr = solves(P.default_params(tol=1e-4, precision="fp32", iter_limit=200_000,
                                        bound_objective_rescaling=1), 1, 0)
    kt = P.time_kernels(d, prm, reps=50, stream=stream)
    pk, src = _peak()
    obj64 = res64["primal_obj"]
    return {"workload": f"energy system 8760 h x 20 regions x 6 technologies, m={lp.m}, n={lp.n}, "
                        f"nnz={lp.nnz}, tol=1e-4",
            "precision": "fp32 iterates, fp32 matrix, fp64 KKT", "tiles": res["tiles"],
            "time_to_tol_s": ms / 1e3, "iters": res["iters"], "iters_per_s": res["iters"] / (ms / 1e3),
            "status": res["status"], "rel_kkt": res["rel_kkt"], "primal_obj": res["primal_obj"],
            "setup_ms": 1e3 * res["setup_s"],
            "fp64": {"time_to_tol_s": ms64 / 1e3, "iters": res64["iters"],
                     "iters_per_s": res64["iters"] / (ms64 / 1e3), "status": res64["status"],
                     "rel_kkt": res64["rel_kkt"], "primal_obj": obj64},
            "obj_rel_diff_vs_fp64": abs(res["primal_obj"] - obj64) / (1.0 + abs(obj64)),
            "speedup_vs_fp64_time_to_tol": ms64 / ms,
            "bound_objective_rescaling": {"time_to_tol_s": msr / 1e3, "iters": resr["iters"],
                                          "status": resr["status"], "rel_kkt": resr["rel_kkt"],
                                          "primal_obj": resr["primal_obj"]},
            "roofline": kernel_roofline(kt, pk, src, "energy", "fp32"), "clocks": clk.summary()}


def _batch_lps(count):
    """lpgen.set_cover_batch(count), generated by one process per core (spawned)."""
    import multiprocessing as mp

    import lpgen
    seeds = list(range(4000, 4000 + count))
    ms = [int(np.random.default_rng(s).integers(2000, 40001)) for s in seeds]
    procs = max(1, min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                       else (os.cpu_count() or 1)))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.starmap(lpgen.set_cover_fixed, zip(seeds, ms), chunksize=4)


def batch_section(args, dev, stream, peak):
    """The batch of 256 uneven covering sub-LPs (m ~ U[2,000, 40,000], n = 4m, 10-50 % of
    the columns fixed to 0/1; 142M nonzeros) to rel. KKT 1e-4 per LP by pdlp_solve_batch
    from host buffers: setup and iteration phase timed apart by the library."""
    import torch

    import paper_2503_10344_gb300 as P

    lps = _batch_lps(args.batch_count)
    prm = P.default_params(tol=1e-4, precision="bf16", tiles=args.tiles)
    P.pdlp_solve_batch(lps, prm, want_y=False)  # warm
    walls, setup, solve, iters = [], [], [], []
    with ClockSampler(dev.index) as clk:
        for _ in range(2):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, _, res = P.pdlp_solve_batch(lps, prm, want_y=False)
            walls.append(time.perf_counter() - t0)
            setup.append(res[0]["setup_s"])
            solve.append(res[0]["solve_s"])
            iters.append(sum(r["iters"] for r in res))
    it = np.array([r["iters"] for r in res])
    # the same batch with one cooperative kernel per check period (persistent = 1)
    prm1 = P.default_params(tol=1e-4, precision="bf16", persistent=1)
    P.pdlp_solve_batch(lps, prm1, want_y=False)  # warm
    _, _, res1 = P.pdlp_solve_batch(lps, prm1, want_y=False)
    kt = P.time_kernels_batch(lps, prm, reps=20)
    pk, src = _peak()
    persistent = {"solve_s": res1[0]["solve_s"], "iters_sum": int(sum(r["iters"] for r in res1)),
                  "optimal": int(sum(r["status"] == P.PDLP_OPTIMAL for r in res1)),
                  "kernel_launches": int(res1[0]["kernel_launches"]),
                  "kernel_launches_two_launch_form": int(res[0]["kernel_launches"])}
    # the launch shapes picked by the autotuner (timed step attempts, cached per shape) instead
    # of the size heuristic
    prma = P.default_params(tol=1e-4, precision="bf16", autotune=1)
    P.pdlp_solve_batch(lps, prma, want_y=False)  # tunes and caches
    _, _, resa = P.pdlp_solve_batch(lps, prma, want_y=False)
    autotuned = {"solve_s": resa[0]["solve_s"], "iters_sum": int(sum(r["iters"] for r in resa)),
                 "optimal": int(sum(r["status"] == P.PDLP_OPTIMAL for r in resa)),
                 "lanes_A": int(resa[0]["lanes_A"]), "lanes_AT": int(resa[0]["lanes_AT"]),
                 "heuristic_lanes": [int(res[0]["lanes_A"]), int(res[0]["lanes_AT"])]}
    return {"workload": f"batch of {len(lps)} set-cover sub-LPs, sum m={sum(l.m for l in lps)}, "
                        f"sum n={sum(l.n for l in lps)}, nnz={sum(l.nnz for l in lps)}, tol=1e-4",
            "precision": {0: "fp64", 1: "fp32", 2: "fp32 iterates, bf16 matrix",
                          3: "fp32 iterates, pattern matrix"}[res[0]["precision_used"]],
            "tiles": res[0]["tiles"], "optimal": int(sum(r["status"] == P.PDLP_OPTIMAL for r in res)),
            "wall_s": statistics.median(walls), "upload_s": res[0]["upload_s"],
            "setup_s": statistics.median(setup),
            "solve_s": statistics.median(solve), "iters_sum": iters[-1],
            "iters_per_s": iters[-1] / solve[-1], "lps_per_s": len(lps) / statistics.median(solve),
            "iters_per_lp": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max())},
            "persistent": persistent, "autotuned": autotuned,
            "roofline": kernel_roofline(kt, pk, src), "clocks": clk.summary()}


def c5_section(args, dev, stream, peak, train=160, test=20, mmin=5_000, mmax=20_000,
               epochs=12):
    """The learned warm start at a reduced scale (the full one: ``--workload warmstart``):
    covering LPs with m ~ U[mmin, mmax], n = 4m; float64 PDLP labels at 1e-6, the network
    trained on the GPU, then every held-out LP solved cold and warm to 1e-4 (bfloat16 /
    pattern iterates); iterations and times (geometric means), fallback rate."""
    from paper_2503_10344_gb300 import warmstart as W
    res = W.run(train, test, mmin, mmax, epochs, 4, 1e-3, log=lambda *a: None)
    s = res["summary"]
    return {"workload": f"learned warm start: {train} training + {test} held-out covering LPs, "
                        f"m ~ U[{mmin}, {mmax}], n = 4m, {epochs} epochs (reduced scale)",
            "generate_s": res["generate_s"], "label_s": res["label_s"], "train_s": res["train_s"],
            "loss_first": res["loss_first"], "loss_last": res["loss_last"], **s}


def c1_section(args, dev, stream, peak):
    """The 200 x 400 MIP relaxation (seeds 1..20): float64 PDLP to rel. KKT 1e-4 and to
    1e-8 through the host API (latency of a small LP: setup, iterations, copies), with
    the two-launch step kernels and with the one-block persistent kernel
    (persistent = 2), then fix-and-propagate (Frac order) from the 1e-4 point with its
    final LP at 1e-8."""
    import lpgen
    import paper_2503_10344_gb300 as P

    out = {"workload": "mip_relaxation m=200 n=400 seeds 1..20 (float64)"}
    lps = [lpgen.mip_relaxation(seed) for seed in range(1, 21)]
    for persistent in (0, 2):
        P.pdlp_solve(lps[0], P.default_params(tol=1e-4, persistent=persistent))  # warm
        rows = []
        for lp in lps:
            row = {}
            for tol in (1e-4, 1e-8):
                t0 = time.perf_counter()
                x, y, r = P.pdlp_solve(lp, P.default_params(tol=tol, persistent=persistent))
                row[tol] = {"wall_s": time.perf_counter() - t0, "solve_s": r["solve_s"],
                            "iters": r["iters"], "ok": r["status"] == P.PDLP_OPTIMAL,
                            "obj": r["primal_obj"], "x": x, "y": y}
            rows.append(row)
        med = lambda key, tol: float(np.median([r[tol][key] for r in rows]))
        out[f"persistent{persistent}"] = {
            "time_to_1e-4_s": {"median_wall": med("wall_s", 1e-4), "median_solve": med("solve_s", 1e-4)},
            "time_to_1e-8_s": {"median_wall": med("wall_s", 1e-8), "median_solve": med("solve_s", 1e-8)},
            "iters_1e-4_median": med("iters", 1e-4), "iters_1e-8_median": med("iters", 1e-8),
            "optimal": int(sum(r[t]["ok"] for r in rows for t in (1e-4, 1e-8)))}
    fp = []
    for lp, row in zip(lps, rows):
        t0 = time.perf_counter()
        _, f = P.fp_run(lp, row[1e-4]["x"], row[1e-4]["y"], strategy="frac", final_lp=True,
                        final_lp_tol=1e-8)
        fp.append((time.perf_counter() - t0, f, row[1e-8]["obj"]))
    feas = [(w, f, o) for w, f, o in fp if f["status"] == P.FP_FEASIBLE]
    out["fp_run"] = {"feasible": len(feas), "median_wall_s": float(np.median([w for w, _, _ in fp])),
                     "median_gap_to_lp": float(np.median([(f["obj"] - o) / max(1.0, abs(f["obj"]))
                                                          for _, f, o in feas])) if feas else None}
    return out


def run_kernels_only(args):
    import torch

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    if args.workload == "batch":
        kt = P.time_kernels_batch(lpgen.set_cover_batch(args.batch_count),
                                  P.default_params(tol=1e-4, precision=args.precision,
                                                   **lane_params(args)), reps=args.reps)
    else:
        if args.workload == "energy":
            lp = lpgen.energy_system()
            prec = "fp32" if args.precision == "bf16" else args.precision
        elif args.workload == "c1":
            lp = lpgen.mip_relaxation(1)  # the 200 x 400 relaxation, float64 unless asked
            prec = "fp64" if args.precision == "bf16" else args.precision
        else:
            lp = lpgen.set_cover(2025)
            prec = args.precision
        d = P.DeviceLP(lp)
        kt = P.time_kernels(d, P.default_params(tol=1e-4, precision=prec, **lane_params(args)),
                            reps=args.reps)
    torch.cuda.synchronize()
    print(json.dumps({k: {"us": 1e3 * v["ms"], "bytes": v["bytes"],
                          "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9}
                      for k, v in kt.items() if v["ms"] > 0}))


def run_batch(args):
    """All LPs of the batch to rel. KKT 1e-4 by pdlp_solve_batch (host buffers: the
    call uploads, sets up, solves and downloads; setup and solve are timed apart).
    With N > 1 processes the LPs are independent problems: each rank solves the
    share ``shard_by_nnz`` gives it (no data-path collective), the timed region is
    the slowest rank's and the iterations are summed over the ranks; the total work
    is the one batch, so the scaling is strong."""
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    every = lpgen.set_cover_batch(args.batch_count)
    if len(every) < ws:
        raise SystemExit(f"a batch of {len(every)} LPs cannot be shared by {ws} ranks")
    mine = shard_by_nnz([l.nnz for l in every], ws)[rank]
    lps = [every[i] for i in mine]

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()

    prm = P.default_params(tol=1e-4, precision=args.precision, **lane_params(args))
    for _ in range(args.warmup):
        P.pdlp_solve_batch(lps, prm, want_y=False)
    times, setup, solve, iters, launches = [], [], [], [], 0
    with ClockSampler(dev.index) as clk:
        barrier()
        for _ in range(args.steps):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            _, _, res = P.pdlp_solve_batch(lps, prm, want_y=False)
            times.append(time.perf_counter() - t0)
            setup.append(res[0]["setup_s"])
            solve.append(res[0]["solve_s"])
            iters.append(sum(r["iters"] for r in res))
            launches += res[0]["kernel_launches"]
        barrier()
    solve_s, all_iters = combine_ranks(sum(solve), sum(iters), ws, dev)
    wall_s, all_launches = combine_ranks(sum(times), launches, ws, dev)
    its = [r["iters"] for r in res]
    ok = sum(r["status"] == P.PDLP_OPTIMAL for r in res)
    if ws > 1:  # the results' gather, outside the timed region
        got = [None] * ws
        torch.distributed.all_gather_object(got, (ok, its))
        ok, its = sum(g[0] for g in got), [i for g in got for i in g[1]]
    it = np.array(its)
    # roofline of the step kernels over this rank's batch, every LP live (HBM: ~3 GB per
    # attempt for the whole batch)
    kt = P.time_kernels_batch(lps, prm, reps=20)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    kern = {k: {"us": 1e3 * v["ms"], "bytes": v["bytes"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                "frac": v["bytes"] / (v["ms"] * 1e-3) / 1e9 / peak}
            for k, v in kt.items() if v["ms"] > 0}
    dom = max(("primal_step", "dual_step"), key=lambda k: kt[k]["ms"])
    if rank == 0:
        line = {"metric": METRIC, "value": all_iters / solve_s, "unit": UNIT + " (sum over the batch)",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * wall_s / args.steps, "higher_is_better": True,
                "scaling": "strong" if ws > 1 else "weak",
                "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": f"batch of {len(every)} set-cover sub-LPs, "
                                       f"sum m={sum(l.m for l in every)}, sum n={sum(l.n for l in every)}, "
                                       f"nnz={sum(l.nnz for l in every)}, tol=1e-4",
                           "precision": args.precision,
                           "parallelism": f"lps sharded by nnz over {ws} ranks" if ws > 1 else "single"},
                "solve_s": solve_s / args.steps, "setup_s": sum(setup) / args.steps,
                "lps_per_s": len(every) / (solve_s / args.steps), "optimal": ok,
                "iters_per_lp": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max())},
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
                             "unit": "GB/s", "frac": kern[dom]["frac"], "traffic": None,
                             "peak_source": "measured" if peaks else "fallback", "kernels": kern},
                "gpu_launches": int(all_launches), "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_variants(args):
    """The algorithmic variants against the default iteration on the same instances and
    precision modes: bound-objective rescaling (pdlp_params.bound_objective_rescaling), the
    reflected restarted Halpern PDHG (pdlp_params.halpern) and normalized-duality-gap
    restarts (pdlp_params.restart_metric = 1); iterations and
    iteration-phase time to rel. KKT 1e-4 (float32 / pattern on the covering LPs and the
    energy system, float64 on the 200 x 400 relaxations)."""
    import torch

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    cases = [("set_cover m=50000 n=200000", lpgen.set_cover(2025), "bf16"),
             ("set_cover m=5000 n=20000", lpgen.set_cover(3, m=5000, n=20000), "bf16"),
             ("energy_system 720 h", lpgen.energy_system(hours=720), "fp32")]
    cases += [(f"mip_relaxation seed {k}", lpgen.mip_relaxation(k), "fp64") for k in range(1, 6)]
    rows = []
    for name, lp, prec in cases:
        d = P.DeviceLP(lp)
        row = {"instance": name, "precision": prec}
        for key, kw in (("default", {}), ("rescaled", {"bound_objective_rescaling": 1}),
                        ("halpern", {"halpern": 1}), ("ndg_restarts", {"restart_metric": 1})):
            prm = P.default_params(tol=1e-4, precision=prec, iter_limit=200_000, **kw)
            P.pdlp_solve_device(d, prm)  # warm
            torch.cuda.synchronize()
            _, _, r = P.pdlp_solve_device(d, prm)
            row[key] = {
                "status": r["status"], "iters": r["iters"], "restarts": r["restarts"],
                "solve_s": r["solve_s"], "setup_s": r["setup_s"], "rel_kkt": r["rel_kkt"],
                "primal_obj": r["primal_obj"]}
        rows.append(row)
    print(json.dumps({"workload": "bound-objective rescaling, reflected restarted Halpern "
                                  "PDHG and normalized-duality-gap restarts against the default "
                                  "iteration",
                      "tol": 1e-4, "runs": rows}), flush=True)


def run_warmstart(args):
    """The learned warm start at full scale: 2,000 training covering LPs and 100 held-out
    ones, m ~ U[5,000, 50,000], n = 4m, 30 epochs; one JSON line with the summary."""
    import __graft_entry__ as G
    G.build()
    from paper_2503_10344_gb300 import warmstart as W
    res = W.run(2000, 100, 5_000, 50_000, 30, 4, 1e-3, log=lambda *a: None)
    res.pop("per_lp", None)
    res.pop("losses", None)
    print(json.dumps({"workload": "learned warm start, full scale", **res}), flush=True)


def run_energy(args):
    """The energy-system LP (8760 h x 20 regions x 6 technologies, 2.1M rows, 2.45M
    columns, 7.9M nonzeros) to rel. KKT 1e-4 with float32 iterates: the workload whose
    vectors and matrix (~0.3 GB per iteration) are far larger than L2, so the step
    kernels run against HBM."""
    import torch

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    lp = lpgen.energy_system()
    d = P.DeviceLP(lp)
    stream = torch.cuda.current_stream()
    prec = "fp32" if args.precision == "bf16" else args.precision  # coefficients in [0.1, 10]
    prm = P.default_params(tol=1e-4, precision=prec, iter_limit=100_000, **lane_params(args))
    wsz = P.workspace_size(lp.m, lp.n, lp.nnz, prm)
    wbuf = torch.empty(wsz + 256, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        P.pdlp_solve_device(d, prm, workspace=wbuf, stream=stream)
    ms, iters, res = [], 0, None
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            _, _, res = P.pdlp_solve_device(d, prm, workspace=wbuf, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
            iters += res["iters"]
    kt = P.time_kernels(d, prm, reps=50, stream=stream)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    kern = {k: {"us": 1e3 * v["ms"], "bytes": v["bytes"], "gbs": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                "frac": v["bytes"] / (v["ms"] * 1e-3) / 1e9 / peak}
            for k, v in kt.items() if v["ms"] > 0}
    dom = max(("primal_step", "dual_step"), key=lambda k: kt[k]["ms"])
    line = {"metric": METRIC, "value": iters / (sum(ms) / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"energy system 8760h x 20 regions x 6 techs, m={lp.m}, n={lp.n}, "
                                   f"nnz={lp.nnz}, tol=1e-4", "precision": prec,
                       "halpern": args.halpern, "restart_metric": args.restart_metric},
            "time_to_tol_s": sum(ms) / 1e3 / args.steps, "iters_per_solve": iters / args.steps,
            "primal_obj": res["primal_obj"], "restarts": res["restarts"],
            "status": res["status"], "rel_kkt": res["rel_kkt"], "setup_ms": 1e3 * res["setup_s"],
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak,
                         "unit": "GB/s", "frac": kern[dom]["frac"], "traffic": None,
                         "peak_source": "measured" if peaks else "fallback", "kernels": kern},
            "gpu_launches": res["kernel_launches"] * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_fp(args):
    """The paper's heuristic end to end on the covering LP (section 2): the LP relaxation
    by PDLP to 1e-4 on the GPU, fix-and-propagate on the host from its point, the final
    LP with every integer fixed; the time breakdown the paper reports (section 4.1)."""
    import torch

    import __graft_entry__ as G
    G.build()
    import lpgen
    import paper_2503_10344_gb300 as P

    lp = lpgen.set_cover(2025)
    prm = P.default_params(tol=1e-4, precision=args.precision)
    P.pdlp_solve(lp, prm)  # warm: graph capture and library load
    rows = []
    for strat in ("type", "frac", "redcost", "dual", "frac_dual", "frac_redcost", "dual_frac",
                  "redcost_frac"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x_lp, y_lp, r = P.pdlp_solve(lp, prm)
        t_lp = time.perf_counter() - t0
        x, f = P.fp_run(lp, x_lp, y_lp, strategy=strat, final_lp=True, final_lp_tol=1e-8)
        total = t_lp + f["search_s"] + f["lp_s"]
        rows.append({"strategy": strat, "status": f["status"], "obj": f["obj"],
                     "lp_bound": r["dual_obj"], "gap": (f["obj"] - r["dual_obj"]) / abs(f["obj"])
                     if f["status"] == P.FP_FEASIBLE else None,
                     "initial_lp_s": t_lp, "search_s": f["search_s"], "final_lp_s": f["lp_s"],
                     "initial_lp_share": t_lp / total, "nodes": f["nodes"]})
    print(json.dumps({"workload": "fix-and-propagate on set_cover m=50000 n=200000 (all binary)",
                      "precision": args.precision, "runs": rows}), flush=True)


def single_gpu_rank(args) -> bool:
    """The energy, fix-and-propagate and kernel-timing workloads measure one GPU: under a
    multi-process launch rank 0 runs them on its own device and the other ranks leave
    without work.  Returns whether this process runs the workload."""
    ws, rank, local = dist_env()
    if ws == 1:
        return True
    if rank != 0:
        return False
    import torch
    torch.cuda.set_device(local)
    return True


if __name__ == "__main__":
    a = parse()
    if a.impl == "gpu" and (a.kernels_only or a.workload in ("energy", "fp", "variants",
                                                              "warmstart")) \
            and not single_gpu_rank(a):
        sys.exit(0)
    if a.kernels_only and a.impl == "gpu":
        run_kernels_only(a)
    elif a.workload == "fp" and a.impl == "gpu":
        run_fp(a)
    elif a.workload == "energy" and a.impl == "gpu":
        run_energy(a)
    elif a.workload == "batch" and a.impl == "gpu":
        run_batch(a)
    elif a.workload == "variants" and a.impl == "gpu":
        run_variants(a)
    elif a.workload == "warmstart" and a.impl == "gpu":
        run_warmstart(a)
    elif a.workload == "c1" and a.impl == "gpu":
        sys.exit("--workload c1 runs with --kernels-only (its solves are the default line's c1 section)")
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
