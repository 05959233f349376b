#!/usr/bin/env python
"""Benchmark: refactorize + solve throughput of the CUDA path on one GB300.

Workload (default): the post-layout power-grid RC mesh, 200 x 200 x 4 nodes
(n = 160,000, nnz(A) ~ 1.05M), in-layer wires log-normal, vias 10x, 0.5%
random long couplings, 2,000 transistor stamps; ordered by the generator's
geometric nested dissection.  One step = one transient time step: new
transistor transconductances -> checked re-factorization (with restart if a
pivot fails) -> solve with a fresh uniform[-1,1] right-hand side -> device
residual.  Inputs for all steps are generated up front and resident in HBM
before the timed region; the factors (~0.7 GB) are far larger than L2.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the CPU oracle
on the same workload instead (the baseline arm).  With torchrun (N > 1)
every rank runs an independent replica on its own GPU ("replicas only":
one factorization does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the serving workloads run one stream per pattern: give the device as many
# hardware work queues as it has (set before any CUDA context exists), so
# that a short launch is not queued behind a long one of another stream
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from paper_2411_14082_gb300 import inputs  # noqa: E402

FP64_PEAK_TFLOPS = 1.25   # GB300 FP64 rate of the profiling recipe (non-tensor ALU)


def max_over_ranks(value, world, device):
    """The largest value over all ranks (the slowest rank's time); value
    itself on one rank.  device: where the process group's tensors live
    ("cuda:i" under NCCL, "cpu" under gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def unit_bytes(n, nnz_a, nnz_lu):
    """Algorithmic bytes of one refactor + solve: the refactor's compulsory
    bytes (A values and slot map, column pointers, factor values written
    with their row ids) and the solve's (factor values and ids read once,
    permutation and intermediate vectors)."""
    b_rf = nnz_a * 12 + 4 * (n + 1) + nnz_lu * 12 + 4 * nnz_a
    b_sv = 12 * nnz_lu + 16 * (n + 1) + 32 * n
    return b_rf + b_sv


def hbm_roofline(bytes_alg, seconds, traffic=None):
    """% of the HBM roofline: algorithmic (compulsory) bytes per unit over the
    unit's time, against the measured copy bandwidth; and the measured DRAM
    traffic rate when a capture exists."""
    peak, src = hbm_peak_gbs()
    gbs = bytes_alg / seconds / 1e9
    out = {"algorithmic_gbs": gbs, "peak_gbs": peak, "peak_source": src, "frac": gbs / peak,
           "bytes_per_unit": bytes_alg}
    if traffic:
        out["dram_gbs"] = traffic / seconds / 1e9
        out["dram_frac"] = traffic / seconds / 1e9 / peak
    return out
# DRAM bytes (read + write) of one refactorization, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over its launches); valid only
# for the kernel source it was taken on
REFACTOR_TRAFFIC = {
    "rc_mesh_200x200x4/library": {"refactor_cu_sha256": "e68bae915649a44f1500d1c55a4d0193e90295ea8f5eb6f02019de0ad691508c",
                                  "bytes": 19.104e9 + 964.9e6},
}


def refactor_traffic(workload):
    """Per-refactorization DRAM traffic if the capture matches the current kernel, else None."""
    import hashlib
    t = REFACTOR_TRAFFIC.get(workload)
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2411_14082_gb300", "csrc", "refactor.cu")
    if t is None or not os.path.exists(src):
        return None
    with open(src, "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != t["refactor_cu_sha256"]:
            return None
    return t["bytes"]
METRIC = "refactor+solve/s"


# ----------------------------------------------------------------------------- workload
def make_workload(name, n_steps, seed, mesh=(200, 200, 4)):
    if name == "mesh":
        ckt = inputs.workload_mesh(nx=mesh[0], ny=mesh[1], nz=mesh[2])
        desc = f"rc_mesh_{mesh[0]}x{mesh[1]}x{mesh[2]}"
    elif name == "mesh_ill":
        # the same mesh with every conductance log-uniform in [1e-9, 1e4] S
        ckt = inputs.workload_mesh(nx=mesh[0], ny=mesh[1], nz=mesh[2], g_range=(1e-9, 1e4))
        desc = f"rc_mesh_ill_{mesh[0]}x{mesh[1]}x{mesh[2]}"
    elif name == "small":
        ckt = inputs.workload_small()
        desc = "mna_grid_40x50_vsrc20"
    elif name == "batch":
        # bordered-block-diagonal grid with power/ground rails; every step is
        # a batch of value sets (one Monte-Carlo corner each: every entry
        # scaled by exp(N(0, ln 1.2)))
        ckt = inputs.bordered_grid(141, 141, n_rails=50, density=0.05)
        desc = "bordered_grid_141x141_rails50"
    else:
        raise ValueError(name)
    n, Ap, Ai, Ax0 = ckt.csc()
    Q = inputs.grid_nd_order(ckt)
    rng = np.random.default_rng(seed)
    vals, rhs = [], []
    for s in range(n_steps):
        if name in ("mesh", "mesh_ill"):
            ckt = inputs.redraw_transistors(ckt, rng)
            vals.append(ckt.values())
        elif name == "batch":
            vals.append(inputs.scale_values(Ax0, rng, 0.2))
        else:
            ckt = inputs.perturb_elements(ckt, rng)
            vals.append(ckt.values())
        rhs.append(inputs.rhs(n, rng))
    return dict(name=desc, n=n, Ap=Ap, Ai=Ai, Ax0=Ax0, Q=Q, vals=vals, rhs=rhs)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 10:
                continue
            if self.uuid and p[1] != self.uuid:
                continue
            try:
                sm.append(float(p[2]))
                mx.append(float(p[3]))
            except ValueError:
                continue
            for nm, v in zip(names, p[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- CPU oracle
ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import oracle as O
from bench import make_workload
first = {first}
w = make_workload({name!r}, first + {steps}, {seed}, {mesh!r})
out = []
for s in range(first, first + {steps}):
    Ax, b = w["vals"][s], w["rhs"][s]
    t0 = time.perf_counter()
    lu = O.factorize(w["n"], w["Ap"], w["Ai"], Ax, w["Q"], 1e-3)
    x = O.solve(lu, b)
    t1 = time.perf_counter()
    res = O.residual(w["n"], w["Ap"], w["Ai"], Ax, x, b)
    out.append(dict(seconds=t1 - t0, residual=res, status=lu.status, rejected=lu.n_rejected))
    if {xfile!r}:
        np.save({xfile!r}.replace("STEP", str(s)), x)
print("ORACLE_JSON " + json.dumps(out), flush=True)
"""


def start_oracle(name, steps, seed, mesh=(200, 200, 4), first=0, xfile=""):
    """The oracle on value sets first .. first+steps-1 of the workload with
    this seed, in its own process; with xfile, each step's solution is saved
    there (numpy .npy; "STEP" in the name is replaced by the step index)."""
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, steps=steps, seed=seed, mesh=tuple(mesh), first=first,
                                 xfile=xfile)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                            stderr=subprocess.STDOUT, env=env, text=True)


def collect_oracle(proc, timeout=1800):
    try:
        out, _ = proc.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        proc.kill()
        return None
    for line in out.splitlines():
        if line.startswith("ORACLE_JSON "):
            return json.loads(line[len("ORACLE_JSON "):])
    sys.stderr.write(out[-2000:])
    return None


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    # every step is one full oracle unit (the smallest sample of this
    # workload); the count is capped so that the run stays within minutes
    steps = max(1, min(args.steps, 2))
    w_name = args.workload
    proc = start_oracle(w_name, steps, args.seed, args.mesh)
    res = collect_oracle(proc)
    if not res:
        print(json.dumps({"impl": "reference", "unavailable": "CPU oracle run failed"}))
        return 0
    secs = [r["seconds"] for r in res]
    value = len(secs) / sum(secs)
    wl = make_workload(w_name, 0, args.seed, args.mesh)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": 0, "steps": steps, "warmup": 0, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wl["name"], "n": int(wl["n"]),
                                        "nnz_a": int(wl["Ap"][-1])},
        "max_rel_residual": max(r["residual"] for r in res),
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} full refactor+solve unit(s) of the workload, "
                                   "single-threaded C oracle", "host": host_info()},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_batch(args, rank, world, local_rank):
    """Batch workload: every step refactorizes and solves `sets` value sets of
    one pattern through gblu_refactorize_batch / gblu_solve_batch."""
    # CPU throughput baseline: one single-threaded oracle process per host
    # core, each on its own value sets of the same pattern (started before
    # the first CUDA call)
    procs, t_cpu0, units = [], None, 3
    if rank == 0 and not args.no_cpu_baseline:
        t_cpu0 = time.perf_counter()
        procs = [start_oracle("batch", units, args.seed + 5000 + p) for p in range(os.cpu_count() or 1)]
    import torch
    import torch.distributed as dist
    from paper_2411_14082_gb300 import gblu

    dev = local_rank
    torch.cuda.set_device(dev)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{dev}"))
    w = make_workload("batch", args.sets, args.seed + 17 * rank)
    n, nnz = w["n"], int(w["Ap"][-1])
    s = gblu.Solver(dev)
    s.analyze(n, w["Ap"], w["Ai"], w["Q"])
    s.factorize(torch.from_numpy(w["Ax0"]).cuda(dev))
    if args.batch_group >= 0:
        s.set_opts(batch_group=args.batch_group)
    # a set whose check fails in the batch is solved again on a handle of its
    # own (restart with pivoting), inside the step, as the batch API asks
    redo = gblu.Solver(dev)
    redo.analyze(n, w["Ap"], w["Ai"], w["Q"])
    redo.factorize(torch.from_numpy(w["Ax0"]).cuda(dev))
    st = s.stats()
    vals = torch.from_numpy(np.stack(w["vals"])).cuda(dev)
    rhs = torch.from_numpy(np.stack(w["rhs"])).cuda(dev)
    xs = torch.empty_like(rhs)
    LUx = torch.empty((args.sets, st["nnz_l"] + st["nnz_u"]), dtype=torch.float64, device=f"cuda:{dev}")
    stream = torch.cuda.current_stream(dev)
    total = args.warmup + args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(total)]
    nfail = 0
    for i in range(total):
        if i == args.warmup:
            torch.cuda.synchronize(dev)
            if world > 1:
                dist.barrier()
            clocks = ClockSampler()
            clocks.start()
            t0 = time.perf_counter()
        ev[i][0].record(stream)
        if args.graph:
            # refactor + solve of the batch replayed from one CUDA graph
            failed = s.step_batch(vals, LUx, rhs, xs)
            ev[i][1].record(stream)
        else:
            _, failed = s.refactorize_batch(vals, LUx)
            ev[i][1].record(stream)
            s.solve_batch(LUx, rhs, xs)
        for k in np.nonzero(failed)[0]:
            redo.refactorize(vals[int(k)])
            redo.solve(rhs[int(k)], xs[int(k)])
        ev[i][2].record(stream)
        nfail += int(failed.sum())
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    elapsed = time.perf_counter() - t0
    clk = clocks.stop()
    t_rf = [ev[i][0].elapsed_time(ev[i][1]) / 1e3 for i in range(args.warmup, total)]
    t_sv = [ev[i][1].elapsed_time(ev[i][2]) / 1e3 for i in range(args.warmup, total)]
    ev_elapsed = sum(ev[i][0].elapsed_time(ev[i][2]) / 1e3 for i in range(args.warmup, total))
    if world > 1:
        ev_elapsed = max_over_ranks(ev_elapsed, world, f"cuda:{dev}")
    res = torch.zeros(4, dtype=torch.float64, device=f"cuda:{dev}")
    worst = 0.0
    for k in range(args.sets):
        s.residual(vals[k], rhs[k], xs[k], out=res)
        worst = max(worst, float(res[0].item()))
    # the other form (graph replay or eager launches) on the same sets, for context
    other = "eager" if args.graph else "graph_replay"
    alt_steps = min(5, args.steps)
    for i in range(alt_steps + 1):   # the first graph call captures
        if i == 1:
            torch.cuda.synchronize(dev)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
        if args.graph:
            _, failed = s.refactorize_batch(vals, LUx)
            s.solve_batch(LUx, rhs, xs)
        else:
            failed = s.step_batch(vals, LUx, rhs, xs)
        for k in np.nonzero(failed)[0]:
            redo.refactorize(vals[int(k)])
            redo.solve(rhs[int(k)], xs[int(k)])
    a1.record(stream)
    torch.cuda.synchronize(dev)
    alt = {"form": other, "value": args.sets * alt_steps / (a0.elapsed_time(a1) / 1e3), "unit": METRIC,
           "ms_per_step": a0.elapsed_time(a1) / alt_steps}
    # the one-matrix path on the same sets, for context (not the metric)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.sets):
        s.refactorize(vals[k])
        s.solve(rhs[k], xs[k])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    single = args.sets / (e0.elapsed_time(e1) / 1e3)
    F = st["flops"]
    value = world * args.sets * args.steps / ev_elapsed
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * ev_elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"] + f"_x{args.sets}", "n": n, "nnz_a": nnz,
                   "nnz_lu": int(st["nnz_l"] + st["nnz_u"]), "sets_per_step": args.sets,
                   "refactor_gflop_per_set": F / 1e9, "ordering": "geometric nested dissection",
                   "batch_group": s.opts()["batch_group"],
                   "form": "graph replay (gblu_step_batch)" if args.graph else
                           "eager launches (gblu_refactorize_batch + gblu_solve_batch)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "max_rel_residual": worst, "residual_ok": bool(worst <= 1e-12), "failed_sets": nfail,
        "failed_sets_note": "sets whose check failed were re-factorized with pivoting on a second handle "
                            "inside the step (their time is in solve_batch)",
        "phases_ms": {"refactor_batch": 1e3 * float(np.mean(t_rf)), "solve_batch": 1e3 * float(np.mean(t_sv)),
                      "note": "graph replay: refactor_batch = the whole replayed step" if args.graph else None,
                      "wall_per_step": 1e3 * elapsed / args.steps},
        "roofline": {"kernel": "refactor batch (all launches)", "bound": "alu",
                     "achieved": args.sets * F / float(np.mean(t_rf)) / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": args.sets * F / float(np.mean(t_rf)) / 1e12 / FP64_PEAK_TFLOPS,
                     "traffic": None},
        "single_path": {"value": single, "unit": METRIC,
                        "note": "the same sets one at a time through gblu_refactorize + gblu_solve"},
        other: alt,
        "cpu_baseline": None,
        # index bytes once per launch, value bytes once per set
        "hbm_roofline": hbm_roofline(
            (4 * nnz + 4 * (n + 1) + 8 * (st["nnz_l"] + st["nnz_u"]))
            + args.sets * (8 * nnz + 16 * (st["nnz_l"] + st["nnz_u"]) + 16 * (n + 1) + 32 * n),
            ev_elapsed / args.steps),
        "clocks": clk,
    }
    if procs:
        res = [collect_oracle(p) for p in procs]
        wall = time.perf_counter() - t_cpu0
        ok = [r for r in res if r]
        if ok:
            done = sum(len(r) for r in ok)
            line["cpu_baseline"] = {
                "value": done / max(max(sum(u["seconds"] for u in r) for r in ok), 1e-9), "unit": METRIC,
                "cores": len(procs), "kind": "oracle",
                "sample": f"{len(procs)} single-threaded oracle processes, {units} sets each of the same pattern; "
                          "value = sets / the longest process's oracle time",
                "wall_s": wall, "max_rel_residual": max(u["residual"] for r in ok for u in r),
                "host": host_info()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve_poisson(args, rank, world, local_rank):
    """C5-like traffic: independent simulations of different sizes share one
    gblu server.  Requests arrive as a Poisson process (open loop), at rates
    set to fractions of the measured service capacity; half of them ask for
    single-precision factors with refinement.  Latency is the server's own
    submit-to-solution time."""
    import threading
    import torch
    from paper_2411_14082_gb300 import gblu

    dev = local_rank
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(args.seed + 17 * rank)
    V = 2
    specs = []
    for i, nt in enumerate(np.exp(rng.uniform(np.log(5000), np.log(args.serve_max_n), args.sims))):
        if i % 2 == 0:   # C1 generator: 2D MNA grid with voltage sources
            side = max(8, int(round(np.sqrt(nt - 20))))
            specs.append((f"mna_{side}x{side}", inputs.mna_grid2d(side, side, seed=args.seed + 2000 + i), "elements"))
        else:            # C2 generator: 4-layer RC mesh with transistor stamps
            side = max(8, int(round(np.sqrt(nt / 4))))
            specs.append((f"mesh_{side}x{side}x4", inputs.rc_mesh3d(side, side, 4, seed=args.seed + 2000 + i,
                                                                   n_fet=max(10, side * side // 20)), "transistors"))
    if args.serve_big:
        specs.append(("mesh_500x500x4", inputs.rc_mesh3d(500, 500, 4, seed=args.seed + 3000), "transistors"))
    srv = gblu.Server(dev, hbm_budget=args.serve_budget_gb << 30, max_batch=args.serve_max_batch)
    pats, refused = [], []
    t0 = time.perf_counter()
    for name, ckt, kind in specs:
        n, Ap, Ai, Ax0 = ckt.csc()
        Q = inputs.grid_nd_order(ckt)
        try:
            pid, slots = srv.add_pattern(n, Ap, Ai, Q, Ax0)
        except gblu.GbluError as e:   # refused by the memory budget
            refused.append({"pattern": name, "n": n, "error": str(e)})
            continue
        vals, rhs = [], []
        for _ in range(V):
            ckt = inputs.redraw_transistors(ckt, rng) if kind == "transistors" else inputs.perturb_elements(ckt, rng)
            vals.append(torch.from_numpy(ckt.values()).pin_memory().numpy())
            rhs.append(torch.from_numpy(inputs.rhs(n, rng)).pin_memory().numpy())
        pats.append(dict(name=name, n=n, id=pid, slots=slots, vals=vals, rhs=rhs,
                         ubytes=unit_bytes(n, len(Ai), srv.pattern_info(pid)["nnz_lu"])))
    t_admit = time.perf_counter() - t0
    # service time of each pattern and mode alone (after one warm request)
    svc = {}
    for p in pats:
        for mode in (0, 1):
            for rep in range(2):
                _, r = srv.wait(srv.submit(p["id"], p["vals"][0], p["rhs"][0], mixed=bool(mode)), timeout=600.0)
            svc[p["name"], mode] = r["latency_s"]
    tbar = float(np.mean(list(svc.values())))
    sweep = []
    for rho in args.serve_rates:
        lam = rho / tbar
        N = args.serve_requests
        ids, lock = [], threading.Lock()
        st0 = srv.stats()

        def dispatch():
            t_next = time.perf_counter()
            for k in range(N):
                t_next += rng.exponential(1.0 / lam)
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                p = pats[int(rng.integers(0, len(pats)))]
                j = int(rng.integers(0, V))
                mode = k % 2
                rid = srv.submit(p["id"], p["vals"][j], p["rhs"][j], mixed=bool(mode))
                with lock:
                    ids.append((rid, mode, p["name"], p["ubytes"], p["n"]))

        clocks = ClockSampler()
        clocks.start()
        t_start = time.perf_counter()
        th = threading.Thread(target=dispatch)
        th.start()
        res = []
        sizes = []
        moved = [0]
        got = 0
        while got < N:
            with lock:
                pending = ids[got:]
            if not pending:
                time.sleep(0.001)
                continue
            for rid, mode, name, ub, nn in pending:
                _, r = srv.wait(rid, timeout=600.0)
                res.append((mode, name, r))
                sizes.append(nn)
                moved[0] += ub
                got += 1
        th.join()
        elapsed = time.perf_counter() - t_start
        clk = clocks.stop()
        lat = np.array([r["latency_s"] for _, _, r in res])
        by_mode = {}
        for mode in (0, 1):
            a = np.array([r["latency_s"] for m, _, r in res if m == mode])
            by_mode["f64" if mode == 0 else "f32_refined"] = {
                "p50_ms": 1e3 * float(np.percentile(a, 50)), "p99_ms": 1e3 * float(np.percentile(a, 99)),
                "fallbacks": int(sum(1 for m, _, r in res if m == mode and r["refine_iters"] < 0))}
        st1 = srv.stats()
        by_size = {}
        for cls, sel in (("n<=100k", [z <= 100000 for z in sizes]), ("n>100k", [z > 100000 for z in sizes])):
            a = np.array([r["latency_s"] for (m_, nm_, r), keep in zip(res, sel) if keep])
            if len(a):
                by_size[cls] = {"requests": int(len(a)), "p50_ms": 1e3 * float(np.percentile(a, 50)),
                                "p99_ms": 1e3 * float(np.percentile(a, 99))}
        slowest = sorted(res, key=lambda t: -t[2]["latency_s"])[:5]
        slow = [{"pattern": nm, "mode": "f64" if m == 0 else "f32_refined", "latency_ms": 1e3 * r["latency_s"],
                 "queue_ms": 1e3 * r["queue_s"], "refine_iters": r["refine_iters"], "repivoted": r["repivoted"]}
                for m, nm, r in slowest]
        sweep.append({"offered_load": rho, "by_size": by_size, "slowest": slow, "arrival_rate_per_s": lam, "requests": N,
                      "served_per_s": N / elapsed, "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                      "latency_ms_p99": 1e3 * float(np.percentile(lat, 99)), "by_mode": by_mode,
                      "mean_batch": float(np.mean([r["batch_size"] for m, _, r in res if m == 0])),
                      "errors": int(sum(1 for _, _, r in res if r["status"] < 0)),
                      "max_rel_residual": float(max(r["berr"] for _, _, r in res)),
                      "batches": st1["batches"] - st0["batches"], "clocks": clk,
                      "hbm_roofline": hbm_roofline(moved[0], elapsed)})
    st = srv.stats()
    srv.close()
    top = sweep[-1]
    ns = [p["n"] for p in pats]
    line = {
        "metric": "served requests/s", "value": world * top["served_per_s"], "unit": "requests/s",
        "n_gpus": world, "steps": args.serve_requests, "warmup": 2, "ms_per_step": 1e3 / top["served_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 and f32+refinement",
        "data": "synthetic",
        "config": {"workload": f"serve_poisson_{len(pats)}_sims", "patterns": len(pats), "n_min": int(min(ns)),
                   "n_max": int(max(ns)), "n_total": int(sum(ns)), "max_batch": args.serve_max_batch,
                   "hbm_budget_gb": args.serve_budget_gb, "mode_mix": "half f64, half f32 + refinement",
                   "arrivals": "Poisson, open loop; rate = offered load / mean solo service time",
                   "mean_solo_service_ms": 1e3 * tbar, "timing": "host wall clock",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "latency_ms_p50": top["latency_ms_p50"], "latency_ms_p99": top["latency_ms_p99"],
        "hbm_roofline": top["hbm_roofline"],
        "max_rel_residual": max(v["max_rel_residual"] for v in sweep),
        "residual_ok": bool(max(v["max_rel_residual"] for v in sweep) <= 1e-12),
        "sweep": sweep, "server": {k: st[k] for k in ("batches", "repivots", "max_batch_seen", "reserved_bytes")},
        "admission_s": t_admit, "refused_patterns": refused,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_uneven(args, rank, world, local_rank):
    """Uneven-pattern batch: 64 MNA grids with n log-uniform in [1k, 50k];
    every step re-factorizes all of them with new values in one launch
    (gblu_refactorize_multi) and solves each."""
    import torch
    from paper_2411_14082_gb300 import gblu

    dev = local_rank
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(args.seed + 17 * rank)
    V = 4   # value sets per pattern, reused cyclically
    pats = []
    t0 = time.perf_counter()
    for i, nt in enumerate(np.exp(rng.uniform(np.log(1000), np.log(50000), args.patterns))):
        side = max(8, int(round(np.sqrt(nt - 20))))
        ny = max(8, int(round((nt - 20) / side)))
        ckt = inputs.mna_grid2d(side, ny, seed=args.seed + 1000 + i)
        n, Ap, Ai, Ax0 = ckt.csc()
        Q = inputs.grid_nd_order(ckt)
        s = gblu.Solver(dev)
        s.analyze(n, Ap, Ai, Q)
        s.factorize(torch.from_numpy(Ax0).cuda(dev))
        vals, rhs = [], []
        for _ in range(V):
            ckt = inputs.perturb_elements(ckt, rng)
            vals.append(torch.from_numpy(ckt.values()).cuda(dev))
            rhs.append(torch.from_numpy(inputs.rhs(n, rng)).cuda(dev))
        st = s.stats()
        pats.append(dict(s=s, n=n, vals=vals, rhs=rhs, flops=st["flops"],
                         ubytes=unit_bytes(n, len(Ai), st["nnz_l"] + st["nnz_u"]),
                         x=torch.empty(n, dtype=torch.float64,
                                                                                         device=f"cuda:{dev}")))
    t_setup = time.perf_counter() - t0
    solvers = [p["s"] for p in pats]
    stream = torch.cuda.current_stream(dev)
    total = args.warmup + args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(total)]
    reps = 0
    for i in range(total):
        if i == args.warmup:
            torch.cuda.synchronize(dev)
            clocks = ClockSampler()
            clocks.start()
        j = i % V
        ev[i][0].record(stream)
        reps += sum(gblu.refactorize_multi(solvers, [p["vals"][j] for p in pats]))
        ev[i][1].record(stream)
        gblu.solve_multi(solvers, [p["rhs"][j] for p in pats], [p["x"] for p in pats])
        ev[i][2].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    t_rf = [ev[i][0].elapsed_time(ev[i][1]) / 1e3 for i in range(args.warmup, total)]
    t_sv = [ev[i][1].elapsed_time(ev[i][2]) / 1e3 for i in range(args.warmup, total)]
    t_all = sum(ev[i][0].elapsed_time(ev[i][2]) / 1e3 for i in range(args.warmup, total))
    res = torch.zeros(4, dtype=torch.float64, device=f"cuda:{dev}")
    worst = 0.0
    j = (total - 1) % V
    for p in pats:
        p["s"].residual(p["vals"][j], p["rhs"][j], p["x"], out=res)
        worst = max(worst, float(res[0].item()))
    # the same systems one handle at a time, for context (not the metric)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        j = (args.warmup + i) % V
        for p in pats:
            p["s"].refactorize(p["vals"][j])
            p["s"].solve(p["rhs"][j], p["x"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    single = len(pats) * args.steps / (e0.elapsed_time(e1) / 1e3)
    F = sum(p["flops"] for p in pats)
    ns = [p["n"] for p in pats]
    line = {
        "metric": "refactor+solve/s (systems)", "value": world * len(pats) * args.steps / t_all,
        "unit": "systems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"uneven_{len(pats)}_mna_grids", "patterns": len(pats),
                   "n_min": int(min(ns)), "n_max": int(max(ns)), "n_total": int(sum(ns)),
                   "refactor_gflop_per_step": F / 1e9,
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "max_rel_residual": worst, "residual_ok": bool(worst <= 1e-12), "repivots": int(reps),
        "phases_ms": {"refactor_multi": 1e3 * float(np.mean(t_rf)), "solves": 1e3 * float(np.mean(t_sv)),
                      "setup_s": t_setup},
        "roofline": {"kernel": "refactor_multi (one launch, all patterns)", "bound": "alu",
                     "achieved": F / float(np.mean(t_rf)) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": F / float(np.mean(t_rf)) / 1e12 / FP64_PEAK_TFLOPS, "traffic": None},
        "single_path": {"value": single, "unit": "systems/s",
                        "note": "the same systems one handle at a time (gblu_refactorize + gblu_solve)"},
        "hbm_roofline": hbm_roofline(sum(p["ubytes"] for p in pats), t_all / args.steps),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args, rank, world, local_rank):
    """Serving workload: closed-loop clients submit solve requests of three
    circuits to one gblu server (resident patterns, continuous batching per
    pattern, patterns overlapping on the device).  A step is one request per
    client; the metric is completed requests per second (host wall clock)."""
    import threading
    import torch
    from paper_2411_14082_gb300 import gblu

    dev = local_rank
    torch.cuda.set_device(dev)
    V = 8   # distinct value sets per pattern, reused cyclically
    specs = [("rc_mesh_200x200x4", inputs.workload_mesh(), 4, "transistors"),
             ("rc_mesh_120x120x4", inputs.workload_mesh(nx=120, ny=120, nz=4), 8, "transistors"),
             ("mna_grid_40x50_vsrc20", inputs.workload_small(), 16, "elements")]
    rng = np.random.default_rng(args.seed + 17 * rank)
    pats = []
    for name, ckt, clients, kind in specs:
        n, Ap, Ai, Ax0 = ckt.csc()
        Q = inputs.grid_nd_order(ckt)
        vals, rhs = [], []
        for _ in range(V):
            ckt = inputs.redraw_transistors(ckt, rng) if kind == "transistors" else inputs.perturb_elements(ckt, rng)
            vals.append(torch.from_numpy(ckt.values()).pin_memory().numpy())
            rhs.append(torch.from_numpy(inputs.rhs(n, rng)).pin_memory().numpy())
        pats.append(dict(name=name, n=n, Ap=Ap, Ai=Ai, Ax0=Ax0, Q=Q, clients=clients, vals=vals, rhs=rhs))
    srv = gblu.Server(dev, hbm_budget=args.serve_budget_gb << 30, max_batch=args.serve_max_batch)
    t0 = time.perf_counter()
    for p in pats:
        p["id"], p["slots"] = srv.add_pattern(p["n"], p["Ap"], p["Ai"], p["Q"], p["Ax0"])
        info = srv.pattern_info(p["id"])
        p["footprint"] = info["footprint_bytes"]
        p["ubytes"] = unit_bytes(p["n"], len(p["Ai"]), info["nnz_lu"])
    t_admit = time.perf_counter() - t0
    lat = {p["name"]: [] for p in pats}
    bsz = {p["name"]: [] for p in pats}
    worst = [0.0]
    bad = []
    lock = threading.Lock()
    start = threading.Barrier(sum(p["clients"] for p in pats) + 1)

    def client(p, c):
        x = torch.empty(p["n"], dtype=torch.float64).pin_memory().numpy()
        mine, sizes, wb = [], [], 0.0
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                start.wait()
            j = (c + i) % V
            _, r = srv.wait(srv.submit(p["id"], p["vals"][j], p["rhs"][j], x), timeout=600.0)
            if r["status"] < 0:
                bad.append(r["status"])
            if i >= args.warmup:
                mine.append(r["latency_s"])
                sizes.append(r["batch_size"])
                wb = max(wb, r["berr"])
        with lock:
            lat[p["name"]].extend(mine)
            bsz[p["name"]].extend(sizes)
            worst[0] = max(worst[0], wb)

    threads = [threading.Thread(target=client, args=(p, c)) for p in pats for c in range(p["clients"])]
    for t in threads:
        t.start()
    clocks = ClockSampler()
    start.wait()
    clocks.start()
    t0 = time.perf_counter()
    for t in threads:
        t.join()
    elapsed = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    done = sum(len(v) for v in lat.values())
    allv = np.concatenate([np.array(v) for v in lat.values()])
    per = {}
    for p in pats:
        a = np.array(lat[p["name"]])
        per[p["name"]] = {"n": p["n"], "clients": p["clients"], "slots": p["slots"],
                          "footprint_gb": p["footprint"] / 1e9, "requests": len(a),
                          "requests_per_s": len(a) / elapsed,
                          "latency_ms_p50": 1e3 * float(np.percentile(a, 50)),
                          "latency_ms_p99": 1e3 * float(np.percentile(a, 99)),
                          "mean_batch": float(np.mean(bsz[p["name"]]))}
    line = {
        "metric": "served requests/s", "value": world * done / elapsed, "unit": "requests/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "serve_3_circuits", "patterns": [p["name"] for p in pats],
                   "clients": sum(p["clients"] for p in pats), "max_batch": args.serve_max_batch,
                   "hbm_budget_gb": args.serve_budget_gb, "timing": "host wall clock, closed-loop clients",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "latency_ms_p50": 1e3 * float(np.percentile(allv, 50)),
        "latency_ms_p99": 1e3 * float(np.percentile(allv, 99)),
        "per_pattern": per, "max_rel_residual": worst[0], "residual_ok": bool(worst[0] <= 1e-12),
        "hbm_roofline": hbm_roofline(sum(len(lat[p["name"]]) * p["ubytes"] for p in pats), elapsed),
        "errors": len(bad), "server": {k: st[k] for k in ("batches", "repivots", "max_batch_seen",
                                                           "reserved_bytes")},
        "admission_s": t_admit, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def host_info():
    """Host cores and CPU model of the machine the oracle ran on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def forms_section(args, s, w, dev, vals, rhs, stream):
    """The other forms of the method, each timed briefly after the headline
    region with CUDA events (context beside the headline, not the metric):
    the mixed-precision step on the same matrix (single-precision factors
    with refinement in double, C4), a 256-set batch of the bordered grid in
    one persistent launch (C3), and the 2,020-unknown MNA grid one step at a
    time (C1).  Each gives its rate, the refactorization's ALU roofline and
    the unit's share of the HBM roofline, and its largest relative residual."""
    import torch
    from paper_2411_14082_gb300 import gblu
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def roof(F, t, peak):
        return {"achieved_tflops": F / t / 1e12, "peak_tflops": peak, "frac": F / t / 1e12 / peak}

    # mixed precision on the same handle and values (C4)
    st = s.stats()
    n, nnz, nlu = w["n"], int(w["Ap"][-1]), st["nnz_l"] + st["nnz_u"]
    x = torch.empty(n, dtype=torch.float64, device=f"cuda:{dev}")
    k = min(5, len(w["vals"]) - 1)
    for i in range(2):
        s.refactorize_f32(vals[i])
        s.solve_refined(vals[i], rhs[i], x, tol=1e-12)
    torch.cuda.synchronize(dev)
    t_rf, t_all, its, berr = [], 0.0, [], 0.0
    for i in range(k):
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        s.refactorize_f32(vals[i])
        e1.record(stream)
        _, it, be = s.solve_refined(vals[i], rhs[i], x, tol=1e-12)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        its.append(it)
        berr = max(berr, be)
        if it >= 0:
            t_rf.append(e0.elapsed_time(e1) / 1e3)
        t_all += e0.elapsed_time(e2) / 1e3
    F = st["flops"]
    out["mixed_precision"] = {
        "workload": w["name"], "value": k / t_all, "unit": METRIC, "steps": k, "ms_per_step": 1e3 * t_all / k,
        "refine_iters": its, "fallbacks": sum(1 for v in its if v < 0), "max_backward_error": berr,
        "roofline_fp32": roof(F, float(np.mean(t_rf)), 152 * 128 * 2 * 2.07e9 / 1e12) if t_rf else None,
        "hbm_roofline": hbm_roofline(unit_bytes(n, nnz, nlu), t_all / k)}
    # batch of value sets (C3)
    wb = make_workload("batch", args.forms_sets, args.seed + 5)
    nb_, nnzb = wb["n"], int(wb["Ap"][-1])
    hb = gblu.Solver(dev)
    hb.analyze(nb_, wb["Ap"], wb["Ai"], wb["Q"])
    hb.factorize(torch.from_numpy(wb["Ax0"]).cuda(dev))
    redo = gblu.Solver(dev)
    redo.analyze(nb_, wb["Ap"], wb["Ai"], wb["Q"])
    redo.factorize(torch.from_numpy(wb["Ax0"]).cuda(dev))
    stb = hb.stats()
    bv = torch.from_numpy(np.stack(wb["vals"])).cuda(dev)
    bb = torch.from_numpy(np.stack(wb["rhs"])).cuda(dev)
    bx = torch.empty_like(bb)
    LUx = torch.empty((args.forms_sets, stb["nnz_l"] + stb["nnz_u"]), dtype=torch.float64, device=f"cuda:{dev}")
    t_b, t_rfb, nfail = 0.0, [], 0
    for i in range(3):   # the first call warms up
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        _, failed = hb.refactorize_batch(bv, LUx)
        e1.record(stream)
        hb.solve_batch(LUx, bb, bx)
        for j in np.nonzero(failed)[0]:
            redo.refactorize(bv[int(j)])
            redo.solve(bb[int(j)], bx[int(j)])
        e2.record(stream)
        torch.cuda.synchronize(dev)
        if i > 0:
            t_b += e0.elapsed_time(e2) / 1e3
            t_rfb.append(e0.elapsed_time(e1) / 1e3)
            nfail += int(failed.sum())
    res = torch.zeros(4, dtype=torch.float64, device=f"cuda:{dev}")
    worst = 0.0
    for j in range(args.forms_sets):
        hb.residual(bv[j], bb[j], bx[j], out=res)
        worst = max(worst, float(res[0].item()))
    Fb = stb["flops"] * args.forms_sets
    out["batch"] = {
        "workload": wb["name"] + f"_x{args.forms_sets}", "value": 2 * args.forms_sets / t_b, "unit": METRIC,
        "steps": 2, "ms_per_step": 1e3 * t_b / 2, "failed_sets_redone": nfail,
        "roofline_fp64": roof(Fb, float(np.mean(t_rfb)), FP64_PEAK_TFLOPS),
        "hbm_roofline": hbm_roofline((4 * nnzb + 4 * (nb_ + 1) + 8 * (stb["nnz_l"] + stb["nnz_u"]))
                                     + args.forms_sets * (8 * nnzb + 16 * (stb["nnz_l"] + stb["nnz_u"])
                                                          + 16 * (nb_ + 1) + 32 * nb_), t_b / 2),
        "max_rel_residual": worst}
    del hb, redo, bv, bb, bx, LUx
    # the small MNA grid (C1), one refactor + solve at a time
    ws = make_workload("small", 25, args.seed + 7)
    ns, nnzs = ws["n"], int(ws["Ap"][-1])
    hs = gblu.Solver(dev)
    hs.analyze(ns, ws["Ap"], ws["Ai"], ws["Q"])
    hs.factorize(torch.from_numpy(ws["Ax0"]).cuda(dev))
    sv = torch.from_numpy(np.stack(ws["vals"])).cuda(dev)
    sb = torch.from_numpy(np.stack(ws["rhs"])).cuda(dev)
    sx = torch.empty_like(sb)
    for i in range(5):
        hs.refactorize(sv[i])
        hs.solve(sb[i], sx[i])
    torch.cuda.synchronize(dev)
    e0, e1 = ev(), ev()
    e0.record(stream)
    for i in range(5, 25):
        hs.refactorize(sv[i])
        hs.solve(sb[i], sx[i])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_s = e0.elapsed_time(e1) / 1e3
    worst = 0.0
    for i in range(5, 25):
        hs.residual(sv[i], sb[i], sx[i], out=res)
        worst = max(worst, float(res[0].item()))
    sts = hs.stats()
    out["small_mna"] = {
        "workload": ws["name"], "value": 20 / t_s, "unit": METRIC, "steps": 20, "ms_per_step": 1e3 * t_s / 20,
        "hbm_roofline": hbm_roofline(unit_bytes(ns, nnzs, sts["nnz_l"] + sts["nnz_u"]), t_s / 20),
        "max_rel_residual": worst, "repivots": sts["n_repivot"]}
    return out


def ordering_variant(args, w, dev, vals, rhs, stream):
    """The headline step with the other ordering (the generator's geometric
    nested dissection when the headline uses the library's, and the reverse),
    timed with events over args.auto_order_steps steps after two warm-up
    steps."""
    import torch
    from paper_2411_14082_gb300 import gblu
    n = w["n"]
    a = gblu.Solver(dev)
    geometric = args.ordering == "library"
    t0 = time.perf_counter()
    a.analyze(n, w["Ap"], w["Ai"], w["Q"] if geometric else None)
    t_an = time.perf_counter() - t0
    a.factorize(torch.from_numpy(w["Ax0"]).cuda(dev))
    st = a.stats()
    x = torch.empty(n, dtype=torch.float64, device=f"cuda:{dev}")
    res = torch.zeros(4, dtype=torch.float64, device=f"cuda:{dev}")
    k = min(args.auto_order_steps, len(w["vals"]) - 2)
    for i in range(2):
        a.refactorize(vals[i])
        a.solve(rhs[i], x)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    worst = 0.0
    e0.record(stream)
    for i in range(2, 2 + k):
        a.refactorize(vals[i])
        a.solve(rhs[i], x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    secs = e0.elapsed_time(e1) / 1e3
    a.residual(vals[1 + k], rhs[1 + k], x, out=res)
    worst = float(res[0].item())
    out = {"value": k / secs, "unit": METRIC, "steps": k, "ms_per_step": 1e3 * secs / k,
           "ordering": ("geometric nested dissection from the generator's coordinates" if geometric
                        else "library (gblu_analyze with Q = NULL)"), "analyze_host_s": t_an,
           "refactor_gflop": st["flops"] / 1e9, "nnz_lu": int(st["nnz_l"] + st["nnz_u"]),
           "last_rel_residual": worst}
    del a
    torch.cuda.synchronize(dev)
    return out


def run_ours(args, rank, world, local_rank):
    oracle_proc = None
    import torch
    import torch.distributed as dist
    from paper_2411_14082_gb300 import gblu

    dev = local_rank
    torch.cuda.set_device(dev)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{dev}"))
    total = args.warmup + args.steps
    w = make_workload(args.workload, total, args.seed + 17 * rank, args.mesh)
    n, nnz = w["n"], int(w["Ap"][-1])
    s = gblu.Solver(dev)
    ss = rs = None
    # the library's own ordering (gblu_analyze without Q), or the generator's
    # geometric nested dissection
    qarg = None if args.ordering == "library" else w["Q"]
    t0 = time.perf_counter()
    if args.static_scaling:
        # static pivoting and scaling: the handle factors Dr P A Dc; a second
        # handle on the original pattern only computes residuals
        ss = gblu.StaticScaling(n, w["Ap"], w["Ai"], w["Ax0"], device=dev)
        s.analyze(n, w["Ap"], ss.Ai_scaled, qarg)
        rs = gblu.Solver(dev)
        rs.analyze(n, w["Ap"], w["Ai"], qarg)
    else:
        s.analyze(n, w["Ap"], w["Ai"], qarg)
    t_an = time.perf_counter() - t0
    if args.solve_ctas >= 0:
        s.set_opts(solve_ctas_per_sm=args.solve_ctas)
    Ax0 = torch.from_numpy(w["Ax0"]).cuda(dev)
    t0 = time.perf_counter()
    s.factorize(ss.values(Ax0) if ss else Ax0)
    torch.cuda.synchronize(dev)
    t_fac = time.perf_counter() - t0
    st = s.stats()
    fac_passes = st["tail_passes"]
    first_how = {0: "pivoting kernel", 1: "predicted structure", 2: "predicted structure, then pivoting kernel"}
    first_detail = {"how": first_how.get(st["first_mode"], "?"), "structure_host": st["first_symbolic_ms"],
                    "kernels": st["tail_kernel_ms"], "schedule_host": st["tail_schedule_ms"],
                    "upload": st["tail_upload_ms"]}
    vals = torch.from_numpy(np.stack(w["vals"])).cuda(dev)
    rhs = torch.from_numpy(np.stack(w["rhs"])).cuda(dev)
    xs = torch.empty_like(rhs)
    res = torch.zeros((total, 4), dtype=torch.float64, device=f"cuda:{dev}")
    tuned = None
    if args.autotune:
        t0 = time.perf_counter()
        opts, tr, ts = s.autotune(vals[0], rhs[0], xs[0], reps=3)
        tuned = {"alpha": opts["alpha"], "warp_column_max": opts["warp_column_max"],
                 "solve_dense_density": opts["solve_dense_density"],
                 "solve_slices": opts["solve_slices"], "refactor_ms": tr, "solve_ms": ts,
                 "tuning_s": time.perf_counter() - t0}
        st = s.stats()
    stream = torch.cuda.current_stream(dev)
    ev_r = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(total)]
    ev_s = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(total)]
    repiv = 0

    mixed = args.precision == "mixed"
    iters = []
    if ss:
        # every step maps values and right-hand side to the scaled system and
        # the solution back (three gather-scale launches inside the timed step)
        sv, sb, sy = torch.empty_like(vals[0]), torch.empty_like(rhs[0]), torch.empty_like(rhs[0])
        raw_vals, raw_rhs, raw_x = vals, rhs, xs

        class _Scaled:
            def __init__(self, f, buf):
                self.f, self.buf = f, buf

            def __getitem__(self, i):
                return self.f(i, self.buf)

        vals = _Scaled(lambda i, b: ss.values(raw_vals[i], out=b), sv)
        rhs = _Scaled(lambda i, b: ss.rhs(raw_rhs[i], out=b), sb)
        xs = _Scaled(lambda i, b: b, sy)
    # re-pivoting protocol of the paper's general-case evaluation: a fraction
    # of the timed runs re-pivot at a random step
    frng = np.random.default_rng(args.seed + 99)
    nforce = int(round(args.repivot_frac * args.steps))
    forced = {int(i) + args.warmup: int(frng.integers(0, n))
              for i in frng.choice(args.steps, size=nforce, replace=False)} if nforce else {}
    genuine = {}
    if forced and args.repivot_mode == "genuine":
        # a real pivot failure instead of a forced one: at a random step with
        # no dependency (its pivot is A's entry itself) and other candidates,
        # the pivot entry of A is scaled by 1e-9, so the check fails and the
        # pivot moves; the values are prepared before the timed region
        f0 = s.export_factors()
        leaves = np.nonzero((np.diff(f0["Up"]) == 1) & (np.diff(f0["Lp"]) > 0))[0]
        for i in forced:
            k = int(leaves[frng.integers(0, len(leaves))])
            c, pr = int(f0["q"][k]), int(f0["piv"][k])
            slot = int(w["Ap"][c]) + int(np.nonzero(w["Ai"][w["Ap"][c]:w["Ap"][c + 1]] == pr)[0][0])
            v = vals[i].clone()
            v[slot] *= 1e-9
            genuine[i] = v
            forced[i] = k
    tail_ms = []

    def step(i):
        nonlocal repiv
        if mixed:
            # single-precision refactor, then refinement in double (falls back
            # to the double-precision refactor when it cannot converge)
            ev_r[i][0].record(stream)
            rep = s.refactorize_f32(vals[i])
            ev_r[i][1].record(stream)
            ev_s[i][0].record(stream)
            _, it, _ = s.solve_refined(vals[i], rhs[i], xs[i], tol=1e-12)
            ev_s[i][1].record(stream)
            iters.append(it)
            repiv += int(rep)
        elif args.graph:
            # refactor + solve replayed from one CUDA graph, one sync per step
            ev_r[i][0].record(stream)
            _, rep = s.step(vals[i], rhs[i], xs[i])
            ev_r[i][1].record(stream)
            ev_s[i][0].record(stream)
            ev_s[i][1].record(stream)
            repiv += int(rep)
        elif i in forced:
            ev_r[i][0].record(stream)
            if i in genuine:
                _, rep = s.refactorize(genuine[i])
            else:
                _, rep = s.refactorize_forced(vals[i], forced[i])
            ev_r[i][1].record(stream)
            repiv += int(rep)
            ts = s.stats()
            tail_ms.append([ts["tail_kernel_ms"], ts["tail_repack_ms"], ts["tail_schedule_ms"],
                            ts["tail_upload_ms"], ts["n_restart_cols"], forced[i], ts["tail_passes"], int(rep),
                            ts["repredictions"]])
            ev_s[i][0].record(stream)
            s.solve(rhs[i], xs[i])
            ev_s[i][1].record(stream)
        else:
            ev_r[i][0].record(stream)
            _, rep = s.refactorize(vals[i])
            ev_r[i][1].record(stream)
            repiv += int(rep)
            ev_s[i][0].record(stream)
            s.solve(rhs[i], xs[i])
            ev_s[i][1].record(stream)
        if ss:
            ss.solution(sy, out=raw_x[i])
            rs.residual(raw_vals[i], raw_rhs[i], raw_x[i], out=res[i])
        else:
            s.residual(genuine[i] if i in genuine else vals[i], rhs[i], xs[i], out=res[i])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    # the FP64 pipe's measured rate, beside the nominal peak (before the
    # timed region, never during it)
    try:
        fp64_probe = gblu.fp64_fma_rate(dev)
    except gblu.GbluError:
        fp64_probe = None
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(uuid)
    clocks.start()
    launches0 = s.stats()["kernel_launches"]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for i in range(args.warmup, total):
        step(i)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    launches = s.stats()["kernel_launches"] - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed = t_start.elapsed_time(t_end) / 1e3
    if world > 1:
        elapsed = max_over_ranks(elapsed, world, f"cuda:{dev}")
    t_ref = [ev_r[i][0].elapsed_time(ev_r[i][1]) / 1e3 for i in range(args.warmup, total)]
    t_sol = [ev_s[i][0].elapsed_time(ev_s[i][1]) / 1e3 for i in range(args.warmup, total)]
    # one unit = refactor + solve of one step, from its first to its last event
    t_unit = [ev_r[i][0].elapsed_time(ev_s[i][1]) / 1e3 for i in range(args.warmup, total)]
    resid = res[args.warmup:, 0].max().item()
    fwd = None
    if mixed and rank == 0 and not args.no_cpu_baseline:
        # forward error of every timed result against the oracle's solution
        # of the same values and right-hand side (oracle processes after the
        # timed region, at most 8 at a time)
        xs_host = [(raw_x[i] if ss else xs[i]).cpu().numpy() for i in range(args.warmup, total)]
        nproc = max(1, min(8, args.steps, os.cpu_count() or 1))
        per = -(-args.steps // nproc)
        pref = os.path.join(tempfile.gettempdir(), f"gblu_mixed_x_{os.getpid()}_STEP.npy")
        procs = [start_oracle(args.workload, min(per, args.steps - p * per), args.seed + 17 * rank, args.mesh,
                              first=args.warmup + p * per, xfile=pref)
                 for p in range(nproc) if p * per < args.steps]
        for p in procs:
            collect_oracle(p)
        fwd = []
        for j, i in enumerate(range(args.warmup, total)):
            f = pref.replace("STEP", str(i))
            if os.path.exists(f):
                xo = np.load(f)
                os.remove(f)
                fwd.append(float(np.abs(xs_host[j] - xo).max() / np.abs(xo).max()))
            else:
                fwd.append(None)

    # ---- end to end through the host-buffer entry point (pinned host memory);
    # with static scaling the host-buffer step would need the scaled values,
    # so the end-to-end leg runs on a plain handle of the original pattern
    eh = s
    if ss:
        eh = gblu.Solver(dev)
        eh.analyze(n, w["Ap"], w["Ai"], qarg)
        eh.factorize(Ax0)
    hv = [torch.from_numpy(v).pin_memory().numpy() for v in w["vals"][args.warmup:]]
    hb = [torch.from_numpy(b).pin_memory().numpy() for b in w["rhs"][args.warmup:]]
    hx = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    eh.step_host(hv[0], hb[0], hx)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        eh.step_host(hv[i], hb[i], hx)
    e2e_t = time.perf_counter() - t0
    if world > 1:
        e2e_t = max_over_ranks(e2e_t, world, f"cuda:{dev}")

    # ---- the same refactor + solve with the library's own ordering
    # (gblu_analyze without Q), timed alone after the headline region
    auto = None
    if args.auto_order_steps > 0 and not (mixed or ss or args.graph or forced):
        auto = ordering_variant(args, w, dev, vals, rhs, stream)
    forms = None
    if args.forms and not (mixed or ss or args.graph or forced) and args.workload == "mesh":
        forms = forms_section(args, s, w, dev, vals, rhs, stream)

    if rank != 0:
        return 0
    if not args.no_cpu_baseline:
        # after every GPU measurement, in a separate process: the oracle
        # solves the first timed step of this run (same seed and value set),
        # which checks that step against it and times it
        oracle_x = os.path.join(tempfile.gettempdir(), f"gblu_oracle_x_{os.getpid()}_STEP.npy")
        oracle_proc = start_oracle(args.workload, 1, args.seed + 17 * rank, args.mesh, first=args.warmup,
                                   xfile=oracle_x)
    cpu = collect_oracle(oracle_proc) if oracle_proc else None
    oracle_check = None
    ox = oracle_x.replace("STEP", str(args.warmup)) if cpu else None
    if cpu and os.path.exists(ox):
        xo = np.load(ox)
        os.remove(ox)
        xg = raw_x[args.warmup] if ss else xs[args.warmup]
        xg = xg.cpu().numpy()
        oracle_check = {"step": args.warmup,
                        "max_rel_diff_x": float(np.abs(xg - xo).max() / np.abs(xo).max()),
                        "gpu_residual": float(res[args.warmup, 0].item()),
                        "oracle_residual": cpu[0]["residual"],
                        "note": "the oracle factorizes the same values with fresh pivoting"}
    F = st["flops"]
    t_rf = float(np.mean(t_ref))
    nnz_lu = st["nnz_l"] + st["nnz_u"]
    b_rf = nnz * 12 + 4 * (n + 1) + nnz_lu * 12 + 4 * nnz          # compulsory bytes
    b_rf_stream = b_rf + 12 * F / 2                                 # each dependency read per use
    value = world * args.steps / elapsed
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w["name"], "n": n, "nnz_a": nnz, "nnz_lu": int(nnz_lu),
                   "refactor_gflop": F / 1e9,
                   "ordering": ("library (gblu_analyze with Q = NULL)" if args.ordering == "library"
                                else "geometric nested dissection from the generator's coordinates"),
                   "l2": "inputs and factors larger than L2 (no flush)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "max_rel_residual": resid, "residual_ok": bool(resid <= 1e-12),
        "repivots": repiv,
        "phases_ms": {"refactor": 1e3 * t_rf, "solve": 1e3 * float(np.mean(t_sol)),
                      "refactor_p50": 1e3 * float(np.median(t_ref)),
                      "refactor_p99": 1e3 * float(np.percentile(t_ref, 99)),
                      "solve_p50": 1e3 * float(np.median(t_sol)),
                      "solve_p99": 1e3 * float(np.percentile(t_sol, 99)),
                      "unit_p50": 1e3 * float(np.median(t_unit)),
                      "unit_p99": 1e3 * float(np.percentile(t_unit, 99)),
                      "analyze_host": 1e3 * t_an, "first_factorize": 1e3 * t_fac,
                      "first_factorize_passes": fac_passes, "first_factorize_parts": first_detail},
        "roofline": {"kernel": "refactor (checked re-factorization, all launches)",
                     "bound": "alu", "achieved": F / t_rf / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": F / t_rf / 1e12 / FP64_PEAK_TFLOPS,
                     "traffic": refactor_traffic(w["name"] + "/" + args.ordering),
                     "peak_source": "FP64 ALU rate: 152 SMs x 2.07 GHz x 4 FLOP/clock",
                     "peak_probe_tflops": fp64_probe,
                     "hbm_view": {"compulsory_gbs": b_rf / t_rf / 1e9,
                                  "streaming_gbs": b_rf_stream / t_rf / 1e9}},
        "hbm_roofline": hbm_roofline(b_rf + 12 * (st["nnz_l"] + st["nnz_u"]) + 16 * (n + 1) + 32 * n,
                                     elapsed / args.steps, None),
        "e2e": {"value": world * args.steps / e2e_t, "unit": METRIC,
                "h2d_bytes_per_step": 8 * (nnz + n), "d2h_bytes_per_step": 8 * n},
        "gpu_launches": int(launches),
        "clocks": clk,
        "structure": {k: st[k] for k in ("nnz_l", "nnz_u", "n_levels", "div_level",
                                          "n_solve_levels_l", "n_solve_levels_u",
                                          "etree_height", "device_bytes")},
    }
    if mixed:
        t_iter = iters[args.warmup:]
        line["dtype"] = "f32 factors, f64 refinement"
        line["config"]["precision"] = "mixed"
        line["refinement"] = {"iters_mean": float(np.mean(t_iter)), "iters_max": int(max(t_iter)),
                              "fallbacks": int(sum(1 for v in t_iter if v < 0)),
                              "fwd_err_vs_oracle": fwd,
                              "max_fwd_err_vs_oracle": max((v for v in fwd if v is not None), default=None)
                              if fwd else None}
        # the single-precision refactor's rate over the steps that kept its
        # factors; a step that fell back (an interrupted single-precision
        # launch plus the double-precision refactor inside the refined solve)
        # is not a single-precision refactor time
        kept = [t for t, v in zip(t_ref, t_iter) if v >= 0]
        line["roofline"]["traffic"] = None
        if kept:
            fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
            ach = F / float(np.mean(kept)) / 1e12
            line["roofline"].update({
                "kernel": "refactor_f32 (single-precision checked re-factorization)", "achieved": ach,
                "peak": fp32_peak, "frac": ach / fp32_peak, "steps_counted": len(kept),
                "peak_source": "FP32 ALU rate: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz (nominal)"})
        else:
            ach = F / float(np.mean(t_unit)) / 1e12
            line["roofline"].update({
                "kernel": "whole step (every step fell back to the double-precision refactor)",
                "achieved": ach, "peak": FP64_PEAK_TFLOPS, "frac": ach / FP64_PEAK_TFLOPS,
                "steps_counted": 0})
        line["e2e"]["note"] = "double-precision host-buffer entry point"
    if tuned:
        line["config"]["autotuned"] = tuned
    if ss:
        line["config"]["static_scaling"] = "maximum-product matching + scaling (Dr P A Dc)"
        line["e2e"]["note"] = "unscaled host-buffer entry point"
    if args.graph:
        line["config"]["graph"] = True
        line["phases_ms"]["note"] = "refactor = the whole graph-replayed step (refactor + solve)"
    if forced:
        tm = np.array(tail_ms)
        plain = [t for j, t in enumerate(t_ref) if j + args.warmup not in forced]
        line["config"]["repivot_frac"] = args.repivot_frac
        line["config"]["repivot_mode"] = args.repivot_mode
        line["repivot"] = {"runs": len(forced), "mean_refactor_ms_all": 1e3 * float(np.mean(t_ref)),
                           "restarts": int(tm[:, 7].sum()),
                           "restarts_kept_every_pivot": int(((tm[:, 6] == 0) & (tm[:, 8] == 0) & (tm[:, 7] == 1)).sum()),
                           "repredictions": [int(v) for v in tm[:, 8]],
                           "restart_refactor_ms": [1e3 * t for j, t in enumerate(t_ref) if j + args.warmup in forced],
                           "mean_refactor_ms_plain": 1e3 * float(np.mean(plain)) if plain else None,
                           "slowdown": float(np.mean(t_ref) / np.mean(plain)) if plain else None,
                           "tail_ms_mean": {"kernel": float(tm[:, 0].mean()), "repack": float(tm[:, 1].mean()),
                                            "schedule": float(tm[:, 2].mean()), "upload": float(tm[:, 3].mean())},
                           "restart_cols_mean": float(tm[:, 4].mean()),
                           "forced_steps": [int(v) for v in tm[:, 5]]}
    line["oracle_check"] = oracle_check
    if auto:
        line["other_ordering"] = auto
    if forms:
        line["forms"] = forms
    if cpu:
        secs = [c["seconds"] for c in cpu]
        line["cpu_baseline"] = {"value": len(secs) / sum(secs), "unit": METRIC, "cores": 1,
                                "kind": "oracle",
                                "sample": "1 full refactor+solve unit: the first timed step of this run "
                                          "(single-threaded C oracle, separate process, run after the "
                                          "GPU measurements; the oracle orders by the generator's "
                                          "geometric nested dissection, an input independent of the "
                                          "library)",
                                "max_rel_residual": max(c["residual"] for c in cpu),
                                "host": host_info()}
    else:
        line["cpu_baseline"] = None
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mesh", choices=["mesh", "mesh_ill", "small", "batch", "serve", "serve_poisson", "uneven"])
    ap.add_argument("--sims", type=int, default=32, help="simulations of the serve_poisson workload")
    ap.add_argument("--serve-max-n", type=int, default=500000)
    ap.add_argument("--serve-big", action="store_true", help="add the 500x500x4 mesh (n = 1M) to serve_poisson")
    ap.add_argument("--serve-requests", type=int, default=120, help="requests per offered-load point")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 0.7, 0.9])
    ap.add_argument("--patterns", type=int, default=64, help="patterns of the uneven workload")
    ap.add_argument("--serve-budget-gb", type=int, default=200, help="device memory budget of the serve workload")
    ap.add_argument("--serve-max-batch", type=int, default=16)
    ap.add_argument("--static-scaling", action="store_true",
                    help="factor the statically pivoted and scaled system (maximum-product matching)")
    ap.add_argument("--autotune", action="store_true", help="tune the schedule options on the matrix first")
    ap.add_argument("--graph", action="store_true", help="time gblu_step (CUDA-graph replay) per step")
    ap.add_argument("--repivot-frac", type=float, default=0.0,
                    help="fraction of timed runs that re-pivot at a random step (general-case protocol)")
    ap.add_argument("--repivot-mode", default="forced", choices=["forced", "genuine"],
                    help="forced: the check of a random step is treated as failed (the paper's protocol); "
                         "genuine: a random step's pivot entry is made tiny so that its pivot really moves")
    ap.add_argument("--precision", default="f64", choices=["f64", "mixed"],
                    help="mixed: single-precision refactor + refinement in double")
    ap.add_argument("--sets", type=int, default=256, help="value sets per step of the batch workload")
    ap.add_argument("--solve-ctas", type=int, default=-1,
                    help="CTAs per SM of the sync-free solves (0: as many as fit; default: the library's)")
    ap.add_argument("--batch-group", type=int, default=-1,
                    help="sets per group of the batch launch (0: from the L2 size; default: the library's)")
    ap.add_argument("--seed", type=int, default=inputs.BASE_SEED + 1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--forms", type=int, default=1,
                    help="1: also time the mixed-precision, batched and small forms briefly (context keys)")
    ap.add_argument("--forms-sets", type=int, default=256, help="value sets of the batched form")
    ap.add_argument("--ordering", default="library", choices=["library", "geometric"],
                    help="library: gblu_analyze without Q (the library's choice); geometric: the "
                         "generator's nested dissection")
    ap.add_argument("--auto-order-steps", type=int, default=5,
                    help="steps of the variant with the other ordering (0: skip)")
    ap.add_argument("--mesh", default="200x200x4",
                    help="grid of the mesh workload (smaller grids for profiling runs)")
    args = ap.parse_args()
    args.mesh = tuple(int(v) for v in args.mesh.lower().split("x"))
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batch":
        return run_batch(args, rank, world, local_rank)
    if args.workload == "serve":
        return run_serve(args, rank, world, local_rank)
    if args.workload == "serve_poisson":
        return run_serve_poisson(args, rank, world, local_rank)
    if args.workload == "uneven":
        return run_uneven(args, rank, world, local_rank)
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
