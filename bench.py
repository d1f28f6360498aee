"""Benchmark: adaptive D2Q21 MLUPS on the 4096^2 high-Mach shear layer.

Workload (one GPU): 4096 x 4096 periodic double shear layer, streams at
+-Mach 2.5 of the cold stream (T_cold = 0.35, temperature ratio 3, tanh width 8),
seeded transverse perturbations in modes 1..8, nu = 1e-5, gamma = 1.4, shifts
in {-2..2}^2, kinetic sensor on, FP32 populations with FP64 Newton. A bench
step is one time step of the whole flow (one launch of the fused step
kernel). The state is 5.7 GB (FP32 form), far larger than L2, so no flush is
needed between steps. The headline times the steps after the warm-up from
the initial state.

Reported beside it: the FP64 plain path on the same flow (MLUPS and the FP32
form's moment error against it), the same FP32 flow once developed (steps
1900-2000 of the workload's 2000) and the mean over all its steps after the
warm-up, the FP32 form's moment error against the FP64 oracle on the 256^2
version of the flow over 200 steps (free-running and with replayed lattice
decisions), the end-to-end figure through the C ABI with host buffers, the
FP64-pipe roofline of the step kernel with the method's own minimum FP64
work beside it, and the CPU oracle on a bounded sample of the same flow (all
cores and one core, CPU model recorded).

Two sub-results run after it on one GPU (skipped under torchrun with N > 1):

* "batched": 256 independent periodic flows, sides log-uniform in
  [64, 1024] (vortex or shear layer, Mach 0.5-3, temperature ratio 1-4,
  nu 1e-5..1e-3, FP32 form), advanced together by one persistent launch per
  step (alb_batch_step: CUDA graph of two steps, autotuned launch shape);
  MLUPS over all flows, beside the same flows stepped one launch per flow.
* "serve": the serving loop under a Poisson stream of requests (50 per
  second for 60 s; sides 64-2048, 100-5000 steps, FP32 or FP64 form, vortex,
  shear-layer or 2D-Riemann initial data, the last with zero-gradient
  ends): completion latency p50/p99, served versus offered node updates;
  flagged requests by initial state; then a stream of the same shape on a
  reduced range (sides 64-512, 100-1000 steps) at about 70 % of the
  measured capacity, drained to completion (bounded).

`--impl reference` times the CPU oracle instead.
Multi-GPU (torchrun, N ranks): every rank runs its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2009_13426_gb300 import costmodel, flows  # noqa: E402

METRIC = "adaptive D2Q21 MLUPS, FP32 form vs FP64 plain at stated error; serve p50/p99"
# DRAM bytes (read + write) per node update of step_kernel<float>, from one
# ncu capture of the 1024^2 case of the same flow (dram__bytes_read.sum +
# dram__bytes_write.sum = 226.9 + 370.5 MB per launch for 1,048,576 nodes,
# mean of the first 3 launches, kinetic sensor on); the traffic
# grows in proportion to the nodes, so a 4096^2 launch moves 16,777,216 x
# this. Measured on the current kernel.
TRAFFIC_BYTES_PER_NODE_FP32 = 569.7
UNIT = "MLUPS"
NU = 1e-5
# The kinetic sensor (Sec. IV.A.2) is on in every timed flow: without it the
# nu = 1e-5 shear layer loses realizability after 300-400 steps in both
# precisions (and in the FP64 oracle), and long serving requests fail.
SENSOR = 1
# step count of the shear-layer workload; its last 100 steps are timed as the
# developed flow
DEVELOPED_STEPS = 2000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", "--n", dest="n", type=int, default=4096,
                    help="grid side of the shear layer (--side under torchrun)")
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--developed-steps", type=int, default=DEVELOPED_STEPS,
                    help="advance the FP32 flow to this step and time the last 100 "
                         "(0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the FP32 form's error against the oracle at 256^2")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-overlap", action="store_true")
    ap.add_argument("--no-d2q49", action="store_true",
                    help="skip the D2Q49 reference-solver line")
    ap.add_argument("--d2q49-side", type=int, default=1024)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=10)
    ap.add_argument("--batched-flows", type=int, default=256,
                    help="use the first N flows of the 256 (smaller profiling runs)")
    ap.add_argument("--no-tune", action="store_true", help="batched: keep the default shape")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-drain", type=float, default=90.0,
                    help="seconds the 70%% run may take after its last arrival")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- distributed

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_mlups(world, nodes, steps, ms_max):
    """Whole-job throughput: every rank advanced `nodes` nodes `steps` times;
    the slowest rank's time bounds the job."""
    return world * nodes * steps / (ms_max * 1e-3) / 1e6


def workload_config(n, world):
    return {"workload": "shear layer %dx%d periodic, Mach 2.5 cold stream, T ratio 3, "
                        "nu 1e-5, kinetic sensor on, FP32 populations, FP64 Newton" % (n, n),
            "nodes": n * n, "u_max": 2, "l2_flush": "not needed: 5.7 GB state >> L2",
            "parallelism": "replica per GPU" if world > 1 else "single GPU"}


# ----------------------------------------------------------------- CPU oracle sample

def cpu_model():
    """The host CPU's model name (lscpu), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _omp():
    """The OpenMP runtime the oracle runs on (its thread count can be set)."""
    import ctypes
    try:
        return ctypes.CDLL("libgomp.so.1")
    except OSError:
        return None


def oracle_sample(n, steps, warmup=1, rows=None, threads=None):
    """The CPU oracle on a bounded sample of the n^2 shear layer: a band of
    `rows` rows of the uniform hot stream and one centred on a shear layer,
    each n wide with zero-gradient ends in y. A sample step is one oracle step
    of both bands. Reported: the measured time per sample step, the sample's
    own rate, and the rate of the full flow estimated by weighting the two
    bands' per-node times by the flow's row mix (2 * rows of n rows lie in
    the two layers)."""
    import oracle as O
    O.lib()
    omp = _omp()
    if threads and omp is not None:
        omp.omp_set_num_threads(int(threads))
    used = omp.omp_get_max_threads() if omp is not None else os.cpu_count()
    try:
        f = flows.shear_layer(n)
        rows = rows or min(64, max(8, n // 8))
        bands = {"uniform": 0, "layer": n // 4 - rows // 2}
        sims = {}
        for name, y0 in bands.items():
            band = [a[y0:y0 + rows].copy() for a in f]
            s = O.Simulation(O.make_config(n, rows, umax=2, nu=NU, bc_y=O.ZERO_GRADIENT,
                                           sensor=bool(SENSOR)))
            assert s.init(*band) == O.OK
            sims[name] = s
        for s in sims.values():
            if warmup:
                s.step(warmup)
        per = {k: 0.0 for k in sims}
        for _ in range(steps):
            for name, s in sims.items():
                t0 = time.perf_counter()
                s.step(1)
                per[name] += time.perf_counter() - t0
    finally:
        if threads and omp is not None:
            omp.omp_set_num_threads(os.cpu_count() or 1)
    total = sum(per.values())
    frac_layer = min(1.0, 2 * rows / n)
    t_node = ((1 - frac_layer) * per["uniform"] + frac_layer * per["layer"]) / (steps * n * rows)
    nodes = 2 * n * rows
    return {"mlups": 1e-6 / t_node, "mlups_sample": nodes * steps / total / 1e6,
            "time_s": total, "ms_per_step": 1e3 * total / steps, "nodes_per_step": nodes,
            "threads": used,
            "sample": "two %dx%d bands of the %d^2 shear layer (uniform stream; shear layer), "
                      "zero-gradient ends in y, %d timed steps each after %d untimed; value "
                      "weights their per-node times by the full flow's row mix"
                      % (n, rows, n, steps, warmup)}


def cpu_baseline(n):
    """The oracle on all host cores (two 64-row bands, 2 steps) and on one core
    (two 8-row bands, 1 step): a bounded sample of a few seconds each."""
    allc = oracle_sample(n, 2, warmup=1)
    one = oracle_sample(n, 1, warmup=1, rows=8, threads=1)
    return {"value": round(allc["mlups"], 4), "unit": UNIT, "cores": allc["threads"],
            "kind": "oracle", "sample": allc["sample"], "cpu_model": cpu_model(),
            "nproc": os.cpu_count(), "timed_s": round(allc["time_s"], 2),
            "single_thread": {"value": round(one["mlups"], 5), "unit": UNIT, "cores": 1,
                              "sample": one["sample"], "timed_s": round(one["time_s"], 2)}}


# ----------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The reference arm: the CPU oracle as it stands on the host cores. Each
    step is one oracle step of the bounded sample above (two 64-row bands of
    the 4096^2 flow); ms_per_step is the measured time of that sample step,
    and the value is the full flow's rate estimated from it."""
    if rank != 0:
        return
    t0 = time.perf_counter()
    res = oracle_sample(args.n, args.steps, warmup=args.warmup)
    cpu = {"value": round(res["mlups"], 4), "unit": UNIT, "cores": res["threads"],
           "kind": "oracle", "sample": res["sample"], "cpu_model": cpu_model(),
           "nproc": os.cpu_count()}
    line = {
        "metric": METRIC, "value": round(res["mlups"], 4), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "impl": "reference",
        "ms_per_step": round(res["ms_per_step"], 1),
        "step": "one oracle step of the sample (%d node updates)" % res["nodes_per_step"],
        "sample_mlups": round(res["mlups_sample"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.n, world),
        "cpu_baseline": cpu,
        "e2e": {"value": round(res["mlups"], 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t0, 1),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm

def _sync_flagged(obj, alb):
    """Synchronise; node failures are counted flags, not errors."""
    try:
        obj.sync()
    except alb.AlbError as e:
        if e.code != alb.ALB_ENEWTON:
            raise


def shear_error_vs_oracle(alb, n=256, steps=200):
    """The FP32 form against the FP64 oracle on the n^2 version of the headline
    flow over `steps` steps: free-running, and with the oracle replaying the
    GPU's lattice decisions (which isolates the step's arithmetic). Also the
    lattice decisions the GPU took differently from what Eq. criterion gives on
    the replayed oracle's moments (FP32 round-off at a threshold)."""
    import oracle as O
    fields = flows.shear_layer(n)
    okw = dict(umax=2, nu=NU, sensor=bool(SENSOR))
    fl = alb.Flow(n, n, u_max=2, nu=NU, precision=alb.ALB_FP32_FORM, sensor=SENSOR)
    fl.init(*fields)
    rep = O.Simulation(O.make_config(n, n, **okw))
    assert rep.init(*fields) == O.OK
    crit = lambda u: np.clip(np.ceil(u + 0.5) - 1, -2, 2).astype(np.int8)
    flips = 0
    for _ in range(steps):
        _, ux, uy, _ = rep.primitives()
        fl.step(1)
        gx, gy = fl.shifts()
        flips += int((gx != crit(ux)).sum() + (gy != crit(uy)).sum())
        rep.step_forced(gx, gy)
    got = fl.moments()
    fl.close()
    free = O.Simulation(O.make_config(n, n, **okw))
    assert free.init(*fields) == O.OK
    free.step(steps)

    def errs(ref):
        r, a, b, e = got
        R, A, B, E = ref
        dm, mm = np.sqrt((a - A) ** 2 + (b - B) ** 2), np.sqrt(A ** 2 + B ** 2)
        mx = max(np.abs(r - R).max() / np.abs(R).max(), dm.max() / mm.max(),
                 np.abs(e - E).max() / np.abs(E).max())
        l2 = max(np.linalg.norm(r - R) / np.linalg.norm(R),
                 np.linalg.norm(dm) / np.linalg.norm(mm),
                 np.linalg.norm(e - E) / np.linalg.norm(E))
        return {"max_rel": float("%.3e" % mx), "l2_rel": float("%.3e" % l2)}

    return {"workload": "shear layer %dx%d (the headline's recipe), %d steps, FP32 form "
                        "against the FP64 oracle" % (n, n, steps),
            "replayed": errs(rep.moments()), "free_running": errs(free.moments()),
            "flipped_decisions": flips,
            "flipped_per_node_step": float("%.3e" % (flips / (n * n * steps)))}


def run_batched(args):
    """256 flows in one persistent launch per step (alb_batch_step)."""
    import torch
    from paper_2009_13426_gb300 import alb

    specs = flows.batched_flows(256)[:args.batched_flows]
    nodes = sum(sp.nx * sp.ny for sp in specs)
    stream = torch.cuda.Stream()
    b = alb.Batch([dict(nx=sp.nx, ny=sp.ny, nu=sp.nu, precision=alb.ALB_FP32_FORM, sensor=SENSOR)
                   for sp in specs], stream=stream)
    try:
        for sp, fl in zip(specs, b.flows):
            fl.init(*sp.fields())
        t = time.perf_counter()
        if not args.no_tune:
            b.tune(trials=2)
        tune_s = time.perf_counter() - t
        tuning = b.tuning(alb.ALB_FP32_FORM)
        b.step(args.warmup)
        _sync_flagged(b, alb)
        s0 = [fl.stats() for fl in b.flows]
        k = args.batched_steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        _sync_flagged(b, alb)
        s1 = [fl.stats() for fl in b.flows]
        tot = {key: sum(x[key] - y[key] for x, y in zip(s1, s0))
               for key in ("fp64_evaluations", "fp64_updates", "fp32_iterations", "newton_calls",
                           "newton_iterations", "reconstructions", "newton_failures",
                           "reconstruction_failures")}
        # the same flows one launch per flow and step (alb_step), same stream
        e0.record(stream)
        for fl in b.flows:
            fl.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_alone = e0.elapsed_time(e1)
    finally:
        b.close()
    launches = k * (2 if tuning["dynamic"] else 1) + (k % 2)
    upd = nodes * k
    tot["node_updates"] = upd
    slots = costmodel.fp64_slots(tot, "fp32")
    tflops = 2.0 * slots / (ms * 1e-3) / 1e12
    return {"workload": "256 periodic flows, side log-uniform 64-1024 (seed 4), vortex or "
                        "shear layer, Mach 0.5-3, T ratio 1-4, nu 1e-5..1e-3, FP32 form",
            "flows": len(specs), "nodes": nodes, "steps": k, "unit": UNIT,
            "value": round(upd / (ms * 1e-3) / 1e6, 2), "ms_per_step": round(ms / k, 3),
            "one_launch_per_flow": {"value": round(upd / (ms_alone * 1e-3) / 1e6, 2),
                                    "launches_per_step": len(specs)},
            "graph": "two steps per CUDA graph replay",
            "launches": launches, "tuning": tuning, "tune_seconds": round(tune_s, 1),
            "per_node": {key: round(v / upd, 4) for key, v in tot.items()
                         if key not in ("newton_failures", "reconstruction_failures",
                                        "node_updates")},
            "roofline": {"bound": "alu", "achieved": round(tflops, 4),
                         "peak": round(costmodel.FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                         "frac": round(tflops / costmodel.FP64_PEAK_TFLOPS, 4),
                         "kernel": "batch_step_kernel<float>"},
            "failures": {"node": tot["newton_failures"],
                         "rebuild": tot["reconstruction_failures"],
                         "node_per_update": float("%.3g" % (tot["newton_failures"] / upd)),
                         "rebuild_per_rebuild": float("%.3g" % (
                             tot["reconstruction_failures"] / max(tot["reconstructions"], 1)))},
            "clamped_flows": sum(1 for sp in specs if sp.clamped)}


def _serve_stream(alb, reqs, window, drain):
    """Submit reqs at their arrival times (fields produced at admission by a
    fill callback), wait `drain` seconds after the window, collect."""
    srv = alb.Server()
    ids = {}
    rejected = 0

    def fill_of(sp):
        def fill(*outs):
            for o, f in zip(outs, sp.fields()):
                o[:] = f
        return fill

    t0 = time.perf_counter()
    try:
        for sp in reqs:
            while time.perf_counter() - t0 < sp.arrival:
                time.sleep(0.0005)
            prec = alb.ALB_FP32_FORM if sp.precision == "fp32" else alb.ALB_FP64_PLAIN
            # the 2D Riemann problem with the paper's zero-gradient ends: periodic
            # ends would add the reversed quadrant jumps at the box's edges
            bc = alb.ALB_ZERO_GRADIENT if sp.kind == "riemann2d" else alb.ALB_PERIODIC
            try:
                rid = srv.submit(sp.steps, fill=fill_of(sp), keep_result=False, nx=sp.nx,
                                 ny=sp.ny, nu=sp.nu, precision=prec, sensor=SENSOR, bc_x=bc,
                                 bc_y=bc)
                ids[rid] = sp
            except alb.AlbError:
                rejected += 1
        end = t0 + window + drain
        done = {}
        while time.perf_counter() < end and len(done) < len(ids):
            for rid in list(ids):
                if rid in done:
                    continue
                st, res = srv.poll(rid)
                if res is not None:
                    done[rid] = res
            time.sleep(0.05)
        stats = srv.stats()
    finally:
        srv.close()
    lat = sorted(r["t_done"] - r["t_submit"] for r in done.values())
    n = len(ids)
    unfinished = n - len(done)

    def pct(q):
        # over all submitted requests, unfinished ones counted as slower than any
        k = int(math.ceil(q * n)) - 1
        return round(lat[k], 3) if 0 <= k < len(lat) else None

    served = stats["node_updates"]
    return {"submitted": n, "completed": len(done), "unfinished": unfinished,
            "rejected": rejected,
            "p50_s": pct(0.50), "p99_s": pct(0.99),
            "completed_p50_s": round(lat[len(lat) // 2], 3) if lat else None,
            "completed_p99_s": round(lat[min(len(lat) - 1, int(0.99 * len(lat)))], 3)
            if lat else None,
            "offered_updates_per_s": float("%.4g" % (sum(sp.nx * sp.ny * sp.steps for sp in reqs)
                                                     / window)),
            "served_mlups": round(served / stats["elapsed_seconds"] / 1e6, 2),
            "busy_fraction": round(stats["busy_seconds"] / stats["elapsed_seconds"], 3),
            "elapsed_s": round(stats["elapsed_seconds"], 1),
            "flagged": sum(1 for r in done.values() if r["status"] == alb.ALB_ENEWTON),
            "flagged_detail": _flag_detail(alb, ids, done),
            "failed": sum(1 for r in done.values()
                          if r["status"] not in (alb.ALB_OK, alb.ALB_ENEWTON)),
            "ns_per_update": {"fp64": round(stats["ns_per_update"][0], 3),
                              "fp32": round(stats["ns_per_update"][1], 3)}}


def _flag_detail(alb, ids, done):
    """Which completed requests were flagged (any node equilibrium or Grad
    rebuild that fell back), by initial state, and how rare the fallbacks
    were: failed node updates per node update, failed rebuilds per rebuild."""
    out = {}
    for kind in ("vortex", "shear", "riemann2d"):
        rs = [r for rid, r in done.items() if ids[rid].kind == kind]
        if not rs:
            continue
        upd = sum(r["stats"]["node_updates"] for r in rs)
        reb = sum(r["stats"]["reconstructions"] for r in rs)
        out[kind] = {"completed": len(rs),
                     "clamped": sum(1 for rid in done if ids[rid].kind == kind and
                                    ids[rid].clamped),
                     "flagged": sum(1 for r in rs if r["status"] == alb.ALB_ENEWTON),
                     "with_node_failures": sum(1 for r in rs if r["stats"]["newton_failures"]),
                     "node_failures_per_update": float("%.3g" % (
                         sum(r["stats"]["newton_failures"] for r in rs) / max(upd, 1))),
                     "rebuild_failures_per_rebuild": float("%.3g" % (
                         sum(r["stats"]["reconstruction_failures"] for r in rs) / max(reb, 1)))}
    return out


def run_serve(args):
    from paper_2009_13426_gb300 import alb

    w = args.serve_seconds
    reqs = flows.serving_requests(rate=50.0, duration=w)
    heavy = _serve_stream(alb, reqs, w, 5.0)
    # The full mix needs about a minute of GPU time per request on average
    # (sides up to 2048, up to 5000 steps, half of them FP64 plain), so a
    # stream at 70 % utilisation would bring about one request per minute and
    # its percentiles would need hours. The second stream keeps the mix's
    # shape on a reduced range (sides 64-512, 100-1000 steps) at a rate of
    # 70 % of the capacity measured in the first run.
    ns = heavy["ns_per_update"]
    small = dict(smin=64, smax=512, steps_min=100, steps_max=1000)
    probe = flows.serving_requests(rate=50.0, duration=60.0, seed=6, **small)
    mean_s = sum(sp.nx * sp.ny * sp.steps * ns["fp32" if sp.precision == "fp32" else "fp64"]
                 for sp in probe) * 1e-9 / len(probe)
    rate = 0.7 / mean_s
    reqs70 = flows.serving_requests(rate=rate, duration=w, seed=7, **small)
    light = _serve_stream(alb, reqs70, w, args.serve_drain)
    light["rate_per_s"] = round(rate, 4)
    light["mix"] = "sides log-uniform 64-512, steps log-uniform 100-1000, otherwise as above"
    return {"workload": "Poisson arrivals, sides log-uniform 64-2048, steps log-uniform "
                        "100-5000, FP32 or FP64 form, vortex / shear layer / 2D Riemann; "
                        "fields made at admission; 80 % HBM admission budget",
            "window_s": w, "rate_50_per_s": heavy, "reduced_mix_at_70pct": light,
            "latency": "submit to results in host memory; p50/p99 over all submitted "
                       "requests (unfinished ones count as slower than any), completed_* "
                       "over the completed ones"}


def run_ours(args, world, rank, local):
    import torch
    from paper_2009_13426_gb300 import alb

    torch.cuda.set_device(local)
    alb.lib()
    n = args.n
    N = n * n
    fields = flows.shear_layer(n)
    stream = torch.cuda.Stream()

    def make(precision):
        fl = alb.Flow(n, n, u_max=2, nu=NU, precision=precision, sensor=SENSOR, stream=stream)
        fl.init(*fields)
        return fl

    def timed(fl, steps, warm):
        for _ in range(warm):
            alb.alb_step(fl.h, 1)
        fl.sync()
        s0 = fl.stats()
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            alb.alb_step(fl.h, 1)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = e0.elapsed_time(e1)
        s1 = fl.stats()
        delta = {k: s1[k] - s0[k] for k in s1}
        return ms, delta

    # FP32 form: the headline
    fl32 = make(alb.ALB_FP32_FORM)
    clocks = ClockSampler(local)
    clocks.start()
    ms32, d32 = timed(fl32, args.steps, args.warmup)
    clk = clocks.stop()
    ms_max = dist_max(ms32, world)
    mlups = aggregate_mlups(world, N, args.steps, ms_max)
    per_launch_ms = ms32 / args.steps
    slots = costmodel.fp64_slots(d32, "fp32")
    achieved_tflops = 2.0 * slots / args.steps / (per_launch_ms * 1e-3) / 1e12
    bytes_per_launch = costmodel.BYTES_PER_NODE["fp32"] * N
    hbm_gbs = bytes_per_launch / (per_launch_ms * 1e-3) / 1e9
    total32 = args.warmup + args.steps

    extra = {}
    if not args.no_fp64:
        fl64 = make(alb.ALB_FP64_PLAIN)
        k64 = args.fp64_steps or max(2, args.steps // 4)
        # advance to the same step count as the FP32 run for the error figure
        ms64, d64 = timed(fl64, k64, max(0, total32 - k64))
        m32 = fl32.moments()
        m64 = fl64.moments()
        s32 = fl32.shifts()
        s64 = fl64.shifts()
        r, a, b, e = m32
        R, A, B, E = m64
        l2 = max(np.linalg.norm(r - R) / np.linalg.norm(R),
                 math.sqrt(np.linalg.norm(a - A) ** 2 + np.linalg.norm(b - B) ** 2)
                 / math.sqrt(np.linalg.norm(A) ** 2 + np.linalg.norm(B) ** 2),
                 np.linalg.norm(e - E) / np.linalg.norm(E))
        linf = max(np.abs(r - R).max() / np.abs(R).max(),
                   np.sqrt((a - A) ** 2 + (b - B) ** 2).max() / np.sqrt(A ** 2 + B ** 2).max(),
                   np.abs(e - E).max() / np.abs(E).max())
        tot = max(abs(r.sum() - R.sum()) / R.sum(), abs(e.sum() - E.sum()) / E.sum())
        slots64 = costmodel.fp64_slots(d64, "fp64")
        extra["fp64_plain"] = {"value": round(N * k64 / (ms64 * 1e-3) / 1e6, 2), "unit": UNIT,
                               "steps": k64, "ms_per_step": round(ms64 / k64, 3),
                               "fp64_slots_per_node": round(slots64 / k64 / N, 1),
                               "fp64_tflops": round(2.0 * slots64 / (ms64 * 1e-3) / 1e12, 4),
                               "counters": {k: d64[k] for k in ("newton_iterations",
                                                                 "newton_calls",
                                                                 "fp64_evaluations",
                                                                 "reconstructions")}}
        extra["error"] = {"fp32_form_vs_fp64_plain_l2_rel": float("%.3e" % l2),
                          "totals_rel": float("%.3e" % tot),
                          "max_rel": float("%.3e" % linf),
                          "lattice_differs_nodes": int((s32[0] != s64[0]).sum()
                                                       + (s32[1] != s64[1]).sum()),
                          "after_steps": total32,
                          "metric": "l2: max over rho, rho*u, rho*E of ||d||_2/||ref||_2; "
                                    "max: same with max-norms (a node whose velocity lies within "
                                    "FP32 round-off of a shift threshold may take another lattice, "
                                    "which changes it at O(1e-2))"}
        fl64.close()

    # The same flow once developed: advanced (untimed) to step
    # developed_steps - 100, then the last 100 steps timed. The vortices of the
    # rolled-up layers need more FP32 Newton steps and refinements per node.
    developed = None
    k_dev = 100
    full_run = None
    if args.developed_steps >= total32 + k_dev:
        clocks_d = ClockSampler(local)
        adv = args.developed_steps - k_dev - total32
        ea0 = torch.cuda.Event(enable_timing=True)
        ea1 = torch.cuda.Event(enable_timing=True)
        ea0.record(stream)
        for _ in range(adv // 100):
            alb.alb_step(fl32.h, 100)
        alb.alb_step(fl32.h, adv % 100)
        ea1.record(stream)
        torch.cuda.synchronize()
        ms_adv = ea0.elapsed_time(ea1)
        clocks_d.start()
        ms_d, dd = timed(fl32, k_dev, 0)
        clk_d = clocks_d.stop()
        ms_d = dist_max(ms_d, world)
        slots_d = costmodel.fp64_slots(dd, "fp32")
        tf_d = 2.0 * slots_d / (ms_d * 1e-3) / 1e12
        developed = {"value": round(aggregate_mlups(world, N, k_dev, ms_d), 2), "unit": UNIT,
                     "steps": [args.developed_steps - k_dev, args.developed_steps],
                     "ms_per_step": round(ms_d / k_dev, 3),
                     "per_node": {k: round(dd[k] / (N * k_dev), 4)
                                  for k in ("fp32_iterations", "fp64_evaluations", "fp64_updates",
                                            "newton_calls", "reconstructions")},
                     "failures": {"node": dd["newton_failures"],
                                  "rebuild": dd["reconstruction_failures"]},
                     "roofline": {"bound": "alu", "achieved": round(tf_d, 4),
                                  "peak": round(costmodel.FP64_PEAK_TFLOPS, 4),
                                  "unit": "TFLOP/s",
                                  "frac": round(tf_d / costmodel.FP64_PEAK_TFLOPS, 4),
                                  "note": "FP64 slots only: the FP32 Newton steps, more "
                                          "than two per node here, are not counted"},
                     "clocks": clk_d}
        r, a, b, e = fl32.moments()
        T = (e / r - 0.5 * ((a / r) ** 2 + (b / r) ** 2)) / 2.5
        developed["state"] = {"finite": bool(np.isfinite(r).all() and np.isfinite(e).all()),
                              "rho_min": float("%.4g" % r.min()),
                              "T_min": float("%.4g" % T.min())}
        # every step of the workload after the warm-up, timed in three pieces
        # with CUDA events on the flow's stream: the headline steps, the
        # advance, the developed steps
        k_all = args.steps + adv + k_dev
        ms_all = dist_max(ms32 + ms_adv + ms_d, world)
        full_run = {"value": round(aggregate_mlups(world, N, k_all, ms_all), 2), "unit": UNIT,
                    "steps": [args.warmup, args.developed_steps],
                    "ms_per_step": round(ms_all / k_all, 3)}
    st = fl32.stats()
    fl32.close()

    # the same flow with shift ranges widened by 0.5, chosen by history or by
    # the neighbourhood
    ovl = None
    if not args.no_overlap:
        ovl = {"shift_overlap": 0.5, "unit": UNIT,
               "criterion": {"value": round(mlups / world, 2),
                             "rebuilt_pulls_per_node": round(d32["reconstructions"]
                                                             / (N * args.steps), 4)}}
        for name, rule in (("history", alb.ALB_RULE_HISTORY),
                           ("neighbourhood", alb.ALB_RULE_NEIGHBOURS)):
            flo = alb.Flow(n, n, u_max=2, nu=NU, precision=alb.ALB_FP32_FORM, stream=stream,
                           shift_overlap=0.5, shift_rule=rule, sensor=SENSOR)
            flo.init(*fields)
            mso, dso = timed(flo, args.steps, args.warmup)
            ovl[name] = {"value": round(N * args.steps / (mso * 1e-3) / 1e6, 2),
                         "ms_per_step": round(mso / args.steps, 3),
                         "rebuilt_pulls_per_node": round(dso["reconstructions"]
                                                         / (N * args.steps), 4)}
            flo.close()

    # the paper's reference solver (App. C.1): D2Q49, 13 moments, FP64, on the
    # same shear-layer recipe at a smaller side
    q49 = None
    if not args.no_d2q49:
        n49 = args.d2q49_side
        f49 = fields if n49 == n else flows.shear_layer(n49)
        fl = alb.Flow(n49, n49, stencil=alb.ALB_D2Q49, moments=13, u_max=2, nu=NU,
                      precision=alb.ALB_FP64_PLAIN, sensor=SENSOR, stream=stream)
        fl.init(*f49)
        k49 = max(2, args.steps // 4)
        ms49, d49 = timed(fl, k49, min(args.warmup, 2))
        N49 = n49 * n49
        q49 = {"workload": "shear layer %dx%d (the headline's recipe), D2Q49, 13 moments, "
                           "FP64" % (n49, n49),
               "value": round(N49 * k49 / (ms49 * 1e-3) / 1e6, 2), "unit": UNIT,
               "steps": k49, "ms_per_step": round(ms49 / k49, 3),
               "kernel": "q49::step_kernel",
               "per_node": {k: round(d49[k] / (N49 * k49), 4)
                            for k in ("newton_iterations", "newton_calls", "reconstructions")},
               "failures": {"node": d49["newton_failures"],
                            "rebuild": d49["reconstruction_failures"]}}
        slots49 = costmodel.q49_slots(d49, N49 * k49)
        if slots49:
            t49 = 2.0 * slots49 / (ms49 * 1e-3) / 1e12
            q49["roofline"] = {"bound": "alu", "achieved": round(t49, 4),
                               "peak": round(costmodel.FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                               "frac": round(t49 / costmodel.FP64_PEAK_TFLOPS, 4)}
        fl.close()

    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).pin_memory() for a in fields]
        outs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(4)]
        fl = alb.Flow(n, n, u_max=2, nu=NU, precision=alb.ALB_FP32_FORM, sensor=SENSOR,
                      stream=stream)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        alb.alb_init(fl.h, *[p.numpy() for p in pinned])
        drift = None
        for _ in range(args.steps):
            alb.alb_step(fl.h, 1)
            tot = alb.alb_totals(fl.h)  # the step's conservation totals, read to the host
            drift = tot if drift is None else drift
        alb.alb_moments(fl.h, [o.numpy() for o in outs])
        dt = time.perf_counter() - t0
        dt = dist_max(dt, world)
        mass_drift = abs(tot[0] - drift[0]) / abs(drift[0])
        fl.close()
        e2e = {"value": round(world * N * args.steps / dt / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(4 * N * 8 / args.steps),
               "d2h_bytes_per_step": int(4 * 8 + 4 * N * 8 / args.steps),
               "note": "alb_init from pinned host fields, then every step alb_step and "
                       "alb_totals (mass, momentum, energy read to the host), then alb_moments "
                       "to pinned host; wall clock; the field copies are divided by the steps",
               "mass_drift": float("%.3e" % mass_drift)}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)

    err256 = None
    if rank == 0 and not args.no_oracle_error:
        err256 = shear_error_vs_oracle(alb)

    batched = serve = None
    if world == 1 and not args.no_batched:
        batched = run_batched(args)
    if world == 1 and not args.no_serve:
        serve = run_serve(args)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(mlups, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(n, world),
        "roofline": {"bound": "alu", "achieved": round(achieved_tflops, 4),
                     "peak": round(costmodel.FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                     "frac": round(achieved_tflops / costmodel.FP64_PEAK_TFLOPS, 4),
                     "traffic": round(TRAFFIC_BYTES_PER_NODE_FP32 * N),
                     "traffic_note": "ncu DRAM bytes per node on the 1024^2 case x nodes: "
                                     "1.36 x the 420 algorithmic bytes, the excess being "
                                     "the threads' stack (spills, call frames) leaving L2",
                     "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                     "kernel": "step_kernel<float>",
                     "fp64_slots_per_node": round(slots / args.steps / N, 1),
                     "method_floor": costmodel.method_floor(mlups / world),
                     "hbm": {"achieved_gbs": round(hbm_gbs, 1),
                             "bytes_per_node": costmodel.BYTES_PER_NODE["fp32"]}},
        "clocks": clk,
        "gpu_launches": args.steps,
        "counters": {k: st[k] for k in ("newton_iterations", "newton_calls", "fp64_evaluations",
                                        "fp64_updates",
                                        "fp32_iterations", "reconstructions",
                                        "newton_failures", "reconstruction_failures")},
    }
    line.update(extra)
    if err256:
        line.setdefault("error", {})["oracle_256"] = err256
    if full_run:
        line["full_run"] = full_run
    if developed:
        line["developed_flow"] = developed
    if ovl:
        line["overlapping_ranges"] = ovl
    if q49:
        line["reference_solver_d2q49"] = q49
    if batched:
        line["batched"] = batched
    if serve:
        line["serve"] = serve
    if world > 1:
        line["batched"] = line["serve"] = "skipped with more than one rank"
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
