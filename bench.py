"""Benchmark: adaptive D2Q21 MLUPS on the 4096^2 high-Mach shear layer.

Workload (one GPU): 4096 x 4096 periodic double shear layer, streams at
+-Mach 2.5 of the cold stream (T_cold = 0.35, temperature ratio 3, tanh width 8),
seeded transverse perturbations in modes 1..8, nu = 1e-5, gamma = 1.4, shifts
in {-2..2}^2, FP32 populations with FP64 Newton. A bench step is one time
step of the whole flow (one launch of the fused step kernel). The state is
5.7 GB (FP32 form), far larger than L2, so no flush is needed between steps.

Reported beside it: the FP64 plain path on the same flow (MLUPS and the FP32
form's moment error against it), the end-to-end figure through the C ABI with
host buffers, the FP64-pipe roofline of the step kernel, and the CPU oracle
on a bounded sample of the same flow.

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
UNIT = "MLUPS"
NU = 1e-5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
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


# ----------------------------------------------------------------- CPU oracle sample

def oracle_sample(n, steps, warmup=1):
    """The CPU oracle on a bounded sample of the n^2 shear layer: a 64-row band
    of the uniform hot stream and a 64-row band centred on a shear layer, each
    n wide with zero-gradient ends in y. Their per-node times are weighted by
    the full flow's row mix (128 of n rows lie in the two layers)."""
    import oracle as O
    f = flows.shear_layer(n)
    rows = 64
    bands = {"uniform": 0, "layer": n // 4 - rows // 2}
    per_node = {}
    total_time = 0.0
    for name, y0 in bands.items():
        band = [a[y0:y0 + rows].copy() for a in f]
        s = O.Simulation(O.make_config(n, rows, umax=2, nu=NU, bc_y=O.ZERO_GRADIENT))
        assert s.init(*band) == O.OK
        if warmup:
            s.step(warmup)
        t0 = time.perf_counter()
        s.step(steps)
        dt = time.perf_counter() - t0
        total_time += dt
        per_node[name] = dt / (steps * n * rows)
    frac_layer = min(1.0, 2 * rows / n)
    t_node = (1 - frac_layer) * per_node["uniform"] + frac_layer * per_node["layer"]
    return {"mlups": 1e-6 / t_node, "time_s": total_time,
            "sample": "two %dx%d bands (uniform stream; shear layer), %d steps each, per-node "
                      "times weighted by the %d^2 flow's row mix" % (n, rows, steps, n)}


# ----------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    if rank != 0:
        return
    cores = os.cpu_count()
    t0 = time.perf_counter()
    res = oracle_sample(args.n, max(1, args.steps // 10), warmup=min(1, args.warmup))
    line = {
        "metric": METRIC, "value": round(res["mlups"], 4), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "impl": "reference",
        "ms_per_step": round(1e3 * args.n * args.n / (res["mlups"] * 1e6), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "shear layer %dx%d, FP64 CPU oracle" % (args.n, args.n)},
        "cpu_baseline": {"value": round(res["mlups"], 4), "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": res["sample"]},
        "e2e": {"value": round(res["mlups"], 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": round(time.perf_counter() - t0, 1),
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm

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
        fl = alb.Flow(n, n, u_max=2, nu=NU, precision=precision, stream=stream)
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
    mlups = world * N * args.steps / (ms_max * 1e-3) / 1e6
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
        extra["fp64_plain"] = {"value": round(N * k64 / (ms64 * 1e-3) / 1e6, 2), "unit": UNIT,
                               "steps": k64, "ms_per_step": round(ms64 / k64, 3)}
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
    st = fl32.stats()
    fl32.close()

    e2e = None
    if not args.no_e2e:
        pinned = [torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).pin_memory() for a in fields]
        outs = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(4)]
        fl = alb.Flow(n, n, u_max=2, nu=NU, precision=alb.ALB_FP32_FORM, stream=stream)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        alb.alb_init(fl.h, *[p.numpy() for p in pinned])
        alb.alb_step(fl.h, args.steps)
        alb.alb_moments(fl.h, [o.numpy() for o in outs])
        dt = time.perf_counter() - t0
        dt = dist_max(dt, world)
        fl.close()
        e2e = {"value": round(world * N * args.steps / dt / 1e6, 2), "unit": UNIT,
               "h2d_bytes_per_step": int(4 * N * 8 / args.steps),
               "d2h_bytes_per_step": int(4 * N * 8 / args.steps),
               "note": "alb_init from pinned host fields + steps + alb_moments to pinned host, "
                       "wall clock; bytes are the per-run copies divided by the steps"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        res = oracle_sample(n, 2, warmup=1)
        cpu = {"value": round(res["mlups"], 4), "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle", "sample": res["sample"]}

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(mlups, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "shear layer %dx%d periodic, Mach 2.5 cold stream, T ratio 3, "
                               "nu 1e-5, FP32 populations, FP64 Newton" % (n, n),
                   "nodes": N, "u_max": 2, "l2_flush": "not needed: 5.7 GB state >> L2",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "achieved": round(achieved_tflops, 4),
                     "peak": round(costmodel.FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                     "frac": round(achieved_tflops / costmodel.FP64_PEAK_TFLOPS, 4),
                     "traffic": None,
                     "peak_source": "FP64: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz",
                     "kernel": "step_kernel<float>",
                     "fp64_slots_per_node": round(slots / args.steps / N, 1),
                     "hbm": {"achieved_gbs": round(hbm_gbs, 1),
                             "bytes_per_node": costmodel.BYTES_PER_NODE["fp32"]}},
        "clocks": clk,
        "gpu_launches": args.steps,
        "counters": {k: st[k] for k in ("newton_iterations", "newton_calls", "fp64_evaluations",
                                        "fp32_iterations", "reconstructions",
                                        "newton_failures", "reconstruction_failures")},
    }
    line.update(extra)
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
