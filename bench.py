"""Throughput of the fused explicit Cahn-Hilliard step on one GB300.

Workload: 2-D Cahn-Hilliard spinodal decomposition, split form (c, mu), on a
2048 x 2048 node Q1 mesh (4,194,304 nodes, 2 DOF per node), f = c^2 (1-c)^2,
kappa = 0.5, M = 1, explicit Euler dt = 1e-3, 10,000 steps, c0 = 0.5 +
U(-0.05, 0.05) from a seed, FP32 state with FP64 mass/energy diagnostics.
One bench step = one whole trajectory (10,000 time steps) plus the FP64
energy/mass evaluation of its end state.

Metric: DOF-steps/s (DOF = nodes x 2 for the split CH form) and the fraction
of the HBM roofline at 8 algorithmic bytes per node-step.  Between timed
trajectories the L2 is flushed by writing a 512 MiB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other arm this
method has) on a bounded sample of the same workload on the host cores.
With N > 1 (torchrun) every rank runs an independent replica: the method is
one domain on one GPU, so there is no data-path collective ("replicas only").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 2048
N_TSTEPS = 10_000
PAR = dict(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3)
DOF_PER_NODE = 2
ALG_BYTES_PER_NODE_STEP = 8  # read c, write c; mu never leaves the chip
WORKLOAD = "ch2d_2048x2048_10000steps"
KERNEL_SRC = os.path.join(ROOT, "paper_2601_06079_gb300", "csrc", "k_explicit2d.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ch2d_2048_dram_traffic.json")


def _config(extra=None):
    cfg = {"workload": WORKLOAD, "nodes": N_SIDE * N_SIDE, "mesh": f"{N_SIDE}x{N_SIDE} Q1 nodes",
           "time_steps_per_bench_step": N_TSTEPS, "dof_per_node": DOF_PER_NODE, "dt": PAR["dt"],
           "kappa": PAR["kappa"], "M": PAR["mobility"], "W": PAR["W"],
           "l2": "flushed between timed trajectories (512 MiB write)",
           "parallelism": "replicas only (one domain per GPU)"}
    if extra:
        cfg.update(extra)
    return cfg


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank, int(os.environ.get("LOCAL_RANK", "0"))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    null when the kernel source changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        h = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
        if t.get("kernel_sha256_16") != h:
            return None
        return float(t["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            sm = [float(r[1]) for r in rows]
            mx = max(float(r[2]) for r in rows)
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            reasons = sorted({names[i] for r in rows for i in range(4)
                              if r[5 + i].strip().lower() == "active"})
            return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                    "samples": len(rows)}
        except Exception:
            return None


def run_ours(args):
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    c0_host = torch.from_numpy(G.ch_initial(1 + rank, (N_SIDE, N_SIDE))).pin_memory()
    solver = pf.Solver((N_SIDE, N_SIDE), h=1.0, model="ch", device=dev, stream=stream)
    solver.set_params(**PAR, shift=0.5)
    c = torch.empty((N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def trajectory():
        solver.step_explicit(c, N_TSTEPS)
        return solver.energy(c)

    # --- device-resident timing: inputs already in HBM ---
    for _ in range(args.warmup):
        c.copy_(c0_host, non_blocking=True)
        trajectory()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    times = []
    with Clocks(local) as clk:
        barrier()
        for i in range(args.steps):
            c.copy_(c0_host, non_blocking=True)
            flush.zero_()
            ev[i][0].record(stream)
            E, M = trajectory()
            ev[i][1].record(stream)
        barrier()
    for a, b in ev:
        times.append(a.elapsed_time(b) / 1e3)
    t_total = sum(times)
    if ws > 1:
        tt = torch.tensor([t_total], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_total = float(tt.item())
    nodes = N_SIDE * N_SIDE
    value = ws * nodes * DOF_PER_NODE * N_TSTEPS * args.steps / t_total
    ms_per_step = 1e3 * t_total / args.steps
    step_launch_s = t_total / (args.steps * N_TSTEPS)

    # --- end to end through the public API with host buffers ---
    out_host = torch.empty_like(c0_host).pin_memory()
    e2e_ev = []
    barrier()
    for i in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(stream)
        c.copy_(c0_host, non_blocking=True)
        E2, M2 = trajectory()
        out_host.copy_(c, non_blocking=True)
        b.record(stream)
        e2e_ev.append((a, b))
    barrier()
    t_e2e = sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3
    if ws > 1:
        tt = torch.tensor([t_e2e], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_e2e = float(tt.item())
    e2e_value = ws * nodes * DOF_PER_NODE * N_TSTEPS * args.steps / t_e2e

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    achieved = ALG_BYTES_PER_NODE_STEP * nodes / step_launch_s / 1e9
    line = {
        "metric": "DOF-steps/s (CH split form, 2 DOF/node) & %HBM roofline",
        "value": value,
        "unit": "DOF-steps/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64 diagnostics)",
        "data": "synthetic (seeded c0 = 0.5 + U(-0.05, 0.05))",
        "config": _config({"node_steps_per_s": value / DOF_PER_NODE,
                           "end_energy": E, "end_mass": M}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _traffic(),
                     "kernel": "k_explicit2d<CH> (fused mu + c update)",
                     "peak_source": f"{peak_kind} hbm_gbs",
                     "per_launch_s": step_launch_s,
                     "alg_bytes_per_launch": ALG_BYTES_PER_NODE_STEP * nodes},
        "e2e": {"value": e2e_value, "unit": "DOF-steps/s",
                "h2d_bytes_per_step": nodes * 4, "d2h_bytes_per_step": nodes * 4 + 16},
        "gpu_launches": args.steps * (N_TSTEPS + 4),
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(sample_steps):
    """FP64 oracle on the host cores: a bounded sample (sample_steps time steps
    of the full 2048^2 mesh), reported in the bench metric's unit."""
    import oracle as O
    import pf_inputs as G

    c0 = G.ch_initial(1, (N_SIDE, N_SIDE))
    P = O.Problem((N_SIDE, N_SIDE), W=PAR["W"], kappa=PAR["kappa"], mob=PAR["mobility"])
    P.ch_explicit(c0, PAR["dt"], 1)  # load / warm
    t = time.perf_counter()
    P.ch_explicit(c0, PAR["dt"], sample_steps)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N_SIDE * N_SIDE * DOF_PER_NODE * sample_steps / dt, "unit": "DOF-steps/s",
            "cores": cores, "kind": "oracle",
            "sample": f"{sample_steps} time steps of the 2048x2048 CH mesh (FP64, OpenMP over "
                      f"element colours), {dt:.1f} s"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    per = []
    for _ in range(args.warmup):
        cpu_baseline(2)
    for _ in range(args.steps):
        b = cpu_baseline(args.cpu_sample_steps)
        per.append(b)
    value = statistics.median(b["value"] for b in per)
    sample_s = args.cpu_sample_steps * N_SIDE * N_SIDE * DOF_PER_NODE / value
    line = {
        "impl": "reference",
        "metric": "DOF-steps/s (CH split form, 2 DOF/node) & %HBM roofline",
        "value": value, "unit": "DOF-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sample_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config({"reference": "FP64 CPU oracle (element loop), bounded sample"}),
        "cpu_baseline": {"value": value, "unit": "DOF-steps/s", "cores": per[0]["cores"],
                         "kind": "oracle", "sample": per[0]["sample"]},
        "e2e": {"value": value, "unit": "DOF-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Untimed launches of the bench workload for ncu captures."""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G

    c = torch.from_numpy(G.ch_initial(1, (N_SIDE, N_SIDE))).cuda()
    solver = pf.Solver((N_SIDE, N_SIDE), h=1.0, model="ch")
    solver.set_params(**PAR, shift=0.5)
    for _ in range(args.warmup + args.steps):
        solver.step_explicit(c, args.tsteps)
    E, M = solver.energy(c)
    torch.cuda.synchronize()
    print(f"profile run done: energy {E:.6f} mass {M:.6f}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="run --steps trajectories of --tsteps time steps untimed (for ncu)")
    ap.add_argument("--tsteps", type=int, default=N_TSTEPS)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
