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

The line also carries "forms": each chosen execution form against its plain
counterpart on the same inputs at the same accuracy -- the fused graph-replayed
CH step vs one launch per step vs the plain two-pass step (2048^2); the
256-instance AC ensemble in one persistent launch vs per-step vs per-instance
launches; the coupled Allen-Cahn / Cahn-Hilliard step (2048^2); the checkpointed adjoint vs the forward trajectory (512^2, 2000
steps); and Newton from the learned warm start vs the plain U^n start for 200
implicit grain-growth steps on 128^3 x 8 fields (surrogate trained in the run
on trajectories from other seeds; the zero-correction ablation -- quadratic
extrapolation through the same network path -- is reported beside it).
--no-forms skips them.

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
# FP32 flop per node of the fused CH step, counted from the kernel's sweep (one
# lane = two nodes): 28 packed FMA (x 2 lanes x 2 flop) + 13 packed add/sub
# (x 2) + 8 scalar add/sub = 146 per lane-row; the warm-up rows of each band
# and the halo lanes of each strip are excluded (they repeat this work).
FLOP_PER_NODE_STEP = 73
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # FP32 lanes x 2 flop x max SM clock
_FP32_PEAK = {}


def fp32_peak(dev, stream):
    """FP32 FMA throughput measured on this GPU in this run (pf_fp32_peak),
    the peak of the ALU rooflines."""
    import torch

    from paper_2601_06079_gb300 import _lib
    if dev not in _FP32_PEAK:
        sink = torch.zeros(4, dtype=torch.float32, device=dev)
        vals = []
        for _ in range(3):
            st, t = _lib.pf_fp32_peak(stream.cuda_stream, sink.data_ptr())
            if st != 0:
                raise RuntimeError(f"pf_fp32_peak failed ({st})")
            vals.append(t)
        _FP32_PEAK[dev] = max(vals)
    return _FP32_PEAK[dev]
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


def job_rate(t_local, units_local, device=None):
    """Whole-job throughput over the ranks of the default process group: the
    units all ranks processed divided by the slowest rank's time (max over
    ranks).  Returns (rate, t_max).  Without an initialised group it is the
    local rate.  `device` holds the reduction tensors (a CUDA device under
    NCCL, None = CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units_local / t_local, t_local
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


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
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix=f"pf_clocks_rank{index}_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        try:
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
    nodes = N_SIDE * N_SIDE
    value, t_total = job_rate(sum(times), nodes * DOF_PER_NODE * N_TSTEPS * args.steps, dev)
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
    e2e_value, t_e2e = job_rate(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3,
                                nodes * DOF_PER_NODE * N_TSTEPS * args.steps, dev)

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    achieved = ALG_BYTES_PER_NODE_STEP * nodes / step_launch_s / 1e9
    alu_peak = fp32_peak(dev, stream)
    alu_achieved = FLOP_PER_NODE_STEP * nodes / step_launch_s / 1e12
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
        # both planes stay in L2 over a trajectory: the FP32 pipe binds, so the
        # same kernel against the measured FP32 FMA peak
        "roofline_alu": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": alu_achieved / alu_peak,
                         "flop_per_node": FLOP_PER_NODE_STEP,
                         "peak_source": "measured FP32 FMA (pf_fp32_peak, this run)",
                         "nominal_peak": NOMINAL_FP32_TFLOPS},
        "e2e": {"value": e2e_value, "unit": "DOF-steps/s",
                "h2d_bytes_per_step": nodes * 4, "d2h_bytes_per_step": nodes * 4 + 16},
        "gpu_launches": args.steps * (N_TSTEPS + 4),
        "clocks": clk.summary(),
    }
    if not args.no_forms:
        line["forms"] = {"explicit_ch_2048": forms_explicit(dev, stream, flush, c0_host),
                         "ensemble_256_ac": forms_ensemble(dev, stream, flush),
                         "coupled_acch_2048": forms_coupled(dev, stream, flush),
                         "implicit_2d_2048": forms_implicit_2d(dev, stream),
                         "implicit_adjoint_ac_1024": forms_implicit_adjoint(dev, stream),
                         "adjoint_ch_512": forms_adjoint(dev, stream),
                         "implicit_warm_start_128": forms_warm_start(dev),
                         "eshelby_129": forms_eshelby(dev, stream, flush),
                         "jvp_128_fanchen8": forms_jvp(dev, stream, flush)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _rel(a, b):
    import torch
    a, b = a.double(), b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _timed(stream, fn, flush=None):
    """Device time (s) of fn() on `stream`, CUDA events, L2 flushed before."""
    import torch
    if flush is not None:
        flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def forms_explicit(dev, stream, flush, c0_host, n_steps=2048):
    """CH 2048^2: fused + graph (default) vs fused per launch vs plain two-pass."""
    import torch

    import paper_2601_06079_gb300 as pf
    solver = pf.Solver((N_SIDE, N_SIDE), h=1.0, model="ch", device=dev, stream=stream)
    solver.set_params(**PAR, shift=0.5)
    c = torch.empty((N_SIDE, N_SIDE), dtype=torch.float32, device=dev)
    out, res = {}, {}
    for form in ("fused_graph", "fused_stream", "two_pass"):
        solver.set_form(form)
        c.copy_(c0_host)
        solver.step_explicit(c, 128)  # warm (graph capture, caches)
        c.copy_(c0_host)
        t = _timed(stream, lambda: solver.step_explicit(c, n_steps), flush)
        res[form] = c.clone()
        nodes = N_SIDE * N_SIDE
        out[form] = {"dof_steps_per_s": nodes * DOF_PER_NODE * n_steps / t,
                     "us_per_step": 1e6 * t / n_steps,
                     "hbm_frac_of_measured_at_8B": 8 * nodes * n_steps / t / 1e9 / _peaks()[0]}
    for form in ("fused_stream", "two_pass"):
        out[form]["rel_l2_vs_fused_graph"] = _rel(res[form], res["fused_graph"])
        out[form]["fused_graph_speedup"] = (out[form]["us_per_step"] /
                                            out["fused_graph"]["us_per_step"])
    out["steps"] = n_steps
    out["accuracy_gate"] = "each form <= 1e-5 rel L2 vs the FP64 oracle (tests/test_gpu_forms.py)"
    return out


def forms_coupled(dev, stream, flush, n=2048, n_steps=1000):
    """Coupled Allen-Cahn / Cahn-Hilliard (Eq. 7 with the Supp. 3 polynomials):
    the fused step on a 2048^2 mesh (3 DOF per node: c, mu, eta; 16 algorithmic
    bytes per node-step: c and eta read and written)."""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    s = pf.Solver((n, n), h=1.0, model="coupled", device=dev, stream=stream)
    s.set_params(kappa=0.3, mobility=1.0, mobility2=150.0, dt=1e-3)
    U0 = torch.from_numpy(G.coupled_initial(1, (n, n))).to(dev)
    U = U0.clone()
    s.step_explicit(U, 16)
    U.copy_(U0)
    t = _timed(stream, lambda: s.step_explicit(U, n_steps), flush)
    nodes = n * n
    return {"mesh": f"{n}x{n}", "steps": n_steps, "dof_per_node": 3,
            "M_c": 1.0, "M_eta": 150.0, "kappa_eta": 0.3, "dt": 1e-3,
            "dof_steps_per_s": 3 * nodes * n_steps / t, "us_per_step": 1e6 * t / n_steps,
            "hbm_frac_of_measured_at_16B": 16 * nodes * n_steps / t / 1e9 / _peaks()[0],
            "accuracy_gate": "<= 1e-5 rel L2 per field vs the FP64 oracle "
                             "(tests/test_gpu_coupled.py)"}


def forms_implicit_2d(dev, stream, n=2048, n_steps=50):
    """2-D implicit backward-Euler steps at the paper's benchmark setting (50
    implicit steps, Fig. 4): Allen-Cahn and split Cahn-Hilliard on 2048^2 with
    dt = 1, 1,000x the explicit CH step of the headline; the explicit step count
    for the same simulated time is given beside it."""
    import numpy as np
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    out = {}
    for model, par, init in (("ac", dict(W=1.0, kappa=1.0, mobility=1.0, dt=1.0),
                              lambda: G.ac_initial(1, (n, n))),
                             ("ch", dict(W=1.0, kappa=0.5, mobility=1.0, dt=1.0),
                              lambda: G.ch_initial(1, (n, n)))):
        s = pf.Solver((n, n), h=1.0, model=model, device=dev, stream=stream)
        s.set_params(**par)
        U = torch.from_numpy(init()).to(dev)
        s.step_implicit(U.clone(), 1)  # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.step_implicit(U, n_steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        dofs = (2 if model == "ch" else 1) * n * n
        out[model] = {"mesh": f"{n}x{n}", "steps": n_steps, "dt": par["dt"],
                      "newton_iters": st["newton_iters"], "gmres_iters": st["gmres_iters"],
                      "converged": bool(st["converged"]), "seconds": t,
                      "ms_per_step": 1e3 * t / n_steps,
                      "dof_steps_per_s": dofs * n_steps / t}
    out["ch"]["explicit_steps_for_same_time"] = int(n_steps * 1.0 / PAR["dt"])
    out["newton_rtol"] = 1e-5
    out["accuracy_gate"] = ("Newton roots vs the oracle's FP64 Newton steps "
                            "(tests/test_gpu_implicit.py)")
    return out


def forms_implicit_adjoint(dev, stream, n=1024, n_steps=10):
    """Sensitivities of an implicit Allen-Cahn trajectory (Supp. 2 adjoint;
    objective of Eq. 19, theta = (L, kappa)) on 1024^2, dt 0.5: the forward
    trajectory alone vs forward + reverse sweep."""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    s = pf.Solver((n, n), h=1.0, model="ac", device=dev, stream=stream)
    s.set_params(W=1.0, kappa=1.0, mobility=1.0, dt=0.5)
    U0 = torch.from_numpy(G.ac_initial(2, (n, n), 0.2, 0.8)).to(dev)
    s.implicit_adjoint(U0, 1)  # warm
    U = U0.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fwd = s.step_implicit(U, n_steps)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    O, g, st = s.implicit_adjoint(U0, n_steps)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    return {"mesh": f"{n}x{n}", "steps": n_steps, "dt": 0.5, "objective": O, "grads": g,
            "forward_s": t_fwd, "forward_plus_adjoint_s": t_adj,
            "adjoint_over_forward": t_adj / t_fwd,
            "forward_gmres_iters": fwd["gmres_iters"], "total_gmres_iters": st["gmres_iters"],
            "accuracy_gate": "<= 0.1 per mille (L and kappa) vs the FP64 oracle adjoint in "
                             "the Table 1 setting (tests/test_gpu_implicit.py)"}


def forms_eshelby(dev, stream, flush, n=129):
    """Eshelby inclusion (Eq. 3-4, eigenstrain of Supp. 3 Eq. III.1, objective
    and sensitivities of Eq. 21-22) on the 100^3 cube with n^3 nodes, E = 22.5,
    nu = 0.3, m = 0.01, l = 0.5, a = 20: the stiffness operator alone (L2
    flushed before each launch), the CG solve (rtol 1e-6) and the volume with
    its adjoint sensitivities (two solves)."""
    import torch

    import paper_2601_06079_gb300 as pf
    h = 100.0 / (n - 1)
    el = pf.Elastic((n, n, n), h, E=22.5, nu=0.3, m=0.01, l=0.5, a=20.0, device=dev,
                    stream=stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1)
    u = torch.rand((3, n, n, n), generator=gen, device=dev) * 2 - 1
    out = el.empty()
    for _ in range(3):
        el.apply(u, out)
    t_apply = sorted(_timed(stream, lambda: el.apply(u, out), flush) for _ in range(21))[10]
    nodes = n ** 3
    # per interior node: 13 mirror pairs x 3 components x 3 adds (two
    # differences and their sum) + 75 FMA (39 diagonal, 36 nonzero couplings)
    flop = 13 * 3 * 3 + 2 * 75
    peak_tflops = fp32_peak(dev, stream)
    el.solve(rtol=1e-6)  # warm
    x = el.empty()
    t_solve = _timed(stream, lambda: el.solve(u=x, rtol=1e-6))
    it_solve = el.stats.iterations
    res = {}

    def sens():
        res["out"] = el.sensitivity(u=x, rtol=1e-6)
    t_sens = _timed(stream, sens)
    V, grads, _ = res["out"]
    return {"mesh": f"{n}^3 nodes, h = {h:g}", "dof": 3 * nodes,
            "apply_us": t_apply * 1e6,
            "apply_roofline": {"bound": "alu", "achieved": flop * nodes / t_apply / 1e12,
                               "peak": peak_tflops, "unit": "TFLOP/s",
                               "peak_source": "measured FP32 FMA (pf_fp32_peak, this run)",
                               "frac": flop * nodes / t_apply / 1e12 / peak_tflops,
                               "hbm_gbs_at_24B_per_node": 24 * nodes / t_apply / 1e9},
            "solve_ms": t_solve * 1e3, "cg_iterations": it_solve,
            "dof_iterations_per_s": 3 * nodes * it_solve / t_solve,
            "sensitivity_ms": t_sens * 1e3, "sensitivity_cg_iterations": el.stats.iterations,
            "volume_change": V - 100.0 ** 3, "dV_dE": grads["E"], "dV_dnu": grads["nu"],
            "accuracy_gate": "operator and loads <= 2e-6 rel vs the FP64 oracle; solution, "
                             "objective <= 1e-5 and dO/dnu <= 1e-4 vs the oracle adjoint "
                             "(tests/test_gpu_elastic.py)"}


def forms_jvp(dev, stream, flush, n=128):
    """The Jacobian-vector product of the implicit step (Eq. 14; Fan-Chen
    Hessian, 8 order parameters, 128^3 nodes) alone, L2 flushed before each
    launch: against HBM (96 B per node: U, v in, J v out) and against the FP32
    ALU, counting per node (one element per node) the Gauss values of U and v
    for 8 fields (960 flop), S2 and T (256), the Hessian action (512), the
    gradient term (240), the weights back (1,104) and the gather (96)."""
    import paper_2601_06079_gb300 as pf  # noqa: F401
    import pf_inputs as G
    import torch
    from paper_2601_06079_gb300 import warmstart as WS
    solver = WS.grain_solver(n, device=dev)
    U = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).to(dev)
    v = torch.from_numpy(G.random_field(2, (8, n, n, n))).to(dev)
    out = torch.empty_like(U)
    for _ in range(3):
        solver.jvp(U, v, out)
    t = sorted(_timed(stream, lambda: solver.jvp(U, v, out), flush) for _ in range(11))[5]
    nodes = n ** 3
    hbm, _ = _peaks()
    flop = 960 + 256 + 512 + 240 + 1104 + 96
    peak_tflops = fp32_peak(dev, stream)
    return {"mesh": f"{n}^3 nodes x 8 order parameters", "us": t * 1e6,
            "hbm": {"achieved_gbs": 96 * nodes / t / 1e9, "peak_gbs": hbm,
                    "frac": 96 * nodes / t / 1e9 / hbm},
            "alu": {"flop_per_node": flop, "achieved_tflops": flop * nodes / t / 1e12,
                    "peak_tflops": peak_tflops, "frac": flop * nodes / t / 1e12 / peak_tflops,
                    "peak_source": "measured FP32 FMA (pf_fp32_peak, this run)"},
            "accuracy_gate": "<= 2e-6 rel vs the FP64 oracle JVP (tests/test_gpu_implicit.py)"}


def forms_ensemble(dev, stream, flush, n_steps=1000):
    """256 uneven AC instances: one persistent graph-captured launch vs one
    launch per step vs one fused launch per instance and step."""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    inst = G.batched_instances(1, count=256)
    shapes = [(p["n"], p["n"]) for p in inst]
    e = pf.Ensemble(shapes, device=dev, stream=stream)
    e.set_params([dict(W=p["W"], kappa=p["kappa"], L=p["L"], dt=0.01) for p in inst])
    fields = [G.ac_initial(1 + i, s) for i, s in enumerate(shapes)]
    st0 = e.pack(fields)
    ty, tune = e.tune(reps=10)
    nodes = int(st0.numel())
    per_class = {}
    for (nx, ny), t, pol in zip(shapes, ty, tune["l2"]):
        per_class.setdefault(f"{nx}x{ny}", {"band_rows": t, "l2": pol})
    uni = {f"{t}/{pol}": v for (t, pol), v in tune["uniform_us"].items()}
    best_uniform = min(uni, key=uni.get)
    out, res = {"instances": 256, "nodes": nodes, "steps": n_steps,
                "tuned_schedule_per_size_class": dict(sorted(per_class.items())),
                "autotuner": {"uniform_us_per_step": uni,
                              "best_uniform": best_uniform,
                              "tuned_us_per_step": tune["tuned_us"],
                              "gain_over_best_uniform": uni[best_uniform] / tune["tuned_us"]}}, {}
    for mode in ("persistent", "per_step", "plain"):
        st = st0.clone()
        e.step(st, 8, mode)  # warm
        st.copy_(st0)
        t = _timed(stream, lambda: e.step(st, n_steps, mode), flush)
        res[mode] = st
        out[mode] = {"node_steps_per_s": nodes * n_steps / t, "ms": 1e3 * t,
                     "hbm_frac_of_measured_at_8B": 8 * nodes * n_steps / t / 1e9 / _peaks()[0]}
    for mode in ("per_step", "plain"):
        out[mode]["bitwise_equal_to_persistent"] = bool(torch.equal(res[mode], res["persistent"]))
        out[mode]["persistent_speedup"] = out[mode]["ms"] / out["persistent"]["ms"]
    return out


def forms_warm_start(dev, n=128, n_eval=200, seeds=4, traj_steps=100, iters=2000, lr=3e-4):
    """3-D grain growth (8 Fan-Chen order parameters, 128^3, dt 0.5): Newton
    from the plain U^n start vs the learned history-2 surrogate (trained here
    on trajectories from other seeds) vs its zero-correction ablation (pure
    quadratic extrapolation through the same network path), same Newton
    tolerance."""
    import numpy as np
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    from paper_2601_06079_gb300 import warmstart as WS
    solver = WS.grain_solver(n, device=dev)
    t0 = time.perf_counter()
    data = WS.trajectories(solver, seeds=list(range(101, 101 + seeds)), n_steps=traj_steps)
    t_data = time.perf_counter() - t0
    surr = pf.Surrogate(device=dev, history=2)
    surr.init(seed=7, last_layer_scale=0.0)
    t0 = time.perf_counter()
    losses = WS.train(surr, data, iters=iters, crop=64, batch=4, lr=lr, seed=1, stiff=0.5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del data
    zero = pf.Surrogate(device=dev, history=2)
    zero.init(seed=7, last_layer_scale=0.0)
    U0 = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).to(dev)
    out = {"mesh": f"{n}^3 nodes x 8 order parameters", "dt": 0.5, "steps": n_eval,
           "newton_rtol": 1e-5, "history": 2,
           "train": {"trajectories": f"seeds 101..{100 + seeds}, {traj_steps} steps each",
                     "iters": iters, "lr": lr, "seconds_data": t_data, "seconds_train": t_train,
                     "loss_first_last_50": [float(np.mean(losses[:50])),
                                            float(np.mean(losses[-50:]))]}}
    res = {}
    WS.run(solver, U0, 4, None)  # warm
    for name, s in (("plain", None), ("learned", surr), ("zero_correction_ablation", zero)):
        U, tot, r0 = WS.run(solver, U0, n_eval, s)
        res[name] = U
        out[name] = {"newton_iters": tot["newton_iters"], "gmres_iters": tot["gmres_iters"],
                     "seconds": tot["seconds"], "predict_seconds": tot["predict_seconds"],
                     "mean_initial_residual": float(np.mean(r0))}
    for name in ("learned", "zero_correction_ablation"):
        out[name]["rel_l2_end_state_vs_plain"] = _rel(res[name], res["plain"])
        out[name]["speedup_vs_plain"] = out["plain"]["seconds"] / out[name]["seconds"]
    # what the trained correction adds on its own: its share of the Newton
    # iterations the learned start saves against the plain start, and the
    # time against the same network path with a zero correction
    saved = out["plain"]["newton_iters"] - out["learned"]["newton_iters"]
    by_net = out["zero_correction_ablation"]["newton_iters"] - out["learned"]["newton_iters"]
    out["learned_share"] = {
        "newton_iters_saved_vs_plain": saved,
        "of_which_by_the_trained_correction": by_net,
        "fraction": by_net / saved if saved else None,
        "seconds_learned_over_ablation": (out["learned"]["seconds"] /
                                          out["zero_correction_ablation"]["seconds"]),
        "reading": "the saving against the plain start comes from extrapolation through "
                   "three states; the trained correction's own share is the fraction above"}
    return out


def forms_adjoint(dev, stream, n=512, n_steps=2000, ckpt=100):
    """CH 512^2, 2000 steps with a per-node mobility field: loss + all gradients
    by the checkpointed discrete adjoint vs the forward trajectory alone."""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    mob = torch.from_numpy(G.gaussian_mobility(3, (n, n))).to(dev)
    c0 = torch.from_numpy(G.ch_initial(5, (n, n))).to(dev)
    s = pf.Solver((n, n), h=1.0, model="ch", device=dev, stream=stream)
    s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3, mobility_field=mob)
    target = c0.clone()
    s.step_explicit(target, n_steps)
    c = c0.clone()
    s.step_explicit(c, 64)
    c.copy_(c0)
    t_fwd = _timed(stream, lambda: s.step_explicit(c, n_steps))
    s.adjoint(c0, target, 200, ckpt)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss, g = s.adjoint(c0, target, n_steps, ckpt)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    # algorithmic bytes per node: forward step with the mobility field 12 B
    # (c in, c out, m in); reverse step 24 B (lambda in, c^n, m, lambda out, the
    # FP64 mobility-gradient read-modify-write counted as 8 B of FP32 traffic);
    # the checkpointed recompute repeats the forward step: 36 B per reverse step
    hbm, kind = _peaks()
    nodes = n * n
    t_rev = max(t_adj - t_fwd, 1e-12)  # recompute + reverse, after the checkpointing forward
    rev_gbs = 36 * nodes * n_steps / t_rev / 1e9
    return {"mesh": f"{n}x{n}", "steps": n_steps, "checkpoint_every": ckpt,
            "forward_ms": 1e3 * t_fwd, "adjoint_ms": 1e3 * t_adj,
            "adjoint_over_forward": t_adj / t_fwd,
            "reverse_step_us": 1e6 * t_rev / n_steps,
            "reverse_roofline": {"bound": "hbm", "bytes_per_node": 36, "achieved": rev_gbs,
                                 "peak": hbm, "unit": "GB/s", "frac": rev_gbs / hbm,
                                 "peak_source": f"{kind} hbm_gbs",
                                 "note": "per reverse step incl. its recompute; 512^2 planes "
                                         "stay in L2"},
            "gradients": "kappa, W, M, 262,144-entry mobility field, c0",
            "accuracy_gate": "<= 1e-4 vs central FD and the oracle adjoint (tests/test_gpu_adjoint.py)"}


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
    # the same oracle on one thread, over a shorter sample
    single = max(1, sample_steps // 10)
    O.set_threads(1)
    t = time.perf_counter()
    P.ch_explicit(c0, PAR["dt"], single)
    dt1 = time.perf_counter() - t
    O.set_threads(0)
    return {"value": N_SIDE * N_SIDE * DOF_PER_NODE * sample_steps / dt, "unit": "DOF-steps/s",
            "cores": cores, "kind": "oracle",
            "sample": f"{sample_steps} time steps of the 2048x2048 CH mesh (FP64, OpenMP over "
                      f"element colours), {dt:.1f} s",
            "single_thread": {"value": N_SIDE * N_SIDE * DOF_PER_NODE * single / dt1,
                              "sample": f"{single} time steps on one thread, {dt1:.1f} s"}}


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
    """Untimed launches of one workload for ncu captures (--target):
    ch        the bench's CH 2048^2 trajectory (--tsteps steps per trajectory)
    surrogate two warm-start predictions on 128^3 x 8 fields (tcgen05 convolutions)
    jvp       three Fan-Chen Jacobian-vector products on 128^3 x 8 fields
    residual  three Fan-Chen implicit residuals on 128^3 x 8 fields
    adjoint   the checkpointed CH adjoint with a mobility field on 512^2 (200 steps,
              checkpoint every 100): forward, recompute and reverse launches
    newton    one implicit grain-growth step on 128^3 x 8 fields (after three
              warm-up steps) inside a profiler range, for ncu
              --profile-from-start off
    newton2d  one implicit split Cahn-Hilliard step on 2048^2 (dt 1, after three
              warm-up steps) inside a profiler range, for ncu
              --profile-from-start off
    ensemble  20 steps of the 256-instance AC ensemble, one launch per step (the
              persistent mode runs the same task body behind a grid barrier)
    coupled   20 coupled Allen-Cahn / Cahn-Hilliard steps on 2048^2
    elastic   five Eshelby stiffness applications on 129^3 x 3 components
    train     four surrogate training steps (history 2, 4 x 64^3 crops, stiffness
              weight 0.5): forward, loss, backward with the tcgen05 weight gradient,
              Adam"""
    import torch

    import paper_2601_06079_gb300 as pf
    import pf_inputs as G

    if args.target == "ch":
        c = torch.from_numpy(G.ch_initial(1, (N_SIDE, N_SIDE))).cuda()
        solver = pf.Solver((N_SIDE, N_SIDE), h=1.0, model="ch")
        solver.set_params(**PAR, shift=0.5)
        for _ in range(args.warmup + args.steps):
            solver.step_explicit(c, args.tsteps)
        E, M = solver.energy(c)
        torch.cuda.synchronize()
        print(f"profile run done: energy {E:.6f} mass {M:.6f}")
    elif args.target == "surrogate":
        n = 128
        s = pf.Surrogate(history=True)
        s.init(seed=1, last_layer_scale=1.0)
        u = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).cuda()
        x = torch.cat([u, 0.99 * u]).reshape(1, 16, n, n, n).contiguous()
        for _ in range(2):
            out = s.predict(x)
        torch.cuda.synchronize()
        print(f"profile run done: guess norm {float(out.norm()):.6f}")
    elif args.target == "jvp":
        from paper_2601_06079_gb300 import warmstart as WS
        n = 128
        solver = WS.grain_solver(n)
        U = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).cuda()
        v = torch.from_numpy(G.random_field(2, (8, n, n, n))).cuda()
        for _ in range(3):
            jv = solver.jvp(U, v)
        torch.cuda.synchronize()
        print(f"profile run done: |Jv| {float(jv.norm()):.6f}")
    elif args.target == "residual":
        from paper_2601_06079_gb300 import warmstart as WS
        n = 128
        solver = WS.grain_solver(n)
        U = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).cuda()
        Un = torch.from_numpy(G.voronoi_grains(2, n=n, n_seeds=64, n_op=8)).cuda()
        for _ in range(3):
            r = solver.implicit_residual(Un, U)
        torch.cuda.synchronize()
        print(f"profile run done: |R| {float(r.norm()):.6f}")
    elif args.target == "adjoint":
        n = 512
        mob = torch.from_numpy(G.gaussian_mobility(3, (n, n))).cuda()
        c0 = torch.from_numpy(G.ch_initial(5, (n, n))).cuda()
        s = pf.Solver((n, n), h=1.0, model="ch")
        s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3, mobility_field=mob)
        target = c0.clone()
        s.step_explicit(target, 200)
        loss, g = s.adjoint(c0, target, 200, 100)
        torch.cuda.synchronize()
        print(f"profile run done: loss {loss:.6e}")
    elif args.target == "newton":
        from paper_2601_06079_gb300 import warmstart as WS
        n = 128
        solver = WS.grain_solver(n)
        U = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=64, n_op=8)).cuda()
        for _ in range(3):
            solver.step_implicit(U, 1)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()  # ncu --profile-from-start off: this step only
        st = solver.step_implicit(U, 1)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(f"profile run done: {st['newton_iters']} Newton, {st['gmres_iters']} GMRES")
    elif args.target == "newton2d":
        n = N_SIDE
        solver = pf.Solver((n, n), h=1.0, model="ch")
        solver.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=1.0)
        U = torch.from_numpy(G.ch_initial(1, (n, n))).cuda()
        solver.step_implicit(U, 3)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()  # ncu --profile-from-start off: this step only
        st = solver.step_implicit(U, 1)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        print(f"profile run done: {st['newton_iters']} Newton, {st['gmres_iters']} GMRES")
    elif args.target == "elastic":
        n = 129
        el = pf.Elastic((n, n, n), 100.0 / (n - 1))
        u = torch.from_numpy(G.random_field(3, (3, n, n, n))).cuda()
        for _ in range(5):
            Ku = el.apply(u)
        torch.cuda.synchronize()
        print(f"profile run done: |Ku| {float(Ku.norm()):.6f}")
    elif args.target == "train":
        s = pf.Surrogate(history=2)
        s.init(seed=1, last_layer_scale=0.1)
        x = torch.from_numpy(G.random_field(6, (4, 24, 64, 64, 64), 0.0, 1.0)).cuda()
        y = x[:, :8].clone() + 0.01 * torch.from_numpy(G.random_field(7, (4, 8, 64, 64, 64))).cuda()
        losses = [s.train_step(x, y, lr=1e-4, stiff=0.5) for _ in range(4)]
        torch.cuda.synchronize()
        print(f"profile run done: losses {losses}")
    elif args.target == "coupled":
        s = pf.Solver((N_SIDE, N_SIDE), h=1.0, model="coupled")
        s.set_params(kappa=0.3, mobility=1.0, mobility2=150.0, dt=1e-3)
        U = torch.from_numpy(G.coupled_initial(1, (N_SIDE, N_SIDE))).cuda()
        s.step_explicit(U, 20)
        torch.cuda.synchronize()
        print(f"profile run done: mean eta {float(U[1].mean()):.6f}")
    else:
        inst = G.batched_instances(1, count=256)
        shapes = [(p["n"], p["n"]) for p in inst]
        e = pf.Ensemble(shapes)
        e.set_params([dict(W=p["W"], kappa=p["kappa"], L=p["L"], dt=0.01) for p in inst])
        st = e.pack([G.ac_initial(1 + i, sh) for i, sh in enumerate(shapes)])
        e.step(st, 20, "per_step")
        torch.cuda.synchronize()
        print(f"profile run done: mean {float(st.mean()):.6f}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-steps", type=int, default=40)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the comparison of execution forms (fused/graph/batched/"
                         "warm start/adjoint) against their plain counterparts")
    ap.add_argument("--profile", action="store_true",
                    help="run one workload untimed for ncu (see --target)")
    ap.add_argument("--tsteps", type=int, default=N_TSTEPS)
    ap.add_argument("--target", default="ch",
                    choices=["ch", "surrogate", "jvp", "residual", "newton", "newton2d", "adjoint",
                             "ensemble",
                             "coupled",
                             "elastic", "train"],
                    help="workload of --profile")
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
