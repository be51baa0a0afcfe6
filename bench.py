#!/usr/bin/env python3
"""Benchmark of the differentiable Projective Dynamics hot path.

Default workload (the largest single-GPU configuration): 64x64x128-cell hex
cantilever (545,025 nodes, 1,635,075 DoFs), corotated energy E = 1e6 Pa,
nu = 0.45, x=0 face fixed, gravity plus seeded surface tractions, h = 0.01 s;
forward rollout (PD + L-BFGS, Alg. 1) with a state checkpoint every 25 steps and
the backward pass (adjoint splitting iteration + L-BFGS, Alg. 2, with the states
of each 25-step segment recomputed from its checkpoint, Sec. 4) to the gradients
w.r.t. the traction field and the initial velocity.  Mixed precision: FP32 local
steps and triangular solves, FP64 factor, vectors and convergence checks.

One bench step is one 25-step checkpoint segment: --steps K times a rollout of
T = 25 K simulation steps forward and backward (K = 20 is the configuration's
500-step horizon), after a warm-up rollout of 25 W steps.  `value` = simulated
fwd+bwd steps per second over the timed rollout.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c5|c2] [--serve] [--probe ...]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica (every global step is one sweep over one factor's elimination tree, so a
rollout does not shard across GPUs and no collective is on the data path); value
= all ranks' simulation steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd sim steps/s at 1e-5 rel error vs FP64 oracle; % HBM roofline; p50/p99"
SEG = 25   # simulation steps per checkpoint segment = one bench step (C5)
# FP32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Algorithmic flops per Gauss point of the forward local step with the corotated
# energy (FMA = 2 flops): F - I from the 8 corners (72 FMA), the Green strain
# H + H^T + H^T H (42), cyclic Jacobi on it (4 sweeps x 3 rotations x 40), sigma - 1
# (12), F V (27 FMA), its Givens QR (3 x 30), the stress U diag(sigma - 1) V^T
# (63), the corner forces (72 FMA) and the energy (6).
LOCAL_FLOPS_PER_GP = 144 + 42 + 4 * 3 * 40 + 12 + 54 + 90 + 63 + 144 + 6
# The same for the Neo-Hookean material (no SVD): F - I (144), det(I + H) - 1 (27),
# 1/J and log J (2), F^-T = cof(F)/J (36), H + H^T + H H^T (63), (F F^T - I) F^-T
# (54), the stress (36), the energy (48) and the corner forces (144).
LOCAL_FLOPS_PER_GP_NH = 144 + 27 + 2 + 36 + 63 + 54 + 36 + 48 + 144
# A linear tetrahedron's one point: F - I from its 3 edge vectors (27 FMA) and the
# forces of its 4 vertices (36 FMA) in place of the hexahedron's 8-corner sums
# (72 FMA each), the rest as for a hexahedron's Gauss point.
LOCAL_FLOPS_PER_TET = LOCAL_FLOPS_PER_GP - 144 - 144 + 54 + 72
WORKLOADS = {
    # tol 1e-7: over 50 steps the mixed path at this tolerance stays within 2.5e-8
    # (positions) and 7e-8 (gradients) of the FP64 path at tol 1e-10
    "c5": dict(name="c5_beam_64x64x128_mixed_ckpt25", K=SEG, tol=1e-7, want=("fext", "v0"), iters_per_step=48.1),
    "c2": dict(name="c2_beam_32x32x64_mixed", K=0, tol=1e-8, want=("w_corot", "w_vol", "v0"),
               iters_per_step=182.0),
    # the same beam of the Neo-Hookean material (Sec. 8): L-BFGS with the PD matrix as
    # initial Hessian forward, the splitting iteration on the Neo-Hookean Hessian backward
    "c2nh": dict(name="c2_beam_32x32x64_neohookean_mixed", K=0, tol=1e-8, want=("w_corot", "w_vol", "v0"),
                 iters_per_step=234.0, nh=True),
    # an unstructured tetrahedral beam (jittered 49x25x25 lattice, Delaunay; the
    # material and tolerance of the C2 beam)
    "tetu": dict(name="unstructured_tet_beam_48x24x24_mixed", K=0, tol=1e-8, want=("w_corot", "w_vol", "v0"),
                 iters_per_step=186.8, tet=True),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3,
                    help="bench steps timed: 25-step checkpoint segments (c5) or 100-step rollouts (c2)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=sorted(WORKLOADS))
    ap.add_argument("--tol", type=float, default=None, help="PD / adjoint tolerance (default per workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 (4x4x8 cantilever) line")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the accuracy leg (the profiled mixed rollout against the FP64 path)")
    ap.add_argument("--serve", action="store_true",
                    help="serving workload instead: quadruped requests under Poisson arrivals")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--T", type=int, default=100, help="simulation steps per rollout (c2, --serve, --probe)")
    ap.add_argument("--probe", choices=["solve", "local", "hvp", "rollout", "quadruped"],
                    help="profiling driver (no timing, no JSON): factorise the workload's beam in mixed "
                         "precision, then run --repeat solves / local steps / Hessian products, or one "
                         "rollout of --T steps forward and backward; 'quadruped' = one 16^3 quadruped "
                         "rollout of --T steps")
    ap.add_argument("--repeat", type=int, default=4)
    ap.add_argument("--profile-events", action="store_true",
                    help="probe rollout: time solves and local steps with CUDA events and print the stats")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="pd_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def solve_bytes(mesh, itemsize):
    """Algorithmic bytes of one solve pair (forward + backward sweep): every
    structural nonzero of the solve panels Q_s = [L11^-1; L21 L11^-1] read once per
    sweep, plus the right-hand side read, the intermediate u written and read and
    the solution written (3 columns per node)."""
    import numpy as np
    first = mesh.export("snode_first")
    rp = mesh.export("row_ptr")
    nc = np.diff(first).astype(np.int64)
    nr = np.diff(rp).astype(np.int64)
    nnz = int(np.sum(nr * nc - nc * (nc - 1) // 2))
    nf3 = 3 * int(first[-1])
    return 2 * nnz * itemsize + nf3 * (8 + 8 + 2 * itemsize), nnz


def oracle_sample(workload, iters_per_step, budget_s=20.0):
    """Bounded CPU sample of the FP64 oracle on the same workload, projected to
    fwd+bwd sim steps/s as 1 / (t_iter * iters_per_step) with the GPU path's
    measured forward + backward iterations per step.

    32x32x64 beam: the oracle's one-time setup (its model and the SuperLU factor of
    L_A, like the GPU's factorisation excluded from steps/s) is timed and reported;
    then the oracle's own PD + L-BFGS forward iterations of step 1 (local step,
    grad g, the A^-1 solve, the Armijo line search: oracle/pd_cpu.py) run for about
    budget_s seconds.  64x64x128 beam: SuperLU's factorisation of L_A (540,800
    unknowns) did not finish within 30 minutes on 8 host cores (18.5 GB resident
    when stopped), so the sample times the parts of an oracle iteration that run
    in bounded time, the local step and grad g, and the projection leaves out the
    solve (it over-estimates the oracle's speed)."""
    import numpy as np
    from oracle import pd_cpu
    from oracle.model import Model
    from oracle.tetmesh import TetModel
    sc = _scene(workload, 1)
    cores = os.cpu_count()
    t0 = time.perf_counter()
    model = TetModel(sc) if WORKLOADS[workload].get("tet") else Model(sc)
    if workload == "c5":
        t_setup = time.perf_counter() - t0
        n = 0
        x = sc.x0.copy()
        t0 = time.perf_counter()
        while True:
            loc = model.local(x)
            model.grad_g(x, x, None, loc)
            n += 1
            if time.perf_counter() - t0 >= budget_s:
                break
        t_iter = (time.perf_counter() - t0) / n
        what = (f"{n} FP64 oracle local-step + grad g evaluations on {sc.name} ({t_iter:.2f} s each, "
                f"numpy/LAPACK on {cores} host cores), projected with the GPU path's {iters_per_step:.1f} "
                f"fwd+bwd iterations per step; the oracle's A^-1 solve is excluded (SuperLU did not factor "
                f"L_A at this size within 30 min)")
    else:
        Afac = pd_cpu.ScalarA(model)
        t_setup = time.perf_counter() - t0
        it = {"n": 0}
        t0 = time.perf_counter()

        def stop(k):
            it["n"] = k
            return time.perf_counter() - t0 >= budget_s
        pd_cpu.pd_lbfgs_step(model, Afac, sc.x0, sc.v0, sc.f_ext, None, None, 1e-12, 5, 100000, stop=stop)
        t_iter = (time.perf_counter() - t0) / max(it["n"], 1)
        what = (f"{it['n']} FP64 oracle PD + L-BFGS iterations of step 1 of {sc.name} ({t_iter:.2f} s each: "
                f"local step, grad g, SuperLU A^-1 solve, Armijo line search; numpy/LAPACK on {cores} host "
                f"cores), projected with the GPU path's {iters_per_step:.1f} fwd+bwd iterations per step; "
                f"oracle setup (model + SuperLU factor of L_A) {t_setup:.1f} s, excluded")
    return {"value": 1.0 / (t_iter * iters_per_step), "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": what, "setup_s": t_setup}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    # iterations per step of the GPU path at this workload (measured; used to
    # project the oracle's timed iterations to simulation steps)
    ips = wl["iters_per_step"]
    res = None
    for _ in range(args.warmup):
        oracle_sample(args.workload, ips, budget_s=2.0)
    vals = []
    for _ in range(args.steps):
        res = oracle_sample(args.workload, ips, budget_s=8.0)
        vals.append(res["value"])
    value = statistics.median(vals)
    res["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["name"], "parallelism": "replicas"},
            "cpu_baseline": res,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def whole_job_rate(elapsed_s, sim_steps_per_rank, world, device):
    """(slowest rank's timed seconds, whole-job simulation steps/s): every rank runs
    an independent replica, so the job's rate is all ranks' steps over the slowest
    rank's time (a MAX all-reduce; called by every rank after the closing barrier)."""
    if world > 1:
        import torch
        t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return elapsed_s, world * sim_steps_per_rank / elapsed_s


def _scene(wl, T):
    from workloads import beam_c2, beam_c5, unstructured_tet_beam
    if wl == "tetu":
        sc = unstructured_tet_beam(48, 24, 24, T=T, index=21, E=1e6)
        sc.neohookean = False
        return sc
    sc = beam_c5(T=T) if wl == "c5" else beam_c2(T=T)
    if wl == "c2nh":
        sc.neohookean = True
    return sc


def _profile_key(wl):
    return {"c5": "c5_beam_64x64x128", "c2": "c2_beam_32x32x64", "c2nh": "c2nh_beam_32x32x64",
            "tetu": "tetu_beam_48x24x24"}[wl]


def _traffic(wl):
    """ncu DRAM bytes of one solve pair at this workload, from the committed
    profile summary (profiles/solve_traffic.txt); None when not captured."""
    path = os.path.join(ROOT, "profiles", "solve_traffic.txt")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    e = d.get(_profile_key(wl))
    if not e:
        return None, None
    return e.get("bytes_per_solve"), e.get("source")


def accuracy_leg(mesh, sc, wc, wv, d, Tr, K, roll_m, g_m, want):
    """The metric's error bound, measured: the profiled mixed rollout (the first Tr
    steps of the timed configuration, its gradients included) against the plain FP64
    path at tol 1e-10 on the same mesh, refactorised in FP64.  At the 64x64x128 beam
    no CPU oracle finishes; the FP64 path is pinned to the oracle on smaller meshes
    by the tests."""
    import numpy as np
    import torch
    from paper_2101_05917_gb300 import api
    from paper_2101_05917_gb300 import _native as N
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh.factorize(wc, wv, None, None, h=sc.h, gravity=tuple(sc.gravity), precision=N.PD_PREC_FP64,
                   neohookean=sc.neohookean)
    o = api.solver_opts(tol_fwd=1e-10, tol_bwd=1e-10, max_iter_fwd=5000, max_iter_bwd=5000, checkpoint_every=K)
    r = mesh.forward(d["x0"], d["v0"], Tr, f_ext=d["f"], opts=o)
    g = mesh.backward(r, Tr, d["lw"], f_ext=d["f"], opts=o, want=want)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    x_ref, x = r.x[-1].cpu().numpy(), roll_m.x[-1].cpu().numpy()
    dx, u = x - x_ref, x_ref - sc.x0
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return {"reference": "plain FP64 path at tol 1e-10, same mesh (pinned to the CPU oracle on smaller meshes)",
            "steps": Tr, "position_rel": float(np.linalg.norm(dx) / np.linalg.norm(x_ref)),
            "displacement_rel": float(np.linalg.norm(dx) / np.linalg.norm(u)),
            "component_max_rel": float(np.abs(dx).max() / np.abs(u).max()),
            "grad_rel": {k: rel(g_m[k].cpu().numpy(), g[k].cpu().numpy()) for k in want},
            "fp64_fwd_iters_per_step": r.stats["fwd_iters"] / Tr, "fp64_s": dt}


def fp64_line(dev, steps=5):
    """Plain FP64 method on the 4x4x8 cantilever (675 DoFs, 50 steps, tol 1e-9):
    fwd+bwd sim steps/s with gradients w.r.t. E (through w_corot), nu and v0."""
    import numpy as np
    import torch
    from paper_2101_05917_gb300 import api
    from paper_2101_05917_gb300 import _native as N
    from workloads import cantilever_c1
    sc = cantilever_c1()
    mesh = api.PDMesh.from_scene(sc, device=dev.index or 0)
    wc, wv, _, _ = api.scene_weights(sc, dev)
    mesh.factorize(wc, None, None, None, h=sc.h, gravity=tuple(sc.gravity), precision=N.PD_PREC_FP64)
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    x0, v0, lw, f = tt(sc.x0), tt(sc.v0), tt(sc.loss_w), tt(sc.f_ext)
    opts = api.solver_opts(tol_fwd=sc.tol_fwd, tol_bwd=sc.tol_bwd, max_iter_fwd=5000, max_iter_bwd=5000)
    lat = []

    def one():
        sm = np.zeros(sc.T)
        o = api.solver_opts(tol_fwd=sc.tol_fwd, tol_bwd=sc.tol_bwd, max_iter_fwd=5000, max_iter_bwd=5000,
                            step_ms=sm)
        roll = mesh.forward(x0, v0, sc.T, f_ext=f, opts=o)
        g = mesh.backward(roll, sc.T, lw, f_ext=f, opts=o, want=("w_corot", "v0"))
        return roll, g, sm
    one()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    it = [0, 0]
    for _ in range(steps):
        roll, g, sm = one()
        lat.append(sm)
        it[0] += roll.stats["fwd_iters"]
        it[1] += g["stats"]["bwd_iters"]
    e1.record(stream)
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1) / 1e3
    # dL/dE and dL/dnu through w = E / (1 + nu) (the only energy of this configuration)
    gw = g["w_corot"].cpu().numpy()
    E = np.asarray(sc.youngs)
    gE = gw / (1 + sc.poisson)
    gnu = float(np.sum(gw * (-E / (1 + sc.poisson) ** 2)))
    lat = np.concatenate(lat)
    mesh.close()
    return {"workload": "c1_cantilever_4x4x8_fp64_T50", "value": steps * sc.T / el, "unit": "steps/s",
            "dtype": "f64", "rollouts": steps, "ms_per_rollout": 1e3 * el / steps, "tol": sc.tol_fwd,
            "fwd_iters_per_step": it[0] / (steps * sc.T), "bwd_iters_per_step": it[1] / (steps * sc.T),
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "grad_norms": {"E": float(np.linalg.norm(gE)), "nu": abs(gnu),
                           "v0": float(g["v0"].norm())},
            "bound": "latency (675 DoFs: every launch is a few CTAs)"}


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2101_05917_gb300 import build as _build
    _build.build()
    from paper_2101_05917_gb300 import api
    from paper_2101_05917_gb300 import _native as N

    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    wl = WORKLOADS[args.workload]
    K = wl["K"]
    tol = args.tol if args.tol is not None else wl["tol"]
    seg = K if K > 0 else args.T             # simulation steps per bench step
    T = seg * args.steps if K > 0 else args.T
    sc = _scene(args.workload, T)
    t0 = time.perf_counter()
    mesh = (api.PDMesh.from_tet_scene if wl.get("tet") else api.PDMesh.from_scene)(sc, device=local)
    t_mesh = time.perf_counter() - t0
    wc, wv, _, _ = api.scene_weights(sc, dev)
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    d = {"x0": tt(sc.x0), "v0": tt(sc.v0), "f": tt(sc.f_ext), "lw": tt(sc.loss_w)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh.factorize(wc, wv, None, None, h=sc.h, gravity=tuple(sc.gravity), precision=N.PD_PREC_MIXED,
                   neohookean=sc.neohookean)
    torch.cuda.synchronize()
    t_factor = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    want = wl["want"]

    def opts_for(profile=False, step_ms=None):
        return api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=5000, max_iter_bwd=5000, checkpoint_every=K,
                               profile=profile, step_ms=step_ms)

    def rollout(Tr, inputs, profile=False, step_ms=None):
        o = opts_for(profile, step_ms)
        roll = mesh.forward(inputs["x0"], inputs["v0"], Tr, f_ext=inputs["f"], opts=o)
        g = mesh.backward(roll, Tr, inputs["lw"], f_ext=inputs["f"], opts=o, want=want)
        return roll, g

    # warm-up: W bench steps (one rollout of W segments, or W rollouts)
    if K > 0:
        rollout(seg * args.warmup, d)
    else:
        for _ in range(args.warmup):
            rollout(T, d)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    flush = None
    if K == 0:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
        flush.fill_(1.0)
    torch.cuda.synchronize()
    ev0.record(stream)
    fstats, bstats, lat = [], [], []
    h0 = time.perf_counter()
    rollouts = 1 if K > 0 else args.steps
    for k in range(rollouts):
        sm = np.zeros(T)
        roll, g = rollout(T, d, step_ms=sm)
        lat.append(sm)
        fstats.append(roll.stats)
        bstats.append(g["stats"])
        if flush is not None:
            flush.fill_(float(k))   # evict the factor panels between timed rollouts
    ev1.record(stream)
    torch.cuda.synchronize()
    host_s = time.perf_counter() - h0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    sim_steps = rollouts * T
    elapsed, value = whole_job_rate(ev0.elapsed_time(ev1) / 1e3, sim_steps, world, dev)
    launches = sum(s["kernel_launches"] for s in fstats + bstats)
    lat = np.concatenate(lat)
    fwd_it = sum(s["fwd_iters"] for s in fstats) / sim_steps
    bwd_it = sum(s["bwd_iters"] for s in bstats) / sim_steps
    fp64_checks = (sum(s["fwd_fp64_iters"] for s in fstats) + sum(s["bwd_fp64_iters"] for s in bstats)) / sim_steps
    g_final = {k: float(g[k].norm()) for k in want}

    # profiled pass after the timed region (CUDA events around every directly
    # launched solve and forward local step; graphs replay the rest of each chunk)
    prof_T = seg if K > 0 else min(T, 10)
    rp, gp = rollout(prof_T, d, profile=True)
    ps = [rp.stats, gp["stats"]]
    solves_timed = sum(s["solves_timed"] for s in ps)
    t_solve = sum(s["solve_ms"] for s in ps) / 1e3 / max(solves_timed, 1)
    locals_timed = rp.stats["local_steps_timed"]
    t_local = rp.stats["local_ms"] / 1e3 / max(locals_timed, 1)
    bytes_solve, nnzq = solve_bytes(mesh, 4)
    peak, peak_kind = peaks()
    achieved = bytes_solve / t_solve / 1e9
    traffic, traffic_src = _traffic(args.workload)
    gps = int(mesh.e) if wl.get("tet") else 8 * int(mesh.e)
    flops_gp = LOCAL_FLOPS_PER_TET if wl.get("tet") else (LOCAL_FLOPS_PER_GP_NH if sc.neohookean else
                                                           LOCAL_FLOPS_PER_GP)
    local_tflops = flops_gp * gps / t_local / 1e12 if locals_timed else None

    # end to end through the public API with host buffers: H2D of the inputs
    # (initial state, external force, loss weights), forward, backward, D2H of the
    # gradients and the loss; the factorisation stays outside, as for `value` (it runs
    # once per material: factorize_s in config)
    T_e = seg * max(1, args.steps // 4) if K > 0 else T
    host = {k: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64).pin_memory()
            for k, a in (("x0", sc.x0), ("v0", sc.v0), ("f", sc.f_ext), ("lw", sc.loss_w))}
    h2d = sum(t.numel() * 8 for t in host.values())
    float((roll.x[-1] * d["lw"]).sum().cpu())   # lazily loaded torch kernels, outside the timed region
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hp = [time.perf_counter()]
    dd = {k: t.to(dev, non_blocking=True) for k, t in host.items()}
    hp.append(time.perf_counter())
    o = opts_for()
    re_ = mesh.forward(dd["x0"], dd["v0"], T_e, f_ext=dd["f"], opts=o)
    hp.append(time.perf_counter())
    ge = mesh.backward(re_, T_e, dd["lw"], f_ext=dd["f"], opts=o, want=want)
    hp.append(time.perf_counter())
    loss = (re_.x[-1] * dd["lw"]).sum()
    out_host = [ge[k].cpu() for k in want] + [loss.cpu()]
    e1.record(stream)
    torch.cuda.synchronize()
    hp.append(time.perf_counter())
    phases = {k: 1e3 * (hp[i + 1] - hp[i]) for i, k in enumerate(("h2d", "forward", "backward", "d2h"))}
    d2h = sum(t.numel() * 8 for t in out_host)
    e2e_value = world * T_e / (e0.elapsed_time(e1) / 1e3)

    accuracy = None
    if rank == 0 and not args.no_accuracy:
        accuracy = accuracy_leg(mesh, sc, wc, wv, d, prof_T, K, rp, gp, want)
    fp64 = None
    if rank == 0 and not args.no_fp64:
        fp64 = fp64_line(dev)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload, fwd_it + bwd_it)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mixed-f32-f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "element_rule": "tetu" if wl.get("tet") else "hex8",
                       "cells": int(mesh.e), "nodes": int(mesh.n),
                       "dofs": 3 * int(mesh.n), "T": T, "sim_steps_per_bench_step": seg,
                       "checkpoint_every": K, "ms_per_sim_step": 1e3 * elapsed / sim_steps,
                       "tol_fwd": tol, "tol_bwd": tol, "lbfgs_m": 5,
                       "fwd_iters_per_step": fwd_it, "bwd_iters_per_step": bwd_it,
                       "fp64_checks_per_step": fp64_checks,
                       "mesh_s": t_mesh, "factorize_s": t_factor, "factor_nnz": int(mesh.info["factor_nnz"]),
                       "timed_host_s": host_s, "grad_norms": g_final,
                       "l2": ("inputs larger than L2: the FP32 solve panels (%.0f MB) stream through every "
                              "solve" % (nnzq * 4 / 1e6)) if K > 0 else
                             "256 MB buffer written between timed rollouts",
                       "parallelism": "replicas"},
            "roofline": {"bound": "hbm", "kernel": "triangular solve pair (solve_pipe_kernel, FP32 panels)",
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src,
                         "bytes_per_launch": bytes_solve, "avg_solve_us": 1e6 * t_solve,
                         "solves_timed": solves_timed,
                         "timing": "CUDA events on the launching stream around every directly launched solve "
                                   "of a profiled %d-step rollout run after the timed region (the timed rollout "
                                   "runs without events)" % prof_T},
            "local_step": {"bound": "alu", "kernel": (
                               "tet_element_kernel (forward, FP32, one unstructured tetrahedron per thread)"
                               if wl.get("tet") else "element_kernel (forward, FP32%s)" % (
                                   ", Neo-Hookean" if sc.neohookean else "")),
                           "avg_us": 1e6 * t_local, "launches_timed": locals_timed,
                           "flops_per_gauss_point": flops_gp, "gauss_points": gps,
                           "achieved": local_tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": (local_tflops / FP32_PEAK_TFLOPS) if local_tflops else None},
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                "max": float(lat.max()), "steps": int(lat.size),
                                "what": "host wall time of one simulation step: forward + recomputation + "
                                        "adjoint"},
            "accuracy": accuracy,
            "fp64": fp64,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "T": T_e,
                    "includes": "H2D of the inputs (x0, v0, f_ext, loss weights), forward, backward, D2H of "
                                "the gradients and the loss; the factorisation (once per material) is outside, "
                                "as for value",
                    "host_phases_ms": phases},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line))
    mesh.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serve(args):
    """Rollout-plus-gradient serving: quadruped requests (N^3 box, N ~ U{8..24},
    T steps, muscle actuation, ground contact with friction) arriving as a Poisson
    stream at twice the serial service rate of a calibration pass; requests/s and
    request latency percentiles."""
    import numpy as np
    from paper_2101_05917_gb300 import build as _build
    _build.build()
    from paper_2101_05917_gb300 import api
    from paper_2101_05917_gb300 import _native as N
    from workloads import quadruped, serving_stream_c4

    T = args.T
    n_req = args.serve_requests
    _, sizes = serving_stream_c4(n_requests=n_req, rate_hz=1.0, T=T)
    scenes = [quadruped(int(Nn), T=T, request=i) for i, Nn in enumerate(sizes)]
    opts = api.solver_opts(tol_fwd=scenes[0].tol_fwd, tol_bwd=scenes[0].tol_bwd, max_iter_fwd=3000,
                           max_iter_bwd=3000)
    srv = api.PDServer(max_slots=args.serve_slots)
    # calibration: the first three requests one at a time (meshes and factors enter the caches)
    serial = []
    for sc in scenes[:3]:
        r = srv.result(srv.submit_scene(sc, opts=opts))
        serial.append(r["latency_ms"] / 1e3)
    rate = 2.0 / statistics.mean(serial)
    gaps, _ = serving_stream_c4(n_requests=n_req, rate_hz=rate, T=T)
    arrivals = gaps
    t0 = time.perf_counter()
    tickets, done = [], {}
    for i, sc in enumerate(scenes):
        while time.perf_counter() - t0 < arrivals[i]:
            time.sleep(0.0005)
        tickets.append(srv.submit_scene(sc, opts=opts))
    for t in tickets:
        done[t] = srv.result(t)
    wall = time.perf_counter() - t0
    srv.close()
    lat = np.array([done[t]["latency_ms"] for t in tickets])
    q = np.array([done[t]["queue_ms"] for t in tickets])
    ok = sum(1 for t in tickets if done[t]["status"] in (N.PD_OK, N.PD_ERR_NOT_CONVERGED))
    line = {
        "metric": "rollout+gradient requests/s under Poisson arrivals; p50/p99 request latency",
        "value": n_req / wall, "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "mixed-f32-f64", "data": "synthetic",
        "config": {"workload": f"c4_quadruped_stream_T{T}", "requests": n_req, "sizes": [int(x) for x in sizes],
                   "arrival_rate_hz": rate, "serial_service_s": serial, "slots": args.serve_slots,
                   "tol_fwd": scenes[0].tol_fwd, "tol_bwd": scenes[0].tol_bwd},
        "sim_steps_per_s": n_req * T / wall,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max())},
        "queue_ms": {"p50": float(np.percentile(q, 50)), "p99": float(np.percentile(q, 99))},
        "fwd_iters_per_step": float(np.mean([done[t]["fwd_iters"] for t in tickets]) / T),
        "bwd_iters_per_step": float(np.mean([done[t]["bwd_iters"] for t in tickets]) / T),
        "completed": ok,
    }
    print(json.dumps(line))


def run_probe(args):
    """Fixed launch sequences for ncu captures (see profiles/)."""
    import numpy as np
    import torch
    from paper_2101_05917_gb300 import build as _build
    _build.build()
    from paper_2101_05917_gb300 import api
    from paper_2101_05917_gb300 import _native as N
    from workloads import quadruped
    dev = torch.device("cuda:0")
    tt = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    sc = quadruped(16, T=args.T) if args.probe == "quadruped" else _scene(args.workload, args.T)
    mesh = api.PDMesh.from_scene(sc)
    wc, wv, wm, fib = api.scene_weights(sc, dev)
    mesh.factorize(wc, wv, wm, fib, h=sc.h, gravity=tuple(sc.gravity), k_contact=sc.k_contact,
                   precision=N.PD_PREC_MIXED, neohookean=sc.neohookean)
    x = tt(sc.x0)
    v = tt(np.random.default_rng(1).standard_normal(sc.x0.shape))
    if args.probe == "solve":
        for _ in range(args.repeat):
            mesh.solve(v, precision=N.PD_PREC_MIXED)
    elif args.probe == "local":
        for _ in range(args.repeat):
            mesh.local_step(x, precision=N.PD_PREC_MIXED)
    elif args.probe == "hvp":
        for _ in range(args.repeat):
            mesh.hessian_vector(x, v, precision=N.PD_PREC_MIXED)
    else:
        tol = (args.tol if args.tol is not None else WORKLOADS[args.workload]["tol"]) \
            if args.probe == "rollout" else sc.tol_fwd
        opts = api.solver_opts(tol_fwd=tol, tol_bwd=tol, max_iter_fwd=3000, max_iter_bwd=3000,
                               profile=args.profile_events)
        act = tt(sc.act[:args.T]) if sc.act is not None else None
        roll = mesh.forward(x, tt(sc.v0), args.T, f_ext=tt(sc.f_ext), act=act, mu=sc.mu, opts=opts)
        g = mesh.backward(roll, args.T, tt(sc.loss_w), f_ext=tt(sc.f_ext), act=act, mu=sc.mu, opts=opts)
        print("forward", roll.stats)
        print("backward", g["stats"])
    torch.cuda.synchronize()
    mesh.close()


def main():
    args = parse()
    if args.probe:
        run_probe(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.serve:
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
