#!/usr/bin/env python
"""Benchmark of the batched differentiable unrolled COSMO path on B300.

Workload (one step = one pass of the whole hot path over one batch):
256 max-cut SDPs on Erdos-Renyi graphs (instance j: seed 2000+j, n ~ U{20..80}
vertices, edge probability ~ U(0.1, 0.5)), unrolled K = 50 iterations with
learnable per-step log rho_k and alpha_k, meta-loss ||r_p^K||^2 + ||r_d^K||^2
summed over instances, forward + backward (every gradient), mixed precision
(float iterates, double reductions).  Metric: unrolled fwd+bwd
instance-iterations per second.

Also reported on the same box: the plain FP64 one-instance-per-launch GPU
form, the roofline of the dominant kernel (PSD Jacobi projection), the CPU
oracle on a bounded sample, the end-to-end number through host buffers, GPU
clocks during the timed region, and the kernels launched.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_INST, K_UNROLL, SEED0 = 256, 50, 2000
METRIC = "unrolled fwd+bwd instance-iters/sec (batched mixed precision)"
WORKLOAD = ("batched differentiable max-cut SDPs: 256 instances, n ~ U{20..80}, "
            "ER p ~ U(0.1,0.5), seeds 2000+j, K=50 unrolled, learnable log rho_k / alpha_k, "
            "loss ||r_p^K||^2+||r_d^K||^2")
FP32_LANES_PER_SM, N_SM, SM_MAX_MHZ = 128, 148, 2032.0


def problems(rank=0, world=1):
    """This rank's shard of the global batch of world x 256 instances (seeds
    2000+j): instances split over the ranks by estimated cost (LPT), so the
    per-GPU work stays that of 256 instances (weak scaling).  One rank: the
    whole 256-instance batch."""
    from synth import maxcut_problem, random_graph_batch
    from paper_2606_13825_b300.dist import shard
    graphs = random_graph_batch(N_INST * world, SEED0, 20, 80, 0.1, 0.5)
    probs = [maxcut_problem(nv, e) for nv, e in graphs]
    return probs if world == 1 else shard(probs, rank, world)[1]


# -------------------------------------------------------------- workloads --
# Each workload: problems, unroll depth, batch options, whether the warm start
# is learned, and a description.  "maxcut" is the headline metric; the others
# are the paper's other problem classes at their stated sizes.
def workload_spec(name, rank=0, world=1):
    from synth import (lovasz_problem, random_graph_batch, cycle_graph, complete_graph,
                       socp_problem, covsteer_problem)
    if name == "maxcut":
        # the library defaults (one CUDA graph per forward / backward) with the
        # autotuner choosing the Jacobi CTA sizes of the PSD size classes
        return dict(probs=problems(rank, world), K=K_UNROLL, opts={"use_graph": 1, "autotune": 1}, value_type="f32",
                    learn_start=False, metric=METRIC, desc=WORKLOAD)
    if name == "lovasz":
        graphs = random_graph_batch(64, 3000 + rank * 64, 100, 200, 0.5, 0.5)
        probs = [lovasz_problem(nv, e) for nv, e in graphs]
        # vertex-transitive graphs (coincident eigenvalues at the optimum)
        for j in range(16):
            nv = 100 + (j * 100) // 15
            probs.append(lovasz_problem(nv, cycle_graph(nv) if j % 2 == 0 else complete_graph(nv)))
        return dict(probs=probs, K=30, opts={"checkpoint_every": 5}, value_type="f32", learn_start=False,
                    metric="unrolled fwd+bwd instance-iters/sec (Lovasz theta, batched mixed precision)",
                    desc="Lovasz theta SDPs: 64 G(n,1/2) graphs n ~ U{100..200} (seeds 3000+j) + 16 "
                         "vertex-transitive cycles/complete graphs n in [100,200]; K=30, checkpoint every 5; "
                         "learnable log rho_k / alpha_k; loss ||r_p^K||^2+||r_d^K||^2")
    if name == "socp":
        probs = [socp_problem(4000 + rank * 64 + j) for j in range(64)]
        # FP32 iterates reach a true relative CG residual of about eps32 * kappa(M)
        # (kappa ~ 1e3-1e4); the recursively updated residual still falls below
        # it, and stopping at 1e-7 instead of 1e-6 takes the worst per-instance
        # rho-gradient error against the FP64 form from 8.0e-3 to 1.7e-3
        return dict(probs=probs, K=100, opts={"cg_tol": 1e-7}, value_type="bf16", learn_start=False,
                    metric="unrolled fwd+bwd instance-iters/sec (sparse SOCP, batched mixed precision)",
                    desc="random sparse SOCPs: 64 instances (seeds 4000+j), n=5000, A 8000x5000 density 1e-3, "
                         "P=M'M+1e-3 I (M 500x5000 density 1e-3), 200 SOCs d ~ U{3..50} + orthant, planted "
                         "solution; K=100; BF16 A values (P FP32), FP32 iterates, CG tol 1e-7; "
                         "loss ||r_p^K||^2+||r_d^K||^2")
    if name in ("lyapunov", "kalman", "mpc"):
        from synth import lyapunov_problem, robust_kalman_problem, robust_mpc_problem
        if name == "lyapunov":
            probs = [lyapunov_problem(6000 + rank * 64 + j, n=40) for j in range(64)]
            desc = "minimum-trace Lyapunov LMIs: 64 instances (seeds 6000+j), n=40 (svec 820, two 40x40 PSD blocks)"
        elif name == "kalman":
            probs = [robust_kalman_problem(7000 + rank * 256 + j, N=100) for j in range(256)]
            desc = "robust Kalman smoothers: 256 instances (seeds 7000+j), N=100 (n=1004, m=1000, 100 SOC(3))"
        else:
            probs = [robust_mpc_problem(8000 + rank * 512 + j, N=50) for j in range(512)]
            desc = "robust MPC: 512 instances (seeds 8000+j), N=50 (n=203, m=505, 51 SOCs)"
        # 64 Lyapunov instances fill 64 of 148 SMs with one CG CTA each: a
        # cluster of 2 per instance measured 1051 -> 823 ms per step; the
        # SOCP classes (256 / 512 instances, short rows) are faster unclustered
        opts = {"use_graph": 1, "cg_cluster": 2 if name == "lyapunov" else 1}
        return dict(probs=probs, K=50, opts=opts, value_type="f32", learn_start=False,
                    metric=f"unrolled fwd+bwd instance-iters/sec ({name}, batched mixed precision)",
                    desc=desc + "; K=50; learnable log rho_k / alpha_k; loss ||r_p^K||^2+||r_d^K||^2")
    if name == "covsteer":
        probs = [covsteer_problem(5000 + rank * 512 + j) for j in range(512)]
        # its CG solves are short (about 12 iterations): staging each instance's
        # matrices in shared memory (the shape rule's CG) costs more than it
        # saves; vectors in shared memory, matrices through L2 measured 35.0 ->
        # 29.5 ms per step (without the warm-start network)
        return dict(probs=probs, K=40, opts={"use_graph": 1, "cg_cluster": -1}, value_type="f32", learn_start=True,
                    metric="unrolled fwd+bwd instance-iters/sec (covariance steering, batched mixed precision)",
                    desc="covariance-steering stand-in SDPs: 512 instances (seeds 5000+j), nx=4, nu=2, T=20, "
                         "PSD blocks 20x p8 + 20x p6 + p4; K=40; App. E warm-start network and log rho_k / alpha_k; "
                         "one CUDA graph per forward / backward")
    raise ValueError(name)


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"cosmo_bench_clocks_rank{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle --
def _oracle_one(args):
    """Forward + backward of one instance with the CPU oracle (one thread)."""
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except Exception:
        pass
    nv, edges, K = args
    from oracle import cosmo as oc
    from synth import maxcut_problem, ZERO
    pr = maxcut_problem(nv, edges)
    rows = np.where(pr.row_types() == ZERO, 100.0, 0.1)
    t0 = time.perf_counter()
    tr = oc.forward(pr, np.tile(rows, (K, 1)), np.full(K, 1.6), 1e-6)
    oc.backward(pr, tr, gloss=1.0)
    return time.perf_counter() - t0


def cpu_oracle_sample(n_inst, K, procs):
    """The oracle as it stands on the n_inst smallest instances of the
    workload (they bound the CPU work to ~10-30 s), one process per core."""
    from synth import random_graph_batch
    graphs = random_graph_batch(N_INST, SEED0, 20, 80, 0.1, 0.5)
    order = np.argsort([g[0] for g in graphs], kind="stable")[:n_inst]
    jobs = [(graphs[i][0], graphs[i][1], K) for i in order]
    import multiprocessing as mp
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(procs) as pool:
        per = pool.map(_oracle_one, jobs)
    wall = time.perf_counter() - t0
    sizes = sorted(int(graphs[i][0]) for i in order)
    return {"value": n_inst * K / wall, "unit": "instance-iters/s", "cores": procs, "kind": "oracle",
            "sample": f"{n_inst} smallest instances of the workload (n={sizes}), K={K}, fwd+bwd, "
                      f"one single-threaded process each (larger instances cost O(n^6) on the CPU)",
            "per_instance_s": [round(t, 3) for t in per]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    procs = 1
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _oracle_one(_smallest_job(K_UNROLL))
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    value = K_UNROLL * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "instance-iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "smallest instance (n=20), K=50, fwd+bwd per step"},
            "cpu_baseline": {"value": value, "unit": "instance-iters/s", "cores": procs, "kind": "oracle",
                             "sample": "one instance (the smallest, n=20) per step, K=50 fwd+bwd"},
            "e2e": {"value": value, "unit": "instance-iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _smallest_job(K):
    from synth import random_graph_batch
    graphs = random_graph_batch(N_INST, SEED0, 20, 80, 0.1, 0.5)
    i = int(np.argmin([g[0] for g in graphs]))
    return (graphs[i][0], graphs[i][1], K)


# ------------------------------------------------------------ App. B CG --
def measured_hbm_gbs():
    """HBM copy bandwidth measured on the B300s (GB/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except Exception:
        return 6400.0, "fallback 6.4 TB/s (of fallback)"


def run_linsys(args, n=50000):
    print(json.dumps(linsys_record(args, n)))
    return 0


def linsys_record(args, n=50000):
    """Reduced-system solve (P + sigma I + A'D(rho)A) x = A'(rho o b) of the
    App. B instance (P diagonal U(0,10), A n/2 x n with 1% N(0,1) nonzeros,
    rho ~ U(0,1)), mixed precision, through a prepared plan (streamed layout
    of A and A', one cooperative launch per solve).  Reports CG iterations
    per second and the achieved HBM bandwidth of the algorithmic bytes per CG
    iteration, (nnz_P + 2 nnz_A)(4 + 4) + 4 (2n + m) + 6n * 4 (A and A'
    streamed once each, 200 MB > L2, so no flush is needed)."""
    import torch
    from synth import linsys_instance
    from paper_2606_13825_b300.solver import ReducedSystem, PcgPlan
    torch.cuda.set_device(0)
    d = linsys_instance(n, seed=6000, density=0.01, row_sampler=True)
    A = d["A"]
    sysm = ReducedSystem([(d["P"], A)], "mixed")
    rho = torch.tensor(d["rho"], dtype=torch.float32, device="cuda")
    rhs = torch.tensor(A.T @ (d["rho"] * d["b"]), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    plan = PcgPlan(sysm)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    info = plan.info()
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(max(1, args.warmup)):
        plan.solve(1e-6, rho, rhs, tol=1e-6, max_iter=2000, x=x, iters=iters)
    torch.cuda.synchronize()
    if args.profile:
        print(json.dumps({"profile_run": True}))
        return 0
    stream = torch.cuda.current_stream()
    times, its = [], []
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.solve(1e-6, rho, rhs, tol=1e-6, max_iter=2000, x=x, iters=iters)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        its.append(int(iters[0]))
    clk = clocks.stop()
    # per-phase breakdown from one more solve with the plan's phase timer on
    # (not part of the timed steps)
    plan.set_timing(True)
    plan.solve(1e-6, rho, rhs, tol=1e-6, max_iter=2000, x=x, iters=iters)
    phases = {k: {"mean_us": round(v[0], 3), "slowest_cta_us": round(v[1], 3)} for k, v in plan.timing().items()}
    plan.set_timing(False)
    m = A.shape[0]
    nnzA, nnzP = A.nnz, d["P"].nnz
    bytes_it = (nnzP + 2 * nnzA) * 8 + 4 * (2 * n + m) + 6 * n * 4
    t_it = sum(times) / sum(its)
    peak, peak_src = measured_hbm_gbs()
    line = {"metric": "App. B reduced-system CG iterations/sec (n=5e4, m=n/2, A 1% dense)",
            "value": 1.0 / t_it, "unit": "CG iterations/s", "iterations_per_solve": its[0],
            "ms_per_solve": 1e3 * float(np.mean(times)), "plan_build_s": t_plan,
            "roofline": {"bound": "hbm", "achieved": bytes_it / t_it / 1e9, "peak": peak,
                         "unit": "GB/s", "frac": bytes_it / t_it / 1e9 / peak,
                         "bytes_per_iteration": bytes_it, "peak_source": peak_src,
                         "timing": "CUDA events around each solve (preconditioner + one cooperative "
                                   "launch), the setup iteration and the discarded last matvec "
                                   "included"},
            "clocks": clk, "plan": info, "phases_per_iteration": phases,
            "config": {"workload": "App. B linear system", "n": n, "m": m, "nnzA": nnzA,
                       "precision": "float values/vectors, double reductions", "tol": 1e-6,
                       "l2": "A and A' (200 MB) exceed L2 each iteration"}}
    return line


def run_solve(args):
    """The vanilla COSMO baseline of Sec. 4 on the batched max-cut workload
    (256 instances, n ~ U{20..80}): every instance solved from zero to the
    normalised KKT tolerance 1e-3 with residual-balancing rho (cosmo_solve
    defaults; CG tolerance 1e-8 as the paper's Table 1).  Reports instances
    solved per second (the batch waits for its slowest instance) and the
    iteration counts (median and max: the Table 1 kind)."""
    import torch
    from paper_2606_13825_b300 import CosmoBatch
    torch.cuda.set_device(0)
    probs = workload_spec("maxcut", 0)["probs"]
    b = CosmoBatch(probs, precision="mixed", cg_tol=1e-8, use_graph=1)
    for _ in range(max(1, args.warmup)):
        b.solve(eps=1e-3)
    torch.cuda.synchronize()
    times, med, mx, conv = [], [], [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        *_, iters, rbp, rbd, rho = b.solve(eps=1e-3)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        med.append(float(np.median(iters[iters > 0])) if (iters > 0).any() else -1)
        mx.append(int(iters.max()))
        conv.append(int((iters > 0).sum()))
    t = float(np.median(times))
    line = {"metric": "vanilla COSMO (residual-balancing rho) solves to 1e-3 per second, max-cut 256 batch",
            "value": len(probs) / t, "unit": "instances/s", "higher_is_better": True,
            "s_per_batch": t, "median_iterations": med[-1], "max_iterations": mx[-1],
            "converged": conv[-1], "instance_iterations_per_s": len(probs) * mx[-1] / t,
            "timing": "wall clock around cosmo_solve (host loop, a readback every 25 iterations)",
            "config": {"workload": "max-cut 256 (n ~ U{20..80}, p ~ U(0.1, 0.5)), zero start", "eps": 1e-3,
                       "rho0": 0.1, "alpha": 1.6, "precision": "mixed"}}
    print(json.dumps(line))
    return 0


def ws_flops(F, O, H=64):
    """Algorithmic flops per element of the warm-start network (App. E):
    forward 2H(F + H + O); reverse pass (layer recompute, both cotangents)
    2H(F + 2H + O); weight sums 2(F + 1)H + 2(H + 1)H + 2(H + 1)O."""
    fwd = 2 * H * (F + H + O)
    bwd = 2 * H * (F + 2 * H + O)
    red = 2 * (F + 1) * H + 2 * (H + 1) * H + 2 * (H + 1) * O
    return fwd, bwd, red


def run_warmstart(args):
    """The App. E warm-start network over the sparse-SOCP batch (64 instances,
    n = 5000, m = 8000: 320k variables and 512k rows): features, both MLPs
    forward, and the reverse pass to both parameter gradients.  Timed with
    CUDA events on the current stream; ALU roofline of the reverse-pass
    kernel of the constraint MLP (FP32 FMA on the CUDA cores)."""
    import torch
    from paper_2606_13825_b300 import CosmoBatch, WarmStartNet, lib
    torch.cuda.set_device(0)
    probs = workload_spec("socp", 0)["probs"]
    b = CosmoBatch(probs, precision="mixed", value_type="bf16")
    net = WarmStartNet(dtype=torch.float32, device="cuda", generator=torch.Generator().manual_seed(3))
    with torch.no_grad():   # a trained-looking output layer (nonzero)
        net.theta_x[-65:].normal_(0, 0.1)
        net.theta_c[-130:].normal_(0, 0.1)
    g = torch.Generator(device="cuda").manual_seed(4)
    gx = torch.randn(b.n_total, device="cuda", generator=g)
    gs = torch.randn(b.m_total, device="cuda", generator=g)
    gy = torch.randn(b.m_total, device="cuda", generator=g)
    tx, tc = net.theta_x.detach(), net.theta_c.detach()

    def step():
        b.ws_forward(tx, tc)
        b.ws_backward(tx, tc, gx, gs, gy)

    for _ in range(args.warmup if args.profile else max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if args.profile:
        print(json.dumps({"profile_run": True, "workload": "warmstart", "steps": args.warmup}))
        return 0
    b.profile("ws_bwd")
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = lib().cosmo_kernel_launch_count()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = (lib().cosmo_kernel_launch_count() - n0) // args.steps
    N = b.n_total + b.m_total
    fx, bx, rx = ws_flops(8, 1)
    fc, bc, rc = ws_flops(12, 2)
    flops = b.n_total * (fx + bx + rx) + b.m_total * (fc + bc + rc)
    line = {"metric": "warm-start network fwd+bwd elements/s (App. E, sparse-SOCP batch)",
            "value": N / (ms * 1e-3), "unit": "elements/s", "higher_is_better": True, "ms_per_step": ms,
            "steps": args.steps, "warmup": args.warmup, "gpu_launches": int(launches) * args.steps,
            "gflop_per_step": flops / 1e9, "tflops": flops / (ms * 1e-3) / 1e12,
            "config": {"workload": "sparse SOCP 64 x (n=5000, m=8000), features + MLP_x / MLP_c forward + "
                                   "reverse to both parameter gradients", "precision": "FP32",
                       "n_total": b.n_total, "m_total": b.m_total}}
    tot_ms, nl = b.profile_read("ws_bwd")
    b.profile(enable=False)
    # FP32 FMA peak of the CUDA cores at the maximum SM clock (2 flops per lane-cycle)
    peak = FP32_LANES_PER_SM * N_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    bwd_s = tot_ms * 1e-3 / args.steps   # both reverse-pass launches of one step
    ach = (b.n_total * bx + b.m_total * bc) / bwd_s / 1e12
    line["roofline"] = {"bound": "alu", "kernel": "k_ws_bwd (both MLPs)", "achieved": ach, "peak": peak,
                        "unit": "TFLOP/s", "frac": ach / peak, "traffic": None, "launches": nl,
                        "share_of_step": bwd_s / (ms * 1e-3)}
    print(json.dumps(line))
    return 0


def run_policy(args):
    """The batched max-cut workload (256 instances, n ~ U{20..80}, K = 50,
    mixed precision, one CUDA graph per forward / backward) trained through
    the closed-loop hyperparameter policy of App. E instead of free per-step
    log rho_k / alpha_k: forward (the policy evaluated on the device after
    every step) + backward to the policy parameters.  CUDA events on the
    current stream, L2 flushed between steps outside the events; the policy
    kernels' own time from a direct-launch copy of the batch."""
    import torch
    from paper_2606_13825_b300 import CosmoBatch, HyperPolicy, lib
    torch.cuda.set_device(0)
    probs = workload_spec("maxcut", 0)["probs"]
    K = K_UNROLL
    res = {}
    for graph in ((0,) if args.profile else (1, 0)):
        b = CosmoBatch(probs, precision="mixed", use_graph=graph)
        pol = HyperPolicy(dtype=torch.float32, device="cuda", generator=torch.Generator().manual_seed(7))
        with torch.no_grad():   # a trained-looking output layer
            g = torch.Generator(device="cuda").manual_seed(8)
            pol.theta_rho[-33:].normal_(0, 0.05, generator=g)
            pol.theta_alpha[-33:].normal_(0, 0.05, generator=g)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

        def step():
            pol.zero_grad(set_to_none=True)
            L = pol(b, K)[3].sum()
            L.backward()

        for _ in range(args.warmup if args.profile else max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        assert not b.status().any(), "device flags raised during warm-up"
        if args.profile:   # direct launches, warm-up steps only: the command profiled under ncu
            print(json.dumps({"profile_run": True, "workload": "maxcut_policy", "steps": args.warmup}))
            return 0
        if not graph:
            b.profile()
        st = torch.cuda.current_stream()
        ms = []
        n0 = lib().cosmo_kernel_launch_count()
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            step()
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[graph] = dict(ms=float(np.median(ms)), launches=(lib().cosmo_kernel_launch_count() - n0) // args.steps)
        if not graph:
            reads = {c: b.profile_read(c, reset=False) for c in b.KERNEL_CLASSES}
            res["kernels"] = {c: round(v[0] / args.steps, 4) for c, v in reads.items() if v[1]}
    t = res[1]["ms"]
    kern = res.get("kernels", {})
    line = {"metric": "closed-loop policy fwd+bwd instance-iters/sec (max-cut 256, K=50, mixed precision)",
            "value": len(probs) * K / (t * 1e-3), "unit": "instance-iters/s", "higher_is_better": True,
            "ms_per_step": t, "steps": args.steps, "warmup": args.warmup, "gpu_launches": int(res[1]["launches"]),
            "direct_launch_ms_per_step": res[0]["ms"], "kernel_ms_per_step_direct": kern,
            "policy_share_direct": (kern.get("pol_fwd", 0) + kern.get("pol_bwd", 0) + kern.get("ws_grad", 0))
            / res[0]["ms"],
            "config": {"workload": WORKLOAD.replace("learnable log rho_k / alpha_k",
                                                    "App. E closed-loop policy (32x32 MLPs, learnable l0)"),
                       "precision": "float iterates and policy, double reductions",
                       "l2": "flushed between steps (256 MB write, outside the events)",
                       "launch": "one CUDA graph per forward / backward"}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- ours --
PSD_TRAFFIC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "psd_fwd_traffic_maxcut256.txt")
PSD_SOURCES = ("kernels_jt.cuh", "kernels_jt2.cuh", "kernels_psd.cuh")


def psd_sources_sha16():
    """Hash of the PSD projection kernels' sources: a DRAM-traffic figure taken
    with ncu holds only for the sources it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for f in PSD_SOURCES:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2606_13825_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def psd_traffic():
    """DRAM bytes (read + write) per forward launch group of the projection on
    the max-cut workload, from the ncu capture summarised in profiles/, or None
    when the kernels changed since it was taken."""
    try:
        kv = {}
        with open(PSD_TRAFFIC) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_sources_sha16") != psd_sources_sha16():
            return None
        return float(kv["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def psd_flops(probs):
    """Algorithmic flops of one PSD-projection launch: symmetric eigen-
    decomposition with vectors 9 p^3 (Golub & Van Loan's count for symmetric
    QR) plus the reconstruction U max(L,0) U' 2 p^3, summed over blocks."""
    from synth.problem import PSD
    return float(sum(11.0 * d ** 3 for p in probs for (ct, d) in p.cones if ct == PSD))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the one-instance-per-launch forms")
    ap.add_argument("--no-linsys", action="store_true", help="skip the App. B CG record")
    ap.add_argument("--profile", action="store_true",
                    help="run only W steps of the workload (the command profiled under ncu)")
    ap.add_argument("--workload", default="maxcut",
                    choices=["maxcut", "lovasz", "socp", "covsteer", "lyapunov", "kalman", "mpc", "linsys",
                             "maxcut_solve", "warmstart", "maxcut_policy"],
                    help="maxcut: the batched differentiable max-cut step (the headline metric); "
                         "lovasz / socp / covsteer / lyapunov / kalman / mpc: the paper's other classes at "
                         "their stated sizes; "
                         "linsys: the App. B reduced-system CG at n=5e4 (HBM roofline of SpMV/CG); "
                         "maxcut_solve: the vanilla COSMO baseline solving the max-cut batch to 1e-3; "
                         "warmstart: the App. E warm-start network forward + reverse on the SOCP batch; "
                         "maxcut_policy: the max-cut step trained through the App. E closed-loop policy")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "linsys":
        return run_linsys(args)
    if args.workload == "maxcut_solve":
        return run_solve(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "maxcut_policy":
        return run_policy(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2606_13825_b300 import CosmoBatch, lib
    from paper_2606_13825_b300.solver import unrolled_residual_loss

    spec = workload_spec(args.workload, rank, world)
    probs, K = spec["probs"], spec["K"]
    n_inst = len(probs)
    opts = dict(spec["opts"])
    use_graph = int(opts.pop("use_graph", 0))
    if args.profile:
        # the profiled command is deterministic: the shape rules' launch
        # configuration (on this workload the one the autotuner keeps: Jacobi
        # at 512 / 256 / 128 threads), no timed candidates before the step
        opts["autotune"] = 0
    b = CosmoBatch(probs, precision="mixed", value_type=spec["value_type"], device=local,
                   use_graph=use_graph, **opts)
    lr = torch.full((K,), math.log(0.1), dtype=torch.float64, device=dev, requires_grad=True)
    ak = torch.full((K,), 1.6, dtype=torch.float64, device=dev, requires_grad=True)
    net = None
    if spec["learn_start"]:
        # the App. E warm-start network (its output layer starts at zero)
        from paper_2606_13825_b300 import WarmStartNet
        net = WarmStartNet(dtype=torch.float32, device=dev, generator=torch.Generator().manual_seed(11))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(batch=b):
        lr.grad = None
        ak.grad = None
        kw = {}
        if net is not None:
            net.zero_grad(set_to_none=True)
            x0, s0, y0 = net(batch)
            kw = dict(x0=x0, s0=s0, y0=y0)
        L, _ = unrolled_residual_loss(batch, lr, ak, **kw)
        L.backward()
        return L

    has_psd = any(ct == 4 for p in probs for (ct, _) in p.cones)
    dom = "psd_fwd" if has_psd else "pcg"          # dominant kernel class
    persist = has_psd and bool(b.info()["fwd_persistent"])
    if persist:
        # the persistent forward: one launch per size class runs every step of
        # a segment (right-hand side, relaxation, projections, dual update)
        dom = "fwd_persist"
    # CUDA events around every launch group of the dominant class: with CUDA
    # graphs they are event nodes of the recorded graphs, read back after
    # each replay, so the roofline kernel is timed inside the timed region
    if not args.profile:
        b.profile(dom)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert not b.status().any(), "device flags raised during warm-up"
    if args.profile:
        print(json.dumps({"profile_run": True, "steps": args.warmup}))
        return 0

    # ---------------- timed region: K steps, L2 flushed between steps -------
    b.profile_read(dom, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = lib().cosmo_kernel_launch_count()
    st = torch.cuda.current_stream()
    total_ms = 0.0
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step()
        e1.record(st)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    launches = lib().cosmo_kernel_launch_count() - n0
    clk = clocks.stop()
    # the roofline kernel, timed live in the timed region
    dom_ms, dom_n = b.profile_read(dom, reset=True)
    if dist:
        from paper_2606_13825_b300.dist import max_over_ranks
        total_ms = max_over_ranks(total_ms, device=dev)
    ms_per_step = total_ms / args.steps
    n_total = n_inst
    if dist:
        tot = torch.tensor([n_inst], dtype=torch.int64, device=dev)
        dist.all_reduce(tot)
        n_total = int(tot)          # every rank's instances (their shards partition the batch)
    value = n_total * K * args.steps / (total_ms / 1e3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    inf = b.info()
    work = {"jacobi_sweeps_per_block": inf["eig_sweeps"] / max(inf["eig_blocks"], 1),
            "cg_iters_per_solve": inf["cg_iters"] / max(inf["cg_solves"], 1),
            "adjoint_cg_iters_per_solve": inf["adj_cg_iters"] / max(inf["adj_cg_solves"], 1)}

    # ---------------- per-kernel breakdown (one extra step, all classes) ----
    tuning = b.tuning()
    bb = b
    if use_graph:
        bb = CosmoBatch(probs, precision="mixed", value_type=spec["value_type"], device=local,
                        use_graph=0, **dict(opts, autotune=0))
        bb.set_tuning(tuning)
        step(bb)
        torch.cuda.synchronize()
    bb.profile(None)
    bb.profile_read(None, reset=True)
    step(bb)
    torch.cuda.synchronize()
    breakdown = {}
    for kname in bb.KERNEL_CLASSES:
        ms, n = bb.profile_read(kname, reset=False)
        if n:
            breakdown[kname] = round(ms, 4)
    bb.profile(enable=False)
    b.profile(enable=False)

    # ---------------- roofline of the dominant kernel ------------------------
    avg_s = dom_ms / max(dom_n, 1) / 1e3
    if has_psd:
        flops = psd_flops(probs)
        kern = ("psd_fwd (cyclic Jacobi eigensolver + reconstruction; a CTA per block, a thread per "
                "block of order <= 8)")
        if persist:
            # one launch group covers the steps of one forward segment
            c = int(opts.get("checkpoint_every", 0) or 0)
            nseg = -(-K // c) if c > 0 else 1
            flops *= K / nseg
            kern = ("fwd_persist (per CTA one instance for every step of a segment: right-hand side, "
                    "relaxation, separable projections, cyclic Jacobi eigensolver + reconstruction, dual update)")
        achieved = flops / avg_s / 1e12
        peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
        roof = {"kernel": kern,
                "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": psd_traffic() if args.workload == "maxcut" and not persist else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the three size-class "
                                  "launches of one forward iteration (profiles/psd_fwd_traffic_maxcut256.txt), "
                                  "null when the kernel sources changed since the capture",
                "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 flop/FMA x 2032 MHz",
                "flops_per_launch": flops, "avg_launch_ms": avg_s * 1e3, "launches_timed": dom_n,
                "algorithmic_count": "sum over blocks of 9p^3 (eigh) + 2p^3 (reconstruction)"
                                     + (", times the steps of a launch" if persist else "")}
    else:
        # CG: every iteration streams A, A' and P once (value + column index)
        # plus ~8 n-vectors of 4 bytes; iterations counted on the device
        vb = 2 if spec["value_type"] == "bf16" else 4
        nnzA = sum(p.A.nnz for p in probs)
        nnzP = sum(p.P.nnz for p in probs)
        inf0 = bb.info()
        it_per_solve = inf0["cg_iters"] / max(inf0["cg_solves"], 1)
        bytes_per_it = (2 * nnzA + nnzP) * (vb + 4) + 8 * 4 * sum(p.A.shape[1] for p in probs)
        bytes_launch = bytes_per_it * it_per_solve
        peak, peak_src = measured_hbm_gbs()
        achieved = bytes_launch / avg_s / 1e9
        roof = {"kernel": "pcg (Jacobi-PCG, CTA per instance, matrix-free SpMV with A, A', P)",
                "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                "bytes_per_launch": bytes_launch, "avg_launch_ms": avg_s * 1e3, "launches_timed": dom_n,
                "algorithmic_count": "per CG iteration (2 nnz(A) + nnz(P)) x (value + int32 index) "
                                     "+ 8 n x 4 bytes, times the mean CG iterations per solve"}

    # ---------------- end to end through host buffers ------------------------
    lr_h = torch.full((K,), math.log(0.1), dtype=torch.float64).pin_memory().numpy()
    ak_h = torch.full((K,), 1.6, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        b.step_host(K, lr_h, ak_h)
    torch.cuda.synchronize()
    total_e2e = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        b.step_host(K, lr_h, ak_h)        # synchronises before returning
        total_e2e += time.perf_counter() - t1
    e2e_value = n_inst * K * args.steps / total_e2e
    e2e = {"value": e2e_value, "unit": "instance-iters/s", "h2d_bytes_per_step": 2 * K * 8,
           "d2h_bytes_per_step": (n_inst + 2 * K) * 8,
           "api": "cosmo_step_host (host log_rho_k, alpha_k in; loss and gradients out; pinned)"}

    # ---------------- plain FP64 one-instance-per-launch GPU form ------------
    def one_instance_form(precision):
        """One instance per batch and per launch (direct launches), on a
        seeded sample of the workload's instances."""
        rng = np.random.default_rng(1)
        sample = rng.choice(n_inst, size=min(8, n_inst) if args.workload == "maxcut" else 2, replace=False)
        tot, iters = 0.0, 0
        o1 = {k: v for k, v in opts.items() if k not in ("autotune",)}
        for i in sample:
            b1 = CosmoBatch([probs[i]], precision=precision, device=local, use_graph=0, **o1)
            l1 = torch.full((K,), math.log(0.1), dtype=torch.float64, device=dev, requires_grad=True)
            a1 = torch.full((K,), 1.6, dtype=torch.float64, device=dev, requires_grad=True)
            L, _ = unrolled_residual_loss(b1, l1, a1)
            L.backward()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            L, _ = unrolled_residual_loss(b1, l1, a1)
            L.backward()
            e1.record(st)
            e1.synchronize()
            tot += e0.elapsed_time(e1) / 1e3
            iters += K
            del b1
        return {"value": iters / tot, "unit": "instance-iters/s",
                "sample": f"{len(sample)} instances (seeded choice, n={sorted(int(probs[i].A.shape[1]) for i in sample)}), "
                          f"each its own {'FP64' if precision == 'fp64' else 'mixed-precision (FP32)'} batch, "
                          f"direct launches, K={K} fwd+bwd"}

    plain = plain32 = None
    if not args.no_plain:
        plain = one_instance_form("fp64")
        plain32 = one_instance_form("mixed")

    cpu = None
    if not args.no_cpu and args.workload == "maxcut":
        ncpu = os.cpu_count() or 1
        cpu = cpu_oracle_sample(16, K, min(16, ncpu))
        cpu["host_cores"] = ncpu

    line = {"metric": spec["metric"], "value": value, "unit": "instance-iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": spec["desc"], "instances_per_gpu": n_inst, "K": K,
                       "precision": "float iterates, double CG/residual/eigen-gap reductions",
                       "l2": "flushed between steps (256 MB write, outside the events)",
                       "launch": ("one CUDA graph per forward / backward (the library default); the "
                                  f"roofline kernel class ({dom}) timed by CUDA-event nodes inside the graphs"
                                  if use_graph else "direct launches on the current stream"),
                       "tuning": {"autotune": bool(opts.get("autotune", 0)), "tuned": tuning["tuned"],
                                  "psd_classes": [f"p<={c['maxp']} x{c['count']}: {c['method']} "
                                                  f"{c['threads']} threads" for c in tuning["classes"]],
                                  "cg_kernel": tuning["cg_kernel"], "tune_ms": round(tuning["tune_ms"], 1)},
                       "parallelism": f"dp{world} (independent instances per GPU, no collective)"},
            "clocks": clk, "gpu_launches": int(launches), "e2e": e2e, "roofline": roof,
            "cpu_baseline": cpu, "plain_fp64": plain,
            "ratio_vs_plain_fp64": (value / world) / plain["value"] if plain else None,
            "plain_fp32_one_instance": plain32,
            "ratio_vs_plain_fp32_one_instance": (value / world) / plain32["value"] if plain32 else None,
            "ratio_fp32_vs_fp64_one_instance": plain32["value"] / plain["value"] if plain else None,
            "kernel_ms_per_step": breakdown, "work": work, "wall_s_timed": t_wall}
    if args.workload == "maxcut" and not args.no_linsys:
        # the HBM-bound CG of the reduced system at App. B scale, its own
        # timed region and clock record
        line["linsys"] = linsys_record(args)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
