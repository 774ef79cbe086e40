"""Benchmark: batched adaptive soft-contact rollouts on GB300.

Workload (one "step" = one batch rollout, the whole hot path): 4096 box pushes
(cube 0.1 m, 1 kg, free joint, mu = 1 pyramidal friction with 8 vertex
contacts, solref 0.002 s), T = 1 s, DOPRI5 rtol 1e-6 / atol 1e-8, forward
only, seeded synthetic inputs.  Metric: env-steps/s = accepted DOPRI5 steps
of all environments per second.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  For N > 1 (torchrun) each rank integrates its
own 4096 environments (weak scaling, no collective on the data path); the
time is the max over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s fwd and fwd+adjoint; p50/p99 MPC-request latency, 1 GB300"
UNIT = "env-steps/s"
WORKLOAD = {"workload": "box_push", "B": 4096, "T_s": 1.0, "rtol": 1e-6, "atol": 1e-8, "h0": 1e-3, "mu": 1.0,
            "contacts": "8 box vertices vs plane, pyramidal 4-edge cone", "solref": [0.002, 1.0]}
# Algorithmic FP64 work of one accepted step, counted by the oracle's
# instrumented scalar over seeded environments (python -m oracle.count_flops):
# each constraint solve counted as started at its final active set (one Newton
# system and one residual check per right-hand side; the CUDA path starts the
# search at the previous right-hand side's active set).  Box pushes: 28,910
# (41,112 with the oracle's own search from the unconstrained acceleration).
FLOP_PER_STEP = 28910.0
FLOP_PER_STEP_SEARCH = 41112.0
# Arm pushing the cube (T = 2 s, 50 intervals): forward 148,516 per accepted
# step; adjoint 492,619 per accepted step (every step once with one tangent in
# the counting derivative scalar: primal recompute + linearised step).
ARM_FLOP_PER_STEP = 148516.0
ARM_ADJ_FLOP_PER_STEP = 492619.0
# FP64 peak derived from the unit counts and clock (152 SMs x 4 FP64 flop/clk
# x 2070 MHz), reported beside the peak measured in the run.
FP64_PEAK_DERIVED_GFLOPS = 152 * 4 * 2.070
L2_BYTES = 126 * 2 ** 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--form", choices=["persistent", "step", "graph"], default="persistent")
    p.add_argument("--lanes", type=int, default=0, help="lanes per environment (0 = autotuned)")
    p.add_argument("--no-extras", action="store_true", help="skip the plain-form and CPU-baseline legs")
    p.add_argument("--envs", type=int, default=4096,
                   help="box pushes per GPU (4096: the benchmark; smaller only to profile a small case)")
    p.add_argument("--horizon", type=float, default=1.0, help="box-push horizon T in s (1: the benchmark)")
    p.add_argument("--serving", action="store_true", help="served-request latency benchmark instead of the rollout bench")
    p.add_argument("--grad-only", action="store_true", help="only the fwd+adjoint leg (one JSON line)")
    p.add_argument("--grad-envs", type=int, default=16384, help="environments of the fwd+adjoint leg")
    p.add_argument("--all", action="store_true", help="every workload (forward, fwd+adjoint, CPU oracle samples)")
    p.add_argument("--pareto", action="store_true", help="integrator comparison: error vs runtime on cube tosses")
    p.add_argument("--pareto-envs", type=int, default=2048)
    p.add_argument("--pareto-sample", type=int, default=32, help="tosses compared with the oracle reference")
    p.add_argument("--adj-lanes", type=int, default=0, help="lanes per environment of the adjoint (0 = autotuned)")
    p.add_argument("--requests", type=int, default=24, help="served requests timed (after the warm-up ones)")
    p.add_argument("--warmup-requests", type=int, default=4)
    p.add_argument("--grad-reps", type=int, default=3, help="timed repeats of the fwd+adjoint leg")
    p.add_argument("--rate", type=float, default=200.0, help="Poisson arrival rate (requests/s)")
    return p.parse_args()


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ distributed plumbing
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, backend):
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum_(t, world):
    """In-place sum of a tensor over the ranks (the parameter-gradient
    exchange of the system-identification step); identity for one rank."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def reduce_sum(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# sources of the forward rollout kernel (the ncu record is valid while they are unchanged)
FORWARD_SOURCES = ("dmx_device.cuh", "dmx_dual.cuh", "dmx_kernels.cuh", "dmx_kernels.h", "dmx_model.h",
                   "dmx_inst_g1.cu", "dmx_inst_g2.cu", "dmx_inst_g4.cu", "dmx_inst_g8.cu", "dmx_inst_g16.cu",
                   "dmx_inst_g32.cu")


# sources of the reverse adjoint kernel (its FP64 counter record is valid while they are unchanged)
ADJOINT_SOURCES = FORWARD_SOURCES + ("dmx_adjoint.h", "dmx_adjoint_rev.cuh", "dmx_vjp.cuh", "dmx_adj_g2.cu",
                                     "dmx_adj_g4.cu", "dmx_adj_g8.cu", "dmx_adj_g16.cu", "dmx_adj_g32.cu")


def _sources_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2506_14186_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def _adjoint_flops_per_step(lanes):
    """Executed FP64 flops per accepted env-step of the reverse adjoint of the
    arm workload (T = 2 s, 50 intervals, K = 32) from the committed ncu counter
    record (2 DFMA + DMUL + DADD thread operations), if it was taken on the
    current kernel sources with the same lane count (else None)."""
    path = os.path.join(ROOT, "profiles", "adjoint_rev_chain_cube.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != _sources_sha(ADJOINT_SOURCES) or rec.get("lanes") != lanes:
        return None
    return rec["fp64_flops_per_launch"] / rec["env_steps"]


def _forward_record(kernel_lanes):
    """The committed ncu record of the persistent kernel (DRAM bytes and FP64
    thread operations per launch), if it was taken on the current kernel
    sources with the same lane count (else None)."""
    path = os.path.join(ROOT, "profiles", "rollout_persistent_box_push.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("source_sha256") != _sources_sha(FORWARD_SOURCES) or rec.get("lanes") != kernel_lanes:
        return None
    return rec


def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def stats_ms(times):
    """Median and p90 (ms) of a list of per-step times (ms)."""
    a = np.asarray(times, dtype=np.float64)
    return float(np.median(a)), float(np.percentile(a, 90))


# ------------------------------------------------------------------ CPU (oracle) timing
def oracle_rate(inp, budget_s=10.0, first=256, max_envs=4096, nthreads=None):
    """Oracle batch rollouts on the host cores over a bounded sample of the
    workload's environments: (env-steps/s, sample description, cores)."""
    import oracle
    from paper_2506_14186_gb300 import workloads as W
    m = oracle.OracleModel(W.box_scene())
    cores = nthreads or os.cpu_count() or 1
    steps, t_used, n_done = 0, 0.0, 0
    chunk = first
    while n_done < max_envs and (n_done == 0 or t_used < budget_s):
        sl = slice(n_done, min(max_envs, n_done + chunk))
        t0 = time.perf_counter()
        r = m.batch_rollout(inp["x0"][sl], inp["T"][sl], rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"],
                            max_steps=inp["max_steps"], nthreads=cores)
        t_used += time.perf_counter() - t0
        steps += int(r["nsteps"].sum())
        n_done = sl.stop
    return steps / t_used, f"first {n_done} of the 4096 environments ({steps} env-steps, {t_used:.1f} s)", cores, t_used


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch

    import paper_2506_14186_gb300 as dmx
    from paper_2506_14186_gb300 import _build, autotune
    from paper_2506_14186_gb300 import workloads as W

    rank, world, local = dist_env()
    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, "nccl")
    sc = W.box_scene()
    inp = W.box_push_inputs(args.envs, seed=1002 + rank, T=args.horizon)
    model = dmx.Model(sc)
    x0 = torch.tensor(np.ascontiguousarray(inp["x0"].T), device=dev)
    T = torch.tensor(inp["T"], device=dev)
    kw = dict(rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
    tuned = {}
    if args.lanes:
        lanes = args.lanes
    else:
        lanes, tuned = autotune.tune_forward(model, x0, T, **kw)
    flush = torch.empty(2 * L2_BYTES // 8, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()

    def step(form=args.form):
        return dmx.rollout(model, x0, T, lanes=lanes, form=form, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    times, nsteps = [], 0
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))                       # evict L2 between timed steps (outside the timing)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            out = step()
            e1.record(st)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            nsteps = int(out["nsteps"].sum().item())
            assert int((out["status"] != 0).sum().item()) == 0, "environment failed"
    torch.cuda.synchronize()
    barrier(world)
    ms, ms_p90 = stats_ms(times)
    ms_max = reduce_max(ms, world, dev)
    steps_all = reduce_sum(nsteps, world, dev)
    value = steps_all / (ms_max * 1e-3)

    # end to end through the C ABI with host buffers (pinned), copies included
    x0_h = torch.from_numpy(np.ascontiguousarray(inp["x0"].T)).pin_memory()
    T_h = torch.from_numpy(np.ascontiguousarray(inp["T"])).pin_memory()
    xT_h = torch.empty((model.nx, 4096), dtype=torch.float64).pin_memory()
    dmx.rollout_host(model, x0_h, T_h, lanes=lanes, xT=xT_h, **kw)
    e2e_t, e2e_steps = [], 0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        r = dmx.rollout_host(model, x0_h, T_h, lanes=lanes, xT=xT_h, **kw)
        e2e_t.append(time.perf_counter() - t0)
        e2e_steps = int(r["nsteps"].sum())
    e2e_s = reduce_max(float(np.median(e2e_t)), world, dev)
    e2e = {"value": reduce_sum(e2e_steps, world, dev) / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(x0_h.numel() * 8 + T_h.numel() * 8),
           "d2h_bytes_per_step": int(xT_h.numel() * 8 + 4096 * 4 * 2)}

    # every rank: the parameter-gradient step ends in an all-reduce over ranks
    sysid = None if args.no_extras else sysid_leg(dmx, dev, world=world, rank=rank)
    result = None
    if rank == 0:
        peak, peak_shapes = dmx.fp64_peak()
        achieved = nsteps * FLOP_PER_STEP / (ms * 1e-3) / 1e12
        rec = _forward_record(lanes)
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": rec.get("dram_bytes_per_launch") if rec else None,
                    "peak_source": "measured in this run: FP64 FMA probe kernel (dmx_fp64_peak), best launch shape "
                                   "of " + ", ".join(f"{k} {v:.3f}" for k, v in peak_shapes.items()) + " TFLOP/s; "
                                   f"derived 152 SMs x 4 flop/clk x 2.07 GHz = {FP64_PEAK_DERIVED_GFLOPS / 1e3:.3f}",
                    "kernel": f"k_rollout_persistent<{lanes}>", "flop_per_env_step": FLOP_PER_STEP,
                    "flop_per_env_step_with_cold_search": FLOP_PER_STEP_SEARCH}
        if rec and rec.get("fp64_flops_per_launch"):
            ex = rec["fp64_flops_per_launch"] / (ms * 1e-3) / 1e12
            roofline["executed"] = {"achieved": ex, "frac": ex / peak, "flop_per_env_step":
                                    rec["fp64_flops_per_launch"] / max(1, rec.get("env_steps", nsteps)),
                                    "source": "ncu FP64 thread operations (2 DFMA + DMUL + DADD), "
                                              "profiles/rollout_persistent_box_push.json"}
        result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": ms_max, "ms_p90": ms_p90, "higher_is_better": True,
                  "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded box pushes)",
                  "config": dict(WORKLOAD, B=args.envs, T_s=args.horizon, form=args.form, lanes=lanes,
                                 parallelism=f"env shards x{world}",
                                 l2="flushed (256 MB write) between timed steps",
                                 env_steps_per_batch=nsteps, autotune_ms=tuned or None),
                  "e2e": e2e, "gpu_launches": args.steps, "roofline": roofline, "clocks": clk.summary()}
        if not args.no_extras:
            extra = {}
            for form in ("graph", "step"):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(0.0)
                e0.record(st)
                out = step(form)
                e1.record(st)
                e1.synchronize()
                t = e0.elapsed_time(e1)
                extra[form] = {"value": int(out["nsteps"].sum().item()) / (t * 1e-3), "ms_per_step": t}
            result["plain_forms"] = extra
            result["sysid"] = sysid
            result["fwd_adjoint"] = grad_leg(dmx, dev, B=args.grad_envs, adj_lanes=args.adj_lanes,
                                             reps=args.grad_reps, peak=peak)
            result["serving"] = serving_leg(dmx, W, requests=args.requests, warmup=args.warmup_requests,
                                            rate=args.rate)
            rate, sample, cores, _ = oracle_rate(inp)
            rate1, sample1, _, _ = oracle_rate(inp, budget_s=0.0, first=32, max_envs=32, nthreads=1)
            result["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                                      "cpu": cpu_model(), "one_thread": {"value": rate1, "sample": sample1}}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return result


def grad_leg(dmx, dev, B=16384, adj_lanes=0, reps=3, peak=None, parity_envs=(0, 5)):
    """Forward (taped) + discrete adjoint (reverse-mode kernel, autotuned lanes)
    of the arm-pushes-cube workload (7 hinges + free cube, 50 torque intervals
    over 2 s, K = 32), loss = squared cube-to-goal distance, on the first B of
    the 16384 environments (all of them by default): `reps` timed repeats
    (median and p90), and the gradient of `parity_envs` against the CPU
    oracle's discrete adjoint along the GPU's step sizes."""
    import torch
    from paper_2506_14186_gb300 import autotune
    from paper_2506_14186_gb300 import workloads as W
    sc = W.chain_cube_scene()
    inp = W.chain_inputs(16384)
    m = dmx.Model(sc)
    x0 = torch.tensor(np.ascontiguousarray(inp["x0"][:B].T), device=dev)
    ctrl = torch.tensor(np.ascontiguousarray(np.transpose(inp["ctrl"][:B], (1, 2, 0))), device=dev)
    T = torch.tensor(inp["T"][:B], device=dev)
    goal = torch.tensor(W.chain_goal(), device=dev)[:, None]
    st = torch.cuda.current_stream()
    fwd_lanes, _ = autotune.tune_forward(m, x0, torch.clamp(T, max=0.2), ctrl=ctrl, NI=50, candidates=(8, 16, 32))
    if adj_lanes:
        m.set_lanes(B, adj_lanes, grad=2)
        adj_ms = None
    else:
        adj_lanes, adj_ms = autotune.tune_adjoint(m, x0, T, ctrl=ctrl, NI=50, K=32)
    m.set_lanes(B, fwd_lanes)
    # warm-up on a short horizon: the stream-ordered pool then holds the tape
    # and adjoint scratch sizes the timed call needs
    w = dmx.rollout(m, x0, torch.clamp(T, max=0.05), ctrl=ctrl, NI=50, K=32, tape=True)
    dmx.rollout_grad(w["tape"], torch.zeros_like(w["xT"]))
    del w
    t_fwd, t_adj, t_tot = [], [], []
    for _ in range(max(1, reps)):
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        out = dmx.rollout(m, x0, T, ctrl=ctrl, NI=50, K=32, tape=True)
        e1.record(st)
        xT_bar = torch.zeros_like(out["xT"])
        xT_bar[7:10] = 2 * (out["xT"][7:10] - goal)
        gx, gu = dmx.rollout_grad(out["tape"], xT_bar)
        e2.record(st)
        e2.synchronize()
        t_fwd.append(e0.elapsed_time(e1))
        t_tot.append(e0.elapsed_time(e2))
        t_adj.append(t_tot[-1] - t_fwd[-1])
    steps = int(out["nsteps"].sum().item())
    t_all = float(np.median(t_tot)) * 1e-3
    t_f = float(np.median(t_fwd)) * 1e-3
    t_a = float(np.median(t_adj)) * 1e-3
    adj_roof = None
    if peak:
        achieved = ARM_ADJ_FLOP_PER_STEP * steps / t_a / 1e12
        adj_roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "kernel": f"k_adjoint_rev<{adj_lanes}>", "flop_per_env_step": ARM_ADJ_FLOP_PER_STEP,
                    "work": "oracle count: every accepted step once in the counting derivative scalar "
                            "(recompute + linearised step), python -m oracle.count_flops chain_cube"}
        fps = _adjoint_flops_per_step(adj_lanes)
        if fps is not None:
            ex = fps * steps / t_a / 1e12
            adj_roof["executed"] = {"achieved": ex, "frac": ex / peak,
                                    "source": "ncu FP64 thread operations, profiles/adjoint_rev_chain_cube.json"}
    parity = None
    if parity_envs:
        parity = _grad_parity(m, out, xT_bar, gx, gu, inp, sc, list(parity_envs))
    return {"workload": "chain_cube (7 hinges + cube, NI=50, T=2 s, K=32)", "envs": B, "adjoint_roofline": adj_roof,
            "grad_rollouts_per_s": B / t_all, "env_steps_per_s": steps / t_all, "forward_s": t_f,
            "adjoint_s": t_a, "total_s_median": t_all, "total_s_p90": float(np.percentile(t_tot, 90)) * 1e-3,
            "reps": len(t_tot), "env_steps": steps, "adjoint_kernel": "reverse",
            "forward_frac": (ARM_FLOP_PER_STEP * steps / t_f / 1e12 / peak) if peak else None,
            "lanes": {"forward": fwd_lanes, "adjoint": adj_lanes, "adjoint_tuning_ms": adj_ms},
            "finite": bool(torch.isfinite(gu).all().item()), "parity_vs_oracle": parity}


def sysid_leg(dmx, dev, world=1, rank=0, B=4096, parity_envs=(0, 1)):
    """System identification step (Sec. 5.1 / App. E.2) on seeded cube tosses:
    observed final positions come from a rollout of a model with other contact
    parameters (mu 0.6, t_c 4 ms instead of 1.0 and 5 ms); the loss is the
    squared final-position error summed over the tosses, and one step is a
    taped forward rollout plus the gradient w.r.t. the model parameters
    (dmx_rollout_grad_params), summed over this GPU's tosses and, with N > 1,
    over all ranks (all-reduce of np doubles: the one collective of the path).
    The per-environment gradients of `parity_envs` are compared with the CPU
    oracle's discrete adjoint along the GPU's step sizes."""
    import torch
    from paper_2506_14186_gb300 import workloads as W
    sc = W.toss_scene()
    true_sc = W.box_scene(solref=(0.004, 1.0), mu=0.6)
    inp = W.toss_inputs(B, seed=1006 + rank)
    m, mt = dmx.Model(sc), dmx.Model(true_sc)
    x0 = torch.tensor(np.ascontiguousarray(inp["x0"].T), device=dev)
    T = torch.tensor(inp["T"], device=dev)
    obs = dmx.rollout(mt, x0, T)["xT"][0:3].clone()
    st = torch.cuda.current_stream()

    def step():
        out = dmx.rollout(m, x0, T, K=16, tape=True)
        xT_bar = torch.zeros_like(out["xT"])
        xT_bar[0:3] = 2 * (out["xT"][0:3] - obs)
        gx, _, pb, ps = dmx.rollout_grad_params(out["tape"], xT_bar)
        allreduce_sum_(ps, world)
        return out, xT_bar, gx, pb, ps
    step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    out, xT_bar, gx, pb, ps = step()
    e1.record(st)
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    parity = None
    if rank == 0 and parity_envs:
        import oracle
        envs = list(parity_envs)
        hlog, n = out["tape"].read()
        idx = torch.tensor(envs, device=dev)
        n = n[idx].cpu().numpy()
        hl = hlog[: int(n.max()), idx].cpu().numpy().T
        o = oracle.OracleModel(sc).batch_replay_grad(inp["x0"][envs], inp["T"][envs], hl, n,
                                                     xT_bar.cpu().numpy().T[envs], params=True)
        g = pb.cpu().numpy().T[envs]
        scale = np.maximum(np.maximum(np.abs(o["p_bar"]), np.abs(o["p_bar"]).max(axis=1, keepdims=True)), 1e-300)
        parity = {"envs": envs, "p_bar": float(np.max(np.abs(g - o["p_bar"]) / scale)), "bar": 1e-6}
    return {"workload": "cube tosses, final-position loss against a model with mu 0.6 and t_c 4 ms",
            "envs_per_gpu": B, "params": ["t_c", "phi_d", "d_o", "d_w", "width", "midpoint", "mu", "mass", "side"],
            "grad_rollouts_per_s": B * world / t, "s": t, "env_steps": int(out["nsteps"].sum().item()),
            "p_bar_sum": ps.cpu().numpy().tolist(), "reduction": "in-library row sums, all-reduce over ranks",
            "kernel": "k_adjoint (forward-mode, one direction per lane)", "parity_vs_oracle": parity}


def _grad_parity(m, out, xT_bar, gx, gu, inp, scene, envs):
    """Largest relative gradient error of the sampled environments against the
    CPU oracle's discrete adjoint along the GPU's accepted step sizes
    (componentwise |g - o| / max(|o|, ||o||_inf))."""
    import torch

    import oracle
    hlog, n = out["tape"].read()
    idx = torch.tensor(envs, device=hlog.device)
    n = n[idx].cpu().numpy()
    hl = hlog[: int(n.max()), idx].cpu().numpy().T
    om = oracle.OracleModel(scene)
    o = om.batch_replay_grad(inp["x0"][envs], inp["T"][envs], hl, n, xT_bar.cpu().numpy().T[envs],
                             ctrl=inp["ctrl"][envs], NI=inp["NI"])
    g_x = gx.cpu().numpy().T[envs]
    g_u = np.transpose(gu.cpu().numpy(), (2, 0, 1))[envs]

    def rel(a, b):
        a, b = a.reshape(len(envs), -1), b.reshape(len(envs), -1)
        scale = np.maximum(np.maximum(np.abs(b), np.abs(b).max(axis=1, keepdims=True)), 1e-300)
        return float(np.max(np.abs(a - b) / scale))
    return {"envs": envs, "x0_bar": rel(g_x, o["x0_bar"]), "ctrl_bar": rel(g_u, o["ctrl_bar"]), "bar": 1e-6}


# ------------------------------------------------------------------ every workload
def _events_time(fn):
    import torch
    st = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    r = fn()
    e1.record(st)
    e1.synchronize()
    return r, e0.elapsed_time(e1) * 1e-3


def _oracle_fwd(scene, inp, n):
    """Oracle batch rollout of the first n environments on all host cores: (env-steps/s, seconds)."""
    import oracle
    m = oracle.OracleModel(scene)
    ctrl = None if inp["ctrl"] is None else inp["ctrl"][:n]
    t0 = time.perf_counter()
    r = m.batch_rollout(inp["x0"][:n], inp["T"][:n], ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"],
                        h0=inp["h0"], max_steps=inp["max_steps"])
    dt = time.perf_counter() - t0
    return float(r["nsteps"].sum()) / dt, dt


def _oracle_grad(scene, inp, n, xT_bar):
    """Oracle forward + discrete adjoint of the first n environments: (grad-rollouts/s, seconds)."""
    import oracle
    m = oracle.OracleModel(scene)
    ctrl = None if inp["ctrl"] is None else inp["ctrl"][:n]
    t0 = time.perf_counter()
    m.batch_grad(inp["x0"][:n], inp["T"][:n], xT_bar[:n], ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"],
                 h0=inp["h0"], max_steps=inp["max_steps"])
    dt = time.perf_counter() - t0
    return n / dt, dt


def run_all(args):
    """Forward and fwd+adjoint rates of the four rollout workloads at their
    stated batch sizes, billiard shots with the discrete and the continuous
    adjoint, with the CPU oracle timed on bounded samples."""
    import torch

    import paper_2506_14186_gb300 as dmx
    from paper_2506_14186_gb300 import _build, autotune
    from paper_2506_14186_gb300 import workloads as W
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    cores = os.cpu_count() or 1

    def d(a):
        return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    def tensors(inp, n):
        ctrl = None if inp["ctrl"] is None else d(np.transpose(inp["ctrl"][:n], (1, 2, 0)))
        return d(inp["x0"][:n].T), d(inp["T"][:n]), ctrl

    def forward(m, inp, n, reps=3):
        x0, T, ctrl = tensors(inp, n)
        kw = dict(ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
        lanes, tuned = autotune.tune_forward(m, x0, torch.clamp(T, max=0.25), **kw)
        best, out = 1e30, None
        for _ in range(reps):
            out, t = _events_time(lambda: dmx.rollout(m, x0, T, lanes=lanes, **kw))
            best = min(best, t)
        steps = int(out["nsteps"].sum().item())
        assert int((out["status"] != 0).sum().item()) == 0
        return {"envs": n, "env_steps": steps, "s": best, "env_steps_per_s": steps / best, "lanes": lanes}

    def gradient(m, inp, n, xT_bar_fn, K=None):
        x0, T, ctrl = tensors(inp, n)
        kw = dict(ctrl=ctrl, NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
        fl, _ = autotune.tune_forward(m, x0, torch.clamp(T, max=0.25), **kw)
        al, _ = autotune.tune_adjoint(m, x0, T, K=K or 32, **kw)
        tuned_k = None
        if K is None:
            K, tuned_k = autotune.tune_checkpoint(m, x0, T, **kw)
        m.set_lanes(n, fl)

        def fwd_adj():
            out = dmx.rollout(m, x0, T, K=K, tape=True, **kw)
            return out, dmx.rollout_grad(out["tape"], xT_bar_fn(out))
        if n <= 4096:
            _events_time(fwd_adj)                        # warm-up (large batches are warm from the tuning)
        (out, (gx, gu)), t = _events_time(fwd_adj)
        steps = int(out["nsteps"].sum().item())
        return {"envs": n, "env_steps": steps, "s": t, "grad_rollouts_per_s": n / t, "env_steps_per_s": steps / t,
                "K": K, "K_tuning_ms": tuned_k, "lanes": {"forward": fl, "adjoint": al},
                "finite": bool(torch.isfinite(gx).all().item())}

    res = {}
    rng = np.random.default_rng(0)
    # 1. bouncing balls, B = 16: forward; gradient of the final height w.r.t. the state (v0 entries)
    sc, inp = W.ball_scene(), W.ball_inputs(16)
    m = dmx.Model(sc)

    def height_bar(out):
        b = torch.zeros_like(out["xT"])
        b[2] = 1.0
        return b
    xb = np.zeros((16, 13)); xb[:, 2] = 1.0
    r = {"forward": forward(m, inp, 16), "fwd_adjoint": gradient(m, inp, 16, height_bar, K=32)}
    rate, sec = _oracle_fwd(sc, inp, 16)
    grate, gsec = _oracle_grad(sc, inp, 16, xb)
    r["cpu_oracle"] = {"env_steps_per_s": rate, "grad_rollouts_per_s": grate, "cores": cores, "sample": "all 16"}
    res["ball_B16"] = r
    # 2. box pushes, B = 4096: forward in the three launch forms
    sc, inp = W.box_scene(), W.box_push_inputs(4096)
    m = dmx.Model(sc)
    r = {"forward": forward(m, inp, 4096)}
    x0, T, _ = tensors(inp, 4096)
    for form in ("graph", "step"):
        out, t = _events_time(lambda: dmx.rollout(m, x0, T, lanes=r["forward"]["lanes"], form=form, rtol=inp["rtol"],
                                                  atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"]))
        r[f"forward_{form}"] = {"s": t, "env_steps_per_s": int(out["nsteps"].sum().item()) / t}
    rate, sec = _oracle_fwd(sc, inp, 512)
    r["cpu_oracle"] = {"env_steps_per_s": rate, "cores": cores, "sample": "first 512 of 4096"}
    res["box_push_B4096"] = r
    # 3. arm pushes cube, B = 16384: forward; forward + adjoint of the squared cube-to-goal distance (K = 32)
    sc, inp = W.chain_cube_scene(), W.chain_inputs(16384)
    m = dmx.Model(sc)
    goal = torch.tensor(W.chain_goal(), device=dev)[:, None]

    def goal_bar(out):
        b = torch.zeros_like(out["xT"])
        b[7:10] = 2 * (out["xT"][7:10] - goal)
        return b
    r = {"forward": forward(m, inp, 16384, reps=1), "fwd_adjoint": gradient(m, inp, 16384, goal_bar, K=32)}
    rate, sec = _oracle_fwd(sc, inp, 64)
    gb = np.zeros((4, 27)); gb[:, 7:10] = 1.0
    grate, gsec = _oracle_grad(sc, inp, 4, gb)
    r["cpu_oracle"] = {"env_steps_per_s": rate, "grad_rollouts_per_s": grate, "cores": cores,
                       "sample": "forward: first 64 of 16384; gradient: first 4"}
    res["chain_cube_B16384"] = r
    # 4. quadruped, B = 8192: forward; forward + adjoint (autotuned lanes and K) on the first 2048
    sc, inp = W.quadruped_scene(), W.quadruped_inputs(8192)
    m = dmx.Model(sc)

    def torso_bar(out):
        b = torch.zeros_like(out["xT"])
        b[0:3] = 1.0
        return b
    r = {"forward": forward(m, inp, 8192, reps=1), "fwd_adjoint": gradient(m, inp, 8192, torso_bar)}
    rate, sec = _oracle_fwd(sc, inp, 64)
    tb = np.zeros((2, 37)); tb[:, 0:3] = 1.0
    grate, gsec = _oracle_grad(sc, inp, 2, tb)
    r["cpu_oracle"] = {"env_steps_per_s": rate, "grad_rollouts_per_s": grate, "cores": cores,
                       "sample": "forward: first 64 of 8192; gradient: first 2"}
    res["quadruped_B8192"] = r
    res["billiard_B4096"] = _billiard_leg(dmx, W, d, cores)
    return {"metric": METRIC, "impl": "ours", "dtype": "f64", "data": "synthetic (seeded)", "all": res}


def _billiard_leg(dmx, W, d, cores, B=4096):
    """Billiard shots (Sec. 4, App. C.4; B = 4096, T = 0.5 s): forward with a
    tape, the discrete adjoint (DTO) and the continuous adjoint by backsolve
    (OTD) of the target ball's final x, plain and straight-through with
    contacts from distance; the CPU oracle's OTD on a sample."""
    import torch
    import oracle
    inp = W.billiard_inputs(B)
    out = {}
    for label, sc, cfd in (("plain", W.billiard_scene(), False), ("cfd", W.billiard_scene(**W.CFD_OPTIONS), True)):
        m = dmx.Model(sc)
        x0, T = d(inp["x0"].T), d(inp["T"])
        w = torch.zeros((26, B), dtype=torch.float64, device=x0.device)
        w[7] = 1.0
        kw = dict(rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
        _events_time(lambda: dmx.rollout(m, x0, T, tape=True, **kw))          # warm-up
        f, tf = _events_time(lambda: dmx.rollout(m, x0, T, tape=True, **kw))
        _, tdto = _events_time(lambda: dmx.rollout_grad(f["tape"], w, cfd=cfd))
        (gx, _, steps, st), totd = _events_time(lambda: dmx.rollout_grad_otd(m, f["xT"], T, w, cfd=cfd, **kw))
        om = oracle.OracleModel(sc)
        n = 64
        t0 = time.perf_counter()
        om.batch_grad_otd(inp["x0"][:n], inp["T"][:n], w[:, :n].T.cpu().numpy(), cfd=cfd, **kw)
        cpu = n / (time.perf_counter() - t0)
        out[label] = {"forward_s": tf, "dto_s": tdto, "otd_s": totd,
                      "forward_env_steps": int(f["nsteps"].sum().item()),
                      "otd_backward_steps": int(steps.sum().item()), "otd_status_ok": bool((st == 0).all().item()),
                      "otd_grad_rollouts_per_s": B / (tf + totd), "dto_grad_rollouts_per_s": B / (tf + tdto),
                      "cpu_oracle_otd_grad_rollouts_per_s": cpu, "cpu_cores": cores, "cpu_sample": f"first {n} of {B}"}
    return out


# ------------------------------------------------------------------ reference arm (the CPU oracle)
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    from paper_2506_14186_gb300 import workloads as W
    inp = W.box_push_inputs(4096)
    for _ in range(args.warmup):
        oracle_rate(inp, budget_s=0.0, first=64, max_envs=64)
    rates, secs = [], []
    for k in range(args.steps):
        rate, sample, cores, sec = oracle_rate(inp, budget_s=0.0, first=256, max_envs=256)
        rates.append(rate)
        secs.append(sec)
    value = float(np.mean(rates))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(secs)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded box pushes)",
            "config": dict(WORKLOAD, parallelism="host threads"), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: the first 256 of the 4096 environments"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ serving
def make_requests(n, seed=5005):
    """Seeded request mix: model in {ball, box, chain_cube} uniform, B ~ U{64..1024},
    T ~ U[0.2, 2] s (arm: NI = round(25 T) torque intervals), half forward-only,
    half forward + adjoint (loss = squared final position of the last body)."""
    from paper_2506_14186_gb300 import workloads as W
    g = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        name = ("ball", "box", "chain_cube")[int(g.integers(0, 3))]
        B = int(g.integers(64, 1025))
        T = float(g.uniform(0.2, 2.0))
        grad = bool(g.integers(0, 2))
        if name == "chain_cube":
            NI = max(1, int(round(25 * T)))
            inp = W.chain_inputs(B, seed=seed + i, T=T, NI=NI)
        else:
            NI = 1
            inp = W.INPUTS[name](B, seed=seed + i, T=T)
        reqs.append({"name": name, "B": B, "T": T, "NI": NI, "grad": grad, "inp": inp})
    return reqs


def serving_leg(dmx, W, requests=40, warmup=5, rate=200.0, seed=5005):
    """Served MPC requests (seeded mix, Poisson arrivals at `rate`): latency
    (submit -> outputs in the caller's host buffers) and rollouts/s of three
    arms on the same requests and arrival times:
      continuous_batching  -- the request server (dmx_submit / dmx_poll): requests
                              admitted as slots and memory free up, kernels of
                              concurrent requests overlap on the device;
      sequential_persistent -- no server: one request at a time in arrival order,
                              the same fused persistent kernels;
      plain_per_request    -- one request at a time, forward pass by one launch
                              per step attempt (plain form).
    Latency of the sequential arms is counted from the arrival time."""
    import torch
    models = {n: dmx.Model(W.SCENES[n]()) for n in ("ball", "box", "chain_cube")}
    total = warmup + requests
    reqs = make_requests(total, seed=seed)
    g = np.random.default_rng(seed + 72)
    arrivals = np.cumsum(g.exponential(1.0 / rate, total))
    host = []
    for r in reqs:
        m = models[r["name"]]
        inp = r["inp"]
        x0 = np.ascontiguousarray(inp["x0"].T)
        ctrl = None if inp["ctrl"] is None else np.ascontiguousarray(np.transpose(inp["ctrl"], (1, 2, 0)))
        xT_bar = None
        if r["grad"]:
            xT_bar = np.zeros((m.nx, r["B"]))
            xT_bar[2] = 1.0                          # d(height of the first free-joint coordinate)
        host.append((m, x0, np.ascontiguousarray(inp["T"]), ctrl, xT_bar))

    def served():
        srv = dmx.Server(device_bytes=96 << 30, max_inflight=32, nstreams=16)
        t0 = time.perf_counter()
        tickets, lat, done = {}, {}, set()
        i = 0
        while len(done) < total:
            now = time.perf_counter() - t0
            while i < total and arrivals[i] <= now:
                m, x0, T, ctrl, xb = host[i]
                r = reqs[i]
                tickets[i] = srv.submit(m, x0, T, ctrl=ctrl, NI=r["NI"], grad=r["grad"], xT_bar=xb)
                i += 1
            for j, t in list(tickets.items()):
                if j in done:
                    continue
                o = srv.poll(t)
                if o is not None:
                    lat[j] = o["latency_s"]
                    done.add(j)
            time.sleep(2e-4)
        makespan = time.perf_counter() - t0
        srv.close()
        return lat, makespan

    def sequential(form):
        def run():
            dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
            t0 = time.perf_counter()
            lat = {}
            for j in range(total):
                while time.perf_counter() - t0 < arrivals[j]:
                    time.sleep(1e-4)
                m, x0, T, ctrl, xb = host[j]
                r = reqs[j]
                out = dmx.rollout(m, dev(x0), dev(T), ctrl=None if ctrl is None else dev(ctrl), NI=r["NI"], form=form,
                                  tape=r["grad"])
                if r["grad"]:
                    gx, gu = dmx.rollout_grad(out["tape"], dev(xb))
                    gx.cpu()
                out["xT"].cpu()
                lat[j] = time.perf_counter() - t0 - arrivals[j]
            return lat, time.perf_counter() - t0
        return run

    res = {}
    for name, fn in (("continuous_batching", served), ("sequential_persistent", sequential("persistent")),
                     ("plain_per_request", sequential("step"))):
        lat, makespan = fn()
        vals = np.array([lat[j] for j in range(warmup, total)])
        rollouts = sum(reqs[j]["B"] for j in range(total))
        res[name] = {"p50_s": float(np.percentile(vals, 50)), "p99_s": float(np.percentile(vals, 99)),
                     "mean_s": float(vals.mean()), "rollouts_per_s": rollouts / makespan, "makespan_s": makespan}
    res["config"] = {"arrivals": f"Poisson {rate}/s", "requests": requests, "warmup_requests": warmup,
                     "mix": "ball/box/chain_cube uniform, B~U{64..1024}, T~U[0.2,2] s, 50% fwd+adjoint"}
    return res


def run_serving(args):
    import torch

    import paper_2506_14186_gb300 as dmx
    from paper_2506_14186_gb300 import _build
    from paper_2506_14186_gb300 import workloads as W
    _build.build()
    torch.cuda.set_device(0)
    res = serving_leg(dmx, W, requests=args.requests, warmup=args.warmup_requests, rate=args.rate)
    head = res["continuous_batching"]
    return {"metric": METRIC, "value": head["p50_s"], "unit": "s (p50 request latency)", "n_gpus": 1,
            "higher_is_better": False, "steps": args.requests, "warmup": args.warmup_requests,
            "dtype": "f64", "data": "synthetic (seeded request mix)", "vs_baseline": None,
            "config": {"workload": "served MPC requests", **res["config"]}, "serving": res}


# ------------------------------------------------------------------ integrator comparison
def toss_reference(scene, inp, n, eps=1e-4, rtol=1e-11):
    """Reference loss (final x of the cube) and gradient w.r.t. the initial
    velocity of the first n tosses: the CPU oracle at rtol 1e-11 and central
    differences (eps = 1e-4) of that tight-tolerance rollout, as the paper's
    ground truth is built (Fig. 12: finite differences of an adaptive solver
    at tolerance 1e-12)."""
    import oracle
    m = oracle.OracleModel(scene)
    X, T = inp["x0"][:n], inp["T"][:n]

    def loss(Xp):
        return m.batch_rollout(Xp, T, rtol=rtol, atol=rtol * 1e-2, h0=1e-4, max_steps=10 ** 6)["xT"][:, 0]
    G = np.zeros((n, 3))
    for k in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, 7 + k] += eps
        Xm[:, 7 + k] -= eps
        G[:, k] = (loss(Xp) - loss(Xm)) / (2 * eps)
    return loss(X), G


def run_pareto(args):
    """Error of the loss and of its gradient vs GPU runtime for fixed-step
    semi-implicit Euler and the adaptive Dormand-Prince and Tsitouras schemes
    (the paper's Fig. 12 and Sec. 3.1 comparison) on 2048 seeded cube tosses
    (T = 1 s, solref 0.005 s): forward and forward+adjoint batch times on the
    GPU; errors of the sampled tosses against the tight-tolerance reference."""
    import torch

    import paper_2506_14186_gb300 as dmx
    from paper_2506_14186_gb300 import _build
    from paper_2506_14186_gb300 import workloads as W
    _build.build()
    torch.cuda.set_device(0)
    sc, inp = W.toss_scene(), W.toss_inputs(args.pareto_envs)
    nref = min(args.pareto_sample, args.pareto_envs)
    t0 = time.perf_counter()
    ref_loss, ref_grad = toss_reference(sc, inp, nref)
    t_ref = time.perf_counter() - t0
    m = dmx.Model(sc)
    B = args.pareto_envs
    x0 = torch.tensor(np.ascontiguousarray(inp["x0"].T), device="cuda")
    T = torch.tensor(inp["T"], device="cuda")
    xT_bar = torch.zeros((13, B), dtype=torch.float64, device="cuda")
    xT_bar[0] = 1.0
    configs = [("euler", {"h0": h}) for h in (2e-3, 1e-3, 5e-4, 2.5e-4, 1.25e-4, 6.25e-5)]
    for method in ("dopri5", "tsit5"):
        configs += [(method, {"rtol": r, "atol": r * 1e-2}) for r in (1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9)]
    points = []
    for method, kw in configs:
        a = dict(kw, max_steps=40000, method=method, K=32)
        dmx.rollout(m, x0, torch.clamp(T, max=0.05), **a)                  # warm-up
        out, t_f = _events_time(lambda: dmx.rollout(m, x0, T, **a))
        (out, (gx, _)), t_g = _events_time(
            lambda: (lambda o: (o, dmx.rollout_grad(o["tape"], xT_bar)))(dmx.rollout(m, x0, T, tape=True, **a)))
        assert int((out["status"] != 0).sum().item()) == 0, (method, kw)
        loss = out["xT"][0, :nref].cpu().numpy()
        grad = gx[7:10, :nref].cpu().numpy().T
        le = np.abs(loss - ref_loss) / np.maximum(np.abs(ref_loss), 1e-12)
        ge = np.linalg.norm(grad - ref_grad, axis=1) / np.linalg.norm(ref_grad, axis=1)
        points.append({"method": method, **{k: v for k, v in kw.items()},
                       "steps_per_env": float(out["nsteps"].double().mean().item()),
                       "forward_s": t_f, "fwd_adjoint_s": t_g,
                       "loss_rel_err_median": float(np.median(le)), "grad_rel_err_median": float(np.median(ge)),
                       "grad_rel_err_p90": float(np.percentile(ge, 90))})

    def front(key_t, key_e):
        pts = sorted(points, key=lambda p: p[key_t])
        out, best = [], float("inf")
        for p in pts:
            if p[key_e] < best:
                best = p[key_e]
                out.append(f"{p['method']} {p.get('h0', p.get('rtol'))}")
        return out
    return {"metric": "error of loss and gradient vs runtime (integrator comparison)", "impl": "ours",
            "dtype": "f64", "data": "synthetic (seeded cube tosses)",
            "config": {"workload": "cube toss", "B": B, "T_s": 1.0, "solref": [0.005, 1.0],
                       "loss": "final x position", "gradient": "w.r.t. the initial velocity",
                       "reference": f"CPU oracle rtol 1e-11, central differences eps 1e-4, first {nref} tosses "
                                    f"({t_ref:.1f} s)"},
            "points": points, "front_gradient": front("fwd_adjoint_s", "grad_rel_err_median"),
            "front_loss": front("forward_s", "loss_rel_err_median")}


def main():
    args = parse()
    if args.serving:
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.all:
        print(json.dumps(run_all(args)), flush=True)
        return
    if args.pareto:
        print(json.dumps(run_pareto(args)), flush=True)
        return
    if args.grad_only:
        import torch
        import paper_2506_14186_gb300 as dmx
        from paper_2506_14186_gb300 import _build
        _build.build()
        print(json.dumps(grad_leg(dmx, torch.device("cuda", 0), B=args.grad_envs, adj_lanes=args.adj_lanes)),
              flush=True)
        return
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
