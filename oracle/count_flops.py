"""Algorithmic FP64 work per accepted step of each workload, counted by the
oracle's instrumented scalar (add/sub/mul/div/sqrt and transcendentals = 1
flop each) over a seeded sample of environments.  TEST/MEASUREMENT
INFRASTRUCTURE: run as `python -m oracle.count_flops [workload ...]`; the
printed figures are the per-unit work the benchmark's rooflines use.

Three figures per workload:
  * forward, with the oracle's active-set search (Newton from the
    unconstrained acceleration in every right-hand side);
  * forward, each constraint solve counted as started at its final active set
    (one Newton system and one residual check): the work of the method when
    the search is warm-started, as the CUDA path does; the benchmark's
    forward roofline uses this figure;
  * adjoint: every accepted step once in the counting derivative scalar
    (primal recompute + linearised step; a reverse sweep costs the
    multiply-adds of the forward linearisation by the transposition
    principle), the benchmark's adjoint roofline.
"""

import sys

import numpy as np

import oracle
from paper_2506_14186_gb300 import workloads as W


def per_step(name, n=64, adjoint=False, **kw):
    sc = W.SCENES[name]()
    inp = W.INPUTS[name](max(n, 64), **kw)
    m = oracle.OracleModel(sc)
    out = {"search": 0, "warm": 0, "adjoint": 0, "steps": 0, "rhs": 0}
    for e in range(n):
        ctrl = None if inp["ctrl"] is None else inp["ctrl"][e]
        a = dict(ctrl=ctrl, T=float(inp["T"][e]), NI=inp["NI"], rtol=inp["rtol"], atol=inp["atol"], h0=inp["h0"],
                 max_steps=inp["max_steps"])
        f, st = m.count_flops(inp["x0"][e], search=True, **a)
        fw, _ = m.count_flops(inp["x0"][e], search=False, **a)
        out["search"] += f; out["warm"] += fw; out["steps"] += st["nsteps"]; out["rhs"] += st["nrhs"]
        if adjoint:
            fa, _ = m.count_adjoint_flops(inp["x0"][e], **a)
            out["adjoint"] += fa
    s = out["steps"]
    return {"search": out["search"] / s, "warm": out["warm"] / s, "adjoint": out["adjoint"] / s if adjoint else None,
            "rhs_per_step": out["rhs"] / s, "steps_per_env": s / n}


if __name__ == "__main__":
    names = sys.argv[1:] or ["ball", "box", "chain_cube", "quadruped"]
    for name in names:
        n = 16 if name in ("chain_cube", "quadruped") else 64
        r = per_step(name, n=n, adjoint=True)
        print(f"{name}: {r['search']:.0f} flop / accepted step with the active-set search, {r['warm']:.0f} "
              f"started at the final active set, adjoint {r['adjoint']:.0f} flop / accepted step; "
              f"{r['rhs_per_step']:.2f} right-hand sides / step, {r['steps_per_env']:.0f} steps / env ({n} envs)")
