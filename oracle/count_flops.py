"""Algorithmic FP64 work per accepted step of each workload, counted by the
oracle's instrumented scalar (add/sub/mul/div/sqrt and transcendentals = 1
flop each) over a seeded sample of environments.  TEST/MEASUREMENT
INFRASTRUCTURE: run as `python -m oracle.count_flops`; the printed figures are
the per-unit work the benchmark's roofline uses."""

import sys

import numpy as np

import oracle
from paper_2506_14186_gb300 import workloads as W


def per_step(name, n=64, **kw):
    sc = W.SCENES[name]()
    inp = W.INPUTS[name](max(n, 64), **kw)
    m = oracle.OracleModel(sc)
    flops = steps = rhs = 0
    for e in range(n):
        ctrl = None if inp["ctrl"] is None else inp["ctrl"][e]
        f, st = m.count_flops(inp["x0"][e], ctrl=ctrl, T=float(inp["T"][e]), NI=inp["NI"], rtol=inp["rtol"],
                              atol=inp["atol"], h0=inp["h0"], max_steps=inp["max_steps"])
        flops += f; steps += st["nsteps"]; rhs += st["nrhs"]
    return flops / steps, flops / rhs, steps / n


if __name__ == "__main__":
    names = sys.argv[1:] or ["ball", "box", "chain_cube", "quadruped"]
    for name in names:
        kw = {}
        if name == "box":
            kw = {}
        fs, fr, ns = per_step(name, n=16 if name in ("chain_cube", "quadruped") else 64)
        print(f"{name}: {fs:.0f} flop / accepted step, {fr:.0f} flop / right-hand side, {ns:.0f} steps / env")
