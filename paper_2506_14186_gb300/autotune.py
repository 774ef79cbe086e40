"""Autotuner: lanes per environment for a (model, batch size, kernel).

Every lane count whose workspace fits in shared memory is timed on the
caller's own inputs (CUDA events, after one warm-up run); the fastest is
recorded in the library (dmx_set_lanes) so that later calls with lanes = 0 use
it.  Results are cached per process by (scene name, B, kind).  The adjoint
kernel is timed on the caller's batch over a short horizon (its lane choice
depends on the batch size and the model, not on the step count).  The
checkpoint interval K of the tape is chosen the same way: taped forward plus
adjoint timed for each candidate K.
"""

from __future__ import annotations

import paper_2506_14186_gb300 as dmx

LANES = (1, 2, 4, 8, 16, 32)
_cache: dict = {}


def tune_forward(model, x0, T, ctrl=None, NI=1, reps=1, candidates=LANES, **kw):
    """Times a forward rollout for each candidate lane count; returns
    (best_lanes, {lanes: ms})."""
    import torch
    key = (model.scene.get("name"), x0.shape[1], 0)
    if key in _cache:
        model.set_lanes(x0.shape[1], _cache[key][0])
        return _cache[key]
    times = {}
    for G in candidates:
        try:
            dmx.rollout(model, x0, T, ctrl=ctrl, NI=NI, lanes=G, **kw)        # warm-up (and fit check)
        except dmx.DmxError:
            continue
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            dmx.rollout(model, x0, T, ctrl=ctrl, NI=NI, lanes=G, **kw)
        e1.record(st)
        e1.synchronize()
        times[G] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    model.set_lanes(x0.shape[1], best)
    _cache[key] = (best, times)
    return best, times


ADJ_LANES = (2, 4, 8, 16, 32)


def tune_adjoint(model, x0, T, ctrl=None, NI=1, horizon=0.1, candidates=ADJ_LANES, **kw):
    """Times the reverse-mode adjoint kernel for each candidate lane count on a
    taped rollout of the caller's batch with horizons capped at `horizon`
    seconds; returns (best_lanes, {lanes: ms})."""
    import torch
    B = x0.shape[1]
    key = (model.scene.get("name"), B, 2)
    if key in _cache:
        model.set_lanes(B, _cache[key][0], grad=2)
        return _cache[key]
    out = dmx.rollout(model, x0, torch.clamp(T, max=horizon), ctrl=ctrl, NI=NI, tape=True, **kw)
    xT_bar = torch.ones_like(out["xT"])
    model.set_adjoint("reverse")
    times = {}
    for G in candidates:
        model.set_lanes(B, G, grad=2)
        try:
            dmx.rollout_grad(out["tape"], xT_bar)                          # warm-up (and fit check)
        except dmx.DmxError:
            continue
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        dmx.rollout_grad(out["tape"], xT_bar)
        e1.record(st)
        e1.synchronize()
        times[G] = e0.elapsed_time(e1)
    best = min(times, key=times.get)
    model.set_lanes(B, best, grad=2)
    _cache[key] = (best, times)
    return best, times


K_CANDIDATES = (8, 16, 32, 64)


def tune_checkpoint(model, x0, T, ctrl=None, NI=1, horizon=0.2, candidates=K_CANDIDATES, **kw):
    """Times a taped forward rollout plus its adjoint (current lane choices)
    for each candidate checkpoint interval K on the caller's batch with
    horizons capped at `horizon` seconds; returns (best_K, {K: ms}).  A K
    whose tape or adjoint scratch does not fit is skipped."""
    import torch
    B = x0.shape[1]
    key = (model.scene.get("name"), B, "K")
    if key in _cache:
        return _cache[key]
    Tc = torch.clamp(T, max=horizon)
    times = {}
    for K in candidates:
        try:
            out = dmx.rollout(model, x0, Tc, ctrl=ctrl, NI=NI, K=K, tape=True, **kw)   # warm-up (and fit check)
            dmx.rollout_grad(out["tape"], torch.ones_like(out["xT"]))
        except dmx.DmxError:
            continue
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        out = dmx.rollout(model, x0, Tc, ctrl=ctrl, NI=NI, K=K, tape=True, **kw)
        dmx.rollout_grad(out["tape"], torch.ones_like(out["xT"]))
        e1.record(st)
        e1.synchronize()
        times[K] = e0.elapsed_time(e1)
    best = min(times, key=times.get)
    _cache[key] = (best, times)
    return best, times
