"""Request server (dmx_submit / dmx_poll): a mix of forward and gradient
requests of three models, batch sizes and horizons, submitted while others
run, gives for every request exactly the result of the same request run alone
through dmx_rollout / dmx_rollout_grad (bitwise); memory-budget admission;
requests that can never fit are refused at submit."""

import numpy as np
import pytest

from paper_2506_14186_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmx():
    import torch
    from paper_2506_14186_gb300 import _build
    _build.build()
    import paper_2506_14186_gb300 as d
    assert torch.cuda.is_available()
    return d


def _requests(dmx):
    import torch  # noqa: F401
    rng = np.random.default_rng(7)
    models = {n: dmx.Model(W.SCENES[n]()) for n in ("ball", "box", "chain_cube")}
    reqs = []
    for i in range(12):
        name = ("ball", "box", "chain_cube")[i % 3]
        B = int(rng.integers(16, 96))
        T = float(rng.uniform(0.1, 0.4))
        NI = 4 if name == "chain_cube" else 1
        inp = W.INPUTS[name](B, seed=100 + i, **({"T": T, "NI": NI} if name == "chain_cube" else {"T": T}))
        grad = i % 2 == 1
        m = models[name]
        x0 = np.ascontiguousarray(inp["x0"].T)
        ctrl = None if inp["ctrl"] is None else np.ascontiguousarray(np.transpose(inp["ctrl"], (1, 2, 0)))
        xT_bar = rng.normal(size=(m.nx, B)) if grad else None
        reqs.append(dict(model=m, x0=x0, T=np.ascontiguousarray(inp["T"]), ctrl=ctrl, NI=NI, grad=grad,
                         xT_bar=xT_bar))
    return reqs


def _alone(dmx, r):
    import torch
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    m = r["model"]
    out = dmx.rollout(m, dev(r["x0"]), dev(r["T"]), ctrl=None if r["ctrl"] is None else dev(r["ctrl"]), NI=r["NI"],
                      K=32, tape=r["grad"])
    res = {"xT": out["xT"].cpu().numpy(), "status": out["status"].cpu().numpy()}
    if r["grad"]:
        gx, gu = dmx.rollout_grad(out["tape"], dev(r["xT_bar"]))
        res["x0_bar"] = gx.cpu().numpy()
        if gu is not None:
            res["ctrl_bar"] = gu.cpu().numpy()
    return res


def test_results_alone_equal_results_in_the_mix(dmx):
    reqs = _requests(dmx)
    srv = dmx.Server(device_bytes=16 << 30, max_inflight=6, nstreams=6)
    tickets = [srv.submit(r["model"], r["x0"], r["T"], ctrl=r["ctrl"], NI=r["NI"], grad=r["grad"], xT_bar=r["xT_bar"])
               for r in reqs]
    outs = [srv.wait(t, timeout=600) for t in tickets]
    srv.close()
    for r, o in zip(reqs, outs):
        a = _alone(dmx, r)
        np.testing.assert_array_equal(o["xT"], a["xT"])
        np.testing.assert_array_equal(o["status"], a["status"])
        assert o["latency_s"] > 0
        if r["grad"]:
            np.testing.assert_array_equal(o["x0_bar"], a["x0_bar"])
            if "ctrl_bar" in a:
                np.testing.assert_array_equal(o["ctrl_bar"], a["ctrl_bar"])


def test_memory_budget_admission(dmx):
    """A budget that holds one request at a time still completes a queue of
    requests; a request larger than the whole budget is refused at submit."""
    m = dmx.Model(W.box_scene())
    inp = W.box_push_inputs(64, T=0.2)
    x0, T = np.ascontiguousarray(inp["x0"].T), np.ascontiguousarray(inp["T"])
    srv = dmx.Server(device_bytes=30_000, max_inflight=4, nstreams=2)
    tickets = [srv.submit(m, x0, T) for _ in range(5)]
    outs = [srv.wait(t, timeout=300) for t in tickets]
    for o in outs[1:]:
        np.testing.assert_array_equal(o["xT"], outs[0]["xT"])
    big = W.box_push_inputs(2000, T=0.2)
    with pytest.raises(dmx.DmxError, match="server budget"):
        srv.submit(m, np.ascontiguousarray(big["x0"].T), np.ascontiguousarray(big["T"]))
    srv.close()


def test_concurrent_requests_overlap_on_the_device(dmx):
    """Requests admitted together run at the same time: four requests of 64
    box pushes (T = 1 s, each far from filling the GPU), submitted at once
    with pageable numpy buffers, all complete within 2x the latency of one
    request alone (issued one after another they would take ~4x), and each
    result equals the one of the request alone."""
    m = dmx.Model(W.box_scene())
    inp = W.box_push_inputs(64, T=1.0)
    x0, T = np.ascontiguousarray(inp["x0"].T), np.ascontiguousarray(inp["T"])
    srv = dmx.Server(device_bytes=4 << 30, max_inflight=8, nstreams=8)
    srv.wait(srv.submit(m, x0, T), timeout=300)                   # warm-up (lane choice, pools)
    alone = [srv.wait(srv.submit(m, x0, T), timeout=300) for _ in range(2)]
    t_alone = min(a["latency_s"] for a in alone)
    tickets = [srv.submit(m, x0, T) for _ in range(4)]
    outs = [srv.wait(t, timeout=300) for t in tickets]
    srv.close()
    t_four = max(o["latency_s"] for o in outs)
    assert t_four < 2.0 * t_alone, (t_four, t_alone)
    for o in outs:
        np.testing.assert_array_equal(o["xT"], alone[0]["xT"])
