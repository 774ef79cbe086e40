"""Multi-process sharding of environments (CPU, gloo, world size 2).

Environments are independent (each has its own step sequence), so the batch
shards across ranks with no collective on the data path; the only collectives
are the timing/count reductions of the benchmark.  These tests run two gloo
ranks on the CPU with the oracle as the per-rank integrator and check
  * that the halves of a batch integrated on two ranks and gathered equal the
    whole batch integrated in one process (bitwise: nothing couples the
    environments),
  * the benchmark's barrier / max / sum reductions over ranks, and
  * the one data-path exchange: model-parameter gradients of each rank's
    tosses summed over the ranks (all-reduce) equal the gradient of the whole
    batch in one process.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2506_14186_gb300 import workloads as W

    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.dist_init(w, "gloo")
    try:
        inp = W.box_push_inputs(8, T=0.05)
        lo, hi = r * 8 // w, (r + 1) * 8 // w
        m = oracle.OracleModel(W.box_scene())
        res = m.batch_rollout(inp["x0"][lo:hi], inp["T"][lo:hi], rtol=inp["rtol"], atol=inp["atol"],
                              h0=inp["h0"], max_steps=inp["max_steps"], nthreads=1)
        parts = [None] * w
        dist.all_gather_object(parts, (lo, hi, res["xT"], res["nsteps"]))
        bench.barrier(w)
        total = bench.reduce_sum(float(res["nsteps"].sum()), w)
        slowest = bench.reduce_max(float(r + 1), w)
        if r == 0:
            np.savez(out, xT=np.concatenate([p[2] for p in parts]), nsteps=np.concatenate([p[3] for p in parts]),
                     ranges=np.array([(p[0], p[1]) for p in parts]), total=total, slowest=slowest)
    finally:
        dist.destroy_process_group()


def test_env_shards_gloo(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2506_14186_gb300 import workloads as W
    oracle.build()
    out = str(tmp_path / "shard.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    assert got["ranges"].tolist() == [[0, 4], [4, 8]]

    inp = W.box_push_inputs(8, T=0.05)
    whole = oracle.OracleModel(W.box_scene()).batch_rollout(inp["x0"], inp["T"], rtol=inp["rtol"], atol=inp["atol"],
                                                           h0=inp["h0"], max_steps=inp["max_steps"], nthreads=2)
    assert np.array_equal(got["xT"], whole["xT"])
    assert np.array_equal(got["nsteps"], whole["nsteps"])
    assert float(got["total"]) == float(whole["nsteps"].sum())
    assert float(got["slowest"]) == 2.0


def test_single_rank_reductions_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(2.0, 1) == 2.0
    bench.barrier(1)
    bench.dist_init(1, "gloo")


def _sysid_worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_2506_14186_gb300 import workloads as W

    bench.dist_init(world, "gloo")
    try:
        inp = W.toss_inputs(6, T=0.3)
        lo, hi = rank * 6 // world, (rank + 1) * 6 // world
        ps = torch.tensor(_param_grads(W.toss_scene(), inp, lo, hi).sum(axis=0))
        bench.allreduce_sum_(ps, world)
        if rank == 0:
            np.save(out, ps.numpy())
    finally:
        dist.destroy_process_group()


def _param_grads(scene, inp, lo, hi):
    """Oracle parameter gradients of the final-x loss of tosses lo..hi-1."""
    import oracle
    m = oracle.OracleModel(scene)
    x0, T = inp["x0"][lo:hi], inp["T"][lo:hi]
    hl, n = [], []
    for e in range(hi - lo):
        r = m.rollout(x0[e], T=float(T[e]))
        hl.append(r["hlog"]); n.append(r["nsteps"])
    H = np.zeros((hi - lo, max(n)))
    for e in range(hi - lo):
        H[e, :n[e]] = hl[e]
    w = np.zeros((hi - lo, 13)); w[:, 0] = 1.0
    return m.batch_replay_grad(x0, T, H, np.array(n, dtype=np.int32), w, params=True, nthreads=1)["p_bar"]


def test_parameter_gradient_allreduce_gloo(tmp_path):
    import torch.multiprocessing as mp

    import oracle
    from paper_2506_14186_gb300 import workloads as W
    oracle.build()
    out = str(tmp_path / "psum.npy")
    mp.start_processes(_sysid_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    whole = _param_grads(W.toss_scene(), W.toss_inputs(6, T=0.3), 0, 6).sum(axis=0)
    np.testing.assert_allclose(got, whole, rtol=1e-12, atol=1e-12 * np.abs(whole).max())
    assert np.abs(whole).max() > 0
