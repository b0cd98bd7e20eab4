"""The replicated (N > 1) paths of bench.py on CPU with gloo, world size 2: the max-over-ranks
timing rule, and the reference arm's rank policy (rank 0 runs, the others return nothing)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(torch, 1.5 + rank, world)
        ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), rank, world) if rank == 1 else "skip"
        out.put((rank, got, ref))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_reference_rank_policy():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]  # every rank sees the slowest rank's time
    assert res[1][2] is None                  # rank 1 of the reference arm does no work


def test_reference_slices_cover_the_operator():
    import numpy as np
    import scipy.sparse as sp

    A = sp.random(103, 50, density=0.1, format="csr", random_state=np.random.default_rng(0))
    sl = bench.reference_slices([(A, 3)], 7)[0]
    assert len(sl) == 7 and sum(s.shape[0] for s, _ in sl) == 103
    assert sum(s.nnz for s, _ in sl) == A.nnz


def test_reference_arm_line():
    """The reference arm's JSON fields on one step (rank 0, N = 1): the oracle on host cores."""
    out = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), 0, 1)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC and out["value"] > 0
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == out["value"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == out["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
