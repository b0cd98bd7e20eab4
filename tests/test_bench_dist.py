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


def _stub_result():
    """A result object shaped like a full run of the bench (every secondary section present and
    as long as a real run makes it)."""
    kern = [{"kernel": f"{o}-{d}-k{k}", "ms": 0.05, "gflops": 1000.0, "gbs": 4000.0, "frac_hbm": 0.6,
             "bytes": 3e8, "flops": 1e8, "fp64_frac": 0.8, "schedule": {"vec": 3, "lpr": 1, "stage": 0, "grid_cap": -1},
             "copy_frac": 0.8} for o, k in (("L", 3), ("G", 3), ("M", 1)) for d in ("f64", "f32")]
    sweep = [{"dtype": d, "format": f, "k": k, "ms": 0.1, "gflops": 500.0, "gbs": 3000.0, "frac_hbm": 0.5,
              "ai_flop_per_byte": 0.3, "speedup_vs_k_spmv": 2.0, "schedule": {"vec": 4, "lpr": 1, "stage": 2, "grid_cap": 0}}
             for d in ("f64", "f32") for f in ("csr", "sell") for k in (1, 2, 3, 4, 8, 16, 32)]
    big = {f"field{i}": [0.123456789] * 40 for i in range(30)}
    out = {"metric": bench.METRIC, "value": 1234.5, "unit": "GFLOP/s", "n_gpus": 1, "steps": 20, "warmup": 5,
           "ms_per_step": 0.35, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
           "data": "synthetic", "config": {"workload": bench.WORKLOAD, "n_cells": 2359296, "k": {"L": 3, "G": 3, "M": 1},
                                           "l2": "inputs larger than L2", "parallelism": "replicas"},
           "roofline": {"bound": "alu", "achieved": 1.07, "peak": 1.25, "unit": "TFLOP/s", "frac": 0.85,
                        "traffic": 3.07e8, "kernel": "L-f64-k3", "peak_source": "nominal", "peak_measured": 1.255,
                        "frac_of_measured": 0.85, "hbm_gbs": 3480.0, "hbm_frac_of_measured": 0.51},
           "kernels": kern, "gpu_launches": 120, "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [],
                                                           "samples": 30},
           "overlapped_step": {"streams": 2, "ms_per_step": 0.32, "value": 1330.0},
           "e2e": {"value": 172.0, "unit": "GFLOP/s", "ms_per_step": 2.47, "h2d_bytes_per_step": 311e6,
                   "d2h_bytes_per_step": 311e6},
           "ksweep": sweep, "poisson": {"k": 3, "rtol": 1e-10, "fp64_cg": {"ms": 252.0, "iters": [1001] * 3, **big},
                                        "ir_fp32_inner": {"ms": 118.0, **big}},
           "multigrid": {"runs": [{"case": "channel-k3", "ms": 30.0, **big}]},
           "batch": {"batch_graph_ms": 80.6, "sequential_fp64_cg_ms": 176.0, **big},
           "learned_guess": {"eval": {"prev_ir": {"ms_per_system": 18.7, **big}, "learned_ir": {"ms_per_system": 21.0}},
                             **big},
           "stencils": big, "refine": big, "projection": big, "extruded": big, "blas1": big, "rbc_spmm": big,
           "paper_context": bench.PAPER_CONTEXT,
           "cpu_baseline": {"value": 1.1, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": "x" * 100,
                            "all_cores": {"value": 10.7, "unit": "GFLOP/s", "cores": 16, "sample": "y" * 100}}}
    return out


def test_headline_line_is_short_and_parses(tmp_path, capsys):
    """The driver keeps only the end of stdout: the last line must be one short JSON object with
    the headline keys, and the full result must land in the detail file."""
    import json

    out = _stub_result()
    assert len(json.dumps(out)) > 20_000  # the full object would not survive a tail of a few KB
    detail = tmp_path / "detail.json"
    with open(detail, "w") as f:
        json.dump(out, f)
    print("earlier progress output " * 200)
    print(json.dumps(bench.headline(out, str(detail))))
    stdout = capsys.readouterr().out
    last = stdout.rstrip("\n").split("\n")[-1]
    assert len(last) < 3072, len(last)
    h = json.loads(stdout[-4096:].rstrip("\n").split("\n")[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
                "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert key in h, key
    assert h["value"] == out["value"] and h["roofline"]["frac"] == out["roofline"]["frac"]
    assert h["e2e"]["h2d_bytes_per_step"] > 0 and h["cpu_baseline"]["kind"] == "oracle"
    assert json.load(open(detail))["ksweep"] == out["ksweep"]
