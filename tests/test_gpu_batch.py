"""Batched uneven Poisson systems in one persistent launch under a CUDA graph, and the
persistent single-system refinement (GPU).  Bar as for the single solves: true relative
residual <= 1e-10 per column, recomputed on the CPU, and the oracle's solution within the
error that residual allows; plus the failure path of the bounded grid barrier."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cg as ocg
from oracle import fvm
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


def _system(g, k, seed):
    A = (-fvm.laplacian(g)).tocsr()
    B = W.zero_mean(W.normal((A.shape[0], k), seed))
    return A, B


def _true_res(A, B, X):
    R = B - A @ X
    R -= R.mean(axis=0, keepdims=True)
    return np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)


SYSTEMS = [(W.unit_periodic_grid(16), 2, 11), (W.channel_grid(20, 16, 12, gamma=1.5), 3, 12),
           (W.unit_periodic_grid(8), 1, 13), (W.channel_grid(12, 9, 7, gamma=1.4), 4, 14)]


def _make(rb, systems, mixed=2, inner="csr"):
    ops, ops32, Bs, As = [], [], [], []
    for g, k, seed in systems:
        A, B = _system(g, k, seed)
        As.append(A)
        Bs.append(B)
        ops.append(rb.Operator.from_scipy(A, k_max=k))
        if inner == "csr":
            ops32.append(rb.Operator.from_scipy(A, dtype="f32", k_max=k))
        else:  # the matrix-free FP32 Laplacian of the same grid
            nodes, per = rb.grid_nodes(g)
            ops32.append(rb.Operator.stencil(nodes, per, scale=-1.0, dtype="f32", k_max=k))
    prm = rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True, max_sweeps=16)
    batch = rb.Batch(ops, ops32, [s[1] for s in systems], prm)
    return batch, As, Bs


@pytest.mark.parametrize("inner", ["csr", "matrix_free"])
@pytest.mark.parametrize("mixed", [1, 2])
def test_batch_matches_oracle_and_replays(rb, mixed, inner):
    batch, As, Bs = _make(rb, SYSTEMS, mixed, inner)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    res = batch.solve(Bd, Xd)
    for (A, B, X, r) in zip(As, Bs, Xd, res):
        assert r.status == rb.RB_OK, r
        Xh = X.cpu().numpy()
        assert np.all(_true_res(A, B, Xh) <= 1e-10)
        Xr, _ = ocg.pcg_columns(A, B, rtol=1e-10, project_mean=True)
        assert np.all(np.linalg.norm(Xh - Xr, axis=0) <= 1e-6 * np.linalg.norm(Xr, axis=0))
    first = [x.clone() for x in Xd]
    # replay of the recorded graph from the same initial guess gives the same answer, bit for bit
    for x in Xd:
        x.zero_()
    res2 = batch.solve(Bd, Xd)
    assert all(r.status == rb.RB_OK for r in res2)
    for a, b in zip(first, Xd):
        assert torch.equal(a, b)
    # new right-hand-side buffers: the graph is recorded again
    Bd2 = [b.clone() * 2.0 for b in Bd]
    Xd2 = [torch.zeros_like(b) for b in Bd2]
    res3 = batch.solve(Bd2, Xd2)
    assert all(r.status == rb.RB_OK for r in res3)
    for a, b in zip(first, Xd2):
        assert torch.allclose(2.0 * a, b, rtol=1e-7, atol=1e-12 * float(a.abs().max()))


def test_batch_equals_single_solves(rb):
    """Each system of the batch gets the answer of the single-system refinement (same algorithm)."""
    batch, As, Bs = _make(rb, SYSTEMS[:3], 2)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    res = batch.solve(Bd, Xd)
    for (g, k, seed), A, B, X, r in zip(SYSTEMS[:3], As, Bs, Xd, res):
        op = rb.Operator.from_scipy(A, k_max=k)
        op32 = rb.Operator.from_scipy(A, dtype="f32", k_max=k)
        x1 = torch.zeros_like(X)
        r1 = rb.cg_solve(op, to_dev(B), x1, A_inner=op32,
                         params=rb.cg_params(rtol=1e-10, mixed=2, project_mean=True, max_sweeps=16))
        assert r1.status == rb.RB_OK
        assert torch.allclose(X, x1, rtol=1e-6, atol=1e-9 * float(x1.abs().max()))
        assert all(abs(a - b) <= max(3, b // 20) for a, b in zip(r.iters, r1.iters)), (r.iters, r1.iters)


def test_batch_bench_configuration(rb):
    """The bench's batch at full size in its launch configuration (64^3 k = 8, 128^3 k = 1,
    three 96 x 64 x 48 channels k = 3, same seeds, one persistent launch per sweep under the
    recorded graph): every column reaches the true 1e-10 residual, recomputed on the CPU with
    the oracle's operators (a property that holds at any size)."""
    systems, As, Bs = [], [], []
    for i, (g, k) in enumerate(zip(W.batch_grids(), W.BATCH_K_DEFAULT)):
        A = (-fvm.laplacian(g)).tocsr()
        B = W.zero_mean(W.normal((g.n_cells, k), W.seed_for(4, k, salt=i)))
        As.append(A)
        Bs.append(B)
        systems.append((rb.Operator.from_scipy(A, k_max=k), rb.Operator.from_scipy(A, dtype="f32", k_max=k), k))
    prm = rb.cg_params(rtol=1e-10, mixed=2, project_mean=True, max_sweeps=16)
    batch = rb.Batch([s[0] for s in systems], [s[1] for s in systems], [s[2] for s in systems], prm)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    res = batch.solve(Bd, Xd)
    for A, B, X, r in zip(As, Bs, Xd, res):
        assert r.status == rb.RB_OK, r
        tr = _true_res(A, B, X.cpu().numpy())
        assert np.all(tr <= 1e-10), tr
        assert np.allclose(r.true_rel_res, tr, rtol=1e-3, atol=1e-14)


def test_batch_at_the_column_limit(rb):
    """64 columns in total (the limit) over systems with 32, 24 and 8 columns: the persistent
    kernel's partial slots for every batch column and its wide-block reductions."""
    systems = [(W.unit_periodic_grid(10), 32, 21), (W.channel_grid(12, 10, 8, gamma=1.5), 24, 22),
               (W.unit_periodic_grid(8), 8, 23)]
    batch, As, Bs = _make(rb, systems, 2)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    res = batch.solve(Bd, Xd)
    for A, B, X, r in zip(As, Bs, Xd, res):
        assert r.status == rb.RB_OK, r
        Xh = X.cpu().numpy()
        assert np.all(_true_res(A, B, Xh) <= 1e-10)
        Xr, _ = ocg.pcg_columns(A, B, rtol=1e-10, project_mean=True)
        assert np.all(np.linalg.norm(Xh - Xr, axis=0) <= 1e-6 * np.linalg.norm(Xr, axis=0))


@pytest.mark.parametrize("k", [1, 3, 8, 16])
def test_persistent_single_system(rb, k):
    g = W.channel_grid(40, 32, 24, gamma=1.5)
    A, B = _system(g, k, 40 + k)
    op = rb.Operator.from_scipy(A, k_max=k)
    op32 = rb.Operator.from_scipy(A, dtype="f32", k_max=k)
    X = torch.zeros((A.shape[0], k), dtype=torch.float64, device="cuda")
    r = rb.cg_solve(op, to_dev(B), X, A_inner=op32,
                    params=rb.cg_params(rtol=1e-10, mixed=2, project_mean=True, persistent=True))
    assert r.status == rb.RB_OK, r
    assert np.all(_true_res(A, B, X.cpu().numpy()) <= 1e-10)
    X2 = torch.zeros_like(X)
    r2 = rb.cg_solve(op, to_dev(B), X2, A_inner=op32, params=rb.cg_params(rtol=1e-10, mixed=2, project_mean=True))
    assert all(abs(a - b) <= max(3, b // 20) for a, b in zip(r.iters, r2.iters)), (r.iters, r2.iters)


def test_batch_barrier_timeout_is_reported(rb):
    """Failure detection without a GPU fault: the barrier waits for one block more than the
    launch has, gives up after 50 ms, the solve returns RB_ETIMEOUT, and the next solve works."""
    batch, As, Bs = _make(rb, SYSTEMS[:2], 2)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    batch.set_barrier(timeout_ms=50.0, extra_arrivals=1)
    res = batch.solve(Bd, Xd)
    assert res[0].status == rb.RB_ETIMEOUT
    batch.set_barrier(timeout_ms=2000.0, extra_arrivals=0)
    for x in Xd:
        x.zero_()
    res = batch.solve(Bd, Xd)
    assert all(r.status == rb.RB_OK for r in res)
    for A, B, X in zip(As, Bs, Xd):
        assert np.all(_true_res(A, B, X.cpu().numpy()) <= 1e-10)


def test_batch_tune_keeps_parity(rb):
    batch, As, Bs = _make(rb, SYSTEMS[:2], 2)
    Bd = [to_dev(B) for B in Bs]
    Xd = [torch.zeros_like(b) for b in Bd]
    ms = batch.tune(Bd, Xd)
    assert ms > 0
    for x in Xd:
        x.zero_()
    res = batch.solve(Bd, Xd)
    assert all(r.status == rb.RB_OK for r in res)
    for A, B, X in zip(As, Bs, Xd):
        assert np.all(_true_res(A, B, X.cpu().numpy()) <= 1e-10)
