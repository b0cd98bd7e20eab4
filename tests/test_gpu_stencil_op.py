"""Parity of the matrix-free FVM Laplacian (rb_fvm_stencil_create, format RB_STENCIL: the
entries formed from per-axis tables) against the oracle's assembled Laplacian (GPU).

Bar: componentwise as for every SpMM, |Y - Y_ref| <= tol (|A| |X|) |c| with tol 1e-12 (FP64)
and 1e-5 (FP32; the oracle fed the RNE-rounded entries and X: the device forms each FP32
entry as a product of FP32-rounded tables, a few ulp away)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fvm, spmm
from tests.conftest import componentwise_ok, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _grids():
    return {
        "channel-24x20x16": W.channel_grid(24, 20, 16),
        "periodic-9^3": W.unit_periodic_grid(9),
        "walled-8x6x10": W.Grid((W.tanh_axis(8, 1.2, 0.0, 2.0), W.tanh_axis(6, 1.5, -1.0, 1.0),
                                 W.tanh_axis(10, 0.8, 0.0, 3.0))),
        "rbc-12x7x9": W.Grid((W.uniform_axis(12), W.uniform_axis(7, 2.0), W.tanh_axis(9, 1.4, 0.0, 1.0))),
        "thin-3x2x4": W.Grid((W.uniform_axis(3), W.tanh_axis(2, 1.1, 0.0, 1.0), W.uniform_axis(4))),
    }


@pytest.mark.parametrize("name", list(_grids()))
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 8, 32, 64])
def test_stencil_spmm_matches_oracle(rb, name, dtype, k):
    g = _grids()[name]
    L = fvm.laplacian(g)
    scale = -1.0 if k % 2 else 2.5
    A = (scale * L).tocsr()
    nodes, per = rb.grid_nodes(g)
    op = rb.Operator.stencil(nodes, per, scale=scale, dtype=dtype, k_max=k)
    assert op.nnz == A.nnz and op.info().format == rb.RB_STENCIL
    npdt = np.float64 if dtype == "f64" else np.float32
    X = W.normal((g.n_cells, k), 1000 + k).astype(npdt)
    c = W.normal(k, 1100 + k)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Y = torch.full((g.n_cells, k), float("nan"), dtype=tdt, device="cuda")
    op.spmm(to_dev(X), Y, c=to_dev(c) if k % 3 == 0 else None)
    Aref = A if dtype == "f64" else spmm.round_f32(A)
    cref = None if k % 3 else (c if dtype == "f64" else c.astype(np.float32).astype(np.float64))
    Xref = X.astype(np.float64)
    ok, worst = componentwise_ok(Y.cpu().numpy(), spmm.spmm(Aref, Xref, cref), spmm.abs_bound(Aref, Xref, cref),
                                 TOL[dtype])
    assert ok, worst


def test_stencil_channel_full_size(rb):
    """The 192 x 128 x 96 channel, k = 3, FP64 and FP32, tuned; and the Jacobi diagonal the
    operator carries (1 / a_ii) against the assembled one."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    L = fvm.laplacian_direct(g)
    nodes, per = rb.grid_nodes(g)
    X = W.normal((g.n_cells, 3), 1200)
    for dtype in ("f64", "f32"):
        op = rb.Operator.stencil(nodes, per, scale=1.0, dtype=dtype, k_max=3)
        npdt = np.float64 if dtype == "f64" else np.float32
        Xd = to_dev(X.astype(npdt))
        Y = torch.empty_like(Xd)
        op.tune(Xd, Y)
        op.spmm(Xd, Y)
        Aref = L if dtype == "f64" else spmm.round_f32(L)
        Xref = X.astype(npdt).astype(np.float64)
        ok, worst = componentwise_ok(Y.cpu().numpy(), spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref), TOL[dtype])
        assert ok, (dtype, worst)


def test_stencil_refuses_bad_schedules(rb):
    g = W.unit_periodic_grid(8)
    nodes, per = rb.grid_nodes(g)
    op = rb.Operator.stencil(nodes, per, k_max=4)
    with pytest.raises(rb.RbError):
        op.set_schedule(4, 2, 2, 0, -1)  # lanes per row: CSR only
    with pytest.raises(rb.RbError):
        op.set_schedule(4, 2, 1, 2, -1)  # TMA staging: CSR only
