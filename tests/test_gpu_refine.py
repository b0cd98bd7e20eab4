"""Parity of the device coarse-to-fine maps of inline mesh refinement (Sec. 3.3) against the
oracle, and of the rectangular SpMMs that apply them to k states at once (GPU).

Bar: CSR structure bit-exact; values within 4 ulp (each weight is the same sequence of IEEE
operations on both sides, so they agree in practice); SpMM componentwise as in the SpMM
tests.  The full-size case is the bench's: the 96 x 64 x 48 channel mapped onto
192 x 128 x 96 and back.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import refine, spmm
from tests.conftest import componentwise_ok, to_dev

pytestmark = pytest.mark.gpu

VAL_RTOL = 4 * 2.0 ** -52


def _walled_grid():
    return W.Grid((W.tanh_axis(8, 1.2, 0.0, 2.0), W.tanh_axis(6, 1.5, -1.0, 1.0), W.tanh_axis(10, 0.8, 0.0, 3.0)))


GRIDS = {
    "walled-8x6x10": _walled_grid,
    "periodic-4^3": lambda: W.unit_periodic_grid(4),
    "channel-12x8x6": lambda: W.channel_grid(12, 8, 6),
    "channel-40x22x36": lambda: W.channel_grid(40, 22, 36),
    "rbc-16^3": lambda: W.rbc_grid(16),
    # axis tables above the shared-memory budget: the per-row (direct) variant
    "long-2800x4x6": lambda: W.Grid((W.uniform_axis(2800, 3.0), W.tanh_axis(4, 1.1, 0.0, 1.0), W.uniform_axis(6))),
}


def _device_map(rb, g, kind):
    nodes, per = rb.grid_nodes(g)
    rp, ci, va, nc = rb.refine_assemble(nodes, per, kind)
    torch.cuda.synchronize()
    return rp, ci, va, nc


def _check_csr(rp, ci, va, A):
    assert np.array_equal(rp.cpu().numpy(), A.indptr.astype(np.int32))
    assert np.array_equal(ci.cpu().numpy(), A.indices.astype(np.int32))
    v = va.cpu().numpy()
    assert np.all(np.abs(v - A.data) <= VAL_RTOL * np.abs(A.data))


@pytest.mark.parametrize("name", list(GRIDS))
def test_prolong_transpose_matches_oracle(rb, name):
    """P^T (the multigrid restriction of residuals): the structure of the oracle's P transposed
    bit for bit, and the values the same bits as the device's own P entries."""
    g = GRIDS[name]()
    rp, ci, va, nc = _device_map(rb, g, rb.RB_REFINE_PROLONG_T)
    P = refine.prolongation(g)
    PT = P.T.tocsr()
    PT.sort_indices()
    assert nc == g.n_cells and rp.numel() - 1 == g.n_cells // 8
    _check_csr(rp, ci, va, PT)
    prp, pci, pva, _ = _device_map(rb, g, rb.RB_REFINE_PROLONG)
    import scipy.sparse as sp

    Pd = sp.csr_matrix((pva.cpu().numpy(), pci.cpu().numpy(), prp.cpu().numpy()), shape=P.shape).T.tocsr()
    Pd.sort_indices()
    assert np.array_equal(va.cpu().numpy(), Pd.data)


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("kind", ["prolong", "restrict"])
def test_refine_map_matches_oracle(rb, name, kind):
    g = GRIDS[name]()
    k = rb.RB_REFINE_PROLONG if kind == "prolong" else rb.RB_REFINE_RESTRICT
    rp, ci, va, nc = _device_map(rb, g, k)
    A = refine.prolongation(g) if kind == "prolong" else refine.restriction(g)
    assert nc == A.shape[1]
    _check_csr(rp, ci, va, A)


def test_refine_invalid_arguments(rb):
    for g in (W.channel_grid(12, 8, 7), W.channel_grid(12, 2, 6)):
        nodes, per = rb.grid_nodes(g)
        with pytest.raises(rb.RbError) as e:
            rb.refine_assemble(nodes, per, rb.RB_REFINE_PROLONG)
        assert "EINVAL" in str(e.value)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_refine_spmm(rb, dtype, k):
    """P and R applied to k columns (rectangular SpMMs), tuned, against the oracle."""
    g = W.channel_grid(40, 22, 36)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    tol = 1e-12 if dtype == "f64" else 1e-5
    for kind, A in ((rb.RB_REFINE_PROLONG, refine.prolongation(g)), (rb.RB_REFINE_RESTRICT, refine.restriction(g))):
        rp, ci, va, nc = _device_map(rb, g, kind)
        op = rb.Operator(rp, ci, va, nc, dtype=dtype, k_max=k)
        X = W.normal((A.shape[1], k), 1500 + k + kind)
        Xd = to_dev(X.astype(npdt))
        Yd = torch.full((A.shape[0], k), float("nan"), dtype=tdt, device="cuda")
        op.tune(Xd, Yd)
        op.spmm(Xd, Yd)
        op.check()
        Aref = A if dtype == "f64" else spmm.round_f32(A)
        Xref = X.astype(npdt).astype(np.float64)
        ok, worst = componentwise_ok(Yd.cpu().numpy(), spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref), tol)
        assert ok, (kind, worst)


def test_refine_full_size_channel(rb):
    """The bench's pair: 96 x 64 x 48 -> 192 x 128 x 96.  Both maps entry by entry against
    the oracle; P then R applied to three FP64 states; a trilinear field carried exactly."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    P, R = refine.prolongation(g), refine.restriction(g)
    rpP, ciP, vaP, ncP = _device_map(rb, g, rb.RB_REFINE_PROLONG)
    _check_csr(rpP, ciP, vaP, P)
    rpR, ciR, vaR, ncR = _device_map(rb, g, rb.RB_REFINE_RESTRICT)
    _check_csr(rpR, ciR, vaR, R)
    opP = rb.Operator(rpP, ciP, vaP, ncP, k_max=3)
    opR = rb.Operator(rpR, ciR, vaR, ncR, k_max=3)
    Xc = W.normal((P.shape[1], 3), 1600)
    Yf = opP.spmm(to_dev(Xc))
    ok, worst = componentwise_ok(Yf.cpu().numpy(), spmm.spmm(P, Xc), spmm.abs_bound(P, Xc), 1e-12)
    assert ok, worst
    Zc = opR.spmm(Yf)
    Yf64 = Yf.cpu().numpy()
    ok, worst = componentwise_ok(Zc.cpu().numpy(), spmm.spmm(R, Yf64), spmm.abs_bound(R, Yf64), 1e-12)
    assert ok, worst
    # the y coordinate of the coarse centres, interpolated to the fine centres (walls: extrapolated)
    yc = 0.5 * (g.axes[1].nodes[::2][:-1] + g.axes[1].nodes[::2][1:])
    yf = 0.5 * (g.axes[1].nodes[:-1] + g.axes[1].nodes[1:])
    nxc, nyc, nzc = (s // 2 for s in g.shape)
    fc = np.broadcast_to(yc[None, :, None], (nzc, nyc, nxc)).ravel().copy()
    ff = np.broadcast_to(yf[None, :, None], (g.shape[2], g.shape[1], g.shape[0])).ravel()
    got = opP.spmm(to_dev(fc)).cpu().numpy()[:, 0]
    assert np.max(np.abs(got - ff)) <= 1e-13
