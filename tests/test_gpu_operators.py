"""Parity of the device operator build against the oracle (GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fvm, mesh
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu

GRIDS = [
    W.unit_periodic_grid(3),
    W.unit_periodic_grid(6),
    W.channel_grid(8, 6, 5, gamma=1.5),
    W.rbc_grid(6, gamma=1.4),
    W.Grid((W.uniform_axis(5, 2.0, periodic=False), W.tanh_axis(7, 1.2), W.uniform_axis(4, 3.0)), "walls-xy"),
    W.Grid((W.tanh_axis(2, 1.0), W.tanh_axis(3, 1.1), W.tanh_axis(2, 0.7)), "all-walls-min"),
    W.channel_grid(41, 33, 29, gamma=1.5),  # several blocks and a ragged tail
]


def _check_csr(rp, ci, va, ref: sp.csr_matrix, rel=1e-12):
    rp, ci, va = rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy()
    assert np.array_equal(rp, ref.indptr)
    assert np.array_equal(ci, ref.indices)
    # componentwise: each value against the largest magnitude in its row
    rowmax = np.maximum.reduceat(np.abs(ref.data), ref.indptr[:-1]) if ref.nnz else np.zeros(0)
    scale = np.repeat(rowmax, np.diff(ref.indptr))
    assert np.all(np.abs(va - ref.data) <= rel * scale)


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g.name)
def test_fvm_operators_match_oracle(rb, g):
    nodes, per = rb.grid_nodes(g)
    for kind, ref in ((rb.RB_FVM_LAPLACIAN, fvm.laplacian(g)), (rb.RB_FVM_DIVERGENCE, fvm.divergence(g)),
                      (rb.RB_FVM_GRADIENT, fvm.gradient(g))):
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, kind)
        assert nc == ref.shape[1]
        _check_csr(rp, ci, va, ref)


def test_fvm_scale_gives_poisson_matrix(rb):
    g = W.channel_grid(10, 8, 6)
    nodes, per = rb.grid_nodes(g)
    rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN, scale=-1.0)
    _check_csr(rp, ci, va, (-fvm.laplacian(g)).tocsr())


def test_fvm_channel_full_size(rb):
    """The 192 x 128 x 96 channel Laplacian (n = 2,359,296): full comparison with the oracle."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    nodes, per = rb.grid_nodes(g)
    rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
    ref = fvm.laplacian_direct(g)
    assert ref.nnz == 16_478_208
    _check_csr(rp, ci, va, ref)


@pytest.mark.parametrize("npts,seed", [(60, 1), (500, 2)])
def test_cot_laplacian_matches_oracle(rb, npts, seed):
    m = W.random_trimesh(npts, seed)
    rp, ci = W.mesh_adjacency(m)
    vals, area, status = rb.mesh_cot_laplacian(to_dev(m.points), to_dev(m.triangles), to_dev(rp), to_dev(ci))
    L, n_clamped = mesh.cot_laplacian(m)
    st = status.cpu().numpy()
    assert st[1] == 0
    assert st[0] == n_clamped
    _check_csr(to_dev(rp), to_dev(ci), vals, L)
    a = mesh.dual_areas(m)
    assert np.allclose(area.cpu().numpy(), a, rtol=1e-13, atol=0)


def test_cot_laplacian_airfoil_full_size(rb):
    """The ~150k-vertex synthetic airfoil mesh: full comparison with the oracle."""
    m = W.airfoil_mesh()
    rp, ci = W.mesh_adjacency(m)
    vals, area, status = rb.mesh_cot_laplacian(to_dev(m.points), to_dev(m.triangles), to_dev(rp), to_dev(ci))
    L, n_clamped = mesh.cot_laplacian(m)
    assert status.cpu().numpy()[1] == 0
    assert status.cpu().numpy()[0] == n_clamped
    _check_csr(to_dev(rp), to_dev(ci), vals, L)
    assert 6.5 <= L.nnz / L.shape[0] <= 7.2
