"""Parity of the device multigrid-preconditioned CG (Sec. 4, Appendix A: CG with a multigrid
preconditioner, its level, restriction and prolongation SpMMs) against the oracle (GPU).

Bars: the hierarchy (level shapes, nonzeros) equal to the oracle's; one V-cycle on every level
within 1e-9 (FP64 cycle; the oracle's coarsest solve is CG to 1e-13, the device's a dense
inverse) or 1e-4 (FP32 cycle) relative to the oracle's, both with their means removed (the
constants are the null space: the cycle's output is defined up to them); the FP64 solve with
the oracle's beta and a true-residual check every iteration in the oracle's iteration count
(+-1) and within 1e-8 of its solution; every solve to a true relative residual <= 1e-10,
recomputed here by the oracle's operator.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fvm, mg
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


def _grids():
    return {
        "channel-32x16x24": W.channel_grid(32, 16, 24),
        "periodic-16": W.unit_periodic_grid(16),
        "rbc-16x16x32": W.Grid((W.uniform_axis(16), W.uniform_axis(16), W.tanh_axis(32, 1.4, 0.0, 1.0))),
    }


def _mg(rb, g, k_max, **kw):
    nodes, per = rb.grid_nodes(g)
    return rb.Multigrid(nodes, per, k_max=k_max, **kw)


def _zm(a):
    return a - a.mean(axis=0, keepdims=True)


@pytest.mark.parametrize("name", ["channel-32x16x24", "periodic-16", "rbc-16x16x32"])
def test_hierarchy_matches_oracle(rb, name):
    g = _grids()[name]
    lv = mg.hierarchy(g)
    m = _mg(rb, g, 1)
    assert m.levels == len(lv)
    axis = mg.line_axis(g)
    assert m.line_axis == (-1 if axis is None else axis)  # the line smoother's axis, as the oracle picks it
    assert _mg(rb, g, 1, smoother="jacobi").line_axis == -1
    inf = m.info()
    for l, L in enumerate(lv):
        assert inf.nnz_A[l] == L.A.nnz
        assert inf.nnz_P[l] == (0 if L.P is None else L.P.nnz)
        assert m.shapes[l][0] * m.shapes[l][1] * m.shapes[l][2] == L.A.shape[0]


@pytest.mark.parametrize("name", ["channel-32x16x24", "periodic-16", "rbc-16x16x32"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3])
@pytest.mark.parametrize("smoother", ["jacobi", "line"])
def test_vcycle_per_level_matches_oracle(rb, name, dtype, k, smoother):
    g = _grids()[name]
    lv = mg.hierarchy(g, smoother=smoother)
    m = _mg(rb, g, k, smoother=smoother)
    tol = 1e-9 if dtype == "f64" else 1e-4
    for l in range(len(lv)):
        n = lv[l].A.shape[0]
        R = _zm(W.normal((n, k), 700 + 10 * l + k))
        Z = m.vcycle(to_dev(R), level=l, dtype=dtype).cpu().numpy()
        for j in range(k):
            zr = mg.vcycle(lv, R[:, j], level=l)
            err = np.linalg.norm(_zm(Z[:, j:j + 1])[:, 0] - (zr - zr.mean())) / np.linalg.norm(zr - zr.mean())
            assert err <= tol, (l, j, err)
    R0 = to_dev(_zm(W.normal((lv[0].A.shape[0], k), 799)))  # a level-0 block
    Z1 = m.vcycle(R0, level=0, dtype=dtype).cpu().numpy()
    Z2 = m.vcycle(R0, level=0, dtype=dtype).cpu().numpy()
    assert np.array_equal(Z1, Z2)  # a second call on the same hierarchy gives the same bits


@pytest.mark.parametrize("shape", [(8, 160, 8), (12, 40, 12)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3])
def test_line_smoother_line_lengths(rb, shape, dtype, k):
    """Wall-normal lines of 160 cells (longer than the 128 whose segments stay in registers:
    the kernel that parks them in the output block) and of 40 and 20 cells (segments of 5, and
    of 2 or 3 cells: unequal splits): one V-cycle per level against the oracle's."""
    g = W.channel_grid(*shape)
    lv = mg.hierarchy(g, smoother="line")
    m = _mg(rb, g, k, smoother="line")
    assert m.line_axis == 1 and m.levels == len(lv) == 2
    tol = 1e-9 if dtype == "f64" else 1e-4
    for l in range(len(lv)):
        n = lv[l].A.shape[0]
        R = _zm(W.normal((n, k), 900 + 10 * l + k))
        Z = m.vcycle(to_dev(R), level=l, dtype=dtype).cpu().numpy()
        for j in range(k):
            zr = mg.vcycle(lv, R[:, j], level=l)
            err = np.linalg.norm(_zm(Z[:, j:j + 1])[:, 0] - (zr - zr.mean())) / np.linalg.norm(zr - zr.mean())
            assert err <= tol, (l, j, err)


def _true_rel_res(A, B, X):
    Rt = B - A @ X
    return np.linalg.norm(_zm(Rt), axis=0) / np.linalg.norm(_zm(B), axis=0)


@pytest.mark.parametrize("name", ["channel-32x16x24", "periodic-16", "rbc-16x16x32"])
@pytest.mark.parametrize("smoother", ["jacobi", "line"])
def test_fp64_solve_follows_the_oracle(rb, name, smoother):
    """FP64 cycle, the oracle's beta, the true residual checked every iteration: the oracle's
    iteration count and solution."""
    g = _grids()[name]
    lv = mg.hierarchy(g, smoother=smoother)
    A = lv[0].A
    k = 3
    B = _zm(W.normal((g.n_cells, k), 720))
    m = _mg(rb, g, k, flexible=False, smoother=smoother)
    X = torch.zeros((g.n_cells, k), dtype=torch.float64, device="cuda")
    res = m.solve(to_dev(B), X, rb.mg_params(mixed=False, check_every=1))
    assert res.status == rb.RB_OK, res
    Xh = X.cpu().numpy()
    assert np.all(_true_rel_res(A, B, Xh) <= 1e-10)
    for j in range(k):
        xr, it = mg.mg_pcg(lv, B[:, j])
        assert abs(res.iters[j] - it) <= 1, (j, res.iters[j], it)
        assert np.linalg.norm(Xh[:, j] - xr) <= 1e-8 * np.linalg.norm(xr)
        assert abs(Xh[:, j].mean()) <= 1e-12 * np.abs(xr).max()  # the zero-mean solution


@pytest.mark.parametrize("name", ["channel-32x16x24", "periodic-16", "rbc-16x16x32"])
@pytest.mark.parametrize("k", [1, 3, 8])
@pytest.mark.parametrize("smoother", ["jacobi", "line"])
def test_mixed_solve_reaches_the_oracle_solution(rb, name, k, smoother):
    """FP32 cycle and CG inside FP64 refinement, flexible beta: the FP64 true residual reaches
    1e-10 and the solution is the oracle's within its conditioning."""
    g = _grids()[name]
    lv = mg.hierarchy(g, smoother=smoother)
    A = lv[0].A
    B = _zm(W.normal((g.n_cells, k), 730 + k))
    m = _mg(rb, g, k, smoother=smoother)
    X = torch.zeros((g.n_cells, k), dtype=torch.float64, device="cuda")
    res = m.solve(to_dev(B), X, rb.mg_params(mixed=True))
    assert res.status == rb.RB_OK, res
    Xh = X.cpu().numpy()
    assert np.all(_true_rel_res(A, B, Xh) <= 1e-10), _true_rel_res(A, B, Xh)
    assert np.all(np.array(res.true_rel_res) <= 1e-10)
    for j in range(min(k, 3)):
        xr, it = mg.mg_pcg(lv, B[:, j])
        assert np.linalg.norm(Xh[:, j] - xr) <= 1e-7 * np.linalg.norm(xr)
        assert res.iters[j] <= 3 * it, (res.iters[j], it)
    if smoother == "line" and m.line_axis >= 0:  # the stretched grids: fewer iterations than point smoothing
        X[:] = 0.0
        rp = _mg(rb, g, k, smoother="jacobi").solve(to_dev(B), X, rb.mg_params(mixed=True))
        assert max(res.iters) < max(rp.iters), (res.iters, rp.iters)


def test_solve_from_a_guess_and_repeat(rb):
    """A nonzero initial guess, and the same solve twice on one hierarchy (the recorded CUDA
    graphs replayed): identical results."""
    g = _grids()["channel-32x16x24"]
    A = (-fvm.laplacian(g)).tocsr()
    k = 3
    B = _zm(W.normal((g.n_cells, k), 740))
    X0 = W.normal((g.n_cells, k), 741)
    m = _mg(rb, g, k)
    outs = []
    for rep in range(2):
        X = to_dev(X0)
        res = m.solve(to_dev(B), X, rb.mg_params(mixed=True))
        assert res.status == rb.RB_OK
        outs.append(X.cpu().numpy())
        assert np.all(_true_rel_res(A, B, outs[-1]) <= 1e-10)
    assert np.array_equal(outs[0], outs[1])
    X = torch.zeros((g.n_cells, k), dtype=torch.float64, device="cuda")
    m.solve(to_dev(B), X, rb.mg_params(mixed=True))
    assert np.linalg.norm(X.cpu().numpy() - outs[0]) <= 1e-8 * np.linalg.norm(outs[0])


def test_strided_blocks_and_fewer_columns(rb):
    """B and X as column slices of wider blocks (ld > k), k below the hierarchy's k_max."""
    g = W.unit_periodic_grid(16)
    A = (-fvm.laplacian(g)).tocsr()
    Bw = W.normal((g.n_cells, 5), 750)
    Bw[:, 1:3] = _zm(Bw[:, 1:3])
    Bd = to_dev(Bw)
    Xd = torch.full((g.n_cells, 6), 7.0, dtype=torch.float64, device="cuda")
    m = _mg(rb, g, 4)
    for mixed in (False, True):
        Xd[:, 2:4] = 0.0
        res = m.solve(Bd[:, 1:3], Xd[:, 2:4], rb.mg_params(mixed=mixed))
        assert res.status == rb.RB_OK
        Xh = Xd.cpu().numpy()
        assert np.all(_true_rel_res(A, Bw[:, 1:3], Xh[:, 2:4]) <= 1e-10)
        assert np.all(Xh[:, [0, 1, 4, 5]] == 7.0)  # the other columns untouched


def test_one_level_and_too_coarse_grids(rb):
    """An odd grid does not coarsen: the cycle is the exact coarse solve (the oracle's CG), a
    solve is refused; a grid whose coarsest level keeps too many cells is refused."""
    g = W.unit_periodic_grid(15)
    lv = mg.hierarchy(g)
    assert len(lv) == 1
    m = _mg(rb, g, 1)
    R = _zm(W.normal((g.n_cells, 1), 760))
    Z = m.vcycle(to_dev(R)).cpu().numpy()[:, 0]
    zr = mg.vcycle(lv, R[:, 0])
    assert np.linalg.norm((Z - Z.mean()) - zr) <= 1e-9 * np.linalg.norm(zr)
    X = torch.zeros((g.n_cells, 1), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbError) as e:
        m.solve(to_dev(R), X)
    assert e.value.status == rb.RB_EINVAL
    with pytest.raises(rb.RbError) as e:
        _mg(rb, W.unit_periodic_grid(17), 1)
    assert e.value.status == rb.RB_EINVAL and "coarsest" in str(e.value)


def test_channel_full_size_k3(rb):
    """The bench's case: the 192 x 128 x 96 channel, k = 3 compatible right-hand sides b = -M u,
    both precisions; the true residual recomputed by the oracle's Laplacian."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    L = fvm.laplacian_direct(g)
    M = fvm.divergence(g)
    k = 3
    U = W.face_field(M.shape[1], k, 2002)
    B = -(M @ U)
    m = _mg(rb, g, k)
    assert m.levels == 5 and m.line_axis == 1
    for mixed in (True, False):
        X = torch.zeros((g.n_cells, k), dtype=torch.float64, device="cuda")
        res = m.solve(to_dev(B), X, rb.mg_params(mixed=mixed))
        assert res.status == rb.RB_OK, res
        Xh = X.cpu().numpy()
        assert np.all(_true_rel_res(-L, B, Xh) <= 1e-10), (mixed, _true_rel_res(-L, B, Xh))
        assert max(res.iters) <= 20, res.iters
