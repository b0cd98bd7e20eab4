"""Pins of the oracle's Poisson solvers and unstructured operator (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import cg, fvm, mesh, spmm


def _fft_periodic_solve(N, b):
    """Exact zero-mean solution of -L p = b on the uniform periodic grid via Fourier modes (P1)."""
    h = 1.0 / N
    bb = b.reshape(N, N, N)  # (k, j, i)
    kk = np.arange(N)
    s = np.sin(np.pi * kk / N) ** 2
    lam = -4 * h * (s[:, None, None] + s[None, :, None] + s[None, None, :])
    bh = np.fft.fftn(bb)
    ph = np.zeros_like(bh)
    nz = lam != 0
    ph[nz] = bh[nz] / (-lam[nz])
    return np.real(np.fft.ifftn(ph)).ravel()


def test_cg_matches_dense_direct_8cube_periodic():
    """P5: Jacobi-CG on 8^3 periodic equals the dense Cholesky solve of (-L + 1 1^T) x = b."""
    g = W.unit_periodic_grid(8)
    A = (-fvm.laplacian(g)).tocsr()
    b = W.zero_mean(W.normal((A.shape[0], 2), 7))
    X, infos = cg.pcg_columns(A, b, rtol=1e-10, project_mean=True)
    Ad = A.toarray()
    kappa = np.linalg.cond(Ad + np.ones_like(Ad))
    for j in range(2):
        xd = cg.dense_pseudo_solve(Ad, b[:, j])
        assert infos[j].status == cg.OK and infos[j].rel_res <= 1e-10
        assert np.linalg.norm(X[:, j] - xd) <= kappa * 1e-10 * np.linalg.norm(xd)
        assert abs(X[:, j].mean()) <= 1e-14 * np.abs(X[:, j]).max()


def test_cg_matches_dense_direct_8cube_channel():
    """P5 on a stretched wall-bounded grid, where the Jacobi diagonal varies."""
    g = W.channel_grid(8, 8, 8, gamma=1.5)
    A = (-fvm.laplacian(g)).tocsr()
    b = W.zero_mean(W.normal((A.shape[0], 1), 8))[:, 0]
    x, info = cg.pcg(A, b, rtol=1e-10, project_mean=True)
    Ad = A.toarray()
    xd = cg.dense_pseudo_solve(Ad, b)
    kappa = np.linalg.cond(Ad + np.ones_like(Ad))
    assert info.status == cg.OK
    assert np.linalg.norm(x - xd) <= kappa * 1e-10 * np.linalg.norm(xd)


def test_cg_matches_fourier_solution_16cube():
    """P1 used as a solver pin: the periodic solution p^ = b^/lambda (kappa != 0)."""
    N = 16
    A = (-fvm.laplacian(W.unit_periodic_grid(N))).tocsr()
    b = W.zero_mean(W.normal((N**3, 1), 9))[:, 0]
    x, info = cg.pcg(A, b, rtol=1e-12, project_mean=True)
    xf = _fft_periodic_solve(N, b)
    assert np.linalg.norm(x - xf) <= 1e-9 * np.linalg.norm(xf)


def test_jacobi_pcg_equals_plain_cg_when_diagonal_constant():
    """With a constant diagonal the Jacobi preconditioner is a scalar: same iterates, same iteration count."""
    A = (-fvm.laplacian(W.unit_periodic_grid(8))).tocsr()
    b = W.zero_mean(W.normal((512, 1), 10))[:, 0]
    x1, i1 = cg.pcg(A, b, rtol=1e-10, jacobi=True, project_mean=True)
    x2, i2 = cg.pcg(A, b, rtol=1e-10, jacobi=False, project_mean=True)
    assert i1.iters == i2.iters
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x2)


def test_projection_makes_field_divergence_free():
    """The pressure solve of the projection method: p from L p = M u* gives M(u* - G p) = 0."""
    g = W.channel_grid(8, 6, 5)
    M, G, L = fvm.divergence(g), fvm.gradient(g), fvm.laplacian(g)
    u = W.face_field(M.shape[1], 1, 11)[:, 0]
    b = M @ u
    assert abs(b.sum()) <= 1e-12 * np.abs(b).sum()  # compatible right-hand side
    p, info = cg.pcg((-L).tocsr(), -b, rtol=1e-12, project_mean=True)
    assert info.status == cg.OK
    assert np.linalg.norm(M @ (u - G @ p)) <= 1e-10 * np.linalg.norm(b)


def test_ir_matches_fp64_solution():
    """P8: FP32-inner refinement reaches the FP64 solution to kappa * 1e-10."""
    g = W.channel_grid(10, 8, 6)
    A = (-fvm.laplacian(g)).tocsr()
    b = W.zero_mean(W.normal((A.shape[0], 1), 12))[:, 0]
    x64, _ = cg.pcg(A, b, rtol=1e-10, project_mean=True)
    xir, info, sweeps = cg.ir_pcg(A, b, rtol=1e-10, inner_rtol=1e-4, project_mean=True)
    assert info.status == cg.OK and info.rel_res <= 1e-10
    assert 2 <= sweeps <= 6
    Ad = A.toarray()
    kappa = np.linalg.cond(Ad + np.ones_like(Ad))
    assert np.linalg.norm(xir - x64) <= kappa * 2e-10 * np.linalg.norm(x64)


def test_reliable_ir_matches_fp64_and_keeps_iterations():
    """P8 for the reliable-update refinement: same solution as FP64 CG within kappa * 1e-10,
    and keeping the direction across sweeps costs few iterations over FP64 CG, unlike
    restarting it (the restarted refinement needs more than 1.4 times as many here)."""
    g = W.channel_grid(16, 12, 10)
    A = (-fvm.laplacian(g)).tocsr()
    b = W.zero_mean(W.normal((A.shape[0], 1), 12))[:, 0]
    x64, i64 = cg.pcg(A, b, rtol=1e-10, project_mean=True)
    xr, ir, sweeps = cg.ir_reliable_pcg(A, b, rtol=1e-10, inner_rtol=1e-2, project_mean=True)
    _, irs, _ = cg.ir_pcg(A, b, rtol=1e-10, inner_rtol=1e-2, project_mean=True)
    assert ir.status == cg.OK and ir.rel_res <= 1e-10
    Ad = A.toarray()
    kappa = np.linalg.cond(Ad + np.ones_like(Ad))
    assert np.linalg.norm(xr - x64) <= kappa * 2e-10 * np.linalg.norm(x64)
    assert ir.iters <= 1.2 * i64.iters < irs.iters / 1.2
    assert 3 <= sweeps <= 8


def test_reliable_ir_block_columns_in_lockstep():
    """The k-column reliable refinement: every column reaches the FP64 solution within
    kappa * 1e-10; columns that are not done share each sweep's iterations (a column that met
    its target keeps iterating), so their counts agree until they finish; k = 1 is the
    single-column solve; the total stays near FP64 CG's."""
    g = W.channel_grid(16, 12, 10)
    A = (-fvm.laplacian(g)).tocsr()
    B = W.zero_mean(W.normal((A.shape[0], 3), 13))
    B[:, 2] *= 1e-3  # a different scale: the same relative tolerance
    X, infos, sweeps = cg.ir_reliable_pcg_block(A, B, rtol=1e-10, inner_rtol=5e-2, project_mean=True)
    Ad = A.toarray()
    kappa = np.linalg.cond(Ad + np.ones_like(Ad))
    for j in range(3):
        x64, i64 = cg.pcg(A, B[:, j], rtol=1e-10, project_mean=True)
        assert infos[j].status == cg.OK and infos[j].rel_res <= 1e-10
        assert np.linalg.norm(X[:, j] - x64) <= kappa * 2e-10 * np.linalg.norm(x64)
        assert infos[j].iters <= 1.3 * i64.iters
    assert max(i.iters for i in infos) - min(i.iters for i in infos) <= max(i.iters for i in infos) // 4
    x1, i1, s1 = cg.ir_reliable_pcg(A, B[:, 0], rtol=1e-10, inner_rtol=5e-2, project_mean=True)
    X1, I1, S1 = cg.ir_reliable_pcg_block(A, B[:, :1], rtol=1e-10, inner_rtol=5e-2, project_mean=True)
    assert np.array_equal(x1, X1[:, 0]) and i1.iters == I1[0].iters and s1 == S1


def test_batch_equals_individual_solves():
    systems = []
    for s, k in ((W.unit_periodic_grid(6), 2), (W.channel_grid(6, 5, 4), 1)):
        A = (-fvm.laplacian(s)).tocsr()
        systems.append((A, W.zero_mean(W.normal((A.shape[0], k), 13 + k))))
    out = cg.batch_solve(systems, rtol=1e-10, project_mean=True)
    for (A, B), (X, infos) in zip(systems, out):
        for j in range(B.shape[1]):
            x, _ = cg.pcg(A, B[:, j], rtol=1e-10, project_mean=True)
            assert np.array_equal(x, X[:, j])


def test_breakdown_and_noconv_status():
    """An indefinite matrix breaks CG down (p.q <= 0); a tiny iteration cap is reported."""
    A = sp.diags([1.0, -1.0, 2.0, 3.0]).tocsr()
    _, info = cg.pcg(A, np.array([1.0, 1.0, 1.0, 1.0]), jacobi=False)
    assert info.status == cg.BREAKDOWN
    A = (-fvm.laplacian(W.unit_periodic_grid(6))).tocsr()
    b = W.zero_mean(W.normal((216, 1), 3))[:, 0]
    _, info = cg.pcg(A, b, max_iter=3, project_mean=True)
    assert info.status == cg.NOCONV and info.iters == 3


# ---------------------------------------------------------------------- unstructured operator


def test_cot_laplacian_linear_precision():
    """Interior vertices of a Delaunay mesh: L2D (a x + b y + c) = 0 exactly (linear precision)."""
    m = W.random_trimesh(300, 5)
    L, n_clamped = mesh.cot_laplacian(m)
    f = 0.7 * m.points[:, 0] - 1.3 * m.points[:, 1] + 0.25
    r = L @ f
    # boundary vertices: on the convex hull of the point set
    from scipy.spatial import ConvexHull

    hull = set(ConvexHull(m.points).vertices.tolist())
    edges = {}
    for t in m.triangles:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            key = (min(a, b), max(a, b))
            edges[key] = edges.get(key, 0) + 1
    bnd = {v for (a, b), c in edges.items() if c == 1 for v in (a, b)}
    assert hull <= bnd
    interior = np.array([i for i in range(m.points.shape[0]) if i not in bnd])
    assert np.abs(r[interior]).max() <= 1e-12 * np.abs(L).max()


def test_cot_laplacian_on_grid_mesh_is_five_point():
    """A right-triangle grid mesh gives the 5-point stencil: weight 1 on axis edges, 0 on diagonals."""
    m = W.grid_trimesh(5, 4, h=0.5)
    L, n_clamped = mesh.cot_laplacian(m)
    assert n_clamped == 0
    nx = 6
    v = 1 + nx * 2  # an interior vertex (i=1, j=2)
    row = dict(zip(L.indices[L.indptr[v]:L.indptr[v + 1]], L.data[L.indptr[v]:L.indptr[v + 1]]))
    for nb in (v - 1, v + 1, v - nx, v + nx):
        assert row[nb] == pytest.approx(1.0, abs=1e-14)
    assert row[v] == pytest.approx(-4.0, abs=1e-14)
    assert all(abs(row[nb]) < 1e-14 for nb in row if nb not in (v, v - 1, v + 1, v - nx, v + nx))


def test_cot_laplacian_invariants_and_pattern():
    m = W.random_trimesh(200, 6)
    L, _ = mesh.cot_laplacian(m)
    rp, ci = W.mesh_adjacency(m)
    assert np.array_equal(L.indptr, rp) and np.array_equal(L.indices, ci)
    assert abs(L - L.T).max() == 0.0
    assert np.abs(L @ np.ones(L.shape[0])).max() <= 1e-13 * np.abs(L).max()
    a = mesh.dual_areas(m)
    u = m.points[m.triangles[:, 1]] - m.points[m.triangles[:, 0]]
    v = m.points[m.triangles[:, 2]] - m.points[m.triangles[:, 0]]
    tri_area = 0.5 * np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
    assert a.sum() == pytest.approx(tri_area.sum(), rel=1e-13)


@pytest.mark.parametrize("nz", [3, 4, 8])
def test_extruded_operator_kron_equals_cellwise(nz):
    """P4 for the extruded operator: the assembled 3-D operator equals the cell-by-cell sum."""
    m = W.random_trimesh(40, 7)
    L, _ = mesh.cot_laplacian(m)
    a = mesh.dual_areas(m)
    dz = 2.0 / nz
    X = W.normal((L.shape[0], nz), 30 + nz)
    Y = mesh.extruded_apply(L, a, nz, dz, X)
    Yl = mesh.extruded_apply_loops(L, a, nz, dz, X)
    assert np.abs(Y - Yl).max() <= 1e-13 * np.abs(Yl).max()
    # zero row sums and symmetry of the 3-D operator
    L3 = mesh.extruded_operator(L, a, nz, dz)
    assert abs(L3 - L3.T).max() <= 1e-15 * abs(L3).max()
    assert np.abs(L3 @ np.ones(L3.shape[0])).max() <= 1e-13 * abs(L3).max()


def test_extruded_spanwise_fourier_mode():
    """A spanwise Fourier mode constant in the plane: L3D (1 (x) cos(2 pi m z/Nz)) = -4 sin^2(pi m/Nz) a/dz."""
    m = W.random_trimesh(30, 8)
    L, _ = mesh.cot_laplacian(m)
    a = mesh.dual_areas(m)
    nz, dz = 8, 0.25
    z = np.arange(nz)
    for mode in (1, 3):
        X = np.ones((L.shape[0], 1)) * np.cos(2 * np.pi * mode * z / nz)[None, :]
        Y = mesh.extruded_apply(L, a, nz, dz, X)
        expect = -4 * np.sin(np.pi * mode / nz) ** 2 * (a / dz)[:, None] * X
        assert np.abs(Y - expect).max() <= 1e-12 * np.abs(expect).max()


def test_airfoil_mesh_shape():
    """The synthetic airfoil mesh: ~7 nonzeros per row, a hole at the body, seeded."""
    m = W.airfoil_mesh(n_points=4000, seed=1)
    rp, ci = W.mesh_adjacency(m)
    n = m.points.shape[0]
    assert 6.5 <= ci.shape[0] / n <= 7.2
    inside = (m.points[:, 0] > 0.05) & (m.points[:, 0] < 0.95) & (np.abs(m.points[:, 1]) < 0.5 * W.naca0012_half_thickness(m.points[:, 0]))
    assert not inside.any()
    m2 = W.airfoil_mesh(n_points=4000, seed=1)
    assert np.array_equal(m.triangles, m2.triangles)


def _reliable_problem(k, seed):
    g = W.channel_grid(24, 16, 12)
    A = (-fvm.laplacian(g)).tocsr()
    B = W.zero_mean(W.normal((g.n_cells, k), seed))
    return A, B


def test_reliable_updates_keep_krylov_progress():
    """The reason for keeping the search direction across sweeps: with a loose inner target
    (many sweeps) the reliable-update refinement needs about as many inner iterations as plain
    FP64 PCG, while restarting each sweep from scratch needs far more.  A wrong rescaling of
    the kept direction (the s_prev / s factors) or a dropped direction loses this."""
    A, B = _reliable_problem(1, 81)
    b = B[:, 0]
    _, info64 = cg.pcg(A, b, rtol=1e-10, project_mean=True)
    for inner in (0.3, 0.1):
        x, info, sweeps = cg.ir_reliable_pcg(A, b, rtol=1e-10, inner_rtol=inner, project_mean=True)
        _, info_r, sweeps_r = cg.ir_pcg(A, b, rtol=1e-10, inner_rtol=inner, project_mean=True)
        assert info.status == cg.OK and sweeps >= 8
        assert info.iters <= 1.15 * info64.iters, (inner, info.iters, info64.iters)
        assert info_r.iters >= 1.5 * info.iters, (inner, info_r.iters, info.iters)


def test_reliable_block_symmetry_and_degenerate_columns():
    """Equal columns give equal results (the lockstep treats them alike); a zero column is done
    at once with x = 0; every other column reaches the tolerance."""
    A, B = _reliable_problem(3, 82)
    B[:, 1] = B[:, 0]
    B[:, 2] = 0.0
    X, infos, _ = cg.ir_reliable_pcg_block(A, B, rtol=1e-10, inner_rtol=5e-2, project_mean=True)
    assert np.array_equal(X[:, 0], X[:, 1]) and infos[0].iters == infos[1].iters
    assert np.all(X[:, 2] == 0.0) and infos[2].iters == 0
    assert infos[0].status == cg.OK and infos[0].rel_res <= 1e-10
