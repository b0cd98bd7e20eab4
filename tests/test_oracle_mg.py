"""Pins of the geometric-multigrid-preconditioned CG oracle (the multigrid hierarchy of Sec. 4
and Appendix A, built geometrically): the V-cycle is a symmetric positive semi-definite
operator (so CG may use it), its iteration count does not grow with the grid while plain
CG's does, and it reaches the plain CG solution."""
import numpy as np

import workloads as W
from oracle import cg as ocg
from oracle import mg


def test_vcycle_is_symmetric_positive():
    g = W.Grid((W.uniform_axis(8, 1.0), W.uniform_axis(8, 2.0), W.uniform_axis(8, 1.5)))
    lv = mg.hierarchy(g)
    assert len(lv) == 2
    n = g.n_cells
    Pi = np.eye(n) - 1.0 / n
    B = np.column_stack([mg.vcycle(lv, Pi[:, i]) for i in range(n)])
    assert np.abs(B - B.T).max() <= 1e-9 * np.abs(B).max()
    w = np.linalg.eigvalsh(0.5 * (B + B.T))
    assert w.min() >= -1e-9 * w.max()
    assert np.sum(w > 1e-9 * w.max()) == n - 1  # only the constants in the null space


def test_iterations_do_not_grow_with_the_grid():
    mg_its, cg_its = [], []
    for n in (8, 16, 32):
        g = W.unit_periodic_grid(n)
        lv = mg.hierarchy(g)
        b = W.zero_mean(W.normal((g.n_cells, 1), 20 + n))[:, 0]
        x, it = mg.mg_pcg(lv, b)
        xr, info = ocg.pcg(lv[0].A, b, rtol=1e-10, project_mean=True)
        assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
        r = b - lv[0].A @ x
        assert np.linalg.norm(r - r.mean()) <= 1e-10 * np.linalg.norm(b)
        mg_its.append(it)
        cg_its.append(info.iters)
    assert max(mg_its) <= 15 and max(mg_its) - min(mg_its) <= 2, mg_its
    assert cg_its[2] >= 3 * cg_its[0], cg_its  # plain CG grows like 1/h


def test_walled_stretched_grid():
    """The channel shape (walls and tanh stretching in y): fewer iterations than plain CG."""
    g = W.channel_grid(32, 16, 24)
    lv = mg.hierarchy(g)
    assert len(lv) == 3
    b = W.zero_mean(W.normal((g.n_cells, 1), 33))[:, 0]
    x, it = mg.mg_pcg(lv, b)
    xr, info = ocg.pcg(lv[0].A, b, rtol=1e-10, project_mean=True)
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
    assert it * 4 <= info.iters, (it, info.iters)


def test_block_cg_terminates_in_ceil_n_over_k():
    """With n distinct eigenvalues and k random right-hand sides the block Krylov space (k new
    directions per iteration) fills after ceil(n / k) iterations: block CG stops there,
    single-column CG after n.  (With eigenvalues of multiplicity >= k the invariant subspace
    holding B has dimension k per eigenvalue and there is no such gain.)"""
    import scipy.sparse as sp

    n = 24
    lam = 1.0 + np.arange(n) ** 1.5
    Q, _ = np.linalg.qr(W.normal((n, n), 40))
    A = sp.csr_matrix(Q @ np.diag(lam) @ Q.T)
    for k in (1, 3, 4, 6):
        B = W.normal((n, k), 41 + k)
        X, it = mg.block_cg(A, B, rtol=1e-9)
        assert it <= -(-n // k), (k, it)
        assert np.allclose(A @ X, B, atol=1e-8 * np.abs(B).max())


def test_block_cg_matches_columnwise_cg_on_poisson():
    """Same solutions as k separate CG solves, in no more iterations (the periodic Laplacian's
    eigenvalues are highly repeated, so there the block brings no finite-termination gain)."""
    g = W.unit_periodic_grid(8)
    A = (-mg.fvm.laplacian(g)).tocsr()
    B = W.zero_mean(W.normal((g.n_cells, 4), 42))
    X, it = mg.block_cg(A, B, rtol=1e-10, project_mean=True)
    Xr, infos = ocg.pcg_columns(A, B, rtol=1e-10, project_mean=True, jacobi=False)
    X = X - X.mean(axis=0, keepdims=True)
    assert np.all(np.linalg.norm(X - Xr, axis=0) <= 1e-8 * np.linalg.norm(Xr, axis=0))
    assert it <= max(i.iters for i in infos)


def test_flexible_beta_equals_standard_with_a_fixed_preconditioner():
    """With the same symmetric V-cycle every iteration, the Polak-Ribiere beta equals the
    Fletcher-Reeves one in exact arithmetic: same iteration count and the same solution."""
    g = W.channel_grid(16, 16, 8)
    lv = mg.hierarchy(g)
    b = W.zero_mean(W.normal((g.n_cells, 1), 44))[:, 0]
    x0, it0 = mg.mg_pcg(lv, b)
    x1, it1 = mg.mg_pcg(lv, b, flexible=True)
    assert abs(it0 - it1) <= 1, (it0, it1)
    assert np.linalg.norm(x1 - x0) <= 1e-9 * np.linalg.norm(x0)


def test_flexible_beta_survives_a_perturbed_preconditioner():
    """A V-cycle whose output is perturbed at the 1e-6 level each iteration (as an FP32 cycle
    is): the flexible form still reaches 1e-10 in about the same number of iterations."""
    g = W.unit_periodic_grid(16)
    lv = mg.hierarchy(g)
    b = W.zero_mean(W.normal((g.n_cells, 1), 45))[:, 0]
    rng = np.random.default_rng(46)
    clean = mg.vcycle

    def noisy(levels, r, level=0, *args, **kw):
        z = clean(levels, r, level, *args, **kw)
        return z * (1.0 + 1e-6 * rng.standard_normal(z.shape)) if level == 0 else z

    mg.vcycle = noisy
    try:
        x, it = mg.mg_pcg(lv, b, flexible=True)
    finally:
        mg.vcycle = clean
    _, it_ref = mg.mg_pcg(lv, b)
    r = b - lv[0].A @ x
    assert np.linalg.norm(r - r.mean()) <= 1e-10 * np.linalg.norm(b)
    assert it <= it_ref + 3, (it, it_ref)


def test_line_axis_and_blocks():
    """The stretched wall-normal axis of a channel is found, an isotropic box has none; the
    line block holds exactly the diagonal and the along-axis couplings of A."""
    g = W.channel_grid(16, 16, 8)
    assert mg.line_axis(g) == 1
    assert mg.line_axis(W.unit_periodic_grid(8)) is None
    # a thin periodic axis does not qualify (its lines would be cyclic)
    assert mg.line_axis(W.Grid((W.uniform_axis(32, 0.1), W.uniform_axis(8), W.uniform_axis(8)))) is None
    A = (-mg.fvm.laplacian(g)).tocsr()
    T = mg.line_block(g, A, 1)
    D = A - T
    assert np.allclose(T.diagonal(), A.diagonal())
    nx = 16
    r, c = D.nonzero()
    assert np.all(np.abs(r - c) != nx)  # no y coupling left outside the blocks ...
    r, c = T.nonzero()
    assert np.all((r == c) | (np.abs(r - c) == nx))  # ... and nothing else inside them
    assert abs(T - T.T).max() == 0.0


def test_line_vcycle_is_symmetric_positive():
    g = W.Grid((W.uniform_axis(8, 1.0), W.tanh_axis(8, 2.0, 0.0, 1.0), W.uniform_axis(8, 1.5)))
    lv = mg.hierarchy(g, smoother="line")
    assert lv[0].T is not None
    n = g.n_cells
    Pi = np.eye(n) - 1.0 / n
    B = np.column_stack([mg.vcycle(lv, Pi[:, i]) for i in range(n)])
    assert np.abs(B - B.T).max() <= 1e-9 * np.abs(B).max()
    w = np.linalg.eigvalsh(0.5 * (B + B.T))
    assert w.min() >= -1e-9 * w.max() and np.sum(w > 1e-9 * w.max()) == n - 1


def test_line_smoothing_on_the_stretched_channel():
    """The walled tanh channel: line smoothing along y needs at most half the iterations of
    point smoothing, and reaches the same solution."""
    g = W.channel_grid(32, 32, 16)
    b = W.zero_mean(W.normal((g.n_cells, 1), 47))[:, 0]
    lp = mg.hierarchy(g)
    ll = mg.hierarchy(g, smoother="line")
    xp, itp = mg.mg_pcg(lp, b)
    xl, itl = mg.mg_pcg(ll, b)
    assert itl * 2 <= itp, (itl, itp)
    assert np.linalg.norm(xl - xp) <= 1e-8 * np.linalg.norm(xp)
