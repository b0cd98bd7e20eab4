"""Stronger Poisson solvers for A = -L (FP64): geometric-multigrid-preconditioned CG, and block
CG over the k columns.

The paper solves its Poisson equations with CG preconditioned by an algebraic multigrid
(Sec. 4, Chronos' aAMG) and reports, in Appendix A, the SpMMs of every level of that
hierarchy (restriction, prolongation and level operators).  That library is closed; the
hierarchy here is geometric, built from the same pieces as the rest of the method:

  * levels: the grid and its repeated 2:1 coarsenings (every other node; each coarse cell is
    8 fine cells), while every axis keeps an even number of at least 4 cells;
  * level operators: A_l = -L on each level's grid (rediscretised, volume-integrated, so that
    the coarse operator matches P^T A P to leading order);
  * transfers: the trilinear prolongation P of the refinement maps and its transpose as the
    restriction of residuals (residuals of the volume-integrated equations are integrals, so
    P^T, not the cell average, carries them), which keeps the cycle symmetric;
  * smoothing: damped Jacobi, nu1 sweeps before and nu2 = nu1 after the coarse correction with
    the same weight (0.8 unless given: the smoothing-factor optimum of damped Jacobi is 4/5 for
    the 2-D and 6/7 for the 3-D Poisson stencil: the local Fourier analysis of damped Jacobi in
    Trottenberg, Oosterlee and Schueller, Multigrid), the coarsest level solved by CG to a tight
    tolerance; on grids stretched
    along one axis (a wall-refined channel) the point smoother leaves error that is smooth
    along that axis but rough across it, which no coarse grid of the full coarsening sees, so
    the line variant relaxes whole grid lines along the strongly coupled axis at once (block
    Jacobi with exact tridiagonal blocks: the classical remedy for anisotropy, e.g. Trottenberg,
    Oosterlee and Schueller, Multigrid, Sec. 5.1);
  * the preconditioner z = B r is one V-cycle from a zero guess; the outer iteration is
    Saad's preconditioned CG (Algorithm 9.1) with the zero-mean projection of singular
    (periodic or all-Neumann) problems.

Block CG (Sec. 5.1 names block-Krylov methods as the way to share more than the matrix across
the k columns): O'Leary's block conjugate gradient, one search block of k directions per
iteration, the k x k systems solved by a pseudo-inverse so that converged or dependent
directions do no harm.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import cg as ocg
from . import fvm, refine


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix       # -L on this level
    dinv: np.ndarray       # 1 / diag(A)
    P: sp.csr_matrix | None  # prolongation from the next coarser level (None on the coarsest)
    T: object = None       # line smoothing: a factorisation of the line-block part of A (None: point Jacobi)


def line_axis(grid, ratio: float = 4.0):
    """The wall-bounded axis along which the couplings of the Laplacian are strongest, if they
    exceed the others' by `ratio` somewhere: a coupling across a face along axis d scales as
    (transverse area) / (centre distance) ~ 1 / w_d^2 relative to the cell volume, so the
    axis with the smallest cell width against the largest of the other axes' widths.  Only
    walled axes qualify (their lines are plain tridiagonal blocks; grids are refined towards
    walls).  None when the grid is isotropic enough for point smoothing."""
    mins = [float(np.diff(a.nodes).min()) for a in grid.axes]
    best, worst = None, 1.0
    for d in range(3):
        if grid.axes[d].periodic:
            continue
        other = max(float(np.diff(grid.axes[e].nodes).max()) for e in range(3) if e != d)
        r = (other / mins[d]) ** 2
        if r > worst:
            best, worst = d, r
    return best if worst >= ratio else None


def line_block(grid, A: sp.csr_matrix, axis: int) -> sp.csr_matrix:
    """The part of A coupling cells along `axis` only (the diagonal and the two neighbours along
    the axis, wrapped on a periodic axis): block diagonal with one tridiagonal (periodic:
    cyclic) block per grid line."""
    n = [a.n for a in grid.axes]
    stride = [1, n[0], n[0] * n[1]][axis]
    A = A.tocoo()
    idx = np.arange(A.shape[0])
    pos = (idx // stride) % n[axis]
    # same line: the two cells differ only in their position along the axis
    same = (A.row - pos[A.row] * stride) == (A.col - pos[A.col] * stride)
    return sp.csr_matrix((A.data[same], (A.row[same], A.col[same])), shape=A.shape)


def hierarchy(grid, min_cells: int = 4, smoother: str = "jacobi") -> list:
    """Levels from fine to coarse.  smoother: "jacobi" (point) or "line" (block Jacobi over the
    grid lines of the strongest-coupling axis of the finest grid, when it has one; the coarse
    grids keep the fine grid's aspect ratios, so every level uses the same axis)."""
    import scipy.sparse.linalg as sla

    levels = []
    g = grid
    axis = line_axis(grid) if smoother == "line" else None
    while True:
        A = (-fvm.laplacian(g)).tocsr()
        can_coarsen = all(a.n % 2 == 0 and a.n // 2 >= min_cells for a in g.axes)
        P = refine.prolongation(g) if can_coarsen else None
        T = sla.splu(line_block(g, A, axis).tocsc()) if axis is not None else None
        levels.append(Level(A, 1.0 / A.diagonal(), P, T))
        if not can_coarsen:
            return levels
        g = refine.coarse_grid(g)


def _smooth(lv: Level, e: np.ndarray, r: np.ndarray, omega: float) -> np.ndarray:
    """One damped sweep: e + omega B^{-1} (r - A e), B = diag(A) or the line blocks of A."""
    s = r - lv.A @ e
    return e + omega * (lv.T.solve(s) if lv.T is not None else lv.dinv * s)


def _project(x, on):
    return x - x.mean() if on else x


def vcycle(levels, r: np.ndarray, level: int = 0, nu: int = 2, omega: float = 0.8,
           project_mean: bool = True) -> np.ndarray:
    """One V(nu, nu) cycle for A_level e = r from e = 0."""
    lv = levels[level]
    if lv.P is None:
        e, _ = ocg.pcg(lv.A, r, rtol=1e-13, project_mean=project_mean)
        return e
    e = np.zeros_like(r)
    for _ in range(nu):
        e = _smooth(lv, e, r, omega)
    rc = lv.P.T @ (r - lv.A @ e)
    e = e + lv.P @ vcycle(levels, _project(rc, project_mean), level + 1, nu, omega, project_mean)
    for _ in range(nu):
        e = _smooth(lv, e, r, omega)
    return _project(e, project_mean)


def mg_pcg(levels, b: np.ndarray, rtol: float = 1e-10, max_iter: int = 500, project_mean: bool = True,
           flexible: bool = False, **kw):
    """CG on A_0 x = b preconditioned by one V-cycle per iteration (Saad Algorithm 9.1).

    flexible: take beta in the Polak-Ribiere form z_new . (r_new - r_old) / (z_old . r_old)
    (Notay's flexible CG), which tolerates a preconditioner that is not exactly the same
    symmetric operator at every iteration, e.g. a V-cycle run in lower precision.  With a
    fixed symmetric preconditioner z_new . r_old = 0 in exact arithmetic, so both forms give
    the same iterates."""
    A = levels[0].A
    b = _project(np.asarray(b, dtype=np.float64), project_mean)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return x, 0
    r = b.copy()
    z = vcycle(levels, r, project_mean=project_mean, **kw)
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        if np.linalg.norm(_project(b - A @ x, project_mean)) <= rtol * nb:
            return _project(x, project_mean), it
        r_old = r + alpha * q
        z = vcycle(levels, r, project_mean=project_mean, **kw)
        rz_new = r @ z
        beta = (z @ (r - r_old)) / rz if flexible else rz_new / rz
        p = z + beta * p
        rz = rz_new
    return _project(x, project_mean), max_iter


def block_cg(A, B: np.ndarray, rtol: float = 1e-10, max_iter: int = 1000, project_mean: bool = False):
    """O'Leary's block CG on A X = B (no preconditioner): X, iterations.  Stops when every
    column's true residual is below rtol times its right-hand side."""
    B = np.asarray(B, dtype=np.float64)
    if project_mean:
        B = B - B.mean(axis=0, keepdims=True)
    nb = np.linalg.norm(B, axis=0)
    X = np.zeros_like(B)
    R = B.copy()
    P = R.copy()
    RR = R.T @ R
    for it in range(1, max_iter + 1):
        Q = A @ P
        alpha = np.linalg.pinv(P.T @ Q) @ RR
        X = X + P @ alpha
        R = R - Q @ alpha
        T = B - A @ X
        if project_mean:
            T = T - T.mean(axis=0, keepdims=True)
        if np.all(np.linalg.norm(T, axis=0) <= rtol * np.where(nb > 0, nb, 1.0)):
            return X, it
        RR_new = R.T @ R
        beta = np.linalg.pinv(RR) @ RR_new
        P = R + P @ beta
        RR = RR_new
    return X, max_iter
