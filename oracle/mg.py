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
    the same weight, the coarsest level solved by CG to a tight tolerance;
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


def hierarchy(grid, min_cells: int = 4) -> list:
    """Levels from fine to coarse."""
    levels = []
    g = grid
    while True:
        A = (-fvm.laplacian(g)).tocsr()
        can_coarsen = all(a.n % 2 == 0 and a.n // 2 >= min_cells for a in g.axes)
        P = refine.prolongation(g) if can_coarsen else None
        levels.append(Level(A, 1.0 / A.diagonal(), P))
        if not can_coarsen:
            return levels
        g = refine.coarse_grid(g)


def _project(x, on):
    return x - x.mean() if on else x


def vcycle(levels, r: np.ndarray, level: int = 0, nu: int = 2, omega: float = 2.0 / 3.0,
           project_mean: bool = True) -> np.ndarray:
    """One V(nu, nu) cycle for A_level e = r from e = 0."""
    lv = levels[level]
    if lv.P is None:
        e, _ = ocg.pcg(lv.A, r, rtol=1e-13, project_mean=project_mean)
        return e
    e = np.zeros_like(r)
    for _ in range(nu):
        e = e + omega * lv.dinv * (r - lv.A @ e)
    rc = lv.P.T @ (r - lv.A @ e)
    e = e + lv.P @ vcycle(levels, _project(rc, project_mean), level + 1, nu, omega, project_mean)
    for _ in range(nu):
        e = e + omega * lv.dinv * (r - lv.A @ e)
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
