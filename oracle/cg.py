"""Poisson solves: Jacobi-preconditioned CG per column, FP32-inner iterative refinement,
and batches of uneven systems (FP64 reference arithmetic).

The paper solves the pressure Poisson equation of the projection method (Sec. 4) with CG
preconditioned by algebraic multigrid; the k flow states or parameters of Sec. 3 share
one matrix, so the k columns are k independent systems A x_j = b_j.  This oracle uses the
textbook preconditioned CG (Saad, Iterative Methods for Sparse Linear Systems,
Algorithm 9.1) with the Jacobi preconditioner D = diag(A).

Readings (the paper fixes none of these):
  * stop when the TRUE residual satisfies ||b - A x||_2 <= rtol ||b||_2 (relative to b,
    not to the first residual); the recurrence residual triggers the check, and when the
    true residual fails the recurrence restarts from r = b - A x, p = D^{-1} r;
  * columns are independent (not block CG); a converged column stops changing;
  * breakdown when p.q <= 0 or is not finite;
  * for the singular periodic/Neumann Laplacian (constant null space) with a compatible
    right-hand side, ``project_mean`` removes the mean from every freshly computed true
    residual and from the final solution, which selects the zero-mean solution.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

OK, NOCONV, BREAKDOWN = 0, 4, 5


@dataclasses.dataclass
class ColumnInfo:
    iters: int
    rel_res: float
    status: int


def _project(v: np.ndarray, on: bool) -> np.ndarray:
    return v - v.mean() if on else v


def pcg(A: sp.csr_matrix, b: np.ndarray, x0: np.ndarray | None = None, rtol: float = 1e-10,
        max_iter: int = 20000, jacobi: bool = True, project_mean: bool = False):
    """Preconditioned CG on one column in FP64 (Saad Algorithm 9.1, Jacobi preconditioner)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    dinv = 1.0 / A.diagonal() if jacobi else np.ones_like(b)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), ColumnInfo(0, 0.0, OK)
    r = _project(b - A @ x, project_mean)
    if np.linalg.norm(r) <= rtol * nb:
        return _project(x, project_mean), ColumnInfo(0, np.linalg.norm(r) / nb, OK)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    it = 0
    while it < max_iter:
        q = A @ p
        pq = p @ q
        if not np.isfinite(pq) or pq <= 0.0:
            return _project(x, project_mean), ColumnInfo(it, np.linalg.norm(b - A @ x) / nb, BREAKDOWN)
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if np.linalg.norm(r) <= rtol * nb:
            rt = _project(b - A @ x, project_mean)
            if np.linalg.norm(rt) <= rtol * nb:
                x = _project(x, project_mean)
                return x, ColumnInfo(it, np.linalg.norm(b - A @ x) / nb, OK)
            # residual replacement: restart the recurrence from the true residual
            r = rt
            z = dinv * r
            p = z.copy()
            rz = r @ z
            continue
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    x = _project(x, project_mean)
    return x, ColumnInfo(it, np.linalg.norm(b - A @ x) / nb, NOCONV)


def pcg_columns(A, B, X0=None, **kw):
    """k independent columns (Sec. 3: the k flow states share the operator)."""
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    infos = []
    for j in range(B.shape[1]):
        X[:, j], info = pcg(A, B[:, j], None if X0 is None else X0[:, j], **kw)
        infos.append(info)
    return X, infos


def pcg_fp32(A32: sp.csr_matrix, b32: np.ndarray, rtol: float, max_iter: int, jacobi: bool = True):
    """The inner solve of the refinement: FP32 matrix and vectors, dot products accumulated in FP64.

    Starts from zero; stops when the recurrence residual reaches rtol ||b||.
    """
    f32 = np.float32
    b32 = np.asarray(b32, dtype=f32)
    dinv = (1.0 / A32.diagonal().astype(np.float64)).astype(f32) if jacobi else np.ones_like(b32)
    x = np.zeros_like(b32)
    r = b32.copy()
    nb = np.sqrt(np.dot(b32.astype(np.float64), b32.astype(np.float64)))
    if nb == 0.0:
        return x, 0
    z = dinv * r
    p = z.copy()
    rz = np.dot(r.astype(np.float64), z.astype(np.float64))
    it = 0
    while it < max_iter:
        q = (A32 @ p).astype(f32)
        pq = np.dot(p.astype(np.float64), q.astype(np.float64))
        if not np.isfinite(pq) or pq <= 0.0:
            break
        alpha = f32(rz / pq)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        if np.sqrt(np.dot(r.astype(np.float64), r.astype(np.float64))) <= rtol * nb:
            break
        z = dinv * r
        rz_new = np.dot(r.astype(np.float64), z.astype(np.float64))
        beta = f32(rz_new / rz)
        rz = rz_new
        p = z + beta * p
    return x, it


def ir_pcg(A: sp.csr_matrix, b: np.ndarray, x0=None, rtol=1e-10, inner_rtol=1e-4, max_sweeps=50,
           inner_max_iter=20000, jacobi=True, project_mean=False):
    """FP32-inner iterative refinement with FP64 residuals and updates.

    Outer loop: r = b - A x in FP64; stop when ||r|| <= rtol ||b||; otherwise solve
    A32 d = r / ||r|| in FP32 (values and vectors rounded to nearest even) with FP64 dot
    accumulation to ``inner_rtol`` (relaxed to half of what the outer tolerance still needs,
    0.5 rtol ||b|| / ||r||, when that is larger), then x += ||r|| d in FP64.
    """
    A32 = A.astype(np.float32)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), ColumnInfo(0, 0.0, OK), 0
    total_inner = 0
    for sweep in range(max_sweeps + 1):
        r = _project(b - A @ x, project_mean)
        nr = np.linalg.norm(r)
        if nr <= rtol * nb:
            x = _project(x, project_mean)
            return x, ColumnInfo(total_inner, np.linalg.norm(b - A @ x) / nb, OK), sweep
        if sweep == max_sweeps:
            break
        tol = max(inner_rtol, 0.5 * rtol * nb / nr)
        d32, it = pcg_fp32(A32, (r / nr).astype(np.float32), tol, inner_max_iter, jacobi)
        total_inner += it
        x = x + nr * d32.astype(np.float64)
    x = _project(x, project_mean)
    return x, ColumnInfo(total_inner, np.linalg.norm(b - A @ x) / nb, NOCONV), max_sweeps


def ir_reliable_pcg(A: sp.csr_matrix, b: np.ndarray, x0=None, rtol=1e-10, inner_rtol=1e-4, max_sweeps=50,
                    max_iter=20000, jacobi=True, project_mean=False):
    """FP32-inner refinement that keeps the search direction across sweeps (reliable updates).

    Each sweep: r = b - A x in FP64 (stop if ||r|| <= rtol ||b||), s = ||r||, r32 = r / s; the
    FP32 recurrence (FP32 matrix and vectors, FP64 dot accumulation) then continues with the
    next direction built from the replaced residual and the previous direction, both in the
    new normalisation: z = D^-1 r32, beta = (r32 . z) / (rz_prev (s_prev / s)^2),
    p32 <- z + beta p32 s_prev / s (the first sweep starts from p32 = z), and runs until
    its residual falls by ``inner_rtol`` (or only to half of what the outer tolerance still
    needs, 0.5 rtol ||b|| / s, when that is larger); then x += s d32 in FP64.  Replacing only the
    residual, not the direction, keeps the Krylov progress, so the iteration count stays
    close to plain FP64 CG.
    """
    f32 = np.float32
    A32 = A.astype(f32)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), ColumnInfo(0, 0.0, OK), 0
    dinv = (1.0 / A32.diagonal().astype(np.float64)).astype(f32) if jacobi else np.ones(b.shape[0], dtype=f32)
    d64 = lambda u, v: float(np.dot(u.astype(np.float64), v.astype(np.float64)))
    p = None
    s_prev = 0.0
    rz = 0.0
    total = 0
    for sweep in range(max_sweeps + 1):
        r = _project(b - A @ x, project_mean)
        s = np.linalg.norm(r)
        if s <= rtol * nb:
            x = _project(x, project_mean)
            return x, ColumnInfo(total, np.linalg.norm(b - A @ x) / nb, OK), sweep
        if sweep == max_sweeps or total >= max_iter:
            break
        r32 = (r / s).astype(f32)
        z = dinv * r32
        rz_new = d64(r32, z)
        if p is None:
            p = z.copy()
        else:
            ratio = s_prev / s
            beta = rz_new / (rz * ratio * ratio)
            p = z + f32(beta) * (p * f32(ratio)).astype(f32)
        rz = rz_new
        rr0 = d64(r32, r32)
        d = np.zeros_like(r32)
        while total < max_iter:
            q = (A32 @ p).astype(f32)
            pq = d64(p, q)
            if not np.isfinite(pq) or pq <= 0.0:
                break
            alpha = f32(rz / pq)
            d = d + alpha * p
            r32 = r32 - alpha * q
            total += 1
            if d64(r32, r32) <= max(inner_rtol**2 * rr0, 0.25 * (rtol * nb / s) ** 2):
                break
            z = dinv * r32
            rz_new = d64(r32, z)
            p = z + f32(rz_new / rz) * p
            rz = rz_new
        x = x + s * d.astype(np.float64)
        s_prev = s
    x = _project(x, project_mean)
    return x, ColumnInfo(total, np.linalg.norm(b - A @ x) / nb, NOCONV), max_sweeps


def batch_solve(systems, **kw):
    """Uneven systems solved one after the other: each column of each system independently."""
    out = []
    for A, B in systems:
        out.append(pcg_columns(A, B, **kw))
    return out


def dense_pseudo_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Zero-mean solution of a singular SPD system with a constant null space.

    (A + 1 1^T) is SPD when A is symmetric positive semi-definite with null space span(1);
    for zero-mean b its solution is the zero-mean solution of A x = b.  Solved by a dense
    Cholesky factorisation.
    """
    n = A.shape[0]
    K = A + np.ones((n, n))
    Lc = np.linalg.cholesky(K)
    y = np.linalg.solve(Lc, b)
    return np.linalg.solve(Lc.T, y)
