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
    """FP32-inner refinement with reliable updates for one right-hand side: the k = 1 case of
    ``ir_reliable_pcg_block`` (same arguments, b a vector; returns x, its ColumnInfo and the
    number of sweeps)."""
    B = np.asarray(b, dtype=np.float64)[:, None]
    X0 = None if x0 is None else np.asarray(x0, dtype=np.float64)[:, None]
    X, infos, sweeps = ir_reliable_pcg_block(A, B, X0, rtol, inner_rtol, max_sweeps, max_iter, jacobi, project_mean)
    return X[:, 0], infos[0], sweeps


def ir_reliable_pcg_block(A: sp.csr_matrix, B: np.ndarray, X0=None, rtol=1e-10, inner_rtol=1e-4, max_sweeps=50,
                          max_iter=20000, jacobi=True, project_mean=False):
    """FP32-inner refinement that keeps the search direction across sweeps (reliable updates),
    for the k columns of B solved together.

    Each sweep, per column not yet converged: r = b - A x in FP64 (the column is done once
    ||r|| <= rtol ||b||), s = ||r||, r32 = r / s; the FP32 recurrence (FP32 matrix and vectors,
    FP64 dot accumulation) then continues with the next direction built from the replaced
    residual and the previous direction, both in the new normalisation: z = D^-1 r32,
    beta = (r32 . z) / (rz_prev (s_prev / s)^2), p32 <- z + beta p32 s_prev / s (the first
    sweep starts from p32 = z).  A column's target for the sweep is a fall of its residual by
    ``inner_rtol``, or only to half of what the outer tolerance still needs
    (0.5 rtol ||b|| / s) when that is larger.  The columns iterate together: one that has met
    its target keeps iterating until every column of the sweep has (the shared operator pass
    costs the same for all of them), and a column whose p . q <= 0 stops.  Then x += s d32 in
    FP64.  Replacing only the residual, not the direction, keeps the Krylov progress, so the
    iteration count stays close to plain FP64 CG.  ``iters`` counts, per column, the inner
    iterations it took part in.
    """
    f32 = np.float32
    A32 = A.astype(f32)
    B = np.asarray(B, dtype=np.float64)
    n, k = B.shape
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64)
    nb = np.linalg.norm(B, axis=0)
    dinv = (1.0 / A32.diagonal().astype(np.float64)).astype(f32) if jacobi else np.ones(n, dtype=f32)
    d64 = lambda u, v: float(np.dot(u.astype(np.float64), v.astype(np.float64)))
    P = [None] * k
    s_prev = np.zeros(k)
    rz = np.zeros(k)
    iters = [0] * k
    done = [bool(nb[j] == 0.0) for j in range(k)]
    for j in range(k):
        if done[j]:
            X[:, j] = 0.0
    sweeps = 0
    for sweep in range(max_sweeps + 1):
        sweeps = sweep
        R32, S, target, active = {}, {}, {}, []
        for j in range(k):
            if done[j]:
                continue
            r = _project(B[:, j] - A @ X[:, j], project_mean)
            s = np.linalg.norm(r)
            if s <= rtol * nb[j]:
                done[j] = True
                continue
            active.append(j)
            r32 = (r / s).astype(f32)
            z = dinv * r32
            rz_new = d64(r32, z)
            if P[j] is None:
                P[j] = z.copy()
            else:
                ratio = s_prev[j] / s
                beta = rz_new / (rz[j] * ratio * ratio)
                P[j] = z + f32(beta) * (P[j] * f32(ratio)).astype(f32)
            rz[j] = rz_new
            R32[j], S[j] = r32, s
            target[j] = max(inner_rtol**2 * d64(r32, r32), 0.25 * (rtol * nb[j] / s) ** 2)
        if not active or sweep == max_sweeps or max(iters) >= max_iter:
            break
        D = {j: np.zeros(n, dtype=f32) for j in active}
        running = list(active)
        met = {j: False for j in active}
        while running and max(iters) < max_iter:
            for j in list(running):
                q = (A32 @ P[j]).astype(f32)
                pq = d64(P[j], q)
                if not np.isfinite(pq) or pq <= 0.0:
                    running.remove(j)
                    continue
                alpha = f32(rz[j] / pq)
                D[j] = D[j] + alpha * P[j]
                R32[j] = R32[j] - alpha * q
                iters[j] += 1
                if d64(R32[j], R32[j]) <= target[j]:
                    met[j] = True
            if all(met[j] for j in running):
                break  # the sweep ends; the next one continues from each column's last direction
            for j in running:
                z = dinv * R32[j]
                rz_new = d64(R32[j], z)
                P[j] = z + f32(rz_new / rz[j]) * P[j]
                rz[j] = rz_new
        for j in active:
            X[:, j] = X[:, j] + S[j] * D[j].astype(np.float64)
            s_prev[j] = S[j]
    infos = []
    for j in range(k):
        X[:, j] = _project(X[:, j], project_mean)
        rel = np.linalg.norm(B[:, j] - A @ X[:, j]) / nb[j] if nb[j] > 0 else 0.0
        infos.append(ColumnInfo(iters[j], rel, OK if done[j] else NOCONV))
    return X, infos, sweeps


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
