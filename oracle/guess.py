"""The Galerkin initial guess: the best combination of given candidate vectors in the energy
norm of the Poisson matrix (FP64).

Not from the paper (its solver starts each step from the previous pressure); it combines the
learned guess with the previous pressures.  For SPD A (semi-definite with a compatible
right-hand side) and candidates v_1 .. v_c, the x0 in their span that minimises the A-norm of
the error x* - x0 is the Ritz-Galerkin solution (Saad, Iterative Methods for Sparse Linear
Systems, Sec. 5.1, the orthogonal projection method with K = L = span{v}): x0 = V c with

    (V^T A V) c = V^T b,

the error then A-orthogonal to every candidate.  Equivalently it minimises the energy
phi(x) = x^T A x / 2 - b^T x, which differs from the squared A-norm error by a constant, so
it is never worse than any single candidate (or than any combination of them).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np


def galerkin_guess(A, b: np.ndarray, cands) -> tuple:
    """x0 = V c minimising ||x* - V c||_A; returns (x0, c).  Dependent candidates (a singular
    Gram matrix) take the minimum-norm c (least squares)."""
    V = np.column_stack([np.asarray(v, dtype=np.float64) for v in cands])
    W = A @ V
    G = V.T @ W
    g = V.T @ np.asarray(b, dtype=np.float64)
    c = np.linalg.lstsq(G, g, rcond=None)[0]
    return V @ c, c


def energy(A, b: np.ndarray, x: np.ndarray) -> float:
    """phi(x) = x^T A x / 2 - b^T x (the A-norm error squared, halved, minus a constant)."""
    return 0.5 * float(x @ (A @ x)) - float(b @ x)
