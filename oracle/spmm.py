"""SpMM over k right-hand sides: the repeated-block product of Sec. 2 (Eq. (1), Algorithm 1).

A = I_k (x) A~ applied to the stacked vector (x_1 ... x_k) equals the sparse-times-dense
product A~ [x_1 ... x_k] (Eq. (1)).  With the vectors interleaved by column (the
array-of-structures layout of Algorithm 1, X[i, j] at position k i + j), the output is

    Y[i, j] = c[j] * sum_{p = ptr[i]}^{ptr[i+1]-1} val[p] * X[idx[p], j]      (Algorithm 1)

Readings (the listing is ambiguous in three places):
  * ``val[p]`` is one value shared by every column: A = I_k (x) A~ has one coefficient per
    nonzero; the listing's two-index ``val[j][k]`` is read as this shared value, with
    per-column variation only through ``c``;
  * the row loop and the output length run over the rows n_r of A~ (the listing writes
    n_c, which differs for the rectangular divergence and gradient);
  * ``c`` is an optional per-column scale (e.g. a per-parameter coefficient of the
    multiple-parameter runs of Sec. 3.4); absent means 1.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def spmm(A: sp.csr_matrix, X: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """The definition: k independent SpMVs, one per column, then the per-column scale."""
    X = np.asarray(X)
    k = X.shape[1]
    Y = np.empty((A.shape[0], k), dtype=np.result_type(A.dtype, X.dtype))
    for j in range(k):
        Y[:, j] = A @ X[:, j]
        if c is not None:
            Y[:, j] *= c[j]
    return Y


def kron_spmv(A: sp.csr_matrix, X: np.ndarray) -> np.ndarray:
    """(I_k (x) A~) applied to the column-stacked vector (x_1; ...; x_k), Eq. (1)'s left-hand side."""
    k = X.shape[1]
    big = sp.kron(sp.identity(k, format="csr"), A, format="csr")
    y = big @ X.T.reshape(-1)  # stack columns one after the other
    return y.reshape(k, A.shape[0]).T


def abs_bound(A: sp.csr_matrix, X: np.ndarray, c: np.ndarray | None = None) -> np.ndarray:
    """(|A~| |X|) scaled by |c|: the denominator of the componentwise error test."""
    absA = A.copy()
    absA.data = np.abs(absA.data)
    return spmm(absA, np.abs(X), None if c is None else np.abs(c))


def round_f32(A: sp.csr_matrix) -> sp.csr_matrix:
    """A copy of A with its values rounded to FP32 (round to nearest even) and kept as FP64."""
    B = A.copy()
    B.data = B.data.astype(np.float32).astype(np.float64)
    return B
