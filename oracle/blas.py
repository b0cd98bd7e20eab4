"""The other basic operations of Sec. 1 on an n x k block, column by column (FP64).

  dot:  out[j] = sum_i X[i, j] Y[i, j]
  axpy: Y[:, j] + alpha[j] X[:, j]
  axty: alpha X[i, j] Y[i, j]   (element-wise product)

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np


def dot(X, Y) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return np.array([float(np.dot(X[:, j], Y[:, j])) for j in range(X.shape[1])])


def axpy(alpha, X, Y) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    return Y + X * np.asarray(alpha, dtype=np.float64)[None, :]


def axty(alpha, X, Y) -> np.ndarray:
    return float(alpha) * np.asarray(X, dtype=np.float64) * np.asarray(Y, dtype=np.float64)
