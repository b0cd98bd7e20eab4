"""Pins of the BLAS-1 oracle (the other basic operations of Sec. 1) against exact rational
arithmetic and closed forms, on blocks whose shapes and per-column scalars differ so that a
transposed axis or a dropped factor fails."""
from fractions import Fraction

import numpy as np

import workloads as W
from oracle import blas


def _small_ints(shape, seed):
    return np.rint(8 * W.normal(shape, seed)).astype(np.float64)  # exact in FP64 and in products


def test_dot_equals_exact_rational_sums():
    X, Y = _small_ints((37, 5), 1), _small_ints((37, 5), 2)
    got = blas.dot(X, Y)
    for j in range(5):
        exact = sum(Fraction(int(X[i, j])) * Fraction(int(Y[i, j])) for i in range(37))
        assert got[j] == float(exact)
    # per column, not per row: a permutation of the columns permutes the results
    p = [3, 0, 4, 1, 2]
    assert np.array_equal(blas.dot(X[:, p], Y[:, p]), got[p])


def test_dot_closed_forms():
    n = 64
    i = np.arange(n)
    c = np.cos(2 * np.pi * 3 * i / n)[:, None]
    s = np.sin(2 * np.pi * 5 * i / n)[:, None]
    # orthogonal discrete Fourier modes; |cos|^2 sums to n / 2
    assert abs(blas.dot(c, s)[0]) < 1e-12
    assert abs(blas.dot(c, c)[0] - n / 2) < 1e-12


def test_axpy_per_column_scalars_exact():
    X, Y = _small_ints((29, 4), 3), _small_ints((29, 4), 4)
    alpha = np.array([1.0, -2.0, 0.5, 0.0])
    got = blas.axpy(alpha, X, Y)
    for j in range(4):
        for i in range(29):
            assert got[i, j] == float(Fraction(int(Y[i, j])) + Fraction(alpha[j]) * Fraction(int(X[i, j])))
    assert np.array_equal(blas.axpy(-alpha, X, blas.axpy(alpha, X, Y)), Y)  # exact inverse here


def test_axty_elementwise_exact():
    X, Y = _small_ints((31, 3), 5), _small_ints((31, 3), 6)
    got = blas.axty(0.25, X, Y)
    for j in range(3):
        for i in range(31):
            assert got[i, j] == float(Fraction(1, 4) * int(X[i, j]) * int(Y[i, j]))
    assert np.array_equal(blas.axty(1.0, X, np.ones_like(Y)), X)
