"""Pins of the Galerkin initial guess (the Ritz-Galerkin projection onto the candidates'
span, Saad Sec. 5.1): its A-norm error is no larger than any candidate's (nor than random
combinations'), it is exact when the solution lies in the span, a single candidate gets the
optimal scale b^T v / v^T A v, and the error is A-orthogonal to every candidate."""
import numpy as np
import pytest

import workloads as W
from oracle import fvm
from oracle import guess as og


def _problem():
    """-L on a small walled channel, a zero-mean b and its zero-mean solution (dense solve of
    the singular system made regular by the rank-one term 1 1^T / n)."""
    g = W.channel_grid(12, 10, 8)
    A = (-fvm.laplacian(g)).tocsr()
    n = g.n_cells
    b = W.zero_mean(W.normal((n, 1), 60))[:, 0]
    x = np.linalg.solve(A.toarray() + np.ones((n, n)) / n, b)
    return A, b, x - x.mean()


def _vec(n, seed):
    return W.normal((n, 1), seed)[:, 0]


def _anorm(A, e):
    return float(np.sqrt(max(e @ (A @ e), 0.0)))


def test_no_worse_than_any_candidate_or_combination():
    A, b, x = _problem()
    rng = np.random.default_rng(61)
    cands = [x + 0.3 * _vec(len(x), 62 + i) for i in range(3)]
    x0, c = og.galerkin_guess(A, b, cands)
    e0 = _anorm(A, x - x0)
    for v in cands:
        assert e0 <= _anorm(A, x - v)
    for _ in range(20):
        w = rng.standard_normal(3)
        assert e0 <= _anorm(A, x - sum(wi * v for wi, v in zip(w, cands))) * (1 + 1e-12)
    r = A @ (x - x0)  # the error is A-orthogonal to the span (the Galerkin condition)
    for v in cands:
        assert abs(v @ r) <= 1e-9 * np.linalg.norm(v) * np.linalg.norm(b)


def test_exact_when_the_solution_is_in_the_span():
    A, b, x = _problem()
    v1 = _vec(len(x), 63)
    v2 = 0.5 * x - v1  # x = 2 v1 + 2 v2
    x0, c = og.galerkin_guess(A, b, [v1, v2])
    assert np.linalg.norm((x0 - x0.mean()) - x) <= 1e-9 * np.linalg.norm(x)
    assert np.allclose(c, [2.0, 2.0], rtol=1e-8)


@pytest.mark.parametrize("scale", [0.3, 1.0, -2.0])
def test_single_candidate_gets_the_optimal_scale(scale):
    A, b, x = _problem()
    v = scale * x + 0.1 * _vec(len(x), 64)
    x0, c = og.galerkin_guess(A, b, [v])
    assert np.isclose(c[0], (b @ v) / (v @ (A @ v)), rtol=1e-12)
    assert _anorm(A, x - x0) <= _anorm(A, x - v)


def test_dependent_candidates():
    A, b, x = _problem()
    v = x + 0.2 * _vec(len(x), 65)
    x0, c = og.galerkin_guess(A, b, [v, 2.0 * v])
    x1, _ = og.galerkin_guess(A, b, [v])
    assert np.linalg.norm(x0 - x1) <= 1e-9 * np.linalg.norm(x1)
    assert og.energy(A, b, x0) <= og.energy(A, b, v) + 1e-12 * abs(og.energy(A, b, v))
