"""Parity of the device Galerkin initial guess (rb_galerkin_guess; the Ritz-Galerkin
projection onto the candidates' span) against the oracle (GPU).

Bars: coefficients within 1e-8 relative of the oracle's and x0 within 1e-10 (relative L2) per
column on well-conditioned candidates; the energy-norm error no larger than every candidate's;
dependent candidates handled; X0 may be one of the candidates; more columns than one
reduction pass holds (k = 40)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fvm
from oracle import guess as og
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


def _system(k, seed):
    g = W.channel_grid(16, 12, 10)
    A = (-fvm.laplacian(g)).tocsr()
    n = g.n_cells
    B = W.zero_mean(W.normal((n, k), seed))
    X = np.linalg.solve(A.toarray() + np.ones((n, n)) / n, B)
    return A, B, X - X.mean(axis=0, keepdims=True)


def _anorm(A, e):
    return float(np.sqrt(max(e @ (A @ e), 0.0)))


@pytest.mark.parametrize("k,n_cand", [(1, 1), (3, 2), (3, 3), (8, 3), (40, 3)])
def test_galerkin_matches_oracle(rb, k, n_cand):
    A, B, X = _system(k, 900 + k)
    n = A.shape[0]
    cands = [X + (0.1 + 0.2 * a) * W.normal((n, k), 910 + a) for a in range(n_cand)]
    op = rb.Operator.from_scipy(A, k_max=k)
    coef = torch.empty((k, n_cand), dtype=torch.float64, device="cuda")
    X0 = rb.galerkin_guess(op, to_dev(B), [to_dev(c) for c in cands], coef=coef).cpu().numpy()
    cd = coef.cpu().numpy()
    for j in range(k):
        x0, c = og.galerkin_guess(A, B[:, j], [v[:, j] for v in cands])
        assert np.allclose(cd[j], c, rtol=1e-8, atol=1e-10), (j, cd[j], c)
        assert np.linalg.norm(X0[:, j] - x0) <= 1e-10 * np.linalg.norm(x0)
        e0 = _anorm(A, X[:, j] - X0[:, j])
        for v in cands:
            assert e0 <= _anorm(A, X[:, j] - v[:, j]) * (1 + 1e-12)


def test_galerkin_dependent_and_aliased(rb):
    """A candidate twice (scaled): the combination equals the single candidate's optimal
    scaling; X0 written over one of the candidate blocks; a strided candidate (ld > k)."""
    k = 3
    A, B, X = _system(k, 920)
    n = A.shape[0]
    v = X + 0.3 * W.normal((n, k), 921)
    op = rb.Operator.from_scipy(A, k_max=k)
    wide = torch.zeros((n, k + 2), dtype=torch.float64, device="cuda")
    wide[:, 1:1 + k] = to_dev(2.0 * v)
    Vd = to_dev(v)
    out = rb.galerkin_guess(op, to_dev(B), [Vd, wide[:, 1:1 + k]], X0=Vd).cpu().numpy()
    for j in range(k):
        x1, c1 = og.galerkin_guess(A, B[:, j], [v[:, j]])
        assert np.linalg.norm(out[:, j] - x1) <= 1e-9 * np.linalg.norm(x1)
    assert torch.all(wide[:, 0] == 0) and torch.all(wide[:, -1] == 0)


def test_galerkin_exact_in_span(rb):
    k = 2
    A, B, X = _system(k, 930)
    n = A.shape[0]
    v1 = W.normal((n, k), 931)
    v2 = 0.5 * X - v1
    op = rb.Operator.from_scipy(A, k_max=k)
    X0 = rb.galerkin_guess(op, to_dev(B), [to_dev(v1), to_dev(v2)]).cpu().numpy()
    X0 -= X0.mean(axis=0, keepdims=True)
    assert np.linalg.norm(X0 - X) <= 1e-9 * np.linalg.norm(X)
