"""Pins of the oracle's SpMM (Eq. (1), Algorithm 1) and of the paper's bound formulas (CPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import bounds, fvm, spmm
from tests.conftest import read_golden


def _rand_csr(nr, nc, density, seed):
    g = np.random.default_rng(seed)
    A = sp.random(nr, nc, density=density, random_state=g, format="csr")
    A.data = g.standard_normal(A.nnz)
    A.sort_indices()
    return A


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_spmm_equals_k_spmvs_and_kron(k):
    """P4: SpMM = k SpMVs = (I_k (x) A~) x = the dense product A X diag(c), on tiny inputs."""
    A = _rand_csr(37, 29, 0.2, k)
    X = W.normal((29, k), 10 + k)
    c = W.normal(k, 20 + k)
    Y = spmm.spmm(A, X)
    Yd = A.toarray() @ X  # dense matrix product: no sparse code involved
    Yk = spmm.kron_spmv(A, X)
    assert np.abs(Y - Yd).max() <= 1e-14 * np.abs(Yd).max()
    assert np.abs(Y - Yk).max() <= 1e-14 * np.abs(Yd).max()
    Yc = spmm.spmm(A, X, c)
    assert np.abs(Yc - Yd * c[None, :]).max() <= 1e-14 * np.abs(Yd * c[None, :]).max()
    # integer entries: every partial sum is exact, so any summation order gives the same bits
    Ai = A.copy()
    Ai.data = np.round(4 * Ai.data)
    Xi = np.round(8 * X)
    assert np.array_equal(spmm.spmm(Ai, Xi), Ai.toarray() @ Xi)
    assert np.array_equal(spmm.kron_spmv(Ai, Xi), Ai.toarray() @ Xi)


def test_spmm_rectangular_operators():
    """The divergence (cells x faces) and gradient (faces x cells) use n_r rows, not n_c."""
    g = W.channel_grid(5, 4, 3)
    M, G = fvm.divergence(g), fvm.gradient(g)
    U = W.normal((M.shape[1], 2), 5)
    P = W.normal((G.shape[1], 3), 6)
    assert spmm.spmm(M, U).shape == (M.shape[0], 2)
    assert np.allclose(spmm.spmm(G, P), G.toarray() @ P, rtol=1e-13, atol=1e-13)


def test_round_f32_is_rne():
    A = _rand_csr(10, 10, 0.5, 3)
    B = spmm.round_f32(A)
    assert np.array_equal(B.data, A.data.astype(np.float32).astype(np.float64))


def test_bound_identity_ub_equals_intensity_ratio():
    """P6: Eq. (pmspmm)'s upper bound is I(m)/I(1) of Eq. (ai), for any sizes."""
    for (nnz, nr, nc) in [(7e6, 1e6, 1e6), (27e6, 1e6, 1e6), (6e6, 1e6, 3e6), (2e3, 1e3, 7e2)]:
        for m in (1, 2, 3, 8, 32, 128):
            a = bounds.speedup_ub(m, nnz, nr, nc)
            b = bounds.speedup_ub_from_intensity(m, nnz, nr, nc)
            assert abs(a - b) <= 1e-12 * b
        assert bounds.speedup_ub(1, nnz, nr, nc) == pytest.approx(1.0, abs=1e-15)
        assert bounds.speedup_lb(1, nnz, nr, nc) == pytest.approx(1.0, abs=1e-15)
        for m in (2, 4, 16):
            assert bounds.speedup_lb(m, nnz, nr, nc) < bounds.speedup_ub(m, nnz, nr, nc) < m


def test_bound_sample_values():
    """Values of the Fig. 2 example (n = 1e6, 7 nnz per row), computed from Eq. (pmspmm)."""
    n = 1e6
    assert bounds.speedup_ub(2, 7 * n, n, n) == pytest.approx(1.7333, abs=1e-4)
    assert bounds.speedup_ub(8, 7 * n, n, n) == pytest.approx(3.8519, abs=1e-4)
    assert bounds.speedup_ub(32, 7 * n, n, n) == pytest.approx(5.5467, abs=1e-4)
    # the lower bound replaces 8 n_c m by 8 nnz m: no reuse of x at all
    nnz = 7 * n
    lb_direct = ((2 * nnz + 1) * 8 / (12 * nnz + 4 * (n + 1) + 8 * (8 * n + 8 * nnz + 8))) / (
        (2 * nnz + 1) / (12 * nnz + 4 * (n + 1) + (8 * n + 8 * nnz + 8)))
    assert bounds.speedup_lb(8, nnz, n, n) == pytest.approx(lb_direct, rel=1e-6)


@pytest.mark.parametrize("name,nnz_row", [("table2_ub_7nnz.txt", 7), ("table3_ub_27nnz.txt", 27)])
def test_tables_2_3_reproduced(name, nnz_row):
    """Tables 2-3 (Theta = 0.65, Pi = 16, gamma = 5) follow from Eqs. (bbtilde), (fullpm) with
    Phi = 1 and the upper bound I(m)/I(1), when the byte count charges 16 B per output entry."""
    betas = [1, 2, 5, 10, 20, 40]
    n = 1e6
    for row in read_golden(name):
        m = int(row[0])
        for beta, printed in zip(betas, row[1:]):
            p_spmm = bounds.speedup_ub_from_intensity(m, nnz_row * n, n, n, y_bytes=16)
            est = bounds.simulation_speedup(m, beta, 5.0, 16.0, p_spmm, 0.65)
            assert abs(est - printed) <= 0.011, (m, beta, est, printed)


def test_iteration_speedups_of_table_5_from_table_4():
    """Table 5's iteration speed-ups are m t_1 / t_m of the Table 4 wall-clock times."""
    rows = read_golden("table4_5_channel.txt")
    t1c, t1f = rows[0][1], rows[0][2]
    for m, tc, tf, pc, pf in rows:
        assert bounds.measured_speedup(m, t1c, tc) == pytest.approx(pc, abs=1.5e-3)
        assert bounds.measured_speedup(m, t1f, tf) == pytest.approx(pf, abs=1.5e-3)


def test_poisson_and_iteration_models_limits():
    """Eqs. (poipm) and (pmite): chi = 1 (pure SpMM) gives P_SpMM; chi = 0 gives 1."""
    for p in (1.0, 1.7, 3.85):
        assert bounds.poisson_speedup(p, 1.0) == pytest.approx(p)
        assert bounds.poisson_speedup(p, 0.0) == pytest.approx(1.0)
        assert bounds.iteration_speedup(p, 1.0) == pytest.approx(p)
        assert bounds.iteration_speedup(p, 0.0) == pytest.approx(1.0)
    # beta~ = beta without refinement (gamma = 0)
    assert bounds.beta_tilde(10.0, 0.0, 16.0) == pytest.approx(10.0)
    # Appendix A: a single matrix with weight 1 reduces to Eq. (pmspmm)
    assert bounds.weighted_ub(8, [(1.0, 7e6, 1e6, 1e6)]) == pytest.approx(bounds.speedup_ub(8, 7e6, 1e6, 1e6))
