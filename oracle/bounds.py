"""Arithmetic-intensity and speed-up models of the paper (FP64 CSR SpMM).

  * ``intensity``        Sec. 2, Eq. (ai): I_SpMM(m) = (2 nnz + 1) m / (12 nnz + 4 (n_r + 1) + m (8 n_r + 8 n_c + 8))
  * ``speedup_ub``       Eq. (pmspmm), upper bound as printed: m[3(nnz + n_r + 1) + 2 n_c] / (3 nnz + (1 + 2m)(n_r + 1) + 2 m n_c)
                         (the printed numerator has an unbalanced bracket; the reading used is
                         the one that equals I(m)/I(1), which the text states it is)
  * ``speedup_lb``       Eq. (pmspmm), lower bound: m[5 nnz + 3(n_r + 1)] / ((3 + 2m) nnz + (1 + 2m)(n_r + 1))
  * ``poisson_speedup``  Eq. (poipm): P_SpMM / (chi + (1 - chi) P_SpMM)
  * ``iteration_speedup``Eq. (pmite): 1 / (1 - Theta + Theta / P_SpMM)
  * ``beta_tilde``       Eq. (bbtilde): Pi (1 + gamma) / (gamma + Pi) beta
  * ``simulation_speedup`` Eq. (fullpm): (1 + beta~)/(Phi m + beta~) * iteration speed-up
  * ``weighted_ub``      Appendix A, weighted upper bound: sum_i omega_i P_ub(nnz_i, n_r_i, n_c_i)

Finding: the printed Tables 2-3 are reproduced (to about 0.01) only when the byte count
charges 16 bytes per output entry (a write-allocate read plus the write) instead of the 8
of Eq. (ai); ``intensity(..., y_bytes=16)`` gives that variant.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations


def intensity(m, nnz, n_r, n_c, y_bytes: int = 8):
    """Eq. (ai) (y_bytes = 8) and the variant that charges 16 bytes per output entry."""
    return (2 * nnz + 1) * m / (8 * nnz + 4 * nnz + 4 * (n_r + 1) + m * (y_bytes * n_r + 8 * n_c + 8))


def speedup_ub(m, nnz, n_r, n_c):
    return m * (3 * (nnz + n_r + 1) + 2 * n_c) / (3 * nnz + (1 + 2 * m) * (n_r + 1) + 2 * m * n_c)


def speedup_lb(m, nnz, n_r, n_c):
    return m * (5 * nnz + 3 * (n_r + 1)) / ((3 + 2 * m) * nnz + (1 + 2 * m) * (n_r + 1))


def speedup_ub_from_intensity(m, nnz, n_r, n_c, y_bytes: int = 8):
    return intensity(m, nnz, n_r, n_c, y_bytes) / intensity(1, nnz, n_r, n_c, y_bytes)


def poisson_speedup(p_spmm, chi):
    return p_spmm / (chi + (1.0 - chi) * p_spmm)


def iteration_speedup(p_spmm, theta):
    return 1.0 / (1.0 - theta + theta / p_spmm)


def beta_tilde(beta, gamma, Pi):
    return Pi * (1.0 + gamma) / (gamma + Pi) * beta


def simulation_speedup(m, beta, gamma, Pi, p_spmm, theta, Phi=1.0):
    bt = beta_tilde(beta, gamma, Pi)
    return (1.0 + bt) / (Phi * m + bt) * iteration_speedup(p_spmm, theta)


def weighted_ub(m, mats):
    """Appendix: mats = [(omega_i, nnz_i, n_r_i, n_c_i)], weights summing to 1."""
    return sum(w * speedup_ub(m, nnz, nr, nc) for (w, nnz, nr, nc) in mats)


def weighted_flop_rate(m, mats_times):
    """Appendix: sum_i omega_i OC_i / t_i with OC_i = (2 nnz_i + 1) m; mats_times = [(omega_i, nnz_i, t_i)]."""
    return sum(w * (2 * nnz + 1) * m / t for (w, nnz, t) in mats_times)


def measured_speedup(m, t_1, t_m):
    """Speed-up definitions of Sec. 2-3 (Poisson and iteration): m t_1 / t_m."""
    return m * t_1 / t_m
