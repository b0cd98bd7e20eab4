"""Pins of the oracle's staggered FVM operators against closed forms and invariants (CPU)."""
import numpy as np
import pytest

import workloads as W
from oracle import fvm

GRIDS = [
    W.unit_periodic_grid(6),
    W.channel_grid(8, 6, 5, gamma=1.5),
    W.rbc_grid(6, gamma=1.4),
    W.Grid((W.uniform_axis(5, 2.0, periodic=False), W.tanh_axis(7, 1.2), W.uniform_axis(4, 3.0)), "walls-xy"),
]


@pytest.mark.parametrize("N", [8, 12])
def test_fourier_eigenvalues_periodic(N):
    """P1: on the uniform periodic N^3 grid (h = 1/N, volume integrated) every Fourier mode
    is an eigenvector with lambda = -4 h sum_d sin^2(pi kappa_d / N)."""
    g = W.unit_periodic_grid(N)
    h = 1.0 / N
    L = fvm.laplacian(g)
    i = np.arange(N)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")  # I: x, ... ; flatten with x fastest below
    for kap in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 1, 2), (N // 2, N // 2 - 1, 1), (N - 1, 1, N // 2)]:
        for fn in (np.cos, np.sin):
            v = fn(2 * np.pi * (kap[0] * I + kap[1] * J + kap[2] * K) / N)
            v = v.transpose(2, 1, 0).ravel()  # order (k, j, i) -> id = i + N (j + N k)
            lam = -4 * h * sum(np.sin(np.pi * kd / N) ** 2 for kd in kap)
            Lv = L @ v
            scale = max(np.abs(v).max(), 1e-300) * 6 * h
            assert np.abs(Lv - lam * v).max() <= 1e-12 * scale


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g.name)
def test_div_grad_equals_direct_laplacian(g):
    """P2: M G equals the Laplacian assembled face by face from A_f / d_f."""
    L = fvm.laplacian(g)
    Ld = fvm.laplacian_direct(g)
    assert L.shape == Ld.shape
    diff = abs(L - Ld)
    assert diff.max() <= 1e-12 * abs(Ld).max()
    assert (L.indptr == Ld.indptr).all() and (L.indices == Ld.indices).all()


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g.name)
def test_zero_row_sums_symmetry_sign(g):
    """P3: L 1 = 0, L = L^T, non-positive diagonal, diagonal dominance of -L."""
    L = fvm.laplacian_direct(g)
    one = np.ones(L.shape[0])
    assert np.abs(L @ one).max() <= 1e-14 * abs(L).max() * 8
    assert abs(L - L.T).max() == 0.0
    d = L.diagonal()
    assert (d < 0).all()
    off = np.asarray(abs(L).sum(axis=1)).ravel() - np.abs(d)
    assert (np.abs(d) >= off * (1 - 1e-14)).all()
    G = fvm.gradient(g)
    M = fvm.divergence(g)
    assert np.abs(G @ one).max() == 0.0  # gradient of a constant
    assert np.abs(one @ M).max() == 0.0  # each face leaves one cell and enters another


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: g.name)
def test_nnz_and_face_counts(g):
    nx, ny, nz = g.shape
    n = g.n_cells
    nf = sum(n if a.periodic else n // a.n * (a.n - 1) for a in g.axes)
    M = fvm.divergence(g)
    assert M.shape == (n, nf)
    walls = sum(0 if a.periodic else 2 * (n // a.n) for a in g.axes)
    assert fvm.laplacian(g).nnz == 7 * n - walls


def test_gradient_of_linear_field_and_orientation():
    """(G p)_f = (p_plus - p_minus)/d_f: for p = y (cell centres) every y-face gives exactly 1,
    which pins the face orientation and the centre distance d_f on a stretched axis."""
    g = W.channel_grid(4, 9, 3, gamma=1.7)
    nx, ny, nz = g.shape
    yc = fvm.cell_centres(g.axes[1])
    p = np.broadcast_to(yc[None, :, None], (nz, ny, nx)).ravel()
    Gp = fvm.gradient(g) @ p
    n = g.n_cells
    gy = Gp[n : n + nx * (ny - 1) * nz]  # the y faces follow the n x faces
    assert np.allclose(gy, 1.0, rtol=0, atol=1e-13)
    assert np.abs(Gp[:n]).max() == 0.0  # p does not vary along x


def test_divergence_of_linear_flux_is_cell_volume():
    """Divergence theorem: for the face field u_f = (face y-coordinate) on y faces, M u equals
    the cell volume on every cell not touching a wall (div of (0, y, 0) is 1).  Pins A_f."""
    g = W.channel_grid(5, 8, 4, gamma=1.3)
    nx, ny, nz = g.shape
    n = g.n_cells
    ny_nodes = g.axes[1].nodes
    nf_x = n
    nf_y = nx * (ny - 1) * nz
    u = np.zeros(fvm.n_faces(g))
    # y faces: ordered (i fastest, then face position j = 1..ny-1, then k)
    ypos = ny_nodes[1:ny]
    u[nf_x : nf_x + nf_y] = np.broadcast_to(ypos[None, :, None], (nz, ny - 1, nx)).ravel()
    div = fvm.divergence(g) @ u
    vol = fvm.cell_volumes(g).reshape(nz, ny, nx)
    interior = div.reshape(nz, ny, nx)[:, 1:-1, :]
    assert np.allclose(interior, vol[:, 1:-1, :], rtol=1e-13, atol=0)


def test_adjointness():
    """<M u, p> = -<u, Omega_s G p> for random u, p (the symmetry-preserving pair)."""
    g = W.channel_grid(6, 5, 4)
    M, G = fvm.divergence(g), fvm.gradient(g)
    om = fvm.staggered_volumes(g)
    u = W.normal(M.shape[1], 1)
    p = W.normal(M.shape[0], 2)
    lhs = (M @ u) @ p
    rhs = -(u * om) @ (G @ p)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(M @ u) @ np.abs(p))


def test_channel_first_cell_height():
    """The tanh stretching with factor 1.5 on 160 cells in [-1, 1] (half height 1) gives a
    first-cell height y+ = Re_tau (y_1 - y_0) close to the 0.65 stated for the channel case
    at Re_tau = 180 (Sec. 4.1); this form gives 0.685."""
    ax = W.tanh_axis(160, 1.5)
    yplus = 180.0 * (ax.nodes[1] - ax.nodes[0])
    assert 0.6 < yplus < 0.75
