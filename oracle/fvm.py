"""Staggered symmetry-preserving finite-volume operators on Cartesian grids (FP64).

Follows the semi-discrete Navier-Stokes form of Sec. 3 (Eq. (ns)): M is the face-to-cell
divergence, Omega_s the staggered (face) control volumes, G = -Omega_s^{-1} M^T the
cell-to-face gradient, and the Laplacian L = M G (the diffusive/Poisson operator).  The
symmetry-preserving construction (Sec. 4) is what makes L symmetric and negative
semi-definite with zero row sums.

Readings of the paper used here (it gives none of these details):
  * face area A_f = product of the two transverse cell widths; d_f = distance between the
    two adjacent cell centres (across the periodic seam where the axis is periodic);
    Omega_s,f = A_f d_f;
  * faces on walls are excluded (no-penetration), which gives homogeneous Neumann
    conditions for the pressure;
  * faces are numbered direction by direction (x, then y, then z); within a direction
    lexicographically with x fastest, the face coordinate along its own axis running over
    0..n-1 (periodic: face i separates cells i-1 mod n and i) or 1..n-1 (walls: face i
    separates cells i-1 and i).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def cell_widths(axis) -> np.ndarray:
    return np.diff(axis.nodes)


def cell_centres(axis) -> np.ndarray:
    return 0.5 * (axis.nodes[:-1] + axis.nodes[1:])


def _face_positions(axis):
    """Positions along the axis of the faces of this direction and their centre distance d_f."""
    n = axis.n
    w = cell_widths(axis)
    if axis.periodic:
        pos = np.arange(n)
        lo = (pos - 1) % n
        d = 0.5 * (w[lo] + w[pos])
    else:
        pos = np.arange(1, n)
        lo = pos - 1
        d = 0.5 * (w[lo] + w[pos])
    return pos, lo, d


def faces(grid):
    """All faces as arrays (minus cell, plus cell, area A_f, centre distance d_f), x then y then z."""
    nx, ny, nz = grid.shape
    widths = [cell_widths(a) for a in grid.axes]
    minus, plus, area, dist = [], [], [], []
    for d in range(3):
        pos, lo, dd = _face_positions(grid.axes[d])
        ranges = [np.arange(nx), np.arange(ny), np.arange(nz)]
        lo_ranges = list(ranges)
        ranges[d] = pos
        lo_ranges[d] = lo
        # face coordinates, x fastest
        K, J, I = np.meshgrid(ranges[2], ranges[1], ranges[0], indexing="ij")
        Kl, Jl, Il = np.meshgrid(lo_ranges[2], lo_ranges[1], lo_ranges[0], indexing="ij")
        plus_c = (I + nx * (J + ny * K)).ravel()
        minus_c = (Il + nx * (Jl + ny * Kl)).ravel()
        others = [e for e in range(3) if e != d]
        wa = widths[others[0]]
        wb = widths[others[1]]
        idx = [I, J, K]
        A = (wa[idx[others[0]]] * wb[idx[others[1]]]).ravel()
        dist_f = _dist_lookup(dd, idx[d], grid.axes[d].periodic).ravel()
        minus.append(minus_c)
        plus.append(plus_c)
        area.append(A)
        dist.append(dist_f)
    return np.concatenate(minus), np.concatenate(plus), np.concatenate(area), np.concatenate(dist)


def _dist_lookup(dd, coord, periodic):
    # dd is indexed by face number along the axis: periodic faces 0..n-1, wall faces 1..n-1
    return dd[coord] if periodic else dd[coord - 1]


def n_faces(grid) -> int:
    return faces(grid)[0].shape[0]


def divergence(grid) -> sp.csr_matrix:
    """M: cells x faces.  +A_f on the cell below the face (its plus face), -A_f on the cell above."""
    mi, pl, A, _ = faces(grid)
    nf = mi.shape[0]
    f = np.arange(nf)
    rows = np.concatenate([mi, pl])
    cols = np.concatenate([f, f])
    vals = np.concatenate([A, -A])
    M = sp.csr_matrix((vals, (rows, cols)), shape=(grid.n_cells, nf))
    M.sort_indices()
    return M


def interpolation(grid) -> sp.csr_matrix:
    """Gamma_{c->s} (faces x cells): the mean of the two cells of each face, the cell-to-face
    interpolator of Eq. (ns) (u_s = Gamma u_c) and of the convective operator C = M U_s Gamma."""
    mi, pl, _, _ = faces(grid)
    nf = mi.shape[0]
    f = np.arange(nf)
    I = sp.csr_matrix((np.full(2 * nf, 0.5), (np.concatenate([f, f]), np.concatenate([mi, pl]))),
                      shape=(nf, grid.n_cells))
    I.sort_indices()
    return I


def face_blocks(grid):
    """(first face, count) of the x, y and z faces in the face numbering."""
    out, start = [], 0
    for d, a in enumerate(grid.axes):
        nd = 1
        for e, b in enumerate(grid.axes):
            nd *= (b.n if (e != d or b.periodic) else b.n - 1)
        out.append((start, nd))
        start += nd
    return out


def staggered_volumes(grid) -> np.ndarray:
    """Omega_s: the face control volumes A_f d_f."""
    _, _, A, d = faces(grid)
    return A * d


def gradient(grid) -> sp.csr_matrix:
    """G = -Omega_s^{-1} M^T (faces x cells): (G p)_f = (p_plus - p_minus) / d_f."""
    M = divergence(grid)
    om = staggered_volumes(grid)
    G = (-sp.diags(1.0 / om) @ M.T).tocsr()
    G.sort_indices()
    return G


def laplacian(grid) -> sp.csr_matrix:
    """L = M G (cells x cells), the volume-integrated Laplacian of the projection method."""
    L = (divergence(grid) @ gradient(grid)).tocsr()
    L.sum_duplicates()
    L.sort_indices()
    return L


def laplacian_direct(grid) -> sp.csr_matrix:
    """L assembled face by face from the coefficients A_f / d_f (independent of M and G).

    Each face adds  c (p_other - p_self)  to both adjacent cells, c = A_f / d_f.
    """
    mi, pl, A, d = faces(grid)
    c = A / d
    n = grid.n_cells
    rows = np.concatenate([mi, pl, mi, pl])
    cols = np.concatenate([pl, mi, mi, pl])
    vals = np.concatenate([c, c, -c, -c])
    L = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    L.sum_duplicates()
    L.sort_indices()
    return L


def cell_volumes(grid) -> np.ndarray:
    wx, wy, wz = (cell_widths(a) for a in grid.axes)
    return (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).ravel()


def jacobi_diag(A: sp.csr_matrix) -> np.ndarray:
    return A.diagonal().astype(np.float64)
