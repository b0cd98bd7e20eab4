"""Unstructured operator of the extruded-airfoil case (FP64).

The paper's third case (Sec. 4.3) is an unstructured airfoil mesh extruded along a
periodic span; Sec. 2 notes that repeated geometries give the repeated-block structure
when the unknowns are ordered suitably.  Ordering the unknowns plane by plane, the 3-D
vertex-centred Laplacian of a mesh extruded into Nz identical periodic planes is

    L3D = dz (I_Nz (x) L2D) + T_z (x) diag(a / dz)

where L2D is the 2-D (per unit depth) Laplacian, a_i the dual-cell areas, and T_z the
periodic second difference [1 -2 1] across the planes.  With the Nz plane values of one
2-D vertex stored next to each other, the first term is an SpMM with k = Nz columns and
the second couples the columns of one row.

Readings (the paper does not state the discretisation of its unstructured operator):
  * L2D is the cotangent-weight Laplacian: off-diagonal w_ij = (cot alpha_ij + cot beta_ij)/2
    over the (one or two) triangles sharing edge ij, diagonal -sum_j w_ij; it has the
    sign convention of the Cartesian L (negative semi-definite, zero row sums);
  * a negative edge weight (possible on boundary edges) is clamped to 0, which keeps
    -L2D an M-matrix;
  * a_i is the barycentric dual area: one third of the area of every incident triangle;
  * boundary edges (outer box and body) carry homogeneous Neumann conditions.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _cot_at(p_apex, p1, p2):
    """cot of the angle at p_apex of the triangle (p_apex, p1, p2)."""
    u = p1 - p_apex
    v = p2 - p_apex
    dot = u[:, 0] * v[:, 0] + u[:, 1] * v[:, 1]
    cross = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
    return dot / cross


def edge_weights(mesh):
    """Summed half-cotangent weight per undirected edge, before clamping: dict-free COO form."""
    P = mesh.points
    t = mesh.triangles.astype(np.int64)
    i, j, k = t[:, 0], t[:, 1], t[:, 2]
    # edge (j,k) is opposite vertex i, etc.
    w_jk = 0.5 * _cot_at(P[i], P[j], P[k])
    w_ki = 0.5 * _cot_at(P[j], P[k], P[i])
    w_ij = 0.5 * _cot_at(P[k], P[i], P[j])
    a = np.concatenate([j, k, i])
    b = np.concatenate([k, i, j])
    w = np.concatenate([w_jk, w_ki, w_ij])
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    n = P.shape[0]
    W = sp.coo_matrix((w, (lo, hi)), shape=(n, n)).tocsr()
    W.sum_duplicates()
    return W  # upper triangle, one entry per edge


def cot_laplacian(mesh, clamp: bool = True):
    """L2D with the pattern of the mesh adjacency (diagonal included).  Returns (L, n_clamped)."""
    W = edge_weights(mesh).tocoo()
    w = W.data.copy()
    n_clamped = int(np.count_nonzero(w < 0)) if clamp else 0
    if clamp:
        w = np.maximum(w, 0.0)
    n = mesh.points.shape[0]
    rows = np.concatenate([W.row, W.col])
    cols = np.concatenate([W.col, W.row])
    vals = np.concatenate([w, w])
    diag = np.zeros(n)
    np.add.at(diag, rows, -vals)
    # one COO with the edges and the diagonal keeps structural zeros (e.g. right-angle edges)
    L = sp.coo_matrix((np.concatenate([vals, diag]), (np.concatenate([rows, np.arange(n)]),
                                                      np.concatenate([cols, np.arange(n)]))), shape=(n, n)).tocsr()
    L.sum_duplicates()
    L.sort_indices()
    return L, n_clamped


def dual_areas(mesh) -> np.ndarray:
    """Barycentric dual-cell areas: a third of each incident triangle's area."""
    P = mesh.points
    t = mesh.triangles.astype(np.int64)
    a, b, c = P[t[:, 0]], P[t[:, 1]], P[t[:, 2]]
    area = 0.5 * np.abs((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    out = np.zeros(P.shape[0])
    for col in range(3):
        np.add.at(out, t[:, col], area / 3.0)
    return out


def periodic_second_difference(nz: int) -> sp.csr_matrix:
    """T_z: the periodic [1 -2 1] matrix across nz planes."""
    e = np.ones(nz)
    T = sp.diags([e[:-1], -2 * e, e[:-1]], [-1, 0, 1], shape=(nz, nz), format="lil")
    T[0, nz - 1] += 1.0
    T[nz - 1, 0] += 1.0
    if nz == 2:  # both neighbours are the same plane
        T = sp.lil_matrix(np.array([[-2.0, 2.0], [2.0, -2.0]]))
    return T.tocsr()


def extruded_operator(L2D: sp.csr_matrix, a: np.ndarray, nz: int, dz: float) -> sp.csr_matrix:
    """L3D = dz (I_Nz (x) L2D) + T_z (x) diag(a / dz), unknowns ordered plane by plane."""
    return (dz * sp.kron(sp.identity(nz), L2D) + sp.kron(periodic_second_difference(nz), sp.diags(a / dz))).tocsr()


def extruded_apply(L2D, a, nz, dz, X: np.ndarray) -> np.ndarray:
    """Y = L3D applied to X (n2D x Nz, one column per plane), through the assembled 3-D operator."""
    L3 = extruded_operator(L2D, a, nz, dz)
    y = L3 @ X.T.reshape(-1)  # plane-by-plane ordering: column z is plane z
    return y.reshape(nz, -1).T


def extruded_apply_loops(L2D: sp.csr_matrix, a, nz, dz, X) -> np.ndarray:
    """The same product written cell by cell (tiny inputs): lateral fluxes dz * L2D row, plus the
    two spanwise neighbours with coefficient a_i / dz across the periodic planes."""
    n = L2D.shape[0]
    Y = np.zeros((n, nz))
    for i in range(n):
        for z in range(nz):
            s = 0.0
            for p in range(L2D.indptr[i], L2D.indptr[i + 1]):
                s += dz * L2D.data[p] * X[L2D.indices[p], z]
            w = a[i] / dz
            s += w * (X[i, (z + 1) % nz] - X[i, z]) + w * (X[i, (z - 1) % nz] - X[i, z])
            Y[i, z] = s
    return Y
