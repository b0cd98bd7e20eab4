"""Wider Laplacian stencils on uniform periodic Cartesian grids (FP64): 13p and 27p.

Sec. 4.1 (channel flow) repeats the SpMM measurement with denser sparsity patterns, as a
higher-order discretisation would have: the first and second neighbours along each axis
(13 nonzeros per row, "13p") and every cell of the surrounding 3 x 3 x 3 block (27 per row,
"27p"), beside the first-neighbour FVM Laplacian (7 per row, "7p").  The paper fixes only
the patterns.  Readings used here (the coefficients do not change the SpMM's work):

  * uniform spacing h_d along each axis, periodic in all three, cells numbered
    lexicographically with x fastest (the same numbering as the FVM operators);
  * both operators volume-integrated like the FVM Laplacian, i.e. the cell volume
    V = hx hy hz times a pointwise approximation of the Laplacian, so that A = -L is
    symmetric positive semi-definite with the constants as null space;
  * 13p: along each axis the fourth-order central second difference
    (-u[-2] + 16 u[-1] - 30 u[0] + 16 u[+1] - u[+2]) / (12 h_d^2);
  * 27p: cubic cells (one h); weight -128, 14, 3, 1 (over 30 h^2) for the centre, the 6 face,
    12 edge and 8 corner neighbours: the 27-point stencil whose leading error is isotropic,
    L u / V = lap u + (h^2 / 12) lap^2 u + O(h^4).

Each row of 13p needs at least 5 cells along every axis and each row of 27p at least 3, so
that the wrapped neighbours are distinct cells.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def _cell_index(shape, i, j, k):
    nx, ny, _ = shape
    return i + nx * (j + ny * k)


def _from_offsets(shape, offsets) -> sp.csr_matrix:
    """L with L[c, c + o] = w for every cell c and every (offset o, weight w), o wrapped."""
    nx, ny, nz = shape
    n = nx * ny * nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    rows = _cell_index(shape, i, j, k)
    R, C, V = [], [], []
    for (dx, dy, dz), w in offsets:
        R.append(rows)
        C.append(_cell_index(shape, (i + dx) % nx, (j + dy) % ny, (k + dz) % nz))
        V.append(np.full(n, w, dtype=np.float64))
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(n, n)).tocsr()
    A.sort_indices()
    return A


def offsets_13p(h):
    """(offset, value) pairs of a 13p row: V times the fourth-order second difference along
    each axis, summed (Sec. 4.1)."""
    h = tuple(float(x) for x in h)
    vol = h[0] * h[1] * h[2]
    offsets = []
    centre = 0.0
    for d in range(3):
        e = [0, 0, 0]
        for o, c in ((-2, -1.0), (-1, 16.0), (1, 16.0), (2, -1.0)):
            e[d] = o
            offsets.append((tuple(e), vol * c / (12.0 * h[d] * h[d])))
        centre += vol * (-30.0) / (12.0 * h[d] * h[d])
    offsets.append(((0, 0, 0), centre))
    return offsets


def offsets_27p(h):
    """(offset, value) pairs of a 27p row on cubic cells of width h: V / (30 h^2) times -128
    (centre), 14 (faces), 3 (edges), 1 (corners) (Sec. 4.1)."""
    h = float(h)
    scale = h ** 3 / (30.0 * h * h)
    weight = {0: -128.0, 1: 14.0, 2: 3.0, 3: 1.0}  # by the number of nonzero offset components
    offsets = []
    for o in itertools.product((-1, 0, 1), repeat=3):
        offsets.append((o, scale * weight[sum(1 for c in o if c != 0)]))
    return offsets


def laplacian_13p(shape, h) -> sp.csr_matrix:
    """13p on the periodic grid of `shape` cells with spacings h (Sec. 4.1)."""
    shape = tuple(int(s) for s in shape)
    if min(shape) < 5:
        raise ValueError("13p needs at least 5 cells along every axis")
    return _from_offsets(shape, offsets_13p(h))


def laplacian_27p(shape, h) -> sp.csr_matrix:
    """27p on the periodic grid of `shape` cubic cells of width h (Sec. 4.1)."""
    shape = tuple(int(s) for s in shape)
    if min(shape) < 3:
        raise ValueError("27p needs at least 3 cells along every axis")
    return _from_offsets(shape, offsets_27p(h))


def row(shape, offsets, r):
    """Columns (sorted) and values of row r alone: the sampled rows of a grid too large to
    assemble here."""
    nx, ny, nz = (int(s) for s in shape)
    i, j, k = r % nx, (r // nx) % ny, r // (nx * ny)
    cols = [int(_cell_index((nx, ny, nz), (i + dx) % nx, (j + dy) % ny, (k + dz) % nz)) for (dx, dy, dz), _ in offsets]
    vals = [w for _, w in offsets]
    order = np.argsort(cols, kind="stable")
    return np.asarray(cols)[order], np.asarray(vals)[order]


def cell_coordinates(shape, h) -> np.ndarray:
    """Cell coordinates (index times spacing) in row order: (n, 3)."""
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([i.ravel() * h[0], j.ravel() * h[1], k.ravel() * h[2]], axis=1).astype(np.float64)
