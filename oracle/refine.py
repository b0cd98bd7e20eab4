"""Coarse-to-fine mapping of cell fields for inline mesh refinement (FP64).

Sec. 3.3 (inline mesh refinement) starts the flow states on a coarser mesh and, once they
have developed, maps them onto the target mesh, consistently, in the manner of classical
adaptive mesh refinement; the mapping applied to the k states at once is a rectangular
SpMM.  The paper does not give the mapping.  Readings used here:

  * the coarse grid is the fine grid with every other node removed along each axis (2:1
    nesting; each coarse cell is the union of 8 fine cells);
  * prolongation P (fine cells x coarse cells): along each axis, linear interpolation in the
    physical cell-centre coordinate between the two coarse centres nearest to the fine
    centre (the coarse cell's left neighbour for a left child, its right neighbour for a
    right child), across the seam of a periodic axis (the neighbour's coordinate shifted by
    the period) and by linear extrapolation from the two first (last) coarse centres next to
    a wall; the 3-D map is the tensor product of the three 1-D ones, so it reproduces every
    field that is linear in each coordinate (trilinear) exactly, on every row;
  * restriction R (coarse cells x fine cells): the volume-weighted mean of the 8 children,
    which conserves the integral of the field.

Cells are numbered x fastest, as the FVM operators; P and R have 8 entries in every row.

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def coarse_nodes(nodes: np.ndarray) -> np.ndarray:
    """Nodes of the 2:1 coarser axis: every other node."""
    if (len(nodes) - 1) % 2 or len(nodes) - 1 < 4:
        raise ValueError("the fine axis needs an even number (>= 4) of cells")
    return np.asarray(nodes, dtype=np.float64)[::2]


def prolongation_1d(nodes: np.ndarray, periodic: bool) -> sp.csr_matrix:
    """Linear interpolation from the coarse cell centres to the fine cell centres of one axis."""
    nodes = np.asarray(nodes, dtype=np.float64)
    cn = coarse_nodes(nodes)
    xf = 0.5 * (nodes[:-1] + nodes[1:])
    xc = 0.5 * (cn[:-1] + cn[1:])
    n_f, n_c = len(xf), len(xc)
    period = nodes[-1] - nodes[0]
    rows, cols, vals = [], [], []
    for t in range(n_f):
        parent = t // 2
        lo, hi = (parent - 1, parent) if t % 2 == 0 else (parent, parent + 1)
        x_lo = x_hi = None
        if lo < 0:
            if periodic:
                lo, x_lo = n_c - 1, xc[n_c - 1] - period
            else:
                lo, hi = 0, 1
        if hi >= n_c:
            if periodic:
                hi, x_hi = 0, xc[0] + period
            else:
                lo, hi = n_c - 2, n_c - 1
        x_lo = xc[lo] if x_lo is None else x_lo
        x_hi = xc[hi] if x_hi is None else x_hi
        w_hi = (xf[t] - x_lo) / (x_hi - x_lo)
        w_lo = (x_hi - xf[t]) / (x_hi - x_lo)
        rows += [t, t]
        cols += [lo, hi]
        vals += [w_lo, w_hi]
    P = sp.coo_matrix((vals, (rows, cols)), shape=(n_f, n_c)).tocsr()
    P.sort_indices()
    return P


def restriction_1d(nodes: np.ndarray) -> sp.csr_matrix:
    """Width-weighted mean of the two children of each coarse cell of one axis."""
    nodes = np.asarray(nodes, dtype=np.float64)
    cn = coarse_nodes(nodes)
    wf = np.diff(nodes)
    wc = np.diff(cn)
    n_c = len(wc)
    rows = np.repeat(np.arange(n_c), 2)
    cols = np.arange(2 * n_c)
    vals = wf / np.repeat(wc, 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_c, 2 * n_c))


def prolongation(grid) -> sp.csr_matrix:
    """P on a 3-D grid: the Kronecker product of the axes' 1-D maps (x fastest)."""
    Px, Py, Pz = (prolongation_1d(a.nodes, a.periodic) for a in grid.axes)
    P = sp.kron(Pz, sp.kron(Py, Px, format="csr"), format="csr")
    P.eliminate_zeros()  # kron stores the zeros of its dense blocks; no weight here is 0
    P.sort_indices()
    return P


def restriction(grid) -> sp.csr_matrix:
    """R on a 3-D grid: the Kronecker product of the axes' 1-D volume-weighted means."""
    Rx, Ry, Rz = (restriction_1d(a.nodes) for a in grid.axes)
    R = sp.kron(Rz, sp.kron(Ry, Rx, format="csr"), format="csr")
    R.eliminate_zeros()
    R.sort_indices()
    return R


def coarse_grid(grid):
    """The 2:1 coarser grid (same periodicity), as a workloads.Grid-like object."""
    import dataclasses

    axes = tuple(dataclasses.replace(a, nodes=coarse_nodes(a.nodes)) for a in grid.axes)
    return dataclasses.replace(grid, axes=axes, name=grid.name + "/2")
