"""Pins of the coarse-to-fine mapping oracle (Sec. 3.3, inline mesh refinement) against what
interpolation and averaging must satisfy, not against its own formulas: trilinear fields
reproduced on every row of a walled grid; the textbook 3/4, 1/4 weights on a uniform axis,
across the periodic seam included; interpolation (weights in [0, 1]) away from walls;
restriction as the volume-weighted transpose of injection, built here by brute force, and
conservation of the integral.  The axes differ in size, spacing and periodicity, so a
transposed axis fails."""
import numpy as np
import pytest

import workloads as W
from oracle import refine


def _walled_grid():
    return W.Grid((W.tanh_axis(8, 1.2, 0.0, 2.0), W.tanh_axis(6, 1.5, -1.0, 1.0), W.tanh_axis(10, 0.8, 0.0, 3.0)))


def _centres(grid):
    c = [0.5 * (a.nodes[:-1] + a.nodes[1:]) for a in grid.axes]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return x.ravel(), y.ravel(), z.ravel()


def _volumes(grid):
    w = [np.diff(a.nodes) for a in grid.axes]
    z, y, x = np.meshgrid(w[2], w[1], w[0], indexing="ij")
    return (x * y * z).ravel()


def test_prolongation_structure_and_constants():
    for g in (_walled_grid(), W.channel_grid(12, 8, 6), W.unit_periodic_grid(4)):
        P = refine.prolongation(g)
        gc = refine.coarse_grid(g)
        assert P.shape == (g.n_cells, gc.n_cells)
        assert np.array_equal(np.diff(P.indptr), np.full(g.n_cells, 8))
        assert np.all(np.diff(P.indices.reshape(-1, 8), axis=1) > 0)
        assert np.allclose(P @ np.ones(gc.n_cells), 1.0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_prolongation_exact_on_trilinear_fields(seed):
    """Every row, walls included (extrapolation there): f = sum of products (a + b x)(c + d y)(e + f z)."""
    g = _walled_grid()
    gc = refine.coarse_grid(g)
    P = refine.prolongation(g)
    r = W.normal(12, seed)
    def f(x, y, z):
        return (r[0] + r[1] * x) * (r[2] + r[3] * y) * (r[4] + r[5] * z) + (r[6] + r[7] * x) * (r[8] + r[9] * z) + r[10] * y
    xf, yf, zf = _centres(g)
    xc, yc, zc = _centres(gc)
    assert np.allclose(P @ f(xc, yc, zc), f(xf, yf, zf), rtol=0, atol=1e-12)
    # a field of x alone, to tell the axes apart
    assert np.allclose(P @ xc, xf, rtol=0, atol=1e-13)
    assert not np.allclose(P @ xc, zf)


def test_prolongation_periodic_axes():
    """Channel grid (periodic x and z, walled y): rows that do not cross a seam reproduce
    linear fields; on the uniform periodic axes every weight, seam rows included, is the
    textbook 3/4 (own parent) or 1/4 (the neighbour), times the y factor."""
    g = W.channel_grid(12, 8, 6)
    gc = refine.coarse_grid(g)
    P = refine.prolongation(g)
    xf, yf, zf = _centres(g)
    xc, yc, zc = _centres(gc)
    nx, ny, nz = g.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    inner = ((i > 0) & (i < nx - 1) & (k > 0) & (k < nz - 1)).ravel()
    for fc, ff in ((xc, xf), (zc, zf), (yc, yf), (xc * zc + yc, xf * zf + yf)):
        assert np.allclose((P @ fc)[inner], ff[inner], rtol=0, atol=1e-12)
    # x and z weights: P restricted to a y-constant field -> the x-z factors
    Px = refine.prolongation_1d(g.axes[0].nodes, True)
    assert np.allclose(np.sort(Px.data.reshape(-1, 2), axis=1), [[0.25, 0.75]] * nx, atol=1e-15)
    parents = np.arange(nx) // 2
    for t in range(nx):
        row = Px.getrow(t)
        w_own = row[0, parents[t]]
        assert abs(w_own - 0.75) <= 1e-15
    # the seam: fine cell 0 takes 1/4 of the last coarse cell
    assert abs(Px[0, nx // 2 - 1] - 0.25) <= 1e-15 and abs(Px[nx - 1, 0] - 0.25) <= 1e-15


def test_prolongation_interpolates_away_from_walls():
    """Away from walls the two coarse centres bracket the fine one: weights in [0, 1]."""
    for a in _walled_grid().axes:
        P1 = refine.prolongation_1d(a.nodes, False)
        n = P1.shape[0]
        for t in range(1, n - 1):
            w = P1.getrow(t).data
            assert np.all(w >= 0) and np.all(w <= 1), (t, w)
        assert np.any(refine.prolongation_1d(a.nodes, False).getrow(0).data < 0)  # extrapolated at the wall


def test_restriction_is_volume_weighted_injection_transpose():
    """R = V_c^-1 I^T V_f with I[f, parent(f)] = 1 (brute force), and the integral is kept."""
    for g in (_walled_grid(), W.channel_grid(12, 8, 6)):
        gc = refine.coarse_grid(g)
        R = refine.restriction(g).toarray()
        nx, ny, nz = g.shape
        I = np.zeros((g.n_cells, gc.n_cells))
        for kk in range(nz):
            for jj in range(ny):
                for ii in range(nx):
                    I[ii + nx * (jj + ny * kk), ii // 2 + (nx // 2) * (jj // 2 + (ny // 2) * (kk // 2))] = 1.0
        Vf, Vc = _volumes(g), _volumes(gc)
        assert np.allclose(R, (I.T * Vf[None, :]) / Vc[:, None], rtol=1e-14, atol=0)
        u = W.normal(g.n_cells, 7)
        assert abs(Vc @ (R @ u) - Vf @ u) <= 1e-13 * (Vf @ np.abs(u))
        assert np.allclose(R @ np.ones(g.n_cells), 1.0, atol=1e-15)


def test_odd_or_tiny_axes_rejected():
    with pytest.raises(ValueError):
        refine.prolongation_1d(np.linspace(0, 1, 8), True)  # 7 cells
    with pytest.raises(ValueError):
        refine.prolongation_1d(np.linspace(0, 1, 3), False)  # 2 cells
