"""Pins of the 13p and 27p stencil oracle (Sec. 4.1) against properties of the continuous
Laplacian, not against its own weights: exactness on polynomials (degree <= 5; 27p with its
isotropic h^2 / 12 lap^2 term), zero row sums and symmetry (the periodic wrap), plane waves
as eigenvectors on every row including the wrapped ones.  The grids have a different size
and, for 13p, a different spacing along each axis, so a transposed axis fails."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle import stencil


def _poly_eval(poly, P):
    return sum(c * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** e for (a, b, e), c in poly.items())


def _diff(poly, axis, times=1):
    out = dict(poly)
    for _ in range(times):
        nxt = {}
        for m, c in out.items():
            if m[axis] == 0:
                continue
            mm = list(m)
            mm[axis] -= 1
            nxt[tuple(mm)] = nxt.get(tuple(mm), 0.0) + c * m[axis]
        out = nxt
    return out


def _lap(poly):
    res = {}
    for d in range(3):
        for m, c in _diff(poly, d, 2).items():
            res[m] = res.get(m, 0.0) + c
    return res


def _random_poly(seed, degree=5):
    r = W.normal(64, seed)
    poly, t = {}, 0
    for m in itertools.product(range(degree + 1), repeat=3):
        if sum(m) <= degree:
            poly[m] = float(np.round(4 * r[t % 64]) / 4)
            t += 1
    return poly


def _interior(shape, reach):
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = ((i >= reach) & (i < nx - reach) & (j >= reach) & (j < ny - reach) & (k >= reach) & (k < nz - reach))
    return m.ravel()


def _structure(L, per_row):
    n = L.shape[0]
    assert np.array_equal(np.diff(L.indptr), np.full(n, per_row))
    for r in range(n):  # sorted, distinct columns
        c = L.indices[L.indptr[r]:L.indptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    assert abs(L - L.T).max() == 0.0
    scale = abs(L).sum(axis=1).A.ravel()
    assert np.all(np.abs(L.sum(axis=1).A.ravel()) <= 1e-14 * scale)


def test_13p_structure_symmetry_null_space():
    _structure(stencil.laplacian_13p((5, 6, 7), (0.3, 0.2, 0.25)), 13)
    _structure(stencil.laplacian_13p((9, 5, 8), (0.1, 0.1, 0.1)), 13)


def test_27p_structure_symmetry_null_space():
    _structure(stencil.laplacian_27p((3, 4, 5), 0.2), 27)
    _structure(stencil.laplacian_27p((6, 3, 7), 0.5), 27)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_13p_exact_on_quintics(seed):
    """Fourth-order axial differences are exact on every polynomial of degree <= 5:
    L p = V lap p at rows whose stencil does not wrap."""
    shape, h = (9, 10, 11), (0.3, 0.2, 0.25)
    L = stencil.laplacian_13p(shape, h)
    P = stencil.cell_coordinates(shape, h)
    poly = _random_poly(seed)
    p = _poly_eval(poly, P)
    got = L @ p
    want = h[0] * h[1] * h[2] * _poly_eval(_lap(poly), P)
    m = _interior(shape, 2)
    assert m.sum() == 5 * 6 * 7
    tol = 1e-12 * (abs(L) @ np.abs(p))
    assert np.all(np.abs(got - want)[m] <= tol[m])


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_27p_isotropic_error_on_quintics(seed):
    """L p = V (lap p + h^2 / 12 lap^2 p) exactly for every polynomial of degree <= 5 at rows
    whose stencil does not wrap: the leading error of the 27-point stencil is isotropic."""
    shape, h = (7, 6, 8), 0.3
    L = stencil.laplacian_27p(shape, h)
    P = stencil.cell_coordinates(shape, (h, h, h))
    poly = _random_poly(seed)
    p = _poly_eval(poly, P)
    got = L @ p
    lap = _lap(poly)
    want = h ** 3 * (_poly_eval(lap, P) + h * h / 12.0 * _poly_eval(_lap(lap), P))
    m = _interior(shape, 1)
    tol = 1e-12 * (abs(L) @ np.abs(p))
    assert np.all(np.abs(got - want)[m] <= tol[m])
    # and the plain 7-point-like reading (no lap^2 term) is wrong for quartics
    wrong = h ** 3 * _poly_eval(lap, P)
    if any(sum(mm) >= 4 for mm, c in poly.items() if c != 0):
        assert np.any(np.abs(got - wrong)[m] > 1e3 * tol[m])


@pytest.mark.parametrize("which", ["13p", "27p"])
def test_plane_waves_are_eigenvectors_on_every_row(which):
    """On a periodic grid every Fourier mode is an eigenvector: the quotient (L v) / v is the
    same on all rows, the wrapped ones included; it is <= 0 and 0 only for the constant."""
    if which == "13p":
        shape, h = (6, 8, 10), (0.3, 0.2, 0.25)
        L = stencil.laplacian_13p(shape, h)
    else:
        shape, h = (5, 6, 8), (0.4, 0.4, 0.4)
        L = stencil.laplacian_27p(shape, 0.4)
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    for a, b, c in ((1, 0, 0), (0, 2, 0), (0, 0, 3), (1, 3, 2), (2, 1, 1)):
        phase = 2 * np.pi * (a * i / nx + b * j / ny + c * k / nz)
        for v in (np.cos(phase), np.sin(phase)):
            Lv = L @ v
            # the pair (cos, sin) spans the mode: L applied to each stays in it with one factor
            big = np.abs(v) > 0.3
            lam = Lv[big] / v[big]
            assert np.all(np.abs(lam - lam[0]) <= 1e-12 * abs(lam[0]))
            assert np.all(np.abs(Lv - lam[0] * v) <= 1e-12 * abs(lam[0]))
            assert lam[0] < 0
    assert np.abs(L @ np.ones(L.shape[0])).max() <= 1e-14 * abs(L).max()


def test_small_grids_rejected():
    with pytest.raises(ValueError):
        stencil.laplacian_13p((4, 6, 6), (1, 1, 1))
    with pytest.raises(ValueError):
        stencil.laplacian_27p((3, 2, 3), 1.0)
