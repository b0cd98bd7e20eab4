"""Pins of the projection-step oracle (Eq. (ns) on m states, Heun RK3; Sec. 3 and Sec. 4)
against the mathematics rather than its own code: the symmetric part of the convective
operator M U_s Gamma is diag(M u_s), so it is skew-symmetric for divergence-free face
velocities (the symmetry-preserving property); every projection leaves M u_s = 0; the
Taylor-Green vortex, an exact solution of the Navier-Stokes equations, is reproduced with an
error that falls at least 4x per halving of h; m stacked states equal m separate runs."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import flow, fvm


def _box(n, L=2 * math.pi):
    return W.Grid((W.uniform_axis(n, L), W.uniform_axis(n, L), W.uniform_axis(n, L)))


def test_interpolation_is_the_face_mean():
    g = W.channel_grid(6, 5, 4)
    I, G = fvm.interpolation(g), fvm.gradient(g)
    assert np.array_equal((I != 0).toarray(), (G != 0).toarray())
    assert np.all(I.data == 0.5)
    assert np.allclose(I @ np.ones(g.n_cells), 1.0)
    blocks = fvm.face_blocks(g)
    assert blocks[-1][0] + blocks[-1][1] == fvm.n_faces(g)


def test_convective_operator_symmetric_part():
    """C + C^T = diag(M u_s) for any face field; skew-symmetric once M u_s = 0."""
    g = _box(6, 1.0)
    ops = flow.operators(g)
    us = W.normal((fvm.n_faces(g), 1), 11)[:, 0]
    C = (ops.M @ sp.diags(us) @ ops.I).toarray()
    assert np.abs(C + C.T - np.diag(ops.M @ us)).max() <= 1e-14 * np.abs(C).max()
    u = W.normal((g.n_cells, 3), 12)
    _, us_p, _ = flow.project(ops, u, 0.5)
    Cp = (ops.M @ sp.diags(us_p[:, 0]) @ ops.I).toarray()
    assert np.abs(Cp + Cp.T).max() <= 1e-10 * np.abs(Cp).max()
    # hence u . C u = 0: no energy from convection
    assert abs(u[:, 0] @ (Cp @ u[:, 0])) <= 1e-10 * np.abs(Cp).max() * (u[:, 0] @ u[:, 0])


@pytest.mark.parametrize("cdt", [1.0, 0.01])
def test_projection_leaves_divergence_free_faces(cdt):
    g = _box(7, 1.0)
    ops = flow.operators(g)
    u = W.normal((g.n_cells, 6), 13)
    uc, us, p = flow.project(ops, u, cdt)
    assert us.shape == (fvm.n_faces(g), 2)
    scale = (abs(ops.M) @ np.abs(us)).max()
    assert np.abs(ops.M @ us).max() <= 1e-10 * scale
    assert np.abs(p.mean(axis=0)).max() <= 1e-12 * np.abs(p).max()


def test_taylor_green_second_order():
    """u = sin x cos y e^{-2 nu t}, v = -cos x sin y e^{-2 nu t} on the 2 pi box, to t = 0.4."""
    nu, T = 0.1, 0.4
    errs = []
    for n in (8, 16):
        g = _box(n)
        ops = flow.operators(g)
        u0 = flow.taylor_green(g, 1)
        u, us, _ = flow.project(ops, u0, 1.0)
        dt = 0.05 * 8 / n
        steps = int(round(T / dt))
        for _ in range(steps):
            u, us, _ = flow.heun3_step(ops, u, us, dt, nu)
        errs.append(np.abs(u - u0 * math.exp(-2 * nu * steps * dt)).max())
        assert np.abs(ops.M @ us).max() <= 1e-9
    assert errs[1] < 3e-3 and errs[0] / errs[1] >= 4.0, errs


@pytest.mark.parametrize("U,k", [(1.0, 1), (-0.7, 2)])
def test_advected_wave_matches_rk3_amplification(U, k):
    """A transverse wave v = eps sin(k x) carried by a uniform stream u = U stays divergence
    free, so the projections change nothing and convection drives the evolution: each step
    multiplies the Fourier mode by R(lam dt), R(z) = 1 + z + z^2/2 + z^3/6 (any third-order
    three-stage Runge-Kutta scheme), lam = -i U sin(k h)/h - nu (2 - 2 cos(k h))/h^2 (central
    convection, three-point diffusion).  Sensitive to the sign of convection and to the
    scheme's weights, which the Taylor-Green vortex (a gradient convective term) is not."""
    n, nu, dt, steps, eps = 16, 0.05, 0.1, 5, 0.3
    g = W.Grid((W.uniform_axis(n, 2 * math.pi), W.uniform_axis(4, 1.0), W.uniform_axis(4, 1.0)))
    ops = flow.operators(g)
    h = 2 * math.pi / n
    x = np.tile(0.5 * h + h * np.arange(n), 16)
    u = np.zeros((g.n_cells, 3))
    u[:, 0] = U
    u[:, 1] = eps * np.sin(k * x)
    us = flow.normal_faces(ops, u, 1)
    for _ in range(steps):
        u, us, _ = flow.heun3_step(ops, u, us, dt, nu)
    lam = -1j * U * math.sin(k * h) / h - nu * (2 - 2 * math.cos(k * h)) / h ** 2
    z = lam * dt
    amp = (1 + z + z * z / 2 + z ** 3 / 6) ** steps
    want = eps * np.imag(amp * np.exp(1j * k * x))
    assert np.abs(u[:, 1] - want).max() <= 1e-9
    assert np.abs(u[:, 0] - U).max() <= 1e-9 and np.abs(u[:, 2]).max() <= 1e-9


def test_states_are_independent():
    """Two stacked states step exactly as two separate runs (every operator is I_m (x) A)."""
    g = _box(6, 1.0)
    ops = flow.operators(g)
    m = 2
    u = W.normal((g.n_cells, 3 * m), 14)
    us = W.normal((fvm.n_faces(g), m), 15)
    U, US, P = flow.heun3_step(ops, u, us, 0.01, 0.05)
    for s in range(m):
        cols = [i * m + s for i in range(3)]
        u1, us1, p1 = flow.heun3_step(ops, u[:, cols], us[:, [s]], 0.01, 0.05)
        assert np.allclose(U[:, cols], u1, rtol=0, atol=1e-13)
        assert np.allclose(US[:, [s]], us1, rtol=0, atol=1e-13)


def test_nonuniform_or_walled_grids_rejected():
    with pytest.raises(ValueError):
        flow.operators(W.channel_grid(6, 6, 6))


def test_mapping_keeps_uniform_streams_and_is_divergence_free():
    """A uniform stream is trilinear, so P reproduces it and the projection leaves it alone;
    a random coarse field maps to divergence-free fine faces."""
    fine = _box(8, 1.0)
    coarse = W.Grid(tuple(W.uniform_axis(4, 1.0) for _ in range(3)))
    m = 2
    u = np.zeros((coarse.n_cells, 3 * m))
    u[:, 0], u[:, 1], u[:, 2 * m + 1] = 0.7, -1.3, 2.1
    uf, usf = flow.map_to_fine(fine, u, 0.1)
    assert np.abs(uf - np.tile(u[:1], (fine.n_cells, 1))).max() <= 1e-12
    ops = flow.operators(fine)
    uf, usf = flow.map_to_fine(fine, W.normal((coarse.n_cells, 3 * m), 16), 0.1)
    scale = (abs(ops.M) @ np.abs(usf)).max()
    assert np.abs(ops.M @ usf).max() <= 1e-10 * scale


def test_refined_run_is_second_order():
    """Taylor-Green run on a coarse box to t = 0.2, mapped onto the 2:1 finer box and run to
    t = 0.4 there: the error against the exact decay (dominated by the trilinear mapping, an
    O(h^2) interpolation) falls at least 3x when both boxes are refined, and the final face
    velocities are divergence free."""
    nu = 0.1
    errs = []
    for nc in (8, 16):
        fine, coarse = _box(2 * nc), _box(nc)
        ops_c = flow.operators(coarse)
        uc, usc, _ = flow.project(ops_c, flow.taylor_green(coarse, 1), 1.0)
        dtc = 0.05 * 8 / nc
        uf, usf = flow.refined_run(fine, uc, usc, nu, dtc, dtc / 2, 4, 8)
        t = 4 * dtc + 8 * dtc / 2
        errs.append(np.abs(uf - flow.taylor_green(fine, 1) * math.exp(-2 * nu * t)).max())
        assert np.abs(flow.operators(fine).M @ usf).max() <= 1e-9
    assert errs[0] / errs[1] >= 3.0, errs
