"""One time step of the projection method on m flow states at once (FP64).

Sec. 3 writes the semi-discrete equations (Eq. (ns)) for a cell-centred velocity u_c with
face velocities u_s = Gamma_{c->s} u_c, the convective operator C(u_s) = M U_s Gamma_{c->s},
the diffusive operator D and the cell-to-cell gradient G_c; Sec. 3.1 stacks m independent
flow states, which share every operator (Eq. (ns-nrhs)): the convective term becomes the
divergence SpMM applied to the axty of the face velocities and the face-interpolated cell
velocities.  Sec. 4 integrates in time with Heun's third-order Runge-Kutta scheme, applied
with a projection at every stage (Sanderse and Koren's formulation).

Readings used here (the paper gives the operators' roles, not these details):
  * uniform periodic grids: the cell volume Omega is one number and the face-to-cell
    interpolator is the transpose of the cell-to-face one, Gamma_{s->c} = Gamma_{c->s}^T
    (Omega^{-1} Gamma^T Omega_s with Omega_s = Omega);
  * D = -nu L with the volume-integrated Laplacian L = M G;
  * G_c p, component d: Gamma_{s->c} applied to G p kept on the faces of direction d only;
  * the state is (u_c, u_s): u_s, the face velocity left by the last projection (divergence
    free), is the one the convective operator uses; a projection takes the predicted cell
    velocity u~, interpolates its face-normal components u~_s, solves L p = M u~_s / (c dt)
    (A = -L, zero-mean p) and sets u_s = u~_s - c dt G p, u_c = u~ - c dt G_c p;
  * Heun's third-order scheme: c = (0, 1/3, 2/3), a21 = 1/3, a31 = 0, a32 = 2/3,
    b = (1/4, 0, 3/4); stage derivatives F = Omega^{-1} (nu L u_c - C(u_s) u_c), the pressure
    entering through the projections.

Layout: u_c is (n, 3 m) with column i m + s for component i of state s; u_s is (n_faces, m).

Test infrastructure only; see the package docstring.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from . import cg as ocg
from . import fvm, refine

HEUN3_C = (0.0, 1.0 / 3.0, 2.0 / 3.0)
HEUN3_A = ((), (1.0 / 3.0,), (0.0, 2.0 / 3.0))
HEUN3_B = (0.25, 0.0, 0.75)


@dataclasses.dataclass
class Operators:
    M: sp.csr_matrix
    G: sp.csr_matrix
    L: sp.csr_matrix
    I: sp.csr_matrix  # Gamma_{c->s}
    blocks: list  # (first face, count) per direction
    vol: float


def operators(grid) -> Operators:
    for a in grid.axes:
        w = np.diff(a.nodes)
        if not a.periodic or np.ptp(w) > 1e-12 * w.max():
            raise ValueError("the projection step takes uniform periodic grids")
    M, G = fvm.divergence(grid), fvm.gradient(grid)
    vol = float(np.prod([a.nodes[1] - a.nodes[0] for a in grid.axes]))
    return Operators(M, G, fvm.laplacian(grid), fvm.interpolation(grid), fvm.face_blocks(grid), vol)


def convection(ops: Operators, u_c: np.ndarray, u_s: np.ndarray) -> np.ndarray:
    """C(u_s) u_c for every component and state: M (u_s * Gamma u_c)."""
    m = u_s.shape[1]
    Y = ops.I @ u_c
    for i in range(3):
        Y[:, i * m:(i + 1) * m] *= u_s
    return ops.M @ Y


def derivative(ops: Operators, u_c, u_s, nu):
    return (nu * (ops.L @ u_c) - convection(ops, u_c, u_s)) / ops.vol


def normal_faces(ops: Operators, u_c: np.ndarray, m: int) -> np.ndarray:
    """Face-normal components of Gamma u_c: direction d's faces take component d."""
    Y = ops.I @ u_c
    u_s = np.zeros((ops.I.shape[0], m))
    for d, (f0, nd) in enumerate(ops.blocks):
        u_s[f0:f0 + nd] = Y[f0:f0 + nd, d * m:(d + 1) * m]
    return u_s


def project(ops: Operators, u_t: np.ndarray, cdt: float, p0=None, rtol: float = 1e-12):
    """Projection of the predicted cell velocity u_t with time step cdt."""
    m = u_t.shape[1] // 3
    ut_s = normal_faces(ops, u_t, m)
    A = (-ops.L).tocsr()
    b = -(ops.M @ ut_s) / cdt  # A p = -M u~_s / cdt, i.e. L p = M u~_s / cdt
    p, _ = ocg.pcg_columns(A, b, p0, rtol=rtol, project_mean=True)
    g = ops.G @ p
    u_s = ut_s - cdt * g
    gm = np.zeros((g.shape[0], 3 * m))
    for d, (f0, nd) in enumerate(ops.blocks):
        gm[f0:f0 + nd, d * m:(d + 1) * m] = g[f0:f0 + nd]
    u_c = u_t - cdt * (ops.I.T @ gm)
    return u_c, u_s, p


def heun3_step(ops: Operators, u_c: np.ndarray, u_s: np.ndarray, dt: float, nu: float, rtol: float = 1e-12):
    """One Heun RK3 step with a projection at every stage; returns (u_c, u_s, p of the last projection)."""
    F = []
    uc_i, us_i = u_c, u_s
    p = None
    for i in range(3):
        if i > 0:
            ut = u_c + dt * sum(a * f for a, f in zip(HEUN3_A[i], F))
            uc_i, us_i, p = project(ops, ut, HEUN3_C[i] * dt, rtol=rtol)
        F.append(derivative(ops, uc_i, us_i, nu))
    ut = u_c + dt * sum(b * f for b, f in zip(HEUN3_B, F))
    return project(ops, ut, dt, rtol=rtol)


def taylor_green(grid, m: int = 1, amp=None) -> np.ndarray:
    """The 2-D Taylor-Green vortex u = a sin x cos y, v = -a cos x sin y (w = 0) at the cell
    centres of a 2 pi periodic box, one amplitude per state: (n, 3 m)."""
    c = [0.5 * (a.nodes[:-1] + a.nodes[1:]) for a in grid.axes]
    z, y, x = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    amp = np.ones(m) if amp is None else np.asarray(amp, dtype=np.float64)
    u = np.zeros((grid.n_cells, 3 * m))
    for s in range(m):
        u[:, s] = amp[s] * (np.sin(x) * np.cos(y)).ravel()
        u[:, m + s] = -amp[s] * (np.cos(x) * np.sin(y)).ravel()
    return u


def map_to_fine(fine_grid, u_c_coarse: np.ndarray, dt: float, rtol: float = 1e-12):
    """Inline mesh refinement's mapping (Sec. 3.3): the coarse cell velocities of every state
    interpolated onto the fine cells by the trilinear prolongation P of ``refine`` (each
    component column alike), then projected on the fine grid, so that the fine state starts
    from divergence-free face velocities and the matching cell velocities.  Returns the fine
    (u_c, u_s)."""
    P = refine.prolongation(fine_grid)
    ops = operators(fine_grid)
    u_c, u_s, _ = project(ops, P @ u_c_coarse, dt, rtol=rtol)
    return u_c, u_s


def refined_run(fine_grid, u_c, u_s, nu: float, dt_coarse: float, dt_fine: float, steps_coarse: int,
                steps_fine: int, rtol: float = 1e-12):
    """The time-split of Sec. 3.3 on m stacked states: `steps_coarse` Heun RK3 steps on the
    2:1 coarser grid (u_c, u_s given there), the mapping onto ``fine_grid``, then `steps_fine`
    steps on it.  Returns the fine (u_c, u_s)."""
    coarse = refine.coarse_grid(fine_grid)
    ops_c = operators(coarse)
    for _ in range(steps_coarse):
        u_c, u_s, _ = heun3_step(ops_c, u_c, u_s, dt_coarse, nu, rtol=rtol)
    u_c, u_s = map_to_fine(fine_grid, u_c, dt_fine, rtol=rtol)
    ops_f = operators(fine_grid)
    for _ in range(steps_fine):
        u_c, u_s, _ = heun3_step(ops_f, u_c, u_s, dt_fine, nu, rtol=rtol)
    return u_c, u_s
