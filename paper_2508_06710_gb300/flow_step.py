"""One time step of the projection method on m stacked flow states, driven through the C ABI.

Sec. 3 writes the semi-discrete Navier-Stokes equations (Eq. (ns)) with cell velocities u_c,
face velocities u_s, the convective operator C(u_s) = M U_s Gamma_{c->s}, the diffusive
operator D = -nu L and the cell-to-cell gradient G_c; stacking m independent flow states
(Eq. (ns-nrhs)) turns every operator into I_m (x) A, so each application is one SpMM over
the states' columns, and the convective term is the divergence SpMM of an axty of the face
velocities with the face-interpolated cell velocities.  Sec. 4 integrates in time with
Heun's third-order Runge-Kutta scheme, with a projection at every stage.

Every arithmetic step runs in the library's kernels (SpMM with per-column scales, axpy,
axty, the Poisson solve by Jacobi- or multigrid-preconditioned CG); this module allocates the
buffers, zero-fills and copies
them, and takes row and column views (the face blocks of each direction, the columns of each
velocity component).  Layout: u_c is (n, 3 m) with column i m + s for component i of state
s; u_s is (n_faces, m), x faces first, then y, then z.

The grid is uniform and periodic along every axis (so the cell volume is one number and the
face-to-cell interpolator is the transpose of the cell-to-face one).  A projection takes the
predicted cell velocity u~, interpolates its face-normal components u~_s, solves
-L p = -M u~_s / (c dt) with zero-mean p, and sets u_s = u~_s - c dt G p and
u_c = u~ - c dt G_c p, G_c p's component d being Gamma_{s->c} applied to G p on the faces of
direction d.
"""
from __future__ import annotations

import time

import numpy as np

from . import (Multigrid, Operator, RbError, axpy, axty, cg_params, cg_solve, cg_workspace_bytes, fvm_assemble,
               mg_params, refine_assemble, RB_FVM_DIVERGENCE, RB_FVM_GRADIENT, RB_FVM_INTERP_C2S, RB_FVM_INTERP_S2C,
               RB_FVM_LAPLACIAN, RB_OK, RB_REFINE_PROLONG)

HEUN3_C = (0.0, 1.0 / 3.0, 2.0 / 3.0)
HEUN3_A = ((), (1.0 / 3.0,), (0.0, 2.0 / 3.0))
HEUN3_B = (0.25, 0.0, 0.75)


class ProjectionStep:
    """Heun RK3 projection steps of m flow states on a uniform periodic grid.

    nodes: the grid's three float64 CUDA node tensors (uniform spacing, periodic axes).
    solver: "jacobi" (rb_cg_solve: Jacobi-PCG, FP64 or FP32-inner refinement by `mixed`) or
    "mg" (rb_mg_solve: multigrid-preconditioned CG, FP64 or FP32 cycle inside FP64 refinement
    by `mixed`) for the pressure equation."""

    def __init__(self, torch, nodes, m, nu, dt, rtol=1e-10, mixed=0, solver="jacobi"):
        self.torch = torch
        nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
        host = [n.cpu().numpy() for n in nodes]
        for a in host:
            w = np.diff(a)
            if np.ptp(w) > 1e-12 * np.max(w):
                raise ValueError("the projection step takes uniform grids")
        per = [True, True, True]
        shape = [len(a) - 1 for a in host]
        self.n = int(np.prod(shape))
        self.vol = float(np.prod([a[1] - a[0] for a in host]))
        self.m, self.nu, self.dt = int(m), float(nu), float(dt)
        m3 = 3 * self.m
        dev = nodes[0].device
        self.dev = dev

        def op(kind, k, scale=1.0, dtype="f64"):
            rp, ci, va, nc = fvm_assemble(nodes, per, kind, scale=scale)
            return Operator(rp, ci, va, nc, dtype=dtype, k_max=k)

        self.M = op(RB_FVM_DIVERGENCE, m3)      # divergence (convective term and projection)
        self.G = op(RB_FVM_GRADIENT, self.m)    # cell-to-face gradient of the pressure
        self.L = op(RB_FVM_LAPLACIAN, m3)       # diffusion
        self.A = op(RB_FVM_LAPLACIAN, self.m, scale=-1.0)  # Poisson matrix -L
        self.A32 = op(RB_FVM_LAPLACIAN, self.m, scale=-1.0, dtype="f32") if mixed and solver == "jacobi" else None
        self.I = op(RB_FVM_INTERP_C2S, m3)      # Gamma_{c->s}
        self.IT = op(RB_FVM_INTERP_S2C, m3)     # Gamma_{s->c} = Gamma_{c->s}^T
        self.nf = self.I.n_rows
        # faces of each direction: periodic axes have n faces per direction
        self.blocks = [(d * self.n, self.n) for d in range(3)]
        f64 = dict(dtype=torch.float64, device=dev)
        if solver == "mg":
            self.mg = Multigrid(nodes, per, k_max=self.m)
            self.prm = mg_params(rtol=rtol, mixed=bool(mixed))
            self.work = None
        elif solver == "jacobi":
            self.mg = None
            self.prm = cg_params(rtol=rtol, mixed=mixed, project_mean=True, check_every=50)
            self.work = torch.empty(cg_workspace_bytes(self.A, self.m, self.prm), dtype=torch.uint8, device=dev)
        else:
            raise ValueError(f"unknown solver {solver!r}")
        self.Y = torch.empty((self.nf, m3), **f64)      # Gamma u, then u_s * Gamma u
        self.Gm = torch.empty((self.nf, m3), **f64)     # G p on each direction's faces, by component
        self.ut_s = torch.empty((self.nf, self.m), **f64)
        self.g = torch.empty((self.nf, self.m), **f64)
        self.B = torch.empty((self.n, self.m), **f64)
        self.P = [torch.zeros((self.n, self.m), **f64) for _ in range(3)]  # one pressure per projection
        self.F = [torch.empty((self.n, m3), **f64) for _ in range(3)]
        self.ut = torch.empty((self.n, m3), **f64)
        self.tmp = torch.empty((self.n, m3), **f64)
        self.us_stage = torch.empty((self.nf, self.m), **f64)

        def col(v, k):
            return torch.full((k,), float(v), **f64)

        self.one_m, self.one_m3 = col(1.0, self.m), col(1.0, m3)
        self.c_diff = col(self.nu / self.vol, m3)
        self.c_conv = col(-1.0 / self.vol, m3)
        self.coef = {}  # alpha arrays of the stage combinations and projections, by value
        self.iters = []
        self.poisson_ms = 0.0

    def _alpha(self, v, k):
        key = (float(v), k)
        if key not in self.coef:
            self.coef[key] = self.torch.full((k,), float(v), dtype=self.torch.float64, device=self.dev)
        return self.coef[key]

    def _cols(self, X, i):
        return X[:, i * self.m:(i + 1) * self.m]

    def derivative(self, u, us, F):
        """F = Omega^{-1} (nu L u - M (u_s * Gamma u)) for every component and state."""
        self.I.spmm(u, self.Y)
        for i in range(3):
            axty(1.0, us, self._cols(self.Y, i))
        self.M.spmm(self.Y, self.tmp, c=self.c_conv)
        self.L.spmm(u, F, c=self.c_diff)
        axpy(self.one_m3, self.tmp, F)

    def project(self, ut, cdt, slot):
        """In place: ut becomes u_c; returns u_s (self.ut_s) after the projection with time cdt."""
        self.I.spmm(ut, self.Y)
        self.ut_s.zero_()
        for d, (f0, nd) in enumerate(self.blocks):
            axpy(self.one_m, self._cols(self.Y, d)[f0:f0 + nd], self.ut_s[f0:f0 + nd])
        self.M.spmm(self.ut_s, self.B, c=self._alpha(-1.0 / cdt, self.m))
        t0 = time.perf_counter()
        if self.mg is not None:
            res = self.mg.solve(self.B, self.P[slot], self.prm)
        else:
            res = cg_solve(self.A, self.B, self.P[slot], A_inner=self.A32, params=self.prm, work=self.work)
        self.poisson_ms += (time.perf_counter() - t0) * 1e3
        if res.status != RB_OK:
            raise RbError(res.status, f"projection solve: {res}")
        self.iters.append(max(res.iters))
        self.G.spmm(self.P[slot], self.g)
        axpy(self._alpha(-cdt, self.m), self.g, self.ut_s)
        self.Gm.zero_()
        for d, (f0, nd) in enumerate(self.blocks):
            axpy(self.one_m, self.g[f0:f0 + nd], self._cols(self.Gm, d)[f0:f0 + nd])
        self.IT.spmm(self.Gm, self.tmp)
        axpy(self._alpha(-cdt, 3 * self.m), self.tmp, ut)
        return self.ut_s

    def _combine(self, u, coeffs):
        """self.ut = u + dt sum_j coeffs[j] F_j."""
        self.ut.copy_(u)
        for a, F in zip(coeffs, self.F):
            if a != 0.0:
                axpy(self._alpha(self.dt * a, 3 * self.m), F, self.ut)

    def step(self, u_c, u_s):
        """One Heun RK3 step; u_c (n, 3 m) and u_s (n_faces, m) are updated in place."""
        f64 = self.torch.float64
        for name, t, shape in (("u_c", u_c, (self.n, 3 * self.m)), ("u_s", u_s, (self.nf, self.m))):
            if tuple(t.shape) != shape or t.dtype != f64 or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous float64 tensor of shape {shape}")
        self.derivative(u_c, u_s, self.F[0])
        for i in (1, 2):
            self._combine(u_c, HEUN3_A[i])
            us_i = self.project(self.ut, HEUN3_C[i] * self.dt, i - 1)
            self.us_stage.copy_(us_i)
            self.derivative(self.ut, self.us_stage, self.F[i])
        self._combine(u_c, HEUN3_B)
        us = self.project(self.ut, self.dt, 2)
        u_c.copy_(self.ut)
        u_s.copy_(us)


class RefinedEnsemble:
    """Inline mesh refinement (Sec. 3.3) of m stacked flow states: the states develop on the
    2:1 coarser grid (every other node of `fine_nodes`, larger time step), are mapped onto the
    fine grid, and continue there.  The mapping interpolates every component of the coarse
    cell velocities with the trilinear prolongation P (one rectangular SpMM over the 3 m
    columns) and projects the result on the fine grid, so that the fine states start from
    divergence-free face velocities and the matching cell velocities.

    Both grids are uniform and periodic (ProjectionStep's requirement); each keeps its own
    operators and Poisson solver."""

    def __init__(self, torch, fine_nodes, m, nu, dt_fine, dt_coarse=None, rtol=1e-10, mixed=2, solver="mg"):
        self.torch = torch
        fine_nodes = [n.to(dtype=torch.float64).contiguous() for n in fine_nodes]
        coarse_nodes = [n[::2].contiguous() for n in fine_nodes]  # every other node
        self.m = int(m)
        self.coarse = ProjectionStep(torch, coarse_nodes, m, nu, 2.0 * dt_fine if dt_coarse is None else dt_coarse,
                                     rtol=rtol, mixed=mixed, solver=solver)
        self.fine = ProjectionStep(torch, fine_nodes, m, nu, dt_fine, rtol=rtol, mixed=mixed, solver=solver)
        rp, ci, va, nc = refine_assemble(fine_nodes, [True, True, True], RB_REFINE_PROLONG)
        self.P = Operator(rp, ci, va, nc, k_max=3 * self.m)

    def map_to_fine(self, u_c_coarse):
        """(u_c, u_s) on the fine grid from the coarse cell velocities (n_coarse, 3 m)."""
        torch = self.torch
        u = torch.empty((self.fine.n, 3 * self.m), dtype=torch.float64, device=self.fine.dev)
        self.P.spmm(u_c_coarse, u)
        us = self.fine.project(u, self.fine.dt, 2)
        return u, us.clone()

    def run(self, u_c, u_s, steps_coarse, steps_fine):
        """`steps_coarse` steps of the coarse states (u_c, u_s given on the coarse grid, updated
        in place), the mapping, `steps_fine` steps on the fine grid; returns the fine (u_c, u_s)
        and the wall time of each phase in ms (synchronised)."""
        torch = self.torch
        t = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps_coarse):
            self.coarse.step(u_c, u_s)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        uf, usf = self.map_to_fine(u_c)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for _ in range(steps_fine):
            self.fine.step(uf, usf)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        t["coarse_ms"], t["map_ms"], t["fine_ms"] = (t1 - t0) * 1e3, (t2 - t1) * 1e3, (t3 - t2) * 1e3
        return uf, usf, t
