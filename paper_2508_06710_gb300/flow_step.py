"""One time step of the projection method on m stacked flow states: a thin wrapper of the
library's rb_projection_* calls (include/rbspmm.h).

Sec. 3 writes the semi-discrete Navier-Stokes equations (Eq. (ns)) with cell velocities u_c,
face velocities u_s, the convective operator C(u_s) = M U_s Gamma_{c->s}, the diffusive
operator D = -nu L and the cell-to-cell gradient G_c; stacking m independent flow states
(Eq. (ns-nrhs)) turns every operator into I_m (x) A, so each application is one SpMM over
the states' columns, and the convective term is the divergence SpMM of an axty of the face
velocities with the face-interpolated cell velocities.  Sec. 4 integrates in time with
Heun's third-order Runge-Kutta scheme, with a projection at every stage.  The library
sequences all of it (rb_projection_step); this module marshals tensors and parameters.

Layout: u_c is (n, 3 m) with column i m + s for component i of state s; u_s is (n_faces, m),
x faces first, then y, then z.  The grid is uniform and periodic along every axis.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import (GridDesc, Operator, ProjectionParams, ProjectionReport, RB_OK, RB_PROJ_JACOBI, RB_PROJ_MG,
               RB_REFINE_PROLONG, RbError, _check, _grid_desc, _ptr, _stream, cg_params, lib, mg_params,
               refine_assemble)

HEUN3_C = (0.0, 1.0 / 3.0, 2.0 / 3.0)


class ProjectionStep:
    """Heun RK3 projection steps of m flow states on a uniform periodic grid (rb_projection_*).

    nodes: the grid's three float64 CUDA node tensors (uniform spacing, periodic axes).
    solver: "jacobi" (rb_cg_solve: Jacobi-PCG, FP64 or FP32-inner refinement by `mixed`) or
    "mg" (rb_mg_solve: multigrid-preconditioned CG, FP64 or FP32 cycle inside FP64 refinement
    by `mixed`) for the pressure equation.  `iters` collects each solve's iteration count and
    `poisson_ms` their wall time."""

    def __init__(self, torch, nodes, m, nu, dt, rtol=1e-10, mixed=0, solver="jacobi", stream=None):
        self.torch = torch
        self._nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
        shape = [int(n.numel()) - 1 for n in self._nodes]
        self.n = int(np.prod(shape))
        self.nf = 3 * self.n
        self.m, self.nu, self.dt = int(m), float(nu), float(dt)
        self.dev = self._nodes[0].device
        if solver == "mg":
            prm, code = mg_params(rtol=rtol, mixed=bool(mixed)), RB_PROJ_MG
        elif solver == "jacobi":
            prm, code = cg_params(rtol=rtol, mixed=mixed, project_mean=True, check_every=50), RB_PROJ_JACOBI
        else:
            raise ValueError(f"unknown solver {solver!r}")
        g = _grid_desc(self._nodes, [True, True, True])
        h = C.c_void_p()
        _check(lib().rb_projection_create(C.byref(g), C.byref(ProjectionParams(self.m, self.nu, self.dt, code, prm)),
                                          _stream(stream), C.byref(h)), "rb_projection_create")
        self.handle = h
        self.iters = []
        self.poisson_ms = 0.0

    def _blocks(self, u_c, u_s):
        f64 = self.torch.float64
        for name, t, shape in (("u_c", u_c, (self.n, 3 * self.m)), ("u_s", u_s, (self.nf, self.m))):
            if tuple(t.shape) != shape or t.dtype != f64 or t.stride(1) != 1 or not t.is_cuda:
                raise ValueError(f"{name} must be a float64 CUDA block of shape {shape} with contiguous rows")
        return u_c.stride(0), u_s.stride(0)

    def _done(self, st, rep, n_solves, what):
        self.iters.extend(int(v) for v in rep.iters[:n_solves])
        self.poisson_ms += rep.poisson_ms
        if st != RB_OK:
            _check(st, what)

    def step(self, u_c, u_s, stream=None):
        """One Heun RK3 step; u_c (n, 3 m) and u_s (n_faces, m) are updated in place."""
        ldu, lds = self._blocks(u_c, u_s)
        rep = ProjectionReport()
        st = lib().rb_projection_step(self.handle, _ptr(u_c), ldu, _ptr(u_s), lds, C.byref(rep), _stream(stream))
        self._done(st, rep, 3, "rb_projection_step")

    def project(self, u_c, cdt, u_s=None, stream=None):
        """One projection with time cdt: u_c (n, 3 m) in place; returns the face velocities."""
        if u_s is None:
            u_s = self.torch.empty((self.nf, self.m), dtype=self.torch.float64, device=self.dev)
        ldu, lds = self._blocks(u_c, u_s)
        rep = ProjectionReport()
        st = lib().rb_projection_project(self.handle, float(cdt), _ptr(u_c), ldu, _ptr(u_s), lds, C.byref(rep),
                                         _stream(stream))
        self._done(st, rep, 1, "rb_projection_project")
        return u_s

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().rb_projection_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


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
        us = self.fine.project(u, self.fine.dt)
        return u, us

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
