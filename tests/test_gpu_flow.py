"""The projection step on m flow states (Eq. (ns), Heun RK3 with per-stage projections; Secs.
3, 4) sequenced from library calls, against the oracle's step (GPU); and the two
interpolator kinds of the device FVM build.

Bar: the interpolators' CSR bit-exact (every value is 1/2 times the scale); the step within
1e-8 of the largest velocity after one step and 1e-7 after four (the Poisson solves stop at
a 1e-10 relative residual on the device and 1e-12 in the oracle, from different initial
guesses); face velocities divergence free to the solver's tolerance.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import flow, fvm
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("grid", ["channel-9x6x5", "periodic-6^3"])
@pytest.mark.parametrize("scale", [1.0, -2.0])
def test_interpolator_kinds_match_oracle(rb, grid, scale):
    g = W.channel_grid(9, 6, 5) if grid.startswith("channel") else W.unit_periodic_grid(6)
    nodes, per = rb.grid_nodes(g)
    I = fvm.interpolation(g) * scale
    for kind, A in ((rb.RB_FVM_INTERP_C2S, I.tocsr()), (rb.RB_FVM_INTERP_S2C, I.T.tocsr())):
        A.sort_indices()
        assert rb.fvm_csr_size(nodes, per, kind) == (A.shape[0], A.shape[1], A.nnz)
        rp, ci, va, nc = rb.fvm_assemble(nodes, per, kind, scale=scale)
        assert nc == A.shape[1]
        assert np.array_equal(rp.cpu().numpy(), A.indptr)
        assert np.array_equal(ci.cpu().numpy(), A.indices)
        assert np.array_equal(va.cpu().numpy(), A.data)


def _box(shape, lengths):
    return W.Grid(tuple(W.uniform_axis(n, L) for n, L in zip(shape, lengths)))


@pytest.mark.parametrize("mixed,solver", [(0, "jacobi"), (2, "jacobi"), (0, "mg"), (2, "mg")])
def test_projection_step_matches_oracle(rb, mixed, solver):
    from paper_2508_06710_gb300.flow_step import ProjectionStep

    g = _box((10, 12, 8), (2 * math.pi, 3.0, 2.5))
    ops = flow.operators(g)
    m, nu, dt = 2, 0.05, 0.01
    u = 0.5 * W.normal((g.n_cells, 3 * m), 1700) + flow.taylor_green(g, m, amp=[1.0, 0.7])
    us = W.normal((fvm.n_faces(g), m), 1701)
    nodes, _ = rb.grid_nodes(g)
    stepper = ProjectionStep(torch, nodes, m, nu, dt, mixed=mixed, solver=solver)
    ud, usd = to_dev(u), to_dev(us)
    scale = np.abs(u).max()
    for s in range(4):
        stepper.step(ud, usd)
        u, us, _ = flow.heun3_step(ops, u, us, dt, nu)
        tol = (1e-8 if s == 0 else 1e-7) * scale
        assert np.abs(ud.cpu().numpy() - u).max() <= tol
        assert np.abs(usd.cpu().numpy() - us).max() <= tol
        U = usd.cpu().numpy()
        assert np.abs(ops.M @ U).max() <= 1e-8 * (abs(ops.M) @ np.abs(U)).max()


def test_projection_step_full_size(rb):
    """The bench's 128^3 periodic 2 pi box, two states (Taylor-Green of amplitude 1 and 0.5 plus
    seeded noise of 0.01): two steps; the faces' divergence against that of the unprojected
    interpolated field; state 1 against a single-state run of the same field; the vortex's
    decay within the noise."""
    from paper_2508_06710_gb300.flow_step import ProjectionStep

    n, nu, dt = 128, 0.01, 0.01
    g = _box((n, n, n), (2 * math.pi,) * 3)
    nodes, _ = rb.grid_nodes(g)
    tg = flow.taylor_green(g, 2, amp=[1.0, 0.5])
    u0 = tg + 0.01 * W.normal(tg.shape, 1800)
    stepper = ProjectionStep(torch, nodes, 2, nu, dt, mixed=2)
    ud = to_dev(u0)
    usd = torch.zeros((3 * g.n_cells, 2), dtype=torch.float64, device="cuda")
    per = [True, True, True]
    I = rb.Operator(*rb.fvm_assemble(nodes, per, rb.RB_FVM_INTERP_C2S), k_max=6)
    M = rb.Operator(*rb.fvm_assemble(nodes, per, rb.RB_FVM_DIVERGENCE), k_max=2)
    # divergence of the face-normal interpolation of u0, before any projection
    Y = I.spmm(ud)
    us0 = torch.cat([Y[d * g.n_cells:(d + 1) * g.n_cells, 2 * d:2 * d + 2] for d in range(3)])
    d0 = M.spmm(us0.contiguous()).abs().max().item()
    stepper.step(ud, usd)
    stepper.step(ud, usd)
    assert len(stepper.iters) == 6 and stepper.poisson_ms > 0.0
    div = M.spmm(usd).abs().max().item()
    assert div <= 1e-6 * d0, (div, d0)  # ||r||_2 <= 1e-10 ||b||_2 bounds the max-norm by ~1.5e-7 ||b||_max
    single = ProjectionStep(torch, nodes, 1, nu, dt, mixed=2)
    u1 = to_dev(u0[:, [1, 3, 5]])
    us1 = torch.zeros((3 * g.n_cells, 1), dtype=torch.float64, device="cuda")
    single.step(u1, us1)
    single.step(u1, us1)
    diff = (ud[:, [1, 3, 5]] - u1).abs().max().item()
    assert diff <= 1e-8, diff
    decay = math.exp(-2 * nu * 2 * dt)
    err = (ud - to_dev(tg) * decay).abs().max().item()
    assert err <= 0.05, err


@pytest.mark.parametrize("mixed", [0, 2])
def test_refined_run_matches_oracle(rb, mixed):
    """Inline mesh refinement (Sec. 3.3): two steps of two states on the 8^3 box, the mapping
    (trilinear P, then a projection) onto 16^3, two steps there; against the oracle's run.
    Bar as for the step (the solves stop at 1e-10 on the device, 1e-12 in the oracle)."""
    from paper_2508_06710_gb300.flow_step import RefinedEnsemble

    fine = _box((16, 16, 16), (2 * math.pi,) * 3)
    coarse = _box((8, 8, 8), (2 * math.pi,) * 3)
    m, nu, dtf = 2, 0.05, 0.02
    u = flow.taylor_green(coarse, m, amp=[1.0, 0.6]) + 0.2 * W.normal((coarse.n_cells, 3 * m), 1900)
    ops_c = flow.operators(coarse)
    u, us, _ = flow.project(ops_c, u, 1.0)
    nodes, _ = rb.grid_nodes(fine)
    run = RefinedEnsemble(torch, nodes, m, nu, dtf, mixed=mixed)
    ud, usd = to_dev(u), to_dev(us)
    uf, usf, t = run.run(ud, usd, 2, 2)
    ur, usr = flow.refined_run(fine, u, us, nu, 2 * dtf, dtf, 2, 2)
    scale = np.abs(u).max()
    assert np.abs(uf.cpu().numpy() - ur).max() <= 1e-7 * scale
    assert np.abs(usf.cpu().numpy() - usr).max() <= 1e-7 * scale
    ops_f = flow.operators(fine)
    U = usf.cpu().numpy()
    assert np.abs(ops_f.M @ U).max() <= 1e-8 * (abs(ops_f.M) @ np.abs(U)).max()
    assert set(t) == {"coarse_ms", "map_ms", "fine_ms"}
    # the mapping alone: P (one SpMM over the 3 m columns) and the fine projection
    uc_map, us_map = run.map_to_fine(to_dev(u))
    ur_map, usr_map = flow.map_to_fine(fine, u, dtf)
    assert np.abs(uc_map.cpu().numpy() - ur_map).max() <= 1e-8 * scale
    assert np.abs(us_map.cpu().numpy() - usr_map).max() <= 1e-8 * scale


def test_projection_abi_strided_and_refusals(rb):
    """rb_projection_step on u_c and u_s held inside wider blocks (ld > 3 m, ld > m) gives the
    contiguous call's result and leaves the other columns alone; a non-uniform or walled grid,
    a wrong shape and overlapping blocks are refused."""
    from paper_2508_06710_gb300.flow_step import ProjectionStep

    g = _box((8, 8, 16), (2 * math.pi, 2.0, 3.0))
    nodes, _ = rb.grid_nodes(g)
    m = 2
    with pytest.raises(rb.RbError) as e:  # 6 and 10 cells do not halve: no multigrid hierarchy
        ProjectionStep(torch, rb.grid_nodes(_box((8, 6, 10), (1.0, 1.0, 1.0)))[0], m, 0.02, 0.01, solver="mg")
    assert e.value.status == rb.RB_EINVAL and "coarsen" in str(e.value)
    u = flow.taylor_green(g, m, amp=[1.0, 0.5]) + 0.1 * W.normal((g.n_cells, 3 * m), 1950)
    us = W.normal((fvm.n_faces(g), m), 1951)
    a = ProjectionStep(torch, nodes, m, 0.02, 0.01, mixed=2, solver="mg")
    b = ProjectionStep(torch, nodes, m, 0.02, 0.01, mixed=2, solver="mg")
    ud, usd = to_dev(u), to_dev(us)
    uw = torch.full((g.n_cells, 3 * m + 3), 9.0, dtype=torch.float64, device="cuda")
    usw = torch.full((fvm.n_faces(g), m + 1), 9.0, dtype=torch.float64, device="cuda")
    uw[:, 1:1 + 3 * m] = ud
    usw[:, :m] = usd
    a.step(ud, usd)
    b.step(uw[:, 1:1 + 3 * m], usw[:, :m])
    assert torch.equal(uw[:, 1:1 + 3 * m], ud) and torch.equal(usw[:, :m], usd)
    assert bool((uw[:, 0] == 9.0).all()) and bool((uw[:, 1 + 3 * m:] == 9.0).all()) and bool((usw[:, m] == 9.0).all())
    with pytest.raises(ValueError):
        a.step(ud[:, :3], usd)
    walled = W.channel_grid(8, 8, 16)
    wn, _ = rb.grid_nodes(walled)
    with pytest.raises(rb.RbError) as e:
        ProjectionStep(torch, wn, m, 0.02, 0.01)
    assert e.value.status == rb.RB_EINVAL
    import ctypes as C

    rep = rb.ProjectionReport()
    st = rb.lib().rb_projection_step(a.handle, C.c_void_p(ud.data_ptr()), 3 * m, C.c_void_p(ud.data_ptr() + 8), m,
                                     C.byref(rep), None)
    assert st == rb.RB_EINVAL and b"overlap" in rb.lib().rb_last_error()
