"""Parity of the device SpMM (CSR, sliced ELL, extruded) and BLAS-1 kernels against the oracle (GPU).

Tolerance: componentwise, |Y - Y_ref| <= tol * (|A| |X|) |c|, tol = 1e-12 for FP64 operators and
1e-5 for FP32 operators (the oracle is fed the FP32-rounded values and X and computes in FP64).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads as W
from oracle import blas, fvm, mesh, spmm
from tests.conftest import componentwise_ok, to_dev

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
KS = [1, 2, 3, 4, 5, 8, 16, 32, 64]


def _rand_csr(nr, nc, nnz_row, seed, long_rows=0):
    g = np.random.default_rng(seed)
    lens = g.poisson(nnz_row, nr)
    if nr > 5:
        lens[::7] = 0  # empty rows
    if long_rows:
        lens[nr // 2] = long_rows  # a row longer than a block can stage
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate([np.sort(g.choice(nc, size=min(l, nc), replace=False)) for l in lens]).astype(np.int32) \
        if nr else np.zeros(0, np.int32)
    lens = np.array([min(l, nc) for l in lens])
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    va = g.standard_normal(rp[-1])
    return sp.csr_matrix((va, ci, rp), shape=(nr, nc))


def _run(rb, A, X, dtype, fmt="csr", c=None, ld_pad=0, tune=False):
    k = X.shape[1]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    op = rb.Operator.from_scipy(A, dtype=dtype, fmt=fmt, k_max=k)
    Xs = np.zeros((A.shape[1], k + ld_pad), dtype=npdt)
    Xs[:, :k] = X.astype(npdt)
    Xd = to_dev(Xs)[:, :k]
    Yd = torch.full((A.shape[0], k + ld_pad), float("nan"), dtype=tdt, device="cuda")
    cd = None if c is None else to_dev(c.astype(np.float64))
    if tune:
        op.tune(Xd, Yd[:, :k])
    op.spmm(Xd, Yd[:, :k], c=cd)
    Y = Yd.cpu().numpy()
    if ld_pad:
        assert np.isnan(Y[:, k:]).all()  # padding lanes untouched
    Aref = A if dtype == "f64" else spmm.round_f32(A)
    Xref = Xs[:, :k].astype(np.float64)
    cref = None if c is None else (c if dtype == "f64" else c.astype(np.float32).astype(np.float64))
    Yref = spmm.spmm(Aref, Xref, cref)
    bound = spmm.abs_bound(Aref, Xref, cref)
    ok, worst = componentwise_ok(Y[:, :k], Yref, bound, TOL[dtype])
    assert ok, f"worst componentwise error {worst:.3e}"
    return op


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("fmt", ["csr", "sell"])
@pytest.mark.parametrize("k", KS)
def test_spmm_random_rectangular(rb, dtype, fmt, k):
    A = _rand_csr(1037, 811, 7, seed=k)
    X = W.normal((811, k), 100 + k)
    _run(rb, A, X, dtype, fmt)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_spmm_scale_padding_and_long_rows(rb, dtype, k):
    """Per-column scale c (Algorithm 1), ld > k (untouched padding), a row too long to stage."""
    A = _rand_csr(2000, 3000, 9, seed=50 + k, long_rows=2900)
    X = W.normal((3000, k), 200 + k)
    c = W.normal(k, 300 + k)
    _run(rb, A, X, dtype, "csr", c=c, ld_pad=3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_spmm_tuned_schedules(rb, dtype, k):
    """The autotuner's pick (vector width, lanes per row, staging) keeps parity."""
    A = _rand_csr(4000, 4000, 27, seed=70 + k)
    X = W.normal((4000, k), 400 + k)
    _run(rb, A, X, dtype, "csr", tune=True)


SCHEDULES = [  # (vec, lpr, stage, grid_cap) for k = 4
    (1, 1, 0, -1), (2, 1, 0, 0), (4, 1, 0, -1), (1, 2, 0, -1), (2, 4, 0, -1), (1, 8, 0, 0),
    (1, 1, 1, 0), (2, 2, 1, 0), (4, 1, 1, 0),
    (1, 1, 2, -1), (2, 1, 2, -1), (4, 1, 2, -1),
]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("sched", SCHEDULES, ids=lambda s: "v%d-l%d-s%d-g%d" % s)
def test_spmm_every_schedule(rb, dtype, sched):
    """Each kernel variant (direct, block-staged, TMA-pipelined; lanes per row; grids) pinned in
    turn: parity on a ragged random matrix with empty rows and one row too long to stage."""
    A = _rand_csr(5003, 4001, 7, seed=90, long_rows=3000)
    k = 4
    X = W.normal((4001, k), 91)
    c = W.normal(k, 92)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    op = rb.Operator.from_scipy(A, dtype=dtype, k_max=k)
    vec, lpr, stage, gc = sched
    op.set_schedule(k, vec, lpr, stage, gc)
    Xd = to_dev(X.astype(npdt))
    Yd = torch.full((A.shape[0], k), float("nan"), dtype=tdt, device="cuda")
    assert op.schedule(Xd, Yd) == {"vec": vec, "lpr": lpr, "stage": stage, "grid_cap": gc}
    op.spmm(Xd, Yd, c=to_dev(c))
    op.check()
    Aref = A if dtype == "f64" else spmm.round_f32(A)
    Xref = X.astype(npdt).astype(np.float64)
    cref = c if dtype == "f64" else c.astype(np.float32).astype(np.float64)
    ok, worst = componentwise_ok(Yd.cpu().numpy(), spmm.spmm(Aref, Xref, cref), spmm.abs_bound(Aref, Xref, cref),
                                 TOL[dtype])
    assert ok, worst


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8, 64])
def test_spmm_tma_pipeline_channel(rb, dtype, k):
    """The TMA-pipelined kernel on a stencil operator at several k (3-wide rows, 16-byte rows)."""
    g = W.channel_grid(40, 31, 23)
    A = fvm.laplacian(g)
    X = W.normal((A.shape[1], k), 300 + k)
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    op = rb.Operator.from_scipy(A, dtype=dtype, k_max=k)
    vec = 3 if k == 3 else min(k, 16 // (8 if dtype == "f64" else 4))
    op.set_schedule(k, vec, 1, 2, -1)
    Y = op.spmm(to_dev(X.astype(npdt)))
    op.check()
    Aref = A if dtype == "f64" else spmm.round_f32(A)
    Xref = X.astype(npdt).astype(np.float64)
    ok, worst = componentwise_ok(Y.cpu().numpy(), spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref), TOL[dtype])
    assert ok, worst


def _ragged_long_rows(nr, nc, seed, every=4999, long_len=3000):
    """Random rows of ~7 nonzeros, some empty, and every `every`-th row longer than a TMA stage
    holds, so that staged and unstaged tiles alternate along one block's walk."""
    g = np.random.default_rng(seed)
    lens = g.poisson(7, nr)
    lens[::13] = 0
    lens[every // 2::every] = long_len
    lens = np.minimum(lens, nc)
    ci = np.concatenate([np.sort(g.choice(nc, size=l, replace=False)) for l in lens]).astype(np.int32)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return sp.csr_matrix((g.standard_normal(rp[-1]), ci, rp), shape=(nr, nc))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 4, 32])
@pytest.mark.parametrize("grid_cap", [1, 3, 7])
def test_spmm_tma_steady_state(rb, dtype, k, grid_cap):
    """The TMA pipeline past its first round: with the grid capped at 1, 3 or 7 blocks every
    block walks tens to hundreds of tiles, so the 3-stage ring wraps over many phases (the
    empty-barrier waits of the later rounds), the producer reloads the boundaries of its next
    32 tiles many times, and staged and unstaged tiles (rows longer than a stage) alternate."""
    nr = 90_000 if k <= 4 else 9_000
    A = _ragged_long_rows(nr, 7_001, seed=500 + k)
    X = W.normal((7_001, k), 510 + k)
    c = W.normal(k, 520 + k)
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    op = rb.Operator.from_scipy(A, dtype=dtype, k_max=k)
    vec = 3 if k == 3 else min(k, 16 // (8 if dtype == "f64" else 4))
    op.set_schedule(k, vec, 1, 2, grid_cap)
    R = 256 // (1 << int(np.ceil(np.log2(k // vec))))  # rows per tile
    tiles = -(-nr // R)
    assert tiles // grid_cap >= 40, "each block must walk many tiles"
    Xd = to_dev(X.astype(npdt))
    for rep in range(2):  # the second call starts from barriers re-initialised by a new launch
        Yd = torch.full((nr, k), float("nan"), dtype=tdt, device="cuda")
        op.spmm(Xd, Yd, c=to_dev(c))
        op.check()
        Aref = A if dtype == "f64" else spmm.round_f32(A)
        Xref = X.astype(npdt).astype(np.float64)
        cref = c if dtype == "f64" else c.astype(np.float32).astype(np.float64)
        ok, worst = componentwise_ok(Yd.cpu().numpy(), spmm.spmm(Aref, Xref, cref), spmm.abs_bound(Aref, Xref, cref),
                                     TOL[dtype])
        assert ok, (rep, worst)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_spmm_fvm_operators(rb, dtype):
    """L (k = 3, velocity components), G (k = 3) and M (k = 1) of a channel grid."""
    g = W.channel_grid(24, 20, 16)
    for A, k in ((fvm.laplacian(g), 3), (fvm.gradient(g), 3), (fvm.divergence(g), 1)):
        X = W.normal((A.shape[1], k), 7 + k)
        _run(rb, A, X, dtype)


def test_spmm_edge_cases(rb):
    # empty operator, single row, k > 32 with unaligned ld is refused cleanly
    A = sp.csr_matrix((0, 5))
    op = rb.Operator.from_scipy(A)
    op.spmm(torch.zeros((5, 2), dtype=torch.float64, device="cuda"), torch.zeros((0, 2), dtype=torch.float64,
                                                                                   device="cuda"))
    A = sp.csr_matrix(np.array([[2.0, 0.0, -1.0]]))
    _run(rb, A, W.normal((3, 4), 1), "f64")
    op = rb.Operator.from_scipy(sp.identity(40, format="csr"))
    X = torch.zeros((40, 64 + 1), dtype=torch.float64, device="cuda")[:, 1:]
    Y = torch.zeros((40, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbError) as e:
        op.spmm(X, Y)
    assert e.value.status in (rb.RB_EINVAL, rb.RB_EUNSUPPORTED)
    with pytest.raises(rb.RbError):  # overlapping X and Y
        Z = torch.zeros((40, 4), dtype=torch.float64, device="cuda")
        op.spmm(Z, Z)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_spmm_no_nonzeros(rb, dtype, k):
    """Rows but no nonzeros: Y = 0 (not NaN, not stale) on every schedule the tuner tries."""
    A = sp.csr_matrix((50, 30))
    op = _run(rb, A, W.normal((30, k), 2), dtype, tune=True)
    assert op.nnz == 0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_spmm_channel_full_size_k3(rb, dtype):
    """192 x 128 x 96 channel Laplacian, k = 3, in the bench's launch configuration."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    A = fvm.laplacian_direct(g)
    X = W.normal((A.shape[1], 3), 2003)
    _run(rb, A, X, dtype)


def _face_starts(g):
    """First rows of the x-, y- and z-face blocks of the gradient of grid g."""
    n = [a.n for a in g.axes]
    counts = []
    for d in range(3):
        c = n[d] if g.axes[d].periodic else n[d] - 1
        for e in range(3):
            if e != d:
                c *= n[e]
        counts.append(c)
    return [0, counts[0], counts[0] + counts[1]]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 4])
@pytest.mark.parametrize("lpr", [1, 2])
def test_spmm_row_blocks_interleaved(rb, dtype, k, lpr):
    """The row-block hint (the gradient's x, y, z face blocks, of unequal lengths on a walled
    grid; and three arbitrary blocks of a random matrix): the direct kernel takes tiles from
    the blocks in turn; every row's result is unchanged."""
    g = W.channel_grid(40, 31, 23)
    G = fvm.gradient(g)
    starts = _face_starts(g)
    assert starts[2] < G.shape[0]
    for A, st in ((G, starts), (_rand_csr(7001, 3001, 5, seed=95), [0, 1000, 4500])):
        X = W.normal((A.shape[1], k), 96 + k)
        npdt = np.float64 if dtype == "f64" else np.float32
        tdt = torch.float64 if dtype == "f64" else torch.float32
        op = rb.Operator.from_scipy(A, dtype=dtype, k_max=k)
        op.set_row_blocks(st)
        vec = 3 if k == 3 else min(k, 16 // (8 if dtype == "f64" else 4))
        op.set_schedule(k, vec, lpr, 0, -1)
        Yd = torch.full((A.shape[0], k), float("nan"), dtype=tdt, device="cuda")
        op.spmm(to_dev(X.astype(npdt)), Yd)
        Aref = A if dtype == "f64" else spmm.round_f32(A)
        Xref = X.astype(npdt).astype(np.float64)
        ok, worst = componentwise_ok(Yd.cpu().numpy(), spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref), TOL[dtype])
        assert ok, worst
    with pytest.raises(rb.RbError):
        op.set_row_blocks([0, 5000, 3000])  # not increasing


@pytest.mark.parametrize("name,k", [("G", 3), ("L", 32)])
@pytest.mark.parametrize("sched", ["tuned", "tma"])
def test_spmm_channel_full_size_fp32_timed_schedules(rb, name, k, sched):
    """The FP32 SpMMs whose tuned schedule the bench times on the full 192 x 128 x 96 channel
    (the gradient with k = 3, the Laplacian with k = 32), on the tuner's pick and forced onto
    the TMA pipeline with one resident wave (tens of tiles per block), against the oracle."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    A = fvm.gradient(g) if name == "G" else fvm.laplacian_direct(g)
    X = W.normal((A.shape[1], k), 2100 + k).astype(np.float32)
    op = rb.Operator.from_scipy(A, dtype="f32", k_max=k)
    Xd = to_dev(X)
    Yd = torch.full((A.shape[0], k), float("nan"), dtype=torch.float32, device="cuda")
    if sched == "tuned":
        op.tune(Xd, Yd)
    else:
        op.set_schedule(k, 3 if k == 3 else 4, 1, 2, -1)
    op.spmm(Xd, Yd)
    op.check()
    Aref = spmm.round_f32(A)
    Xref = X.astype(np.float64)
    ok, worst = componentwise_ok(Yd.cpu().numpy(), spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref), TOL["f32"])
    assert ok, (op.schedule(Xd, Yd), worst)


# ------------------------------------------------------------------------------- extruded


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nz,sched", [(3, None), (8, None), (16, None), (64, None), (16, (4, 1, 1, 0)),
                                      (16, (2, 1, 2, 0)), (64, (4, 2, 0, -1)), (64, (4, 1, 2, 0))])
def test_extruded_spmm(rb, dtype, nz, sched):
    """The spanwise epilogue in every kernel: direct (lanes per row 1 and 2), block-staged, TMA."""
    m = W.random_trimesh(300, nz)
    L, _ = mesh.cot_laplacian(m)
    a = mesh.dual_areas(m)
    dz = W.EXTRUDED_SPAN / nz
    w = a / dz
    X = W.normal((L.shape[0], nz), 500 + nz)
    npdt = np.float64 if dtype == "f64" else np.float32
    op = rb.Operator.from_scipy(L, dtype=dtype, k_max=nz, extruded_nz=nz, z_weight=torch.as_tensor(w), dz=dz)
    if sched:
        op.set_schedule(nz, *sched)
    Y = op.spmm(to_dev(X.astype(npdt))).cpu().numpy()
    if dtype == "f64":
        Lr, wr, dzr, Xr = L, w, dz, X
    else:
        Lr = spmm.round_f32(L)
        wr = w.astype(np.float32).astype(np.float64)
        dzr = float(np.float32(dz))
        Xr = X.astype(np.float32).astype(np.float64)
    # oracle: the assembled 3-D operator dz (I (x) L2D) + T_z (x) diag(w)
    Yref = mesh.extruded_apply(Lr, wr * dzr, nz, dzr, Xr)
    absL = abs(Lr)
    bound = dzr * spmm.spmm(absL, np.abs(Xr)) + 4 * wr[:, None] * np.abs(Xr).max(axis=1, keepdims=True)
    ok, worst = componentwise_ok(Y, Yref, bound, TOL[dtype] * 4)
    assert ok, worst


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_extruded_spmm_scaled(rb, dtype):
    """Extruded operator with a per-column (per-plane) scale c: Y = c * (dz L X + spanwise term)."""
    nz = 8
    m = W.random_trimesh(257, 11)
    L, _ = mesh.cot_laplacian(m)
    a = mesh.dual_areas(m)
    dz = W.EXTRUDED_SPAN / nz
    w = a / dz
    X = W.normal((L.shape[0], nz), 611)
    c = W.normal(nz, 612)
    npdt = np.float64 if dtype == "f64" else np.float32
    op = rb.Operator.from_scipy(L, dtype=dtype, k_max=nz, extruded_nz=nz, z_weight=torch.as_tensor(w), dz=dz)
    Y = op.spmm(to_dev(X.astype(npdt)), c=to_dev(c)).cpu().numpy()
    rnd = (lambda v: v) if dtype == "f64" else (lambda v: np.asarray(v, np.float32).astype(np.float64))
    Lr = L if dtype == "f64" else spmm.round_f32(L)
    wr, dzr, Xr, cr = rnd(w), float(rnd(dz)), rnd(X), rnd(c)
    Yref = mesh.extruded_apply(Lr, wr * dzr, nz, dzr, Xr) * cr[None, :]
    bound = (dzr * spmm.spmm(abs(Lr), np.abs(Xr)) + 4 * wr[:, None] * np.abs(Xr).max(axis=1, keepdims=True)) \
        * np.abs(cr)[None, :]
    ok, worst = componentwise_ok(Y, Yref, bound, TOL[dtype] * 4)
    assert ok, worst


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_spmm_sell_scaled(rb, dtype, k):
    """Sliced ELL with a per-column scale c."""
    A = _rand_csr(777, 901, 6, seed=130 + k)
    X = W.normal((901, k), 131 + k)
    c = W.normal(k, 132 + k)
    _run(rb, A, X, dtype, "sell", c=c)


def test_extruded_airfoil_full_size(rb):
    """The ~150k-vertex airfoil mesh extruded into 64 periodic planes (k = 64), FP64."""
    m = W.airfoil_mesh()
    L, _ = mesh.cot_laplacian(m)
    a = mesh.dual_areas(m)
    nz = W.EXTRUDED_NZ
    dz = W.EXTRUDED_SPAN / nz
    X = W.normal((L.shape[0], nz), 3064)
    op = rb.Operator.from_scipy(L, k_max=nz, extruded_nz=nz, z_weight=torch.as_tensor(a / dz), dz=dz)
    Y = op.spmm(to_dev(X)).cpu().numpy()
    Yref = mesh.extruded_apply(L, a, nz, dz, X)
    bound = dz * spmm.spmm(abs(L), np.abs(X)) + 4 * (a / dz)[:, None] * np.abs(X).max(axis=1, keepdims=True)
    ok, worst = componentwise_ok(Y, Yref, bound, 4e-12)
    assert ok, worst


# ------------------------------------------------------------------------------- BLAS-1


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 64])
@pytest.mark.parametrize("n", [1, 1000, 300_001])
def test_dot_axpy_axty(rb, dtype, k, n):
    """Contiguous blocks (the flat 16-byte streaming kernels for k <= 8, all k for axpy/axty)."""
    npdt = np.float64 if dtype == "f64" else np.float32
    X = W.normal((n, k), 1).astype(npdt)
    Y = W.normal((n, k), 2).astype(npdt)
    alpha = W.normal(k, 3)
    Xd, Yd = to_dev(X), to_dev(Y)
    d = rb.dot(Xd, Yd).cpu().numpy()
    dref = blas.dot(X, Y)
    scale = blas.dot(np.abs(X), np.abs(Y))
    tol = 1e-13 if dtype == "f64" else 1e-6
    assert np.all(np.abs(d - dref) <= tol * scale + 1e-300)
    # bit-reproducible
    assert np.array_equal(d, rb.dot(Xd, Yd).cpu().numpy())
    rb.axpy(to_dev(alpha), Xd, Yd)
    aref = blas.axpy(alpha if dtype == "f64" else alpha.astype(np.float32), X, Y)
    got = Yd.cpu().numpy().astype(np.float64)
    tol2 = 1e-15 if dtype == "f64" else 2e-7
    assert np.all(np.abs(got - aref) <= tol2 * (np.abs(X * alpha[None, :]) + np.abs(Y)) + 1e-300)
    Yd2 = to_dev(Y)
    rb.axty(0.5, Xd, Yd2)
    tref = blas.axty(0.5, X, Y)
    tol3 = 1e-15 if dtype == "f64" else 2e-7
    assert np.all(np.abs(Yd2.cpu().numpy() - tref) <= tol3 * np.abs(tref) + 1e-300)
    # alpha = 1 (the Jacobi product, one multiply per entry): the correctly rounded x y, bit for
    # bit (the FP64 product of two FP32 values is exact, so rounding it once gives the FP32 one)
    Yd3 = to_dev(Y)
    rb.axty(1.0, Xd, Yd3)
    assert np.array_equal(Yd3.cpu().numpy(), blas.axty(1.0, X, Y).astype(npdt))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_dot_axpy_axty_strided(rb, dtype, k):
    """Rows wider than k (ld = k + 3): the row-and-chunk kernels; padding left untouched."""
    npdt = np.float64 if dtype == "f64" else np.float32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    n = 12_345
    X = W.normal((n, k), 11).astype(npdt)
    Y = W.normal((n, k), 12).astype(npdt)
    alpha = W.normal(k, 13)
    Xw = torch.full((n, k + 3), float("nan"), dtype=tdt, device="cuda")
    Yw = torch.full((n, k + 3), float("nan"), dtype=tdt, device="cuda")
    Xw[:, :k] = to_dev(X)
    Yw[:, :k] = to_dev(Y)
    d = rb.dot(Xw[:, :k], Yw[:, :k]).cpu().numpy()
    scale = blas.dot(np.abs(X), np.abs(Y))
    tol = 1e-13 if dtype == "f64" else 1e-6
    assert np.all(np.abs(d - blas.dot(X, Y)) <= tol * scale + 1e-300)
    rb.axpy(to_dev(alpha), Xw[:, :k], Yw[:, :k])
    aref = blas.axpy(alpha if dtype == "f64" else alpha.astype(np.float32), X, Y)
    got = Yw[:, :k].cpu().numpy().astype(np.float64)
    tol2 = 1e-15 if dtype == "f64" else 2e-7
    assert np.all(np.abs(got - aref) <= tol2 * (np.abs(X * alpha[None, :]) + np.abs(Y)) + 1e-300)
    assert torch.isnan(Yw[:, k:]).all()
    for a in (0.5, 1.0):  # both axty kernels: the scaled product and the unit one
        Yw[:, :k] = to_dev(Y)
        rb.axty(a, Xw[:, :k], Yw[:, :k])
        tref = blas.axty(a, X, Y)
        got = Yw[:, :k].cpu().numpy()
        if a == 1.0:
            assert np.array_equal(got, tref.astype(npdt))
        else:
            assert np.all(np.abs(got - tref) <= (1e-15 if dtype == "f64" else 2e-7) * np.abs(tref) + 1e-300)
        assert torch.isnan(Yw[:, k:]).all()


def test_fma_peak_is_plausible(rb):
    """The measured FMA roofs: FP64 within GB300's nominal rate (152 SMs x 2 FMAs per clock x 2
    flops at up to 2.07 GHz, 1.26 TFLOP/s) and above half of it; FP32 far above FP64."""
    f64 = rb.fma_peak("f64")
    f32 = rb.fma_peak("f32")
    assert 0.5 * 1.26 < f64 <= 1.05 * 1.26, f64
    assert f32 > 20 * f64, (f32, f64)
