"""Parity of the double-float SpMM (RB_DF64: FP64 values as pairs hi + lo of FP32 numbers, the
products and sums formed with TwoProd and TwoSum) against the FP64 oracle (GPU).

Bars:
  * rb_df64_split / rb_df64_join: bit-exact against the format's definition, hi = RN32(x),
    lo = RN32(x - hi), x' = RN64(hi + lo), computed here with numpy's IEEE conversions;
  * the SpMM: componentwise |Y - Y_ref| <= tol_i (|A| |X|)_ij |c_j| against the oracle's FP64
    product of the ORIGINAL FP64 operator and block, with tol_i = (n_i^2 + 10 n_i + 10) 2^-48
    for a row of n_i nonzeros (the worst case of the accumulation: TwoSum and TwoProd are
    exact, the low-part sum E rounds n_i times, the products' low parts and the input splits
    round once each); for the FVM operators (n_i <= 7) that is below 1e-12, the FP64 bar.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import workloads as W
from oracle import fvm, spmm
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu

KS = [1, 2, 3, 4, 5, 6, 8, 16, 32, 64]


def _split_ref(x):
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def _df_block(rb, X, ld_pad=0):
    """X (float64 numpy) as a double-float device block, optionally inside a wider one."""
    n, k = X.shape
    hi, lo = _split_ref(X)
    full = np.zeros((n, k + ld_pad, 2), dtype=np.float32)
    full[:, :k, 0], full[:, :k, 1] = hi, lo
    return to_dev(full)[:, :k]


def _row_tol(A):
    n = np.diff(A.indptr).astype(np.float64)
    return ((n * n + 10 * n + 10) * 2.0 ** -48)[:, None]


def _check(A, X, Y, c=None, tol=None):
    Yref = spmm.spmm(A, X, c)
    bound = spmm.abs_bound(A, X, c)
    lim = (_row_tol(A) if tol is None else tol) * bound
    err = np.abs(Y - Yref)
    worst = float((err / np.maximum(bound, 1e-300)).max()) if err.size else 0.0
    assert np.all(err <= lim + 1e-300), f"worst componentwise error {worst:.3e}"
    return worst


def _rand_csr(nr, nc, nnz_row, seed, long_rows=0):
    g = np.random.default_rng(seed)
    lens = np.minimum(g.poisson(nnz_row, nr), nc)
    if nr > 5:
        lens[::7] = 0  # empty rows
    if long_rows:
        lens[nr // 2] = min(long_rows, nc)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate([np.sort(g.choice(nc, size=l, replace=False)) for l in lens]).astype(np.int32)
    va = g.standard_normal(rp[-1]) * np.exp(g.uniform(-3, 3, rp[-1]))  # six decades of magnitude
    return sp.csr_matrix((va, ci, rp), shape=(nr, nc))


def _run(rb, A, X, c=None, ld_pad=0, sched=None, tune=False):
    k = X.shape[1]
    op = rb.Operator.from_scipy(A, dtype="df64", k_max=k)
    Xd = _df_block(rb, X, ld_pad)
    Yfull = torch.full((A.shape[0], k + ld_pad, 2), float("nan"), dtype=torch.float32, device="cuda")
    Yd = Yfull[:, :k]
    if sched is not None:
        op.set_schedule(k, *sched)
    if tune:
        op.tune(Xd, Yd)
    cd = None if c is None else to_dev(c.astype(np.float64))
    op.spmm(Xd, Yd, c=cd)
    Y = rb.df_join(Yd).cpu().numpy()
    if ld_pad:
        assert torch.isnan(Yfull[:, k:]).all()  # the padding columns untouched
    return op, Y


def test_split_and_join_are_the_definition(rb):
    g = np.random.default_rng(11)
    X = g.standard_normal((1001, 5)) * np.exp(g.uniform(-40, 40, (1001, 5)))
    X[0, 0], X[1, 1], X[2, 2] = 0.0, -0.0, 1.0 + 2.0 ** -40
    D = rb.df_split(to_dev(X))
    assert D.shape == (1001, 5, 2) and D.dtype == torch.float32
    hi, lo = _split_ref(X)
    Dh = D.cpu().numpy()
    assert np.array_equal(Dh[..., 0].view(np.uint32), hi.view(np.uint32))
    assert np.array_equal(Dh[..., 1].view(np.uint32), lo.view(np.uint32))
    J = rb.df_join(D).cpu().numpy()
    assert np.array_equal(J, hi.astype(np.float64) + lo.astype(np.float64))
    assert np.all(np.abs(J - X) <= 2.0 ** -48 * np.abs(X))  # 48 bits of the 53 survive
    # strided blocks: columns 1..3 of wider blocks, the rest untouched
    Xw = to_dev(X)
    Dw = torch.full((1001, 7, 2), 5.0, dtype=torch.float32, device="cuda")
    rb.df_split(Xw[:, 1:4], out=Dw[:, 2:5])
    Dwh = Dw.cpu().numpy()
    assert np.array_equal(Dwh[:, 2:5, 0], hi[:, 1:4]) and np.array_equal(Dwh[:, 2:5, 1], lo[:, 1:4])
    assert np.all(Dwh[:, [0, 1, 5, 6]] == 5.0)


@pytest.mark.parametrize("k", KS)
def test_spmm_random_rectangular(rb, k):
    A = _rand_csr(3001, 2203, 8, 100 + k, long_rows=300)
    X = W.normal((A.shape[1], k), 200 + k)
    _run(rb, A, X)
    _run(rb, A, X, tune=True)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8])
def test_spmm_every_schedule(rb, k):
    """Every valid (vec, lpr, grid_cap) of the double-float kernel; staged schedules refused."""
    A = _rand_csr(5003, 4001, 12, 300 + k, long_rows=500)
    X = W.normal((A.shape[1], k), 400 + k)
    ran = 0
    for vec in (1, 2, 3, 4):
        if k % vec or (k // vec) > 32:
            continue
        kp = 1 << max(0, (k // vec - 1).bit_length())
        for lpr in (1, 2, 4, 8):
            if kp * lpr > 32:
                continue
            for gc in (-1, 0, 7):
                _run(rb, A, X, sched=(vec, lpr, 0, gc))
                ran += 1
    assert ran >= 3
    op = rb.Operator.from_scipy(A, dtype="df64", k_max=k)
    for stage in (1, 2):
        with pytest.raises(rb.RbError) as e:
            op.set_schedule(k, 1, 1, stage, -1)
        assert e.value.status == rb.RB_EINVAL


@pytest.mark.parametrize("k", [1, 3, 8])
def test_spmm_scaled_and_strided(rb, k):
    A = _rand_csr(2000, 2000, 6, 500 + k)
    X = W.normal((2000, k), 600 + k)
    c = np.linspace(-2.5, 3.0, k) + 1.0 / 3.0  # not exact in FP32: the split of c matters
    _run(rb, A, X, c=c, ld_pad=3)


def test_spmm_empty_and_tiny(rb):
    A = sp.csr_matrix((np.zeros(0), np.zeros(0, np.int32), np.zeros(4, np.int32)), shape=(3, 5))
    _, Y = _run(rb, A, W.normal((5, 2), 1))
    assert np.all(Y == 0.0)
    A = sp.csr_matrix(np.array([[1.0 + 2.0 ** -30, -1.0, 0.0], [0.0, 0.0, 0.0], [2.0 ** -20, 0.0, 3.0]]))
    X = np.array([[1.0, 2.0 ** -30], [1.0, 0.0], [-(2.0 ** -25), 1.0]])
    _, Y = _run(rb, A, X)
    Yref = A @ X
    # cancellation: row 0, column 0 is 2^-30 exactly, far below FP32's resolution of 1
    assert Y[0, 0] == Yref[0, 0] == 2.0 ** -30
    assert np.array_equal(Y[1], [0.0, 0.0])


@pytest.mark.parametrize("kind", ["laplacian", "gradient", "divergence"])
@pytest.mark.parametrize("k", [1, 3, 4])
def test_fvm_operators_at_fp64_bar(rb, kind, k):
    """The staggered FVM operators of a stretched channel: within 1e-12 (|A||X|), the FP64 bar."""
    g = W.channel_grid(24, 16, 12, gamma=1.5)
    A = {"laplacian": fvm.laplacian_direct, "gradient": fvm.gradient, "divergence": fvm.divergence}[kind](g)
    A = A.tocsr()
    assert np.diff(A.indptr).max() <= 7
    X = W.normal((A.shape[1], k), 700 + k)
    _, Y = _run(rb, A, X)
    _check(A, X, Y, tol=1e-12)


def test_channel_full_size_k3(rb):
    """The 192 x 128 x 96 channel Laplacian, k = 3, the tuned schedule: sampled rows against the
    oracle (rows computed one by one) at the FP64 bar, and the whole result against the native
    FP64 SpMM within 2e-12 (|A||X|)."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    nodes, per = rb.grid_nodes(g)
    rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
    k = 3
    X = W.normal((nc, k), 2025)
    Xd64 = to_dev(X)
    op64 = rb.Operator(rp, ci, va, nc, dtype="f64", k_max=k)
    opdf = rb.Operator(rp, ci, va, nc, dtype="df64", k_max=k)
    Xdf = rb.df_split(Xd64)
    Ydf = torch.empty((opdf.n_rows, k, 2), dtype=torch.float32, device="cuda")
    opdf.tune(Xdf, Ydf)
    opdf.spmm(Xdf, Ydf)
    Y = rb.df_join(Ydf)
    Y64 = op64.spmm(Xd64)
    absA = rb.Operator(rp, ci, va.abs(), nc, dtype="f64", k_max=k)
    bound = absA.spmm(Xd64.abs())
    rel = ((Y - Y64).abs() / bound.clamp_min(1e-300)).max().item()
    assert rel <= 2e-12, rel
    L = fvm.laplacian_direct(g).tocsr()
    rows = np.random.default_rng(5).choice(L.shape[0], 4000, replace=False)
    Ls = L[rows]
    Yh = Y.cpu().numpy()[rows]
    ref = Ls @ X
    lim = 1e-12 * (abs(Ls) @ np.abs(X))
    assert np.all(np.abs(Yh - ref) <= lim)


def test_refusals(rb):
    A = _rand_csr(100, 100, 4, 9)
    with pytest.raises(rb.RbError) as e:
        rb.Operator.from_scipy(A, dtype="df64", fmt="sell")
    assert e.value.status == rb.RB_EINVAL
    big = A.copy()
    big.data[0] = 1e39
    with pytest.raises(rb.RbError) as e:
        rb.Operator.from_scipy(big, dtype="df64")
    assert e.value.status == rb.RB_EINVAL and "FP32 range" in str(e.value)
    op = rb.Operator.from_scipy(A, dtype="df64", k_max=2)
    with pytest.raises(ValueError):  # a float64 block is not a double-float block
        op.spmm(to_dev(np.ones((100, 2))))
    op64 = rb.Operator.from_scipy(A, dtype="f64", k_max=2)
    with pytest.raises(ValueError):  # nor the other way round
        op64.spmm(_df_block(rb, np.ones((100, 2))))


def _stencil_df(rb, g, k, scale=1.0):
    nodes, per = rb.grid_nodes(g)
    return rb.Operator.stencil(nodes, per, scale=scale, dtype="df64", k_max=k)


@pytest.mark.parametrize("name", ["channel-24x16x12", "periodic-10", "rbc-8x8x16", "channel-13x6x5"])
@pytest.mark.parametrize("k", [1, 3, 4, 8])
def test_stencil_df_at_fp64_bar(rb, name, k):
    """The matrix-free Laplacian in double-float arithmetic (factorised entries V c): within
    1e-12 (|L||X|) of the oracle's assembled FP64 Laplacian, scale -1 included (A = -L); odd
    and even axes, walls and periodic axes."""
    g = {"channel-24x16x12": W.channel_grid(24, 16, 12, gamma=1.5), "periodic-10": W.unit_periodic_grid(10),
         "rbc-8x8x16": W.Grid((W.uniform_axis(8), W.uniform_axis(8), W.tanh_axis(16, 1.4, 0.0, 1.0))),
         "channel-13x6x5": W.channel_grid(13, 6, 5, gamma=2.0)}[name]
    L = fvm.laplacian_direct(g).tocsr()
    X = W.normal((g.n_cells, k), 800 + k)
    for scale in (1.0, -1.0):
        op = _stencil_df(rb, g, k, scale)
        Yd = op.spmm(_df_block(rb, X))
        Y = rb.df_join(Yd).cpu().numpy()
        _check((scale * L).tocsr(), X, Y, tol=1e-12)


def test_stencil_df_scaled_strided(rb):
    g = W.channel_grid(16, 12, 8, gamma=1.5)
    L = fvm.laplacian_direct(g).tocsr()
    k = 3
    X = W.normal((g.n_cells, k), 830)
    c = np.array([0.5, -1.0 / 3.0, 2.5])
    op = _stencil_df(rb, g, k)
    Xd = _df_block(rb, X, ld_pad=2)
    Yw = torch.full((g.n_cells, k + 1, 2), float("nan"), dtype=torch.float32, device="cuda")
    op.spmm(Xd, Yw[:, :k], c=to_dev(c))
    assert torch.isnan(Yw[:, k]).all()
    Y = rb.df_join(Yw[:, :k]).cpu().numpy()
    _check(L, X, Y, c=c, tol=1e-12)


def test_stencil_df_channel_full_size_k3(rb):
    """The 192 x 128 x 96 channel, k = 3: the whole product against the native FP64 CSR SpMM
    within 2e-12 (|L||X|) and sampled rows against the oracle within 1e-12."""
    g = W.channel_grid(*W.CHANNEL_SHAPE, gamma=1.5)
    nodes, per = rb.grid_nodes(g)
    rp, ci, va, nc = rb.fvm_assemble(nodes, per, rb.RB_FVM_LAPLACIAN)
    k = 3
    X = W.normal((nc, k), 2026)
    Xd64 = to_dev(X)
    op = rb.Operator.stencil(nodes, per, dtype="df64", k_max=k)
    Xdf = rb.df_split(Xd64)
    Ydf = torch.empty((op.n_rows, k, 2), dtype=torch.float32, device="cuda")
    op.tune(Xdf, Ydf)
    op.spmm(Xdf, Ydf)
    Y = rb.df_join(Ydf)
    op64 = rb.Operator(rp, ci, va, nc, dtype="f64", k_max=k)
    Y64 = op64.spmm(Xd64)
    bound = rb.Operator(rp, ci, va.abs(), nc, dtype="f64", k_max=k).spmm(Xd64.abs())
    rel = ((Y - Y64).abs() / bound.clamp_min(1e-300)).max().item()
    assert rel <= 2e-12, rel
    Lc = fvm.laplacian_direct(g).tocsr()
    rows = np.random.default_rng(6).choice(Lc.shape[0], 4000, replace=False)
    Ls = Lc[rows]
    assert np.all(np.abs(Y.cpu().numpy()[rows] - Ls @ X) <= 1e-12 * (abs(Ls) @ np.abs(X)))
