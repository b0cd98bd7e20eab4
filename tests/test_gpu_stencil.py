"""Parity of the device 13p / 27p stencil assembly (Sec. 4.1's denser patterns) against the
oracle, and of the SpMM and Poisson solve on those operators (GPU).

Bar: the CSR structure (row pointers, column indices) bit-exact; values within 4 ulp (the
host forms each coefficient with the oracle's operations, the 27p volume factor h^3 may round
differently); SpMM componentwise as in the SpMM tests; CG to a true 1e-10 residual and the
oracle's solution.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cg as ocg
from oracle import spmm, stencil
from tests.conftest import componentwise_ok, to_dev

pytestmark = pytest.mark.gpu

VAL_RTOL = 4 * 2.0 ** -52


def _assemble(rb, shape, h, kind, scale=1.0):
    rp, ci, va, n = rb.stencil_assemble(shape, h, kind, scale=scale)
    torch.cuda.synchronize()
    return rp.cpu().numpy(), ci.cpu().numpy(), va.cpu().numpy(), n


def _oracle(shape, h, kind):
    return stencil.laplacian_13p(shape, h) if kind == 13 else stencil.laplacian_27p(shape, h[0])


CASES = [  # (kind, shape, h): the smallest grids, ragged last blocks, anisotropic 13p
    (13, (5, 5, 5), (0.2, 0.2, 0.2)),
    (13, (5, 6, 7), (0.3, 0.2, 0.25)),
    (13, (8, 9, 10), (0.125, 0.5, 0.1)),
    (13, (33, 5, 6), (1.0, 2.0, 3.0)),
    (27, (3, 3, 3), (0.5, 0.5, 0.5)),
    (27, (3, 4, 5), (0.2, 0.2, 0.2)),
    (27, (11, 12, 13), (0.1, 0.1, 0.1)),
    (27, (40, 3, 7), (1.0 / 40, 1.0 / 40, 1.0 / 40)),
]


@pytest.mark.parametrize("kind,shape,h", CASES, ids=lambda v: str(v))
def test_stencil_assembly_matches_oracle(rb, kind, shape, h):
    rp, ci, va, n = _assemble(rb, shape, h, kind)
    L = _oracle(shape, h, kind)
    assert n == L.shape[0]
    assert np.array_equal(rp, L.indptr.astype(np.int32))
    assert np.array_equal(ci, L.indices.astype(np.int32))
    assert np.all(np.abs(va - L.data) <= VAL_RTOL * np.abs(L.data))


def test_stencil_scale(rb):
    """scale multiplies every value (-1: the SPD Poisson matrix)."""
    shape, h = (6, 5, 7), (0.3, 0.2, 0.25)
    _, _, va1, _ = _assemble(rb, shape, h, 13)
    _, ci2, va2, _ = _assemble(rb, shape, h, 13, scale=-1.0)
    assert np.array_equal(va2, -va1)


def test_stencil_invalid_arguments(rb):
    for shape, h, kind in (((4, 6, 6), (1, 1, 1), 13), ((5, 5, 2), (1, 1, 1), 27), ((5, 5, 5), (1, 1, 2), 27),
                           ((5, 5, 5), (1, 0, 1), 13), ((5, 5, 5), (1, 1, 1), 7)):
        with pytest.raises(rb.RbError) as e:
            rb.stencil_assemble(shape, h, kind)
        assert "EINVAL" in str(e.value)


@pytest.mark.parametrize("kind", [13, 27])
def test_stencil_full_size(rb, kind):
    """The 160^3 grid of the stencil bench (4,096,000 cells): structure and zero row sums on
    every row, sampled rows against the oracle row by row, symmetry on the sampled rows."""
    shape = (160, 160, 160)
    h = (1.0 / 160,) * 3
    rp, ci, va, n = rb.stencil_assemble(shape, h, kind)
    assert torch.equal(rp, kind * torch.arange(n + 1, dtype=torch.int32, device="cuda"))
    C = ci.view(n, kind)
    assert bool((C[:, 1:] > C[:, :-1]).all())
    assert int(C.min()) >= 0 and int(C.max()) < n
    V = va.view(n, kind)
    assert float((V.sum(dim=1).abs() / V.abs().sum(dim=1)).max()) <= 1e-14
    offs = stencil.offsets_13p(h) if kind == 13 else stencil.offsets_27p(h[0])
    g = np.random.default_rng(160 + kind)
    sample = np.concatenate([[0, 1, 159, 160 * 160 - 1, n - 1, n // 2], g.integers(0, n, 200)])
    Cs, Vs = C[torch.as_tensor(sample, device="cuda")].cpu().numpy(), V[torch.as_tensor(sample, device="cuda")].cpu().numpy()
    for r, cr, vr in zip(sample, Cs, Vs):
        oc, ov = stencil.row(shape, offs, int(r))
        assert np.array_equal(cr, oc)
        assert np.all(np.abs(vr - ov) <= VAL_RTOL * np.abs(ov))
        # symmetry: row c holds r with the same value
        rows_c = C[torch.as_tensor(cr.astype(np.int64), device="cuda")].cpu().numpy()
        vals_c = V[torch.as_tensor(cr.astype(np.int64), device="cuda")].cpu().numpy()
        for t in range(kind):
            hit = np.nonzero(rows_c[t] == r)[0]
            assert hit.size == 1 and vals_c[t][hit[0]] == vr[t]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("kind", [13, 27])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_spmm_on_stencils(rb, dtype, kind, k):
    """The SpMM on 13- and 27-entry rows (odd lengths: the unrolled nonzero loops' remainders),
    tuned and on every staging variant."""
    shape, h = ((9, 10, 11), (0.3, 0.2, 0.25)) if kind == 13 else ((11, 12, 13), (0.1, 0.1, 0.1))
    rp, ci, va, n = rb.stencil_assemble(shape, h, kind)
    L = _oracle(shape, h, kind)
    X = W.normal((n, k), 1300 + kind + k)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    npdt = np.float64 if dtype == "f64" else np.float32
    op = rb.Operator(rp, ci, va, n, dtype=dtype, k_max=k)
    Xd = to_dev(X.astype(npdt))
    Aref = L if dtype == "f64" else spmm.round_f32(L)
    Xref = X.astype(npdt).astype(np.float64)
    Yref, bound = spmm.spmm(Aref, Xref), spmm.abs_bound(Aref, Xref)
    tol = 1e-12 if dtype == "f64" else 1e-5
    scheds = [None] + [(v, lpr, st, gc) for v in (1,) for (lpr, st, gc) in ((1, 0, -1), (2, 0, 0), (4, 0, -1),
                                                                            (1, 1, 0), (1, 2, -1))]
    for sc in scheds:
        Yd = torch.full((n, k), float("nan"), dtype=tdt, device="cuda")
        if sc is None:
            op.tune(Xd, Yd)
        else:
            op.set_schedule(k, *sc)
        op.spmm(Xd, Yd)
        op.check()
        ok, worst = componentwise_ok(Yd.cpu().numpy(), Yref, bound, tol)
        assert ok, (sc, worst)


@pytest.mark.parametrize("kind", [13, 27])
@pytest.mark.parametrize("mixed", [0, 2])
def test_cg_on_stencils(rb, kind, mixed):
    """Poisson solves with A = -L (13p, 27p) on zero-mean right-hand sides: true residual 1e-10
    and the oracle's CG solution."""
    shape, h = ((12, 10, 14), (0.1, 0.12, 0.09)) if kind == 13 else ((13, 12, 11), (0.1, 0.1, 0.1))
    rp, ci, va, n = rb.stencil_assemble(shape, h, kind, scale=-1.0)
    A = (-_oracle(shape, h, kind)).tocsr()
    k = 3
    B = W.zero_mean(W.normal((n, k), 1400 + kind))
    op = rb.Operator(rp, ci, va, n, k_max=k)
    opi = rb.Operator(rp, ci, va, n, dtype="f32", k_max=k) if mixed else None
    X = to_dev(np.zeros_like(B))
    res = rb.cg_solve(op, to_dev(B), X, A_inner=opi, params=rb.cg_params(rtol=1e-10, mixed=mixed, project_mean=True))
    assert res.status == rb.RB_OK, res
    Xn = X.cpu().numpy()
    R = B - A @ Xn
    R -= R.mean(axis=0, keepdims=True)
    tr = np.linalg.norm(R, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(tr <= 1e-10), tr
    Xr, _ = ocg.pcg_columns(A, B, rtol=1e-10, project_mean=True)
    err = np.linalg.norm(Xn - Xr, axis=0) / np.linalg.norm(Xr, axis=0)
    assert np.all(err <= 1e-7), err
