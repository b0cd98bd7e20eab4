"""rb_dot_noalloc, the dot product for callers that cannot give the library device memory
(GPU).

Such a caller (a plain C program or a plugin that does not own the GPU's memory pool, or a
code path that must not call cudaMalloc because it can synchronise the device) calls the
entry point through the C ABI with only its inputs and its output; the partial sums live in
a fixed array inside the library.  This file is collected last so that a run stopping at the
first failure has run every other test already; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W
from oracle import blas as oblas
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


def _call(rb, n, k, code, X, Y, stream):
    lib = rb.lib()
    out = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.rb_dot_noalloc(n, k, code, C.c_void_p(X.data_ptr() if n else 0), k,
                            C.c_void_p(Y.data_ptr() if n else 0), k, C.c_void_p(out.data_ptr()), stream)
    assert st == rb.RB_OK, lib.rb_last_error()
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype,k,n", [("f64", 1, 300_001), ("f64", 3, 77_777), ("f32", 8, 100_000),
                                       ("f64", 64, 5_000), ("f32", 64, 9_999)])
def test_dot_noalloc_matches_rb_dot_twice(rb, dtype, k, n):
    npdt = np.float64 if dtype == "f64" else np.float32
    code = rb.RB_F64 if dtype == "f64" else rb.RB_F32
    Xh = W.normal((n, k), 801).astype(npdt)
    Yh = W.normal((n, k), 802).astype(npdt)
    X, Y = to_dev(Xh), to_dev(Yh)
    ref = rb.dot(X, Y).cpu().numpy()  # the existing entry point, with its workspace
    exact = oblas.dot(Xh, Yh)  # the FP64 oracle on the same (FP32-valued) inputs
    scale = oblas.dot(np.abs(Xh), np.abs(Yh))
    tol = 1e-13 if dtype == "f64" else 1e-6
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # the shared scratch keeps the previous call's sums: two calls in a row
        got = _call(rb, n, k, code, X, Y, stream)
        assert np.all(np.abs(got - ref) <= tol * scale + 1e-300), (call, got, ref)
        assert np.all(np.abs(got - exact) <= tol * scale + 1e-300), (call, got, exact)


def test_dot_noalloc_large_then_small(rb):
    """A call on many rows (all 256 partial-sum rows of the scratch used) followed on the same
    stream by calls that use one row of it, and by an empty one: stale rows of the earlier
    call must not leak into the later sums."""
    k = 5
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    Xh, Yh = W.normal((4_000_000, k), 811), W.normal((4_000_000, k), 812)
    X, Y = to_dev(Xh), to_dev(Yh)
    big = _call(rb, Xh.shape[0], k, rb.RB_F64, X, Y, stream)
    assert np.all(np.abs(big - oblas.dot(Xh, Yh)) <= 1e-13 * oblas.dot(np.abs(Xh), np.abs(Yh)))
    for n in (37, 1):
        xs, ys = Xh[:n], Yh[:n]
        got = _call(rb, n, k, rb.RB_F64, to_dev(xs), to_dev(ys), stream)
        assert np.all(np.abs(got - oblas.dot(xs, ys)) <= 1e-13 * oblas.dot(np.abs(xs), np.abs(ys)) + 1e-300), n
        assert np.all(np.abs(got - rb.dot(to_dev(xs), to_dev(ys)).cpu().numpy()) <= 1e-13 * oblas.dot(np.abs(xs), np.abs(ys)) + 1e-300)
    empty = _call(rb, 0, k, rb.RB_F64, X, Y, stream)
    assert np.array_equal(empty, np.zeros(k))


def test_dot_noalloc_rejects_too_many_columns(rb):
    lib = rb.lib()
    X = torch.zeros((10, 65), dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    st = lib.rb_dot_noalloc(10, 65, rb.RB_F64, C.c_void_p(X.data_ptr()), 65, C.c_void_p(X.data_ptr()), 65,
                            C.c_void_p(out.data_ptr()), None)
    assert st == rb.RB_EINVAL
    assert b"scratch" in lib.rb_last_error()
