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
from tests.conftest import to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,k,n", [("f64", 1, 300_001), ("f64", 3, 77_777), ("f32", 8, 100_000),
                                       ("f64", 64, 5_000), ("f32", 64, 9_999)])
def test_dot_noalloc_matches_rb_dot_twice(rb, dtype, k, n):
    npdt = np.float64 if dtype == "f64" else np.float32
    code = rb.RB_F64 if dtype == "f64" else rb.RB_F32
    X = to_dev(W.normal((n, k), 801).astype(npdt))
    Y = to_dev(W.normal((n, k), 802).astype(npdt))
    ref = rb.dot(X, Y).cpu().numpy()  # the existing entry point, with its workspace
    scale = rb.dot(X.abs(), Y.abs()).cpu().numpy()
    tol = 1e-13 if dtype == "f64" else 1e-6
    lib = rb.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):  # the shared scratch keeps the previous call's sums: two calls in a row
        out = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.rb_dot_noalloc(n, k, code, C.c_void_p(X.data_ptr()), k, C.c_void_p(Y.data_ptr()), k,
                                C.c_void_p(out.data_ptr()), stream)
        assert st == rb.RB_OK, lib.rb_last_error()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= tol * scale + 1e-300), (call, got, ref)


def test_dot_noalloc_rejects_too_many_columns(rb):
    lib = rb.lib()
    X = torch.zeros((10, 65), dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    st = lib.rb_dot_noalloc(10, 65, rb.RB_F64, C.c_void_p(X.data_ptr()), 65, C.c_void_p(X.data_ptr()), 65,
                            C.c_void_p(out.data_ptr()), None)
    assert st == rb.RB_EINVAL
    assert b"scratch" in lib.rb_last_error()
