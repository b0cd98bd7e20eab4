"""The C ABI library builds, loads without a GPU and exports every symbol the header declares (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rbspmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:rb_status|size_t|const char\*)\s+(rb_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2508_06710_gb300 import build

    build.build()
    import paper_2508_06710_gb300 as rb

    return rb.lib()


def test_header_declares_the_documented_calls():
    names = _declared()
    assert len(names) == len(set(names))
    for n in ("rb_operator_create", "rb_spmm", "rb_dot", "rb_axpy", "rb_axty", "rb_cg_solve"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    import paper_2508_06710_gb300 as rb

    assert set(_declared()) <= set(rb.SYMBOLS) | {n for n in _declared() if hasattr(lib, n)}
    assert set(rb.SYMBOLS) <= set(_declared())


def test_host_side_validation_without_gpu(lib):
    """Argument checks return RB_EINVAL before touching the device."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    assert lib.rb_version().decode().count(".") == 2
    h = C.c_void_p()
    assert lib.rb_operator_create(None, None, 0, 0, None, C.byref(h)) == rb.RB_EINVAL
    assert b"null" in lib.rb_last_error()
    assert lib.rb_spmm(None, None, 1, None, 1, 1, None, None) == rb.RB_EINVAL
    assert lib.rb_dot(10, 0, 0, None, 1, None, 1, None, None, 0, None) == rb.RB_EINVAL
    assert lib.rb_dot_workspace_bytes(100, 3) > 0 and lib.rb_dot_workspace_bytes(100, 65) == 0
    g = rb.GridDesc()
    for d in range(3):
        g.n[d] = 2
        g.periodic[d] = 1  # a periodic axis needs >= 3 cells
    nr, nc, nnz = C.c_int32(), C.c_int32(), C.c_int64()
    assert lib.rb_fvm_csr_size(C.byref(g), 0, C.byref(nr), C.byref(nc), C.byref(nnz)) == rb.RB_EINVAL
    # an extruded operator whose row 1 stores no diagonal entry (host arrays; refused before
    # any device work, since the spanwise -2 w_i is folded into the stored diagonal)
    rp = (C.c_int32 * 3)(0, 2, 3)
    ci = (C.c_int32 * 3)(0, 1, 0)
    va = (C.c_double * 3)(2.0, -1.0, -1.0)
    zw = (C.c_double * 2)(0.5, 0.5)
    csr = rb.CsrDesc(2, 2, 3, C.addressof(rp), C.addressof(ci), C.addressof(va), 0)
    blk = rb.BlockDesc(3, 3, C.addressof(zw), 0.1)
    assert lib.rb_operator_create(C.byref(csr), C.byref(blk), rb.RB_F64, rb.RB_CSR, None, C.byref(h)) == rb.RB_EINVAL
    assert b"diagonal" in lib.rb_last_error()


def test_stencil_validation_without_gpu(lib):
    """rb_stencil_assemble refuses bad grids before any device work (null outputs here)."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    def call(n, h, kind):
        return lib.rb_stencil_assemble((C.c_int32 * 3)(*n), (C.c_double * 3)(*h), kind, 1.0, None, None, None, None)

    for n, h, kind, msg in (((4, 6, 6), (1, 1, 1), 13, b">= 5 cells"), ((5, 5, 2), (1, 1, 1), 27, b">= 3 cells"),
                            ((5, 5, 5), (1, 1, 2), 27, b"cubic"), ((5, 5, 5), (1, 0, 1), 13, b"positive"),
                            ((5, 5, 5), (1, float("nan"), 1), 13, b"positive"), ((5, 5, 5), (1, 1, 1), 7, b"unknown kind"),
                            ((1000, 1000, 100), (1, 1, 1), 27, b"32-bit"), ((5, 5, 5), (1, 1, 1), 13, b"null output")):
        assert call(n, h, kind) == rb.RB_EINVAL
        assert msg in lib.rb_last_error(), (n, h, kind, lib.rb_last_error())
    assert lib.rb_stencil_assemble(None, None, 13, 1.0, None, None, None, None) == rb.RB_EINVAL


def test_refine_validation_without_gpu(lib):
    """rb_refine_assemble refuses odd or small axes, null node arrays and unknown kinds first."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    nodes = (C.c_double * 9)(*range(9))
    for n, kind, msg in (((8, 7, 8), 0, b"even number"), ((8, 2, 8), 1, b"even number"), ((8, 8, 8), 3, b"unknown kind"),
                         ((8, 8, 8), 0, b"null output"), ((8, 8, 8), 2, b"null output"), ((8, 5, 8), 2, b"even number")):
        g = rb.GridDesc()
        for d in range(3):
            g.n[d] = n[d]
            g.periodic[d] = 1
            g.nodes[d] = C.addressof(nodes)
        assert lib.rb_refine_assemble(C.byref(g), kind, None, None, None, None) == rb.RB_EINVAL
        assert msg in lib.rb_last_error(), (n, kind, lib.rb_last_error())
    g = rb.GridDesc()
    for d in range(3):
        g.n[d] = 8
    assert lib.rb_refine_assemble(C.byref(g), 0, None, None, None, None) == rb.RB_EINVAL
    assert b"null nodes" in lib.rb_last_error()


def test_fvm_sizes_match_oracle(lib):
    """Row, column and nonzero counts of the device builder equal the oracle's (no GPU work)."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb
    import workloads as W
    from oracle import fvm

    for g in (W.unit_periodic_grid(5), W.channel_grid(7, 6, 5), W.rbc_grid(4)):
        gd = rb.GridDesc()
        for d in range(3):
            gd.n[d] = g.axes[d].n
            gd.periodic[d] = 1 if g.axes[d].periodic else 0
        I = fvm.interpolation(g)
        for kind, ref in ((0, fvm.laplacian(g)), (1, fvm.divergence(g)), (2, fvm.gradient(g)), (3, I), (4, I.T.tocsr())):
            nr, nc, nnz = C.c_int32(), C.c_int32(), C.c_int64()
            assert lib.rb_fvm_csr_size(C.byref(gd), kind, C.byref(nr), C.byref(nc), C.byref(nnz)) == 0
            assert (nr.value, nc.value, nnz.value) == (ref.shape[0], ref.shape[1], ref.nnz)


def test_multigrid_validation_without_gpu(lib):
    """rb_mg_create / rb_mg_solve / rb_mg_vcycle refuse bad parameters before any device work."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    nodes = (C.c_double * 9)(*range(9))
    g = rb.GridDesc()
    for d in range(3):
        g.n[d] = 8
        g.periodic[d] = 1
        g.nodes[d] = C.addressof(nodes)
    h = C.c_void_p()
    for k_max, prm, msg in ((0, None, b"k_max"), (65, None, b"k_max"), (3, rb.MgParams(0, 0.5, 4, 1, 1, 1), b"nu"),
                            (3, rb.MgParams(2, 1.5, 4, 1, 1, 1), b"omega"), (3, rb.MgParams(2, 0.5, 1, 1, 1, 1), b"min_cells")):
        st = lib.rb_mg_create(C.byref(g), k_max, None if prm is None else C.byref(prm), None, C.byref(h))
        assert st == rb.RB_EINVAL and msg in lib.rb_last_error(), (k_max, lib.rb_last_error())
        assert not h.value
    g.nodes[1] = None
    assert lib.rb_mg_create(C.byref(g), 1, None, None, C.byref(h)) == rb.RB_EINVAL
    assert b"null nodes" in lib.rb_last_error()
    rep = rb.CgReport()
    assert lib.rb_mg_solve(None, C.byref(rb.mg_params()), None, 1, None, 1, 1, C.byref(rep), None) == rb.RB_EINVAL
    assert lib.rb_mg_vcycle(None, 0, 0, None, 1, None, 1, 1, None) == rb.RB_EINVAL


def test_galerkin_validation_without_gpu(lib):
    """rb_galerkin_guess refuses bad sizes and null arguments before any device work."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    assert lib.rb_galerkin_workspace_bytes(100, 3, 3) > 0
    assert lib.rb_galerkin_workspace_bytes(100, 3, 4) == 0 and lib.rb_galerkin_workspace_bytes(100, 65, 1) == 0
    ptrs = (C.c_void_p * 1)(None)
    lds = (C.c_int64 * 1)(3)
    assert lib.rb_galerkin_guess(None, 3, 1, ptrs, lds, None, 3, None, 3, None, None, 0, None) == rb.RB_EINVAL
    assert b"null operator" in lib.rb_last_error()


def test_double_float_validation_without_gpu(lib):
    """RB_DF64 operators: CSR only, not extruded, values inside FP32's range; the split and join
    calls check their blocks (host arrays: every refusal comes before device work)."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    h = C.c_void_p()
    rp = (C.c_int32 * 3)(0, 2, 3)
    ci = (C.c_int32 * 3)(0, 1, 0)
    va = (C.c_double * 3)(2.0, -1.0, 1e39)
    csr = rb.CsrDesc(2, 2, 3, C.addressof(rp), C.addressof(ci), C.addressof(va), 0)
    assert lib.rb_operator_create(C.byref(csr), None, rb.RB_DF64, rb.RB_SELL, None, C.byref(h)) == rb.RB_EINVAL
    assert b"CSR" in lib.rb_last_error()
    zw = (C.c_double * 2)(0.5, 0.5)
    blk = rb.BlockDesc(3, 3, C.addressof(zw), 0.1)
    assert lib.rb_operator_create(C.byref(csr), C.byref(blk), rb.RB_DF64, rb.RB_CSR, None, C.byref(h)) == rb.RB_EINVAL
    assert b"extruded" in lib.rb_last_error()
    assert lib.rb_operator_create(C.byref(csr), None, rb.RB_DF64, rb.RB_CSR, None, C.byref(h)) == rb.RB_EINVAL
    assert b"FP32 range" in lib.rb_last_error()
    assert lib.rb_operator_create(C.byref(csr), None, 3, rb.RB_CSR, None, C.byref(h)) == rb.RB_EINVAL
    buf = (C.c_double * 64)()
    a = C.addressof(buf)
    assert lib.rb_df64_split(4, 0, a, 1, a + 256, 1, None) == rb.RB_EINVAL  # k = 0
    assert lib.rb_df64_split(4, 2, a, 1, a + 256, 2, None) == rb.RB_EINVAL  # ldx < k
    assert lib.rb_df64_split(4, 2, a, 2, a + 8, 2, None) == rb.RB_EINVAL  # overlapping blocks
    assert b"overlap" in lib.rb_last_error()
    assert lib.rb_df64_join(4, 2, a + 4, 2, a + 256, 2, None) == rb.RB_EINVAL  # misaligned
    assert lib.rb_df64_join(4, 2, None, 2, a, 2, None) == rb.RB_EINVAL
    assert lib.rb_df64_split(0, 2, None, 2, None, 2, None) == rb.RB_OK  # nothing to do


def test_projection_validation_without_gpu(lib):
    """rb_projection_create and rb_projection_step refuse bad arguments before device work."""
    import ctypes as C

    import paper_2508_06710_gb300 as rb

    g = rb.GridDesc()
    for d in range(3):
        g.n[d] = 8
        g.periodic[d] = 1
    h = C.c_void_p()
    good = rb.ProjectionParams(2, 0.01, 0.01, rb.RB_PROJ_MG, rb.mg_params())

    def create(prm, grid=g):
        return lib.rb_projection_create(C.byref(grid), C.byref(prm), None, C.byref(h))

    for bad in (rb.ProjectionParams(0, 0.01, 0.01, 0, rb.mg_params()),     # m < 1
                rb.ProjectionParams(22, 0.01, 0.01, 0, rb.mg_params()),    # 3 m > RB_MAX_K
                rb.ProjectionParams(2, 0.01, 0.0, 0, rb.mg_params()),      # dt = 0
                rb.ProjectionParams(2, -1.0, 0.01, 0, rb.mg_params()),     # nu < 0
                rb.ProjectionParams(2, 0.01, 0.01, 7, rb.mg_params()),     # unknown solver
                rb.ProjectionParams(2, 0.01, 0.01, 0, rb.mg_params(project_mean=False))):
        assert create(bad) == rb.RB_EINVAL
    walled = rb.GridDesc()
    for d in range(3):
        walled.n[d] = 8
        walled.periodic[d] = 1 if d < 2 else 0
    assert create(good, walled) == rb.RB_EINVAL and b"periodic" in lib.rb_last_error()
    assert lib.rb_projection_create(None, C.byref(good), None, C.byref(h)) == rb.RB_EINVAL
    rep = rb.ProjectionReport()
    assert lib.rb_projection_step(None, None, 6, None, 2, C.byref(rep), None) == rb.RB_EINVAL
    assert lib.rb_projection_destroy(None) == rb.RB_OK
