"""Repeated-block SpMM for CFD operators on one GB300 (sm_103a): Python binding.

A thin ctypes layer over the C ABI in include/rbspmm.h: it marshals torch tensors (device
memory, streams) into pointers and sizes and turns status codes into exceptions.  Every
computation runs in the library's CUDA kernels; there is no Python or CPU fallback: if
librbspmm.so is missing the calls raise.

Layout: a block of k right-hand sides is a 2-D tensor (n, k) whose rows are contiguous
(stride (ld, 1), ld >= k): the k columns of one row are interleaved, as in Algorithm 1.  A
double-float block (dtype "df64": FP64 values as pairs hi + lo of FP32 numbers) is a float32
tensor (n, k, 2) with strides (2 ld, 2, 1): the same bytes as an (n, k) float64 block.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbspmm.so")

RB_OK, RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_ENOCONV, RB_EBREAKDOWN, RB_ETIMEOUT, RB_EUNSUPPORTED = range(8)
STATUS_NAMES = ["RB_OK", "RB_EINVAL", "RB_ENOMEM", "RB_ECUDA", "RB_ENOCONV", "RB_EBREAKDOWN", "RB_ETIMEOUT",
                "RB_EUNSUPPORTED"]
RB_F64, RB_F32, RB_DF64 = 0, 1, 2
RB_CSR, RB_SELL, RB_AUTO, RB_STENCIL = 0, 1, 2, 3
RB_FVM_LAPLACIAN, RB_FVM_DIVERGENCE, RB_FVM_GRADIENT, RB_FVM_INTERP_C2S, RB_FVM_INTERP_S2C = 0, 1, 2, 3, 4
RB_STENCIL_13P, RB_STENCIL_27P = 13, 27
RB_REFINE_PROLONG, RB_REFINE_RESTRICT, RB_REFINE_PROLONG_T = 0, 1, 2
RB_MAX_K = 64

# exported C symbols, in the order include/rbspmm.h declares them
SYMBOLS = ["rb_last_error", "rb_version", "rb_fma_peak", "rb_fvm_csr_size", "rb_fvm_assemble", "rb_stencil_assemble",
           "rb_refine_assemble", "rb_mesh_cot_laplacian", "rb_fvm_stencil_create",
           "rb_operator_create", "rb_operator_destroy", "rb_operator_set_row_blocks", "rb_operator_info",
           "rb_operator_check", "rb_spmm", "rb_df64_split", "rb_df64_join",
           "rb_tune_spmm", "rb_set_spmm_schedule", "rb_get_spmm_schedule", "rb_dot_workspace_bytes", "rb_dot",
           "rb_dot_noalloc", "rb_axpy", "rb_axty", "rb_cg_workspace_bytes", "rb_cg_solve", "rb_batch_create", "rb_batch_destroy",
           "rb_batch_solve", "rb_batch_tune", "rb_batch_set_barrier", "rb_guess_param_count", "rb_guess_create",
           "rb_guess_destroy", "rb_guess_init_params", "rb_guess_set_params", "rb_guess_get_params", "rb_guess_get_grad", "rb_guess_predict",
           "rb_guess_loss_grad", "rb_guess_adam_step", "rb_guess_read_activation", "rb_guess_select",
           "rb_mg_create", "rb_mg_destroy", "rb_mg_info", "rb_mg_vcycle", "rb_mg_solve",
           "rb_projection_create", "rb_projection_destroy", "rb_projection_step", "rb_projection_project",
           "rb_galerkin_workspace_bytes", "rb_galerkin_guess"]


class RbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


# ----------------------------------------------------------------------------- C structs
class GridDesc(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("periodic", C.c_int32 * 3), ("nodes", C.c_void_p * 3)]


class CsrDesc(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("vals", C.c_void_p), ("on_device", C.c_int32)]


class BlockDesc(C.Structure):
    _fields_ = [("k_max", C.c_int32), ("extruded_nz", C.c_int32), ("z_weight", C.c_void_p), ("dz", C.c_double)]


class OpInfo(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int64), ("dtype", C.c_int32),
                ("format", C.c_int32), ("sell_c", C.c_int32), ("sell_sigma", C.c_int32),
                ("sell_padded_nnz", C.c_int64), ("device_bytes", C.c_int64), ("has_diag", C.c_int32),
                ("extruded_nz", C.c_int32)]


class SpmmSchedule(C.Structure):
    _fields_ = [("vec", C.c_int32), ("lpr", C.c_int32), ("stage", C.c_int32), ("grid_cap", C.c_int32)]


class MgParams(C.Structure):
    _fields_ = [("nu", C.c_int32), ("omega", C.c_double), ("min_cells", C.c_int32), ("flexible", C.c_int32),
                ("matrix_free", C.c_int32), ("smoother", C.c_int32)]


RB_MG_MAX_LEVELS = 16


class MgInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n", (C.c_int32 * 3) * RB_MG_MAX_LEVELS),
                ("nnz_A", C.c_int64 * RB_MG_MAX_LEVELS), ("nnz_P", C.c_int64 * RB_MG_MAX_LEVELS),
                ("device_bytes", C.c_int64), ("line_axis", C.c_int32)]


class GuessCfg(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("levels", C.c_int32),
                ("channels", C.c_int32 * 4), ("periodic", C.c_int32 * 3)]


class AdamParams(C.Structure):
    _fields_ = [("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double)]


class CgParams(C.Structure):
    _fields_ = [("rtol", C.c_double), ("max_iter", C.c_int32), ("precond", C.c_int32), ("mixed", C.c_int32),
                ("inner_rtol", C.c_double), ("max_sweeps", C.c_int32), ("project_mean", C.c_int32),
                ("check_every", C.c_int32), ("persistent", C.c_int32)]


class CgReport(C.Structure):
    _fields_ = [("iters", C.c_int32 * RB_MAX_K), ("true_rel_res", C.c_double * RB_MAX_K),
                ("status", C.c_int32 * RB_MAX_K), ("spmm_calls", C.c_int32), ("sweeps", C.c_int32),
                ("host_syncs", C.c_int32), ("ms", C.c_double)]


RB_PROJ_JACOBI, RB_PROJ_MG = 0, 1


class ProjectionParams(C.Structure):
    _fields_ = [("m", C.c_int32), ("nu", C.c_double), ("dt", C.c_double), ("solver", C.c_int32), ("cg", CgParams)]


class ProjectionReport(C.Structure):
    _fields_ = [("iters", C.c_int32 * 3), ("status", C.c_int32), ("poisson_ms", C.c_double)]


_lib = None


def lib():
    """The loaded native library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run paper_2508_06710_gb300.build.build() (needs nvcc)")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "rb_last_error": (C.c_char_p, []),
        "rb_version": (C.c_char_p, []),
        "rb_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.c_void_p]),
        "rb_fvm_csr_size": (C.c_int, [C.POINTER(GridDesc), C.c_int, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]),
        "rb_fvm_assemble": (C.c_int, [C.POINTER(GridDesc), C.c_int, dbl, vp, vp, vp, vp]),
        "rb_stencil_assemble": (C.c_int, [C.POINTER(i32), C.POINTER(dbl), C.c_int, dbl, vp, vp, vp, vp]),
        "rb_refine_assemble": (C.c_int, [C.POINTER(GridDesc), C.c_int, vp, vp, vp, vp]),
        "rb_mesh_cot_laplacian": (C.c_int, [i32, vp, i32, vp, vp, vp, i64, vp, vp, vp, vp]),
        "rb_operator_create": (C.c_int, [C.POINTER(CsrDesc), C.POINTER(BlockDesc), C.c_int, C.c_int, vp,
                                         C.POINTER(vp)]),
        "rb_fvm_stencil_create": (C.c_int, [C.POINTER(GridDesc), dbl, C.c_int, i32, vp, C.POINTER(vp)]),
        "rb_operator_destroy": (C.c_int, [vp]),
        "rb_operator_set_row_blocks": (C.c_int, [vp, i32, C.POINTER(i32)]),
        "rb_operator_info": (C.c_int, [vp, C.POINTER(OpInfo)]),
        "rb_spmm": (C.c_int, [vp, vp, i64, vp, i64, i32, vp, vp]),
        "rb_df64_split": (C.c_int, [i64, i32, vp, i64, vp, i64, vp]),
        "rb_df64_join": (C.c_int, [i64, i32, vp, i64, vp, i64, vp]),
        "rb_tune_spmm": (C.c_int, [vp, vp, i64, vp, i64, i32, vp]),
        "rb_set_spmm_schedule": (C.c_int, [vp, i32, C.POINTER(SpmmSchedule)]),
        "rb_get_spmm_schedule": (C.c_int, [vp, i32, i64, i64, vp, vp, C.POINTER(SpmmSchedule)]),
        "rb_operator_check": (C.c_int, [vp, vp]),
        "rb_dot_workspace_bytes": (sz, [i64, i32]),
        "rb_dot": (C.c_int, [i64, i32, C.c_int, vp, i64, vp, i64, vp, vp, sz, vp]),
        "rb_dot_noalloc": (C.c_int, [i64, i32, C.c_int, vp, i64, vp, i64, vp, vp]),
        "rb_axpy": (C.c_int, [i64, i32, C.c_int, vp, vp, i64, vp, i64, vp]),
        "rb_axty": (C.c_int, [i64, i32, C.c_int, dbl, vp, i64, vp, i64, vp]),
        "rb_cg_workspace_bytes": (sz, [vp, i32, C.POINTER(CgParams)]),
        "rb_cg_solve": (C.c_int, [vp, vp, C.POINTER(CgParams), vp, i64, vp, i64, i32, vp, sz, C.POINTER(CgReport),
                                  vp]),
        "rb_batch_create": (C.c_int, [i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(i32), C.POINTER(CgParams),
                                      C.POINTER(vp)]),
        "rb_batch_destroy": (C.c_int, [vp]),
        "rb_batch_solve": (C.c_int, [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(i64),
                                     C.POINTER(CgReport), vp]),
        "rb_batch_tune": (C.c_int, [vp, C.POINTER(vp), C.POINTER(i64), C.POINTER(vp), C.POINTER(i64),
                                    C.POINTER(C.c_double), vp]),
        "rb_batch_set_barrier": (C.c_int, [vp, C.c_double, i32]),
        "rb_guess_param_count": (C.c_int, [C.POINTER(GuessCfg), C.POINTER(i64)]),
        "rb_guess_create": (C.c_int, [C.POINTER(GuessCfg), C.POINTER(vp)]),
        "rb_guess_destroy": (C.c_int, [vp]),
        "rb_guess_init_params": (C.c_int, [vp, vp, dbl, vp]),
        "rb_guess_set_params": (C.c_int, [vp, vp, vp]),
        "rb_guess_get_params": (C.c_int, [vp, vp, vp]),
        "rb_guess_get_grad": (C.c_int, [vp, vp, vp]),
        "rb_guess_predict": (C.c_int, [vp, vp, vp, vp, vp, vp]),
        "rb_guess_loss_grad": (C.c_int, [vp, vp, vp, vp, vp, i32, vp, vp]),
        "rb_guess_adam_step": (C.c_int, [vp, C.POINTER(AdamParams), dbl, vp]),
        "rb_guess_read_activation": (C.c_int, [vp, i32, vp, C.POINTER(i64), vp]),
        "rb_guess_select": (C.c_int, [vp, vp, vp, vp, vp, i32, dbl, vp, vp, vp, vp]),
        "rb_mg_create": (C.c_int, [C.POINTER(GridDesc), i32, C.POINTER(MgParams), vp, C.POINTER(vp)]),
        "rb_mg_destroy": (C.c_int, [vp]),
        "rb_mg_info": (C.c_int, [vp, C.POINTER(MgInfo)]),
        "rb_mg_vcycle": (C.c_int, [vp, i32, C.c_int, vp, i64, vp, i64, i32, vp]),
        "rb_mg_solve": (C.c_int, [vp, C.POINTER(CgParams), vp, i64, vp, i64, i32, C.POINTER(CgReport), vp]),
        "rb_projection_create": (C.c_int, [C.POINTER(GridDesc), C.POINTER(ProjectionParams), vp, C.POINTER(vp)]),
        "rb_projection_destroy": (C.c_int, [vp]),
        "rb_projection_step": (C.c_int, [vp, vp, i64, vp, i64, C.POINTER(ProjectionReport), vp]),
        "rb_projection_project": (C.c_int, [vp, C.c_double, vp, i64, vp, i64, C.POINTER(ProjectionReport), vp]),
        "rb_galerkin_workspace_bytes": (sz, [i64, i32, i32]),
        "rb_galerkin_guess": (C.c_int, [vp, i32, i32, C.POINTER(vp), C.POINTER(i64), vp, i64, vp, i64, vp, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int, what: str):
    if status != RB_OK:
        raise RbError(status, f"{what}: {lib().rb_last_error().decode()}")


def version() -> str:
    return lib().rb_version().decode()


def fma_peak(dtype="f64", stream=None) -> float:
    """Measured FMA throughput of the GPU in TFLOP/s (rb_fma_peak)."""
    v = C.c_double()
    _check(lib().rb_fma_peak({"f64": RB_F64, "f32": RB_F32}[dtype], C.byref(v), _stream(stream)), "rb_fma_peak")
    return v.value


# ----------------------------------------------------------------------------- tensor helpers
def _torch():
    import torch

    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _block(t, name, pairs=False):
    """(tensor, n, k, ld) of a row-major 2-D block whose rows are contiguous, or (pairs) of a
    double-float block (float32, (n, k, 2), strides (2 ld, 2, 1)); ld in elements (pairs)."""
    if pairs:
        torch = _torch()
        if t.dim() != 3 or t.dtype != torch.float32 or t.shape[2] != 2 or t.stride(2) != 1 or t.stride(1) != 2 or t.stride(0) % 2:
            raise ValueError(f"{name}: a double-float block is float32 (n, k, 2) with strides (2 ld, 2, 1)")
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        return t, t.shape[0], t.shape[1], max(t.stride(0) // 2, t.shape[1])
    if t.dim() == 3:
        raise ValueError(f"{name}: a double-float block goes only to a df64 operator or df_join")
    if t.dim() == 1:
        t = t.view(-1, 1)
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D tensor with contiguous rows (stride (ld, 1))")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    return t, t.shape[0], t.shape[1], max(t.stride(0), t.shape[1])


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return RB_F64
    if t.dtype == torch.float32:
        return RB_F32
    raise ValueError("blocks must be float64 or float32")


# ----------------------------------------------------------------------------- operator build
def _grid_desc(nodes, periodic):
    g = GridDesc()
    for d in range(3):
        g.n[d] = int(nodes[d].numel() - 1)
        g.periodic[d] = 1 if periodic[d] else 0
        g.nodes[d] = nodes[d].data_ptr()
    return g


def fvm_csr_size(nodes, periodic, kind):
    g = _grid_desc(nodes, periodic)
    nr, nc, nnz = C.c_int32(), C.c_int32(), C.c_int64()
    _check(lib().rb_fvm_csr_size(C.byref(g), kind, C.byref(nr), C.byref(nc), C.byref(nnz)), "rb_fvm_csr_size")
    return nr.value, nc.value, nnz.value


def fvm_assemble(nodes, periodic, kind, scale=1.0, stream=None):
    """CSR (row_ptr, col_idx, vals, n_cols) of the staggered FVM operator on the grid whose axis
    node coordinates are the float64 CUDA tensors ``nodes`` (x, y, z)."""
    torch = _torch()
    nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
    nr, nc, nnz = fvm_csr_size(nodes, periodic, kind)
    dev = nodes[0].device
    rp = torch.empty(nr + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(nnz, dtype=torch.int32, device=dev)
    va = torch.empty(nnz, dtype=torch.float64, device=dev)
    g = _grid_desc(nodes, periodic)
    _check(lib().rb_fvm_assemble(C.byref(g), kind, float(scale), _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)),
           "rb_fvm_assemble")
    return rp, ci, va, nc


def stencil_assemble(shape, h, kind, scale=1.0, device="cuda", stream=None):
    """CSR (row_ptr, col_idx, vals, n) of the 13p or 27p Laplacian (``RB_STENCIL_13P`` /
    ``RB_STENCIL_27P``) on the uniform periodic grid of ``shape`` cells with spacings ``h``."""
    torch = _torch()
    n_arr = (C.c_int32 * 3)(*[int(v) for v in shape])
    h_arr = (C.c_double * 3)(*[float(v) for v in h])
    rows = int(shape[0]) * int(shape[1]) * int(shape[2])
    rp = torch.empty(rows + 1, dtype=torch.int32, device=device)
    ci = torch.empty(int(kind) * rows, dtype=torch.int32, device=device)
    va = torch.empty(int(kind) * rows, dtype=torch.float64, device=device)
    _check(lib().rb_stencil_assemble(n_arr, h_arr, int(kind), float(scale), _ptr(rp), _ptr(ci), _ptr(va),
                                     _stream(stream)), "rb_stencil_assemble")
    return rp, ci, va, rows


def refine_assemble(nodes, periodic, kind, stream=None):
    """CSR (row_ptr, col_idx, vals, n_cols) of the prolongation (``RB_REFINE_PROLONG``, fine x
    coarse), the restriction (``RB_REFINE_RESTRICT``, coarse x fine) or the transposed
    prolongation (``RB_REFINE_PROLONG_T``, coarse x fine) between the grid whose axis node
    coordinates are the float64 CUDA tensors ``nodes`` and its 2:1 coarsening."""
    torch = _torch()
    nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
    n_fine = 1
    for n in nodes:
        n_fine *= int(n.numel() - 1)
    rows, cols = (n_fine, n_fine // 8) if kind == RB_REFINE_PROLONG else (n_fine // 8, n_fine)
    dev = nodes[0].device
    rp = torch.empty(rows + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(8 * n_fine if kind == RB_REFINE_PROLONG_T else 8 * rows, dtype=torch.int32, device=dev)
    va = torch.empty(ci.numel(), dtype=torch.float64, device=dev)
    g = _grid_desc(nodes, periodic)
    _check(lib().rb_refine_assemble(C.byref(g), int(kind), _ptr(rp), _ptr(ci), _ptr(va), _stream(stream)),
           "rb_refine_assemble")
    return rp, ci, va, cols


def grid_nodes(grid, device="cuda"):
    """Device node tensors and periodic flags of a ``workloads.Grid``."""
    torch = _torch()
    nodes = [torch.as_tensor(a.nodes, dtype=torch.float64, device=device) for a in grid.axes]
    return nodes, [a.periodic for a in grid.axes]


def mesh_cot_laplacian(points, triangles, row_ptr, col_idx, stream=None):
    """Values and dual areas of the cotangent Laplacian on the given adjacency pattern.
    Returns (vals, area, status) with status a device int64[2] (clamped edges, pattern error)."""
    torch = _torch()
    dev = points.device
    n = points.shape[0]
    nnz = col_idx.numel()
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    area = torch.empty(n, dtype=torch.float64, device=dev)
    status = torch.empty(2, dtype=torch.int64, device=dev)
    _check(lib().rb_mesh_cot_laplacian(n, _ptr(points.contiguous()), triangles.shape[0], _ptr(triangles.contiguous()),
                                       _ptr(row_ptr), _ptr(col_idx), nnz, _ptr(vals), _ptr(area), _ptr(status),
                                       _stream(stream)), "rb_mesh_cot_laplacian")
    return vals, area, status


# ----------------------------------------------------------------------------- operators
class Operator:
    """A = I_k (x) A~ stored once on the device (CSR or sliced ELL, FP64 or FP32; CSR as
    double-float pairs with dtype "df64")."""

    def __init__(self, row_ptr, col_idx, vals, n_cols, dtype="f64", fmt="csr", k_max=1, extruded_nz=0,
                 z_weight=None, dz=0.0, stream=None):
        torch = _torch()
        on_dev = bool(row_ptr.is_cuda)
        self._keep = (row_ptr.to(torch.int32).contiguous(), col_idx.to(torch.int32).contiguous(),
                      vals.to(torch.float64).contiguous(),
                      None if z_weight is None else z_weight.to(torch.float64).contiguous())
        rp, ci, va, zw = self._keep
        d = CsrDesc(rp.numel() - 1, int(n_cols), ci.numel(), rp.data_ptr(), ci.data_ptr() if ci.numel() else None,
                    va.data_ptr() if va.numel() else None, 1 if on_dev else 0)
        b = BlockDesc(int(k_max), int(extruded_nz), None if zw is None else zw.data_ptr(), float(dz))
        h = C.c_void_p()
        dt = {"f64": RB_F64, "f32": RB_F32, "df64": RB_DF64}[dtype]
        fm = {"csr": RB_CSR, "sell": RB_SELL, "auto": RB_AUTO}[fmt]
        _check(lib().rb_operator_create(C.byref(d), C.byref(b), dt, fm, _stream(stream) if on_dev else None,
                                        C.byref(h)), "rb_operator_create")
        self.handle = h
        self.dtype = dtype
        self._keep = None
        inf = self.info()
        self.n_rows, self.n_cols, self.nnz = inf.n_rows, inf.n_cols, inf.nnz
        self.extruded_nz = inf.extruded_nz

    @classmethod
    def stencil(cls, nodes, periodic, scale=1.0, dtype="f64", k_max=1, stream=None):
        """The FVM Laplacian of the grid times `scale` as a matrix-free operator (rb_fvm_stencil_create):
        per-axis tables instead of stored entries."""
        torch = _torch()
        nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
        g = _grid_desc(nodes, periodic)
        h = C.c_void_p()
        _check(lib().rb_fvm_stencil_create(C.byref(g), float(scale), {"f64": RB_F64, "f32": RB_F32, "df64": RB_DF64}[dtype],
                                           int(k_max), _stream(stream), C.byref(h)), "rb_fvm_stencil_create")
        self = cls.__new__(cls)
        self.handle = h
        self.dtype = dtype
        self._keep = None
        inf = self.info()
        self.n_rows, self.n_cols, self.nnz = inf.n_rows, inf.n_cols, inf.nnz
        self.extruded_nz = 0
        return self

    @classmethod
    def from_scipy(cls, A, **kw):
        torch = _torch()
        A = A.tocsr()
        return cls(torch.as_tensor(A.indptr.astype("int32")), torch.as_tensor(A.indices.astype("int32")),
                   torch.as_tensor(A.data.astype("float64")), A.shape[1], **kw)

    def info(self) -> OpInfo:
        inf = OpInfo()
        _check(lib().rb_operator_info(self.handle, C.byref(inf)), "rb_operator_info")
        return inf

    def _blocks(self, X, Y):
        """Checks that X and Y hold the operator's type: float64 (f64), float32 (f32) or
        double-float pairs (df64)."""
        torch = _torch()
        pairs = self.dtype == "df64"
        want = torch.float32 if self.dtype in ("f32", "df64") else torch.float64
        X, _, k, ldx = _block(X, "X", pairs)
        Y, _, _, ldy = _block(Y, "Y", pairs)
        if X.dtype != want or Y.dtype != want:
            raise ValueError(f"X and Y must be {want} blocks for a {self.dtype} operator")
        return X, k, ldx, Y, ldy

    def spmm(self, X, Y=None, c=None, stream=None):
        torch = _torch()
        if Y is None:
            shape = (self.n_rows, X.shape[1], 2) if self.dtype == "df64" else (self.n_rows, X.shape[1] if X.dim() > 1 else 1)
            Y = torch.empty(shape, dtype=X.dtype, device=X.device)
        X, k, ldx, Y, ldy = self._blocks(X, Y)
        _check(lib().rb_spmm(self.handle, _ptr(X), ldx, _ptr(Y), ldy, k, _ptr(c), _stream(stream)), "rb_spmm")
        return Y

    def tune(self, X, Y, stream=None):
        X, k, ldx, Y, ldy = self._blocks(X, Y)
        _check(lib().rb_tune_spmm(self.handle, _ptr(X), ldx, _ptr(Y), ldy, k, _stream(stream)), "rb_tune_spmm")

    def set_schedule(self, k, vec, lpr=1, stage=0, grid_cap=-1):
        s = SpmmSchedule(vec, lpr, stage, grid_cap)
        _check(lib().rb_set_spmm_schedule(self.handle, k, C.byref(s)), "rb_set_spmm_schedule")

    def schedule(self, X, Y):
        X, k, ldx, Y, ldy = self._blocks(X, Y)
        s = SpmmSchedule()
        _check(lib().rb_get_spmm_schedule(self.handle, k, ldx, ldy, _ptr(X), _ptr(Y), C.byref(s)),
               "rb_get_spmm_schedule")
        return {"vec": s.vec, "lpr": s.lpr, "stage": s.stage, "grid_cap": s.grid_cap}

    def set_row_blocks(self, starts):
        """Rows in len(starts) blocks starting at these rows that address the same columns in order
        (rb_operator_set_row_blocks); [] or [0] removes the hint."""
        starts = [int(v) for v in starts] or [0]
        _check(lib().rb_operator_set_row_blocks(self.handle, len(starts), (C.c_int32 * len(starts))(*starts)),
               "rb_operator_set_row_blocks")

    def check(self, stream=None):
        """Raises RbError(RB_ETIMEOUT) if a pipelined SpMM kernel gave up a bounded wait."""
        _check(lib().rb_operator_check(self.handle, _stream(stream)), "rb_operator_check")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().rb_operator_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- double-float blocks
def df_split(X, out=None, stream=None):
    """The double-float block (float32 (n, k, 2)) of the float64 block X (rb_df64_split)."""
    torch = _torch()
    X, n, k, ldx = _block(X, "X")
    if X.dtype != torch.float64:
        raise ValueError("X must be a float64 block")
    if out is None:
        out = torch.empty((n, k, 2), dtype=torch.float32, device=X.device)
    out, nd, kd, ldd = _block(out, "out", pairs=True)
    if nd != n or kd != k:
        raise ValueError("out must be a double-float block of X's shape")
    _check(lib().rb_df64_split(n, k, _ptr(X), ldx, _ptr(out), ldd, _stream(stream)), "rb_df64_split")
    return out


def df_join(D, out=None, stream=None):
    """The float64 block hi + lo of the double-float block D (rb_df64_join)."""
    torch = _torch()
    D, n, k, ldd = _block(D, "D", pairs=True)
    if out is None:
        out = torch.empty((n, k), dtype=torch.float64, device=D.device)
    out, no, ko, ldx = _block(out, "out")
    if out.dtype != torch.float64 or no != n or ko != k:
        raise ValueError("out must be a float64 block of D's shape")
    _check(lib().rb_df64_join(n, k, _ptr(D), ldd, _ptr(out), ldx, _stream(stream)), "rb_df64_join")
    return out


# ----------------------------------------------------------------------------- basic operations
def dot(X, Y, out=None, work=None, stream=None):
    torch = _torch()
    X, n, k, ldx = _block(X, "X")
    Y, _, _, ldy = _block(Y, "Y")
    if out is None:
        out = torch.empty(k, dtype=torch.float64, device=X.device)
    wb = lib().rb_dot_workspace_bytes(n, k)
    if work is None:
        work = torch.empty(wb, dtype=torch.uint8, device=X.device)
    _check(lib().rb_dot(n, k, _dtype_code(X), _ptr(X), ldx, _ptr(Y), ldy, _ptr(out), _ptr(work), work.numel(),
                        _stream(stream)), "rb_dot")
    return out


def dot_noalloc(X, Y, out, stream=None):
    """Per-column dot products without a workspace (see rb_dot_noalloc): for callers that
    cannot give the library device memory.  `out` (k float64 on the device) is caller-owned."""
    X, n, k, ldx = _block(X, "X")
    Y, _, _, ldy = _block(Y, "Y")
    _check(lib().rb_dot_noalloc(n, k, _dtype_code(X), _ptr(X), ldx, _ptr(Y), ldy, _ptr(out), _stream(stream)),
           "rb_dot_noalloc")
    return out


def axpy(alpha, X, Y, stream=None):
    X, n, k, ldx = _block(X, "X")
    Y, _, _, ldy = _block(Y, "Y")
    _check(lib().rb_axpy(n, k, _dtype_code(X), _ptr(alpha), _ptr(X), ldx, _ptr(Y), ldy, _stream(stream)), "rb_axpy")
    return Y


def axty(alpha, X, Y, stream=None):
    X, n, k, ldx = _block(X, "X")
    Y, _, _, ldy = _block(Y, "Y")
    _check(lib().rb_axty(n, k, _dtype_code(X), float(alpha), _ptr(X), ldx, _ptr(Y), ldy, _stream(stream)),
           "rb_axty")
    return Y


def galerkin_guess(A: "Operator", B, cands, X0=None, coef=None, work=None, stream=None):
    """X0 = the combination of the candidate blocks (each (n, k), float64, CUDA) with the
    smallest energy-norm error for A X = B, column by column (rb_galerkin_guess).  X0 may be
    one of the candidates; coef (k x len(cands) float64, CUDA) receives the coefficients."""
    torch = _torch()
    B, n, k, ldb = _block(B, "B")
    cs = [_block(c, "candidate") for c in cands]
    for c in cs:
        if c[1] != n or c[2] != k:
            raise ValueError("every candidate must have the shape of B")
    if X0 is None:
        X0 = torch.empty((n, k), dtype=torch.float64, device=B.device)
    X0, nx, kx, ldx = _block(X0, "X0")
    if nx != n or kx != k:
        raise ValueError("X0 must have the shape of B")
    nc = len(cs)
    wb = lib().rb_galerkin_workspace_bytes(n, k, nc)
    if work is None:
        work = torch.empty(wb, dtype=torch.uint8, device=B.device)
    ptrs = (C.c_void_p * nc)(*[c[0].data_ptr() for c in cs])
    lds = (C.c_int64 * nc)(*[c[3] for c in cs])
    _check(lib().rb_galerkin_guess(A.handle, k, nc, ptrs, lds, _ptr(B), ldb, _ptr(X0), ldx, _ptr(coef), _ptr(work),
                                   work.numel(), _stream(stream)), "rb_galerkin_guess")
    return X0


# ----------------------------------------------------------------------------- Poisson solve
@dataclass
class CgResult:
    status: int
    iters: list
    true_rel_res: list
    col_status: list
    spmm_calls: int
    sweeps: int
    host_syncs: int
    ms: float
    extra: dict = field(default_factory=dict)


def cg_params(rtol=1e-10, max_iter=20000, precond=True, mixed=False, inner_rtol=None, max_sweeps=60,
              project_mean=False, check_every=32, persistent=False) -> CgParams:
    """mixed: False/0 = FP64 CG, 1 (or True) = restarted FP32-inner refinement, 2 = refinement
    with reliable updates (the search direction survives each sweep).  persistent: each sweep's
    inner iterations in one cooperative launch (refinement only)."""
    m = int(mixed)
    if inner_rtol is None:  # measured best on the channel and 128^3 Poisson problems (see the design notes)
        inner_rtol = 5e-2 if m == 2 else 1e-4
    return CgParams(rtol, max_iter, 1 if precond else 0, m, inner_rtol, max_sweeps, 1 if project_mean else 0,
                    check_every, 1 if persistent else 0)


def cg_workspace_bytes(A: Operator, k: int, params: CgParams) -> int:
    return int(lib().rb_cg_workspace_bytes(A.handle, k, C.byref(params)))


def cg_solve(A: Operator, B, X, A_inner: Operator | None = None, params: CgParams | None = None, work=None,
             stream=None, raise_on_fail=False) -> CgResult:
    """Solves A X[:, j] = B[:, j] for every column j; X holds the initial guess on entry."""
    torch = _torch()
    params = params or cg_params()
    B, n, k, ldb = _block(B, "B")
    X, _, _, ldx = _block(X, "X")
    wb = cg_workspace_bytes(A, k, params)
    if work is None:
        work = torch.empty(wb, dtype=torch.uint8, device=X.device)
    rep = CgReport()
    st = lib().rb_cg_solve(A.handle, None if A_inner is None else A_inner.handle, C.byref(params), _ptr(B), ldb,
                           _ptr(X), ldx, k, _ptr(work), work.numel(), C.byref(rep), _stream(stream))
    if st not in (RB_OK, RB_ENOCONV, RB_EBREAKDOWN) or (raise_on_fail and st != RB_OK):
        _check(st, "rb_cg_solve")
    return CgResult(st, list(rep.iters[:k]), list(rep.true_rel_res[:k]), list(rep.status[:k]), rep.spmm_calls,
                    rep.sweeps, rep.host_syncs, rep.ms)


class Batch:
    """Uneven Poisson systems solved together: one persistent launch per refinement sweep,
    the whole solve recorded once as a CUDA graph and replayed per call."""

    def __init__(self, ops, ops_inner, ks, params: CgParams):
        n = len(ops)
        self._ops = list(ops) + list(ops_inner)  # keep the operators alive
        self.ks = [int(k) for k in ks]
        self.n_sys = n
        h = C.c_void_p()
        _check(lib().rb_batch_create(n, (C.c_void_p * n)(*[o.handle.value for o in ops]),
                                     (C.c_void_p * n)(*[o.handle.value for o in ops_inner]),
                                     (C.c_int32 * n)(*self.ks), C.byref(params), C.byref(h)), "rb_batch_create")
        self.handle = h

    def _arrays(self, Bs, Xs):
        n = self.n_sys
        bb = [_block(b, "B") for b in Bs]
        xx = [_block(x, "X") for x in Xs]
        return ((C.c_void_p * n)(*[b[0].data_ptr() for b in bb]), (C.c_int64 * n)(*[b[3] for b in bb]),
                (C.c_void_p * n)(*[x[0].data_ptr() for x in xx]), (C.c_int64 * n)(*[x[3] for x in xx]))

    def solve(self, Bs, Xs, stream=None):
        pB, lB, pX, lX = self._arrays(Bs, Xs)
        reps = (CgReport * self.n_sys)()
        st = lib().rb_batch_solve(self.handle, pB, lB, pX, lX, reps, _stream(stream))
        if st not in (RB_OK, RB_ENOCONV, RB_EBREAKDOWN, RB_ETIMEOUT):
            _check(st, "rb_batch_solve")
        out = []
        for i, r in enumerate(reps):
            k = self.ks[i]
            out.append(CgResult(st, list(r.iters[:k]), list(r.true_rel_res[:k]), list(r.status[:k]), r.spmm_calls,
                                r.sweeps, r.host_syncs, r.ms))
        return out

    def tune(self, Bs, Xs, stream=None):
        pB, lB, pX, lX = self._arrays(Bs, Xs)
        ms = C.c_double()
        _check(lib().rb_batch_tune(self.handle, pB, lB, pX, lX, C.byref(ms), _stream(stream)), "rb_batch_tune")
        return ms.value

    def set_barrier(self, timeout_ms=2000.0, extra_arrivals=0):
        _check(lib().rb_batch_set_barrier(self.handle, float(timeout_ms), int(extra_arrivals)), "rb_batch_set_barrier")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().rb_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multigrid:
    """Geometric multigrid hierarchy of -L on a Cartesian grid (rb_mg_create): the V-cycle
    preconditioner and the multigrid-preconditioned CG solve of the pressure equation."""

    def __init__(self, nodes, periodic, k_max=1, nu=2, omega=0.8, min_cells=4, flexible=True, matrix_free=True,
                 smoother="line", stream=None):
        torch = _torch()
        self._nodes = [n.to(dtype=torch.float64).contiguous() for n in nodes]
        g = _grid_desc(self._nodes, periodic)
        prm = MgParams(int(nu), float(omega), int(min_cells), 1 if flexible else 0, 1 if matrix_free else 0,
                       {"jacobi": 0, "line": 1}[smoother])
        h = C.c_void_p()
        _check(lib().rb_mg_create(C.byref(g), int(k_max), C.byref(prm), _stream(stream), C.byref(h)), "rb_mg_create")
        self.handle = h
        self.k_max = int(k_max)
        inf = self.info()
        self.levels = inf.levels
        self.line_axis = inf.line_axis
        self.shapes = [tuple(inf.n[l][d] for d in range(3)) for l in range(inf.levels)]
        self.n = self.shapes[0][0] * self.shapes[0][1] * self.shapes[0][2]

    def info(self) -> MgInfo:
        inf = MgInfo()
        _check(lib().rb_mg_info(self.handle, C.byref(inf)), "rb_mg_info")
        return inf

    def vcycle(self, R, Z=None, level=0, dtype="f64", stream=None):
        """Z = B_level R (one V-cycle on that level); R, Z float64 (n_level, k) CUDA blocks."""
        torch = _torch()
        R, n, k, ldr = _block(R, "R")
        sh = self.shapes[level] if 0 <= level < self.levels else None
        if sh is None or n != sh[0] * sh[1] * sh[2]:
            raise ValueError(f"R must have one row per cell of level {level} ({sh})")
        if Z is None:
            Z = torch.empty((n, k), dtype=torch.float64, device=R.device)
        Z, nz, _, ldz = _block(Z, "Z")
        if nz != n or Z.shape[1] != k:
            raise ValueError("Z must have the shape of R")
        _check(lib().rb_mg_vcycle(self.handle, int(level), {"f64": RB_F64, "f32": RB_F32}[dtype], _ptr(R), ldr,
                                  _ptr(Z), ldz, k, _stream(stream)), "rb_mg_vcycle")
        return Z

    def solve(self, B, X, params: CgParams | None = None, stream=None, raise_on_fail=False) -> CgResult:
        """Solves -L X[:, j] = B[:, j] (X holds the initial guess on entry)."""
        params = params or mg_params()
        B, n, k, ldb = _block(B, "B")
        X, nx, kx, ldx = _block(X, "X")
        if n != self.n or nx != self.n or kx != k:
            raise ValueError(f"B and X must be ({self.n}, k) blocks of the same k")
        rep = CgReport()
        st = lib().rb_mg_solve(self.handle, C.byref(params), _ptr(B), ldb, _ptr(X), ldx, k, C.byref(rep),
                               _stream(stream))
        if st not in (RB_OK, RB_ENOCONV, RB_EBREAKDOWN) or (raise_on_fail and st != RB_OK):
            _check(st, "rb_mg_solve")
        return CgResult(st, list(rep.iters[:k]), list(rep.true_rel_res[:k]), list(rep.status[:k]), rep.spmm_calls,
                        rep.sweeps, rep.host_syncs, rep.ms)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().rb_mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_params(rtol=1e-10, max_iter=500, mixed=True, inner_rtol=1e-4, max_sweeps=30, project_mean=True,
              check_every=4) -> CgParams:
    """Parameters of Multigrid.solve: mixed = FP32 cycle and CG inside FP64 refinement."""
    return CgParams(rtol, max_iter, 1, 1 if mixed else 0, inner_rtol, max_sweeps, 1 if project_mean else 0,
                    check_every, 0)


def guess_cfg(nx, ny, nz, channels=(8, 16, 32, 48), periodic=(1, 1, 0)) -> GuessCfg:
    """Network of len(channels) levels on an nx x ny x nz grid (x fastest); periodic = (x, y, z)."""
    ch = list(channels) + [0] * (4 - len(channels))
    return GuessCfg(nx, ny, nz, len(channels), (C.c_int32 * 4)(*ch), (C.c_int32 * 3)(*periodic))


def guess_param_count(cfg: GuessCfg) -> int:
    n = C.c_int64()
    _check(lib().rb_guess_param_count(C.byref(cfg), C.byref(n)), "rb_guess_param_count")
    return n.value


class Guess:
    """The learned initial guess network (3-D U-Net) of one grid: parameters, Adam state and
    activation buffers live in the library; vectors are FP64 device tensors of n cells."""

    def __init__(self, cfg: GuessCfg):
        self.cfg = cfg
        self.n_params = guess_param_count(cfg)
        self.n = cfg.nx * cfg.ny * cfg.nz
        h = C.c_void_p()
        _check(lib().rb_guess_create(C.byref(cfg), C.byref(h)), "rb_guess_create")
        self.handle = h

    def init_params(self, normals, head_scale=1.0, stream=None):
        """He initialisation from given N(0, 1) draws (float32 device tensor, n_params entries)."""
        assert normals.dtype == _torch().float32 and normals.numel() == self.n_params and normals.is_contiguous()
        _check(lib().rb_guess_init_params(self.handle, _ptr(normals), float(head_scale), _stream(stream)),
               "rb_guess_init_params")

    def set_params(self, theta, stream=None):
        assert theta.dtype == _torch().float32 and theta.numel() == self.n_params and theta.is_contiguous()
        _check(lib().rb_guess_set_params(self.handle, _ptr(theta), _stream(stream)), "rb_guess_set_params")

    def params(self, stream=None):
        t = _torch().empty(self.n_params, dtype=_torch().float32, device="cuda")
        _check(lib().rb_guess_get_params(self.handle, _ptr(t), _stream(stream)), "rb_guess_get_params")
        return t

    def grad(self, stream=None):
        t = _torch().empty(self.n_params, dtype=_torch().float32, device="cuda")
        _check(lib().rb_guess_get_grad(self.handle, _ptr(t), _stream(stream)), "rb_guess_get_grad")
        return t

    def _vec(self, v, name):
        assert v.dtype == _torch().float64 and v.is_cuda and v.numel() == self.n and v.is_contiguous(), name
        return _ptr(v)

    def predict(self, b, p1, p2, out=None, stream=None):
        out = _torch().empty(self.n, dtype=_torch().float64, device="cuda") if out is None else out
        _check(lib().rb_guess_predict(self.handle, self._vec(b, "b"), self._vec(p1, "p1"), self._vec(p2, "p2"),
                                      self._vec(out, "out"), _stream(stream)), "rb_guess_predict")
        return out

    def loss_grad(self, b, p1, p2, p, accumulate=False, loss=None, stream=None):
        _check(lib().rb_guess_loss_grad(self.handle, self._vec(b, "b"), self._vec(p1, "p1"), self._vec(p2, "p2"),
                                        self._vec(p, "p"), int(bool(accumulate)), _ptr(loss), _stream(stream)),
               "rb_guess_loss_grad")

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0, stream=None):
        h = AdamParams(lr, beta1, beta2, eps)
        _check(lib().rb_guess_adam_step(self.handle, C.byref(h), float(grad_scale), _stream(stream)),
               "rb_guess_adam_step")

    def activation(self, index, stream=None):
        n = C.c_int64()
        _check(lib().rb_guess_read_activation(self.handle, index, None, C.byref(n), _stream(stream)),
               "rb_guess_read_activation")
        t = _torch().empty(n.value, dtype=_torch().float32, device="cuda")
        _check(lib().rb_guess_read_activation(self.handle, index, _ptr(t), C.byref(n), _stream(stream)),
               "rb_guess_read_activation")
        return t

    def select(self, A: Operator, b, cand0, cand1, x0, sweeps=0, omega=2.0 / 3.0, stream=None):
        """x0 = the candidate (after `sweeps` damped Jacobi sweeps) with the smaller residual;
        returns (res tensor[2], choice tensor[1]) on the device."""
        torch = _torch()
        res = torch.empty(2, dtype=torch.float64, device="cuda")
        choice = torch.empty(1, dtype=torch.int32, device="cuda")
        _check(lib().rb_guess_select(self.handle, A.handle, self._vec(b, "b"), self._vec(cand0, "c0"),
                                     self._vec(cand1, "c1"), int(sweeps), float(omega), self._vec(x0, "x0"),
                                     _ptr(res), _ptr(choice), _stream(stream)), "rb_guess_select")
        return res, choice

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().rb_guess_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
