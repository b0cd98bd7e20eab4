// The matrix-free FVM Laplacian (format RB_STENCIL, stencil7.cuh): creation from a grid and
// its SpMM over k interleaved columns (Sec. 2, Eq. (1), Algorithm 1 with the entries formed
// from per-axis tables instead of read).
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "stencil7.cuh"

namespace rb {

namespace {

// Y[i, :] = c * (A X)[i, :] over a persistent grid; thread layout as in the CSR kernels: the
// KP chunks of VEC columns of a row in adjacent lanes, consecutive rows in consecutive lanes
// groups, so X's centre rows, its x neighbours and Y move as coalesced vectors
template <typename T, int VEC, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_spmm_stencil7(Stencil7<T> st, int64_t n, int k, int kp,
                                                             const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                             int64_t ldy, const double* __restrict__ cs) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  T c[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) c[q] = SCALE ? (T)cs[chunk * VEC + q] : T(1);
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    T acc[VEC], dinv;
    stencil7_apply<T, VEC>(st, X, ldx, row, chunk * VEC, acc, dinv);
    Vec<T, VEC> y;
#pragma unroll
    for (int q = 0; q < VEC; ++q) y.v[q] = SCALE ? acc[q] * c[q] : acc[q];
    stv<T, VEC>(Y + row * ldy + chunk * VEC, y);
  }
}

// The same product with a run of RUN consecutive cells along x per thread (stencil7_apply_run)
template <typename T, int VEC, int RUN, bool SCALE, bool CONTIG>
__global__ void __launch_bounds__(kThreads) k_spmm_stencil7_run(Stencil7<T> st, FastDiv drun, FastDiv drow,
                                                                 int64_t n_runs, int k,
                                                                 int kp, const T* __restrict__ X, int64_t ldx,
                                                                 T* __restrict__ Y, int64_t ldy,
                                                                 const double* __restrict__ cs) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  T cc[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) cc[q] = SCALE ? (T)cs[chunk * VEC + q] : T(1);
  for (int64_t u = (int64_t)blockIdx.x * R + threadIdx.x / kp; u < n_runs; u += (int64_t)gridDim.x * R) {
    Vec<T, VEC> x0[RUN], y[RUN];
    const int64_t row0 = stencil7_apply_run<T, VEC, RUN, CONTIG>(st, drun, drow, u, X + chunk * VEC, ldx, x0, y);
    if constexpr (SCALE) {
#pragma unroll
      for (int c = 0; c < RUN; ++c)
#pragma unroll
        for (int q = 0; q < VEC; ++q) y[c].v[q] *= cc[q];
    }
    store_run<T, VEC, RUN, CONTIG>(Y + chunk * VEC + row0 * ldy, ldy, y);
  }
}

// Jacobi diagonal of the operator in both precisions (as rb_operator_create forms it from the
// FP64 diagonal): 1 / a_ii and the FP32 reciprocal of the FP32-rounded entry
__global__ void k_stencil7_dinv(Stencil7<double> st, int64_t n, double* __restrict__ d64, float* __restrict__ d32) {
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n; row += (int64_t)gridDim.x * blockDim.x) {
    const double a = st.scale * stencil7_coef(st, row).diag;
    d64[row] = a != 0.0 ? 1.0 / a : 0.0;
    d32[row] = a != 0.0 ? (float)(1.0 / (double)(float)a) : 0.0f;
  }
}

template <typename T>
Stencil7<T> view(const rb_op* op) {
  Stencil7<T> s;
  for (int d = 0; d < 3; ++d) {
    s.n[d] = op->st_n[d];
    s.per[d] = op->st_per[d];
    s.w[d] = static_cast<const T*>(op->st_w[d]);
    s.ic[d] = static_cast<const T*>(op->st_ic[d]);
  }
  s.scale = (T)op->st_scale;
  s.init_div();
  return s;
}

template <typename T, int VEC>
rb_status launch(const rb_op* op, const SpmmSched& sc, const T* X, int64_t ldx, T* Y, int64_t ldy, int k,
                 const double* cs, cudaStream_t s) {
  const int R = kThreads / sc.kp;
  constexpr int RUN = 4;
  if (op->st_n[0] % RUN == 0) {  // runs of four cells along x
    const int64_t n_runs = op->n_rows / RUN;
    const int64_t rblocks = (n_runs + R - 1) / R;
    FastDiv drun, drow;
    drun.init((uint32_t)(op->st_n[0] / RUN));
    drow.init((uint32_t)op->st_n[1]);
    const bool contig = sc.kp == 1 && ldx == VEC && ldy == VEC && ((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0;
    auto go = [&](auto kern) {
      kern<<<wave_grid(kern, rblocks), kThreads, 0, s>>>(view<T>(op), drun, drow, n_runs, k, sc.kp, X, ldx, Y, ldy, cs);
    };
    if (cs) {
      if (contig) go(&k_spmm_stencil7_run<T, VEC, RUN, true, true>);
      else go(&k_spmm_stencil7_run<T, VEC, RUN, true, false>);
    } else {
      if (contig) go(&k_spmm_stencil7_run<T, VEC, RUN, false, true>);
      else go(&k_spmm_stencil7_run<T, VEC, RUN, false, false>);
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
  }
  const int64_t blocks = ((int64_t)op->n_rows + R - 1) / R;
  if (cs) {
    auto* kern = &k_spmm_stencil7<T, VEC, true>;
    kern<<<wave_grid(kern, blocks), kThreads, 0, s>>>(view<T>(op), op->n_rows, k, sc.kp, X, ldx, Y, ldy, cs);
  } else {
    auto* kern = &k_spmm_stencil7<T, VEC, false>;
    kern<<<wave_grid(kern, blocks), kThreads, 0, s>>>(view<T>(op), op->n_rows, k, sc.kp, X, ldx, Y, ldy, cs);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T>
rb_status launch_t(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                   const double* cs, cudaStream_t s) {
  const T* x = static_cast<const T*>(X);
  T* y = static_cast<T*>(Y);
  switch (sc.vec) {
    case 1: return launch<T, 1>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 2: return launch<T, 2>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 3: return launch<T, 3>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 4: return launch<T, 4>(op, sc, x, ldx, y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported vector width %d", sc.vec);
  return RB_EUNSUPPORTED;
}

}  // namespace

rb_status stencil_df_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                            int k, const double* cs, cudaStream_t s);
rb_status stencil_df_tables(const rb_grid_desc* grid, double scale, double* const w64[3], double* const ic64[3],
                            void* tab[3], int64_t* bytes, cudaStream_t s);

rb_status stencil_spmm_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                              int k, const double* cs, cudaStream_t s) {
  if (op->dtype == RB_DF64) return stencil_df_launch(op, sc, X, ldx, Y, ldy, k, cs, s);
  if (op->dtype == RB_F64) return launch_t<double>(op, sc, X, ldx, Y, ldy, k, cs, s);
  return launch_t<float>(op, sc, X, ldx, Y, ldy, k, cs, s);
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_fvm_stencil_create(const rb_grid_desc* grid, double scale, rb_dtype dtype, int32_t k_max,
                                           rb_stream_t stream, rb_op_t* out) {
  clear_error();
  RB_REQUIRE(grid && out, "rb_fvm_stencil_create: null argument");
  *out = nullptr;
  RB_REQUIRE(dtype == RB_F64 || dtype == RB_F32 || dtype == RB_DF64, "rb_fvm_stencil_create: unknown dtype %d",
             (int)dtype);
  RB_REQUIRE(k_max >= 1 && k_max <= RB_MAX_K, "rb_fvm_stencil_create: k_max %d outside [1, %d]", k_max, RB_MAX_K);
  RB_REQUIRE(std::isfinite(scale), "rb_fvm_stencil_create: scale is not finite");
  for (int d = 0; d < 3; ++d) RB_REQUIRE(grid->nodes[d] != nullptr, "rb_fvm_stencil_create: null nodes[%d]", d);
  int32_t nr = 0, nc = 0;
  int64_t nnz = 0;
  RB_TRY(rb_fvm_csr_size(grid, RB_FVM_LAPLACIAN, &nr, &nc, &nnz));  // validates the grid
  cudaStream_t s = S(stream);
  rb_op* op = new rb_op();
  op->n_rows = op->n_cols = nr;
  op->nnz = nnz;
  op->dtype = dtype;
  op->format = RB_STENCIL;
  op->k_max = k_max;
  op->max_row_len = 7;
  op->avg_row_len = nr ? (double)nnz / nr : 0.0;
  op->st_scale = scale;
  for (int d = 0; d < 3; ++d) op->st_n[d] = grid->n[d], op->st_per[d] = grid->periodic[d] ? 1 : 0;
  double *w64[3] = {}, *ic64[3] = {};
  float *w32[3] = {}, *ic32[3] = {};
  rb_status st = RB_OK;
  auto alloc = [&](void** p, size_t bytes) {
    if (st != RB_OK) return;
    cudaError_t e = cudaMalloc(p, bytes + 64);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes + 64);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    else op->device_bytes += (int64_t)bytes + 64;
  };
  for (int d = 0; d < 3; ++d) {
    const size_t n = (size_t)grid->n[d] + 1;
    alloc((void**)&w64[d], n * 8);
    alloc((void**)&ic64[d], n * 8);
    alloc((void**)&w32[d], n * 4);
    alloc((void**)&ic32[d], n * 4);
  }
  alloc((void**)&op->err, sizeof(int));
  alloc((void**)&op->dinv64, (size_t)nr * 8);
  alloc((void**)&op->dinv32, (size_t)nr * 4);
  if (st == RB_OK) st = stencil7_tables(grid, w64, ic64, w32, ic32, s);
  if (st == RB_OK && nr > 0) {
    Stencil7<double> v;
    for (int d = 0; d < 3; ++d) v.n[d] = op->st_n[d], v.per[d] = op->st_per[d], v.w[d] = w64[d], v.ic[d] = ic64[d];
    v.scale = scale;
    v.init_div();
    const int grid_blocks = (int)std::min<int64_t>(((int64_t)nr + 255) / 256, kMaxGrid);
    k_stencil7_dinv<<<grid_blocks, 256, 0, s>>>(v, nr, op->dinv64, op->dinv32);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "stencil operator tables", __FILE__, __LINE__);
    op->has_diag = 1;
  }
  // keep the tables of the operator's type (double-float: the factorised pair tables)
  if (st == RB_OK && dtype == RB_DF64) {
    void* tab[3] = {nullptr, nullptr, nullptr};
    st = stencil_df_tables(grid, scale, w64, ic64, tab, &op->device_bytes, s);
    for (int d = 0; d < 3; ++d) op->st_w[d] = tab[d];
  }
  for (int d = 0; d < 3; ++d) {
    if (dtype == RB_DF64) {
      for (void* q : {(void*)w64[d], (void*)ic64[d], (void*)w32[d], (void*)ic32[d]})
        if (q) cudaFree(q);
    } else if (dtype == RB_F64) {
      op->st_w[d] = w64[d], op->st_ic[d] = ic64[d];
      if (w32[d]) cudaFree(w32[d]);
      if (ic32[d]) cudaFree(ic32[d]);
    } else {
      op->st_w[d] = w32[d], op->st_ic[d] = ic32[d];
      if (w64[d]) cudaFree(w64[d]);
      if (ic64[d]) cudaFree(ic64[d]);
    }
  }
  if (st != RB_OK) {
    const std::string msg = rb_last_error();
    rb_operator_destroy(op);
    set_error("%s", msg.c_str());
    return st;
  }
  *out = op;
  return RB_OK;
}
