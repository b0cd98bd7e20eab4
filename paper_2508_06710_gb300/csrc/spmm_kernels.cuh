// Kernel launch and template dispatch of the SpMM (Sec. 2, Eq. (1), Algorithm 1) for one
// value type; included by one translation unit per type so that the FP64 and FP32
// instantiations compile in parallel.
#pragma once

#include "common.cuh"
#include "spmm_impl.cuh"
#include "spmm_tma.cuh"

namespace rb {
namespace {


// shared memory of one block of the TMA pipeline (the ring of stages); two blocks fit on an SM
constexpr size_t kTmaSmemLimit = 100 * 1024;

template <typename T, int VEC, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_spmm_sell(int n_slots, const int32_t* __restrict__ sptr,
                                                         const int32_t* __restrict__ swidth,
                                                         const int32_t* __restrict__ srow,
                                                         const int32_t* __restrict__ scol, const T* __restrict__ sval,
                                                         const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                         int64_t ldy, int k, int kp, const double* __restrict__ cs) {
  const int R = kThreads / kp;
  const int t = threadIdx.x;
  const int chunk = t % kp;
  if (chunk * VEC >= k) return;
  const T* Xc = X + chunk * VEC;
  // slot index g = slice * 32 + lane in slice; a persistent grid strides over the slots
  for (int64_t g = (int64_t)blockIdx.x * R + t / kp; g < n_slots; g += (int64_t)gridDim.x * R) {
    const int row = __ldg(srow + g);
    if (row < 0) continue;
    const int sl = (int)(g >> 5), r = (int)(g & 31);
    const int base = __ldg(sptr + sl) + r;
    const int width = __ldg(swidth + sl);
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
#pragma unroll 2
    for (int j = 0; j < width; ++j) {
      const int c = __ldg(scol + base + j * 32);
      const T v = __ldg(sval + base + j * 32);
      const Vec<T, VEC> x = ldv<T, VEC>(Xc + (int64_t)c * ldx);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(v, x.v[e], acc[e]);
    }
    Vec<T, VEC> y;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      if constexpr (SCALE) y.v[e] = acc[e] * (T)cs[chunk * VEC + e];
      else y.v[e] = acc[e];
    }
    stv<T, VEC>(Y + (int64_t)row * ldy + chunk * VEC, y);
  }
}

template <typename T, int VEC>
rb_status launch_sell(const rb_op* op, const SpmmSched& sc, const T* X, int64_t ldx, T* Y, int64_t ldy, int k,
                      const double* cs, cudaStream_t s) {
  const int R = kThreads / sc.kp;
  const int64_t slots = (int64_t)op->n_slices * 32;
  int64_t grid = (slots + R - 1) / R;
  if (grid == 0) return RB_OK;
  auto* kern = cs ? &k_spmm_sell<T, VEC, true> : &k_spmm_sell<T, VEC, false>;
  grid = wave_grid(kern, grid);
  kern<<<(unsigned)grid, kThreads, 0, s>>>((int)slots, op->sell_ptr, op->sell_width, op->sell_row, op->sell_col,
                                           static_cast<const T*>(op->sell_val), X, ldx, Y, ldy, k, sc.kp, cs);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T, int VEC, int LPR, int EPI>
rb_status launch_csr(const rb_op* op, const SpmmSched& sc, const T* X, int64_t ldx, T* Y, int64_t ldy, int k,
                     const double* cs, cudaStream_t s) {
  CsrArgs<T> a;
  fill_csr_args(op, sc, a);
  a.X = X;
  a.ldx = ldx;
  a.Y = Y;
  a.ldy = ldy;
  a.k = k;
  a.cs = cs;
  const int R = sc.rows_per_block();
  int64_t grid = ((int64_t)op->n_rows + R - 1) / R;
  if (grid == 0) return RB_OK;
  if (sc.stage == 2) {
    if constexpr (LPR == 1) {
      auto* kern = &k_spmm_tma<T, VEC, EPI>;
      const int cap = tma_capacity<T>(op, R, kTmaSmemLimit);
      const size_t smem = tma_layout<T>(R, cap).total;
      RB_TRY(opt_in_smem(reinterpret_cast<const void*>(kern), smem));
      grid = wave_grid(kern, grid, smem, kTmaThreads);
      if (sc.grid_cap > 0) grid = std::min<int64_t>(grid, sc.grid_cap);  // fewer blocks, more tiles each
      kern<<<(unsigned)grid, kTmaThreads, smem, s>>>(a, R, cap, op->err);
      RB_CUDA(cudaGetLastError());
      return RB_OK;
    }
    set_error("spmm: the TMA pipeline takes one lane per row");
    return RB_EUNSUPPORTED;
  }
  if (sc.stage) {
    const size_t smem = csr_smem_bytes<T>(R, a.stage_cap);
    k_spmm_csr<T, VEC, LPR, EPI><<<(unsigned)std::min<int64_t>(grid, INT32_MAX), kThreads, smem, s>>>(a);
  } else {
    auto* kern = a.nblk > 1 ? &k_spmm_direct_blk<T, VEC, LPR, EPI> : &k_spmm_direct<T, VEC, LPR, EPI>;
    if (sc.grid_cap < 0) grid = wave_grid(kern, grid);  // one resident wave, grid-stride
    else if (sc.grid_cap > 0) grid = std::min<int64_t>(grid, sc.grid_cap);
    kern<<<(unsigned)std::min<int64_t>(grid, INT32_MAX), kThreads, 0, s>>>(a);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T, int VEC, int LPR>
rb_status dispatch_epi(const rb_op* op, const SpmmSched& sc, const T* X, int64_t ldx, T* Y, int64_t ldy, int k,
                       const double* cs, cudaStream_t s) {
  if (op->ext_nz > 0) {
    if constexpr (VEC != 3) {  // the spanwise epilogue takes widths dividing Nz: never 3
      if (cs) return launch_csr<T, VEC, LPR, kEpiExt | kEpiScale>(op, sc, X, ldx, Y, ldy, k, cs, s);
      return launch_csr<T, VEC, LPR, kEpiExt>(op, sc, X, ldx, Y, ldy, k, cs, s);
    }
    set_error("spmm: the extruded epilogue takes vector widths dividing Nz");
    return RB_EUNSUPPORTED;
  }
  if (cs) return launch_csr<T, VEC, LPR, kEpiScale>(op, sc, X, ldx, Y, ldy, k, cs, s);
  return launch_csr<T, VEC, LPR, 0>(op, sc, X, ldx, Y, ldy, k, cs, s);
}

template <typename T, int VEC>
rb_status dispatch_lpr(const rb_op* op, const SpmmSched& sc, const T* X, int64_t ldx, T* Y, int64_t ldy, int k,
                       const double* cs, cudaStream_t s) {
  if (op->format == RB_SELL && op->ext_nz == 0) return launch_sell<T, VEC>(op, sc, X, ldx, Y, ldy, k, cs, s);
  switch (sc.lpr) {
    case 1: return dispatch_epi<T, VEC, 1>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 2: return dispatch_epi<T, VEC, 2>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 4: return dispatch_epi<T, VEC, 4>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 8: return dispatch_epi<T, VEC, 8>(op, sc, X, ldx, Y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported lanes per row %d", sc.lpr);
  return RB_EUNSUPPORTED;
}

template <typename T>
rb_status dispatch_vec(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                       const double* cs, cudaStream_t s) {
  const T* x = static_cast<const T*>(X);
  T* y = static_cast<T*>(Y);
  switch (sc.vec) {
    case 1: return dispatch_lpr<T, 1>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 2: return dispatch_lpr<T, 2>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 3: return dispatch_lpr<T, 3>(op, sc, x, ldx, y, ldy, k, cs, s);
    case 4: return dispatch_lpr<T, 4>(op, sc, x, ldx, y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported vector width %d", sc.vec);
  return RB_EUNSUPPORTED;
}

}  // namespace
}  // namespace rb
