// Wider Laplacian stencils on uniform periodic Cartesian grids (Sec. 4.1: the 13p and 27p
// sparsity patterns measured beside the first-neighbour 7p), written into CSR on the device.
//
// Every row has the same number of entries (13 or 27), so row r starts at KIND r and no scan
// is needed.  One thread builds one row with its columns already in order: along each axis
// the wrapped neighbour indices are sorted once (a 5- or 3-element network in registers), and
// with cells numbered x fastest, visiting z, then y, then x in sorted order gives increasing
// columns.  A block stages its rows in shared memory and writes them out with consecutive
// threads on consecutive entries.
#include "common.cuh"

namespace rb {
namespace {

constexpr int kStencilThreads = 128;

// Coefficients of one operator (scale included): 13p uses c[d][0] for the first neighbours
// along axis d, c[d][1] for the second ones and centre; 27p uses w[m] for a neighbour whose
// offset has m nonzero components (w[0] the centre).
struct StencilCoef {
  double c[3][2];
  double centre;
  double w[4];
};

// sorts N (index, offset) pairs by index: odd-even transposition, every index known at
// compile time, so both arrays stay in registers
template <int N>
__device__ __forceinline__ void sort_axis(int (&v)[N], int (&o)[N]) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
#pragma unroll
    for (int a = r & 1; a + 1 < N; a += 2) {
      const bool sw = v[a] > v[a + 1];
      const int v0 = sw ? v[a + 1] : v[a], v1 = sw ? v[a] : v[a + 1];
      const int o0 = sw ? o[a + 1] : o[a], o1 = sw ? o[a] : o[a + 1];
      v[a] = v0, v[a + 1] = v1, o[a] = o0, o[a + 1] = o1;
    }
  }
}

// neighbour indices t + o (o = -R..R) along an axis of n >= 2R + 1 cells, wrapped, sorted
template <int R>
__device__ __forceinline__ void axis_neighbours(int t, int n, int (&v)[2 * R + 1], int (&o)[2 * R + 1]) {
#pragma unroll
  for (int a = 0; a < 2 * R + 1; ++a) {
    const int off = a - R;
    int x = t + off;
    x += (x < 0) ? n : 0;
    x -= (x >= n) ? n : 0;
    v[a] = x;
    o[a] = off;
  }
  sort_axis<2 * R + 1>(v, o);
}

template <int KIND>
__global__ void __launch_bounds__(kStencilThreads) k_stencil(int nx, int ny, int nz, StencilCoef cf,
                                                             int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                                                             double* __restrict__ va) {
  __shared__ double s_val[kStencilThreads * KIND];
  __shared__ int32_t s_col[kStencilThreads * KIND];
  const int n = nx * ny * nz;
  const int r0 = blockIdx.x * kStencilThreads;
  const int rows = min(kStencilThreads, n - r0);
  const int r = r0 + threadIdx.x;
  if (threadIdx.x < rows) {
    const int i = r % nx, q = r / nx;
    const int j = q % ny, k = q / ny;
    int* col0 = s_col + threadIdx.x * KIND;
    double* val0 = s_val + threadIdx.x * KIND;
    int p = 0;
    if constexpr (KIND == 13) {
      int xv[5], xo[5], yv[5], yo[5], zv[5], zo[5];
      axis_neighbours<2>(i, nx, xv, xo);
      axis_neighbours<2>(j, ny, yv, yo);
      axis_neighbours<2>(k, nz, zv, zo);
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        if (zo[a] != 0) {
          col0[p] = i + nx * (j + ny * zv[a]);
          val0[p++] = (zo[a] == 1 || zo[a] == -1) ? cf.c[2][0] : cf.c[2][1];
          continue;
        }
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          if (yo[b] != 0) {
            col0[p] = i + nx * (yv[b] + ny * k);
            val0[p++] = (yo[b] == 1 || yo[b] == -1) ? cf.c[1][0] : cf.c[1][1];
            continue;
          }
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            col0[p] = xv[c] + nx * (j + ny * k);
            val0[p++] = xo[c] == 0 ? cf.centre : (xo[c] == 1 || xo[c] == -1) ? cf.c[0][0] : cf.c[0][1];
          }
        }
      }
    } else {
      int xv[3], xo[3], yv[3], yo[3], zv[3], zo[3];
      axis_neighbours<1>(i, nx, xv, xo);
      axis_neighbours<1>(j, ny, yv, yo);
      axis_neighbours<1>(k, nz, zv, zo);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            col0[p] = xv[c] + nx * (yv[b] + ny * zv[a]);
            const int m = (zo[a] != 0) + (yo[b] != 0) + (xo[c] != 0);
            val0[p++] = m == 0 ? cf.w[0] : m == 1 ? cf.w[1] : m == 2 ? cf.w[2] : cf.w[3];
          }
    }
    rp[r] = KIND * r;
    if (r == n - 1) rp[n] = KIND * n;
  }
  __syncthreads();
  const int64_t base = (int64_t)KIND * r0;
  for (int e = threadIdx.x; e < rows * KIND; e += kStencilThreads) {
    ci[base + e] = s_col[e];
    va[base + e] = s_val[e];
  }
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_stencil_assemble(const int32_t n[3], const double h[3], rb_stencil_kind kind, double scale,
                                         int32_t* row_ptr, int32_t* col_idx, double* vals, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(n != nullptr && h != nullptr, "rb_stencil_assemble: null n or h");
  RB_REQUIRE(kind == RB_STENCIL_13P || kind == RB_STENCIL_27P, "rb_stencil_assemble: unknown kind %d", (int)kind);
  const int reach = kind == RB_STENCIL_13P ? 2 : 1;
  for (int d = 0; d < 3; ++d) {
    RB_REQUIRE(n[d] >= 2 * reach + 1, "rb_stencil_assemble: %d-point stencil needs >= %d cells along axis %d (got %d)",
               (int)kind, 2 * reach + 1, d, n[d]);
    RB_REQUIRE(std::isfinite(h[d]) && h[d] > 0.0, "rb_stencil_assemble: spacing h[%d] must be positive", d);
  }
  RB_REQUIRE(kind != RB_STENCIL_27P || (h[0] == h[1] && h[1] == h[2]),
             "rb_stencil_assemble: the 27-point stencil takes cubic cells (equal h)");
  const int64_t rows = (int64_t)n[0] * n[1] * n[2];
  RB_REQUIRE(rows * (int64_t)kind <= INT32_MAX, "rb_stencil_assemble: %lld nonzeros exceed 32-bit row pointers",
             (long long)(rows * (int64_t)kind));
  RB_REQUIRE(row_ptr && col_idx && vals, "rb_stencil_assemble: null output array");
  StencilCoef cf{};
  if (kind == RB_STENCIL_13P) {
    const double vol = h[0] * h[1] * h[2];
    double centre = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double q = 12.0 * h[d] * h[d];
      cf.c[d][0] = scale * (vol * 16.0 / q);
      cf.c[d][1] = scale * (vol * -1.0 / q);
      centre += vol * -30.0 / q;
    }
    cf.centre = scale * centre;
  } else {
    const double hh = h[0];
    const double unit = hh * hh * hh / (30.0 * hh * hh);
    const double wt[4] = {-128.0, 14.0, 3.0, 1.0};
    for (int m = 0; m < 4; ++m) cf.w[m] = scale * (unit * wt[m]);
  }
  cudaStream_t s = S(stream);
  const unsigned grid = (unsigned)((rows + kStencilThreads - 1) / kStencilThreads);
  if (kind == RB_STENCIL_13P)
    k_stencil<13><<<grid, kStencilThreads, 0, s>>>(n[0], n[1], n[2], cf, row_ptr, col_idx, vals);
  else
    k_stencil<27><<<grid, kStencilThreads, 0, s>>>(n[0], n[1], n[2], cf, row_ptr, col_idx, vals);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}
