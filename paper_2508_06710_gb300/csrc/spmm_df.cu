// SpMM over k interleaved columns (Sec. 2, Eq. (1), Algorithm 1) in double-float arithmetic:
// operator values and the blocks X, Y hold FP64 numbers as unevaluated sums hi + lo of two
// FP32 numbers (Dekker, "A floating-point technique for extending the available precision",
// Numer. Math. 18, 1971), and every product and sum is formed with the error-free
// transformations
//   TwoProd (the FMA form): p = RN(a b), q = fma(a, b, -p), so a b = p + q exactly;
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = RN(a + b), b' = s - a, r = (a - (s - b')) + (b - b'),
//   so a + b = s + r exactly.
// The accumulation of a row keeps (S, E): S the FP32 running sum of the leading products, E the
// FP32 sum of TwoSum's exact rounding errors and each product's low part
// vh xh - p + vh xl + vl xh (vl xl, below 2^-48 of the product, dropped); the result is
// TwoSum(S, E).  Twelve FP32 instructions per nonzero and column, on the FP32 pipe, instead of
// one FP64 FMA on GB300's FP64 pipe (1/64 of the FP32 rate); the bytes moved are FP64's (a pair
// is 8 bytes).  Error: about 2^-48 of sum_p |val[p] X[idx[p], j]| per nonzero of the row, from
// the rounding of E and the dropped term.
//
// A pair is stored {hi, lo} (hi at the lower address) and is loaded and stored as one 8-byte
// word, so the k-interleaved blocks move exactly as FP64 blocks of the same shape.  Only the
// CSR direct schedule exists for this type (one lane or LPR lanes per row).
#include <algorithm>

#include "common.cuh"
#include "spmm_impl.cuh"

namespace rb {

namespace {

// the pair held in the bits of an 8-byte word: hi in the low half (the lower address)
__device__ __forceinline__ void df_bits(double w, float& hi, float& lo) {
  hi = __int_as_float(__double2loint(w));
  lo = __int_as_float(__double2hiint(w));
}

__device__ __forceinline__ double df_word(float hi, float lo) {
  return __hiloint2double(__float_as_int(lo), __float_as_int(hi));
}

// TwoSum with rounded-to-nearest operations that the compiler may not contract into FMAs
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& r) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (S, E) += (vh + vl) (xh + xl)
__device__ __forceinline__ void df_mac(float vh, float vl, float xh, float xl, float& S, float& E) {
  const float p = __fmul_rn(vh, xh);
  float q = __fmaf_rn(vh, xh, -p);
  q = __fmaf_rn(vh, xl, q);
  q = __fmaf_rn(vl, xh, q);
  float s, r;
  two_sum(S, p, s, r);
  S = s;
  E = __fadd_rn(E, __fadd_rn(r, q));
}

struct DfArgs {
  int n_rows = 0;
  const int32_t* __restrict__ rp = nullptr;
  const int32_t* __restrict__ ci = nullptr;
  const double* __restrict__ va = nullptr;  // pairs, as 8-byte words
  const double* __restrict__ X = nullptr;   // pairs
  int64_t ldx = 0;
  double* __restrict__ Y = nullptr;         // pairs
  int64_t ldy = 0;
  int k = 1;
  int kp = 1;
  const double* __restrict__ cs = nullptr;  // per-column scale (FP64), or null
};

template <int VEC, int LPR, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_spmm_df(DfArgs a) {
  const int R = kThreads / (a.kp * LPR);
  const int t = threadIdx.x;
  const int sub = t % LPR;
  const int rc = t / LPR;
  const int chunk = rc % a.kp;
  const int rloc = rc / a.kp;
  const int64_t stride = (int64_t)gridDim.x * R;
  // the column scale c split into pairs as the block values are, once per thread
  float ch[VEC], cl[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    ch[e] = 1.0f, cl[e] = 0.0f;
    if constexpr (SCALE) {
      if (chunk * VEC + e < a.k) {
        const double cd = a.cs[chunk * VEC + e];
        ch[e] = __double2float_rn(cd);
        cl[e] = __double2float_rn(cd - (double)ch[e]);
      }
    }
  }
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    float S[VEC], E[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) S[e] = 0.0f, E[e] = 0.0f;
    int rs = 0, re = 0;
    if (active) {
      rs = __ldg(a.rp + row);
      re = __ldg(a.rp + row + 1);
    }
    const double* Xc = a.X + chunk * VEC;
#pragma unroll 2
    for (int p = rs + sub; p < re; p += LPR) {
      const int c = __ldg(a.ci + p);
      float vh, vl;
      df_bits(__ldg(a.va + p), vh, vl);
      const Vec<double, VEC> x = ldv<double, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        float xh, xl;
        df_bits(x.v[e], xh, xl);
        df_mac(vh, vl, xh, xl, S[e], E[e]);
      }
    }
    if constexpr (LPR > 1) {  // the lanes' partial sums, combined exactly up to E's rounding
#pragma unroll
      for (int off = LPR / 2; off >= 1; off >>= 1) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const float So = __shfl_xor_sync(0xffffffffu, S[e], off);
          const float Eo = __shfl_xor_sync(0xffffffffu, E[e], off);
          float s, r;
          two_sum(S[e], So, s, r);
          S[e] = s;
          E[e] = __fadd_rn(E[e], __fadd_rn(Eo, r));
        }
      }
    }
    if (active && sub == 0) {
      Vec<double, VEC> y;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        float hi, lo;
        two_sum(S[e], E[e], hi, lo);
        if constexpr (SCALE) {  // (hi + lo) (ch + cl), renormalised by TwoSum
          const float p = __fmul_rn(hi, ch[e]);
          float q = __fmaf_rn(hi, ch[e], -p);
          q = __fmaf_rn(hi, cl[e], q);
          q = __fmaf_rn(lo, ch[e], q);
          two_sum(p, q, hi, lo);
        }
        y.v[e] = df_word(hi, lo);
      }
      stv<double, VEC>(a.Y + row * a.ldy + chunk * VEC, y);
    }
  }
}

template <int VEC, int LPR>
rb_status launch_df(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                    const double* cs, cudaStream_t s) {
  DfArgs a;
  a.n_rows = op->n_rows;
  a.rp = op->row_ptr;
  a.ci = op->col_idx;
  a.va = static_cast<const double*>(op->vals);
  a.X = static_cast<const double*>(X);
  a.ldx = ldx;
  a.Y = static_cast<double*>(Y);
  a.ldy = ldy;
  a.k = k;
  a.kp = sc.kp;
  a.cs = cs;
  const int R = sc.rows_per_block();
  int64_t grid = ((int64_t)op->n_rows + R - 1) / R;
  if (grid == 0) return RB_OK;
  auto* kern = cs ? &k_spmm_df<VEC, LPR, true> : &k_spmm_df<VEC, LPR, false>;
  if (sc.grid_cap < 0) grid = wave_grid(kern, grid);
  else if (sc.grid_cap > 0) grid = std::min<int64_t>(grid, sc.grid_cap);
  kern<<<(unsigned)std::min<int64_t>(grid, INT32_MAX), kThreads, 0, s>>>(a);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <int VEC>
rb_status launch_df_lpr(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                        int k, const double* cs, cudaStream_t s) {
  switch (sc.lpr) {
    case 1: return launch_df<VEC, 1>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 2: return launch_df<VEC, 2>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 4: return launch_df<VEC, 4>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 8: return launch_df<VEC, 8>(op, sc, X, ldx, Y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported lanes per row %d", sc.lpr);
  return RB_EUNSUPPORTED;
}

// hi = RN32(x), lo = RN32(x - hi) (the difference is exact in FP64)
__global__ void k_df_split(int64_t n, int k, const double* __restrict__ X, int64_t ldx, double* __restrict__ D,
                           int64_t ldd) {
  const int64_t total = n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / k;
    const int c = (int)(i - r * k);
    const double x = X[r * ldx + c];
    const float hi = __double2float_rn(x);
    const float lo = __double2float_rn(x - (double)hi);
    D[r * ldd + c] = df_word(hi, lo);
  }
}

// x = RN64(hi + lo)
__global__ void k_df_join(int64_t n, int k, const double* __restrict__ D, int64_t ldd, double* __restrict__ X,
                          int64_t ldx) {
  const int64_t total = n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / k;
    const int c = (int)(i - r * k);
    float hi, lo;
    df_bits(D[r * ldd + c], hi, lo);
    X[r * ldx + c] = (double)hi + (double)lo;
  }
}

rb_status check_pair_block(const char* fn, int64_t n, int k, const void* A, int64_t lda, const void* B, int64_t ldb) {
  RB_REQUIRE(n >= 0, "%s: negative n", fn);
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "%s: k = %d outside [1, %d]", fn, k, RB_MAX_K);
  RB_REQUIRE(lda >= k && ldb >= k, "%s: leading dimensions smaller than k", fn);
  RB_REQUIRE(n == 0 || (A && B), "%s: null block", fn);
  RB_REQUIRE((uintptr_t)A % 8 == 0 && (uintptr_t)B % 8 == 0, "%s: blocks not 8-byte aligned", fn);
  const uintptr_t ab = (uintptr_t)A, ae = ab + (uintptr_t)(((n - 1) * lda + k) * 8);
  const uintptr_t bb = (uintptr_t)B, be = bb + (uintptr_t)(((n - 1) * ldb + k) * 8);
  RB_REQUIRE(n == 0 || ae <= bb || be <= ab, "%s: the blocks overlap", fn);
  return RB_OK;
}

}  // namespace

rb_status spmm_launch_df(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                         int k, const double* cs, cudaStream_t s) {
  switch (sc.vec) {
    case 1: return launch_df_lpr<1>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 2: return launch_df_lpr<2>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 3: return launch_df_lpr<3>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 4: return launch_df_lpr<4>(op, sc, X, ldx, Y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported vector width %d", sc.vec);
  return RB_EUNSUPPORTED;
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_df64_split(int64_t n, int32_t k, const double* X, int64_t ldx, void* D, int64_t ldd,
                                   rb_stream_t stream) {
  clear_error();
  RB_TRY(check_pair_block("rb_df64_split", n, k, X, ldx, D, ldd));
  if (n == 0) return RB_OK;
  const int64_t blocks = (n * k + kThreads - 1) / kThreads;
  k_df_split<<<wave_grid(&k_df_split, blocks), kThreads, 0, S(stream)>>>(n, k, X, ldx, static_cast<double*>(D), ldd);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

extern "C" rb_status rb_df64_join(int64_t n, int32_t k, const void* D, int64_t ldd, double* X, int64_t ldx,
                                  rb_stream_t stream) {
  clear_error();
  RB_TRY(check_pair_block("rb_df64_join", n, k, D, ldd, X, ldx));
  if (n == 0) return RB_OK;
  const int64_t blocks = (n * k + kThreads - 1) / kThreads;
  k_df_join<<<wave_grid(&k_df_join, blocks), kThreads, 0, S(stream)>>>(n, k, static_cast<const double*>(D), ldd, X,
                                                                         ldx);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}
