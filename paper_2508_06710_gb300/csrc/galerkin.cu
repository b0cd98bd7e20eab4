// The Galerkin initial guess for k independent systems A x_j = b_j sharing one operator:
// x0_j = sum_a c_aj v_aj, the combination of up to three candidate vectors per system that
// minimises the energy norm of the error (the Ritz-Galerkin projection onto their span,
// Saad, Iterative Methods, Sec. 5.1):
//
//   (V_j^T A V_j) c_j = V_j^T b_j
//
// Not from the paper (its solver starts each step from the previous pressure): the learned
// guess of this library is one candidate, the previous pressures the others.  Three steps:
//   W_a = A V_a          one SpMM per candidate block (all k columns at once)
//   G, g                 one fused pass: v_a . w_b (a <= b) and v_a . b per column, reduced
//                        in FP64 in a fixed order; the last block solves each column's small
//                        system (Cholesky that drops dependent candidates) and keeps the
//                        result only if its energy phi = c^T G c / 2 - c^T g is no larger than
//                        the best single candidate's (so rounding cannot make it worse)
//   X0 = sum_a c_a V_a   elementwise
#include <algorithm>

#include "common.cuh"
#include "reduce.cuh"

namespace rb {

SpmmSched pick_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y);
rb_status spmm_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                      const double* cs, cudaStream_t s);
rb_status spmm_validate(const rb_op* op, const void* X, int64_t ldx, const void* Y, int64_t ldy, int k);

namespace {

constexpr int kMaxCand = 3;
constexpr int kGroup = 28;                                  // columns per reduction pass (9 x 28 <= 256 sums)
constexpr int kNQ = kMaxCand * (kMaxCand + 1) / 2 + kMaxCand;  // Gram entries a <= b, and v_a . b

struct GalArgs {
  int64_t n;
  int k, c, j0, kc, kp;  // columns j0 .. j0 + kc of k; kp = next_pow2(kc) lanes per row
  const double* v[kMaxCand];
  int64_t ldv[kMaxCand];
  const double* w[kMaxCand];  // W_a = A V_a, ld = k
  const double* b;
  int64_t ldb;
  double* coef;      // k x c, this call's output (device)
  double* user_coef; // the caller's copy (may be null)
  double* partials;
  unsigned* counter;
};

// Solves the c x c system of one column: Cholesky that skips a pivot not above 1e-12 of its
// diagonal (a candidate dependent on the earlier ones gets coefficient 0).
__device__ void small_solve(int c, const double (&G)[kMaxCand][kMaxCand], const double (&g)[kMaxCand],
                            double (&x)[kMaxCand]) {
  double Lm[kMaxCand][kMaxCand] = {};
  bool on[kMaxCand];
  for (int i = 0; i < c; ++i) {
    double d = G[i][i];
    for (int p = 0; p < i; ++p)
      if (on[p]) d -= Lm[i][p] * Lm[i][p];
    on[i] = d > 1e-12 * fabs(G[i][i]) && isfinite(d);
    Lm[i][i] = on[i] ? sqrt(d) : 1.0;
    for (int r = i + 1; r < c; ++r) {
      double s = G[r][i];
      for (int p = 0; p < i; ++p)
        if (on[p]) s -= Lm[r][p] * Lm[i][p];
      Lm[r][i] = on[i] ? s / Lm[i][i] : 0.0;
    }
  }
  double y[kMaxCand];
  for (int i = 0; i < c; ++i) {
    double s = g[i];
    for (int p = 0; p < i; ++p) s -= Lm[i][p] * y[p];
    y[i] = on[i] ? s / Lm[i][i] : 0.0;
  }
  for (int i = c - 1; i >= 0; --i) {
    double s = y[i];
    for (int p = i + 1; p < c; ++p) s -= Lm[p][i] * x[p];
    x[i] = on[i] ? s / Lm[i][i] : 0.0;
  }
}

// Quantities per column, in order: G_ab for a <= b (row-major upper triangle), then g_a.
__global__ void __launch_bounds__(kThreads) k_gram(GalArgs a) {
  __shared__ RedSmem<kNQ> red;
  const int R = kThreads / a.kp;
  const int chunk = threadIdx.x % a.kp;
  const bool col_ok = chunk < a.kc;
  const int j = a.j0 + chunk;
  double s[kNQ][1];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) s[q][0] = 0.0;
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / a.kp; row < a.n; row += (int64_t)gridDim.x * R) {
      double v[kMaxCand] = {}, w[kMaxCand] = {};
#pragma unroll
      for (int p = 0; p < kMaxCand; ++p) {
        if (p < a.c) {
          v[p] = __ldg(a.v[p] + row * a.ldv[p] + j);
          w[p] = __ldg(a.w[p] + row * a.k + j);
        }
      }
      const double bv = __ldg(a.b + row * a.ldb + j);
      int q = 0;
#pragma unroll
      for (int p = 0; p < kMaxCand; ++p)
#pragma unroll
        for (int r = p; r < kMaxCand; ++r, ++q)
          if (r < a.c) s[q][0] = fma(v[p], w[r], s[q][0]);
#pragma unroll
      for (int p = 0; p < kMaxCand; ++p)
        if (p < a.c) s[q + p][0] = fma(v[p], bv, s[q + p][0]);
    }
  }
  const double tot = block_reduce<kNQ, 1>(s, a.kp, 1, a.kc, red);
  const int m = kNQ * a.kc;
  if (!publish_partials<kNQ>(tot, m, a.partials, a.counter, red)) return;
  const double all = final_sum<kNQ>(a.partials, m, gridDim.x, red);
  __shared__ double s_tot[kNQ * kGroup];
  if ((int)threadIdx.x < m) s_tot[threadIdx.x] = all;
  __syncthreads();
  const int jj = threadIdx.x;
  if (jj < a.kc) {
    // thread t < m held quantity t / kc of column t % kc
    double G[kMaxCand][kMaxCand] = {}, g[kMaxCand] = {};
    int q = 0;
    for (int p = 0; p < kMaxCand; ++p)
      for (int r = p; r < kMaxCand; ++r, ++q)
        if (r < a.c) G[p][r] = G[r][p] = s_tot[q * a.kc + jj];
    for (int p = 0; p < a.c; ++p) g[p] = s_tot[(q + p) * a.kc + jj];
    double x[kMaxCand] = {};
    small_solve(a.c, G, g, x);
    // energy of the combination against each single candidate (phi_a = G_aa / 2 - g_a)
    double phi = 0.0;
    for (int p = 0; p < a.c; ++p) {
      double gx = 0.0;
      for (int r = 0; r < a.c; ++r) gx += G[p][r] * x[r];
      phi += x[p] * (0.5 * gx - g[p]);
    }
    int best = -1;
    double best_phi = isfinite(phi) ? phi : INFINITY;
    for (int p = 0; p < a.c; ++p) {
      const double ph = 0.5 * G[p][p] - g[p];
      if (ph < best_phi) best = p, best_phi = ph;
    }
    if (best >= 0)
      for (int p = 0; p < a.c; ++p) x[p] = (p == best) ? 1.0 : 0.0;
    for (int p = 0; p < a.c; ++p) {
      a.coef[(int64_t)(a.j0 + jj) * a.c + p] = x[p];
      if (a.user_coef) a.user_coef[(int64_t)(a.j0 + jj) * a.c + p] = x[p];
    }
  }
}

// X0[i, j] = sum_a coef[j][a] V_a[i, j]; each element read and written by one thread, so X0 may
// be one of the candidates
__global__ void __launch_bounds__(kThreads) k_combine(GalArgs a, double* __restrict__ x0, int64_t ldx) {
  const int64_t total = a.n * a.k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / a.k;
    const int j = (int)(e - row * a.k);
    double s = 0.0;
    for (int p = 0; p < a.c; ++p) s = fma(a.coef[(int64_t)j * a.c + p], a.v[p][row * a.ldv[p] + j], s);
    x0[row * ldx + j] = s;
  }
}

struct GalLayout {
  size_t w, coef, partials, counter, total;
};

GalLayout gal_layout(int64_t n, int k, int c) {
  GalLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  L.w = take(sizeof(double) * (size_t)c * n * k);
  L.coef = take(sizeof(double) * (size_t)k * c);
  L.partials = take(sizeof(double) * (size_t)kNQ * kGroup * kMaxGrid);
  L.counter = take(sizeof(unsigned) * 4);
  L.total = off;
  return L;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" size_t rb_galerkin_workspace_bytes(int64_t n, int32_t k, int32_t n_cand) {
  if (n < 0 || k < 1 || k > RB_MAX_K || n_cand < 1 || n_cand > kMaxCand) return 0;
  return gal_layout(n, k, n_cand).total;
}

extern "C" rb_status rb_galerkin_guess(rb_op_t A, int32_t k, int32_t n_cand, const double* const* cand,
                                       const int64_t* ldc, const double* B, int64_t ldb, double* X0, int64_t ldx,
                                       double* coef, void* work, size_t work_bytes, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(A, "rb_galerkin_guess: null operator");
  RB_REQUIRE(A->dtype == RB_F64 && A->n_rows == A->n_cols, "rb_galerkin_guess: A must be a square FP64 operator");
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "rb_galerkin_guess: k = %d outside [1, %d]", k, RB_MAX_K);
  RB_REQUIRE(n_cand >= 1 && n_cand <= kMaxCand, "rb_galerkin_guess: n_cand = %d outside [1, %d]", n_cand, kMaxCand);
  RB_REQUIRE(cand && ldc && B && X0, "rb_galerkin_guess: null argument");
  RB_REQUIRE(ldb >= k && ldx >= k, "rb_galerkin_guess: leading dimension smaller than k");
  const int64_t n = A->n_rows;
  const GalLayout L = gal_layout(n, k, n_cand);
  RB_REQUIRE(work && work_bytes >= L.total, "rb_galerkin_guess: workspace too small (%zu < %zu)", work_bytes, L.total);
  RB_REQUIRE((uintptr_t)work % 256 == 0, "rb_galerkin_guess: workspace not 256-byte aligned");
  char* base = static_cast<char*>(work);
  GalArgs a{};
  a.n = n;
  a.k = k;
  a.c = n_cand;
  a.b = B;
  a.ldb = ldb;
  a.coef = reinterpret_cast<double*>(base + L.coef);
  a.user_coef = coef;
  a.partials = reinterpret_cast<double*>(base + L.partials);
  a.counter = reinterpret_cast<unsigned*>(base + L.counter);
  cudaStream_t s = S(stream);
  for (int p = 0; p < n_cand; ++p) {
    RB_REQUIRE(cand[p] && ldc[p] >= k, "rb_galerkin_guess: candidate %d null or ld < k", p);
    double* w = reinterpret_cast<double*>(base + L.w) + (size_t)p * n * k;
    RB_TRY(spmm_validate(A, cand[p], ldc[p], w, k, k));
    a.v[p] = cand[p];
    a.ldv[p] = ldc[p];
    a.w[p] = w;
  }
  if (n == 0) return RB_OK;
  RB_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned) * 4, s));
  for (int p = 0; p < n_cand; ++p)
    RB_TRY(spmm_launch(A, pick_sched(A, k, a.ldv[p], k, a.v[p], a.w[p]), a.v[p], a.ldv[p], const_cast<double*>(a.w[p]),
                       k, k, nullptr, s));
  for (int j0 = 0; j0 < k; j0 += kGroup) {
    a.j0 = j0;
    a.kc = std::min(kGroup, k - j0);
    a.kp = next_pow2(a.kc);
    const int64_t blocks = (n + kThreads / a.kp - 1) / (kThreads / a.kp);
    k_gram<<<wave_grid(&k_gram, blocks), kThreads, 0, s>>>(a);
  }
  const int cg = (int)std::min<int64_t>((n * k + kThreads - 1) / kThreads, kMaxGrid);
  k_combine<<<std::max(cg, 1), kThreads, 0, s>>>(a, X0, ldx);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}
