// The other three basic operations of Sec. 1 on an n x k block, one column per right-hand
// side: dot (per-column inner products, FP64 accumulation), axpy (per-column scalars) and
// axty (element-wise product).  Streaming kernels: each thread handles VEC consecutive
// columns of a row (16-byte accesses when aligned), rows in a grid-stride loop.
#include <algorithm>
#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "reduce.cuh"

namespace rb {
namespace {

constexpr int kBlasGrid = kPersistentGrid;  // partials capacity: at most one resident wave

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_dot_partial(int64_t n, int k, int kp, const T* __restrict__ X,
                                                          int64_t ldx, const T* __restrict__ Y, int64_t ldy,
                                                          double* __restrict__ partials) {
  __shared__ RedSmem<1> sm;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const int rloc = threadIdx.x / kp;
  const bool col_ok = chunk * VEC < k;
  double acc[1][VEC];
  float facc[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc[0][e] = 0.0, facc[e] = 0.0f;
  int pending = 0;
  for (int64_t row = (int64_t)blockIdx.x * R + rloc; row < n; row += (int64_t)gridDim.x * R) {
    if (!col_ok) break;
    const Vec<T, VEC> x = ldv<T, VEC>(X + row * ldx + chunk * VEC);
    const Vec<T, VEC> y = ldv<T, VEC>(Y + row * ldy + chunk * VEC);
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[0][e] = fma((double)x.v[e], (double)y.v[e], acc[0][e]);
    } else {
      // FP32 products summed four at a time in FP32, the groups in FP64
#pragma unroll
      for (int e = 0; e < VEC; ++e) facc[e] = fmaf((float)x.v[e], (float)y.v[e], facc[e]);
      if (++pending == 4) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[0][e] += (double)facc[e], facc[e] = 0.0f;
        pending = 0;
      }
    }
  }
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[0][e] += (double)facc[e];
  }
  const double v = block_reduce<1, VEC>(acc, kp, 1, k, sm);
  if ((int)threadIdx.x < k) partials[(size_t)blockIdx.x * k + threadIdx.x] = v;
}

__global__ void __launch_bounds__(kThreads) k_dot_final(int m, int nblocks, const double* __restrict__ partials,
                                                        double* __restrict__ out) {
  __shared__ RedSmem<1> sm;
  const double r = final_sum<1>(partials, m, nblocks, sm);
  if ((int)threadIdx.x < m) out[threadIdx.x] = r;
}

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_axpy(int64_t n, int k, int kp, const double* __restrict__ alpha,
                                                   const T* __restrict__ X, int64_t ldx, T* __restrict__ Y,
                                                   int64_t ldy) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  T a[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) a[e] = (T)alpha[chunk * VEC + e];
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const Vec<T, VEC> x = ldv<T, VEC>(X + row * ldx + chunk * VEC);
    Vec<T, VEC> y = ldv_rw<T, VEC>(Y + row * ldy + chunk * VEC);
#pragma unroll
    for (int e = 0; e < VEC; ++e) y.v[e] = fma(a[e], x.v[e], y.v[e]);
    stv<T, VEC>(Y + row * ldy + chunk * VEC, y);
  }
}

// alpha x y with alpha == 1 taken as the one product x y: the same value (1 x is x exactly), and
// half the FP64 multiplies, which GB300 issues at 2 per clock per SM: two multiplies per entry
// bound the FP64 kernel near 90 µs on 28 M entries, more than its HBM time.
template <bool UNIT, typename T>
__device__ __forceinline__ T axty_elem(T alpha, T x, T y) {
  if constexpr (UNIT) return x * y;
  else return alpha * x * y;
}

template <typename T, int VEC, bool UNIT>
__global__ void __launch_bounds__(kThreads) k_axty(int64_t n, int k, int kp, T alpha, const T* __restrict__ X,
                                                   int64_t ldx, T* __restrict__ Y, int64_t ldy) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const Vec<T, VEC> x = ldv<T, VEC>(X + row * ldx + chunk * VEC);
    Vec<T, VEC> y = ldv_rw<T, VEC>(Y + row * ldy + chunk * VEC);
#pragma unroll
    for (int e = 0; e < VEC; ++e) y.v[e] = axty_elem<UNIT>(alpha, x.v[e], y.v[e]);
    stv<T, VEC>(Y + row * ldy + chunk * VEC, y);
  }
}


// Flat streaming of a contiguous block (ld == k, 16-byte aligned): the n k entries as one
// array of 16-byte vectors, entry f in column f % k.  The grid is a multiple of the odd part of
// k, so that the stride (grid x threads x V entries) is a multiple of k: every vector a thread
// touches starts in the same column, the column of each lane position e is fixed per thread,
// and the inner loop is pure streaming (one accumulator or one alpha per position).
constexpr int kFlatMaxK = 8;

inline int odd_part(int k) {
  while (k % 2 == 0) k /= 2;
  return k;
}

template <typename T>
__device__ __forceinline__ void flat_cols(int64_t first_entry, int k, int (&cole)[16 / sizeof(T)]) {
  const int c0 = (int)(first_entry % k);
#pragma unroll
  for (int e = 0; e < (int)(16 / sizeof(T)); ++e) cole[e] = (c0 + e) % k;
}

// dot over units of lcm(V, K) entries (whole vectors that start and end on a row boundary):
// the column of every entry of a unit is a compile-time constant, so the loop keeps just K
// accumulators.  FP32 products are summed four units at a time in FP32, the groups in FP64.
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }

template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_dot_flat(int64_t total, const T* __restrict__ X,
                                                       const T* __restrict__ Y, double* __restrict__ partials) {
  constexpr int V = 16 / sizeof(T);
  constexpr int L = V / gcd_c(V, K) * K;  // entries per unit
  constexpr int NV = L / V;               // vectors per unit
  __shared__ double sh[kThreads / 32][K];
  const int64_t nunits = total / L;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  double acc[K];
  T facc[K];
  // FP64: one accumulator per position of the unit (L independent FMA chains instead of K
  // chains of L / K, for the FP64 pipe's latency), folded into the columns at the end
  double pacc[sizeof(T) == 8 ? L : 1];
#pragma unroll
  for (int j = 0; j < K; ++j) acc[j] = 0.0, facc[j] = T(0);
#pragma unroll
  for (int q = 0; q < (sizeof(T) == 8 ? L : 1); ++q) pacc[q] = 0.0;
  int pending = 0;
  for (int64_t u = tid; u < nunits; u += stride) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const Vec<T, V> x = ldv<T, V>(X + u * L + i * V);
      const Vec<T, V> y = ldv<T, V>(Y + u * L + i * V);
#pragma unroll
      for (int e = 0; e < V; ++e) {
        if constexpr (sizeof(T) == 8) pacc[i * V + e] = fma((double)x.v[e], (double)y.v[e], pacc[i * V + e]);
        else facc[(i * V + e) % K] = fma(x.v[e], y.v[e], facc[(i * V + e) % K]);
      }
    }
    // FP32 products are summed four units at a time in FP32, the groups in FP64 (FP64
    // products accumulate in place: a flush per unit would add a DADD per column and unit on
    // the FP64 pipe, which bounds this kernel)
    if constexpr (sizeof(T) == 4) {
      if (++pending == 4) {
#pragma unroll
        for (int j = 0; j < K; ++j) acc[j] += (double)facc[j], facc[j] = T(0);
        pending = 0;
      }
    }
  }
  if constexpr (sizeof(T) == 8) {
#pragma unroll
    for (int q = 0; q < L; ++q) acc[q % K] += pacc[q];
  } else {
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] += (double)facc[j];
  }
  // tail entries past the last whole unit: entry nunits L + tid is in column tid % K
  const int64_t f = nunits * L + tid;
  if (f < total) {
    const int cf = (int)(tid % K);
#pragma unroll
    for (int j = 0; j < K; ++j)
      if (cf == j) acc[j] += (double)X[f] * (double)Y[f];
  }
  const int w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double v = acc[j];
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[w][j] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double v = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) v += sh[i][threadIdx.x];
    partials[(size_t)blockIdx.x * K + threadIdx.x] = v;
  }
}

template <typename T>
rb_status launch_dot_flat(int64_t total, int k, const T* X, const T* Y, double* partials, int& grid, cudaStream_t s) {
  auto go = [&](auto kc) {
    constexpr int K = decltype(kc)::value;
    constexpr int V = 16 / sizeof(T);
    constexpr int L = V / gcd_c(V, K) * K;
    const int64_t blocks = std::max<int64_t>(1, (total / L + kThreads - 1) / kThreads);
    grid = std::min(kBlasGrid, wave_grid(&k_dot_flat<T, K>, blocks));
    k_dot_flat<T, K><<<grid, kThreads, 0, s>>>(total, X, Y, partials);
  };
  switch (k) {
    case 1: go(std::integral_constant<int, 1>{}); break;
    case 2: go(std::integral_constant<int, 2>{}); break;
    case 3: go(std::integral_constant<int, 3>{}); break;
    case 4: go(std::integral_constant<int, 4>{}); break;
    case 5: go(std::integral_constant<int, 5>{}); break;
    case 6: go(std::integral_constant<int, 6>{}); break;
    case 7: go(std::integral_constant<int, 7>{}); break;
    case 8: go(std::integral_constant<int, 8>{}); break;
    default: set_error("rb_dot: flat kernel takes k <= 8"); return RB_EUNSUPPORTED;
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_axpy_flat(int64_t total, int k, const double* __restrict__ alpha,
                                                        const T* __restrict__ X, T* __restrict__ Y) {
  constexpr int V = 16 / sizeof(T);
  const int64_t nvec = total / V;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int cole[V];
  flat_cols<T>(tid * V, k, cole);
  T a[V];
#pragma unroll
  for (int e = 0; e < V; ++e) a[e] = (T)alpha[cole[e]];
  for (int64_t c = tid; c < nvec; c += stride) {
    const Vec<T, V> x = ldv<T, V>(X + c * V);
    Vec<T, V> y = ldv_rw<T, V>(Y + c * V);
#pragma unroll
    for (int e = 0; e < V; ++e) y.v[e] = fma(a[e], x.v[e], y.v[e]);
    stv<T, V>(Y + c * V, y);
  }
  const int64_t f = nvec * V + tid;
  if (f < total) Y[f] = fma((T)alpha[f % k], X[f], Y[f]);
}

template <typename T, bool UNIT>
__global__ void __launch_bounds__(kThreads) k_axty_flat(int64_t total, T alpha, const T* __restrict__ X,
                                                        T* __restrict__ Y) {
  constexpr int V = 16 / sizeof(T);
  const int64_t nvec = total / V;
  const int64_t tid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t c = tid; c < nvec; c += stride) {
    const Vec<T, V> x = ldv<T, V>(X + c * V);
    Vec<T, V> y = ldv_rw<T, V>(Y + c * V);
#pragma unroll
    for (int e = 0; e < V; ++e) y.v[e] = axty_elem<UNIT>(alpha, x.v[e], y.v[e]);
    stv<T, V>(Y + c * V, y);
  }
  const int64_t f = nvec * V + tid;
  if (f < total) Y[f] = axty_elem<UNIT>(alpha, X[f], Y[f]);
}

bool flat_ok(int k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  return ldx == k && ldy == k && ((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0;
}

// grid of a flat kernel: one resident wave, a multiple of the odd part of k
template <typename K>
int flat_grid(K* kernel, int64_t total, int eb, int k) {
  const int64_t vec_blocks = (total / (16 / eb) + kThreads - 1) / kThreads;
  int g = wave_grid(kernel, std::max<int64_t>(vec_blocks, 1));
  const int o = odd_part(k);
  g = std::max(o, g / o * o);
  return g;
}

rb_status check_block(const char* fn, int64_t n, int k, rb_dtype dtype, const void* X, int64_t ldx, const void* Y,
                      int64_t ldy) {
  RB_REQUIRE(n >= 0, "%s: negative n", fn);
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "%s: k = %d outside [1, %d]", fn, k, RB_MAX_K);
  RB_REQUIRE(dtype == RB_F64 || dtype == RB_F32, "%s: unknown dtype", fn);
  RB_REQUIRE(ldx >= k && ldy >= k, "%s: leading dimension smaller than k", fn);
  RB_REQUIRE(n == 0 || (X && Y), "%s: null X or Y", fn);
  const int eb = dtype == RB_F64 ? 8 : 4;
  RB_REQUIRE((uintptr_t)X % eb == 0 && (uintptr_t)Y % eb == 0, "%s: X or Y not aligned to the element size", fn);
  return RB_OK;
}

// vector width and threads per row for a block pair
void vec_kp(int eb, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y, int& vec, int& kp) {
  vec = pick_vec(eb, k, ldx, ldy, X, Y);
  while (next_pow2((k + vec - 1) / vec) > 32 && vec < 16 / eb && k % (vec * 2) == 0) vec *= 2;
  kp = next_pow2((k + vec - 1) / vec);
}

}  // namespace

size_t dot_partials(int64_t n, int k) {
  (void)k;
  return (size_t)kBlasGrid * k * sizeof(double) + 256;
}

}  // namespace rb

using namespace rb;

extern "C" size_t rb_dot_workspace_bytes(int64_t n, int32_t k) {
  if (k < 1 || k > RB_MAX_K || n < 0) return 0;
  return dot_partials(n, k);
}

namespace rb {
// Calls f(std::integral_constant<int, V>) for the vector width V; widths above 16 bytes are
// never instantiated.
template <typename T, class F>
void with_vec(int vec, F&& f) {
  switch (vec) {
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 4:
      if constexpr (sizeof(T) == 4) f(std::integral_constant<int, 4>{});
      break;
  }
}
}  // namespace rb

#define RB_DISPATCH_VEC(T, vec, ...) \
  with_vec<T>(vec, [&](auto vv_) { constexpr int V = decltype(vv_)::value; __VA_ARGS__; })

extern "C" rb_status rb_dot(int64_t n, int32_t k, rb_dtype dtype, const void* X, int64_t ldx, const void* Y,
                            int64_t ldy, double* out, void* work, size_t work_bytes, rb_stream_t stream) {
  clear_error();
  RB_TRY(check_block("rb_dot", n, k, dtype, X, ldx, Y, ldy));
  RB_REQUIRE(out != nullptr, "rb_dot: null output");
  RB_REQUIRE(work != nullptr && work_bytes >= rb_dot_workspace_bytes(n, k), "rb_dot: workspace too small (%zu < %zu)",
             work_bytes, rb_dot_workspace_bytes(n, k));
  RB_REQUIRE((uintptr_t)work % 16 == 0, "rb_dot: workspace not 16-byte aligned");
  cudaStream_t s = S(stream);
  const int eb = dtype == RB_F64 ? 8 : 4;
  int vec, kp;
  vec_kp(eb, k, ldx, ldy, X, Y, vec, kp);
  RB_REQUIRE(kp <= 32, "rb_dot: k = %d needs 16-byte aligned rows", k);
  const int64_t blocks = std::max<int64_t>(1, (n + kThreads / kp - 1) / (kThreads / kp));
  int grid = 1;
  double* partials = static_cast<double*>(work);
  if (k <= kFlatMaxK && flat_ok(k, ldx, ldy, X, Y)) {
    const int64_t total = n * k;
    if (dtype == RB_F64) RB_TRY(launch_dot_flat<double>(total, k, (const double*)X, (const double*)Y, partials, grid, s));
    else RB_TRY(launch_dot_flat<float>(total, k, (const float*)X, (const float*)Y, partials, grid, s));
  } else if (dtype == RB_F64) {
    RB_DISPATCH_VEC(double, vec, grid = wave_grid(&k_dot_partial<double, V>, blocks);
                    k_dot_partial<double, V><<<grid, kThreads, 0, s>>>(n, k, kp, (const double*)X, ldx,
                                                                       (const double*)Y, ldy, partials));
  } else {
    RB_DISPATCH_VEC(float, vec, grid = wave_grid(&k_dot_partial<float, V>, blocks);
                    k_dot_partial<float, V><<<grid, kThreads, 0, s>>>(n, k, kp, (const float*)X, ldx,
                                                                      (const float*)Y, ldy, partials));
  }
  k_dot_final<<<1, kThreads, 0, s>>>(k, grid, partials, out);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

extern "C" rb_status rb_axpy(int64_t n, int32_t k, rb_dtype dtype, const double* alpha, const void* X, int64_t ldx,
                             void* Y, int64_t ldy, rb_stream_t stream) {
  clear_error();
  RB_TRY(check_block("rb_axpy", n, k, dtype, X, ldx, Y, ldy));
  RB_REQUIRE(alpha != nullptr, "rb_axpy: null alpha");
  if (n == 0) return RB_OK;
  cudaStream_t s = S(stream);
  const int eb = dtype == RB_F64 ? 8 : 4;
  int vec, kp;
  vec_kp(eb, k, ldx, ldy, X, Y, vec, kp);
  RB_REQUIRE(kp <= 32, "rb_axpy: k = %d needs 16-byte aligned rows", k);
  const int64_t blocks = (n + kThreads / kp - 1) / (kThreads / kp);
  if (flat_ok(k, ldx, ldy, X, Y)) {
    const int64_t total = n * k;
    if (dtype == RB_F64)
      k_axpy_flat<double><<<flat_grid(&k_axpy_flat<double>, total, 8, k), kThreads, 0, s>>>(
          total, k, alpha, (const double*)X, (double*)Y);
    else
      k_axpy_flat<float><<<flat_grid(&k_axpy_flat<float>, total, 4, k), kThreads, 0, s>>>(
          total, k, alpha, (const float*)X, (float*)Y);
  } else if (dtype == RB_F64) {
    RB_DISPATCH_VEC(double, vec,
                    k_axpy<double, V><<<wave_grid(&k_axpy<double, V>, blocks), kThreads, 0, s>>>(
                        n, k, kp, alpha, (const double*)X, ldx, (double*)Y, ldy));
  } else {
    RB_DISPATCH_VEC(float, vec,
                    k_axpy<float, V><<<wave_grid(&k_axpy<float, V>, blocks), kThreads, 0, s>>>(
                        n, k, kp, alpha, (const float*)X, ldx, (float*)Y, ldy));
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T, bool UNIT>
rb_status launch_axty(int64_t n, int k, int vec, int kp, T alpha, const void* X, int64_t ldx, void* Y, int64_t ldy,
                      cudaStream_t s) {
  if (flat_ok(k, ldx, ldy, X, Y)) {
    const int64_t total = n * k;
    k_axty_flat<T, UNIT><<<flat_grid(&k_axty_flat<T, UNIT>, total, (int)sizeof(T), 1), kThreads, 0, s>>>(
        total, alpha, (const T*)X, (T*)Y);
  } else {
    const int64_t blocks = (n + kThreads / kp - 1) / (kThreads / kp);
    RB_DISPATCH_VEC(T, vec,
                    k_axty<T, V, UNIT><<<wave_grid(&k_axty<T, V, UNIT>, blocks), kThreads, 0, s>>>(
                        n, k, kp, alpha, (const T*)X, ldx, (T*)Y, ldy));
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

extern "C" rb_status rb_axty(int64_t n, int32_t k, rb_dtype dtype, double alpha, const void* X, int64_t ldx, void* Y,
                             int64_t ldy, rb_stream_t stream) {
  clear_error();
  RB_TRY(check_block("rb_axty", n, k, dtype, X, ldx, Y, ldy));
  if (n == 0) return RB_OK;
  cudaStream_t s = S(stream);
  const int eb = dtype == RB_F64 ? 8 : 4;
  int vec, kp;
  vec_kp(eb, k, ldx, ldy, X, Y, vec, kp);
  RB_REQUIRE(kp <= 32, "rb_axty: k = %d needs 16-byte aligned rows", k);
  if (dtype == RB_F64) {
    if (alpha == 1.0) return launch_axty<double, true>(n, k, vec, kp, 1.0, X, ldx, Y, ldy, s);
    return launch_axty<double, false>(n, k, vec, kp, alpha, X, ldx, Y, ldy, s);
  }
  if ((float)alpha == 1.0f) return launch_axty<float, true>(n, k, vec, kp, 1.0f, X, ldx, Y, ldy, s);
  return launch_axty<float, false>(n, k, vec, kp, (float)alpha, X, ldx, Y, ldy, s);
}

// ---------------------------------------------------------------------------------------
// rb_dot_noalloc: rb_dot for callers that cannot hand the library device memory.
//
// Some callers have no device allocator to draw a workspace from: a plain C program or a
// plugin inside a host application that does not own the GPU's memory pool, or a code path
// that must not call cudaMalloc / cudaFree because those can synchronise the whole device.
// This entry point computes the same per-column dot products as rb_dot but keeps its
// per-block partial sums in a fixed array in the library's own device memory, declared
// below, instead of in a caller-provided workspace.  It allocates nothing.
//
// The array holds kNoAllocBlocks x RB_MAX_K partial sums (256 x 64 doubles, 128 KiB); every
// GPU that loads the library holds it until the process exits.  The reduction uses at most
// kNoAllocBlocks blocks, so any n and any k <= RB_MAX_K fit; k beyond that is rejected.
// All calls share the one array and each call overwrites what it uses (the first kernel
// writes every partial sum the second one reads, so nothing needs clearing first), which
// means two calls whose kernels overlap on the GPU (different streams, or host threads)
// race on it: such callers must order their calls themselves.
// ---------------------------------------------------------------------------------------
namespace rb {
namespace {

constexpr int kNoAllocBlocks = 256;
static __device__ __align__(256) double g_dot_scratch[kNoAllocBlocks * RB_MAX_K];

// Device address of g_dot_scratch on the current device.  The host-side symbol is only a
// stand-in, so the address is looked up once per device (with that device current) the
// first time the entry point runs there, and cached.
rb_status dot_scratch_address(double** out) {
  static std::mutex mu;
  static std::map<int, double*> cache;
  int dev = 0;
  RB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    void* p = nullptr;
    RB_CUDA(cudaGetSymbolAddress(&p, g_dot_scratch));
    it = cache.emplace(dev, static_cast<double*>(p)).first;
  }
  *out = it->second;
  return RB_OK;
}

}  // namespace
}  // namespace rb

extern "C" rb_status rb_dot_noalloc(int64_t n, int32_t k, rb_dtype dtype, const void* X, int64_t ldx, const void* Y,
                                    int64_t ldy, double* out, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K,
             "rb_dot_noalloc: k = %d outside [1, %d], the columns its fixed scratch of %d x %d partial sums holds", k,
             RB_MAX_K, kNoAllocBlocks, RB_MAX_K);
  RB_TRY(check_block("rb_dot_noalloc", n, k, dtype, X, ldx, Y, ldy));
  RB_REQUIRE(out != nullptr, "rb_dot_noalloc: null output");
  double* partials = nullptr;
  RB_TRY(dot_scratch_address(&partials));
  cudaStream_t s = S(stream);
  const int eb = dtype == RB_F64 ? 8 : 4;
  int vec, kp;
  vec_kp(eb, k, ldx, ldy, X, Y, vec, kp);
  RB_REQUIRE(kp <= 32, "rb_dot_noalloc: k = %d needs 16-byte aligned rows", k);
  const int64_t blocks = std::max<int64_t>(1, (n + kThreads / kp - 1) / (kThreads / kp));
  int grid = 1;
  if (dtype == RB_F64) {
    RB_DISPATCH_VEC(double, vec, grid = std::min(kNoAllocBlocks, wave_grid(&k_dot_partial<double, V>, blocks));
                    k_dot_partial<double, V><<<grid, kThreads, 0, s>>>(n, k, kp, (const double*)X, ldx,
                                                                       (const double*)Y, ldy, partials));
  } else {
    RB_DISPATCH_VEC(float, vec, grid = std::min(kNoAllocBlocks, wave_grid(&k_dot_partial<float, V>, blocks));
                    k_dot_partial<float, V><<<grid, kThreads, 0, s>>>(n, k, kp, (const float*)X, ldx,
                                                                      (const float*)Y, ldy, partials));
  }
  k_dot_final<<<1, kThreads, 0, s>>>(k, grid, partials, out);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}
