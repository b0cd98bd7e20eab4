// Shared definitions of the repeated-block SpMM library: error state, the operator object,
// vector loads over the k interleaved columns, and block/grid reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <string>

#include "../../include/rbspmm.h"

namespace rb {

// ------------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
rb_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define RB_CUDA(call)                                                   \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) return rb::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define RB_REQUIRE(cond, ...)          \
  do {                                 \
    if (!(cond)) {                     \
      rb::set_error(__VA_ARGS__);      \
      return RB_EINVAL;                \
    }                                  \
  } while (0)

#define RB_TRY(expr)                \
  do {                              \
    rb_status s_ = (expr);          \
    if (s_ != RB_OK) return s_;     \
  } while (0)

inline cudaStream_t S(rb_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

constexpr int kThreads = 256;  // threads per block of every streaming kernel
constexpr int kMaxGrid = 152 * 8;  // 152 SMs x 8 resident blocks of 256 threads

// ------------------------------------------------------------------------------------------
// Schedules and the operator object
// ------------------------------------------------------------------------------------------
// One launch shape of the SpMM kernels: VEC consecutive columns per thread (16-byte loads
// when VEC * sizeof(T) == 16), KP = next power of two of k / VEC threads per row (so the
// threads of a row are aligned within a warp), LPR threads splitting one row's nonzeros
// (reduced with warp shuffles), and whether the block's nonzeros are staged in shared
// memory before use.
struct SpmmSched {
  int vec = 1;
  int kp = 1;
  int lpr = 1;
  int stage = 0;      // 1: stage the block's nonzeros in shared memory first
  int grid_cap = 0;   // direct kernel: persistent grid of at most this many blocks (0: one per row block)
  int rows_per_block() const { return kThreads / (kp * lpr); }
};

constexpr int kPersistentGrid = 152 * 8;  // 8 resident blocks of 256 threads on each of 152 SMs

// Blocks of `kernel` (kThreads threads, `smem` dynamic bytes) that fit on the device at
// once: multiprocessors x resident blocks per multiprocessor (cached per kernel).  Grid-
// stride kernels launch at most this many blocks, so they run in one wave whatever their
// register count, and never more than kPersistentGrid.
int resident_blocks(const void* kernel, size_t smem, int threads = kThreads);

// Raises `kernel`'s dynamic shared memory limit to at least `bytes` on the current device.
// The attribute belongs to the device, so the largest value set is remembered per (device,
// kernel); a host thread that moves to another device sets it again there.
rb_status opt_in_smem(const void* kernel, size_t bytes);

template <typename K>
inline int wave_grid(K* kernel, int64_t work_blocks, size_t smem = 0, int threads = kThreads) {
  const int cap = resident_blocks(reinterpret_cast<const void*>(kernel), smem, threads);
  return (int)std::max<int64_t>(1, std::min<int64_t>(work_blocks, cap));
}

}  // namespace rb

struct rb_op {
  int32_t n_rows = 0, n_cols = 0;
  int64_t nnz = 0;
  rb_dtype dtype = RB_F64;
  rb_format format = RB_CSR;
  int32_t k_max = 1;
  // CSR (arrays padded by 64 bytes so that aligned vector and bulk copies may read past nnz)
  int32_t* row_ptr = nullptr;
  int32_t* col_idx = nullptr;
  void* vals = nullptr;
  int32_t max_row_len = 0;
  double avg_row_len = 0.0;
  // sliced ELL (C rows per slice, column-major inside a slice)
  int32_t sell_c = 0, sell_sigma = 0, n_slices = 0;
  int64_t sell_nnz = 0;
  int32_t* sell_ptr = nullptr;   // n_slices + 1 offsets (entries)
  int32_t* sell_width = nullptr; // n_slices
  int32_t* sell_row = nullptr;   // n_slices * C: original row of each slot (-1: empty)
  int32_t* sell_col = nullptr;
  void* sell_val = nullptr;
  // Jacobi
  int32_t has_diag = 0;
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  // extruded along a periodic direction
  int32_t ext_nz = 0;
  double dz = 0.0;
  double* zw64 = nullptr;
  float* zw32 = nullptr;
  int64_t device_bytes = 0;
  // matrix-free 7-point Laplacian of a Cartesian grid (format RB_STENCIL): per-axis cell
  // widths and inverse centre distances in the operator's type, and the scale
  int32_t st_n[3] = {0, 0, 0}, st_per[3] = {0, 0, 0};
  void* st_w[3] = {nullptr, nullptr, nullptr};
  void* st_ic[3] = {nullptr, nullptr, nullptr};
  double st_scale = 1.0;
  int32_t n_rblk = 1;                     // row blocks addressing the same columns in order
  int32_t rblk_off[4] = {0, 0, 0, 0};      // their starts and the end (rb_operator_set_row_blocks)
  int* err = nullptr;  // device status word: nonzero after a bounded wait in a kernel gave up
  std::map<int, rb::SpmmSched> tuned;  // k -> schedule chosen by rb_tune_spmm
};

namespace rb {

// ------------------------------------------------------------------------------------------
// Vector access to VEC consecutive columns
// ------------------------------------------------------------------------------------------
template <typename T, int VEC>
struct Vec {
  T v[VEC];
};

template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv(const T* p) {
  Vec<T, VEC> r;
  if constexpr (sizeof(T) * VEC == 16) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    memcpy(&r, &q, 16);
  } else if constexpr (sizeof(T) * VEC == 8) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    memcpy(&r, &q, 8);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = __ldg(p + e);
  }
  return r;
}

// Plain (non read-only path) load, for data written earlier by the same kernel sequence.
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv_rw(const T* p) {
  Vec<T, VEC> r;
  if constexpr (sizeof(T) * VEC == 16) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    memcpy(&r, &q, 16);
  } else if constexpr (sizeof(T) * VEC == 8) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    memcpy(&r, &q, 8);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = p[e];
  }
  return r;
}

// L2-coherent load (bypasses L1 and the read-only path): for data other blocks of the same
// launch have written, as in the persistent solver between grid barriers.
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv_cg(const T* p) {
  Vec<T, VEC> r;
  if constexpr (sizeof(T) * VEC == 16) {
    const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
    memcpy(&r, &q, 16);
  } else if constexpr (sizeof(T) * VEC == 8) {
    const float2 q = __ldcg(reinterpret_cast<const float2*>(p));
    memcpy(&r, &q, 8);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = __ldcg(p + e);
  }
  return r;
}

// An L2 eviction policy that keeps lines longer (evict_last), for data re-read across a
// kernel (the SpMM's gathered X) while the matrix and the outputs stream past.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ double ld_keep(const double* p, uint64_t pol) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_keep(const float* p, uint64_t pol) {
  float v;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
  return v;
}

// ldv with the evict_last L2 policy (read-only data)
template <typename T, int VEC>
__device__ __forceinline__ Vec<T, VEC> ldv_keep(const T* p, uint64_t pol) {
  Vec<T, VEC> r;
  if constexpr (sizeof(T) == 8 && VEC == 2) {
    asm volatile("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p), "l"(pol));
  } else if constexpr (sizeof(T) == 4 && VEC == 4) {
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(p), "l"(pol));
  } else if constexpr (sizeof(T) == 4 && VEC == 2) {
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(r.v[0]), "=f"(r.v[1]) : "l"(p), "l"(pol));
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) r.v[e] = ld_keep(p + e, pol);
  }
  return r;
}

template <typename T, int VEC>
__device__ __forceinline__ void stv(T* p, const Vec<T, VEC>& r) {
  if constexpr (sizeof(T) * VEC == 16) {
    float4 q;
    memcpy(&q, &r, 16);
    *reinterpret_cast<float4*>(p) = q;
  } else if constexpr (sizeof(T) * VEC == 8) {
    float2 q;
    memcpy(&q, &r, 8);
    *reinterpret_cast<float2*>(p) = q;
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) p[e] = r.v[e];
  }
}

__host__ __device__ inline int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Largest VEC in {4, 2, 1} (4 only for 4-byte types: 16-byte loads) that divides k and the
// leading dimensions and keeps every row start aligned.
inline int pick_vec(int elem_bytes, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  for (int v = 16 / elem_bytes; v > 1; v >>= 1) {
    const uintptr_t a = (uintptr_t)v * elem_bytes;
    if (k % v == 0 && ldx % v == 0 && ldy % v == 0 && ((uintptr_t)X % a) == 0 && ((uintptr_t)Y % a) == 0) return v;
  }
  return 1;
}

// Whether VEC elements per thread can be loaded as one access: 8- and 16-byte accesses need
// the leading dimensions and bases aligned; other widths (3, or 4 doubles) use scalar loads.
inline bool vec_ok(int elem_bytes, int vec, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  if (vec < 1 || k % vec) return false;
  const int w = vec * elem_bytes;
  if (w == 8 || w == 16) {
    const uintptr_t a = (uintptr_t)w;
    return ldx % vec == 0 && ldy % vec == 0 && ((uintptr_t)X % a) == 0 && ((uintptr_t)Y % a) == 0;
  }
  return true;
}

// ------------------------------------------------------------------------------------------
// Reductions: per-column sums over the rows handled by a block.  Threads are laid out as
// (row, chunk) with KP chunks per row, KP a power of two dividing 32, so lanes with equal
// lane % KP hold the same columns.  The warp stage folds lanes with xor offsets >= KP; the
// block stage sums the warps in order.  Fixed order throughout: bit-reproducible.
// ------------------------------------------------------------------------------------------
template <typename A, int NV>
__device__ __forceinline__ void warp_fold(A (&a)[NV], int kp) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off >= kp) {
#pragma unroll
      for (int e = 0; e < NV; ++e) a[e] += __shfl_xor_sync(0xffffffffu, a[e], off);
    }
  }
}

}  // namespace rb
