// SpMM with the matrix streamed through shared memory by TMA bulk copies.
//
// A persistent block owns tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... of R rows.  One
// producer warp keeps a ring of kTmaStages shared-memory stages filled: for each tile it
// waits until the consumers have released the stage (mbarrier "empty"), then issues bulk
// copies of the tile's row pointers and of its contiguous range of column indices and
// values, all completing on the stage's "full" mbarrier.  The eight consumer warps wait for
// "full", read the tile's nonzeros from shared memory (each value and index is fetched from
// HBM once and reused by the KP lanes of the row and all k columns), gather the rows of X,
// release the stage and write Y.  The boundaries of the producer's next 32 tiles are loaded
// in one warp-wide load, so the copy of a tile never waits on a row-pointer round trip.
//
// Every mbarrier wait is bounded (tma.cuh); on a timeout the thread records an error code
// in *err and leaves its loop, and the producer drains the copies it has issued before the
// block exits.
#pragma once

#include "spmm_impl.cuh"
#include "tma.cuh"

namespace rb {

constexpr int kTmaStages = 3;
constexpr int kTmaThreads = kThreads + 32;  // 8 consumer warps + 1 producer warp

__host__ __device__ inline size_t align128(size_t v) { return (v + 127) & ~(size_t)127; }

struct TmaLayout {
  int R, cap;
  size_t rp_off, ci_off, va_off, stage_bytes, hdr_off, bar_off, total;
};

template <typename T>
__host__ __device__ inline TmaLayout tma_layout(int R, int cap) {
  TmaLayout L;
  L.R = R;
  L.cap = cap;
  size_t off = 0;
  L.rp_off = off;
  off += align128((size_t)round4(R + 1) * 4);
  L.ci_off = off;
  off += align128((size_t)cap * 4);
  L.va_off = off;
  off += align128((size_t)cap * sizeof(T));
  L.stage_bytes = off;
  L.hdr_off = kTmaStages * L.stage_bytes;
  L.bar_off = L.hdr_off + 128;
  L.total = L.bar_off + 2 * kTmaStages * sizeof(uint64_t);
  return L;
}

// Staged nonzeros per stage: 1.25x the average row plus slack, a multiple of 4, and the
// whole ring within `limit` bytes of shared memory.
template <typename T>
inline int tma_capacity(const rb_op* op, int R, size_t limit) {
  int cap = round4((int)((double)R * (op->avg_row_len * 1.25 + 1.0)) + 16);
  while (cap > 16 && tma_layout<T>(R, cap).total > limit) cap -= 16;
  return cap;
}

template <typename T, int VEC, int EPI>
__global__ void __launch_bounds__(kTmaThreads) k_spmm_tma(CsrArgs<T> a, int R, int cap, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char sm[];
  const TmaLayout L = tma_layout<T>(R, cap);
  int* hdr = reinterpret_cast<int*>(sm + L.hdr_off);  // per stage: first staged nonzero, staged flag
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + kTmaStages;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = (a.n_rows + R - 1) / R;
  const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmaStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kThreads / 32);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == kThreads / 32) {
    // ------------------------------------------------------------------- producer warp
    int b = 0, e = 0;
    int armed = 0;
    int ok = 1;
    for (int i = 0; i < my_tiles; ++i) {
      if ((i & 31) == 0) {  // boundaries of this block's next 32 tiles, one per lane
        const int64_t ti = (int64_t)blockIdx.x + (int64_t)(i + lane) * gridDim.x;
        const int64_t r0 = ti * R < a.n_rows ? ti * R : a.n_rows;
        const int64_t r1 = r0 + R < a.n_rows ? r0 + R : a.n_rows;
        b = __ldg(a.rp + r0);
        e = __ldg(a.rp + r1);
      }
      const int p0 = __shfl_sync(0xffffffffu, b, i & 31);
      const int p1 = __shfl_sync(0xffffffffu, e, i & 31);
      if (lane == 0) {
        const int s = i % kTmaStages;
        const uint32_t ph = (uint32_t)(i / kTmaStages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u)) {
          atomicExch(err, 1);
          ok = 0;
        } else {
          const int t = (int)blockIdx.x + i * (int)gridDim.x;
          const int r0 = t * R;
          const int nr = min(R, a.n_rows - r0);
          const int p0a = p0 & ~3;
          const int cnt = (p1 - p0a + 3) & ~3;
          const int staged = cnt <= cap ? 1 : 0;
          hdr[2 * s] = p0a;
          hdr[2 * s + 1] = staged;
          const uint32_t rp_bytes = (uint32_t)round4(nr + 1) * 4u;
          const uint32_t bytes = rp_bytes + (staged ? (uint32_t)cnt * (4u + (uint32_t)sizeof(T)) : 0u);
          unsigned char* st = sm + (size_t)s * L.stage_bytes;
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_g2s(st + L.rp_off, a.rp + r0, rp_bytes, &full[s]);
          if (staged && cnt > 0) {
            bulk_g2s(st + L.ci_off, a.ci + p0a, (uint32_t)cnt * 4u, &full[s]);
            bulk_g2s(st + L.va_off, a.va + p0a, (uint32_t)cnt * (uint32_t)sizeof(T), &full[s]);
          }
          armed = i + 1;
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
    }
    // no copy may be in flight when the block exits
    if (lane == 0) {
      for (int i = armed > kTmaStages ? armed - kTmaStages : 0; i < armed; ++i)
        if (!mbar_wait(&full[i % kTmaStages], (uint32_t)(i / kTmaStages) & 1u)) atomicExch(err, 2);
    }
    return;
  }

  // --------------------------------------------------------------------- consumer warps
  const int chunk = threadIdx.x % a.kp;
  const int rloc = threadIdx.x / a.kp;
  for (int i = 0; i < my_tiles; ++i) {
    const int s = i % kTmaStages;
    const uint32_t ph = (uint32_t)(i / kTmaStages) & 1u;
    const bool got = mbar_wait(&full[s], ph);
    if (!__all_sync(0xffffffffu, got)) {  // leave as a whole warp
      if (lane == 0) atomicExch(err, 3);
      break;
    }
    const unsigned char* st = sm + (size_t)s * L.stage_bytes;
    const int* s_rp = reinterpret_cast<const int*>(st + L.rp_off);
    const int* s_ci = reinterpret_cast<const int*>(st + L.ci_off);
    const T* s_va = reinterpret_cast<const T*>(st + L.va_off);
    const int p0a = hdr[2 * s];
    const int staged = hdr[2 * s + 1];
    const int t = (int)blockIdx.x + i * (int)gridDim.x;
    const int64_t row = (int64_t)t * R + rloc;
    const bool active = rloc < R && row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int ee = 0; ee < VEC; ++ee) acc[ee] = T(0);
    if (active) {
      const int rs = s_rp[rloc] - p0a;
      const int re = s_rp[rloc + 1] - p0a;
      const T* Xc = a.X + chunk * VEC;
      if (staged) {
#pragma unroll 2
        for (int p = rs; p < re; ++p) {
          const int c = s_ci[p];
          const T v = s_va[p];
          const Vec<T, VEC> x = ldv<T, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
          for (int ee = 0; ee < VEC; ++ee) acc[ee] = fma(v, x.v[ee], acc[ee]);
        }
      } else {
#pragma unroll 2
        for (int p = rs; p < re; ++p) {
          const int c = __ldg(a.ci + p0a + p);
          const T v = __ldg(a.va + p0a + p);
          const Vec<T, VEC> x = ldv<T, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
          for (int ee = 0; ee < VEC; ++ee) acc[ee] = fma(v, x.v[ee], acc[ee]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // this warp no longer reads the stage
    if (active) store_row<T, VEC, EPI>(a, row, chunk, acc);
  }
}

}  // namespace rb
