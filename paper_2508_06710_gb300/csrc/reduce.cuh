// Deterministic per-column reductions over the rows of an n x k block.
//
// Threads are laid out as (row, chunk): thread t handles chunk t % KP (VEC consecutive
// columns) of some rows, KP a power of two <= 32, so within a warp the lanes with equal
// lane % KP hold the same columns.  A block folds its warps with xor shuffles (offsets >=
// KP), then sums the 8 warps in order; each block writes one partial per (quantity,
// column); the last block to finish (atomic ticket) sums the partials of all blocks in a
// fixed order.  The result does not depend on timing: bit-reproducible for fixed sizes.
#pragma once

#include "common.cuh"

namespace rb {

constexpr int kWarps = kThreads / 32;

// Shared scratch for block_reduce: kWarps * NQ * KP * VEC doubles (KP * VEC <= 64).
template <int NQ>
struct RedSmem {
  double v[kWarps][NQ][64];
  double fin[kThreads];  // one value per thread: [warp][lane] or flat
  int last;
};

// In: acc[q][e] for the thread's chunk.  Out: thread t < NQ * k receives the block total of
// quantity q = t / k, column j = t % k (other threads receive 0).
// With LPR > 1 lanes per row (thread t = (row * KP + chunk) * LPR + sub), only the sub == 0
// lanes may hold nonzero values; pass lpr so the fold and the chunk index account for it.
// The warp stage runs in the accumulators' own type A (FP32 for the FP32 solve, FP64
// otherwise); the warp totals are widened to FP64 for the block and grid stages.
template <int NQ, int VEC, typename A>
__device__ __forceinline__ double block_reduce(A (&acc)[NQ][VEC], int kp, int lpr, int k, RedSmem<NQ>& sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int width = kp * lpr;
#pragma unroll
  for (int q = 0; q < NQ; ++q) warp_fold<A, VEC>(acc[q], width);
  if (lane < width && (lane % lpr) == 0) {
    const int chunk = lane / lpr;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int e = 0; e < VEC; ++e) sm.v[w][q][chunk * VEC + e] = (double)acc[q][e];
  }
  __syncthreads();
  double r = 0.0;
  if ((int)threadIdx.x < NQ * k) {
    const int q = threadIdx.x / k, j = threadIdx.x % k;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) r += sm.v[ww][q][j];
  }
  return r;
}

// Writes this block's totals to partials[blockIdx.x * m + t] (m = NQ * k outputs) and
// returns true in every thread of the LAST block to arrive, after a fence that makes all
// blocks' partials visible.  The last block resets the ticket counter to zero.
template <int NQ>
__device__ __forceinline__ bool publish_partials(double v, int m, double* partials, unsigned* counter,
                                                 RedSmem<NQ>& sm) {
  if ((int)threadIdx.x < m) partials[(size_t)blockIdx.x * m + threadIdx.x] = v;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(counter, 1u);
    sm.last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  const bool last = sm.last != 0;
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

// In the last block: returns to thread t < m the sum over all blocks of partial t, summed
// in a fixed order (strided per thread group, then folded).  m <= 256.
template <int NQ>
__device__ __forceinline__ double final_sum(const double* partials, int m, int nblocks, RedSmem<NQ>& sm) {
  const int mp = next_pow2(m);  // outputs padded to a power of two
  const int groups = kThreads / mp > 0 ? kThreads / mp : 1;
  const int t = threadIdx.x;
  const int o = t % mp, g = t / mp;
  double s = 0.0;
  if (o < m && g < groups) {
    // unrolled so that the loads are in flight together; the additions keep their order
#pragma unroll 8
    for (int b = g; b < nblocks; b += groups) s += __ldcg(partials + (size_t)b * m + o);
  }
  // fold the groups: within a warp when mp <= 32, then across warps through shared memory
  const int lane = t & 31, w = t >> 5;
  if (mp <= 32) {
    for (int off = 16; off >= mp; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane < mp) sm.fin[w * 32 + lane] = s;
    __syncthreads();
    double r = 0.0;
    if (t < m)
      for (int ww = 0; ww < kWarps; ++ww) r += sm.fin[ww * 32 + t];
    __syncthreads();
    return r;
  }
  // mp > 32: each group spans mp / 32 warps; groups = 256 / mp <= 4
  double* flat = sm.fin;
  flat[t] = s;
  __syncthreads();
  double r = 0.0;
  if (t < m)
    for (int gg = 0; gg < groups; ++gg) r += flat[gg * mp + t];
  __syncthreads();
  return r;
}

}  // namespace rb
