// Building blocks of the CSR SpMM shared by the standalone SpMM and the fused CG kernels:
// staging a block's rows (row pointers, column indices, values) in shared memory, and the
// per-(row, chunk) accumulation over the row's nonzeros.
#pragma once

#include "common.cuh"

namespace rb {

template <typename T>
struct CsrArgs {
  int n_rows = 0;
  const int32_t* __restrict__ rp = nullptr;
  const int32_t* __restrict__ ci = nullptr;
  const T* __restrict__ va = nullptr;
  const T* __restrict__ X = nullptr;
  int64_t ldx = 0;
  T* __restrict__ Y = nullptr;
  int64_t ldy = 0;
  int k = 1;
  int kp = 1;
  int stage_cap = 0;  // nonzeros a block may stage in shared memory (0: read from global)
  const double* __restrict__ cs = nullptr;
  // extruded operator: Y = A' X + w_i (x_{z-1} + x_{z+1}) across the k periodic columns, A'
  // the stored values (dz A~ with -2 w_i folded into the diagonal)
  const T* __restrict__ zw = nullptr;
  // row blocks that address the same columns in the same order (the x, y, z faces of a
  // gradient): the direct kernel takes tiles from the blocks in turn (nblk > 1)
  int nblk = 1;
  int blk_off[4] = {0, 0, 0, 0};  // block starts and the end (nblk + 1 entries)
};

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }

template <typename T>
__host__ __device__ inline size_t csr_smem_bytes(int R, int cap) {
  return (size_t)4 * round4(R + 1) + (size_t)4 * round4(cap) + sizeof(T) * (size_t)cap;
}

// Nonzeros a block of R rows stages: room for 1.25x the average row plus slack, kept under
// 48 KB so that several blocks share an SM.
// `limit` is the dynamic shared memory the kernel may use: 48 KB minus its static shared
// memory, so that no launch needs the opt-in for more than 48 KB per block.
template <typename T>
inline int stage_capacity(const rb_op* op, int R, int stage, size_t limit) {
  if (!stage) return 0;
  int cap = (int)((double)R * (op->avg_row_len * 1.25 + 1.0)) + 32;
  cap = round4(cap);
  while (cap > 4 && csr_smem_bytes<T>(R, cap) > limit) cap -= 4;
  return cap;
}

template <typename T>
inline void fill_csr_args(const rb_op* op, const SpmmSched& sc, CsrArgs<T>& a, size_t smem_limit = 48 * 1024) {
  a.n_rows = op->n_rows;
  a.rp = op->row_ptr;
  a.ci = op->col_idx;
  a.va = static_cast<const T*>(op->vals);
  a.kp = sc.kp;
  a.stage_cap = stage_capacity<T>(op, sc.rows_per_block(), sc.stage, smem_limit);
  a.zw = (sizeof(T) == 8) ? reinterpret_cast<const T*>(op->zw64) : reinterpret_cast<const T*>(op->zw32);
  a.nblk = op->n_rblk > 1 ? op->n_rblk : 1;
  for (int b = 0; b <= a.nblk && b < 4; ++b) a.blk_off[b] = op->rblk_off[b];
  if (a.nblk == 1) a.blk_off[0] = 0, a.blk_off[1] = op->n_rows;
}

struct TileInfo {
  int r0, nr, base, cnt;
  bool staged;
};

// Loads the row pointers of rows [r0, r0 + nr) and, when they fit, the block's nonzeros
// into shared memory.  Called by all threads of the block; ends with a barrier.
template <typename T>
__device__ __forceinline__ TileInfo stage_rows(const CsrArgs<T>& a, int r0, int R, int32_t* s_rp, int32_t* s_ci,
                                               T* s_va) {
  TileInfo ti;
  ti.r0 = r0;
  ti.nr = min(R, a.n_rows - r0);
  __syncthreads();  // previous users of the shared arrays are done
  for (int i = threadIdx.x; i <= ti.nr; i += blockDim.x) s_rp[i] = __ldg(a.rp + r0 + i);
  __syncthreads();
  ti.base = s_rp[0];
  ti.cnt = s_rp[ti.nr] - ti.base;
  ti.staged = a.stage_cap > 0 && ti.cnt <= a.stage_cap;
  if (ti.staged) {
    const int32_t* ci = a.ci + ti.base;
    const T* va = a.va + ti.base;
    for (int e = threadIdx.x; e < ti.cnt; e += blockDim.x) {
      s_ci[e] = __ldg(ci + e);
      s_va[e] = __ldg(va + e);
    }
  }
  __syncthreads();
  return ti;
}

// acc += sum over the nonzeros p = rs + sub, rs + sub + LPR, ... of row rloc of
// val[p] * X[idx[p], chunk * VEC .. chunk * VEC + VEC).
// Must be called by every thread of the warp when LPR > 1 (the reduction shuffles);
// inactive threads contribute zero.
template <typename T, int VEC, int LPR>
__device__ __forceinline__ void row_accumulate(const CsrArgs<T>& a, const TileInfo& ti, const int32_t* s_rp,
                                               const int32_t* s_ci, const T* s_va, int rloc, int chunk, int sub,
                                               bool active, T (&acc)[VEC]) {
  const int rs = active ? s_rp[rloc] - ti.base : 0;
  const int re = active ? s_rp[rloc + 1] - ti.base : 0;
  const T* Xc = a.X + chunk * VEC;
  if (ti.staged) {
#pragma unroll 2
    for (int p = rs + sub; p < re; p += LPR) {
      const int c = s_ci[p];
      const T v = s_va[p];
      const Vec<T, VEC> x = ldv<T, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(v, x.v[e], acc[e]);
    }
  } else {
    const int32_t* ci = a.ci + ti.base;
    const T* va = a.va + ti.base;
#pragma unroll 2
    for (int p = rs + sub; p < re; p += LPR) {
      const int c = __ldg(ci + p);
      const T v = __ldg(va + p);
      const Vec<T, VEC> x = ldv<T, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(v, x.v[e], acc[e]);
    }
  }
  if constexpr (LPR > 1) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
    }
  }
}

// The spanwise coupling of the extruded operator: w_i (x_{z-1} + x_{z+1}) across the k (= Nz)
// periodic columns of row `row`, added to acc.  The operator's stored values already carry
// dz and, on the diagonal, the -2 w_i of the second difference (folded in when the operator
// was created), so two FP64 instructions per entry remain here instead of five.
template <typename T, int VEC>
__device__ __forceinline__ void extruded_epilogue(const CsrArgs<T>& a, int64_t row, int chunk, T (&acc)[VEC]) {
  const int nz = a.k;
  const T* xr = a.X + row * a.ldx;
  const Vec<T, VEC> xs = ldv<T, VEC>(xr + chunk * VEC);
  const int z0 = chunk * VEC;
  const T left = __ldg(xr + (z0 == 0 ? nz - 1 : z0 - 1));
  const T right = __ldg(xr + (z0 + VEC == nz ? 0 : z0 + VEC));
  const T w = __ldg(a.zw + row);
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const T xm = (e == 0) ? left : xs.v[e - 1];
    const T xp = (e == VEC - 1) ? right : xs.v[e + 1];
    acc[e] = fma(w, xm + xp, acc[e]);
  }
}

// Direct accumulation for one (row, chunk, sub) without shared-memory staging: the row's
// index and value loads are issued by all KP * LPR lanes of the row and served as one
// broadcast.  Must be called by every lane of the warp when LPR > 1.
// COHERENT: gather X through L2 only (X written by other blocks of the same launch).
template <typename T, int VEC, int LPR, bool COHERENT = false, bool KEEP = false>
__device__ __forceinline__ void row_accumulate_direct(const CsrArgs<T>& a, int64_t row, int chunk, int sub,
                                                      bool active, T (&acc)[VEC]) {
  int rs = 0, re = 0;
  if (active) {
    rs = __ldg(a.rp + row);
    re = __ldg(a.rp + row + 1);
  }
  const T* Xc = a.X + chunk * VEC;
  // FP64: unrolled by two only: with four, rows of 2 or 6 nonzeros (gradient, divergence) run
  // a remainder whose predicated-off FMAs still take FP64-pipe issue slots (+50% on G, k = 3).
  // FP32 with up to three columns per lane: four gathers in flight per lane hide more of
  // their latency (L f32 k = 3 40.7 -> 39.7 us, M f32 k = 1 35.0 -> 33.3 us); with 16-byte
  // gathers (VEC = 4) four deep was slower (k = 4 and 8, the extruded k = 64).
  constexpr int kUnroll = (sizeof(T) == 4 && VEC < 4) ? 4 : 2;
  // KEEP (the CG's q = A p): the gathered p lines get the evict_last L2 policy, so that the
  // next kernel of the iteration, which reads p again, finds them in L2 (the plain SpMM, whose
  // X is not read again, runs faster without it)
  uint64_t keep = 0;
  if constexpr (KEEP) keep = l2_keep_policy();
#pragma unroll kUnroll
  for (int p = rs + sub; p < re; p += LPR) {
    const int c = __ldg(a.ci + p);
    const T v = __ldg(a.va + p);
    Vec<T, VEC> x;
    if constexpr (COHERENT) x = ldv_cg<T, VEC>(Xc + (int64_t)c * a.ldx);
    else if constexpr (KEEP) x = ldv_keep<T, VEC>(Xc + (int64_t)c * a.ldx, keep);
    else x = ldv<T, VEC>(Xc + (int64_t)c * a.ldx);
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = fma(v, x.v[e], acc[e]);
  }
  if constexpr (LPR > 1) {
#pragma unroll
    for (int off = LPR / 2; off >= 1; off >>= 1) {
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
    }
  }
}

// Epilogue variants, chosen at compile time so that a launch without a column scale or
// without the spanwise coupling issues none of their instructions (not even predicated off).
constexpr int kEpiExt = 1;    // extruded operator: add the periodic spanwise second difference
constexpr int kEpiScale = 2;  // per-column scale c (Algorithm 1), NULL otherwise

template <typename T, int VEC, int EPI>
__device__ __forceinline__ void store_row(const CsrArgs<T>& a, int64_t row, int chunk, T (&acc)[VEC]) {
  if constexpr ((EPI & kEpiExt) != 0) extruded_epilogue<T, VEC>(a, row, chunk, acc);
  Vec<T, VEC> y;
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    if constexpr ((EPI & kEpiScale) != 0) y.v[e] = acc[e] * (T)a.cs[chunk * VEC + e];
    else y.v[e] = acc[e];
  }
  stv<T, VEC>(a.Y + row * a.ldy + chunk * VEC, y);
}

// SpMM without staging: a persistent grid strides over blocks of R = 256 / (KP LPR) rows;
// no block-wide barrier anywhere, so every warp keeps its gathers in flight independently.
// The same kernel for an operator whose rows come in blocks addressing the same columns in the
// same order (its row-block hint): tile q of block b is work item q * nblk + b, so that the
// tiles at one position of every block, which gather the same region of X, run at about the
// same time and find X in L2.  A separate kernel, so that the plain one's code is unaffected.
template <typename T, int VEC, int LPR, int EPI>
__global__ void __launch_bounds__(kThreads) k_spmm_direct_blk(CsrArgs<T> a) {
  const int R = kThreads / (a.kp * LPR);
  const int t = threadIdx.x;
  const int sub = t % LPR;
  const int rc = t / LPR;
  const int chunk = rc % a.kp;
  const int rloc = rc / a.kp;
  int64_t tiles = 0;
  for (int b = 0; b < a.nblk; ++b) tiles = max(tiles, (int64_t)(a.blk_off[b + 1] - a.blk_off[b] + R - 1) / R);
  for (int64_t w = blockIdx.x; w < tiles * a.nblk; w += gridDim.x) {
    const int b = (int)(w % a.nblk);
    const int64_t row = a.blk_off[b] + (w / a.nblk) * R + rloc;
    const bool active = row < a.blk_off[b + 1] && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
    row_accumulate_direct<T, VEC, LPR>(a, row, chunk, sub, active, acc);
    if (active && sub == 0) store_row<T, VEC, EPI>(a, row, chunk, acc);
  }
}

template <typename T, int VEC, int LPR, int EPI>
__global__ void __launch_bounds__(kThreads) k_spmm_direct(CsrArgs<T> a) {
  const int R = kThreads / (a.kp * LPR);
  const int t = threadIdx.x;
  const int sub = t % LPR;
  const int rc = t / LPR;
  const int chunk = rc % a.kp;
  const int rloc = rc / a.kp;
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
    row_accumulate_direct<T, VEC, LPR>(a, row, chunk, sub, active, acc);
    if (active && sub == 0) store_row<T, VEC, EPI>(a, row, chunk, acc);
  }
}

template <typename T, int VEC, int LPR, int EPI>
__global__ void __launch_bounds__(kThreads) k_spmm_csr(CsrArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int R = kThreads / (a.kp * LPR);
  int32_t* s_rp = reinterpret_cast<int32_t*>(smem_raw);
  int32_t* s_ci = s_rp + round4(R + 1);
  T* s_va = reinterpret_cast<T*>(s_ci + round4(a.stage_cap));
  const int t = threadIdx.x;
  const int sub = t % LPR;
  const int rc = t / LPR;
  const int chunk = rc % a.kp;
  const int rloc = rc / a.kp;
  for (int64_t tile = blockIdx.x; tile * R < a.n_rows; tile += gridDim.x) {
    const int r0 = (int)(tile * R);
    const TileInfo ti = stage_rows<T>(a, r0, R, s_rp, s_ci, s_va);
    const bool active = rloc < ti.nr && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
    row_accumulate<T, VEC, LPR>(a, ti, s_rp, s_ci, s_va, rloc, chunk, sub, active, acc);
    if (active && sub == 0) store_row<T, VEC, EPI>(a, (int64_t)r0 + rloc, chunk, acc);
  }
}

}  // namespace rb
