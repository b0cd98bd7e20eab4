// Learned initial guess for the Poisson solve: a 3-D U-Net trained and evaluated with
// hand-written kernels.  The 3x3x3 convolutions (forward, input gradient, weight gradient)
// run on the tensor cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators
// in tensor memory); pooling, the 2x2x2 transposed convolution, the head, the loss and Adam
// are streaming kernels on the CUDA cores.
//
// Activations are BF16, channel-last: the c channels of cell v at base[v * ld + c], ld a
// multiple of 8 so that every 8-channel group is one aligned 16-byte chunk (one row of a
// tensor-core core matrix).  A decoder level's input is one buffer [cells][2 c]: the
// transposed convolution writes channels [0, c), the encoder writes its output into
// channels [c, 2 c) directly, so the skip concatenation costs nothing.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "umma.cuh"

namespace rb {
namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------------------ geometry

struct Dims {
  int nx = 1, ny = 1, nz = 1;
  int px = 1, py = 1, pz = 0;  // periodic flags
  __host__ __device__ int n() const { return nx * ny * nz; }
};

// Neighbour (x + dx, y + dy, z + dz) of cell v: its index, or -1 outside a walled axis.
__device__ __forceinline__ int neighbour(const Dims& d, int x, int y, int z, int dx, int dy, int dz) {
  x += dx;
  y += dy;
  z += dz;
  if (x < 0 || x >= d.nx) {
    if (!d.px) return -1;
    x = x < 0 ? x + d.nx : x - d.nx;
  }
  if (y < 0 || y >= d.ny) {
    if (!d.py) return -1;
    y = y < 0 ? y + d.ny : y - d.ny;
  }
  if (z < 0 || z >= d.nz) {
    if (!d.pz) return -1;
    z = z < 0 ? z + d.nz : z - d.nz;
  }
  return x + d.nx * (y + d.ny * z);
}

// tap index (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1), offsets in -1..1
__device__ __forceinline__ void tap_offsets(int tap, int& dx, int& dy, int& dz) {
  dz = tap / 9 - 1;
  dy = (tap / 3) % 3 - 1;
  dx = tap % 3 - 1;
}

// ------------------------------------------------------------------ 3x3x3 convolution (MMA)
//
// Implicit GEMM: D[cell m][out channel n] = sum_K A[m][K] B[n][K], K = tap * c_in + ci.
// A is gathered from the input cells' neighbours (16 bytes = 8 channels of one tap per
// copy, zeros past a wall), B is the weight matrix [NP][kpad] (K-major, zero padded), held
// in shared memory for the whole launch.  One CTA of 128 threads (thread = cell row of the
// 128-cell tile) runs a ring of kStages A slots of kKS K-columns: cp.async gathers run
// kAhead stages ahead, one thread issues a stage's two MMAs and commits them to the slot's
// mbarrier, which frees the slot for the gather kStages - kAhead stages later.  Two TMEM accumulators alternate
// between tiles, and a tile's epilogue (TMEM -> registers -> bias, ReLU / mask -> BF16) runs
// after the next tile's first MMAs have been issued.
//
// The same kernel computes the input gradient of a convolution: correlation of the output
// gradient with the weights flipped in all three offsets and transposed (c_in <-> c_out),
// with the padding rules unchanged.

constexpr int kConvThreads = 128;
constexpr int kKS = 32;                     // K columns per stage (two K = 16 MMAs)
constexpr int kStages = 8;                  // A ring slots
constexpr int kAhead = 4;                   // stages gathered ahead of the one being issued
// A slot is refilled kStages - kAhead stages after its MMAs were issued, so the gathers never
// wait for the tensor cores' latency of the stage just issued.
constexpr int kAStage = 128 * kKS * 2;      // bytes of one A stage (8 KB)
constexpr uint32_t kSboA = (kKS / 8) * 128; // A: core matrices adjacent along M
constexpr size_t kMaxConvSmem = 200 * 1024;
constexpr int kMaxChunks = 512;             // K_pad / 8 of any convolution (27 c_in <= 4096)

struct Conv3Args {
  const bf16* x = nullptr;
  int ldx = 0, cin = 0;  // input channels (multiple of 8)
  Dims d;
  int n_vox = 0;
  const bf16* w = nullptr;  // [NP][kpad]
  int kpad = 0;             // multiple of kKS, >= 27 cin
  const float* bias = nullptr;
  int relu = 0;
  const bf16* mask = nullptr;  // zero the output where mask <= 0 (input-gradient pass)
  int ldm = 0;
  bf16* y = nullptr;
  int ldy = 0, cout = 0;  // output channels (multiple of 8, <= NP)
  int* err = nullptr;
};

__host__ __device__ constexpr uint32_t tmem_cols_for(int np2) {
  return np2 <= 32 ? 32u : (np2 <= 64 ? 64u : (np2 <= 128 ? 128u : 256u));
}

template <int NP>
__global__ void __launch_bounds__(kConvThreads) k_conv3_mma(Conv3Args a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t slot_bar[kStages];
  __shared__ __align__(8) uint64_t acc_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int chunk_tab[kMaxChunks];
  constexpr uint32_t kCols = tmem_cols_for(2 * NP);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sB = smem_u32(smem);
  const uint32_t sA = sB + (uint32_t)(NP * a.kpad * 2);
  const uint32_t sbo_b = (uint32_t)(a.kpad / 8) * 128;
  const int S = a.kpad / kKS;
  const int n_tiles = (a.n_vox + 127) / 128;
  const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int T = my_tiles * S;
  const uint32_t idesc = umma_idesc_bf16(128, NP, false, false);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&slot_bar[i], 1);
    mbar_init(&acc_bar[0], 1);
    mbar_init(&acc_bar[1], 1);
    mbar_init(&drain_bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCols);

  // weights -> shared, K-major canonical layout: core (n / 8, q) at (n / 8) sbo_b + 128 q
  const int kc = a.kpad / 8;
  for (int i = tid; i < NP * kc; i += kConvThreads) {
    const int n = i / kc, q = i - n * kc;
    cp_async16(sB + (uint32_t)(n >> 3) * sbo_b + (uint32_t)q * 128 + (uint32_t)(n & 7) * 16,
               a.w + (size_t)n * a.kpad + (size_t)q * 8, 16);
  }

  // per 16-byte K chunk q (8 channels of one tap): packed (dx+1) | (dy+1) << 2 | (dz+1) << 4 |
  // ci0 << 8, or -1 past the 27 taps; built once per CTA so the gathers divide nothing
  for (int q = tid; q < kc; q += kConvThreads) {
    const int kk = q * 8, tap = kk / a.cin;
    chunk_tab[q] = tap < 27 ? ((tap % 3) | ((tap / 3) % 3) << 2 | (tap / 9) << 4 | (kk - tap * a.cin) << 8) : -1;
  }
  __syncthreads();
  // the cell of this thread in the tile last decomposed (tiles change every S stages)
  int cur_ti = -1, cx = 0, cy = 0, cz = 0;
  bool cvalid = false;

  // gather of stage j (tile j / S, K columns [(j % S) kKS, +kKS)) into ring slot j % kStages
  auto load_stage = [&](int j) {
    const int ti = j / S, s = j - ti * S;
    if (ti != cur_ti) {
      cur_ti = ti;
      const int v = ((int)blockIdx.x + ti * (int)gridDim.x) * 128 + tid;
      cvalid = v < a.n_vox;
      const int r = v / a.d.nx;
      cx = v - r * a.d.nx;
      cz = r / a.d.ny;
      cy = r - cz * a.d.ny;
    }
    const uint32_t dst = sA + (uint32_t)(j % kStages) * kAStage + (uint32_t)(tid >> 3) * kSboA + (uint32_t)(tid & 7) * 16;
#pragma unroll
    for (int jq = 0; jq < kKS / 8; ++jq) {
      const int e = chunk_tab[s * (kKS / 8) + jq];
      const bf16* src = a.x;
      uint32_t bytes = 0;
      if (cvalid && e >= 0) {
        const int nb = neighbour(a.d, cx, cy, cz, (e & 3) - 1, ((e >> 2) & 3) - 1, ((e >> 4) & 3) - 1);
        if (nb >= 0) {
          src = a.x + (size_t)nb * a.ldx + (e >> 8);
          bytes = 16;
        }
      }
      cp_async16(dst + (uint32_t)jq * 128, src, bytes);
    }
  };

  uint32_t tmem = 0;
  int fail = 0;
  auto epilogue = [&](int e) {
    const int b = e & 1;
    if (!mbar_wait(&acc_bar[b], (uint32_t)(e >> 1) & 1u)) fail = 1;
    tc_fence_after();
    const int t = (int)blockIdx.x + e * (int)gridDim.x;
    const int v = t * 128 + tid;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * NP);
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float acc[16];
      tmem_ld16(taddr + (uint32_t)c0, acc);  // whole warp, valid cell or not
      if (fail || v >= a.n_vox) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = c0 + 8 * h;
        if (cb >= a.cout) continue;
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float val = acc[8 * h + i];
          if (a.bias) val += __ldg(a.bias + cb + i);
          if (a.relu) val = fmaxf(val, 0.0f);
          o[i] = val;
        }
        if (a.mask) {
          const uint4 mq = *reinterpret_cast<const uint4*>(a.mask + (size_t)v * a.ldm + cb);
          const bf16* mv = reinterpret_cast<const bf16*>(&mq);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (!(__bfloat162float(mv[i]) > 0.0f)) o[i] = 0.0f;
        }
        uint4 q;
        __nv_bfloat162* qp = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) qp[i] = __floats2bfloat162_rn(o[2 * i], o[2 * i + 1]);
        *reinterpret_cast<uint4*>(a.y + (size_t)v * a.ldy + cb) = q;
      }
    }
  };

  // prologue: weights and the first kAhead stages (the weights ride in group 0)
  for (int j = 0; j < kAhead; ++j) {
    if (j < T) load_stage(j);
    cp_async_commit();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  tmem = tmem_slot;

  for (int j = 0; j < T; ++j) {
    const int ti = j / S, s = j - ti * S;
    cp_async_wait<kAhead - 1>();  // stage j has landed (this thread's copies)
    fence_proxy_async();
    if (__syncthreads_or(fail)) break;
    if (tid == 0) {
      tc_fence_after();
      const int slot = j % kStages;
      const uint32_t d = tmem + (uint32_t)((ti & 1) * NP);
#pragma unroll
      for (int ks = 0; ks < kKS / 16; ++ks) {
        const uint64_t ad = umma_sdesc(sA + (uint32_t)slot * kAStage + (uint32_t)ks * 256, 128, kSboA);
        const uint64_t bd = umma_sdesc(sB + (uint32_t)(s * (kKS / 16) + ks) * 256, 128, sbo_b);
        umma_bf16(d, ad, bd, idesc, (s > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&slot_bar[slot]);
      if (s == S - 1) umma_commit(&acc_bar[ti & 1]);
    }
    // gather stage j + kAhead into the slot of stage j + kAhead - kStages once its MMAs are done
    const int jn = j + kAhead;
    if (jn < T) {
      const int jo = jn - kStages;
      if (jo >= 0 && !mbar_wait(&slot_bar[jo % kStages], (uint32_t)(jo / kStages) & 1u)) fail = 1;
      if (!fail) load_stage(jn);
    }
    cp_async_commit();
    if (s == 0 && ti > 0) epilogue(ti - 1);
    if (j == T - 1) epilogue(ti);
  }
  cp_async_wait_all();
  // drain: every MMA this CTA issued has completed before TMEM is released
  if (tid == 0) {
    umma_commit(&drain_bar);
    if (!mbar_wait(&drain_bar, 0)) fail = 1;
  }
  if (fail && a.err) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ------------------------------------------------ 3x3x3 convolution on 128-cell rows (MMA)
//
// When a grid row holds exactly W = 128 or 64 cells (the MMA's M), the 27 taps need no
// gathered copy: each CTA keeps the three input lines (z - 1, z, z + 1) of four consecutive y
// rows in a shared-memory ring, one line = W + 2 cells (the row and its x neighbours, wrapped or zero)
// of 8 channels (16 bytes) per channel group, and the A operand of tap (dz, dy, dx) is a
// descriptor into line (z + dz, y + dy) starting at cell dx + 1: core matrices of 8 cells are
// 128 bytes apart (SBO), and the second K core of an MMA is the next channel group (LBO =
// the group stride) or, with 8 channels, the next x offset (LBO = 16 bytes; the third x
// offset of a line pairs with zero weights).  Each input line is loaded for three y rows
// instead of being gathered for 27 taps.  A CTA walks `chunk` consecutive rows of one z
// plane; the loads of row y + 2 overlap the MMAs of row y and the epilogue of row y - 1.
// Row widths W: 128 cells (MMA M = 128, accumulator row m in TMEM lane m) and 64 cells
// (M = 64: row m in lane 32 (m / 16) + m % 16, the first 16 lanes of each warp's quarter).
// rows per work item: long runs reuse the ring (2 halo rows per run), short runs give more
// items; the launch picks the longest run that still yields enough items to fill the GPU
// Forward and input-gradient launches: the rows of each z plane are cut into the most equal
// runs that still give one run per resident CTA (resident / nz runs per plane, at least one),
// so that no CTA waits for a second run while others idle.  (Runs of 16 rows over 1024
// items and 912 resident CTAs at 128^3 left 112 CTAs a second run: the launch took 32
// row-steps for an average of 18.)
inline int row_chunk_fill(int ny, int nz, int resident) {
  const int parts = std::max(1, std::min(ny, resident / std::max(nz, 1)));
  return (ny + parts - 1) / parts;
}
inline int row_chunk(int ny, int nz, int want_items) {
  int c = 16;
  while (c > 2 && nz * ((ny + c - 1) / c) < want_items) c /= 2;
  return c;
}
__host__ __device__ constexpr int row_pos(int W) { return W + 2; }
__host__ __device__ constexpr uint32_t line_bytes(int W) { return (uint32_t)(W + 2) * 16; }
__host__ __device__ constexpr uint32_t group_bytes(int W) { return 12 * line_bytes(W); }  // 3 z lines x 4 slots

__host__ __device__ inline int row_k(int cin) { return cin == 8 ? 9 * 4 * 8 : 27 * cin; }
inline size_t row_smem(int np, int cin, int W) {
  return (size_t)np * row_k(cin) * 2 + (size_t)(cin / 8) * group_bytes(W) + 256;
}

template <int NP, int W>
__global__ void __launch_bounds__(kConvThreads) k_conv3_row(Conv3Args a, int chunk) {
  constexpr uint32_t kLineBytes = line_bytes(W), kGroupBytes = group_bytes(W);
  constexpr int kRowPos = row_pos(W);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t acc_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  constexpr uint32_t kCols = tmem_cols_for(2 * NP);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int G = a.cin / 8;
  const int krow = row_k(a.cin);
  const uint32_t sB = smem_u32(smem);
  const uint32_t sL = sB + (uint32_t)(NP * krow * 2);
  const uint32_t sbo_b = (uint32_t)(krow / 8) * 128;
  const int ny = a.d.ny, nz = a.d.nz;
  const int chunks_y = (ny + chunk - 1) / chunk;
  const int items = nz * chunks_y;
  const uint32_t idesc = umma_idesc_bf16(W, NP, false, false);

  if (tid == 0) {
    mbar_init(&acc_bar[0], 1);
    mbar_init(&acc_bar[1], 1);
    mbar_init(&drain_bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCols);
  // With 8-channel inputs the third x offset of a line is paired with a zero-weight core that
  // reads 16 bytes into the next line of the ring (or the pad after the last): those bytes must
  // be finite (0 x NaN = NaN), so the whole ring and the pad start as zeros; every line
  // written later holds finite activations.
  for (uint32_t off = (uint32_t)tid * 16; off < (uint32_t)G * kGroupBytes + 256; off += kConvThreads * 16)
    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(sL + off), "r"(0u) : "memory");
  const int kcw = krow / 8;
  for (int i = tid; i < NP * kcw; i += kConvThreads) {
    const int n = i / kcw, q = i - n * kcw;
    cp_async16(sB + (uint32_t)(n >> 3) * sbo_b + (uint32_t)q * 128 + (uint32_t)(n & 7) * 16,
               a.w + (size_t)n * krow + (size_t)q * 8, 16);
  }
  cp_async_commit();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // base descriptors (start address sL or sB); see the MMA issue below
  const uint64_t adesc_g1 = umma_sdesc(sL, 16, 128);
  const uint64_t adesc_gn = umma_sdesc(sL, kGroupBytes, 128);
  const uint64_t bdesc0 = umma_sdesc(sB, 128, sbo_b);

  auto line_addr = [&](int cg, int dzi, int yy) -> uint32_t {
    return sL + (uint32_t)cg * kGroupBytes + (uint32_t)(dzi * 4 + (yy & 3)) * kLineBytes;
  };
  // the three z lines of row yy into ring slot yy & 3
  // this thread's line positions (pos = tid, and tid + 128 for the last halo cells): the cell
  // each copies (wrapped, or none past a wall) is the same for every line
  constexpr int kPos = (kRowPos + kConvThreads - 1) / kConvThreads;
  int p_off[kPos];
  bool p_ok[kPos];
#pragma unroll
  for (int k = 0; k < kPos; ++k) {
    const int pos = tid + k * kConvThreads;
    int x = pos - 1;
    p_ok[k] = pos < kRowPos;
    if (x < 0 || x >= W) {
      if (a.d.px) x = x < 0 ? x + W : x - W;
      else p_ok[k] = false;
    }
    p_off[k] = x * a.ldx;
  }
  auto load_row = [&](int z, int yy) {
    int yw = yy;
    bool yok = true;
    if (yw < 0 || yw >= ny) {
      if (a.d.py) yw = yw < 0 ? yw + ny : yw - ny;
      else yok = false;
    }
    for (int dzi = 0; dzi < 3; ++dzi) {
      int zz = z + dzi - 1;
      bool ok = yok;
      if (zz < 0 || zz >= nz) {
        if (a.d.pz) zz = zz < 0 ? zz + nz : zz - nz;
        else ok = false;
      }
      const bf16* row = a.x + ((size_t)zz * ny + yw) * W * a.ldx;
      for (int cg = 0; cg < G; ++cg) {
        const uint32_t dst = line_addr(cg, dzi, yy);
#pragma unroll
        for (int k = 0; k < kPos; ++k) {
          if (tid + k * kConvThreads >= kRowPos) break;
          const bool okx = ok && p_ok[k];
          cp_async16(dst + (uint32_t)(tid + k * kConvThreads) * 16,
                     okx ? (const void*)(row + p_off[k] + cg * 8) : (const void*)a.x, okx ? 16u : 0u);
        }
      }
    }
  };

  // the biases of the output channels, once (zero without biases or past cout)
  float bias_r[NP];
#pragma unroll
  for (int i = 0; i < NP; ++i) bias_r[i] = (a.bias && i < a.cout) ? __ldg(a.bias + i) : 0.0f;
  int fail = 0;
  int tcount = 0;  // tiles (rows) this CTA has issued: selects the accumulator and barrier phase
  auto epilogue = [&](int e, int z, int y) {
    const int b = e & 1;
    if (!mbar_wait(&acc_bar[b], (uint32_t)(e >> 1) & 1u)) fail = 1;
    tc_fence_after();
    // this thread's cell of the row: the accumulator row in its TMEM lane (see above)
    const int lane = tid & 31;
    const int xc = W == 128 ? tid : (lane < 16 ? warp * 16 + lane : -1);
    const int v = (z * ny + y) * W + xc;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * NP);
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float acc[16];
      tmem_ld16(taddr + (uint32_t)c0, acc);
      if (fail || xc < 0) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = c0 + 8 * h;
        if (cb >= a.cout) continue;
        float o[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float val = acc[8 * h + i] + bias_r[c0 + 8 * h + i];
          if (a.relu) val = fmaxf(val, 0.0f);
          o[i] = val;
        }
        if (a.mask) {
          const uint4 mq = *reinterpret_cast<const uint4*>(a.mask + (size_t)v * a.ldm + cb);
          const bf16* mv = reinterpret_cast<const bf16*>(&mq);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (!(__bfloat162float(mv[i]) > 0.0f)) o[i] = 0.0f;
        }
        uint4 q;
        __nv_bfloat162* qp = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) qp[i] = __floats2bfloat162_rn(o[2 * i], o[2 * i + 1]);
        *reinterpret_cast<uint4*>(a.y + (size_t)v * a.ldy + cb) = q;
      }
    }
  };

  for (int it = blockIdx.x; it < items && !fail; it += gridDim.x) {
    const int z = it / chunks_y;
    const int y0 = (it - z * chunks_y) * chunk;
    const int y1 = min(ny, y0 + chunk);
    load_row(z, y0 - 1);
    load_row(z, y0);
    load_row(z, y0 + 1);
    cp_async_commit();
    int prev_y = -1;
    for (int y = y0; y < y1; ++y) {
      cp_async_wait<0>();  // rows y - 1 .. y + 1 (and the weights) have landed
      fence_proxy_async();
      if (__syncthreads_or(fail)) break;
      if (tid == 0) {
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)((tcount & 1) * NP);
        // Descriptors differ only in their start address (bits 0-13, in 16-byte units), and
        // every shared address here is below 256 KB: each MMA's descriptor is a base
        // descriptor plus its byte offset / 16, with no carry out of the field.
        uint64_t bdesc = bdesc0;
        uint32_t kk = 0;
        if (G == 1) {
          for (int li = 0; li < 9; ++li) {
            const uint64_t a = adesc_g1 + ((line_addr(0, li / 3, y + li % 3 - 1) - sL) >> 4);
#pragma unroll
            for (int h = 0; h < 2; ++h, ++kk, bdesc += 16)
              umma_bf16(d, a + 2u * h, bdesc, idesc, kk > 0 ? 1u : 0u);
          }
        } else {
          for (int tap = 0; tap < 27; ++tap) {
            const int dzi = tap / 9, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            const uint64_t a = adesc_gn + ((line_addr(0, dzi, y + dy) - sL + (uint32_t)(1 + dx) * 16) >> 4);
            for (int cp = 0; cp < G / 2; ++cp, ++kk, bdesc += 16)
              umma_bf16(d, a + (uint64_t)((2u * cp * kGroupBytes) >> 4), bdesc, idesc, kk > 0 ? 1u : 0u);
          }
        }
        umma_commit(&acc_bar[tcount & 1]);
      }
      // row y + 2 goes into the ring slot of row y - 2, read last by the MMAs of row y - 1
      if (prev_y >= 0 && !mbar_wait(&acc_bar[(tcount - 1) & 1], (uint32_t)((tcount - 1) >> 1) & 1u)) fail = 1;
      if (y + 2 <= y1 && !fail) load_row(z, y + 2);
      cp_async_commit();
      if (prev_y >= 0) epilogue(tcount - 1, z, prev_y);
      prev_y = y;
      ++tcount;
    }
    if (prev_y >= 0) epilogue(tcount - 1, z, prev_y);
  }
  cp_async_wait_all();
  if (tid == 0) {
    umma_commit(&drain_bar);
    if (!mbar_wait(&drain_bar, 0)) fail = 1;
  }
  if (fail && a.err) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ------------------------------------------- 3x3x3 convolution on slabs of short rows (MMA)
//
// Grids whose rows are short (W = 16, 32 or 64 cells: the network's coarser levels) take an
// M = 128 tile as R = 128 / W whole rows of one z plane.  The three x offsets go into N instead of A:
// B stacks the weights of dx = -1, 0, +1 as three column blocks of PW columns, so one MMA of a
// (dz, dy) tap line and input-channel pair gives, for every cell p of the tile, in[p] W_dx for
// all three dx at once; the epilogue forms out[x] = D[x - 1][dx = -1] + D[x][0] + D[x + 1][+1]
// with warp shuffles along the row (across the two warps of a 64-cell row through shared
// memory; wrapped on a periodic x; nothing past a wall).  The A
// operand then needs no x halo: tap line (dz, dy) is R consecutive rows of the CTA's slab,
// rows y0 - 1 .. y0 + R of the three z planes, stored per 8-channel group (core matrices of 8
// cells 128 bytes apart; the pair's second group one group slab further, LBO).  A tile costs
// 9 C_in / 16 MMAs of N = 3 PW, against 27 C_in / 16 of N = PW for taps one at a time, and
// loads (R + 2) / R of its three planes' rows instead of gathering 27 copies of every cell.
// K of the stacked weights: 9 tap lines x C channels, as MMAs of two 8-channel K cores; with
// C = 8 the cores of an MMA are two z lines of one y offset (z offsets -1, 0 and +1, zero
// weights): 6 MMAs of 16
__host__ __device__ constexpr int stack_k(int C) { return C == 8 ? 96 : 9 * C; }
// dz slabs of a group: the three planes, and for 8-channel inputs a zero fourth (the partner of
// the last plane's cores)
__host__ __device__ constexpr int slab_planes(int cin) { return cin == 8 ? 4 : 3; }
__host__ __device__ constexpr uint32_t slab_group_bytes(int W) { return (uint32_t)(128 / W + 2) * W * 16; }
inline size_t slab_smem(int nt, int cin, int W) {
  return (size_t)nt * stack_k(cin) * 2 + (size_t)slab_planes(cin) * (cin / 8) * slab_group_bytes(W);
}

template <int NT, int W>
__global__ void __launch_bounds__(kConvThreads) k_conv3_slab(Conv3Args a, int pw) {
  constexpr int R = 128 / W;
  constexpr uint32_t kGS = slab_group_bytes(W);
  constexpr uint32_t kCols = tmem_cols_for(NT);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = a.cin / 8, ktot = stack_k(a.cin);
  const uint32_t sB = smem_u32(smem);
  const uint32_t sS = sB + (uint32_t)(NT * ktot * 2);
  const uint32_t sbo_b = (uint32_t)(ktot / 8) * 128;
  const int ny = a.d.ny, nz = a.d.nz;
  const int tiles_y = ny / R, n_tiles = nz * tiles_y;
  const uint32_t idesc = umma_idesc_bf16(128, NT, false, false);
  // i / G as the high word of i * ceil(2^32 / G): exact for i < 2^32 / G (the copy indices
  // here are below 2^16)
  const uint32_t g_magic = G == 1 ? 0u : (uint32_t)((0x100000000ull + (uint64_t)G - 1) / (uint64_t)G);

  if (tid == 0) {
    mbar_init(&acc_bar, 1);
    mbar_init(&drain_bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCols);
  // weights [NT][ktot] -> K-major canonical layout: core (n / 8, q) at (n / 8) sbo_b + 128 q
  const int kcw = ktot / 8;
  for (int i = tid; i < NT * kcw; i += kConvThreads) {
    const int n = i / kcw, q = i - n * kcw;
    cp_async16(sB + (uint32_t)(n >> 3) * sbo_b + (uint32_t)q * 128 + (uint32_t)(n & 7) * 16,
               a.w + (size_t)n * ktot + (size_t)q * 8, 16);
  }
  cp_async_commit();
  if (G == 1)  // the zero fourth plane (finite bytes behind zero weights)
    for (uint32_t off = (uint32_t)tid * 16; off < kGS; off += kConvThreads * 16)
      asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(sS + 3 * kGS + off), "r"(0u) : "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  // this thread's cell: row r, position x of the tile, accumulator row tid (TMEM lane tid)
  const int x = tid % W, r = tid / W;
  const bool has_l = x > 0 || a.d.px, has_r = x < W - 1 || a.d.px;
  // neighbours along the row within the warp (rows of W >= 32 cells span W / 32 warps: the
  // first and last lanes of a warp trade with the adjacent warps through shared memory)
  constexpr int WL = W < 32 ? W : 32;
  const int seg = lane & ~(WL - 1);
  const int src_l = seg | ((lane + WL - 1) & (WL - 1)), src_r = seg | ((lane + 1) & (WL - 1));
  constexpr int WPR = W / 32;  // warps per row (0 for W = 16)
  __shared__ float xl[WPR > 1 ? 4 : 1][16], xr[WPR > 1 ? 4 : 1][16];
  const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
  int fail = 0;
  uint32_t phase = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int z = t / tiles_y, y0 = (t - z * tiles_y) * R;
    // slab [dz][group][row y0 - 1 + rr][cell][8 channels]; a thread's consecutive copies read
    // consecutive 16-byte pieces of one cell
    const int total = 3 * (R + 2) * W * G;
    for (int i = tid; i < total; i += kConvThreads) {
      int rest = G == 1 ? i : (int)__umulhi((uint32_t)i, g_magic);  // i / G
      const int cg = i - rest * G;
      const int xx = rest % W;
      rest /= W;
      const int rr = rest % (R + 2), dzi = rest / (R + 2);
      int yy = y0 - 1 + rr, zz = z + dzi - 1;
      bool ok = true;
      if (yy < 0 || yy >= ny) {
        if (a.d.py) yy = yy < 0 ? yy + ny : yy - ny;
        else ok = false;
      }
      if (zz < 0 || zz >= nz) {
        if (a.d.pz) zz = zz < 0 ? zz + nz : zz - nz;
        else ok = false;
      }
      const uint32_t dst = sS + (uint32_t)(dzi * G + cg) * kGS + (uint32_t)(rr * W + xx) * 16;
      cp_async16(dst, ok ? (const void*)(a.x + ((size_t)(zz * ny + yy) * W + xx) * a.ldx + cg * 8) : (const void*)a.x,
                 ok ? 16u : 0u);
    }
    cp_async_commit();
    cp_async_wait<0>();  // the slab (and, on the first tile, the weights) has landed
    fence_proxy_async();
    if (__syncthreads_or(fail)) break;
    if (tid == 0) {
      tc_fence_after();
      uint32_t kk = 0;
      if (G == 1) {  // cores: planes (0, 1) and (2, zero) of each y offset
        for (int dyi = 0; dyi < 3; ++dyi)
          for (int pr = 0; pr < 2; ++pr, ++kk) {
            const uint64_t ad = umma_sdesc(sS + (uint32_t)(2 * pr) * kGS + (uint32_t)(dyi * W) * 16, kGS, 128);
            umma_bf16(tmem, ad, umma_sdesc(sB + kk * 256, 128, sbo_b), idesc, kk > 0 ? 1u : 0u);
          }
      } else {
        for (int li = 0; li < 9; ++li) {
          const int dzi = li / 3, dyi = li % 3;
          for (int pr = 0; pr < G / 2; ++pr, ++kk) {
            const uint64_t ad = umma_sdesc(sS + (uint32_t)(dzi * G + 2 * pr) * kGS + (uint32_t)(dyi * W) * 16, kGS, 128);
            umma_bf16(tmem, ad, umma_sdesc(sB + kk * 256, 128, sbo_b), idesc, kk > 0 ? 1u : 0u);
          }
        }
      }
      umma_commit(&acc_bar);
    }
    if (!mbar_wait(&acc_bar, phase)) fail = 1;
    phase ^= 1u;
    tc_fence_after();
    const int v = (z * ny + y0 + r) * W + x;
    for (int c0 = 0; c0 < pw; c0 += 16) {
      float pm[16], pc[16], pp[16];
      tmem_ld16(taddr + (uint32_t)c0, pm);             // dx = -1 block (whole warp)
      tmem_ld16(taddr + (uint32_t)(pw + c0), pc);      // dx = 0
      tmem_ld16(taddr + (uint32_t)(2 * pw + c0), pp);  // dx = +1
      float lv[16], rv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        lv[i] = __shfl_sync(0xffffffffu, pm[i], src_l);
        rv[i] = __shfl_sync(0xffffffffu, pp[i], src_r);
      }
      if constexpr (WPR > 1) {
        const int wr = warp % WPR, w0 = warp - wr;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (lane == 31) xl[warp][i] = pm[i];
          if (lane == 0) xr[warp][i] = pp[i];
        }
        __syncthreads();
        const int wl = w0 + (wr + WPR - 1) % WPR, wn = w0 + (wr + 1) % WPR;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (lane == 0) lv[i] = xl[wl][i];
          if (lane == 31) rv[i] = xr[wn][i];
        }
        __syncthreads();  // xl, xr are rewritten by the next column chunk
      }
      float o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) o[i] = pc[i] + (has_l ? lv[i] : 0.0f) + (has_r ? rv[i] : 0.0f);
      if (fail) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = c0 + 8 * h;
        if (cb >= a.cout) continue;
        float q8[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float val = o[8 * h + i];
          if (a.bias) val += __ldg(a.bias + cb + i);
          if (a.relu) val = fmaxf(val, 0.0f);
          q8[i] = val;
        }
        if (a.mask) {
          const uint4 mq = *reinterpret_cast<const uint4*>(a.mask + (size_t)v * a.ldm + cb);
          const bf16* mv = reinterpret_cast<const bf16*>(&mq);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (!(__bfloat162float(mv[i]) > 0.0f)) q8[i] = 0.0f;
        }
        uint4 q;
        __nv_bfloat162* qp = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
        for (int i = 0; i < 4; ++i) qp[i] = __floats2bfloat162_rn(q8[2 * i], q8[2 * i + 1]);
        *reinterpret_cast<uint4*>(a.y + (size_t)v * a.ldy + cb) = q;
      }
    }
    tc_fence_before();  // this tile's TMEM reads precede the next tile's MMAs (next barrier)
  }
  cp_async_wait_all();
  // every MMA this CTA issued has completed before TMEM is released (also after a wait gave up)
  if (tid == 0) {
    umma_commit(&drain_bar);
    if (!mbar_wait(&drain_bar, 0)) fail = 1;
  }
  if (fail && a.err) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ------------------------------------------------------- weight gradient of a 3x3x3 conv (MMA)
//
// D[m][n] = sum over cells v of A[m][v] B[n][v] with m = tap * c_in + ci (plus one row
// m = 27 c_in of ones, which yields the bias gradient) and n the output channel:
// A[m][v] = x[neighbour(v, tap)][ci], B[n][v] = g[v][n] (g the ReLU-masked output gradient).
// Both operands are MN-major in shared memory (8 consecutive channels of one cell form a
// 16-byte row), K = cells.  CTA (m tile, split) accumulates its share of the cells in TMEM and
// writes an FP32 partial [split][mpad][NP]; a second kernel sums the splits in a fixed order.

constexpr int kWS = 32;                          // cells per stage
constexpr uint32_t kLboWA = 16 * 128;            // A: core matrices adjacent along K (cells)
constexpr int kWAStage = 128 * kWS * 2;          // 8 KB

struct WgradArgs {
  const bf16* x = nullptr;
  int ldx = 0, cin = 0;  // convolution input (channels, multiple of 8)
  const bf16* g = nullptr;
  int ldg = 0, cout = 0;  // masked output gradient
  Dims d;
  int n_vox = 0;
  int rows = 0;  // 27 cin: index of the ones row
  int mpad = 0;
  int cells_per_split = 0;  // multiple of kWS
  float* part = nullptr;
  int np = 0;      // columns of a partial row (output channels padded)
  int go_cta = 0;  // output groups of 8 channels per CTA (line-buffer kernel)
  int* err = nullptr;
};

template <int NP>
__global__ void __launch_bounds__(kConvThreads) k_wgrad_mma(WgradArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t slot_bar[kStages];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_slot;
  constexpr uint32_t kCols = tmem_cols_for(NP);
  constexpr uint32_t kLboWB = (NP / 8) * 128;
  constexpr int kWBStage = NP * kWS * 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sA = smem_u32(smem);
  const uint32_t sB = sA + (uint32_t)kStages * kWAStage;
  const int mt = blockIdx.x, split = blockIdx.y;
  const int v0 = split * a.cells_per_split;
  const int v1 = min(a.n_vox, v0 + a.cells_per_split);
  const int T = v1 > v0 ? (v1 - v0 + kWS - 1) / kWS : 0;
  const uint32_t idesc = umma_idesc_bf16(128, NP, true, true);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) mbar_init(&slot_bar[i], 1);
    mbar_init(&done_bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, kCols);

  // this thread's A row groups (grp = tid / 32 + 4 r): gather (tap offsets, ci0), the ones
  // row, or zeros; fixed for the CTA's m tile, so decoded once
  constexpr int kAG = (kWS * 16) / kConvThreads;  // A groups per thread per stage (4)
  int gcode[kAG];
#pragma unroll
  for (int r = 0; r < kAG; ++r) {
    const int m = mt * 128 + (tid / kWS + r * (kConvThreads / kWS)) * 8;
    if (m < a.rows) {
      const int tap = m / a.cin;
      gcode[r] = (tap % 3) | ((tap / 3) % 3) << 2 | (tap / 9) << 4 | (m - tap * a.cin) << 8;
    } else {
      gcode[r] = m == a.rows ? -1 : -2;  // -1: the ones row, -2: zeros
    }
  }
  const int kcell = tid % kWS;  // the cell column of every copy this thread makes

  auto load_stage = [&](int j) {
    const int slot = j % kStages;
    const uint32_t a_base = sA + (uint32_t)slot * kWAStage;
    const uint32_t b_base = sB + (uint32_t)slot * kWBStage;
    const int v = v0 + j * kWS + kcell;
    const bool valid = v < v1;
    int x = 0, y = 0, z = 0;
    if (valid) {
      const int r = v / a.d.nx;
      x = v - r * a.d.nx;
      z = r / a.d.ny;
      y = r - z * a.d.ny;
    }
    // A: 32 cells x 16 groups of 8 rows
#pragma unroll
    for (int r = 0; r < kAG; ++r) {
      const int grp = tid / kWS + r * (kConvThreads / kWS);
      const uint32_t dst = a_base + (uint32_t)(kcell >> 3) * kLboWA + (uint32_t)grp * 128 + (uint32_t)(kcell & 7) * 16;
      const int e = gcode[r];
      if (e < 0) {
        uint4 q = make_uint4(0, 0, 0, 0);
        if (e == -1 && valid) q.x = 0x3F80u;  // BF16 1.0 in the low half: the bias row
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(q.x), "r"(q.y), "r"(q.z), "r"(q.w)
                     : "memory");
        continue;
      }
      const bf16* src = a.x;
      uint32_t bytes = 0;
      if (valid) {
        const int nb = neighbour(a.d, x, y, z, (e & 3) - 1, ((e >> 2) & 3) - 1, ((e >> 4) & 3) - 1);
        if (nb >= 0) {
          src = a.x + (size_t)nb * a.ldx + (e >> 8);
          bytes = 16;
        }
      }
      cp_async16(dst, src, bytes);
    }
    // B: 32 cells x NP / 8 groups
#pragma unroll
    for (int r = 0; r < (kWS * (NP / 8) + kConvThreads - 1) / kConvThreads; ++r) {
      const int grp = tid / kWS + r * (kConvThreads / kWS);
      if (grp >= NP / 8) break;
      const uint32_t dst = b_base + (uint32_t)(kcell >> 3) * kLboWB + (uint32_t)grp * 128 + (uint32_t)(kcell & 7) * 16;
      const bool ok = valid && grp * 8 < a.cout;
      cp_async16(dst, ok ? (const void*)(a.g + (size_t)v * a.ldg + grp * 8) : (const void*)a.g, ok ? 16u : 0u);
    }
  };

  for (int j = 0; j < kAhead; ++j) {
    if (j < T) load_stage(j);
    cp_async_commit();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int fail = 0;
  for (int j = 0; j < T; ++j) {
    cp_async_wait<kAhead - 1>();
    fence_proxy_async();
    if (__syncthreads_or(fail)) break;
    if (tid == 0) {
      tc_fence_after();
      const int slot = j % kStages;
#pragma unroll
      for (int ks = 0; ks < kWS / 16; ++ks) {
        const uint64_t ad = umma_sdesc(sA + (uint32_t)slot * kWAStage + (uint32_t)ks * 2 * kLboWA, kLboWA, 128);
        const uint64_t bd = umma_sdesc(sB + (uint32_t)slot * kWBStage + (uint32_t)ks * 2 * kLboWB, kLboWB, 128);
        umma_bf16(tmem, ad, bd, idesc, (j > 0 || ks > 0) ? 1u : 0u);
      }
      umma_commit(&slot_bar[slot]);
    }
    const int jn = j + kAhead;
    if (jn < T) {
      const int jo = jn - kStages;
      if (jo >= 0 && !mbar_wait(&slot_bar[jo % kStages], (uint32_t)(jo / kStages) & 1u)) fail = 1;
      if (!fail) load_stage(jn);
    }
    cp_async_commit();
  }
  cp_async_wait_all();
  if (tid == 0) {
    umma_commit(&done_bar);
    if (!mbar_wait(&done_bar, 0)) fail = 1;
  }
  fail = __syncthreads_or(fail);
  tc_fence_after();
  // epilogue: lane = row m of the tile, NP FP32 columns -> partial (zeros when T == 0)
  const int m = warp * 32 + lane;
  float* dst = a.part + ((size_t)split * a.mpad + (size_t)mt * 128 + m) * NP;
#pragma unroll
  for (int c0 = 0; c0 < NP; c0 += 16) {
    float acc[16];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, acc);
#pragma unroll
    for (int i = 0; i < 16; i += 4) {
      float4 q = (T > 0 && !fail) ? make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]) : make_float4(0, 0, 0, 0);
      *reinterpret_cast<float4*>(dst + c0 + i) = q;
    }
  }
  if (fail && a.err) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// Weight gradient on rows of W cells (a multiple of 16) with no operand tile built per row:
// D[(j, ci)][(j', co)] = sum over the row's cells x of line_j[x][ci] g[x + j' - 1][co], K = the
// cells.  A (MN-major) is the nine input lines (dy, dz) around the row, line j = 3 (dy + 1) +
// (dz + 1) as M core j (8 channels of one line per core, cores one line apart: M = 128 holds the
// nine and seven don't-care cores); B (MN-major) is the row's output gradient with its x halo,
// the N cores 16 bytes apart, so that core j' reads g shifted by j' - 1 cells: dx = 1 - j'
// (N = 32: the fourth core is don't-care).  So tap (dz, dy, dx) and channel pair come out
// of one MMA per 16 cells for all 27 taps of an 8-channel group pair, the operands read where
// the copies put them.  A CTA takes runs of `chunk` rows of one z plane; a run's lines are
// stored in order [y line][dz] per 8-channel group (no slot reuse within a run), so the nine
// lines of every row are consecutive.  The bias gradient (sum of g) is summed per thread.
// Accumulators: one 32-column block per (input group, output group), in TMEM for the CTA's
// runs (at most two output groups per CTA: more are spread over the grid's y dimension); the
// partial [split][m = tap c_in + ci (+ the bias row 27 c_in)][n = co] goes to k_wgrad_reduce.
__host__ __device__ constexpr int wlin_halo(int W) { return W + 4; }  // g line: cells -1 .. W + 2
inline size_t wgrad_lin_smem(int W, int G, int Go, int chunk) {
  return ((size_t)G * (chunk + 2) * 3 + 7) * W * 16 + 3 * (size_t)Go * wlin_halo(W) * 16;
}

template <int W>
__global__ void __launch_bounds__(kConvThreads) k_wgrad_lin(WgradArgs a, int chunk, int runs_per_split) {
  constexpr uint32_t kLB = W * 16;                   // one line: W cells x 8 channels
  constexpr uint32_t kGH = wlin_halo(W) * 16;        // one g line with its halo
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mma_bar[2];  // rows alternate between the two
  __shared__ uint32_t tmem_slot;
  __shared__ float bred[4][16];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // this CTA's output groups: cgo0 .. cgo0 + Go - 1 of the layer's (grid dimension y)
  const int G = a.cin / 8, cgo0 = blockIdx.y * a.go_cta, Go = min(a.go_cta, (a.cout + 7) / 8 - cgo0);
  const uint32_t cols = tmem_cols_for(32 * G * a.go_cta);
  const int nlines = G * (chunk + 2) * 3 + 7;
  const uint32_t sL = smem_u32(smem);
  const uint32_t sG = sL + (uint32_t)nlines * kLB;  // three g buffers of Go lines each
  const int ny = a.d.ny, nz = a.d.nz;
  const int runs_y = (ny + chunk - 1) / chunk, items = nz * runs_y;
  const int it0 = blockIdx.x * runs_per_split, it1 = min(items, it0 + runs_per_split);
  const uint32_t idesc = umma_idesc_bf16(128, 32, true, true);

  if (tid == 0) {
    mbar_init(&mma_bar[0], 1);
    mbar_init(&mma_bar[1], 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, cols);
  // every byte the MMAs may read starts finite: the don't-care cores read lines past a
  // run's window and the g halo past the row
  const uint32_t total_bytes = (uint32_t)nlines * kLB + 3u * a.go_cta * kGH;
  for (uint32_t off = (uint32_t)tid * 16; off < total_bytes; off += kConvThreads * 16)
    asm volatile("st.shared.v4.b32 [%0], {%1, %1, %1, %1};" ::"r"(sL + off), "r"(0u) : "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // this thread's copies of a row's lines: copy k is piece i = tid + 128 k of (dzi, x, cg), the
  // same for every row, so its offsets are worked out once (up to kWT copies a thread)
  constexpr int kWT = 6;
  const int per = W * G;
  const bool tabled = 3 * per <= kWT * kConvThreads;
  uint32_t t_dst[kWT], t_src[kWT];
  int t_dz[kWT];
#pragma unroll
  for (int k = 0; k < kWT; ++k) {
    const int i = tid + k * kConvThreads;
    const int dzi = i / per, rem = i - dzi * per;
    const int x = rem / G, cg = rem - x * G;
    t_dz[k] = i < 3 * per ? dzi : -1;
    t_dst[k] = (uint32_t)((cg * (chunk + 2)) * 3 + dzi) * kLB + (uint32_t)x * 16;
    t_src[k] = (uint32_t)(x * a.ldx + cg * 8);
  }
  // line (cg, yl, dzi) of the current run: input row y0 - 1 + yl of plane z + dzi - 1
  auto load_lines = [&](int z, int y0, int yl) {
    int yy = y0 - 1 + yl;
    bool yok = true;
    if (yy < 0 || yy >= ny) {
      if (a.d.py) yy = yy < 0 ? yy + ny : yy - ny;
      else yok = false;
    }
    if (tabled) {
      // the row's start in each of the three planes (or none past a wall)
      const bf16* pb[3];
      bool pok[3];
#pragma unroll
      for (int dzi = 0; dzi < 3; ++dzi) {
        int zz = z + dzi - 1;
        pok[dzi] = yok;
        if (zz < 0 || zz >= nz) {
          if (a.d.pz) zz = zz < 0 ? zz + nz : zz - nz;
          else pok[dzi] = false;
        }
        pb[dzi] = a.x + (size_t)(zz * ny + yy) * W * a.ldx;
      }
      const uint32_t yoff = sL + (uint32_t)(yl * 3) * kLB;
#pragma unroll
      for (int k = 0; k < kWT; ++k) {
        if (t_dz[k] < 0) break;
        const int dz = t_dz[k];
        const bool ok = dz == 0 ? pok[0] : (dz == 1 ? pok[1] : pok[2]);
        const bf16* b = dz == 0 ? pb[0] : (dz == 1 ? pb[1] : pb[2]);
        cp_async16(yoff + t_dst[k], ok ? (const void*)(b + t_src[k]) : (const void*)a.x, ok ? 16u : 0u);
      }
      return;
    }
    for (int i = tid; i < 3 * per; i += kConvThreads) {
      const int dzi = i / per, rem = i - dzi * per;
      const int x = rem / G, cg = rem - x * G;
      int zz = z + dzi - 1;
      bool ok = yok;
      if (zz < 0 || zz >= nz) {
        if (a.d.pz) zz = zz < 0 ? zz + nz : zz - nz;
        else ok = false;
      }
      const uint32_t dst = sL + (uint32_t)((cg * (chunk + 2) + yl) * 3 + dzi) * kLB + (uint32_t)x * 16;
      cp_async16(dst, ok ? (const void*)(a.x + ((size_t)(zz * ny + yy) * W + x) * a.ldx + cg * 8) : (const void*)a.x,
                 ok ? 16u : 0u);
    }
  };
  // the output gradient of row (z, y) with its halo into g buffer `buf`: cell h - 1 at h
  auto load_g = [&](int z, int y, int buf) {
    const int nh = W + 2;  // cells -1 .. W (the two spare cells stay zero)
    for (int i = tid; i < nh * Go; i += kConvThreads) {
      const int h = i / Go, cgo = i - h * Go;
      int x = h - 1;
      bool ok = (cgo0 + cgo) * 8 < a.cout;
      if (x < 0 || x >= W) {
        if (a.d.px) x = x < 0 ? x + W : x - W;
        else ok = false;
      }
      const uint32_t dst = sG + (uint32_t)(buf * Go + cgo) * kGH + (uint32_t)h * 16;
      cp_async16(dst, ok ? (const void*)(a.g + ((size_t)(z * ny + y) * W + x) * a.ldg + (cgo0 + cgo) * 8) : (const void*)a.g,
                 ok ? 16u : 0u);
    }
  };

  float bsum[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) bsum[i] = 0.0f;
  int fail = 0;
  int rows_done = 0;  // rows whose MMAs were issued
  // row r's MMAs commit to mma_bar[r & 1], as that barrier's phase r / 2
  auto wait_row = [&](int r) {
    if (r >= 0 && !mbar_wait(&mma_bar[r & 1], (uint32_t)(r >> 1) & 1u)) fail = 1;
  };
  for (int it = it0; it < it1; ++it) {
    const int z = it / runs_y, y0 = (it - z * runs_y) * chunk, y1 = min(ny, y0 + chunk);
    // the previous run's MMAs read the line buffer: all done before it is overwritten
    wait_row(rows_done - 2);
    wait_row(rows_done - 1);
    if (!fail) {
      for (int yl = 0; yl < 3; ++yl) load_lines(z, y0, yl);
      load_g(z, y0, rows_done % 3);
    }
    cp_async_commit();
    for (int y = y0; y < y1; ++y) {
      // row y + 1's output gradient goes into the buffer row y - 2's MMAs read (row y - 1's
      // may still run)
      if (y > y0) wait_row(rows_done - 2);
      if (!fail) {
        if (y + 2 <= y1) load_lines(z, y0, y - y0 + 3);
        if (y + 1 < y1) load_g(z, y + 1, (rows_done + 1) % 3);
      }
      cp_async_commit();
      cp_async_wait<1>();  // row y's lines and output gradient have landed
      fence_proxy_async();
      if (__syncthreads_or(fail)) break;
      const uint32_t gb = sG + (uint32_t)((rows_done % 3) * Go) * kGH;
      if (tid < W) {
#pragma unroll
        for (int cgo = 0; cgo < 2; ++cgo) {
          if (cgo >= Go) break;
          uint32_t q[4];
          asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3])
                       : "r"(gb + (uint32_t)cgo * kGH + (uint32_t)(tid + 1) * 16));
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q[i]));
            bsum[cgo * 8 + 2 * i] += f.x;
            bsum[cgo * 8 + 2 * i + 1] += f.y;
          }
        }
      }
      if (tid == 0) {
        tc_fence_after();
        const int yl = y - y0;
#pragma unroll 1
        for (int ks = 0; ks < W / 16; ++ks)
          for (int cg = 0; cg < G; ++cg) {
            const uint64_t ad =
                umma_sdesc(sL + (uint32_t)((cg * (chunk + 2) + yl) * 3) * kLB + (uint32_t)ks * 256, 128, kLB);
            for (int cgo = 0; cgo < Go; ++cgo) {
              const uint64_t bd = umma_sdesc(gb + (uint32_t)cgo * kGH + (uint32_t)ks * 256, 128, 16);
              umma_bf16(tmem + (uint32_t)((cg * Go + cgo) * 32), ad, bd, idesc,
                        (rows_done > 0 || ks > 0) ? 1u : 0u);
            }
          }
        umma_commit(&mma_bar[rows_done & 1]);
      }
      ++rows_done;
    }
  }
  cp_async_wait_all();
  wait_row(rows_done - 2);
  wait_row(rows_done - 1);
  fail = __syncthreads_or(fail);
  tc_fence_after();
  // partials: lane m = j * 8 + ci of accumulator (cg, cgo), columns j' * 8 + co
  const int m = warp * 32 + lane, j = m >> 3, ci = m & 7;
  const int dyi = j / 3, dzi = j - 3 * dyi;
  float* part = a.part + (size_t)blockIdx.x * a.mpad * a.np + cgo0 * 8;
  for (int cg = 0; cg < G; ++cg)
    for (int cgo = 0; cgo < Go; ++cgo) {
      float a0[16], a1[16];  // columns j' = 0, 1 and j' = 2, 3
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((cg * Go + cgo) * 32);
      tmem_ld16(ta, a0);
      tmem_ld16(ta + 16u, a1);
      if (j >= 9) continue;
      const float z0 = rows_done > 0 && !fail ? 1.0f : 0.0f;  // zeros from a CTA without rows
      float* dst = part + (size_t)(dzi * 9 + dyi * 3) * a.cin * a.np + (size_t)(cg * 8 + ci) * a.np + cgo * 8;
      const size_t tap_stride = (size_t)a.cin * a.np;  // dx = 1 - j': tap offsets 2, 1, 0
#pragma unroll
      for (int i = 0; i < 8; i += 4) {
        *reinterpret_cast<float4*>(dst + 2 * tap_stride + i) =
            make_float4(z0 * a0[i], z0 * a0[i + 1], z0 * a0[i + 2], z0 * a0[i + 3]);
        *reinterpret_cast<float4*>(dst + tap_stride + i) =
            make_float4(z0 * a0[8 + i], z0 * a0[9 + i], z0 * a0[10 + i], z0 * a0[11 + i]);
        *reinterpret_cast<float4*>(dst + i) = make_float4(z0 * a1[i], z0 * a1[i + 1], z0 * a1[i + 2], z0 * a1[i + 3]);
      }
    }
  // the bias row: per channel, warps' sums in order
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    float v = bsum[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) bred[warp][i] = v;
  }
  __syncthreads();
  if (tid < 8 * Go && tid < 16) {
    const float v = ((bred[0][tid] + bred[1][tid]) + bred[2][tid]) + bred[3][tid];
    part[(size_t)(27 * a.cin) * a.np + tid] = (rows_done > 0 && !fail) ? v : 0.0f;
  }
  if (fail && a.err) atomicExch(a.err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, cols);
}

// Sums over the splits of a [splits][stride] FP32 partial for the block's 32 consecutive
// columns (lane = column f; ok: f is a real column): warp w adds splits w, w + warps, ... in
// order, then warp 0 adds the warps' sums in warp order: a fixed order, so the result does not
// depend on scheduling.  Each warp reads 128 contiguous bytes per split.  Valid in warp 0.
__device__ __forceinline__ float split_column_sum(const float* __restrict__ part, int splits, size_t stride, int f,
                                                  bool ok, float (*sh)[32]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float s = 0.0f;
  if (ok) {
    const float* p = part + f;
#pragma unroll 4
    for (int sp = warp; sp < splits; sp += nw) s += __ldcs(p + (size_t)sp * stride);
  }
  sh[warp][lane] = s;
  __syncthreads();
  float t = 0.0f;
  if (warp == 0) {
    t = sh[0][lane];
    for (int w = 1; w < nw; ++w) t += sh[w][lane];
  }
  __syncthreads();
  return t;
}

// Sums the splits of a weight-gradient partial [split][m < mpad][n < np] and adds it into the
// parameter gradient in the [c_out][tap][c_in] layout (+ biases, row m = 27 cin_pad).
// cin_pad: channels of the GEMM input (>= cin).
__global__ void k_wgrad_reduce(const float* __restrict__ part, int splits, int mpad, int np, int cin_pad, int cin,
                               int cout, float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ float sh[32][32];
  const int rows = 27 * cin_pad;
  const int total = (rows + 1) * np;
  for (int f0 = blockIdx.x * 32; f0 < total; f0 += gridDim.x * 32) {
    const int f = f0 + (threadIdx.x & 31);
    const float v = split_column_sum(part, splits, (size_t)mpad * np, f, f < total, sh);
    if (threadIdx.x >= 32 || f >= total) continue;
    const int m = f / np, n = f - m * np;
    if (n >= cout) continue;
    if (m == rows) {
      gb[n] += v;
    } else {
      const int tap = m / cin_pad, ci = m - tap * cin_pad;
      if (ci < cin) gw[((size_t)n * 27 + tap) * cin + ci] += v;
    }
  }
}

// threads per block of the split reductions: a warp per 4 splits or more, at most 32 warps
inline int split_sum_threads(int splits) { return 32 * std::min(32, std::max(1, splits / 4)); }
inline int split_sum_blocks(int64_t columns) { return (int)std::max<int64_t>(1, std::min<int64_t>(8192, (columns + 31) / 32)); }

// ------------------------------------------------------------------------ streaming kernels

constexpr int kRedThreads = 256;
constexpr int kRedGrid = 608;

template <int NQ>
__device__ void block_sum_store(double (&v)[NQ], double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32][NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    for (int o = 16; o >= 1; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[w][q] = v[q];
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int i = 0; i < kRedThreads / 32; ++i) s += sh[i][threadIdx.x];
    part[(size_t)blockIdx.x * NQ + threadIdx.x] = s;
  }
}

// out[q] = scale * sum over blocks; one block of 256 threads per quantity q (grid nq), each
// thread a fixed strided subset, then a fixed-shape tree: the same order on every run.
__global__ void __launch_bounds__(256) k_finish(const double* __restrict__ part, int nblk, int nq,
                                                double* __restrict__ out, double scale) {
  __shared__ double sh[256];
  const int q = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 256) s += part[(size_t)b * nq + q];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[q] = scale * sh[0];
}

// sums of b^2 and p1^2 (for the scales s_b, s_p)
__global__ void k_sumsq2(const double* __restrict__ b, const double* __restrict__ p1, int n, double* part) {
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double bb = b[i], pp = p1[i];
    v[0] += bb * bb;
    v[1] += pp * pp;
  }
  block_sum_store<2>(v, part);
}

// s[0] = mean b^2, s[1] = mean p1^2 -> scales; x0[v] = (b / s_b, p1 / s_p, p2 / s_p, 0 ...) in BF16, ld 8
__global__ void k_make_input(const double* __restrict__ b, const double* __restrict__ p1, const double* __restrict__ p2,
                             int n, const double* __restrict__ ms, double* __restrict__ scal, bf16* __restrict__ x0) {
  const double sb = ms[0] > 0.0 ? sqrt(ms[0]) : 1.0;
  const double sp = ms[1] > 0.0 ? sqrt(ms[1]) : 1.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    scal[0] = sb;
    scal[1] = sp;
  }
  const double ib = 1.0 / sb, ip = 1.0 / sp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
    h[0] = __floats2bfloat162_rn((float)(b[i] * ib), (float)(p1[i] * ip));
    h[1] = __floats2bfloat162_rn((float)(p2[i] * ip), 0.0f);
    h[2] = __floats2bfloat162_rn(0.0f, 0.0f);
    h[3] = h[2];
    *reinterpret_cast<uint4*>(x0 + (size_t)i * 8) = q;
  }
}

// 2x2x2 average pooling: out[coarse][c] = mean of the 8 fine cells; thread per (coarse, 8 channels)
__global__ void k_pool(const bf16* __restrict__ in, int ldi, Dims fine, int c, bf16* __restrict__ out, int ldo) {
  const int cx = fine.nx / 2, cy = fine.ny / 2, cz = fine.nz / 2;
  const int groups = c / 8;
  const int total = cx * cy * cz * groups;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int gq = i % groups, v = i / groups;
    const int x = v % cx, r = v / cx, y = r % cy, z = r / cy;
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const int fv = (2 * x + (o & 1)) + fine.nx * ((2 * y + ((o >> 1) & 1)) + fine.ny * (2 * z + (o >> 2)));
      const uint4 q = *reinterpret_cast<const uint4*>(in + (size_t)fv * ldi + gq * 8);
      const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
      for (int e = 0; e < 8; ++e) s[e] += __bfloat162float(h[e]);
    }
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(s[2 * e] * 0.125f, s[2 * e + 1] * 0.125f);
    *reinterpret_cast<uint4*>(out + (size_t)v * ldo + gq * 8) = q;
  }
}

// the block's copy of a transposed convolution's weights (count a multiple of 8 BF16 values,
// W from cudaMalloc): 16-byte pieces, then a barrier
__device__ __forceinline__ void stage_weights(const bf16* __restrict__ W, int count, bf16* sw) {
  const uint4* src = reinterpret_cast<const uint4*>(W);
  uint4* dst = reinterpret_cast<uint4*>(sw);
  for (int i = threadIdx.x; i < count / 8; i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
}

// fine cell index of coarse cell (x, y, z) and offset o = a * 4 + b * 2 + c (z, y, x offsets)
__device__ __forceinline__ int fine_of(const Dims& fine, int x, int y, int z, int o) {
  return (2 * x + (o & 1)) + fine.nx * ((2 * y + ((o >> 1) & 1)) + fine.ny * (2 * z + (o >> 2)));
}

// 2x2x2 stride-2 transposed convolution, W [cout][8][cin] BF16 in shared memory; thread per
// (fine cell, 8 output channels); writes channels [0, cout) of the decoder input (ld ldo)
__global__ void k_up(const bf16* __restrict__ in, int ldi, int cin, const bf16* __restrict__ W,
                     const float* __restrict__ bias, Dims fine, int cout, bf16* __restrict__ out, int ldo) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  bf16* sw = reinterpret_cast<bf16*>(sm_raw);
  stage_weights(W, cout * 8 * cin, sw);
  const int groups = cout / 8;
  const int total = fine.n() * groups;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int gq = i % groups, fv = i / groups;
    const int x = fv % fine.nx, r = fv / fine.nx, y = r % fine.ny, z = r / fine.ny;
    const int o = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
    const int cv = (x >> 1) + (fine.nx >> 1) * ((y >> 1) + (fine.ny >> 1) * (z >> 1));
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = bias[gq * 8 + e];
    const bf16* xin = in + (size_t)cv * ldi;
    for (int ci = 0; ci < cin; ci += 8) {
      const uint4 q = *reinterpret_cast<const uint4*>(xin + ci);
      const bf16* h = reinterpret_cast<const bf16*>(&q);
      float xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = __bfloat162float(h[u]);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        // the 8 weights W[gq 8 + e][o][ci .. ci + 7]: one 16-byte shared-memory load
        const uint4 wq = *reinterpret_cast<const uint4*>(sw + ((gq * 8 + e) * 8 + o) * cin + ci);
        const bf16* wh = reinterpret_cast<const bf16*>(&wq);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[e] += __bfloat162float(wh[u]) * xv[u];
      }
    }
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int e = 0; e < 4; ++e) h[e] = __floats2bfloat162_rn(acc[2 * e], acc[2 * e + 1]);
    *reinterpret_cast<uint4*>(out + (size_t)fv * ldo + gq * 8) = q;
  }
}

// input gradient of the transposed convolution, masked by the ReLU of its input:
// g_in[v][ci] = bf16(sum_{o, co} gu[fine(v, o)][co] W[co][o][ci]) * (x[v][ci] > 0)
__global__ void k_up_dx(const bf16* __restrict__ gu, int ldg, int cout, const bf16* __restrict__ W, int cin,
                        const bf16* __restrict__ xin, int ldx, Dims fine, bf16* __restrict__ gin, int ldgi) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  bf16* sw = reinterpret_cast<bf16*>(sm_raw);
  stage_weights(W, cout * 8 * cin, sw);
  const int cx = fine.nx / 2, cy = fine.ny / 2, cz = fine.nz / 2;
  const int groups = cin / 8;
  const int total = cx * cy * cz * groups;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int gq = i % groups, v = i / groups;
    const int x = v % cx, r = v / cx, y = r % cy, z = r / cy;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int o = 0; o < 8; ++o) {
      const bf16* g = gu + (size_t)fine_of(fine, x, y, z, o) * ldg;
      for (int co = 0; co < cout; co += 8) {
        const uint4 q = *reinterpret_cast<const uint4*>(g + co);
        const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float gv = __bfloat162float(h[u]);
          // W[co + u][o][gq 8 .. gq 8 + 7]: one 16-byte shared-memory load
          const uint4 wq = *reinterpret_cast<const uint4*>(sw + ((co + u) * 8 + o) * cin + gq * 8);
          const bf16* wr = reinterpret_cast<const bf16*>(&wq);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] += __bfloat162float(wr[e]) * gv;
        }
      }
    }
    const uint4 mq = *reinterpret_cast<const uint4*>(xin + (size_t)v * ldx + gq * 8);
    const bf16* mh = reinterpret_cast<const bf16*>(&mq);
    uint4 q;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&q);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // round first (the stored gradient), then mask: the same as masking the rounded value
      __nv_bfloat162 rv = __floats2bfloat162_rn(acc[2 * e], acc[2 * e + 1]);
      if (!(__bfloat162float(mh[2 * e]) > 0.0f)) rv.x = __float2bfloat16(0.0f);
      if (!(__bfloat162float(mh[2 * e + 1]) > 0.0f)) rv.y = __float2bfloat16(0.0f);
      h[e] = rv;
    }
    *reinterpret_cast<uint4*>(gin + (size_t)v * ldgi + gq * 8) = q;
  }
}

// weight and bias gradient of the transposed convolution, dW[co][o][ci] = sum over coarse cells v
// of g[fine(v, o)][co] x[v][ci] and db[co] = sum over fine cells of g[.][co]: an outer-product
// sum per child o.  Tiles of 8 co x 8 ci for one o (tile index o fastest, then the co group,
// then the ci group), tb tiles per block (blockIdx.y: the tile group), each tile held in
// registers by ln lanes (ln a power of two, the lanes of a tile adjacent in a warp) that stride
// over the block's range of cells_per_split coarse cells (blockIdx.x).  The lanes then add up
// by a fixed xor tree, and the block writes its share of part[blockIdx.x][8 cin cout + cout]
// (W in [co][o][ci] order, then the biases, which the tiles of the first ci group sum over o).
constexpr int kUpDwThreads = 256;
__global__ void __launch_bounds__(kUpDwThreads, 2)
    k_up_dw(const bf16* __restrict__ x, int ldx, int cin, const bf16* __restrict__ gu, int ldg, int cout, Dims fine,
            int tb, int ln, int cells_per_split, float* __restrict__ part) {
  __shared__ float sb[64][8];  // tb <= 64: each tile's bias sums
  const int tile = threadIdx.x / ln, j = threadIdx.x & (ln - 1);
  const int gco = cout / 8;
  const int n_tiles = gco * cin;  // 8 (cout / 8) (cin / 8)
  const int tg = blockIdx.y * tb + tile;
  const bool valid = tile < tb && tg < n_tiles;
  const int o = tg & 7, rest = tg >> 3, cog = rest % gco, cig = rest / gco;
  const bool with_bias = valid && cig == 0;
  const int cx = fine.nx / 2, cy = fine.ny / 2;
  const int nc = cx * cy * (fine.nz / 2);
  const int c0 = blockIdx.x * cells_per_split, c1 = min(nc, c0 + cells_per_split);
  float acc[8][8], bs[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    bs[r] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.0f;
  }
  if (valid) {
#pragma unroll 2
    for (int v = c0 + j; v < c1; v += ln) {
      const int xx = v % cx, rr = v / cx;
      const uint4 xq = __ldg(reinterpret_cast<const uint4*>(x + (size_t)v * ldx + cig * 8));
      const uint4 gq =
          __ldg(reinterpret_cast<const uint4*>(gu + (size_t)fine_of(fine, xx, rr % cy, rr / cy, o) * ldg + cog * 8));
      const __nv_bfloat162* xh = reinterpret_cast<const __nv_bfloat162*>(&xq);
      const __nv_bfloat162* gh = reinterpret_cast<const __nv_bfloat162*>(&gq);
      float xv[8], gv[8];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 fx = __bfloat1622float2(xh[e]), fg = __bfloat1622float2(gh[e]);
        xv[2 * e] = fx.x, xv[2 * e + 1] = fx.y, gv[2 * e] = fg.x, gv[2 * e + 1] = fg.y;
      }
#pragma unroll
      for (int r = 0; r < 8; ++r) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] += gv[r] * xv[c];
        if (with_bias) bs[r] += gv[r];
      }
    }
  }
  for (int m = ln >> 1; m >= 1; m >>= 1) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], m);
      bs[r] += __shfl_xor_sync(0xffffffffu, bs[r], m);
    }
  }
  const int n_w = 8 * cin * cout;
  float* dst = part + (size_t)blockIdx.x * (n_w + cout);
  if (valid) {
    // lane j writes the rows r with r = j (ln >= 8) or r = j mod ln (ln < 8)
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if ((ln >= 8 ? r : (r & (ln - 1))) != j) continue;
      float4* d = reinterpret_cast<float4*>(dst + ((size_t)(cog * 8 + r) * 8 + o) * cin + cig * 8);
      d[0] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
      d[1] = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
    }
  }
  if (j == 0 && tile < tb) {
#pragma unroll
    for (int r = 0; r < 8; ++r) sb[tile][r] = bs[r];
  }
  __syncthreads();
  // biases: the 8 tiles of one (co group, first ci group) pair, o = 0 .. 7 in order
  if ((int)threadIdx.x < tb) {
    const int q = threadIdx.x >> 3, r = threadIdx.x & 7;
    const int t0 = blockIdx.y * tb + q * 8;
    if (t0 < n_tiles && (t0 >> 3) / gco == 0) {
      float sum = 0.0f;
      for (int oo = 0; oo < 8; ++oo) sum += sb[q * 8 + oo][r];
      dst[n_w + ((t0 >> 3) % gco) * 8 + r] = sum;
    }
  }
}

// dst[i] += sum over blocks part[b][i] for the transposed convolution's (co, o, ci) + bias
// layout, the blocks summed in a fixed order
__global__ void k_sum_parts(const float* __restrict__ part, int nblk, int n, float* __restrict__ dst) {
  __shared__ float sh[32][32];
  for (int f0 = blockIdx.x * 32; f0 < n; f0 += gridDim.x * 32) {
    const int f = f0 + (threadIdx.x & 31);
    const float v = split_column_sum(part, nblk, (size_t)n, f, f < n, sh);
    if (threadIdx.x < 32 && f < n) dst[f] += v;
  }
}

// head: y[v] = sum_c W[c] x[v][c] + b (FP32), with per-block partial sums of y
__global__ void k_head(const bf16* __restrict__ x, int ldx, int c, const float* __restrict__ W,
                       const float* __restrict__ b, int n, float* __restrict__ y, double* part) {
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = b[0];
    for (int cc = 0; cc < c; cc += 8) {
      const uint4 q = *reinterpret_cast<const uint4*>(x + (size_t)i * ldx + cc);
      const bf16* h = reinterpret_cast<const bf16*>(&q);
#pragma unroll
      for (int e = 0; e < 8; ++e) s += W[cc + e] * __bfloat162float(h[e]);
    }
    y[i] = s;
    v[0] += s;
  }
  block_sum_store<1>(v, part);
}

// sums of p1 (for the mean of the guess)
__global__ void k_sum1(const double* __restrict__ a, int n, double* part) {
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += a[i];
  block_sum_store<1>(v, part);
}

// guess = p1 - mean(p1) + s_p (y - mean(y)); means[0] = mean y, means[1] = mean p1
__global__ void k_guess_out(const double* __restrict__ p1, const float* __restrict__ y, int n,
                            const double* __restrict__ scal, const double* __restrict__ means, double* __restrict__ out) {
  const double sp = scal[1], my = means[0], mp = means[1];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = p1[i] - mp + sp * ((double)y[i] - my);
}

// sum of (p - p1) (mean of the scaled target, times s_p)
__global__ void k_sum_diff(const double* __restrict__ p, const double* __restrict__ p1, int n, double* part) {
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[0] += p[i] - p1[i];
  block_sum_store<1>(v, part);
}

// d = (y - mean y) - (t - mean t), t = (p - p1) / s_p; gy = 2 d / n; partial sums of d^2.
// means[0] = mean y, means[2] = mean (p - p1).  The difference of the two pressures and its
// scaling in FP64 (they cancel), the rest in FP32 like y: this GPU's FP64 pipe runs about 1/60
// of the FP32 rate, and a thread's few terms sum in FP32 before the FP64 block and grid sums.
__global__ void k_loss(const double* __restrict__ p, const double* __restrict__ p1, const float* __restrict__ y, int n,
                       const double* __restrict__ scal, const double* __restrict__ means, float* __restrict__ gy,
                       double* part) {
  const double isp = 1.0 / scal[1], mt = means[2] * isp;
  const float my = (float)means[0], two_n = 2.0f / (float)n;
  float acc = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float t = (float)((p[i] - p1[i]) * isp - mt);
    const float d = (y[i] - my) - t;
    gy[i] = two_n * d;
    acc += d * d;
  }
  double v[1] = {acc};
  block_sum_store<1>(v, part);
}

// head backward: partial sums of gy * x[c] (c < C) and of gy; g_pre = bf16(W[c] gy) masked by x > 0.
// A thread's sums in FP32 (its few cells), the block and grid sums in FP64.
template <int C>
__global__ void k_head_bwd(const bf16* __restrict__ x, int ldx, const float* __restrict__ W,
                           const float* __restrict__ gy, int n, bf16* __restrict__ gpre, int ldg, double* part) {
  float v[C + 1];
#pragma unroll
  for (int q = 0; q <= C; ++q) v[q] = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float g = gy[i];
#pragma unroll
    for (int cc = 0; cc < C; cc += 8) {
      const uint4 q = *reinterpret_cast<const uint4*>(x + (size_t)i * ldx + cc);
      const bf16* h = reinterpret_cast<const bf16*>(&q);
      uint4 o;
      __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const float x0 = __bfloat162float(h[e]), x1 = __bfloat162float(h[e + 1]);
        v[cc + e] += g * x0;
        v[cc + e + 1] += g * x1;
        __nv_bfloat162 r = __floats2bfloat162_rn(W[cc + e] * g, W[cc + e + 1] * g);
        if (!(x0 > 0.0f)) r.x = __float2bfloat16(0.0f);
        if (!(x1 > 0.0f)) r.y = __float2bfloat16(0.0f);
        oh[e / 2] = r;
      }
      *reinterpret_cast<uint4*>(gpre + (size_t)i * ldg + cc) = o;
    }
    v[C] += g;
  }
  double vd[C + 1];
#pragma unroll
  for (int q = 0; q <= C; ++q) vd[q] = v[q];
  block_sum_store<C + 1>(vd, part);
}

// encoder output gradient: bf16((g_skip + g_pool / 8) * (act > 0)); thread per (cell, 8 channels).
// g_skip = channels [c, 2c) of the decoder-input gradient (ld lds), act = channels [c, 2c) of
// the decoder input (the encoder output), g_pool the coarse gradient of the pooled tensor.
__global__ void k_combine(const bf16* __restrict__ gskip, int lds, const bf16* __restrict__ gpool, int ldp,
                          const bf16* __restrict__ act, int lda, Dims fine, int c, bf16* __restrict__ out, int ldo) {
  const int groups = c / 8;
  const int total = fine.n() * groups;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int gq = i % groups, v = i / groups;
    const int x = v % fine.nx, r = v / fine.nx, y = r % fine.ny, z = r / fine.ny;
    const int cv = (x >> 1) + (fine.nx >> 1) * ((y >> 1) + (fine.ny >> 1) * (z >> 1));
    const uint4 qs = *reinterpret_cast<const uint4*>(gskip + (size_t)v * lds + gq * 8);
    const uint4 qp = *reinterpret_cast<const uint4*>(gpool + (size_t)cv * ldp + gq * 8);
    const uint4 qa = *reinterpret_cast<const uint4*>(act + (size_t)v * lda + gq * 8);
    const bf16* hs = reinterpret_cast<const bf16*>(&qs);
    const bf16* hp = reinterpret_cast<const bf16*>(&qp);
    const bf16* ha = reinterpret_cast<const bf16*>(&qa);
    uint4 o;
    __nv_bfloat162* oh = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float a0 = __bfloat162float(hs[e]) + __bfloat162float(hp[e]) * 0.125f;
      float a1 = __bfloat162float(hs[e + 1]) + __bfloat162float(hp[e + 1]) * 0.125f;
      if (!(__bfloat162float(ha[e]) > 0.0f)) a0 = 0.0f;
      if (!(__bfloat162float(ha[e + 1]) > 0.0f)) a1 = 0.0f;
      oh[e / 2] = __floats2bfloat162_rn(a0, a1);
    }
    *reinterpret_cast<uint4*>(out + (size_t)v * ldo + gq * 8) = o;
  }
}

// Adam (Kingma and Ba 2015, Algorithm 1) on FP32 masters; c1 = 1 / (1 - beta1^t),
// c2 = 1 / (1 - beta2^t); the gradient is scaled first and zeroed after use.
__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v, float* __restrict__ g,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2, float gscale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    g[i] = 0.0f;
  }
}

// BF16 copies of a 3x3x3 convolution's weights W[co][tap][ci] (ci < cin):
//   forward  wf[n][k]: n = co < np, k = tap * cin_pad + ci < kpad (zero elsewhere)
//   gradient wd[n][k]: n = ci < npd, k = tap' * cout + co < kpadd with tap' = 26 - tap
__global__ void k_pack_conv3(const float* __restrict__ W, int cin, int cin_pad, int cout, bf16* __restrict__ wf,
                             int np, int kpad, bf16* __restrict__ wd, int npd, int kpadd) {
  const int tf = np * kpad, td = npd * kpadd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tf + td; i += gridDim.x * blockDim.x) {
    if (i < tf) {
      const int n = i / kpad, k = i - n * kpad;
      const int tap = k / cin_pad, ci = k - tap * cin_pad;
      float val = 0.0f;
      if (n < cout && tap < 27 && ci < cin) val = W[((size_t)n * 27 + tap) * cin + ci];
      wf[i] = __float2bfloat16(val);
    } else {
      const int j = i - tf;
      const int n = j / kpadd, k = j - n * kpadd;
      const int tp = k / cout, co = k - tp * cout;
      float val = 0.0f;
      if (n < cin && tp < 27) val = W[((size_t)co * 27 + (26 - tp)) * cin + n];
      wd[j] = __float2bfloat16(val);
    }
  }
}

// BF16 weights of a 3x3x3 convolution in the row kernel's K order, [np][row_k(C)] for an input
// of C channels: with C = 8 the K cores per (dz, dy) line are x offsets -1, 0, +1 and a zero
// core; otherwise K = tap * C + c.  Forward (dgrad = 0): rows n = output channel < cout,
// c = input channel < cin.  Input gradient: rows n = input channel < cin, c = output channel,
// taps flipped.
__global__ void k_pack_row(const float* __restrict__ W, int cin, int cout, int dgrad, int C, int np,
                           bf16* __restrict__ dst) {
  const int kr = row_k(C);
  const int nrows = dgrad ? cin : cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np * kr; i += gridDim.x * blockDim.x) {
    const int n = i / kr, K = i - n * kr;
    int tap, c;
    if (C == 8) {
      const int core = K >> 3, r = core & 3;
      c = K & 7;
      tap = r < 3 ? (core >> 2) * 3 + r : -1;
    } else {
      tap = K / C;
      c = K - tap * C;
    }
    float v = 0.0f;
    if (tap >= 0 && n < nrows) {
      if (!dgrad) {
        if (c < cin) v = W[((size_t)n * 27 + tap) * cin + c];
      } else if (c < cout) {
        v = W[((size_t)c * 27 + (26 - tap)) * cin + n];
      }
    }
    dst[i] = __float2bfloat16(v);
  }
}

// BF16 weights of a 3x3x3 convolution for the slab kernel, [3 pw][stack_k(C)] for an
// input of C channels: row n = (dx + 1) pw + o (o < pw, zero rows past the real channels),
// column K = ((dz + 1) 3 + (dy + 1)) C + c (C = 8: see stack_k).  Forward (dgrad = 0): o = output channel < cout,
// c = input channel < cin.  Input gradient: o = input channel < cin, c = output channel,
// taps flipped.
__global__ void k_pack_slab(const float* __restrict__ W, int cin, int cout, int dgrad, int C, int pw,
                            bf16* __restrict__ dst) {
  const int ktot = stack_k(C), nt = 3 * pw;
  const int nrows = dgrad ? cin : cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt * ktot; i += gridDim.x * blockDim.x) {
    const int n = i / ktot, K = i - n * ktot;
    const int part = n / pw, o = n - part * pw;
    int li, c;
    if (C == 8) {  // MMA m = 2 (dy + 1) + pair, core kc: plane dz + 1 = 2 pair + kc (3: zero)
      const int m = K >> 4, kc = (K >> 3) & 1, dzi = 2 * (m & 1) + kc;
      c = K & 7;
      li = dzi < 3 ? dzi * 3 + (m >> 1) : -1;
    } else {
      li = K / C;
      c = K - li * C;
    }
    const int tap = li * 3 + part;  // (dz + 1) 9 + (dy + 1) 3 + (dx + 1)
    float v = 0.0f;
    if (li >= 0 && o < nrows) {
      if (!dgrad) {
        if (c < cin) v = W[((size_t)o * 27 + tap) * cin + c];
      } else if (c < cout) {
        v = W[((size_t)c * 27 + (26 - tap)) * cin + o];
      }
    }
    dst[i] = __float2bfloat16(v);
  }
}

__global__ void k_to_bf16(const float* __restrict__ a, int n, bf16* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = __float2bfloat16(a[i]);
}

// activation inspection: [n][c] of a BF16 buffer with leading dimension ld -> FP32
__global__ void k_bf16_to_f32(const bf16* __restrict__ a, int lda, int n, int c, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * c; i += gridDim.x * blockDim.x) {
    const int v = i / c, cc = i - v * c;
    out[i] = __bfloat162float(a[(size_t)v * lda + cc]);
  }
}

// guess selection: r = b - A c for two candidates (A c already in ac0 / ac1), sums of r^2, b^2
// The judge's two candidates are kept interleaved, [n][2] (cell i: candidate 0 then 1), so that
// each smoothing sweep applies A to both in one k = 2 SpMM (the matrix read once for the two).
__global__ void k_pack2(const double* __restrict__ c0, const double* __restrict__ c1, int n, double* __restrict__ xs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    xs[2 * i] = c0[i];
    xs[2 * i + 1] = c1[i];
  }
}

// damped Jacobi on both candidates: x += omega D^-1 (b - A x)
__global__ void k_jacobi2(const double* __restrict__ b, const double* __restrict__ ax, const double* __restrict__ dinv,
                          double omega, int n, double* __restrict__ xs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = omega * dinv[i];
    xs[2 * i] += w * (b[i] - ax[2 * i]);
    xs[2 * i + 1] += w * (b[i] - ax[2 * i + 1]);
  }
}

__global__ void k_resid2(const double* __restrict__ b, const double* __restrict__ ax, int n, double* part) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double bi = b[i], r0 = bi - ax[2 * i], r1 = bi - ax[2 * i + 1];
    v[0] += r0 * r0;
    v[1] += r1 * r1;
    v[2] += bi * bi;
  }
  block_sum_store<3>(v, part);
}

__global__ void k_pick(const double* __restrict__ xs, int n, const double* __restrict__ sums, double* __restrict__ res,
                       int* __restrict__ choice, double* __restrict__ x0) {
  const double bb = sums[2] > 0.0 ? sums[2] : 1.0;
  const int pick = sums[1] < sums[0] ? 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    res[0] = sqrt(sums[0] / bb);
    res[1] = sqrt(sums[1] / bb);
    *choice = pick;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x0[i] = xs[2 * i + pick];
}

// ------------------------------------------------------------------------------ host side

int round_up(int v, int m) { return (v + m - 1) / m * m; }

enum LayerKind { kConv3 = 0, kUp = 1, kHead = 2 };

struct Layer {
  LayerKind kind;
  int level = 0;
  int cin = 0, cout = 0;  // cin as in the parameter vector (3 for enc0a)
  int cin_pad = 0;        // channels of the GEMM input
  int64_t w_off = 0, b_off = 0;
  int np = 0, kpad = 0, npd = 0, kpadd = 0, mpad = 0;  // conv3 packing
  bf16* wf = nullptr;
  bf16* wd = nullptr;
  bf16* wf_row = nullptr;  // row-kernel layouts (level-0 rows of 128 cells), or null
  bf16* wd_row = nullptr;
  bf16* wf_slab = nullptr;  // slab-kernel layouts (rows of 16 or 32 cells), or null
  bf16* wd_slab = nullptr;
  int pw_f = 0, pw_d = 0;   // their column blocks: output channels rounded up to 16
  bf16* wu = nullptr;  // up: BF16 [cout][8][cin]
};

}  // namespace
}  // namespace rb

struct rb_guess {
  rb_guess_cfg cfg{};
  int L = 0;
  std::vector<int> ch;
  std::vector<rb::Dims> dims;
  std::vector<rb::Layer> layers;
  int64_t n_params = 0;
  int64_t adam_t = 0;
  float* theta = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* grad = nullptr;
  // activations (BF16)
  rb::bf16* x0 = nullptr;                 // [n0][8]
  std::vector<rb::bf16*> enc_a, cat, pooled, dec_a, dec_b;
  rb::bf16* bottom = nullptr;
  float* y = nullptr;
  float* gy = nullptr;
  // gradients (BF16)
  std::vector<rb::bf16*> g_b, g_a, g_cat, g_eb, g_ea, g_pool;
  rb::bf16* g_bottom = nullptr;
  // scratch
  double* red = nullptr;    // reduction partials
  double* scal = nullptr;   // [0] s_b, [1] s_p, [2..5] sums / means, [6] loss
  float* wpart = nullptr;   // weight-gradient partials
  size_t wpart_floats = 0;
  double* sel = nullptr;    // [4 n] A x0, A x1 and the smoothed candidates of the guess selection
  int* err = nullptr;
  std::vector<void*> allocs;
};

namespace rb {
namespace {

template <typename T>
rb_status galloc(rb_guess* g, T** p, size_t count) {
  void* q = nullptr;
  RB_CUDA(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
  RB_CUDA(cudaMemset(q, 0, std::max<size_t>(count, 1) * sizeof(T)));
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return RB_OK;
}

int conv_np(int c) { return round_up(c, 16); }

rb_status check_cfg(const rb_guess_cfg* c) {
  RB_REQUIRE(c != nullptr, "rb_guess: null configuration");
  RB_REQUIRE(c->levels >= 2 && c->levels <= 4, "rb_guess: levels must be 2..4 (got %d)", c->levels);
  const int f = 1 << (c->levels - 1);
  RB_REQUIRE(c->nx > 0 && c->ny > 0 && c->nz > 0 && c->nx % f == 0 && c->ny % f == 0 && c->nz % f == 0,
             "rb_guess: grid %d x %d x %d not divisible by 2^(levels-1) = %d", c->nx, c->ny, c->nz, f);
  RB_REQUIRE((int64_t)c->nx * c->ny * c->nz < (1LL << 30), "rb_guess: grid too large");
  for (int l = 0; l < c->levels; ++l)
    RB_REQUIRE(c->channels[l] >= 8 && c->channels[l] % 8 == 0, "rb_guess: channels[%d] = %d not a positive multiple of 8",
               l, c->channels[l]);
  return RB_OK;
}

void build_layers(const rb_guess_cfg& c, std::vector<Layer>& out, int64_t& n) {
  out.clear();
  n = 0;
  auto add = [&](LayerKind k, int level, int cin, int cout) {
    Layer ly;
    ly.kind = k;
    ly.level = level;
    ly.cin = cin;
    ly.cout = cout;
    ly.cin_pad = round_up(cin, 8);
    ly.w_off = n;
    n += (k == kConv3 ? 27LL * cin * cout : (k == kUp ? 8LL * cin * cout : cin));
    ly.b_off = n;
    n += cout;
    if (k == kConv3) {
      ly.np = conv_np(cout);
      ly.kpad = round_up(27 * ly.cin_pad, kKS);
      ly.npd = conv_np(ly.cin_pad);
      ly.kpadd = round_up(27 * cout, kKS);
      ly.mpad = round_up(27 * ly.cin_pad + 1, 128);
    }
    out.push_back(ly);
  };
  const int L = c.levels;
  int cin = 3;
  for (int l = 0; l < L; ++l) {
    add(kConv3, l, cin, c.channels[l]);
    add(kConv3, l, c.channels[l], c.channels[l]);
    cin = c.channels[l];
  }
  for (int l = L - 2; l >= 0; --l) {
    add(kUp, l, c.channels[l + 1], c.channels[l]);
    add(kConv3, l, 2 * c.channels[l], c.channels[l]);
    add(kConv3, l, c.channels[l], c.channels[l]);
  }
  add(kHead, 0, c.channels[0], 1);
}

int guess_sm_count() {
  thread_local int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
  }
  return sms;
}

// CTAs of `kernel` that one SM holds at once: the tightest of threads, registers, shared
// memory (dynamic + static + the per-block reserve) and tensor memory (512 columns per SM).
int blocks_per_sm(const void* kernel, size_t dyn_smem, int threads, uint32_t tmem_cols) {
  cudaFuncAttributes fa{};
  int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0, resv = 0;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = std::min(blk_sm, thr_sm / threads);
  const int regs = std::max(1, fa.numRegs) * threads;
  n = std::min(n, regs_sm / regs);
  const size_t per_block = dyn_smem + fa.sharedSizeBytes + (size_t)resv;
  n = std::min<int>(n, (int)(smem_sm / std::max<size_t>(per_block, 1)));
  n = std::min<int>(n, (int)(512 / tmem_cols));
  return std::max(1, n);
}

size_t conv_smem(int np, int kpad) { return (size_t)np * kpad * 2 + (size_t)kStages * kAStage; }

template <int NP>
rb_status launch_conv3_np(const Conv3Args& a, size_t smem, cudaStream_t s) {
  auto* kern = &k_conv3_mma<NP>;
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(kern), smem));
  const int n_tiles = (a.n_vox + 127) / 128;
  thread_local int per_sm = 0;
  thread_local size_t per_sm_smem = 0;
  if (per_sm == 0 || per_sm_smem != smem) {
    per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), smem, kConvThreads, tmem_cols_for(2 * NP));
    per_sm_smem = smem;
  }
  const int grid = std::max(1, std::min(n_tiles, per_sm * guess_sm_count()));
  kern<<<grid, kConvThreads, smem, s>>>(a);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

}  // namespace
}  // namespace rb

namespace rb {
namespace {

// layer indices in the flat order
int enc_idx(int l, int s) { return 2 * l + s; }
int dec_base(const rb_guess* g, int l) { return 2 * g->L + 3 * (g->L - 2 - l); }
int head_idx(const rb_guess* g) { return 2 * g->L + 3 * (g->L - 1); }

template <int NP, int W>
rb_status launch_row_np(const Conv3Args& a, size_t smem, cudaStream_t s) {
  auto* kern = &k_conv3_row<NP, W>;
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(kern), smem));
  thread_local int per_sm = 0;
  thread_local size_t per_sm_smem = 0;
  if (per_sm == 0 || per_sm_smem != smem) {
    per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), smem, kConvThreads, tmem_cols_for(2 * NP));
    per_sm_smem = smem;
  }
  const int chunk = row_chunk_fill(a.d.ny, a.d.nz, per_sm * guess_sm_count());
  const int items = a.d.nz * ((a.d.ny + chunk - 1) / chunk);
  const int grid = std::max(1, std::min(items, per_sm * guess_sm_count()));
  kern<<<grid, kConvThreads, smem, s>>>(a, chunk);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// the row kernel takes grids whose rows are 128 or 64 cells and inputs of 8 or an even number
// of 8-channel groups
bool row_kernel_fits(const Dims& d, int cin, int np) {
  return (d.nx == 128 || d.nx == 64) && (cin == 8 || (cin % 16 == 0)) && np <= 64 &&
         row_smem(np, cin, d.nx) <= kMaxConvSmem;
}

rb_status row_launch(const Conv3Args& a, int np, cudaStream_t s) {
  const size_t smem = row_smem(np, a.cin, a.d.nx);
  const bool w128 = a.d.nx == 128;
  switch (np) {
    case 16: return w128 ? launch_row_np<16, 128>(a, smem, s) : launch_row_np<16, 64>(a, smem, s);
    case 32: return w128 ? launch_row_np<32, 128>(a, smem, s) : launch_row_np<32, 64>(a, smem, s);
    case 48: return w128 ? launch_row_np<48, 128>(a, smem, s) : launch_row_np<48, 64>(a, smem, s);
    case 64: return w128 ? launch_row_np<64, 128>(a, smem, s) : launch_row_np<64, 64>(a, smem, s);
  }
  set_error("rb_guess: no row convolution kernel for %d output channels", np);
  return RB_EUNSUPPORTED;
}

template <int NT, int W>
rb_status launch_slab_nt(const Conv3Args& a, int pw, size_t smem, cudaStream_t s) {
  auto* kern = &k_conv3_slab<NT, W>;
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(kern), smem));
  thread_local int per_sm = 0;
  thread_local size_t per_sm_smem = 0;
  if (per_sm == 0 || per_sm_smem != smem) {
    per_sm = blocks_per_sm(reinterpret_cast<const void*>(kern), smem, kConvThreads, tmem_cols_for(NT));
    per_sm_smem = smem;
  }
  const int n_tiles = a.d.nz * (a.d.ny / (128 / W));
  const int grid = std::max(1, std::min(n_tiles, per_sm * guess_sm_count()));
  kern<<<grid, kConvThreads, smem, s>>>(a, pw);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// the slab kernel takes rows of 16, 32 or 64 cells (whole rows per 128-cell tile), inputs of
// 8 channels or an even number of 8-channel groups and at most 192 stacked output columns
bool slab_kernel_fits(const Dims& d, int cin, int pw) {
  return (d.nx == 16 || d.nx == 32 || d.nx == 64) && d.ny % (128 / d.nx) == 0 && (cin == 8 || cin % 16 == 0) &&
         pw % 16 == 0 && 3 * pw <= 192 && slab_smem(3 * pw, cin, d.nx) <= kMaxConvSmem;
}

template <int NT>
rb_status slab_launch_w(const Conv3Args& a, int pw, size_t smem, cudaStream_t s) {
  switch (a.d.nx) {
    case 16: return launch_slab_nt<NT, 16>(a, pw, smem, s);
    case 32: return launch_slab_nt<NT, 32>(a, pw, smem, s);
    case 64: return launch_slab_nt<NT, 64>(a, pw, smem, s);
  }
  set_error("rb_guess: no slab convolution kernel for rows of %d cells", a.d.nx);
  return RB_EUNSUPPORTED;
}

rb_status slab_launch(const Conv3Args& a, int pw, cudaStream_t s) {
  const size_t smem = slab_smem(3 * pw, a.cin, a.d.nx);
  switch (3 * pw) {
    case 48: return slab_launch_w<48>(a, pw, smem, s);
    case 96: return slab_launch_w<96>(a, pw, smem, s);
    case 144: return slab_launch_w<144>(a, pw, smem, s);
    case 192: return slab_launch_w<192>(a, pw, smem, s);
  }
  set_error("rb_guess: no slab convolution kernel for %d output channels", pw);
  return RB_EUNSUPPORTED;
}

rb_status conv3_launch(const Conv3Args& a, int np, cudaStream_t s) {
  const size_t smem = conv_smem(np, a.kpad);
  RB_REQUIRE(a.kpad / 8 <= kMaxChunks, "rb_guess: convolution with %d input channels too wide", a.cin);
  RB_REQUIRE(smem <= kMaxConvSmem, "rb_guess: convolution weights (%d x %d) exceed shared memory", np, a.kpad);
  switch (np) {
    case 16: return launch_conv3_np<16>(a, smem, s);
    case 32: return launch_conv3_np<32>(a, smem, s);
    case 48: return launch_conv3_np<48>(a, smem, s);
    case 64: return launch_conv3_np<64>(a, smem, s);
    case 96: return launch_conv3_np<96>(a, smem, s);
    case 128: return launch_conv3_np<128>(a, smem, s);
  }
  set_error("rb_guess: no convolution kernel for %d output channels", np);
  return RB_EUNSUPPORTED;
}

// y = relu?(conv(x) + b): forward of layer ly at its level
rb_status conv3_fwd(rb_guess* g, const Layer& ly, const bf16* x, int ldx, bf16* y, int ldy, cudaStream_t s) {
  Conv3Args a;
  a.x = x;
  a.ldx = ldx;
  a.cin = ly.cin_pad;
  a.d = g->dims[ly.level];
  a.n_vox = a.d.n();
  a.w = ly.wf;
  a.kpad = ly.kpad;
  a.bias = g->theta + ly.b_off;
  a.relu = 1;
  a.y = y;
  a.ldy = ldy;
  a.cout = ly.cout;
  a.err = g->err;
  if (ly.wf_slab) {
    a.w = ly.wf_slab;
    return slab_launch(a, ly.pw_f, s);
  }
  if (ly.wf_row) {
    a.w = ly.wf_row;
    return row_launch(a, ly.np, s);
  }
  return conv3_launch(a, ly.np, s);
}

// gin = conv^T(gpre) (masked by mask > 0 when mask != nullptr)
rb_status conv3_dgrad(rb_guess* g, const Layer& ly, const bf16* gpre, int ldg, const bf16* mask, int ldm, bf16* gin,
                      int ldgi, cudaStream_t s) {
  Conv3Args a;
  a.x = gpre;
  a.ldx = ldg;
  a.cin = ly.cout;
  a.d = g->dims[ly.level];
  a.n_vox = a.d.n();
  a.w = ly.wd;
  a.kpad = ly.kpadd;
  a.mask = mask;
  a.ldm = ldm;
  a.y = gin;
  a.ldy = ldgi;
  a.cout = ly.cin_pad;
  a.err = g->err;
  if (ly.wd_slab) {
    a.w = ly.wd_slab;
    return slab_launch(a, ly.pw_d, s);
  }
  if (ly.wd_row) {
    a.w = ly.wd_row;
    return row_launch(a, ly.npd, s);
  }
  return conv3_launch(a, ly.npd, s);
}

struct WgradPlan {
  int m_tiles = 0, splits = 0, cells = 0;
};

WgradPlan wgrad_plan(const Layer& ly, int n) {
  WgradPlan p;
  p.m_tiles = ly.mpad / 128;
  const int target = std::max(1, (4 * guess_sm_count()) / p.m_tiles);
  p.cells = round_up(std::max(1, (n + target - 1) / target), kWS);
  p.splits = (n + p.cells - 1) / p.cells;
  return p;
}

template <int NP>
rb_status launch_wgrad_np(const WgradArgs& a, const WgradPlan& p, cudaStream_t s) {
  const size_t smem = (size_t)kStages * (kWAStage + NP * kWS * 2);
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(&k_wgrad_mma<NP>), smem));
  k_wgrad_mma<NP><<<dim3(p.m_tiles, p.splits), kConvThreads, smem, s>>>(a);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// The line-buffer weight gradient: rows of 16 to 128 cells, at most two output groups (its
// per-thread bias sums) and eight 32-column accumulators (256 TMEM columns)
struct LinWPlan {
  int chunk = 0, splits = 0, per_split = 0, go_cta = 0, go_tiles = 0;
  size_t smem = 0;
};

// output groups per CTA: two, or one where two would need more than eight accumulators
int wgrad_lin_go(const Layer& ly) {
  const int G = ly.cin_pad / 8, Go = (ly.cout + 7) / 8;
  return (Go >= 2 && 2 * G <= 8) ? 2 : 1;
}

bool wgrad_lin_fits(const Layer& ly, const Dims& d) {
  const int G = ly.cin_pad / 8, go = wgrad_lin_go(ly);
  return (d.nx == 16 || d.nx == 32 || d.nx == 64 || d.nx == 128) && G * go <= 8 &&
         wgrad_lin_smem(d.nx, G, go, 2) <= kMaxConvSmem;
}

const void* wgrad_lin_kernel(int W) {
  switch (W) {
    case 16: return (const void*)&k_wgrad_lin<16>;
    case 32: return (const void*)&k_wgrad_lin<32>;
    case 64: return (const void*)&k_wgrad_lin<64>;
    default: return (const void*)&k_wgrad_lin<128>;
  }
}

// runs of the longest chunk (16, 8, 4, 2 rows) whose line buffer leaves room for four CTAs per
// SM (the kernel waits on a block barrier every row: more CTAs hide it), then one wave of CTAs
// with equal shares of the runs
constexpr size_t kWlinSmemTarget = 56 * 1024;
LinWPlan wgrad_lin_plan(const Layer& ly, const Dims& d) {
  LinWPlan p;
  const int G = ly.cin_pad / 8, Go = wgrad_lin_go(ly);
  p.go_cta = Go;
  p.go_tiles = ((ly.cout + 7) / 8 + Go - 1) / Go;
  p.chunk = 2;
  for (int c = 16; c >= 2; c /= 2)
    if (wgrad_lin_smem(d.nx, G, Go, c) <= kWlinSmemTarget || c == 2) {
      p.chunk = std::min(c, std::max(2, d.ny));
      break;
    }
  p.smem = wgrad_lin_smem(d.nx, G, Go, p.chunk);
  const int resident = blocks_per_sm(wgrad_lin_kernel(d.nx), p.smem, kConvThreads, tmem_cols_for(32 * G * Go)) *
                       guess_sm_count();
  const int items = d.nz * ((d.ny + p.chunk - 1) / p.chunk);
  const int target = std::max(1, resident / p.go_tiles);
  p.per_split = std::max(1, (items + target - 1) / target);
  p.splits = (items + p.per_split - 1) / p.per_split;
  return p;
}

template <int W>
rb_status launch_wgrad_lin(const WgradArgs& a, const LinWPlan& p, cudaStream_t s) {
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(&k_wgrad_lin<W>), p.smem));
  k_wgrad_lin<W><<<dim3(p.splits, p.go_tiles), kConvThreads, p.smem, s>>>(a, p.chunk, p.per_split);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

rb_status conv3_wgrad(rb_guess* g, const Layer& ly, const bf16* x, int ldx, const bf16* gpre, int ldg, cudaStream_t s) {
  const Dims d = g->dims[ly.level];
  if (wgrad_lin_fits(ly, d)) {
    const LinWPlan lp = wgrad_lin_plan(ly, d);
    WgradArgs a;
    a.x = x;
    a.ldx = ldx;
    a.cin = ly.cin_pad;
    a.g = gpre;
    a.ldg = ldg;
    a.cout = ly.cout;
    a.d = d;
    a.n_vox = d.n();
    a.rows = 27 * ly.cin_pad;
    a.mpad = ly.mpad;
    a.np = ly.np;
    a.go_cta = lp.go_cta;
    a.part = g->wpart;
    a.err = g->err;
    rb_status st;
    switch (d.nx) {
      case 16: st = launch_wgrad_lin<16>(a, lp, s); break;
      case 32: st = launch_wgrad_lin<32>(a, lp, s); break;
      case 64: st = launch_wgrad_lin<64>(a, lp, s); break;
      default: st = launch_wgrad_lin<128>(a, lp, s); break;
    }
    RB_TRY(st);
    k_wgrad_reduce<<<split_sum_blocks((int64_t)(a.rows + 1) * ly.np), split_sum_threads(lp.splits), 0, s>>>(
        g->wpart, lp.splits, ly.mpad, ly.np, ly.cin_pad, ly.cin, ly.cout, g->grad + ly.w_off, g->grad + ly.b_off);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
  }
  const WgradPlan p = wgrad_plan(ly, d.n());
  WgradArgs a;
  a.x = x;
  a.ldx = ldx;
  a.cin = ly.cin_pad;
  a.g = gpre;
  a.ldg = ldg;
  a.cout = ly.cout;
  a.d = d;
  a.n_vox = d.n();
  a.rows = 27 * ly.cin_pad;
  a.mpad = ly.mpad;
  a.cells_per_split = p.cells;
  a.part = g->wpart;
  a.err = g->err;
  rb_status st;
  switch (ly.np) {
    case 16: st = launch_wgrad_np<16>(a, p, s); break;
    case 32: st = launch_wgrad_np<32>(a, p, s); break;
    case 48: st = launch_wgrad_np<48>(a, p, s); break;
    case 64: st = launch_wgrad_np<64>(a, p, s); break;
    default:
      set_error("rb_guess: no weight-gradient kernel for %d output channels", ly.np);
      return RB_EUNSUPPORTED;
  }
  RB_TRY(st);
  k_wgrad_reduce<<<split_sum_blocks((int64_t)(a.rows + 1) * ly.np), split_sum_threads(p.splits), 0, s>>>(
      g->wpart, p.splits, ly.mpad, ly.np, ly.cin_pad, ly.cin, ly.cout, g->grad + ly.w_off, g->grad + ly.b_off);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// k_up_dw's launch: tiles of 8 x 8 outputs, up to 64 per block; lanes per tile the largest power
// of two that keeps the block within 256 threads; one wave of two blocks per SM split into
// equal ranges of coarse cells
struct UpDwPlan {
  int tb = 0, ln = 0, gy = 0, cells = 0, splits = 0;
};
UpDwPlan up_dw_plan(const rb_guess* g, const Layer& ly) {
  UpDwPlan p;
  const int nc = g->dims[ly.level].n() / 8;
  const int n_tiles = ly.cout * ly.cin / 8;
  p.tb = std::min(n_tiles, 64);
  p.ln = 1;
  while (p.ln * 2 * p.tb <= kUpDwThreads) p.ln *= 2;
  p.gy = (n_tiles + p.tb - 1) / p.tb;
  const int target = std::max(1, 2 * guess_sm_count() / p.gy);
  p.cells = std::max(1, (nc + target - 1) / target);
  p.splits = std::max(1, (nc + p.cells - 1) / p.cells);
  return p;
}

size_t wpart_need(const rb_guess* g) {
  size_t need = 1;
  for (const Layer& ly : g->layers) {
    if (ly.kind == kConv3) {
      const WgradPlan p = wgrad_plan(ly, g->dims[ly.level].n());
      need = std::max(need, (size_t)p.splits * ly.mpad * ly.np);
      if (wgrad_lin_fits(ly, g->dims[ly.level]))
        need = std::max(need, (size_t)wgrad_lin_plan(ly, g->dims[ly.level]).splits * ly.mpad * ly.np);
    } else if (ly.kind == kUp) {
      need = std::max(need, (size_t)up_dw_plan(g, ly).splits * (8 * ly.cin * ly.cout + ly.cout));
    }
  }
  return need;
}

rb_status refresh_weights(rb_guess* g, cudaStream_t s) {
  for (Layer& ly : g->layers) {
    if (ly.kind == kConv3) {
      const int total = ly.np * ly.kpad + ly.npd * ly.kpadd;
      k_pack_conv3<<<std::min(1024, (total + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, ly.cin, ly.cin_pad, ly.cout,
                                                                       ly.wf, ly.np, ly.kpad, ly.wd, ly.npd, ly.kpadd);
      if (ly.wf_row) {
        const int t = ly.np * row_k(ly.cin_pad);
        k_pack_row<<<std::min(1024, (t + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, ly.cin, ly.cout, 0, ly.cin_pad,
                                                                   ly.np, ly.wf_row);
      }
      if (ly.wd_row) {
        const int t = ly.npd * row_k(ly.cout);
        k_pack_row<<<std::min(1024, (t + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, ly.cin, ly.cout, 1, ly.cout,
                                                                   ly.npd, ly.wd_row);
      }
      if (ly.wf_slab) {
        const int t = 3 * ly.pw_f * stack_k(ly.cin_pad);
        k_pack_slab<<<std::min(1024, (t + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, ly.cin, ly.cout, 0, ly.cin_pad,
                                                                    ly.pw_f, ly.wf_slab);
      }
      if (ly.wd_slab) {
        const int t = 3 * ly.pw_d * stack_k(ly.cout);
        k_pack_slab<<<std::min(1024, (t + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, ly.cin, ly.cout, 1, ly.cout,
                                                                    ly.pw_d, ly.wd_slab);
      }
    } else if (ly.kind == kUp) {
      const int total = 8 * ly.cin * ly.cout;
      k_to_bf16<<<std::min(1024, (total + 255) / 256), 256, 0, s>>>(g->theta + ly.w_off, total, ly.wu);
    }
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

int grid_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>(kRedGrid, (work + 255) / 256)); }

rb_status forward(rb_guess* g, const double* b, const double* p1, const double* p2, cudaStream_t s) {
  const int L = g->L;
  const int n0 = g->dims[0].n();
  k_sumsq2<<<kRedGrid, kRedThreads, 0, s>>>(b, p1, n0, g->red);
  k_finish<<<2, 256, 0, s>>>(g->red, kRedGrid, 2, g->scal + 2, 1.0 / n0);
  k_make_input<<<grid_for(n0), 256, 0, s>>>(b, p1, p2, n0, g->scal + 2, g->scal, g->x0);
  RB_CUDA(cudaGetLastError());
  for (int l = 0; l < L; ++l) {
    const int c = g->ch[l];
    const bf16* in = l == 0 ? g->x0 : g->pooled[l - 1];
    const int ldin = l == 0 ? 8 : g->ch[l - 1];
    RB_TRY(conv3_fwd(g, g->layers[enc_idx(l, 0)], in, ldin, g->enc_a[l], c, s));
    bf16* out = l < L - 1 ? g->cat[l] + c : g->bottom;
    const int ldo = l < L - 1 ? 2 * c : c;
    RB_TRY(conv3_fwd(g, g->layers[enc_idx(l, 1)], g->enc_a[l], c, out, ldo, s));
    if (l < L - 1) {
      k_pool<<<grid_for((int64_t)g->dims[l + 1].n() * (c / 8)), 256, 0, s>>>(out, ldo, g->dims[l], c, g->pooled[l], c);
      RB_CUDA(cudaGetLastError());
    }
  }
  for (int l = L - 2; l >= 0; --l) {
    const int c = g->ch[l], cc = g->ch[l + 1];
    const int base = dec_base(g, l);
    const Layer& up = g->layers[base];
    const bf16* in = l == L - 2 ? g->bottom : g->dec_b[l + 1];
    const size_t sm = (size_t)up.cout * 8 * up.cin * 2;
    k_up<<<grid_for((int64_t)g->dims[l].n() * (c / 8)), 256, sm, s>>>(in, cc, cc, up.wu, g->theta + up.b_off, g->dims[l],
                                                                      c, g->cat[l], 2 * c);
    RB_CUDA(cudaGetLastError());
    RB_TRY(conv3_fwd(g, g->layers[base + 1], g->cat[l], 2 * c, g->dec_a[l], c, s));
    RB_TRY(conv3_fwd(g, g->layers[base + 2], g->dec_a[l], c, g->dec_b[l], c, s));
  }
  const Layer& hd = g->layers[head_idx(g)];
  k_head<<<kRedGrid, kRedThreads, 0, s>>>(g->dec_b[0], g->ch[0], g->ch[0], g->theta + hd.w_off, g->theta + hd.b_off, n0,
                                          g->y, g->red);
  k_finish<<<1, 256, 0, s>>>(g->red, kRedGrid, 1, g->scal + 2, 1.0 / n0);  // scal[2] = mean y
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <int C>
rb_status head_bwd_c(rb_guess* g, cudaStream_t s) {
  const Layer& hd = g->layers[head_idx(g)];
  const int n0 = g->dims[0].n();
  k_head_bwd<C><<<kRedGrid, kRedThreads, 0, s>>>(g->dec_b[0], C, g->theta + hd.w_off, g->gy, n0, g->g_b[0], C, g->red);
  // parameter gradient: head W (C sums) and b, added into grad
  k_finish<<<C + 1, 256, 0, s>>>(g->red, kRedGrid, C + 1, g->scal + 8, 1.0);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

__global__ void k_add_head_grad(const double* __restrict__ sums, int c, float* __restrict__ gw, float* __restrict__ gb) {
  const int i = threadIdx.x;
  if (i < c) gw[i] += (float)sums[i];
  if (i == c) gb[0] += (float)sums[c];
}

rb_status backward(rb_guess* g, cudaStream_t s) {
  const int L = g->L;
  const Layer& hd = g->layers[head_idx(g)];
  switch (g->ch[0]) {
    case 8: RB_TRY(head_bwd_c<8>(g, s)); break;
    case 16: RB_TRY(head_bwd_c<16>(g, s)); break;
    case 24: RB_TRY(head_bwd_c<24>(g, s)); break;
    case 32: RB_TRY(head_bwd_c<32>(g, s)); break;
    default:
      set_error("rb_guess: the head takes 8, 16, 24 or 32 channels at level 0");
      return RB_EUNSUPPORTED;
  }
  k_add_head_grad<<<1, 64, 0, s>>>(g->scal + 8, g->ch[0], g->grad + hd.w_off, g->grad + hd.b_off);
  // decoder, finest level first
  for (int l = 0; l <= L - 2; ++l) {
    const int c = g->ch[l], cc = g->ch[l + 1];
    const int base = dec_base(g, l);
    const Layer& up = g->layers[base];
    const Layer& la = g->layers[base + 1];
    const Layer& lb = g->layers[base + 2];
    RB_TRY(conv3_wgrad(g, lb, g->dec_a[l], c, g->g_b[l], c, s));
    RB_TRY(conv3_dgrad(g, lb, g->g_b[l], c, g->dec_a[l], c, g->g_a[l], c, s));
    RB_TRY(conv3_wgrad(g, la, g->cat[l], 2 * c, g->g_a[l], c, s));
    RB_TRY(conv3_dgrad(g, la, g->g_a[l], c, nullptr, 0, g->g_cat[l], 2 * c, s));
    // transposed convolution: input gradient (masked by its input's ReLU) and weight gradient
    const bf16* upin = l == L - 2 ? g->bottom : g->dec_b[l + 1];
    bf16* gin = l == L - 2 ? g->g_bottom : g->g_b[l + 1];
    const size_t sm = (size_t)up.cout * 8 * up.cin * 2;
    k_up_dx<<<grid_for((int64_t)g->dims[l + 1].n() * (cc / 8)), 256, sm, s>>>(g->g_cat[l], 2 * c, c, up.wu, cc, upin,
                                                                                cc, g->dims[l], gin, cc);
    const UpDwPlan up_p = up_dw_plan(g, up);
    k_up_dw<<<dim3(up_p.splits, up_p.gy), up_p.tb * up_p.ln, 0, s>>>(upin, cc, cc, g->g_cat[l], 2 * c, c, g->dims[l],
                                                                    up_p.tb, up_p.ln, up_p.cells, g->wpart);
    const int n_out = 8 * cc * c + c;
    k_sum_parts<<<split_sum_blocks(n_out), split_sum_threads(up_p.splits), 0, s>>>(g->wpart, up_p.splits, n_out,
                                                                        g->grad + up.w_off);  // W then b, contiguous
    RB_CUDA(cudaGetLastError());
  }
  // encoder, bottom first
  for (int l = L - 1; l >= 0; --l) {
    const int c = g->ch[l];
    const Layer& la = g->layers[enc_idx(l, 0)];
    const Layer& lb = g->layers[enc_idx(l, 1)];
    bf16* geb = l == L - 1 ? g->g_bottom : g->g_eb[l];
    if (l < L - 1) {
      k_combine<<<grid_for((int64_t)g->dims[l].n() * (c / 8)), 256, 0, s>>>(g->g_cat[l] + c, 2 * c, g->g_pool[l + 1], c,
                                                                            g->cat[l] + c, 2 * c, g->dims[l], c, geb, c);
      RB_CUDA(cudaGetLastError());
    }
    RB_TRY(conv3_wgrad(g, lb, g->enc_a[l], c, geb, c, s));
    RB_TRY(conv3_dgrad(g, lb, geb, c, g->enc_a[l], c, g->g_ea[l], c, s));
    const bf16* in = l == 0 ? g->x0 : g->pooled[l - 1];
    const int ldin = l == 0 ? 8 : g->ch[l - 1];
    RB_TRY(conv3_wgrad(g, la, in, ldin, g->g_ea[l], c, s));
    if (l > 0) RB_TRY(conv3_dgrad(g, la, g->g_ea[l], c, nullptr, 0, g->g_pool[l], g->ch[l - 1], s));
  }
  return RB_OK;
}

rb_status guess_check(rb_guess* g, cudaStream_t s) {
  int h = 0;
  RB_CUDA(cudaMemcpyAsync(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  if (h) {
    RB_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    set_error("rb_guess: a tensor-core kernel gave up a bounded wait");
    return RB_ETIMEOUT;
  }
  return RB_OK;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_guess_param_count(const rb_guess_cfg* cfg, int64_t* n) {
  clear_error();
  RB_TRY(check_cfg(cfg));
  RB_REQUIRE(n != nullptr, "rb_guess_param_count: null output");
  std::vector<Layer> ls;
  build_layers(*cfg, ls, *n);
  return RB_OK;
}

extern "C" rb_status rb_guess_destroy(rb_guess_t g) {
  clear_error();
  if (!g) return RB_OK;
  for (void* p : g->allocs) cudaFree(p);
  delete g;
  return RB_OK;
}

extern "C" rb_status rb_guess_create(const rb_guess_cfg* cfg, rb_guess_t* out) {
  clear_error();
  RB_TRY(check_cfg(cfg));
  RB_REQUIRE(out != nullptr, "rb_guess_create: null output");
  *out = nullptr;
  rb_guess* g = new rb_guess();
  g->cfg = *cfg;
  g->L = cfg->levels;
  for (int l = 0; l < g->L; ++l) {
    g->ch.push_back(cfg->channels[l]);
    Dims d;
    d.nx = cfg->nx >> l;
    d.ny = cfg->ny >> l;
    d.nz = cfg->nz >> l;
    d.px = cfg->periodic[0] != 0;
    d.py = cfg->periodic[1] != 0;
    d.pz = cfg->periodic[2] != 0;
    g->dims.push_back(d);
  }
  build_layers(*cfg, g->layers, g->n_params);
  auto fail = [&](rb_status st) {
    const std::string msg = rb_last_error();
    rb_guess_destroy(g);
    set_error("%s", msg.c_str());
    return st;
  };
  for (const Layer& ly : g->layers) {
    if (ly.kind != kConv3) continue;
    if (conv_smem(ly.np, ly.kpad) > kMaxConvSmem || conv_smem(ly.npd, ly.kpadd) > kMaxConvSmem) {
      set_error("rb_guess_create: a %d -> %d convolution's weights exceed shared memory", ly.cin, ly.cout);
      return fail(RB_EINVAL);
    }
    if (ly.np > 64) {
      set_error("rb_guess_create: at most 64 output channels per convolution (got %d)", ly.cout);
      return fail(RB_EINVAL);
    }
  }
  for (const Layer& ly : g->layers)
    if (ly.kind == kUp && (size_t)8 * ly.cin * ly.cout * sizeof(bf16) > 48 * 1024) {
      set_error("rb_guess_create: a %d -> %d up-sampling's weights exceed 48 KB of shared memory", ly.cin, ly.cout);
      return fail(RB_EINVAL);
    }
  const int L = g->L;
  rb_status st = RB_OK;
  auto A = [&](auto** p, size_t count) {
    if (st == RB_OK) st = galloc(g, p, count);
  };
  A(&g->theta, g->n_params);
  A(&g->adam_m, g->n_params);
  A(&g->adam_v, g->n_params);
  A(&g->grad, g->n_params);
  const size_t n0 = g->dims[0].n();
  A(&g->x0, n0 * 8);
  g->enc_a.assign(L, nullptr);
  g->cat.assign(L, nullptr);
  g->pooled.assign(L, nullptr);
  g->dec_a.assign(L, nullptr);
  g->dec_b.assign(L, nullptr);
  g->g_b.assign(L, nullptr);
  g->g_a.assign(L, nullptr);
  g->g_cat.assign(L, nullptr);
  g->g_eb.assign(L, nullptr);
  g->g_ea.assign(L, nullptr);
  g->g_pool.assign(L, nullptr);
  for (int l = 0; l < L; ++l) {
    const size_t n = g->dims[l].n();
    const int c = g->ch[l];
    A(&g->enc_a[l], n * c);
    A(&g->g_ea[l], n * c);
    if (l > 0) A(&g->g_pool[l], n * g->ch[l - 1]);
    if (l < L - 1) {
      A(&g->cat[l], n * 2 * c);
      A(&g->pooled[l], (size_t)g->dims[l + 1].n() * c);
      A(&g->dec_a[l], n * c);
      A(&g->dec_b[l], n * c);
      A(&g->g_b[l], n * c);
      A(&g->g_a[l], n * c);
      A(&g->g_cat[l], n * 2 * c);
      A(&g->g_eb[l], n * c);
    } else {
      A(&g->bottom, n * c);
      A(&g->g_bottom, n * c);
    }
  }
  A(&g->y, n0);
  A(&g->gy, n0);
  A(&g->red, (size_t)kRedGrid * 64);
  A(&g->scal, 128);
  A(&g->sel, 4 * n0);
  A(&g->err, 1);
  for (Layer& ly : g->layers) {
    if (ly.kind == kConv3) {
      A(&ly.wf, (size_t)ly.np * ly.kpad);
      A(&ly.wd, (size_t)ly.npd * ly.kpadd);
      const Dims& d = g->dims[ly.level];
      if (row_kernel_fits(d, ly.cin_pad, ly.np)) A(&ly.wf_row, (size_t)ly.np * row_k(ly.cin_pad));
      if (ly.cin == ly.cin_pad && row_kernel_fits(d, ly.cout, ly.npd)) A(&ly.wd_row, (size_t)ly.npd * row_k(ly.cout));
      const int pwf = round_up(ly.cout, 16), pwd = round_up(ly.cin_pad, 16);
      if (slab_kernel_fits(d, ly.cin_pad, pwf)) {
        ly.pw_f = pwf;
        A(&ly.wf_slab, (size_t)3 * pwf * stack_k(ly.cin_pad));
      }
      if (ly.cin == ly.cin_pad && slab_kernel_fits(d, ly.cout, pwd)) {
        ly.pw_d = pwd;
        A(&ly.wd_slab, (size_t)3 * pwd * stack_k(ly.cout));
      }
    } else if (ly.kind == kUp) {
      A(&ly.wu, (size_t)8 * ly.cin * ly.cout);
    }
  }
  if (st == RB_OK) {
    g->wpart_floats = wpart_need(g);
    A(&g->wpart, g->wpart_floats);
  }
  if (st == RB_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = cuda_fail(e, "cudaDeviceSynchronize", __FILE__, __LINE__);
  }
  if (st != RB_OK) return fail(st);
  *out = g;
  return RB_OK;
}

extern "C" rb_status rb_guess_set_params(rb_guess_t g, const float* theta, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && theta, "rb_guess_set_params: null argument");
  cudaStream_t s = S(stream);
  RB_CUDA(cudaMemcpyAsync(g->theta, theta, g->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s));
  RB_CUDA(cudaMemsetAsync(g->adam_m, 0, g->n_params * sizeof(float), s));
  RB_CUDA(cudaMemsetAsync(g->adam_v, 0, g->n_params * sizeof(float), s));
  RB_CUDA(cudaMemsetAsync(g->grad, 0, g->n_params * sizeof(float), s));
  g->adam_t = 0;
  return refresh_weights(g, s);
}

__global__ void k_init_layer(const float* __restrict__ nrm, int64_t n_w, int64_t n_b, float scale,
                             float* __restrict__ th) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_w + n_b; i += (int64_t)gridDim.x * blockDim.x)
    th[i] = i < n_w ? nrm[i] * scale : 0.0f;
}

extern "C" rb_status rb_guess_init_params(rb_guess_t g, const float* normals, double head_scale, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && normals, "rb_guess_init_params: null argument");
  cudaStream_t s = S(stream);
  for (const Layer& ly : g->layers) {
    const int64_t n_w = ly.b_off - ly.w_off;
    const double fan = ly.kind == kConv3 ? 27.0 * ly.cin : (double)ly.cin;
    double scale = std::sqrt(2.0 / fan);
    if (ly.kind == kHead) scale *= head_scale;
    k_init_layer<<<grid_for(n_w + ly.cout), 256, 0, s>>>(normals + ly.w_off, n_w, ly.cout, (float)scale,
                                                         g->theta + ly.w_off);
  }
  RB_CUDA(cudaGetLastError());
  RB_CUDA(cudaMemsetAsync(g->adam_m, 0, g->n_params * sizeof(float), s));
  RB_CUDA(cudaMemsetAsync(g->adam_v, 0, g->n_params * sizeof(float), s));
  RB_CUDA(cudaMemsetAsync(g->grad, 0, g->n_params * sizeof(float), s));
  g->adam_t = 0;
  return refresh_weights(g, s);
}

extern "C" rb_status rb_guess_get_params(rb_guess_t g, float* theta, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && theta, "rb_guess_get_params: null argument");
  RB_CUDA(cudaMemcpyAsync(theta, g->theta, g->n_params * sizeof(float), cudaMemcpyDeviceToDevice, S(stream)));
  return RB_OK;
}

extern "C" rb_status rb_guess_get_grad(rb_guess_t g, float* grad, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && grad, "rb_guess_get_grad: null argument");
  RB_CUDA(cudaMemcpyAsync(grad, g->grad, g->n_params * sizeof(float), cudaMemcpyDeviceToDevice, S(stream)));
  return RB_OK;
}

extern "C" rb_status rb_guess_predict(rb_guess_t g, const double* b, const double* p1, const double* p2, double* p_out,
                                      rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && b && p1 && p2 && p_out, "rb_guess_predict: null argument");
  cudaStream_t s = S(stream);
  const int n0 = g->dims[0].n();
  RB_TRY(forward(g, b, p1, p2, s));
  k_sum1<<<kRedGrid, kRedThreads, 0, s>>>(p1, n0, g->red);
  k_finish<<<1, 256, 0, s>>>(g->red, kRedGrid, 1, g->scal + 3, 1.0 / n0);  // scal[3] = mean p1
  k_guess_out<<<grid_for(n0), 256, 0, s>>>(p1, g->y, n0, g->scal, g->scal + 2, p_out);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

__global__ void k_add_loss(const double* __restrict__ sum, double* __restrict__ dst) { *dst += *sum; }

extern "C" rb_status rb_guess_loss_grad(rb_guess_t g, const double* b, const double* p1, const double* p2,
                                        const double* p, int32_t accumulate, double* loss, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && b && p1 && p2 && p, "rb_guess_loss_grad: null argument");
  cudaStream_t s = S(stream);
  const int n0 = g->dims[0].n();
  if (!accumulate) RB_CUDA(cudaMemsetAsync(g->grad, 0, g->n_params * sizeof(float), s));
  RB_TRY(forward(g, b, p1, p2, s));
  k_sum_diff<<<kRedGrid, kRedThreads, 0, s>>>(p, p1, n0, g->red);
  k_finish<<<1, 256, 0, s>>>(g->red, kRedGrid, 1, g->scal + 4, 1.0 / n0);  // scal[4] = mean (p - p1)
  // k_loss reads means[0] = mean y (scal[2]) and means[2] = mean (p - p1) (scal[4])
  k_loss<<<kRedGrid, kRedThreads, 0, s>>>(p, p1, g->y, n0, g->scal, g->scal + 2, g->gy, g->red);
  k_finish<<<1, 256, 0, s>>>(g->red, kRedGrid, 1, g->scal + 6, 1.0 / n0);  // scal[6] = loss
  RB_CUDA(cudaGetLastError());
  if (loss) {
    k_add_loss<<<1, 1, 0, s>>>(g->scal + 6, loss);
    RB_CUDA(cudaGetLastError());
  }
  return backward(g, s);
}

extern "C" rb_status rb_guess_adam_step(rb_guess_t g, const rb_adam_params* h, double grad_scale, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && h, "rb_guess_adam_step: null argument");
  RB_REQUIRE(h->lr > 0 && h->beta1 >= 0 && h->beta1 < 1 && h->beta2 >= 0 && h->beta2 < 1 && h->eps > 0,
             "rb_guess_adam_step: invalid hyper-parameters");
  cudaStream_t s = S(stream);
  RB_TRY(guess_check(g, s));
  g->adam_t += 1;
  const double c1 = 1.0 / (1.0 - std::pow(h->beta1, (double)g->adam_t));
  const double c2 = 1.0 / (1.0 - std::pow(h->beta2, (double)g->adam_t));
  k_adam<<<grid_for(g->n_params), 256, 0, s>>>(g->theta, g->adam_m, g->adam_v, g->grad, g->n_params, (float)h->lr,
                                               (float)h->beta1, (float)h->beta2, (float)h->eps, (float)c1, (float)c2,
                                               (float)grad_scale);
  RB_CUDA(cudaGetLastError());
  return refresh_weights(g, s);
}

extern "C" rb_status rb_guess_read_activation(rb_guess_t g, int32_t index, float* out, int64_t* count,
                                              rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && count, "rb_guess_read_activation: null argument");
  RB_REQUIRE(index >= -1 && index < (int)g->layers.size(), "rb_guess_read_activation: index %d out of range", index);
  const int L = g->L;
  const bf16* src = nullptr;
  int ld = 0, c = 0, n = 0;
  if (index == -1) {
    src = g->x0, ld = 8, c = 3, n = g->dims[0].n();
  } else {
    const Layer& ly = g->layers[index];
    const int l = ly.level;
    n = g->dims[l].n();
    c = ly.cout;
    if (ly.kind == kHead) {
      *count = n;
      if (out) RB_CUDA(cudaMemcpyAsync(out, g->y, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, S(stream)));
      return RB_OK;
    }
    if (index < 2 * L) {
      if (index % 2 == 0) src = g->enc_a[l], ld = c;
      else if (l < L - 1) src = g->cat[l] + c, ld = 2 * c;
      else src = g->bottom, ld = c;
    } else {
      const int r = (index - 2 * L) % 3;
      if (r == 0) src = g->cat[l], ld = 2 * c;
      else if (r == 1) src = g->dec_a[l], ld = c;
      else src = g->dec_b[l], ld = c;
    }
  }
  *count = (int64_t)n * c;
  if (out) {
    k_bf16_to_f32<<<grid_for((int64_t)n * c), 256, 0, S(stream)>>>(src, ld, n, c, out);
    RB_CUDA(cudaGetLastError());
  }
  return RB_OK;
}

extern "C" rb_status rb_spmm(rb_op_t A, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t k, const double* c,
                             rb_stream_t stream);

// damped Jacobi sweep on two vectors: x_i += omega dinv (b - (A x)_i)
extern "C" rb_status rb_guess_select(rb_guess_t g, rb_op_t A, const double* b, const double* cand0,
                                     const double* cand1, int32_t sweeps, double omega, double* x0, double* res,
                                     int32_t* choice, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(g && A && b && cand0 && cand1 && x0 && res && choice, "rb_guess_select: null argument");
  const int n0 = g->dims[0].n();
  RB_REQUIRE(A->n_rows == n0 && A->n_cols == n0 && A->dtype == RB_F64,
             "rb_guess_select: A must be the FP64 %d x %d operator of the grid", n0, n0);
  RB_REQUIRE(sweeps >= 0 && sweeps <= 1000, "rb_guess_select: sweeps = %d outside [0, 1000]", sweeps);
  RB_REQUIRE(sweeps == 0 || (A->has_diag && A->dinv64), "rb_guess_select: smoothing needs A's diagonal");
  cudaStream_t s = S(stream);
  double* ax = g->sel;                   // [n][2]: A x_0, A x_1, interleaved
  double* xs = g->sel + 2 * (size_t)n0;  // [n][2]: the (smoothed) candidates, interleaved
  k_pack2<<<grid_for(n0), 256, 0, s>>>(cand0, cand1, n0, xs);
  RB_CUDA(cudaGetLastError());
  for (int it = 0; it <= sweeps; ++it) {
    RB_TRY(rb_spmm(A, xs, 2, ax, 2, 2, nullptr, stream));  // both candidates, one pass over A
    if (it < sweeps) {
      k_jacobi2<<<grid_for(n0), 256, 0, s>>>(b, ax, A->dinv64, omega, n0, xs);
      RB_CUDA(cudaGetLastError());
    }
  }
  k_resid2<<<kRedGrid, kRedThreads, 0, s>>>(b, ax, n0, g->red);
  k_finish<<<3, 256, 0, s>>>(g->red, kRedGrid, 3, g->scal + 16, 1.0);
  k_pick<<<grid_for(n0), 256, 0, s>>>(xs, n0, g->scal + 16, res, choice, x0);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}
