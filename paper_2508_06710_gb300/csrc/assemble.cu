// Operator build on the device.
//
// (1) Staggered symmetry-preserving FVM operators on a Cartesian grid (Sec. 3, semi-discrete
//     equations (ns); Sec. 4): the divergence M (faces -> cells), the gradient
//     G = -Omega_s^{-1} M^T (cells -> faces) and the Laplacian L = M G, written straight
//     into CSR by one thread per row.  Each face contributes A_f / d_f to L, with A_f the
//     product of the two transverse cell widths and d_f the distance between the adjacent
//     cell centres; faces on walls are excluded.  Row pointers follow in closed form from
//     the number of wall faces met before each row, so no scan is needed.
// (2) The cotangent-weight Laplacian of a triangle mesh (the unstructured operator of the
//     extruded-airfoil case, Sec. 4.3): one thread per triangle adds the half cotangent of
//     each angle to the weight of the opposite edge (at most two contributions per edge,
//     whose sum does not depend on their order), then one thread per row clamps negative
//     weights and forms the diagonal.
// (3) The coarse-to-fine maps of inline mesh refinement (Sec. 3.3): prolongation P (fine cells
//     x coarse cells) and restriction R (coarse x fine) between a grid and its 2:1 coarsening
//     (every other node), 8 entries per row in both, so again no scan.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "stencil7.cuh"

namespace rb {
namespace {

struct GridDev {
  int n[3];
  int per[3];
  const double* nodes[3];
};

__device__ __forceinline__ double width(const GridDev& g, int d, int t) { return g.nodes[d][t + 1] - g.nodes[d][t]; }

// distance between the centres of cells t-1 (periodic wrap) and t along axis d
__device__ __forceinline__ double centre_dist(const GridDev& g, int d, int t) {
  const int lo = (t == 0) ? g.n[d] - 1 : t - 1;
  return 0.5 * (width(g, d, lo) + width(g, d, t));
}

// Cell widths and reciprocal centre distances along each axis, as the row kernels read them:
// either computed where needed (GeomDirect) or from tables that each block builds once in
// shared memory (GeomTab: 2 (nx + ny + nz) doubles), which takes the FP64 divisions (a few
// dozen FP64-pipe instructions each, six per Laplacian row) out of the per-row work.  A face
// coefficient is A_f * (1 / d_f) in both (one rounding more than A_f / d_f; both neighbours of
// a face compute it from the same operands, so L stays exactly symmetric).
struct GeomDirect {
  const GridDev* g;
  double s;  // scale of icd: the operator's scale for L and G (folded in), 1 for M
  __device__ double w(int d, int t) const { return width(*g, d, t); }
  __device__ double icd(int d, int t) const { return s / centre_dist(*g, d, t); }
};
struct GeomTab {
  const double* wt[3];
  const double* it[3];
  __device__ double w(int d, int t) const { return wt[d][t]; }
  __device__ double icd(int d, int t) const { return it[d][t]; }
};

inline size_t geom_tab_bytes(const GridDev& g) { return 16 * (size_t)(g.n[0] + g.n[1] + g.n[2]); }
constexpr size_t kGeomTabMax = 48 * 1024;

// whole block: the tables in shared memory (icd scaled by s)
__device__ GeomTab build_geom_tab(const GridDev& g, double* smem, double s) {
  GeomTab t;
  double* p = smem;
  for (int d = 0; d < 3; ++d) {
    t.wt[d] = p;
    p += g.n[d];
  }
  for (int d = 0; d < 3; ++d) {
    t.it[d] = p;
    p += g.n[d];
  }
  for (int d = 0; d < 3; ++d)
    for (int i = threadIdx.x; i < g.n[d]; i += blockDim.x) {
      const_cast<double*>(t.wt[d])[i] = width(g, d, i);
      const_cast<double*>(t.it[d])[i] = s / centre_dist(g, d, i);
    }
  __syncthreads();
  return t;
}

// number of (cell, wall face) incidences over the cells before `id` (lexicographic, x fastest)
__device__ __forceinline__ int64_t walls_before(const GridDev& g, int i, int j, int k) {
  const int64_t Nx = g.n[0], Ny = g.n[1], Nz = g.n[2];
  int64_t w = 0;
  if (!g.per[0]) w += 2 * ((int64_t)j + Ny * k) + (i > 0 ? 1 : 0);
  if (!g.per[1]) w += 2 * Nx * k + (j > 0 ? Nx : 0) + ((j == 0 || j == Ny - 1) ? i : 0);
  if (!g.per[2]) w += (k > 0 ? Nx * Ny : 0) + ((k == 0 || k == Nz - 1) ? (int64_t)i + Nx * j : 0);
  return w;
}

__device__ __forceinline__ int face_dim(const GridDev& g, int dir, int axis) {
  return (axis == dir && !g.per[axis]) ? g.n[axis] - 1 : g.n[axis];
}

__device__ __forceinline__ int64_t face_offset(const GridDev& g, int dir) {
  int64_t off = 0;
  for (int d = 0; d < dir; ++d) off += (int64_t)face_dim(g, d, 0) * face_dim(g, d, 1) * face_dim(g, d, 2);
  return off;
}

// index of the face of direction `dir` at position p along dir (0..n-1 periodic, 1..n-1 walls)
// and transverse cell coordinates c[]
__device__ __forceinline__ int64_t face_index(const GridDev& g, int dir, const int c[3], int p) {
  int f[3] = {c[0], c[1], c[2]};
  f[dir] = g.per[dir] ? p : p - 1;
  return face_offset(g, dir) + f[0] + (int64_t)face_dim(g, dir, 0) * (f[1] + (int64_t)face_dim(g, dir, 1) * f[2]);
}

// product of the two transverse widths, in increasing axis order
template <class Geom>
__device__ __forceinline__ double face_area(const Geom& G, int dir, const int c[3]) {
  const int a = dir == 0 ? 1 : 0;
  const int b = dir == 2 ? 1 : 2;
  return G.w(a, c[a]) * G.w(b, c[b]);
}

// Sorts a row's (column, value) pairs by column with a fixed compare-exchange network
// (every index known at compile time, so the arrays stay in registers); absent entries carry
// the column INT64_MAX and sort to the end.  Odd-even transposition: N rounds.
template <int N>
__device__ __forceinline__ void sort_pairs(int64_t (&col)[N], double (&val)[N]) {
#pragma unroll
  for (int r = 0; r < N; ++r) {
#pragma unroll
    for (int a = r & 1; a + 1 < N; a += 2) {
      const bool sw = col[a] > col[a + 1];
      const int64_t c0 = sw ? col[a + 1] : col[a], c1 = sw ? col[a] : col[a + 1];
      const double v0 = sw ? val[a + 1] : val[a], v1 = sw ? val[a] : val[a + 1];
      col[a] = c0, col[a + 1] = c1, val[a] = v0, val[a + 1] = v1;
    }
  }
}

// cell coordinates of row id (n < 2^31: 32-bit division)
__device__ __forceinline__ void cell_of(const GridDev& g, int64_t id, int (&c)[3]) {
  const unsigned u = (unsigned)id, nx = (unsigned)g.n[0], ny = (unsigned)g.n[1];
  const unsigned q = u / nx;
  c[0] = (int)(u - q * nx);
  c[1] = (int)(q % ny);
  c[2] = (int)(q / ny);
}

// The row writers store the row's entries at ci[start - obase ..], va[start - obase ..]: the
// global arrays (obase 0) or a block's staging buffer in shared memory (obase = the first
// entry of the block's rows).
template <class Geom>
__device__ __forceinline__ void laplacian_row(const GridDev& g, const Geom& G, double scale, int32_t* __restrict__ rp,
                                              int32_t* __restrict__ ci, double* __restrict__ va, int64_t id,
                                              int64_t obase = 0) {
  int c[3];
  cell_of(g, id, c);
  const int64_t start = 7 * id - walls_before(g, c[0], c[1], c[2]);
  int64_t col[7];
  double val[7];
  int cnt = 1;
  double diag = 0.0;
  const int64_t stride[3] = {1, g.n[0], (int64_t)g.n[0] * g.n[1]};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double A = face_area(G, d, c);
    const int t = c[d];
    // minus neighbour across the face at position t (slot 2d), plus neighbour across the face
    // at position t + 1 (slot 2d + 1); a wall leaves its slot absent
    const bool has_m = g.per[d] || t > 0, has_p = g.per[d] || t < g.n[d] - 1;
    const int tn = (t == 0) ? g.n[d] - 1 : t - 1;
    const int tp = (t == g.n[d] - 1) ? 0 : t + 1;
    const double cm = has_m ? A * G.icd(d, t) : 0.0;
    const double cp = has_p ? A * G.icd(d, tp) : 0.0;
    col[2 * d] = has_m ? id + (int64_t)(tn - t) * stride[d] : INT64_MAX;
    val[2 * d] = cm;
    col[2 * d + 1] = has_p ? id + (int64_t)(tp - t) * stride[d] : INT64_MAX;
    val[2 * d + 1] = cp;
    diag += cm;
    diag += cp;
    cnt += (int)has_m + (int)has_p;
  }
  col[6] = id;
  val[6] = -diag;
  sort_pairs<7>(col, val);
  rp[id] = (int32_t)start;
#pragma unroll
  for (int e = 0; e < 7; ++e)
    if (e < cnt) {
      ci[start - obase + e] = (int32_t)col[e];
      va[start - obase + e] = val[e];  // the scale is in G.icd
    }
}

// HALF: the face-to-cell interpolator (1/2 on each face of the cell) instead of +-A_f
template <class Geom, bool HALF = false>
__device__ __forceinline__ void divergence_row(const GridDev& g, const Geom& G, double scale, int32_t* __restrict__ rp,
                                               int32_t* __restrict__ ci, double* __restrict__ va, int64_t id,
                                               int64_t obase = 0) {
  int c[3];
  cell_of(g, id, c);
  const int64_t start = 6 * id - walls_before(g, c[0], c[1], c[2]);
  int64_t col[6];
  double val[6];
  int cnt = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double A = face_area(G, d, c);
    const int t = c[d];
    // minus face (this cell lies above it) in slot 2d, plus face (below it) in slot 2d + 1
    const bool has_m = g.per[d] || t > 0, has_p = g.per[d] || t < g.n[d] - 1;
    const int tp = (t == g.n[d] - 1) ? 0 : t + 1;
    col[2 * d] = has_m ? face_index(g, d, c, t) : INT64_MAX;
    val[2 * d] = HALF ? 0.5 : -A;
    col[2 * d + 1] = has_p ? face_index(g, d, c, tp) : INT64_MAX;
    val[2 * d + 1] = HALF ? 0.5 : A;
    cnt += (int)has_m + (int)has_p;
  }
  sort_pairs<6>(col, val);
  rp[id] = (int32_t)start;
#pragma unroll
  for (int e = 0; e < 6; ++e)
    if (e < cnt) {
      ci[start - obase + e] = (int32_t)col[e];
      va[start - obase + e] = scale * val[e];
    }
}

// the face's two cells for a compile-time direction (every index a constant: no local arrays);
// HALF: the cell-to-face interpolator (1/2 on both cells) instead of -+1/d_f
template <int DIR, bool HALF, class Geom>
__device__ __forceinline__ void gradient_face(const GridDev& g, const Geom& G, double scale, int32_t* __restrict__ rp,
                                              int32_t* __restrict__ ci, double* __restrict__ va, int64_t f,
                                              int64_t local) {
  const unsigned fx = (unsigned)face_dim(g, DIR, 0), fy = (unsigned)face_dim(g, DIR, 1);
  const unsigned u = (unsigned)local, q = u / fx;
  int c[3];
  c[0] = (int)(u - q * fx);
  c[1] = (int)(q % fy);
  c[2] = (int)(q / fy);
  const int p = g.per[DIR] ? c[DIR] : c[DIR] + 1;  // face position along DIR
  const int lo = (p == 0) ? g.n[DIR] - 1 : p - 1;
  const int64_t sx = 1, sy = g.n[0], sz = (int64_t)g.n[0] * g.n[1];
  const int64_t base = c[0] * sx + c[1] * sy + c[2] * sz - (int64_t)c[DIR] * (DIR == 0 ? sx : DIR == 1 ? sy : sz);
  const int64_t sd = DIR == 0 ? sx : DIR == 1 ? sy : sz;
  const int64_t idm = base + lo * sd, idp = base + p * sd;
  const double inv = HALF ? 0.5 * scale : G.icd(DIR, p);  // scale / d_f
  const double vm = HALF ? inv : -inv;
  const int64_t s = 2 * f;
  rp[f] = (int32_t)s;
  if (idm < idp) {
    ci[s] = (int32_t)idm, va[s] = vm;
    ci[s + 1] = (int32_t)idp, va[s + 1] = inv;
  } else {
    ci[s] = (int32_t)idp, va[s] = inv;
    ci[s + 1] = (int32_t)idm, va[s + 1] = vm;
  }
}

template <class Geom, bool HALF = false>
__device__ __forceinline__ void gradient_row(const GridDev& g, const Geom& G, double scale, int32_t* __restrict__ rp,
                                             int32_t* __restrict__ ci, double* __restrict__ va, int64_t f) {
  const int64_t n0 = (int64_t)face_dim(g, 0, 0) * face_dim(g, 0, 1) * face_dim(g, 0, 2);
  const int64_t n1 = (int64_t)face_dim(g, 1, 0) * face_dim(g, 1, 1) * face_dim(g, 1, 2);
  if (f < n0) gradient_face<0, HALF>(g, G, scale, rp, ci, va, f, f);
  else if (f < n0 + n1) gradient_face<1, HALF>(g, G, scale, rp, ci, va, f, f - n0);
  else gradient_face<2, HALF>(g, G, scale, rp, ci, va, f, f - n0 - n1);
}

// FK_C2S has the gradient's pattern and FK_S2C the divergence's, with 1/2 for every entry
enum FvmKernelKind { FK_LAP = 0, FK_DIV = 1, FK_GRAD = 2, FK_C2S = 3, FK_S2C = 4 };

constexpr int kFvmThreads = 256;

// first CSR entry of row r < rows of the Laplacian (7 per cell) or the divergence (6 per cell)
template <int KIND>
__device__ __forceinline__ int64_t row_start(const GridDev& g, int64_t r) {
  constexpr int per = KIND == FK_LAP ? 7 : 6;
  int c[3];
  cell_of(g, r, c);
  return per * r - walls_before(g, c[0], c[1], c[2]);
}

// One thread per row, grid-stride over tiles of 256 rows.  With TAB the block first builds
// the axis tables; for the Laplacian and the divergence it also stages each tile's entries
// (one contiguous range of the CSR arrays) in shared memory and writes them out coalesced,
// instead of each thread storing its row's 6-7 entries with a stride across the warp.
template <int KIND, bool TAB>
__global__ void __launch_bounds__(kFvmThreads) k_fvm(GridDev g, double scale, int32_t* __restrict__ rp,
                                                     int32_t* __restrict__ ci, double* __restrict__ va, int64_t rows,
                                                     int64_t nnz) {
  extern __shared__ double geom_smem[];
  if (blockIdx.x == 0 && threadIdx.x == 0) rp[rows] = (int32_t)nnz;
  constexpr bool kStage = TAB && KIND != FK_GRAD && KIND != FK_C2S;
  constexpr int kPer = KIND == FK_LAP ? 7 : 6;
  auto body = [&](const auto& G, double* s_va, int32_t* s_ci) {
    for (int64_t r0 = (int64_t)blockIdx.x * kFvmThreads; r0 < rows; r0 += (int64_t)gridDim.x * kFvmThreads) {
      const int64_t id = r0 + threadIdx.x;
      if constexpr (kStage) {
        const int64_t base = row_start<KIND>(g, r0);
        const int64_t end = r0 + kFvmThreads >= rows ? nnz : row_start<KIND>(g, r0 + kFvmThreads);
        if (id < rows) {
          if constexpr (KIND == FK_LAP) laplacian_row(g, G, scale, rp, s_ci, s_va, id, base);
          else divergence_row<std::decay_t<decltype(G)>, KIND == FK_S2C>(g, G, scale, rp, s_ci, s_va, id, base);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < (int)(end - base); e += kFvmThreads) {
          ci[base + e] = s_ci[e];
          va[base + e] = s_va[e];
        }
        __syncthreads();
      } else if (id < rows) {
        if constexpr (KIND == FK_LAP) laplacian_row(g, G, scale, rp, ci, va, id);
        else if constexpr (KIND == FK_DIV || KIND == FK_S2C)
          divergence_row<std::decay_t<decltype(G)>, KIND == FK_S2C>(g, G, scale, rp, ci, va, id);
        else gradient_row<std::decay_t<decltype(G)>, KIND == FK_C2S>(g, G, scale, rp, ci, va, id);
      }
    }
  };
  // L and G take the scale into their reciprocal distances; M and the interpolators multiply
  // their entries by it
  const double icd_scale = (KIND == FK_LAP || KIND == FK_GRAD) ? scale : 1.0;
  if constexpr (TAB) {
    const GeomTab G = build_geom_tab(g, geom_smem, icd_scale);
    double* s_va = geom_smem + 2 * (g.n[0] + g.n[1] + g.n[2]);
    int32_t* s_ci = reinterpret_cast<int32_t*>(s_va + kPer * kFvmThreads);
    body(G, s_va, s_ci);
  } else {
    GeomDirect G{&g, icd_scale};
    body(G, nullptr, nullptr);
  }
}

// ---------------------------------------------------------------------------- triangle mesh

__device__ __forceinline__ int find_col(const int32_t* ci, int lo, int hi, int c) {
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (ci[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double cot_at(double ax, double ay, double bx, double by, double cx, double cy) {
  const double ux = bx - ax, uy = by - ay, vx = cx - ax, vy = cy - ay;
  return (ux * vx + uy * vy) / fabs(ux * vy - uy * vx);
}

__global__ void k_cot_triangles(int n_tri, int n_vert, const double* __restrict__ P, const int32_t* __restrict__ tri,
                                const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                double* __restrict__ va, double* __restrict__ area, int32_t* __restrict__ bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tri) return;
  const int v[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
  for (int a = 0; a < 3; ++a)
    if (v[a] < 0 || v[a] >= n_vert) {
      atomicExch(bad, 3);
      return;
    }
  double x[3], y[3];
  for (int a = 0; a < 3; ++a) x[a] = P[2 * v[a]], y[a] = P[2 * v[a] + 1];
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    // half cotangent of the angle at vertex a weights the opposite edge (b, c)
    const double w = 0.5 * cot_at(x[a], y[a], x[b], y[b], x[c], y[c]);
    const int pb = find_col(ci, rp[v[b]], rp[v[b] + 1], v[c]);
    const int pc = find_col(ci, rp[v[c]], rp[v[c] + 1], v[b]);
    if (pb >= rp[v[b] + 1] || ci[pb] != v[c] || pc >= rp[v[c] + 1] || ci[pc] != v[b]) {
      atomicExch(bad, 1);
      continue;
    }
    atomicAdd(va + pb, w);
    atomicAdd(va + pc, w);
  }
  if (area) {
    const double ar = 0.5 * fabs((x[1] - x[0]) * (y[2] - y[0]) - (y[1] - y[0]) * (x[2] - x[0]));
    for (int a = 0; a < 3; ++a) atomicAdd(area + v[a], ar / 3.0);
  }
}

__global__ void k_cot_rows(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           double* __restrict__ va, unsigned long long* __restrict__ clamped,
                           int32_t* __restrict__ bad) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = 0.0;
  int dpos = -1;
  unsigned long long nc = 0;
  for (int p = rp[r]; p < rp[r + 1]; ++p) {
    const int c = ci[p];
    if (c == r) {
      dpos = p;
      continue;
    }
    double w = va[p];
    if (w < 0.0) {
      if (c > r) ++nc;  // count each undirected edge once
      w = 0.0;
      va[p] = 0.0;
    }
    s += w;
  }
  if (dpos < 0) {
    atomicExch(bad, 2);
    return;
  }
  va[dpos] = -s;
  if (nc && clamped) atomicAdd(clamped, nc);
}

rb_status grid_from_desc(const rb_grid_desc* gd, GridDev& g) {
  RB_REQUIRE(gd != nullptr, "fvm: null grid");
  for (int d = 0; d < 3; ++d) {
    g.n[d] = gd->n[d];
    g.per[d] = gd->periodic[d] ? 1 : 0;
    g.nodes[d] = gd->nodes[d];
    RB_REQUIRE(g.n[d] >= (g.per[d] ? 3 : 2), "fvm: axis %d has %d cells (need >= %d)", d, g.n[d], g.per[d] ? 3 : 2);
  }
  const int64_t n = (int64_t)g.n[0] * g.n[1] * g.n[2];
  RB_REQUIRE(7 * n < INT32_MAX, "fvm: grid too large for int32 CSR indexing");
  return RB_OK;
}

void sizes(const GridDev& g, int64_t& n, int64_t& nf, int64_t& walls) {
  n = (int64_t)g.n[0] * g.n[1] * g.n[2];
  nf = 0;
  walls = 0;
  for (int d = 0; d < 3; ++d) {
    nf += g.per[d] ? n : n / g.n[d] * (g.n[d] - 1);
    if (!g.per[d]) walls += 2 * (n / g.n[d]);
  }
}

// Tables in shared memory when the three axes fit (2 (nx + ny + nz) doubles within 48 KB),
// then a grid of a few resident waves, each block building its tables once; else the direct
// form, one block per 256 rows.
template <int KIND>
rb_status launch_fvm(const GridDev& g, double scale, int32_t* rp, int32_t* ci, double* va, int64_t rows, int64_t nnz,
                     cudaStream_t s) {
  const int bs = kFvmThreads;
  const int64_t blocks = (rows + bs - 1) / bs;
  const size_t stage = (KIND == FK_GRAD || KIND == FK_C2S) ? 0 : (size_t)(KIND == FK_LAP ? 7 : 6) * bs * (8 + 4);
  const size_t smem = geom_tab_bytes(g) + stage;
  if (smem <= kGeomTabMax) {
    auto* kern = &k_fvm<KIND, true>;
    const int grid = wave_grid(kern, blocks, smem, bs);
    kern<<<grid, bs, smem, s>>>(g, scale, rp, ci, va, rows, nnz);
  } else {
    k_fvm<KIND, false><<<(unsigned)std::max<int64_t>(1, blocks), bs, 0, s>>>(g, scale, rp, ci, va, rows, nnz);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// ------------------------------------------------------------------------------------------
// Inline mesh refinement maps.  The coarse grid is the fine one with every other node, so
// coarse cell I along an axis is fine cells 2I and 2I + 1 and its centre is the midpoint of
// fine nodes 2I and 2I + 2.
// ------------------------------------------------------------------------------------------
constexpr int kMapThreads = 128;

// Along axis d: the two coarse cells whose centres interpolate fine cell t (left child: the
// parent and its left neighbour; right child: the parent and its right neighbour; across a
// periodic seam the neighbour's centre shifted by the period; at a wall the two cells next to
// it, extrapolating), returned sorted by index with their linear weights.
__device__ __forceinline__ void prolong_axis(const GridDev& g, int d, int t, int (&c)[2], double (&w)[2]) {
  const double* x = g.nodes[d];
  const int nf = g.n[d], nc = nf / 2, parent = t >> 1;
  int lo = (t & 1) ? parent : parent - 1;
  int hi = lo + 1;
  const double period = x[nf] - x[0];
  double shift_lo = 0.0, shift_hi = 0.0;
  if (lo < 0) {
    if (g.per[d]) lo = nc - 1, shift_lo = -period;
    else lo = 0, hi = 1;
  }
  if (hi >= nc) {
    if (g.per[d]) hi = 0, shift_hi = period;
    else lo = nc - 2, hi = nc - 1;
  }
  double x_lo = 0.5 * (x[2 * lo] + x[2 * lo + 2]);
  double x_hi = 0.5 * (x[2 * hi] + x[2 * hi + 2]);
  if (shift_lo != 0.0) x_lo = x_lo + shift_lo;
  if (shift_hi != 0.0) x_hi = x_hi + shift_hi;
  const double xf = 0.5 * (x[t] + x[t + 1]);
  const double w_hi = (xf - x_lo) / (x_hi - x_lo);
  const double w_lo = (x_hi - xf) / (x_hi - x_lo);
  const bool sw = lo > hi;  // the seam puts the neighbour's index on the other side
  c[0] = sw ? hi : lo, c[1] = sw ? lo : hi;
  w[0] = sw ? w_hi : w_lo, w[1] = sw ? w_lo : w_hi;
}

// The two coarse cells and weights of one axis position: P's (fine position t) or R's (coarse
// position p: the children 2p, 2p + 1 and their widths over the parent's).
struct AxisMap {
  int c[2];
  double w[2];
};

template <bool RESTRICT>
__device__ __forceinline__ AxisMap axis_map(const GridDev& g, int d, int t) {
  AxisMap m;
  if constexpr (RESTRICT) {
    const double* x = g.nodes[d];
    const double wc = x[2 * t + 2] - x[2 * t];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      m.c[a] = 2 * t + a;
      m.w[a] = (x[2 * t + a + 1] - x[2 * t + a]) / wc;
    }
  } else {
    prolong_axis(g, d, t, m.c, m.w);
  }
  return m;
}

// Axis positions per row: P's rows run over fine positions, R's over coarse ones.
template <bool RESTRICT>
__host__ __device__ inline int map_len(const GridDev& g, int d) { return RESTRICT ? g.n[d] / 2 : g.n[d]; }

// Per-axis tables (AxisMap for every position of the three axes) in shared memory, 24 bytes
// per position, when they fit in this budget; the weights then cost each block its share of
// (nx + ny + nz) divisions pairs instead of six FP64 divisions per row.
constexpr size_t kMapTabMax = 32 * 1024;

// RESTRICT = false: P's rows (one per fine cell); true: R's rows (one per coarse cell, the
// children in index order).  TAB: a persistent grid whose blocks build the axis tables once
// and stride over 128-row tiles; else one tile per block with the weights computed per row.
// Each tile is staged in shared memory and written out by consecutive threads.
template <bool RESTRICT, bool TAB>
__global__ void __launch_bounds__(kMapThreads) k_refine_map(GridDev g, int32_t* __restrict__ rp,
                                                            int32_t* __restrict__ ci, double* __restrict__ va) {
  __shared__ double s_val[kMapThreads * 8];
  __shared__ int32_t s_col[kMapThreads * 8];
  extern __shared__ AxisMap s_tab[];
  const int l0 = map_len<RESTRICT>(g, 0), l1 = map_len<RESTRICT>(g, 1), l2 = map_len<RESTRICT>(g, 2);
  if constexpr (TAB) {
    for (int t = threadIdx.x; t < l0 + l1 + l2; t += kMapThreads) {
      const int d = t < l0 ? 0 : (t < l0 + l1 ? 1 : 2);
      const int q = t - (d == 0 ? 0 : (d == 1 ? l0 : l0 + l1));
      // the axis as a compile-time index, so that the grid stays in registers
      s_tab[t] = d == 0 ? axis_map<RESTRICT>(g, 0, q) : (d == 1 ? axis_map<RESTRICT>(g, 1, q) : axis_map<RESTRICT>(g, 2, q));
    }
    __syncthreads();
  }
  const int ncx = g.n[0] / 2, ncy = g.n[1] / 2;
  const int rows = l0 * l1 * l2;
  const int sx = RESTRICT ? g.n[0] : ncx, sy = RESTRICT ? g.n[1] : ncy;  // column grid
  const int stride = TAB ? gridDim.x * kMapThreads : rows;
  for (int r0 = blockIdx.x * kMapThreads; r0 < rows; r0 += stride) {
    const int nr = min(kMapThreads, rows - r0);
    const int r = r0 + threadIdx.x;
    if (threadIdx.x < nr) {
      const int i = r % l0, q = r / l0, j = q % l1, k = q / l1;
      AxisMap m[3];
      if constexpr (TAB) {
        m[0] = s_tab[i], m[1] = s_tab[l0 + j], m[2] = s_tab[l0 + l1 + k];
      } else {
        m[0] = axis_map<RESTRICT>(g, 0, i), m[1] = axis_map<RESTRICT>(g, 1, j), m[2] = axis_map<RESTRICT>(g, 2, k);
      }
      int e = threadIdx.x * 8;
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc, ++e) {
            s_col[e] = m[0].c[cc] + sx * (m[1].c[b] + sy * m[2].c[a]);
            s_val[e] = m[2].w[a] * (m[1].w[b] * m[0].w[cc]);
          }
      rp[r] = 8 * r;
      if (r == rows - 1) rp[rows] = 8 * rows;
    }
    __syncthreads();
    const int64_t base = 8 * (int64_t)r0;
    for (int e = threadIdx.x; e < nr * 8; e += kMapThreads) {
      ci[base + e] = s_col[e];
      va[base + e] = s_val[e];
    }
    __syncthreads();  // the staging buffers are refilled by the next tile
  }
}

template <bool RESTRICT>
rb_status launch_refine_map(const GridDev& g, int32_t* rp, int32_t* ci, double* va, cudaStream_t s) {
  const int64_t rows = (int64_t)map_len<RESTRICT>(g, 0) * map_len<RESTRICT>(g, 1) * map_len<RESTRICT>(g, 2);
  const int64_t tiles = (rows + kMapThreads - 1) / kMapThreads;
  const size_t tab = sizeof(AxisMap) * (size_t)(map_len<RESTRICT>(g, 0) + map_len<RESTRICT>(g, 1) + map_len<RESTRICT>(g, 2));
  if (tab <= kMapTabMax) {
    auto* kern = &k_refine_map<RESTRICT, true>;
    kern<<<wave_grid(kern, tiles, tab, kMapThreads), kMapThreads, tab, s>>>(g, rp, ci, va);
  } else {
    k_refine_map<RESTRICT, false><<<(unsigned)tiles, kMapThreads, 0, s>>>(g, rp, ci, va);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// P^T (N_c x N), the restriction of the multigrid cycle: row I of the 1-D transpose along an
// axis lists the fine positions t whose interpolation uses coarse cell I (two to five of them:
// 2I - 1 .. 2I + 2 inside, wrapped at a periodic seam, one more next to a wall where P
// extrapolates), sorted, with P's weights.  P = P_z (x) P_y (x) P_x, so P^T's row (I, J, K) is
// the product of the three 1-D rows: cx[I] cy[J] cz[K] entries, columns sorted when z runs
// outermost, and its offset has a closed form in the per-axis prefix sums of the counts.
struct TAxis {
  int cnt, pre;  // entries of this 1-D row, entries of the rows before it on the axis
  int t[8];
  double w[8];
};

__device__ void prolong_t_axis(const GridDev& g, int d, int I, TAxis& r) {
  const int nf = g.n[d];
  r.cnt = 0;
  for (int o = -3; o <= 4; ++o) {
    int t = 2 * I + o;
    if (g.per[d]) t = ((t % nf) + nf) % nf;
    else if (t < 0 || t >= nf) continue;
    bool seen = false;
    for (int q = 0; q < r.cnt; ++q) seen |= r.t[q] == t;
    if (seen) continue;
    int c[2];
    double w[2];
    prolong_axis(g, d, t, c, w);
    if (c[0] == I || c[1] == I) {
      r.t[r.cnt] = t;
      r.w[r.cnt] = c[0] == I ? w[0] : w[1];
      ++r.cnt;
    }
  }
  for (int q = 1; q < r.cnt; ++q)  // insertion sort by fine position
    for (int u = q; u > 0 && r.t[u - 1] > r.t[u]; --u) {
      const int tt = r.t[u];
      r.t[u] = r.t[u - 1], r.t[u - 1] = tt;
      const double ww = r.w[u];
      r.w[u] = r.w[u - 1], r.w[u - 1] = ww;
    }
}

constexpr size_t kProlongTTabMax = 200 * 1024;

__global__ void __launch_bounds__(kMapThreads) k_prolong_t(GridDev g, int32_t* __restrict__ rp,
                                                           int32_t* __restrict__ ci, double* __restrict__ va) {
  extern __shared__ TAxis s_ax[];
  const int ncx = g.n[0] / 2, ncy = g.n[1] / 2, ncz = g.n[2] / 2;
  for (int p = threadIdx.x; p < ncx + ncy + ncz; p += kMapThreads) {
    const int d = p < ncx ? 0 : (p < ncx + ncy ? 1 : 2);
    prolong_t_axis(g, d, p - (d == 0 ? 0 : (d == 1 ? ncx : ncx + ncy)), s_ax[p]);
  }
  __syncthreads();
  if (threadIdx.x < 3) {  // exclusive prefix of the counts along each axis
    const int d = threadIdx.x;
    const int b = d == 0 ? 0 : (d == 1 ? ncx : ncx + ncy), len = d == 0 ? ncx : (d == 1 ? ncy : ncz);
    int acc = 0;
    for (int q = 0; q < len; ++q) {
      s_ax[b + q].pre = acc;
      acc += s_ax[b + q].cnt;
    }
  }
  __syncthreads();
  const TAxis* ax = s_ax;
  const TAxis* ay = s_ax + ncx;
  const TAxis* az = s_ax + ncx + ncy;
  const int64_t sx = 2 * (int64_t)g.n[0], sy = 2 * (int64_t)g.n[1];  // entries per axis (each t in two rows)
  const int64_t rows = (int64_t)ncx * ncy * ncz;
  const int nfx = g.n[0], nfy = g.n[1];
  for (int64_t r = (int64_t)blockIdx.x * kMapThreads + threadIdx.x; r < rows; r += (int64_t)gridDim.x * kMapThreads) {
    const int I = (int)(r % ncx), J = (int)((r / ncx) % ncy), Kz = (int)(r / ((int64_t)ncx * ncy));
    const TAxis &X = ax[I], &Y = ay[J], &Z = az[Kz];
    int64_t e = (int64_t)Z.pre * sy * sx + (int64_t)Z.cnt * ((int64_t)Y.pre * sx + (int64_t)Y.cnt * X.pre);
    rp[r] = (int32_t)e;
    if (r == rows - 1) rp[rows] = (int32_t)(e + (int64_t)X.cnt * Y.cnt * Z.cnt);
    for (int a = 0; a < Z.cnt; ++a)
      for (int b = 0; b < Y.cnt; ++b)
        for (int c = 0; c < X.cnt; ++c, ++e) {
          ci[e] = X.t[c] + nfx * (Y.t[b] + nfy * Z.t[a]);
          va[e] = Z.w[a] * (Y.w[b] * X.w[c]);  // the product in P's order: bit-identical entries
        }
  }
}

rb_status launch_prolong_t(const GridDev& g, int32_t* rp, int32_t* ci, double* va, cudaStream_t s) {
  const size_t tab = sizeof(TAxis) * (size_t)(g.n[0] / 2 + g.n[1] / 2 + g.n[2] / 2);
  RB_REQUIRE(tab <= kProlongTTabMax, "rb_refine_assemble: P^T needs %zu bytes of axis tables (limit %zu)", tab,
             kProlongTTabMax);
  RB_TRY(opt_in_smem(reinterpret_cast<const void*>(&k_prolong_t), tab));
  const int64_t rows = (int64_t)(g.n[0] / 2) * (g.n[1] / 2) * (g.n[2] / 2);
  const int64_t tiles = (rows + kMapThreads - 1) / kMapThreads;
  k_prolong_t<<<wave_grid(&k_prolong_t, tiles, tab, kMapThreads), kMapThreads, tab, s>>>(g, rp, ci, va);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// Per-axis tables of the matrix-free operators (stencil7.cuh): cell widths and inverse centre
// distances of each axis (the Laplacian), and the 1-D prolongation and its transpose (the
// transfers), in FP64 and rounded to FP32.
__global__ void k_stencil7_axis(GridDev g, int d, double* __restrict__ w64, double* __restrict__ ic64,
                                float* __restrict__ w32, float* __restrict__ ic32) {
  const int n = g.n[d];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n; t += gridDim.x * blockDim.x) {
    if (t < n) {
      const double w = width(g, d, t);
      w64[t] = w;
      w32[t] = (float)w;
    }
    double ic = 0.0;
    if (g.per[d]) ic = 1.0 / centre_dist(g, d, t == n ? 0 : t);
    else if (t > 0 && t < n) ic = 1.0 / centre_dist(g, d, t);
    ic64[t] = ic;
    ic32[t] = (float)ic;
  }
}

__global__ void k_transfer_axis(GridDev g, int d, PAxis<double>* __restrict__ pa64, TAxisTab<double>* __restrict__ ta64,
                                PAxis<float>* __restrict__ pa32, TAxisTab<float>* __restrict__ ta32) {
  const int nf = g.n[d], nc = nf / 2;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nf + nc; t += gridDim.x * blockDim.x) {
    if (t < nf) {
      int c[2];
      double w[2];
      prolong_axis(g, d, t, c, w);
      pa64[t] = PAxis<double>{c[0], c[1], w[0], w[1]};
      pa32[t] = PAxis<float>{c[0], c[1], (float)w[0], (float)w[1]};
    } else {
      const int I = t - nf;
      TAxis r;
      prolong_t_axis(g, d, I, r);
      TAxisTab<double> a{};
      TAxisTab<float> b{};
      a.cnt = b.cnt = r.cnt;
      for (int q = 0; q < r.cnt; ++q) {
        a.t[q] = b.t[q] = r.t[q];
        a.w[q] = r.w[q];
        b.w[q] = (float)r.w[q];
      }
      ta64[I] = a;
      ta32[I] = b;
    }
  }
}

}  // namespace

rb_status stencil7_tables(const rb_grid_desc* grid, double* w64[3], double* ic64[3], float* w32[3], float* ic32[3],
                          cudaStream_t s) {
  GridDev g;
  RB_TRY(grid_from_desc(grid, g));
  for (int d = 0; d < 3; ++d) {
    k_stencil7_axis<<<(g.n[d] + 1 + 127) / 128, 128, 0, s>>>(g, d, w64[d], ic64[d], w32[d], ic32[d]);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

rb_status transfer_tables(const rb_grid_desc* fine, PAxis<double>* pa64[3], TAxisTab<double>* ta64[3],
                          PAxis<float>* pa32[3], TAxisTab<float>* ta32[3], cudaStream_t s) {
  GridDev g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = fine->n[d];
    g.per[d] = fine->periodic[d] ? 1 : 0;
    g.nodes[d] = fine->nodes[d];
    RB_REQUIRE(g.n[d] >= 4 && g.n[d] % 2 == 0, "transfer tables: axis %d has %d cells (need an even number >= 4)", d,
               g.n[d]);
  }
  for (int d = 0; d < 3; ++d) {
    const int m = g.n[d] + g.n[d] / 2;
    k_transfer_axis<<<(m + 127) / 128, 128, 0, s>>>(g, d, pa64[d], ta64[d], pa32[d], ta32[d]);
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

namespace {
}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_fvm_csr_size(const rb_grid_desc* grid, rb_fvm_kind kind, int32_t* n_rows, int32_t* n_cols,
                                     int64_t* nnz) {
  clear_error();
  GridDev g;
  RB_TRY(grid_from_desc(grid, g));
  RB_REQUIRE(n_rows && n_cols && nnz, "rb_fvm_csr_size: null output");
  int64_t n, nf, walls;
  sizes(g, n, nf, walls);
  switch (kind) {
    case RB_FVM_LAPLACIAN: *n_rows = (int32_t)n, *n_cols = (int32_t)n, *nnz = 7 * n - walls; break;
    case RB_FVM_DIVERGENCE: *n_rows = (int32_t)n, *n_cols = (int32_t)nf, *nnz = 6 * n - walls; break;
    case RB_FVM_GRADIENT: *n_rows = (int32_t)nf, *n_cols = (int32_t)n, *nnz = 2 * nf; break;
    case RB_FVM_INTERP_C2S: *n_rows = (int32_t)nf, *n_cols = (int32_t)n, *nnz = 2 * nf; break;
    case RB_FVM_INTERP_S2C: *n_rows = (int32_t)n, *n_cols = (int32_t)nf, *nnz = 6 * n - walls; break;
    default: set_error("rb_fvm_csr_size: unknown kind %d", (int)kind); return RB_EINVAL;
  }
  return RB_OK;
}

extern "C" rb_status rb_fvm_assemble(const rb_grid_desc* grid, rb_fvm_kind kind, double scale, int32_t* row_ptr,
                                     int32_t* col_idx, double* vals, rb_stream_t stream) {
  clear_error();
  GridDev g;
  RB_TRY(grid_from_desc(grid, g));
  RB_REQUIRE(row_ptr && col_idx && vals, "rb_fvm_assemble: null output array");
  for (int d = 0; d < 3; ++d) RB_REQUIRE(g.nodes[d] != nullptr, "rb_fvm_assemble: null nodes[%d]", d);
  int64_t n, nf, walls;
  sizes(g, n, nf, walls);
  cudaStream_t s = S(stream);
  switch (kind) {
    case RB_FVM_LAPLACIAN: return launch_fvm<FK_LAP>(g, scale, row_ptr, col_idx, vals, n, 7 * n - walls, s);
    case RB_FVM_DIVERGENCE: return launch_fvm<FK_DIV>(g, scale, row_ptr, col_idx, vals, n, 6 * n - walls, s);
    case RB_FVM_GRADIENT: return launch_fvm<FK_GRAD>(g, scale, row_ptr, col_idx, vals, nf, 2 * nf, s);
    case RB_FVM_INTERP_C2S: return launch_fvm<FK_C2S>(g, scale, row_ptr, col_idx, vals, nf, 2 * nf, s);
    case RB_FVM_INTERP_S2C: return launch_fvm<FK_S2C>(g, scale, row_ptr, col_idx, vals, n, 6 * n - walls, s);
    default: set_error("rb_fvm_assemble: unknown kind %d", (int)kind); return RB_EINVAL;
  }
}

extern "C" rb_status rb_mesh_cot_laplacian(int32_t n_vert, const double* points, int32_t n_tri,
                                           const int32_t* triangles, const int32_t* row_ptr, const int32_t* col_idx,
                                           int64_t nnz, double* vals, double* area, int64_t* n_clamped,
                                           rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(n_vert >= 0 && n_tri >= 0 && nnz >= 0, "rb_mesh_cot_laplacian: negative size");
  RB_REQUIRE(n_vert == 0 || (points && row_ptr && col_idx && vals), "rb_mesh_cot_laplacian: null array");
  RB_REQUIRE(n_tri == 0 || triangles, "rb_mesh_cot_laplacian: null triangles");
  if (n_vert == 0) return RB_OK;
  cudaStream_t s = S(stream);
  // status words in the caller's device array: [0] clamped edges, [1] pattern error flag
  RB_REQUIRE(n_clamped != nullptr, "rb_mesh_cot_laplacian: n_clamped (device int64[2]) is required");
  RB_CUDA(cudaMemsetAsync(vals, 0, (size_t)nnz * sizeof(double), s));
  if (area) RB_CUDA(cudaMemsetAsync(area, 0, (size_t)n_vert * sizeof(double), s));
  RB_CUDA(cudaMemsetAsync(n_clamped, 0, 2 * sizeof(int64_t), s));
  unsigned long long* cl = reinterpret_cast<unsigned long long*>(n_clamped);
  int32_t* bad = reinterpret_cast<int32_t*>(n_clamped + 1);
  if (n_tri > 0)
    k_cot_triangles<<<(n_tri + 255) / 256, 256, 0, s>>>(n_tri, n_vert, points, triangles, row_ptr, col_idx, vals, area, bad);
  k_cot_rows<<<(n_vert + 255) / 256, 256, 0, s>>>(n_vert, row_ptr, col_idx, vals, cl, bad);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

extern "C" rb_status rb_refine_assemble(const rb_grid_desc* fine, rb_refine_kind kind, int32_t* row_ptr,
                                        int32_t* col_idx, double* vals, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(fine != nullptr, "rb_refine_assemble: null grid");
  RB_REQUIRE(kind == RB_REFINE_PROLONG || kind == RB_REFINE_RESTRICT || kind == RB_REFINE_PROLONG_T,
             "rb_refine_assemble: unknown kind %d", (int)kind);
  GridDev g;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = fine->n[d];
    g.per[d] = fine->periodic[d] ? 1 : 0;
    g.nodes[d] = fine->nodes[d];
    RB_REQUIRE(g.n[d] >= 4 && g.n[d] % 2 == 0, "rb_refine_assemble: axis %d has %d cells (need an even number >= 4)",
               d, g.n[d]);
    RB_REQUIRE(g.nodes[d] != nullptr, "rb_refine_assemble: null nodes[%d]", d);
  }
  const int64_t n_fine = (int64_t)g.n[0] * g.n[1] * g.n[2];
  RB_REQUIRE(8 * n_fine <= INT32_MAX, "rb_refine_assemble: grid too large for int32 CSR indexing");
  RB_REQUIRE(row_ptr && col_idx && vals, "rb_refine_assemble: null output array");
  cudaStream_t s = S(stream);
  if (kind == RB_REFINE_PROLONG) return launch_refine_map<false>(g, row_ptr, col_idx, vals, s);
  if (kind == RB_REFINE_PROLONG_T) return launch_prolong_t(g, row_ptr, col_idx, vals, s);
  return launch_refine_map<true>(g, row_ptr, col_idx, vals, s);
}
