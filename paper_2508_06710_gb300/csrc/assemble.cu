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
#include <algorithm>

#include "common.cuh"

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

__device__ __forceinline__ double face_area(const GridDev& g, int dir, const int c[3]) {
  // product of the two transverse widths, in increasing axis order
  const int a = dir == 0 ? 1 : 0;
  const int b = dir == 2 ? 1 : 2;
  return width(g, a, c[a]) * width(g, b, c[b]);
}

template <int N>
__device__ __forceinline__ void sort_pairs(int64_t (&col)[N], double (&val)[N], int cnt) {
  for (int a = 1; a < cnt; ++a) {
    const int64_t kc = col[a];
    const double kv = val[a];
    int b = a - 1;
    while (b >= 0 && col[b] > kc) {
      col[b + 1] = col[b];
      val[b + 1] = val[b];
      --b;
    }
    col[b + 1] = kc;
    val[b + 1] = kv;
  }
}

__global__ void k_laplacian(GridDev g, double scale, int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                            double* __restrict__ va, int64_t n, int64_t nnz) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id == 0) rp[n] = (int32_t)nnz;
  if (id >= n) return;
  const int i = (int)(id % g.n[0]);
  const int j = (int)((id / g.n[0]) % g.n[1]);
  const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
  const int c[3] = {i, j, k};
  const int64_t start = 7 * id - walls_before(g, i, j, k);
  int64_t col[7];
  double val[7];
  int cnt = 0;
  double diag = 0.0;
  const int64_t stride[3] = {1, g.n[0], (int64_t)g.n[0] * g.n[1]};
  for (int d = 0; d < 3; ++d) {
    const double A = face_area(g, d, c);
    const int t = c[d];
    // minus neighbour across the face at position t
    if (g.per[d] || t > 0) {
      const int tn = (t == 0) ? g.n[d] - 1 : t - 1;
      const double cf = A / centre_dist(g, d, t);
      col[cnt] = id + (int64_t)(tn - t) * stride[d];
      val[cnt++] = cf;
      diag += cf;
    }
    // plus neighbour across the face at position t + 1
    if (g.per[d] || t < g.n[d] - 1) {
      const int tp = (t == g.n[d] - 1) ? 0 : t + 1;
      const double cf = A / centre_dist(g, d, tp);
      col[cnt] = id + (int64_t)(tp - t) * stride[d];
      val[cnt++] = cf;
      diag += cf;
    }
  }
  col[cnt] = id;
  val[cnt++] = -diag;
  sort_pairs<7>(col, val, cnt);
  rp[id] = (int32_t)start;
  for (int e = 0; e < cnt; ++e) {
    ci[start + e] = (int32_t)col[e];
    va[start + e] = scale * val[e];
  }
}

__global__ void k_divergence(GridDev g, double scale, int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                             double* __restrict__ va, int64_t n, int64_t nnz) {
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id == 0) rp[n] = (int32_t)nnz;
  if (id >= n) return;
  const int i = (int)(id % g.n[0]);
  const int j = (int)((id / g.n[0]) % g.n[1]);
  const int k = (int)(id / ((int64_t)g.n[0] * g.n[1]));
  const int c[3] = {i, j, k};
  const int64_t start = 6 * id - walls_before(g, i, j, k);
  int64_t col[6];
  double val[6];
  int cnt = 0;
  for (int d = 0; d < 3; ++d) {
    const double A = face_area(g, d, c);
    const int t = c[d];
    if (g.per[d] || t > 0) {  // minus face: this cell lies above it
      col[cnt] = face_index(g, d, c, t);
      val[cnt++] = -A;
    }
    if (g.per[d] || t < g.n[d] - 1) {  // plus face: this cell lies below it
      const int tp = (t == g.n[d] - 1) ? 0 : t + 1;
      col[cnt] = face_index(g, d, c, tp);
      val[cnt++] = A;
    }
  }
  sort_pairs<6>(col, val, cnt);
  rp[id] = (int32_t)start;
  for (int e = 0; e < cnt; ++e) {
    ci[start + e] = (int32_t)col[e];
    va[start + e] = scale * val[e];
  }
}

__global__ void k_gradient(GridDev g, double scale, int32_t* __restrict__ rp, int32_t* __restrict__ ci,
                           double* __restrict__ va, int64_t nf) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f == 0) rp[nf] = (int32_t)(2 * nf);
  if (f >= nf) return;
  int dir = 0;
  int64_t local = f;
  for (; dir < 2; ++dir) {
    const int64_t cnt = (int64_t)face_dim(g, dir, 0) * face_dim(g, dir, 1) * face_dim(g, dir, 2);
    if (local < cnt) break;
    local -= cnt;
  }
  const int fx = face_dim(g, dir, 0), fy = face_dim(g, dir, 1);
  int c[3];
  c[0] = (int)(local % fx);
  c[1] = (int)((local / fx) % fy);
  c[2] = (int)(local / ((int64_t)fx * fy));
  const int p = g.per[dir] ? c[dir] : c[dir] + 1;  // face position along dir
  const int lo = (p == 0) ? g.n[dir] - 1 : p - 1;
  int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
  cm[dir] = lo;
  cp[dir] = p;
  const int64_t idm = cm[0] + (int64_t)g.n[0] * (cm[1] + (int64_t)g.n[1] * cm[2]);
  const int64_t idp = cp[0] + (int64_t)g.n[0] * (cp[1] + (int64_t)g.n[1] * cp[2]);
  const double inv = 1.0 / centre_dist(g, dir, p);
  const int64_t s = 2 * f;
  rp[f] = (int32_t)s;
  if (idm < idp) {
    ci[s] = (int32_t)idm, va[s] = -scale * inv;
    ci[s + 1] = (int32_t)idp, va[s + 1] = scale * inv;
  } else {
    ci[s] = (int32_t)idp, va[s] = scale * inv;
    ci[s + 1] = (int32_t)idm, va[s + 1] = -scale * inv;
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
  const int bs = 256;
  switch (kind) {
    case RB_FVM_LAPLACIAN:
      k_laplacian<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(g, scale, row_ptr, col_idx, vals, n, 7 * n - walls);
      break;
    case RB_FVM_DIVERGENCE:
      k_divergence<<<(unsigned)((n + bs - 1) / bs), bs, 0, s>>>(g, scale, row_ptr, col_idx, vals, n, 6 * n - walls);
      break;
    case RB_FVM_GRADIENT:
      k_gradient<<<(unsigned)((nf + bs - 1) / bs), bs, 0, s>>>(g, scale, row_ptr, col_idx, vals, nf);
      break;
    default: set_error("rb_fvm_assemble: unknown kind %d", (int)kind); return RB_EINVAL;
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
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
