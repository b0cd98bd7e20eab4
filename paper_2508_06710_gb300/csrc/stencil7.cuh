// Matrix-free operators of Cartesian FVM grids: the 7-point Laplacian and the refinement
// transfers applied from per-axis tables instead of stored entries.
//
// The repeated-block structure of Sec. 2 reads each matrix entry once for all k columns; on a
// Cartesian grid the entries themselves repeat: every coefficient of the symmetry-preserving
// Laplacian (Sec. 3, Eq. (ns); L = M G) is a product of one-dimensional quantities,
//   across the x face between cells (i-1, j, k) and (i, j, k):  w_y[j] w_z[k] / d_x[i],
// w the cell widths and d the distances between neighbouring cell centres (wrapped on a
// periodic axis), and likewise for y and z; the diagonal is minus the sum of the six.  So the
// operator is the grid's 2 (n_x + n_y + n_z) + 3 numbers, and an SpMM with it reads only X
// and writes only Y (the "stencil descriptor" form: no index or value streams at all).  The
// trilinear prolongation P of the refinement maps and its transpose are products of per-axis
// 1-D maps in the same way.
//
// Tables (device arrays, in the operator's type T):
//   w[d][t]   width of cell t along axis d, t < n[d]
//   ic[d][f]  1 / d_f for face f = 0 .. n[d] of axis d (face f between cells f - 1 and f),
//             0 on the wall faces f = 0 and f = n[d] of a bounded axis (excluded faces: the
//             homogeneous Neumann condition); on a periodic axis face n[d] is face 0
#pragma once

#include <cstring>

#include "common.cuh"

namespace rb {

// Unsigned 32-bit division by a divisor fixed for a whole launch, as one multiply-high, an add
// and two shifts: Granlund and Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), the round-up method for N = 32: with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0),
// t = floor(m n / 2^32).  Exact for every n < 2^32 and 1 <= d < 2^31.  The rows of the grids
// here are below 2^31, so (i, j, k) come from two of these instead of 64-bit divisions.
struct FastDiv {
  uint32_t m = 0;
  int s1 = 0, s2 = 0;
  __host__ void init(uint32_t d) {
    int l = 0;
    while ((uint64_t)1 << l < d) ++l;
    m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    const uint32_t t = __umulhi(m, n);
    return (t + ((n - t) >> s1)) >> s2;
  }
};

template <typename T>
struct Stencil7 {
  int n[3];
  int per[3];
  const T* w[3];
  const T* ic[3];
  T scale;          // the operator is scale * L
  FastDiv dx, dxy;  // division by n[0] and by n[0] n[1]
  __host__ void init_div() {
    dx.init((uint32_t)n[0]);
    dxy.init((uint32_t)n[0] * (uint32_t)n[1]);
  }
};

// The row's cell (i, j, k), its six face coefficients of L and the diagonal -sum of them
template <typename T>
struct Coef7 {
  int i, j, k;
  T cxm, cxp, cym, cyp, czm, czp, diag;
};

template <typename T>
__device__ __forceinline__ Coef7<T> stencil7_coef(const Stencil7<T>& s, int64_t row) {
  Coef7<T> c;
  const uint32_t r32 = (uint32_t)row;
  c.k = (int)s.dxy.div(r32);
  const uint32_t rem = r32 - (uint32_t)c.k * (uint32_t)(s.n[0] * s.n[1]);
  c.j = (int)s.dx.div(rem);
  c.i = (int)(rem - (uint32_t)c.j * (uint32_t)s.n[0]);
  const T wx = __ldg(s.w[0] + c.i), wy = __ldg(s.w[1] + c.j), wz = __ldg(s.w[2] + c.k);
  const T ayz = wy * wz, axz = wx * wz, axy = wx * wy;
  c.cxm = ayz * __ldg(s.ic[0] + c.i), c.cxp = ayz * __ldg(s.ic[0] + c.i + 1);
  c.cym = axz * __ldg(s.ic[1] + c.j), c.cyp = axz * __ldg(s.ic[1] + c.j + 1);
  c.czm = axy * __ldg(s.ic[2] + c.k), c.czp = axy * __ldg(s.ic[2] + c.k + 1);
  c.diag = -(((c.cxm + c.cxp) + (c.cym + c.cyp)) + (c.czm + c.czp));
  return c;
}

// (A X)[row, col0 .. col0 + VEC) into acc, and the inverse diagonal of A into dinv.
// COHERENT: X read through L2 only (X written by other blocks of the same launch).
template <typename T, int VEC, bool COHERENT = false>
__device__ __forceinline__ void stencil7_apply(const Stencil7<T>& s, const T* __restrict__ X, int64_t ldx, int64_t row,
                                               int col0, T (&acc)[VEC], T& dinv) {
  const Coef7<T> cf = stencil7_coef(s, row);
  const int i = cf.i, j = cf.j, k = cf.k;
  const int nx = s.n[0], ny = s.n[1];
  const int64_t plane = (int64_t)nx * ny;
  const T cxm = cf.cxm, cxp = cf.cxp, cym = cf.cym, cyp = cf.cyp, czm = cf.czm, czp = cf.czp, diag = cf.diag;
  dinv = T(1) / (s.scale * diag);
  // neighbour rows (a wall neighbour has coefficient 0: any valid row will do, take this one)
  const int im = i > 0 ? i - 1 : (s.per[0] ? nx - 1 : i), ip = i + 1 < nx ? i + 1 : (s.per[0] ? 0 : i);
  const int jm = j > 0 ? j - 1 : (s.per[1] ? ny - 1 : j), jp = j + 1 < ny ? j + 1 : (s.per[1] ? 0 : j);
  const int nz = s.n[2];
  const int km = k > 0 ? k - 1 : (s.per[2] ? nz - 1 : k), kp = k + 1 < nz ? k + 1 : (s.per[2] ? 0 : k);
  const T* xc = X + col0;
  auto ld = [&](int64_t r) { return COHERENT ? ldv_cg<T, VEC>(xc + r * ldx) : ldv<T, VEC>(xc + r * ldx); };
  const Vec<T, VEC> x0 = ld(row);
  const Vec<T, VEC> a = ld(row - i + im);
  const Vec<T, VEC> b = ld(row - i + ip);
  const Vec<T, VEC> c = ld(row + (int64_t)(jm - j) * nx);
  const Vec<T, VEC> d = ld(row + (int64_t)(jp - j) * nx);
  const Vec<T, VEC> e = ld(row + (int64_t)(km - k) * plane);
  const Vec<T, VEC> f = ld(row + (int64_t)(kp - k) * plane);
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    T y = diag * x0.v[q];
    y = fma(cxm, a.v[q], y);
    y = fma(cxp, b.v[q], y);
    y = fma(cym, c.v[q], y);
    y = fma(cyp, d.v[q], y);
    y = fma(czm, e.v[q], y);
    y = fma(czp, f.v[q], y);
    acc[q] = s.scale * y;
  }
}

// A run of RUN consecutive cells along x (n_x a multiple of RUN): the row split, the y and z
// factors and the neighbour base addresses are formed once per run, and the x neighbours inside
// the run come from registers.  CONTIG: X rows hold exactly the k = VEC columns (ld = VEC,
// 16-byte aligned bases), so a run of RUN * VEC values moves as 16-byte vectors.
template <typename T, int VEC, int RUN, bool CONTIG>
__device__ __forceinline__ void load_run(const T* __restrict__ p, int64_t ldx, Vec<T, VEC> (&v)[RUN]) {
  if constexpr (CONTIG && (sizeof(T) * VEC * RUN) % 16 == 0) {
    constexpr int NV = sizeof(T) * VEC * RUN / 16;
    T buf[VEC * RUN];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
      memcpy(reinterpret_cast<char*>(buf) + 16 * q, &f, 16);
    }
#pragma unroll
    for (int c = 0; c < RUN; ++c)
#pragma unroll
      for (int q = 0; q < VEC; ++q) v[c].v[q] = buf[c * VEC + q];
  } else {
#pragma unroll
    for (int c = 0; c < RUN; ++c) v[c] = ldv<T, VEC>(p + (int64_t)c * ldx);
  }
}

template <typename T, int VEC, int RUN, bool CONTIG>
__device__ __forceinline__ void store_run(T* __restrict__ p, int64_t ldy, const Vec<T, VEC> (&y)[RUN]) {
  if constexpr (CONTIG && (sizeof(T) * VEC * RUN) % 16 == 0) {
    constexpr int NV = sizeof(T) * VEC * RUN / 16;
    T buf[VEC * RUN];
#pragma unroll
    for (int c = 0; c < RUN; ++c)
#pragma unroll
      for (int q = 0; q < VEC; ++q) buf[c * VEC + q] = y[c].v[q];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      float4 f;
      memcpy(&f, reinterpret_cast<char*>(buf) + 16 * q, 16);
      reinterpret_cast<float4*>(p)[q] = f;
    }
  } else {
#pragma unroll
    for (int c = 0; c < RUN; ++c) stv<T, VEC>(p + (int64_t)c * ldy, y[c]);
  }
}

// (A X) for the RUN cells of run u (u = i0 / RUN + (n_x / RUN)(j + n_y k); drun divides by
// n_x / RUN, drow by n_y), columns xc .. xc + VEC: the centre values into x0, the products into
// y; returns the run's first row
template <typename T, int VEC, int RUN, bool CONTIG>
__device__ __forceinline__ int64_t stencil7_apply_run(const Stencil7<T>& st, const FastDiv& drun, const FastDiv& drow,
                                                      int64_t u, const T* __restrict__ xc, int64_t ldx,
                                                      Vec<T, VEC> (&x0)[RUN], Vec<T, VEC> (&y)[RUN]) {
  const int nx = st.n[0], ny = st.n[1], nz = st.n[2];
  const uint32_t runs_x = (uint32_t)(nx / RUN);
  const uint32_t line = drun.div((uint32_t)u);  // j + ny k
  const int i0 = (int)((uint32_t)u - line * runs_x) * RUN;
  const int kz = (int)drow.div(line);
  const int j = (int)(line - (uint32_t)kz * (uint32_t)ny);
  const int64_t row0 = (int64_t)line * nx + i0;
  const T wy = __ldg(st.w[1] + j), wz = __ldg(st.w[2] + kz);
  const T ayz = wy * wz;
  const T icym = __ldg(st.ic[1] + j), icyp = __ldg(st.ic[1] + j + 1);
  const T iczm = __ldg(st.ic[2] + kz), iczp = __ldg(st.ic[2] + kz + 1);
  const int jm = j > 0 ? j - 1 : (st.per[1] ? ny - 1 : j), jp = j + 1 < ny ? j + 1 : (st.per[1] ? 0 : j);
  const int km = kz > 0 ? kz - 1 : (st.per[2] ? nz - 1 : kz), kp2 = kz + 1 < nz ? kz + 1 : (st.per[2] ? 0 : kz);
  const int64_t plane = (int64_t)nx * ny;
  Vec<T, VEC> ym[RUN], yp[RUN], zm[RUN], zp[RUN];
  load_run<T, VEC, RUN, CONTIG>(xc + row0 * ldx, ldx, x0);
  load_run<T, VEC, RUN, CONTIG>(xc + (row0 + (int64_t)(jm - j) * nx) * ldx, ldx, ym);
  load_run<T, VEC, RUN, CONTIG>(xc + (row0 + (int64_t)(jp - j) * nx) * ldx, ldx, yp);
  load_run<T, VEC, RUN, CONTIG>(xc + (row0 + (int64_t)(km - kz) * plane) * ldx, ldx, zm);
  load_run<T, VEC, RUN, CONTIG>(xc + (row0 + (int64_t)(kp2 - kz) * plane) * ldx, ldx, zp);
  // x neighbours of the run's ends (wrapped on a periodic axis; at a wall the coefficient is 0)
  const int il = i0 > 0 ? i0 - 1 : (st.per[0] ? nx - 1 : i0);
  const int ir = i0 + RUN < nx ? i0 + RUN : (st.per[0] ? 0 : i0 + RUN - 1);
  const Vec<T, VEC> xl = ldv<T, VEC>(xc + (row0 - i0 + il) * ldx);
  const Vec<T, VEC> xr = ldv<T, VEC>(xc + (row0 - i0 + ir) * ldx);
  T icx[RUN + 1], wx[RUN];
#pragma unroll
  for (int c = 0; c <= RUN; ++c) icx[c] = __ldg(st.ic[0] + i0 + c);
#pragma unroll
  for (int c = 0; c < RUN; ++c) wx[c] = __ldg(st.w[0] + i0 + c);
#pragma unroll
  for (int c = 0; c < RUN; ++c) {
    const T cxm = ayz * icx[c], cxp = ayz * icx[c + 1];
    const T axz = wx[c] * wz, axy = wx[c] * wy;
    const T cym = axz * icym, cyp = axz * icyp, czm = axy * iczm, czp = axy * iczp;
    const T diag = -(((cxm + cxp) + (cym + cyp)) + (czm + czp));
    const Vec<T, VEC>& left = c == 0 ? xl : x0[c > 0 ? c - 1 : 0];
    const Vec<T, VEC>& right = c == RUN - 1 ? xr : x0[c < RUN - 1 ? c + 1 : 0];
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      T a = diag * x0[c].v[q];
      a = fma(cxm, left.v[q], a);
      a = fma(cxp, right.v[q], a);
      a = fma(cym, ym[c].v[q], a);
      a = fma(cyp, yp[c].v[q], a);
      a = fma(czm, zm[c].v[q], a);
      a = fma(czp, zp[c].v[q], a);
      y[c].v[q] = st.scale * a;
    }
  }
  return row0;
}

// ----------------------------------------------------------------------------- transfers

// The 1-D prolongation of one fine position: the two coarse positions and their weights
template <typename T>
struct PAxis {
  int c0, c1;
  T w0, w1;
};

// The 1-D transpose of one coarse position: the fine positions that use it (at most 8) and
// their weights, sorted by position
template <typename T>
struct TAxisTab {
  int cnt;
  int t[8];
  T w[8];
};

template <typename T>
struct Transfer3 {
  int nf[3];               // fine cells per axis (coarse: nf / 2)
  const PAxis<T>* pa[3];   // per fine position
  const TAxisTab<T>* ta[3];  // per coarse position
  FastDiv fx, fxy, cx, cxy;  // division by the fine and the coarse row lengths and planes
  __host__ void init_div() {
    fx.init((uint32_t)nf[0]);
    fxy.init((uint32_t)nf[0] * (uint32_t)nf[1]);
    cx.init((uint32_t)(nf[0] / 2));
    cxy.init((uint32_t)(nf[0] / 2) * (uint32_t)(nf[1] / 2));
  }
};

// (P E_c)[fine row, col0 .. col0 + VEC): trilinear interpolation from the coarse block
template <typename T, int VEC>
__device__ __forceinline__ void prolong_apply(const Transfer3<T>& tr, const T* __restrict__ Ec, int k, int64_t row,
                                              int col0, T (&acc)[VEC]) {
  const int nx = tr.nf[0], ny = tr.nf[1];
  const uint32_t r32 = (uint32_t)row;
  const int kk = (int)tr.fxy.div(r32);
  const uint32_t rem = r32 - (uint32_t)kk * (uint32_t)(nx * ny);
  const int j = (int)tr.fx.div(rem);
  const int i = (int)(rem - (uint32_t)j * (uint32_t)nx);
  const PAxis<T> px = tr.pa[0][i], py = tr.pa[1][j], pz = tr.pa[2][kk];
  const int cnx = nx / 2, cny = ny / 2;
  const int cx[2] = {px.c0, px.c1}, cy[2] = {py.c0, py.c1}, cz[2] = {pz.c0, pz.c1};
  const T wx[2] = {px.w0, px.w1}, wy[2] = {py.w0, py.w1}, wz[2] = {pz.w0, pz.w1};
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[q] = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T wab = wz[a] * wy[b];
      const int64_t base = (int64_t)cnx * (cy[b] + (int64_t)cny * cz[a]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const T wt = wab * wx[c];
        const Vec<T, VEC> v = ldv<T, VEC>(Ec + (base + cx[c]) * k + col0);
#pragma unroll
        for (int q = 0; q < VEC; ++q) acc[q] = fma(wt, v.v[q], acc[q]);
      }
    }
}

// (P^T R_f)[coarse row, col0 .. col0 + VEC): the weighted sum over the fine cells whose
// interpolation uses this coarse cell
template <typename T, int VEC>
__device__ __forceinline__ void restrict_apply(const Transfer3<T>& tr, const T* __restrict__ Rf, int k, int64_t row,
                                               int col0, T (&acc)[VEC]) {
  const int cnx = tr.nf[0] / 2, cny = tr.nf[1] / 2;
  const uint32_t r32 = (uint32_t)row;
  const int K3 = (int)tr.cxy.div(r32);
  const uint32_t rem = r32 - (uint32_t)K3 * (uint32_t)(cnx * cny);
  const int J = (int)tr.cx.div(rem);
  const int I = (int)(rem - (uint32_t)J * (uint32_t)cnx);
  const TAxisTab<T>& tx = tr.ta[0][I];
  const TAxisTab<T>& ty = tr.ta[1][J];
  const TAxisTab<T>& tz = tr.ta[2][K3];
  const int nx = tr.nf[0], ny = tr.nf[1];
#pragma unroll
  for (int q = 0; q < VEC; ++q) acc[q] = T(0);
  // the x list in registers (fixed bound, guarded), y and z lists from the cached table
  const int ncx = tx.cnt, ncy = ty.cnt, ncz = tz.cnt;
  int xt[8];
  T xw[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    xt[c] = c < ncx ? tx.t[c] : 0;
    xw[c] = c < ncx ? tx.w[c] : T(0);
  }
  // y positions four at a time (a coarse cell has at most 4 of them away from a wall): the
  // gathers of four fine rows are in flight together, not one row's after another's
  for (int a = 0; a < ncz; ++a) {
    const T wa = tz.w[a];
    const int64_t za = (int64_t)ny * tz.t[a];
    for (int b0 = 0; b0 < ncy; b0 += 4) {
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) {
        const int b = b0 + bb;
        if (b < ncy) {
          const T wab = wa * ty.w[b];
          const T* base = Rf + (int64_t)nx * (ty.t[b] + za) * k + col0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (c < ncx) {
              const Vec<T, VEC> v = ldv<T, VEC>(base + (int64_t)xt[c] * k);
              const T wt = wab * xw[c];
#pragma unroll
              for (int q = 0; q < VEC; ++q) acc[q] = fma(wt, v.v[q], acc[q]);
            }
          }
        }
      }
    }
  }
}

// Device tables of a Laplacian stencil (both precisions) and of the transfers between a
// grid and its 2:1 coarsening, built from the grid's device node coordinates.
rb_status stencil7_tables(const rb_grid_desc* g, double* w64[3], double* ic64[3], float* w32[3], float* ic32[3],
                          cudaStream_t s);
rb_status transfer_tables(const rb_grid_desc* fine, PAxis<double>* pa64[3], TAxisTab<double>* ta64[3],
                          PAxis<float>* pa32[3], TAxisTab<float>* ta32[3], cudaStream_t s);

}  // namespace rb
