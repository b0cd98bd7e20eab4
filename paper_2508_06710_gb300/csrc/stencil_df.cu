// The matrix-free FVM Laplacian (format RB_STENCIL) in double-float arithmetic (RB_DF64): the
// SpMM over k interleaved columns (Sec. 2, Eq. (1), Algorithm 1) with the entries formed from
// per-axis tables, every product and sum an error-free FP32 transformation (TwoProd, TwoSum)
// as in the double-float CSR SpMM, so that an FP64-accurate product reads only X and writes
// only Y and does its arithmetic on the FP32 pipe.
//
// Factorised entries.  On a Cartesian grid the Laplacian's coefficient across the x face
// between cells i - 1 and i is w_y[j] w_z[k] / d_x[i] = V_ijk (ic_x[i] / w_x[i]), V = w_x w_y w_z
// the cell volume, and likewise for the other faces; the diagonal is minus their sum.  So
//   (L x)_ijk = V_ijk [ D_ijk x_ijk + sum over the six neighbours of c_nb x_nb ],
// with per-axis tables (FP64, split into pairs once): c-[t] = ic[t] / w[t] (face below cell t),
// c+[t] = ic[t + 1] / w[t] (face above; 0 on a wall face), ds[t] = -(c-[t] + c+[t]), and
// D_ijk = ds_x[i] + ds_y[j] + ds_z[k].  Per cell: V (two pair products, the operator's scale
// folded into the x widths) and D (two pair sums); per column: seven multiply-adds of the
// accumulation (S, E) of the double-float CSR kernel, its TwoSum, and the product by V.
//
// Table layout: for axis d, cell t, four pairs {w (x: scale w), c-, c+, ds} = 32 bytes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "stencil7.cuh"

namespace rb {

namespace {

__device__ __forceinline__ void df_bits(double w, float& hi, float& lo) {
  hi = __int_as_float(__double2loint(w));
  lo = __int_as_float(__double2hiint(w));
}
__device__ __forceinline__ double df_word(float hi, float lo) {
  return __hiloint2double(__float_as_int(lo), __float_as_int(hi));
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& r) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_of(double w) {
  DF r;
  df_bits(w, r.h, r.l);
  return r;
}
// (a h + a l)(b h + b l), renormalised (a l b l dropped)
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float q = __fmaf_rn(a.h, b.h, -p);
  q = __fmaf_rn(a.h, b.l, q);
  q = __fmaf_rn(a.l, b.h, q);
  DF r;
  two_sum(p, q, r.h, r.l);
  return r;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  DF r;
  two_sum(s, e, r.h, r.l);
  return r;
}
// (S, E) += a x, as in the double-float CSR SpMM
__device__ __forceinline__ void df_mac(DF a, DF x, float& S, float& E) {
  const float p = __fmul_rn(a.h, x.h);
  float q = __fmaf_rn(a.h, x.h, -p);
  q = __fmaf_rn(a.h, x.l, q);
  q = __fmaf_rn(a.l, x.h, q);
  float s, r;
  two_sum(S, p, s, r);
  S = s;
  E = __fadd_rn(E, __fadd_rn(r, q));
}

struct AxisTab {
  DF w, cm, cp, ds;
};
__device__ __forceinline__ AxisTab load_tab(const double* __restrict__ t, int i) {
  const double2 u = __ldg(reinterpret_cast<const double2*>(t) + 2 * i);
  const double2 v = __ldg(reinterpret_cast<const double2*>(t) + 2 * i + 1);
  return AxisTab{df_of(u.x), df_of(u.y), df_of(v.x), df_of(v.y)};
}

struct StencilDf {
  int n[3];
  int per[3];
  const double* tab[3];
  FastDiv dx, dxy;
};

template <int VEC, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_spmm_stencil_df(StencilDf st, int64_t n, int k, int kp,
                                                               const double* __restrict__ X, int64_t ldx,
                                                               double* __restrict__ Y, int64_t ldy,
                                                               const double* __restrict__ cs) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  DF cc[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) {
    cc[q] = DF{1.0f, 0.0f};
    if constexpr (SCALE) {
      const double c = cs[chunk * VEC + q];
      cc[q].h = __double2float_rn(c);
      cc[q].l = __double2float_rn(c - (double)cc[q].h);
    }
  }
  const int nx = st.n[0], ny = st.n[1], nz = st.n[2];
  const int64_t plane = (int64_t)nx * ny;
  const double* xc = X + chunk * VEC;
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const uint32_t r32 = (uint32_t)row;
    const int kz = (int)st.dxy.div(r32);
    const uint32_t rem = r32 - (uint32_t)kz * (uint32_t)(nx * ny);
    const int j = (int)st.dx.div(rem);
    const int i = (int)(rem - (uint32_t)j * (uint32_t)nx);
    const AxisTab tx = load_tab(st.tab[0], i), ty = load_tab(st.tab[1], j), tz = load_tab(st.tab[2], kz);
    const DF V = df_mul(tx.w, df_mul(ty.w, tz.w));
    const DF D = df_add(tx.ds, df_add(ty.ds, tz.ds));
    // neighbour rows (a wall neighbour has coefficient 0: this row stands in for it)
    const int im = i > 0 ? i - 1 : (st.per[0] ? nx - 1 : i), ip = i + 1 < nx ? i + 1 : (st.per[0] ? 0 : i);
    const int jm = j > 0 ? j - 1 : (st.per[1] ? ny - 1 : j), jp = j + 1 < ny ? j + 1 : (st.per[1] ? 0 : j);
    const int km = kz > 0 ? kz - 1 : (st.per[2] ? nz - 1 : kz), kp2 = kz + 1 < nz ? kz + 1 : (st.per[2] ? 0 : kz);
    const Vec<double, VEC> x0 = ldv<double, VEC>(xc + row * ldx);
    const Vec<double, VEC> a = ldv<double, VEC>(xc + (row - i + im) * ldx);
    const Vec<double, VEC> b = ldv<double, VEC>(xc + (row - i + ip) * ldx);
    const Vec<double, VEC> c = ldv<double, VEC>(xc + (row + (int64_t)(jm - j) * nx) * ldx);
    const Vec<double, VEC> d = ldv<double, VEC>(xc + (row + (int64_t)(jp - j) * nx) * ldx);
    const Vec<double, VEC> e = ldv<double, VEC>(xc + (row + (int64_t)(km - kz) * plane) * ldx);
    const Vec<double, VEC> f = ldv<double, VEC>(xc + (row + (int64_t)(kp2 - kz) * plane) * ldx);
    Vec<double, VEC> y;
#pragma unroll
    for (int q = 0; q < VEC; ++q) {
      float S = 0.0f, E = 0.0f;
      df_mac(D, df_of(x0.v[q]), S, E);
      df_mac(tx.cm, df_of(a.v[q]), S, E);
      df_mac(tx.cp, df_of(b.v[q]), S, E);
      df_mac(ty.cm, df_of(c.v[q]), S, E);
      df_mac(ty.cp, df_of(d.v[q]), S, E);
      df_mac(tz.cm, df_of(e.v[q]), S, E);
      df_mac(tz.cp, df_of(f.v[q]), S, E);
      DF s;
      two_sum(S, E, s.h, s.l);
      DF r = df_mul(s, V);
      if constexpr (SCALE) r = df_mul(r, cc[q]);
      y.v[q] = df_word(r.h, r.l);
    }
    stv<double, VEC>(Y + row * ldy + chunk * VEC, y);
  }
}

template <int VEC>
rb_status launch_df(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                    const double* cs, cudaStream_t s) {
  StencilDf st;
  for (int d = 0; d < 3; ++d) {
    st.n[d] = op->st_n[d];
    st.per[d] = op->st_per[d];
    st.tab[d] = static_cast<const double*>(op->st_w[d]);
  }
  st.dx.init((uint32_t)st.n[0]);
  st.dxy.init((uint32_t)st.n[0] * (uint32_t)st.n[1]);
  const int R = kThreads / sc.kp;
  const int64_t blocks = ((int64_t)op->n_rows + R - 1) / R;
  auto go = [&](auto kern) {
    kern<<<wave_grid(kern, blocks), kThreads, 0, s>>>(st, op->n_rows, k, sc.kp, static_cast<const double*>(X), ldx,
                                                      static_cast<double*>(Y), ldy, cs);
  };
  if (cs) go(&k_spmm_stencil_df<VEC, true>);
  else go(&k_spmm_stencil_df<VEC, false>);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

}  // namespace

rb_status stencil_df_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                            int k, const double* cs, cudaStream_t s) {
  switch (sc.vec) {
    case 1: return launch_df<1>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 2: return launch_df<2>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 3: return launch_df<3>(op, sc, X, ldx, Y, ldy, k, cs, s);
    case 4: return launch_df<4>(op, sc, X, ldx, Y, ldy, k, cs, s);
  }
  set_error("spmm: unsupported vector width %d", sc.vec);
  return RB_EUNSUPPORTED;
}

// The per-axis pair tables from the FP64 widths and inverse centre distances (device arrays of
// n[d] and n[d] + 1 entries): built on the host in FP64, split into pairs, uploaded.
rb_status stencil_df_tables(const rb_grid_desc* grid, double scale, double* const w64[3], double* const ic64[3],
                            void* tab[3], int64_t* bytes, cudaStream_t s) {
  for (int d = 0; d < 3; ++d) {
    const int n = grid->n[d];
    std::vector<double> w(n + 1), ic(n + 1);
    RB_CUDA(cudaMemcpyAsync(w.data(), w64[d], sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaMemcpyAsync(ic.data(), ic64[d], sizeof(double) * (n + 1), cudaMemcpyDeviceToHost, s));
    RB_CUDA(cudaStreamSynchronize(s));
    std::vector<float> t((size_t)n * 8);
    auto put = [&](int cell, int slot, double v) {
      const float hi = (float)v;
      t[(size_t)cell * 8 + 2 * slot] = hi;
      t[(size_t)cell * 8 + 2 * slot + 1] = (float)(v - (double)hi);
    };
    for (int c = 0; c < n; ++c) {
      const double cm = ic[c] / w[c], cp = ic[c + 1] / w[c];
      RB_REQUIRE(std::isfinite(cm) && std::isfinite(cp) && std::fabs(cm) < 3e38 && std::fabs(cp) < 3e38 &&
                     std::fabs(w[c] * (d == 0 ? scale : 1.0)) < 3e38,
                 "rb_fvm_stencil_create: axis %d's coefficients leave the FP32 range of RB_DF64 pairs", d);
      put(c, 0, d == 0 ? scale * w[c] : w[c]);
      put(c, 1, cm);
      put(c, 2, cp);
      put(c, 3, -(cm + cp));
    }
    void* p = nullptr;
    RB_CUDA(cudaMalloc(&p, t.size() * sizeof(float) + 64));
    tab[d] = p;
    *bytes += (int64_t)(t.size() * sizeof(float) + 64);
    RB_CUDA(cudaMemcpyAsync(p, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    RB_CUDA(cudaStreamSynchronize(s));
  }
  return RB_OK;
}

}  // namespace rb
