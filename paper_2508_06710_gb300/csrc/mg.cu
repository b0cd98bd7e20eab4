// Multigrid-preconditioned CG for the Poisson matrix A = -L of a Cartesian FVM grid, on k
// columns that share the operator.  The paper's Poisson solver is CG with a multigrid
// preconditioner (Sec. 4), and Appendix A (Table 9) lists the SpMMs of its hierarchy: the
// level operators, the restrictions and the prolongations.  Its algebraic hierarchy comes
// from a closed library; the hierarchy here is geometric and built from the library's own
// operator assemblies:
//
//   levels     the grid and its repeated 2:1 coarsenings (every other node), while every axis
//              keeps an even count of at least 2 min_cells cells
//   A_l        -L rediscretised on level l (rb_fvm_assemble with scale -1)
//   P_l, P_l^T the trilinear prolongation from level l + 1 and its transpose, the restriction
//              of residuals (rb_refine_assemble, RB_REFINE_PROLONG and RB_REFINE_PROLONG_T)
//   coarsest   solved exactly: a dense inverse of A_L + s 1 1^T (s > 0; the zero-mean
//              pseudo-inverse solution for the singular operator), computed on the device by
//              Gauss-Jordan elimination when the hierarchy is built
//
// One V(nu, nu) cycle z = B r from a zero guess, per level:
//   e = omega D^-1 r; nu - 1 damped Jacobi sweeps e <- e + omega D^-1 (r - A e);
//   r_c = P^T (r - A e); e_c = cycle of the next level on r_c; e <- e + P e_c;
//   nu sweeps e <- e + omega D^-1 (r - A e)
// Each sweep is one SpMM-shaped kernel (the product, the update and the Jacobi scaling fused;
// Jacobi needs the old iterate, so sweeps alternate between two buffers), the residual and the
// prolongation-add too; the restriction is the library's SpMM.  The k columns travel together
// through every kernel (Eq. (1): each matrix entry is read once for all of them).  Constants
// (the null space) picked up by the smoother pass through the cycle harmlessly: they leave
// every residual unchanged and are removed from the solution at the end.
//
// Outer iteration: PCG (Saad, Alg. 9.1) with z = B r, per column; beta in the flexible
// Polak-Ribiere form -alpha (q . z_new) / (r . z)_old (Notay) when requested, which tolerates
// an FP32 cycle.  Two precisions:
//   mixed = 0: FP64 throughout (operators, vectors, cycle); convergence is decided on the true
//              residual b - A x every check_every iterations;
//   mixed != 0: FP64 iterative refinement: r = b - A x (FP64 operator), the scaled residual
//              r / ||r|| solved by the same PCG in FP32 (FP32 operators, vectors and cycle; dot
//              products summed in FP32 per thread, in FP64 across threads and blocks) to
//              inner_rtol, then x += ||r|| d in FP64.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"
#include "spmm_impl.cuh"
#include "stencil7.cuh"

namespace rb {

SpmmSched pick_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y);
rb_status spmm_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                      const double* cs, cudaStream_t s);

namespace {

constexpr int K = RB_MAX_K;
constexpr int kMgMaxLevels = 16;
constexpr int kMgMaxCoarse = 4096;  // cells of the coarsest level (its dense inverse: 128 MiB)

enum MgState : int { MG_ACTIVE = 0, MG_DONE = 2, MG_BREAKDOWN = 3, MG_NOCONV = 4 };

struct MgScal {
  // the CG recurrence (of the FP64 solve, or of a refinement sweep's FP32 solve)
  double rz[K], alpha[K], beta[K], itol2[K];
  int state[K], iters[K];
  // the true residual b - A x (FP64)
  double bb[K], tol2[K], mean[K], scale[K], rr_true[K];
  int ostate[K];
  int n_active, n_oactive;
  unsigned counter[8];
};

__device__ __forceinline__ void mg_recount(MgScal* sc, int k) {
  int na = 0, no = 0;
  for (int j = 0; j < k; ++j) {
    na += sc->state[j] == MG_ACTIVE;
    no += sc->ostate[j] == MG_ACTIVE;
  }
  sc->n_active = na;
  sc->n_oactive = no;
}

// vector width for blocks of k columns with leading dimension k (the library's own buffers,
// 256-byte aligned): 16- or 8-byte accesses where k allows, 3 for multiples of 3
int mg_vec(int eb, int k) {
  if (k * eb == 16 || k * eb == 8) return k;
  if (k % 3 == 0 && k <= 96) return 3;
  for (int w = 16 / eb; w >= 1; w >>= 1)
    if (k % w == 0) return w;
  return 1;
}

// ------------------------------------------------------------------------- cycle kernels

// e = omega D^-1 r (the first sweep from e = 0: no product)
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_smooth0(int64_t n, int k, int kp, const T* __restrict__ r,
                                                          const T* __restrict__ dinv, T omega, T* __restrict__ e,
                                                          const int* __restrict__ gate) {
  if (gate && *gate == 0) return;  // every column of the solve has finished
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const int64_t o = row * k + chunk * VEC;
    const Vec<T, VEC> rv = ldv<T, VEC>(r + o);
    const T w = omega * __ldg(dinv + row);
    Vec<T, VEC> ev;
#pragma unroll
    for (int q = 0; q < VEC; ++q) ev.v[q] = w * rv.v[q];
    stv<T, VEC>(e + o, ev);
  }
}

// Dot products of the last sweep of a cycle used as the CG preconditioner: r . z and q . z
// per column, and the new beta and r . z formed by the last block.
struct MgDots {
  MgScal* sc = nullptr;
  double* partials = nullptr;
  const void* q = nullptr;  // this iteration's q = A p (same type as the cycle)
  int init = 0;             // first z of a solve or sweep: beta = 0
  int flexible = 0;
};

enum SweepMode : int { SW_JACOBI = 0, SW_RESID = 1 };

// One product-shaped pass over level l: with e the iterate (a.X) and r the level's right-hand
// side, writes out = e + omega D^-1 (r - A e) (SW_JACOBI) or out = r - A e (SW_RESID).  With
// DOTS (the last sweep of the outer cycle), also r . out and q . out per column.
template <typename T, int VEC, int MODE, bool DOTS, bool ST>
__global__ void __launch_bounds__(kThreads) k_mg_sweep(CsrArgs<T> a, Stencil7<T> st, const T* __restrict__ r,
                                                        const T* __restrict__ dinv, T omega, T* __restrict__ out,
                                                        MgDots dd, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ RedSmem<2> red;
  const int R = kThreads / a.kp;
  const int t = threadIdx.x;
  const int chunk = t % a.kp, rloc = t / a.kp;
  T d0[VEC], d1[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) d0[q] = d1[q] = T(0);
  const T* qv_base = static_cast<const T*>(dd.q);
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = T(0);
    if constexpr (ST) {
      T unused;
      if (active) stencil7_apply<T, VEC>(st, a.X, a.ldx, row, chunk * VEC, acc, unused);
    } else {
      row_accumulate_direct<T, VEC, 1>(a, row, chunk, 0, active, acc);
    }
    if (active) {
      const int64_t o = row * a.k + chunk * VEC;
      const Vec<T, VEC> rv = ldv<T, VEC>(r + o);
      Vec<T, VEC> y;
      if constexpr (MODE == SW_RESID) {
#pragma unroll
        for (int q = 0; q < VEC; ++q) y.v[q] = rv.v[q] - acc[q];
      } else {
        const Vec<T, VEC> ev = ldv<T, VEC>(a.X + o);
        const T w = omega * __ldg(dinv + row);
#pragma unroll
        for (int q = 0; q < VEC; ++q) y.v[q] = fma(w, rv.v[q] - acc[q], ev.v[q]);
      }
      if constexpr (DOTS) {
        if (dd.init) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) d0[q] = fma(rv.v[q], y.v[q], d0[q]);
        } else {
          const Vec<T, VEC> qv = ldv<T, VEC>(qv_base + o);
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            d0[q] = fma(rv.v[q], y.v[q], d0[q]);
            d1[q] = fma(qv.v[q], y.v[q], d1[q]);
          }
        }
      }
      stv<T, VEC>(out + o, y);
    }
  }
  if constexpr (DOTS) {
    T part[2][VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) part[0][q] = d0[q], part[1][q] = d1[q];
    const double v = block_reduce<2, VEC>(part, a.kp, 1, a.k, red);
    MgScal* sc = dd.sc;
    if (!publish_partials<2>(v, 2 * a.k, dd.partials, &sc->counter[2], red)) return;
    const double tot = final_sum<2>(dd.partials, 2 * a.k, gridDim.x, red);
    // thread t < 2k holds quantity t / k of column t % k
    __shared__ double s_tot[2 * K];
    if ((int)threadIdx.x < 2 * a.k) s_tot[threadIdx.x] = tot;
    __syncthreads();
    const int j = threadIdx.x;
    if (j < a.k) {
      const double rz_new = s_tot[j], qz = s_tot[a.k + j];
      double beta = 0.0;
      if (!dd.init && sc->state[j] == MG_ACTIVE) {
        const double rz_old = sc->rz[j];
        beta = dd.flexible ? -sc->alpha[j] * qz / rz_old : rz_new / rz_old;
        if (!isfinite(beta)) beta = 0.0;
      }
      sc->beta[j] = beta;
      sc->rz[j] = rz_new;
    }
  }
}

// e += P e_c (the coarse correction; a.X = e_c, a.Y = e, P's rows are this level's cells)
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_prolong_add(CsrArgs<T> a, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int R = kThreads / a.kp;
  const int t = threadIdx.x;
  const int chunk = t % a.kp, rloc = t / a.kp;
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = T(0);
    row_accumulate_direct<T, VEC, 1>(a, row, chunk, 0, active, acc);
    if (active) {
      const int64_t o = row * a.ldy + chunk * VEC;
      Vec<T, VEC> y = ldv_rw<T, VEC>(a.Y + o);
#pragma unroll
      for (int q = 0; q < VEC; ++q) y.v[q] += acc[q];
      stv<T, VEC>(a.Y + o, y);
    }
  }
}

// Matrix-free transfers (stencil7.cuh): e += P e_c over the fine rows, r_c = P^T r over the
// coarse rows
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_prolong_st(Transfer3<T> tr, int64_t n, int k, int kp,
                                                             const T* __restrict__ ec, T* __restrict__ e,
                                                             const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    T acc[VEC];
    prolong_apply<T, VEC>(tr, ec, k, row, chunk * VEC, acc);
    const int64_t o = row * k + chunk * VEC;
    Vec<T, VEC> y = ldv_rw<T, VEC>(e + o);
#pragma unroll
    for (int q = 0; q < VEC; ++q) y.v[q] += acc[q];
    stv<T, VEC>(e + o, y);
  }
}

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_restrict_st(Transfer3<T> tr, int64_t nc, int k, int kp,
                                                              const T* __restrict__ rf, T* __restrict__ rc,
                                                              const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < nc; row += (int64_t)gridDim.x * R) {
    T acc[VEC];
    restrict_apply<T, VEC>(tr, rf, k, row, chunk * VEC, acc);
    Vec<T, VEC> y;
#pragma unroll
    for (int q = 0; q < VEC; ++q) y.v[q] = acc[q];
    stv<T, VEC>(rc + row * k + chunk * VEC, y);
  }
}

// ------------------------------------------------------------------- line smoothing
// Block Jacobi over the grid lines along one wall-bounded axis (the strongly coupled one of a
// wall-refined grid): the block of a line is the tridiagonal part of A along it (A's diagonal
// and its two couplings along the axis).  Thomas' algorithm: with l_j, u_j the couplings to
// positions j - 1 and j + 1 and b_j the diagonal, den_0 = b_0, den_j = b_j - l_j c_{j-1},
// c_j = u_j / den_j (the factors, fixed with the operator, computed once per level), then per
// right-hand side s: d_j = (s_j - l_j d_{j-1}) / den_j forward and x_j = d_j - c_j x_{j+1}
// backward.

struct LineGeom {
  int axis, len, stride;  // the axis, its cell count, the row stride along it
  int nlines;             // lines (rows / len)
  FastDiv div_inner;      // lines are numbered (inner, outer): inner < stride
  int inner;              // = stride (rows before the line axis in the numbering)
};

// first row of line t: inner part below the axis, outer part above it
__device__ __forceinline__ int64_t line_base(const LineGeom& lg, int t) {
  if (lg.stride == 1) return (int64_t)t * lg.len;
  const uint32_t o = lg.div_inner.div((uint32_t)t);
  const uint32_t i = (uint32_t)t - o * (uint32_t)lg.inner;
  return (int64_t)o * lg.len * lg.inner + i;
}

template <typename T>
__device__ __forceinline__ void along(const Coef7<T>& c, int axis, T& lo, T& up) {
  lo = axis == 0 ? c.cxm : (axis == 1 ? c.cym : c.czm);
  up = axis == 0 ? c.cxp : (axis == 1 ? c.cyp : c.czp);
}

// the factors c_j and 1 / den_j of every line, from the FP64 tables, in both precisions
__global__ void k_line_factors(Stencil7<double> st, LineGeom lg, double* __restrict__ c64,
                               double* __restrict__ id64, double* __restrict__ a64, float* __restrict__ c32,
                               float* __restrict__ id32, float* __restrict__ a32) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < lg.nlines; t += gridDim.x * blockDim.x) {
    const int64_t b0 = line_base(lg, t);
    double cprev = 0.0;
    for (int j = 0; j < lg.len; ++j) {
      const int64_t row = b0 + (int64_t)j * lg.stride;
      const Coef7<double> cf = stencil7_coef(st, row);
      double lo, up;
      along(cf, lg.axis, lo, up);
      lo *= st.scale, up *= st.scale;
      const double den = st.scale * cf.diag - lo * cprev;
      const double c = up / den;
      c64[row] = c, id64[row] = 1.0 / den, a64[row] = -lo / den;
      c32[row] = (float)c, id32[row] = (float)(1.0 / den), a32[row] = (float)(-lo / den);
      cprev = c;
    }
  }
}

// The 7-point operator seen from one grid line along axis d (cells t = 0 .. len - 1): the
// face area across d is the product of the other two axes' widths, fixed on the line, and the
// coefficient across another axis e is w_d[t] times a factor fixed on the line (the third
// axis' width times 1 / d_f of the face across e).  A cell then costs two table reads along
// the line, and its neighbours along d are the line's own cells, carried from cell to cell.
template <typename T>
struct LineSten {
  const T* wd;   // widths along the line
  const T* icd;  // 1 / d_f of the faces along the line
  T area;        // face area across d
  T f1m, f1p, f2m, f2p;        // e1 < e2 the other axes: the factors of the lower / upper face
  int o1m, o1p, o2m, o2p;  // row offsets of those neighbours (wrapped, or 0 at a wall)
  int wrap;                // along a periodic d: offset from cell 0 to cell len - 1 (else 0)
};

template <typename P>
__device__ __forceinline__ P sel3(int a, P v0, P v1, P v2) {
  return a == 0 ? v0 : (a == 1 ? v1 : v2);
}

// the line along axis d whose cell t = 0 is row b0
template <typename T>
__device__ __forceinline__ LineSten<T> line_sten(const Stencil7<T>& s, int d, int64_t b0) {
  const uint32_t r32 = (uint32_t)b0;
  const int p2 = (int)s.dxy.div(r32);
  const uint32_t rem = r32 - (uint32_t)p2 * (uint32_t)(s.n[0] * s.n[1]);
  const int p1 = (int)s.dx.div(rem);
  const int p0 = (int)(rem - (uint32_t)p1 * (uint32_t)s.n[0]);
  const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  const int64_t plane = (int64_t)s.n[0] * s.n[1];
  LineSten<T> L;
  L.wd = sel3(d, s.w[0], s.w[1], s.w[2]);
  L.icd = sel3(d, s.ic[0], s.ic[1], s.ic[2]);
  const int pe1 = sel3(e1, p0, p1, p2), pe2 = sel3(e2, p0, p1, p2);
  const T* w1 = sel3(e1, s.w[0], s.w[1], s.w[2]);
  const T* w2 = sel3(e2, s.w[0], s.w[1], s.w[2]);
  const T* ic1 = sel3(e1, s.ic[0], s.ic[1], s.ic[2]);
  const T* ic2 = sel3(e2, s.ic[0], s.ic[1], s.ic[2]);
  const T we1 = __ldg(w1 + pe1), we2 = __ldg(w2 + pe2);
  L.area = we1 * we2;
  L.f1m = we2 * __ldg(ic1 + pe1), L.f1p = we2 * __ldg(ic1 + pe1 + 1);
  L.f2m = we1 * __ldg(ic2 + pe2), L.f2p = we1 * __ldg(ic2 + pe2 + 1);
  auto offs = [&](int e, int pe, int& om, int& op) {  // rows < 2^31: offsets fit in 32 bits
    const int ne = sel3(e, s.n[0], s.n[1], s.n[2]), per = sel3(e, s.per[0], s.per[1], s.per[2]);
    const int str = sel3(e, 1, s.n[0], (int)plane);
    const int pm = pe > 0 ? pe - 1 : (per ? ne - 1 : pe), pp = pe + 1 < ne ? pe + 1 : (per ? 0 : pe);
    om = (pm - pe) * str, op = (pp - pe) * str;
  };
  offs(e1, pe1, L.o1m, L.o1p);
  offs(e2, pe2, L.o2m, L.o2p);
  const int nd = sel3(d, s.n[0], s.n[1], s.n[2]);
  L.wrap = sel3(d, s.per[0], s.per[1], s.per[2]) ? (nd - 1) * sel3(d, 1, s.n[0], (int)plane) : 0;
  return L;
}

enum LineMode : int { LN_ZERO = 0, LN_JACOBI = 1 };

constexpr int kSeg = kThreads / 32;  // segments per line: one warp each

// out = e + omega T^-1 (r - A e) over each line (LN_ZERO: e = 0, out = omega T^-1 r); with DOTS
// the last sweep of the outer cycle, also r . out and q . out per column.
//
// Partition method: Thomas' two recurrences are first order, d_j = a_j d_{j-1} + b_j with
// a_j = -l_j / den_j, b_j = s_j / den_j, and x_j = d_j - c_j x_{j+1}; a segment of a line
// composes its cells' maps into one affine map, the segments' maps are joined in shared
// memory, and each segment then finishes its cells from its entry value.  A block holds
// 32 / KP lines (the lanes of a warp: KP column chunks of each line in adjacent lanes, lines
// next to each other, so that loads along the other axes are coalesced) and kSeg segments (the
// warps).  Passes: (1) residual, b_j kept in `out`, forward composition; (2) d_j into `out`,
// with the backward composition accumulated forward (x_j0 = sum_j P_j d_j + P x_j1, P the
// running product of -c); (3) backward substitution and the damped update.
template <typename T, int VEC, int MODE, bool DOTS>
__global__ void __launch_bounds__(kThreads) k_mg_line(Stencil7<T> st, LineGeom lg, int k, int kp,
                                                       const T* __restrict__ e, const T* __restrict__ r,
                                                       const T* __restrict__ cfac, const T* __restrict__ idn,
                                                       const T* __restrict__ aco, T omega, T* __restrict__ out,
                                                       MgDots dd, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ RedSmem<2> red;
  __shared__ T sA[kSeg][32][VEC], sB[kSeg][32][VEC];
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int chunk = lane % kp, ll = lane / kp, LW = 32 / kp;
  const bool col_ok = chunk * VEC < k;
  const int j0 = (seg * lg.len) / kSeg, j1 = ((seg + 1) * lg.len) / kSeg;
  T d0[VEC], d1[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) d0[q] = d1[q] = T(0);
  const T* qv_base = static_cast<const T*>(dd.q);
  for (int line0 = blockIdx.x * LW; line0 < lg.nlines; line0 += gridDim.x * LW) {  // uniform over the block
    const int t = line0 + ll;
    const bool on = col_ok && t < lg.nlines;
    const int64_t b0 = on ? line_base(lg, t) : 0;
    // pass 1: b_j = s_j / den_j into out; forward map of the segment: d_out = A d_in + B
    T A[VEC], B[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) A[q] = T(1), B[q] = T(0);
    // FP64: the residual in the line's own form (e_{j-1}, e_j, e_{j+1} carried along the line,
    // four of the six coefficients one product each), which takes most of the generic form's
    // FP64 arithmetic off the slow FP64 pipe; FP32 keeps the generic form, whose fewer
    // registers keep the whole grid of blocks resident
    constexpr bool kLineForm = sizeof(T) == 8 && MODE != LN_ZERO;
    LineSten<T> ls{};
    Vec<T, VEC> xp{}, x0{}, xn{};
    T icm = T(0);
    const int64_t sk = (int64_t)lg.stride * k;
    if constexpr (kLineForm) {
      if (on) {
        ls = line_sten(st, lg.axis, b0);
        const T* ec = e + (b0 + (int64_t)j0 * lg.stride) * k + chunk * VEC;
        x0 = ldv<T, VEC>(ec);
        xp = j0 > 0 ? ldv<T, VEC>(ec - sk) : (ls.wrap ? ldv<T, VEC>(ec + (int64_t)ls.wrap * k) : x0);
        icm = __ldg(ls.icd + j0);
      }
    }
    if (on) {
      for (int j = j0; j < j1; ++j) {
        const int64_t row = b0 + (int64_t)j * lg.stride;
        const int64_t o = row * k + chunk * VEC;
        const Vec<T, VEC> rv = ldv<T, VEC>(r + o);
        T sv[VEC];
        if constexpr (MODE == LN_ZERO) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) sv[q] = rv.v[q];
        } else if constexpr (kLineForm) {
          const T* ec = e + o;
          xn = j + 1 < lg.len ? ldv<T, VEC>(ec + sk) : (ls.wrap ? ldv<T, VEC>(ec - (int64_t)ls.wrap * k) : x0);
          const Vec<T, VEC> a1 = ldv<T, VEC>(ec + (int64_t)ls.o1m * k), b1 = ldv<T, VEC>(ec + (int64_t)ls.o1p * k);
          const Vec<T, VEC> a2 = ldv<T, VEC>(ec + (int64_t)ls.o2m * k), b2 = ldv<T, VEC>(ec + (int64_t)ls.o2p * k);
          const T wt = __ldg(ls.wd + j), icp = __ldg(ls.icd + j + 1);
          const T c1m = wt * ls.f1m, c1p = wt * ls.f1p, c2m = wt * ls.f2m, c2p = wt * ls.f2p;
          const T cdm = ls.area * icm, cdp = ls.area * icp;
          const T diag = -(((c1m + c1p) + (c2m + c2p)) + (cdm + cdp));
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            T y = diag * x0.v[q];
            y = fma(c1m, a1.v[q], y);
            y = fma(c1p, b1.v[q], y);
            y = fma(c2m, a2.v[q], y);
            y = fma(c2p, b2.v[q], y);
            y = fma(cdm, xp.v[q], y);
            y = fma(cdp, xn.v[q], y);
            sv[q] = rv.v[q] - st.scale * y;
          }
          xp = x0, x0 = xn, icm = icp;
        } else {
          T ae[VEC], unused;
          stencil7_apply<T, VEC>(st, e, k, row, chunk * VEC, ae, unused);
#pragma unroll
          for (int q = 0; q < VEC; ++q) sv[q] = rv.v[q] - ae[q];
        }
        const T id = __ldg(idn + row), a = __ldg(aco + row);
        Vec<T, VEC> bv;
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          bv.v[q] = sv[q] * id;
          A[q] = a * A[q];
          B[q] = fma(a, B[q], bv.v[q]);
        }
        stv<T, VEC>(out + o, bv);
      }
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) sA[seg][lane][q] = A[q], sB[seg][lane][q] = B[q];
    __syncthreads();
    T din[VEC];  // d just before the segment: the earlier segments' maps applied to d = 0
#pragma unroll
    for (int q = 0; q < VEC; ++q) din[q] = T(0);
    for (int s2 = 0; s2 < seg; ++s2)
#pragma unroll
      for (int q = 0; q < VEC; ++q) din[q] = fma(sA[s2][lane][q], din[q], sB[s2][lane][q]);
    __syncthreads();  // sA / sB are reused below
    // pass 2: d_j into out; backward map of the segment accumulated forward: x_j0 = S + P x_j1
    T P[VEC], S[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) P[q] = T(1), S[q] = T(0);
    if (on) {
      for (int j = j0; j < j1; ++j) {
        const int64_t row = b0 + (int64_t)j * lg.stride;
        const int64_t o = row * k + chunk * VEC;
        const T a = __ldg(aco + row), c = __ldg(cfac + row);
        Vec<T, VEC> dv = ldv_rw<T, VEC>(out + o);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          din[q] = fma(a, din[q], dv.v[q]);
          dv.v[q] = din[q];
          S[q] = fma(P[q], din[q], S[q]);
          P[q] = -c * P[q];
        }
        stv<T, VEC>(out + o, dv);
      }
    }
#pragma unroll
    for (int q = 0; q < VEC; ++q) sA[seg][lane][q] = P[q], sB[seg][lane][q] = S[q];
    __syncthreads();
    T xin[VEC];  // x just after the segment: the later segments' maps from x_len = 0
#pragma unroll
    for (int q = 0; q < VEC; ++q) xin[q] = T(0);
    for (int s2 = kSeg - 1; s2 > seg; --s2)
#pragma unroll
      for (int q = 0; q < VEC; ++q) xin[q] = fma(sA[s2][lane][q], xin[q], sB[s2][lane][q]);
    __syncthreads();
    // pass 3: backward substitution, damped update (and the dot products)
    if (on) {
      for (int j = j1 - 1; j >= j0; --j) {
        const int64_t row = b0 + (int64_t)j * lg.stride;
        const int64_t o = row * k + chunk * VEC;
        const T c = __ldg(cfac + row);
        const Vec<T, VEC> dv = ldv_rw<T, VEC>(out + o);
        Vec<T, VEC> y;
        if constexpr (MODE == LN_ZERO) {
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            xin[q] = dv.v[q] - c * xin[q];
            y.v[q] = omega * xin[q];
          }
        } else {
          const Vec<T, VEC> ev = ldv<T, VEC>(e + o);
#pragma unroll
          for (int q = 0; q < VEC; ++q) {
            xin[q] = dv.v[q] - c * xin[q];
            y.v[q] = fma(omega, xin[q], ev.v[q]);
          }
        }
        if constexpr (DOTS) {
          const Vec<T, VEC> rv = ldv<T, VEC>(r + o);
          if (dd.init) {
#pragma unroll
            for (int q = 0; q < VEC; ++q) d0[q] = fma(rv.v[q], y.v[q], d0[q]);
          } else {
            const Vec<T, VEC> qv = ldv<T, VEC>(qv_base + o);
#pragma unroll
            for (int q = 0; q < VEC; ++q) {
              d0[q] = fma(rv.v[q], y.v[q], d0[q]);
              d1[q] = fma(qv.v[q], y.v[q], d1[q]);
            }
          }
        }
        stv<T, VEC>(out + o, y);
      }
    }
  }
  if constexpr (DOTS) {
    T part[2][VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) part[0][q] = d0[q], part[1][q] = d1[q];
    const double v = block_reduce<2, VEC>(part, kp, 1, k, red);
    MgScal* sc = dd.sc;
    if (!publish_partials<2>(v, 2 * k, dd.partials, &sc->counter[2], red)) return;
    const double tot = final_sum<2>(dd.partials, 2 * k, gridDim.x, red);
    __shared__ double s_tot[2 * K];
    if ((int)threadIdx.x < 2 * k) s_tot[threadIdx.x] = tot;
    __syncthreads();
    const int jj = threadIdx.x;
    if (jj < k) {
      const double rz_new = s_tot[jj], qz = s_tot[k + jj];
      double beta = 0.0;
      if (!dd.init && sc->state[jj] == MG_ACTIVE) {
        const double rz_old = sc->rz[jj];
        beta = dd.flexible ? -sc->alpha[jj] * qz / rz_old : rz_new / rz_old;
        if (!isfinite(beta)) beta = 0.0;
      }
      sc->beta[jj] = beta;
      sc->rz[jj] = rz_new;
    }
  }
}

// z = Ainv r on the coarsest level (Ainv dense FP64, nc x nc): one block per row, lanes over
// (m, column), the m lanes folded through shared memory in a fixed order
template <typename T>
__global__ void __launch_bounds__(kThreads) k_mg_coarse(int nc, int k, const double* __restrict__ ainv,
                                                         const T* __restrict__ r, T* __restrict__ z,
                                                         const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ double s[kThreads];
  const int kp = next_pow2(k);
  const int j = threadIdx.x % kp, lane = threadIdx.x / kp, lanes = kThreads / kp;
  const int i = blockIdx.x;
  double acc = 0.0;
  if (j < k)
    for (int m = lane; m < nc; m += lanes) acc = fma(__ldg(ainv + (int64_t)i * nc + m), (double)r[(int64_t)m * k + j], acc);
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = lanes / 2; w >= 1; w >>= 1) {
    if (lane < w) s[threadIdx.x] += s[threadIdx.x + w * kp];
    __syncthreads();
  }
  if (lane == 0 && j < k) z[(int64_t)i * k + j] = (T)s[j];
}

// ---------------------------------------------------------------------- CG kernels

// q = A p, p . q; the last block forms alpha = (r . z) / (p . q) per column
template <typename T, int VEC, bool ST>
__global__ void __launch_bounds__(kThreads) k_mgcg_q(CsrArgs<T> a, Stencil7<T> st, MgScal* __restrict__ sc,
                                                      double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<1> red;
  const int R = kThreads / a.kp;
  const int t = threadIdx.x;
  const int chunk = t % a.kp, rloc = t / a.kp;
  T d[VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) d[q] = T(0);
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = T(0);
    if constexpr (ST) {
      T unused;
      if (active) stencil7_apply<T, VEC>(st, a.X, a.ldx, row, chunk * VEC, acc, unused);
    } else {
      row_accumulate_direct<T, VEC, 1, false, true>(a, row, chunk, 0, active, acc);
    }
    if (active) {
      const int64_t o = row * a.k + chunk * VEC;
      const Vec<T, VEC> pv = ldv<T, VEC>(a.X + o);
      Vec<T, VEC> qv;
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        qv.v[q] = acc[q];
        d[q] = fma(pv.v[q], acc[q], d[q]);
      }
      stv<T, VEC>(a.Y + o, qv);
    }
  }
  T part[1][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) part[0][q] = d[q];
  const double v = block_reduce<1, VEC>(part, a.kp, 1, a.k, red);
  if (!publish_partials<1>(v, a.k, partials, &sc->counter[0], red)) return;
  const double tot = final_sum<1>(partials, a.k, gridDim.x, red);
  const int j = threadIdx.x;
  if (j < a.k) {
    double al = 0.0;
    if (sc->state[j] == MG_ACTIVE) {
      if (!(tot > 0.0) || !isfinite(tot) || !isfinite(sc->rz[j])) {
        // a refinement sweep's FP32 solve ends there (the FP64 residual decides); the FP64
        // solve reports the breakdown
        sc->state[j] = sizeof(T) == 4 ? MG_DONE : MG_BREAKDOWN;
      } else {
        al = sc->rz[j] / tot;
      }
    }
    sc->alpha[j] = al;
  }
  __syncthreads();
  if (threadIdx.x == 0) mg_recount(sc, a.k);
}

// x += alpha p, r -= alpha q, r . r; the last block counts the iteration and, for a
// refinement sweep's inner solve (INNER), stops columns whose r . r reached itol2
template <typename T, int VEC, bool INNER>
__global__ void __launch_bounds__(kThreads) k_mgcg_xr(int64_t n, int k, int kp, T* __restrict__ x,
                                                       T* __restrict__ r, const T* __restrict__ p,
                                                       const T* __restrict__ q, MgScal* __restrict__ sc,
                                                       double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<1> red;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const bool col_ok = chunk * VEC < k;
  T al[VEC], d[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) al[e] = col_ok ? (T)sc->alpha[chunk * VEC + e] : T(0), d[e] = T(0);
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
      const int64_t o = row * k + chunk * VEC;
      const Vec<T, VEC> pv = ldv<T, VEC>(p + o);
      const Vec<T, VEC> qv = ldv<T, VEC>(q + o);
      Vec<T, VEC> rv = ldv_rw<T, VEC>(r + o);
      Vec<T, VEC> xv = ldv_rw<T, VEC>(x + o);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        // a column that is not iterating (alpha = 0) keeps x and r bit for bit
        xv.v[e] = al[e] != T(0) ? fma(al[e], pv.v[e], xv.v[e]) : xv.v[e];
        rv.v[e] = al[e] != T(0) ? fma(-al[e], qv.v[e], rv.v[e]) : rv.v[e];
        d[e] = fma(rv.v[e], rv.v[e], d[e]);
      }
      stv<T, VEC>(x + o, xv);
      stv<T, VEC>(r + o, rv);
    }
  }
  T part[1][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = d[e];
  const double v = block_reduce<1, VEC>(part, kp, 1, k, red);
  if (!publish_partials<1>(v, k, partials, &sc->counter[1], red)) return;
  const double tot = final_sum<1>(partials, k, gridDim.x, red);
  const int j = threadIdx.x;
  if (j < k && sc->state[j] == MG_ACTIVE) {
    sc->iters[j] += 1;
    if (INNER && tot <= sc->itol2[j]) sc->state[j] = MG_DONE;
    if (!isfinite(tot)) sc->state[j] = INNER ? MG_DONE : MG_BREAKDOWN;
  }
  __syncthreads();
  if (threadIdx.x == 0) mg_recount(sc, k);
}

// p = z + beta p (beta = 0 where a column is not iterating); INIT: p = z, whatever p held
// (the buffers are shared by the FP64 and FP32 solves: stale bits may read as NaN, and
// 0 * NaN is NaN)
template <typename T, int VEC, bool INIT>
__global__ void __launch_bounds__(kThreads) k_mgcg_p(int64_t n, int k, int kp, const T* __restrict__ z,
                                                      T* __restrict__ p, const MgScal* __restrict__ sc) {
  if (sc->n_active == 0) return;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  T be[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) be[e] = (T)sc->beta[chunk * VEC + e];
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const int64_t o = row * k + chunk * VEC;
    const Vec<T, VEC> zv = ldv<T, VEC>(z + o);
    if constexpr (INIT) {
      stv<T, VEC>(p + o, zv);
    } else {
      Vec<T, VEC> pv = ldv_rw<T, VEC>(p + o);
#pragma unroll
      for (int e = 0; e < VEC; ++e) pv.v[e] = fma(be[e], pv.v[e], zv.v[e]);
      stv<T, VEC>(p + o, pv);
    }
  }
}

// ------------------------------------------------------------- FP64 true residual, refinement

enum ResidKind : int { TR_INIT = 0, TR_CHECK = 1 };

// rt = b - A x (FP64), per column sum and sum of squares (and of b at TR_INIT); the last block
// forms the projected norms and marks columns whose true residual meets the tolerance
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_true_resid(CsrArgs<double> a, const double* __restrict__ b,
                                                             int64_t ldb, double* __restrict__ rt, int kind,
                                                             int project, double rtol2, MgScal* __restrict__ sc,
                                                             double* __restrict__ partials) {
  __shared__ RedSmem<4> red;
  const int R = kThreads / a.kp;
  const int t = threadIdx.x;
  const int chunk = t % a.kp, rloc = t / a.kp;
  double s[4][VEC];
#pragma unroll
  for (int q = 0; q < VEC; ++q) s[0][q] = s[1][q] = s[2][q] = s[3][q] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    double acc[VEC];
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] = 0.0;
    row_accumulate_direct<double, VEC, 1>(a, row, chunk, 0, active, acc);
    if (active) {
      Vec<double, VEC> y;
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const double bv = __ldg(b + row * ldb + chunk * VEC + q);
        y.v[q] = bv - acc[q];
        s[0][q] += y.v[q];
        s[1][q] = fma(y.v[q], y.v[q], s[1][q]);
        if (kind == TR_INIT) {
          s[2][q] += bv;
          s[3][q] = fma(bv, bv, s[3][q]);
        }
      }
      stv<double, VEC>(rt + row * a.k + chunk * VEC, y);
    }
  }
  const double v = block_reduce<4, VEC>(s, a.kp, 1, a.k, red);
  if (!publish_partials<4>(v, 4 * a.k, partials, &sc->counter[3], red)) return;
  const double tot = final_sum<4>(partials, 4 * a.k, gridDim.x, red);
  __shared__ double s_tot[4 * K];
  if ((int)threadIdx.x < 4 * a.k) s_tot[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < a.k) {
    const double n = (double)a.n_rows;
    const double mean = project ? s_tot[j] / n : 0.0;
    double rr = s_tot[a.k + j] - n * mean * mean;
    if (rr < 0.0) rr = 0.0;  // rounding; a NaN stays NaN (fmax would hide it)
    if (kind == TR_INIT) {
      const double mb = project ? s_tot[2 * a.k + j] / n : 0.0;
      double bb = s_tot[3 * a.k + j] - n * mb * mb;
      if (bb < 0.0) bb = 0.0;
      sc->bb[j] = bb;
      sc->tol2[j] = rtol2 * bb;
      sc->ostate[j] = MG_ACTIVE;
      sc->state[j] = MG_ACTIVE;
      sc->iters[j] = 0;
    }
    sc->mean[j] = mean;
    sc->rr_true[j] = rr;
    sc->scale[j] = sqrt(rr);
    if (sc->ostate[j] == MG_ACTIVE) {
      if (!isfinite(rr)) {
        sc->ostate[j] = MG_BREAKDOWN;
        sc->state[j] = MG_BREAKDOWN;
      } else if (rr <= sc->tol2[j]) {
        sc->ostate[j] = MG_DONE;
        sc->state[j] = MG_DONE;
      }
    }
    if (sc->state[j] == MG_BREAKDOWN) sc->ostate[j] = MG_BREAKDOWN;
  }
  __syncthreads();
  if (threadIdx.x == 0) mg_recount(sc, a.k);
}

// out = (rt - mean) * inv (per column), in the solve's type T; zero for columns that are not
// iterating (their share of the cycle then stays zero).  MODE 0: the FP64 solve's initial
// residual (inv = 1); MODE 1: a refinement sweep's scaled FP32 residual, inv = 1 / ||rt||,
// with the sweep's inner target set per column and its state reopened.
template <typename T, int VEC, int MODE>
__global__ void __launch_bounds__(kThreads) k_mg_rhs(int64_t n, int k, int kp, const double* __restrict__ rt,
                                                      T* __restrict__ out, MgScal* __restrict__ sc, double inner_rtol,
                                                      double rtol) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  double mean[VEC], inv[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int j = chunk * VEC + e;
    const bool on = sc->ostate[j] == MG_ACTIVE;
    mean[e] = sc->mean[j];
    inv[e] = !on ? 0.0 : (MODE == 1 ? 1.0 / sc->scale[j] : 1.0);
  }
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const int64_t o = row * k + chunk * VEC;
    Vec<T, VEC> y;
#pragma unroll
    for (int e = 0; e < VEC; ++e) y.v[e] = (T)((__ldg(rt + o + e) - mean[e]) * inv[e]);
    stv<T, VEC>(out + o, y);
  }
  if (MODE == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
    for (int j = 0; j < k; ++j) {
      if (sc->ostate[j] == MG_ACTIVE) {
        // this sweep's target: inner_rtol of its residual, or only what the outer tolerance
        // still needs (half of it) when that is looser, so the last sweep does not overshoot
        const double need = 0.5 * sqrt(sc->tol2[j]) / sc->scale[j];
        const double tgt = fmax(inner_rtol, need);
        sc->itol2[j] = tgt * tgt;
        sc->state[j] = MG_ACTIVE;
      } else if (sc->state[j] == MG_ACTIVE) {
        sc->state[j] = MG_DONE;
      }
    }
    mg_recount(sc, k);
  }
}

// x64 += ||r|| d (the refinement update, FP64) for columns still open
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_refine_add(int64_t n, int k, int kp, double* __restrict__ x,
                                                             const float* __restrict__ d, const MgScal* __restrict__ sc) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  double s[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int j = chunk * VEC + e;
    s[e] = sc->ostate[j] == MG_ACTIVE ? sc->scale[j] : 0.0;
  }
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R) {
    const int64_t o = row * k + chunk * VEC;
#pragma unroll
    for (int e = 0; e < VEC; ++e) x[o + e] = fma(s[e], (double)d[o + e], x[o + e]);
  }
}

// column means of x removed (the zero-mean solution of a singular problem), two passes
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_colsum(int64_t n, int k, int kp, const double* __restrict__ x,
                                                         MgScal* __restrict__ sc, double* __restrict__ partials) {
  __shared__ RedSmem<1> red;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  double s[1][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) s[0][e] = 0.0;
  if (chunk * VEC < k)
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R)
#pragma unroll
      for (int e = 0; e < VEC; ++e) s[0][e] += x[row * k + chunk * VEC + e];
  const double v = block_reduce<1, VEC>(s, kp, 1, k, red);
  if (!publish_partials<1>(v, k, partials, &sc->counter[4], red)) return;
  const double tot = final_sum<1>(partials, k, gridDim.x, red);
  if ((int)threadIdx.x < k) sc->mean[threadIdx.x] = tot / (double)n;
}

template <int VEC>
__global__ void __launch_bounds__(kThreads) k_mg_submean(int64_t n, int k, int kp, double* __restrict__ x,
                                                          const MgScal* __restrict__ sc) {
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  double m[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) m[e] = sc->mean[chunk * VEC + e];
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < n; row += (int64_t)gridDim.x * R)
#pragma unroll
    for (int e = 0; e < VEC; ++e) x[row * k + chunk * VEC + e] -= m[e];
}

__global__ void k_mg_mark_noconv(MgScal* sc, int k) {
  const int j = threadIdx.x;
  if (j < k) {
    if (sc->ostate[j] == MG_ACTIVE) sc->ostate[j] = MG_NOCONV;
    if (sc->state[j] == MG_ACTIVE) sc->state[j] = MG_NOCONV;
  }
  __syncthreads();
  if (j == 0) mg_recount(sc, k);
}

// block copies between a caller's strided block and the library's (ld = k), with conversion
template <typename TI, typename TO>
__global__ void k_mg_copy(int64_t n, int k, const TI* __restrict__ src, int64_t lds, TO* __restrict__ dst, int64_t ldd) {
  const int64_t total = n * k;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / k;
    const int j = (int)(i - row * k);
    dst[row * ldd + j] = (TO)src[row * lds + j];
  }
}

// ------------------------------------------------------- coarsest level: dense inverse

__global__ void k_dense_from_csr(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ va, double* __restrict__ M) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) M[(int64_t)i * n + j] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int p = rp[i]; p < rp[i + 1]; ++p) M[(int64_t)i * n + ci[p]] += va[p];
    __syncthreads();
  }
}

// M += s 1 1^T with s = trace(M) / n^2 (the constant vector's eigenvalue becomes the mean
// diagonal entry): one block
__global__ void k_dense_shift(int n, double* __restrict__ M) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += M[(int64_t)i * n + i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double s = red[0] / ((double)n * n);
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) M[e] += s;
}

// Gauss-Jordan inversion in place, pivot p (no pivoting: the shifted matrix is symmetric
// positive definite).  Step 1 (one block): save column p, scale row p by 1 / M[p][p].
__global__ void k_gj_pivot(int n, int p, double* __restrict__ M, double* __restrict__ col) {
  const double piv = M[(int64_t)p * n + p];
  for (int i = threadIdx.x; i < n; i += blockDim.x) col[i] = M[(int64_t)i * n + p];
  __syncthreads();
  const double inv = 1.0 / piv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) M[(int64_t)p * n + j] = (j == p) ? inv : M[(int64_t)p * n + j] * inv;
}

// Step 2: every other row i: M[i][j] -= col[i] M[p][j] (j != p), M[i][p] = -col[i] M[p][p]
__global__ void k_gj_update(int n, int p, double* __restrict__ M, const double* __restrict__ col) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    if (i == p) continue;
    const double f = col[i];
    M[e] = (j == p) ? -f * M[(int64_t)p * n + p] : fma(-f, M[(int64_t)p * n + j], M[e]);
  }
}

__global__ void k_every_other(int n_out, const double* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_out) dst[i] = src[2 * i];
}

}  // namespace
}  // namespace rb

// ------------------------------------------------------------------------ the hierarchy

struct rb_mg_level {
  int n[3] = {0, 0, 0};
  int64_t cells = 0;
  rb_op* A[2] = {nullptr, nullptr};   // -L: [0] FP64, [1] FP32
  rb_op* P[2] = {nullptr, nullptr};   // prolongation from the next level (this level's rows)
  rb_op* PT[2] = {nullptr, nullptr};  // its transpose (the next level's rows)
  rb_op* S32 = nullptr;               // -L matrix-free in FP32 (the FP32 cycle's operator)
  rb_op* S64 = nullptr;               // -L matrix-free in FP64 (line smoothing of the FP64 cycle)
  void* line_mem = nullptr;           // line smoothing: c_j and 1 / den_j per cell, FP64 then FP32
  double *lc64 = nullptr, *lid64 = nullptr, *la64 = nullptr;
  float *lc32 = nullptr, *lid32 = nullptr, *la32 = nullptr;
  // matrix-free transfers to the next level: per-axis 1-D maps (FP32)
  rb::PAxis<float>* pa32[3] = {nullptr, nullptr, nullptr};
  rb::TAxisTab<float>* ta32[3] = {nullptr, nullptr, nullptr};
  void* tab_mem = nullptr;  // one allocation holding the transfer tables (both precisions)
  // level vectors, n x k_max doubles each (used as FP32 by the FP32 cycle)
  void *rhs = nullptr, *ea = nullptr, *eb = nullptr, *res = nullptr, *out = nullptr;
};

struct rb_mg {
  int L = 0, k_max = 1;
  int line_axis = -1;  // axis of the line smoother, -1: point Jacobi
  rb_mg_params prm{};
  std::vector<rb_mg_level> lv;
  int nc = 0;              // coarsest cells
  double* ainv = nullptr;  // its dense inverse (nc x nc)
  // solve vectors (n0 x k_max doubles each): the FP64 solution and residual, and the CG's
  // x, r, p, q, z (FP64 for mixed = 0, FP32 for a refinement sweep)
  double *x64 = nullptr, *rt = nullptr;
  void *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr;
  rb::MgScal* sc = nullptr;
  double* partials = nullptr;
  int64_t device_bytes = 0;
  // CUDA graphs of check_every CG iterations, per (precision, k, chunk, flexible)
  std::map<std::vector<int>, cudaGraphExec_t> graphs;
  cudaStream_t cap = nullptr;  // private stream for graph capture
};

namespace rb {
namespace {

constexpr int kMgPartials = 4 * K * kMaxGrid;  // 4 quantities x k columns x blocks

template <typename T>
rb_status mg_alloc(rb_mg* g, T** p, size_t count) {
  void* q = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16) + 64;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  e = cudaMemset(q, 0, bytes);
  if (e != cudaSuccess) {
    cudaFree(q);
    return cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
  }
  *p = static_cast<T*>(q);
  g->device_bytes += (int64_t)bytes;
  return RB_OK;
}

void mg_free(rb_mg* g) {
  if (!g) return;
  for (auto& l : g->lv) {
    for (int d = 0; d < 2; ++d) {
      if (l.A[d]) rb_operator_destroy(l.A[d]);
      if (l.P[d]) rb_operator_destroy(l.P[d]);
      if (l.PT[d]) rb_operator_destroy(l.PT[d]);
    }
    if (l.S32) rb_operator_destroy(l.S32);
    if (l.S64) rb_operator_destroy(l.S64);
    for (void* p : {l.rhs, l.ea, l.eb, l.res, l.out, l.tab_mem, l.line_mem})
      if (p) cudaFree(p);
  }
  for (void* p : {(void*)g->ainv, (void*)g->x64, (void*)g->rt, g->x, g->r, g->p, g->q, g->z, (void*)g->sc,
                  (void*)g->partials})
    if (p) cudaFree(p);
  for (auto& kv : g->graphs)
    if (kv.second) cudaGraphExecDestroy(kv.second);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

// An operator from a device CSR (the library copies it), in both precisions
rb_status make_ops(int nr, int nc, int64_t nnz, const int32_t* rp, const int32_t* ci, const double* va, int k_max,
                   cudaStream_t s, rb_op* out[2]) {
  rb_csr_desc d{nr, nc, nnz, rp, ci, va, 1};
  rb_block_desc b{k_max, 0, nullptr, 0.0};
  RB_TRY(rb_operator_create(&d, &b, RB_F64, RB_CSR, s, &out[0]));
  RB_TRY(rb_operator_create(&d, &b, RB_F32, RB_CSR, s, &out[1]));
  return RB_OK;
}

struct DevCsr {
  int32_t *rp = nullptr, *ci = nullptr;
  double* va = nullptr;
  ~DevCsr() {
    if (rp) cudaFree(rp);
    if (ci) cudaFree(ci);
    if (va) cudaFree(va);
  }
  rb_status alloc(int64_t rows, int64_t nnz) {
    RB_CUDA(cudaMalloc(&rp, (size_t)(rows + 1) * 4 + 64));
    RB_CUDA(cudaMalloc(&ci, (size_t)std::max<int64_t>(nnz, 1) * 4 + 64));
    RB_CUDA(cudaMalloc(&va, (size_t)std::max<int64_t>(nnz, 1) * 8 + 64));
    return RB_OK;
  }
};

LineGeom line_geom(const rb_mg_level& lv, int axis) {
  LineGeom lg{};
  lg.axis = axis;
  lg.len = lv.n[axis];
  lg.stride = axis == 0 ? 1 : (axis == 1 ? lv.n[0] : lv.n[0] * lv.n[1]);
  lg.inner = lg.stride;
  lg.nlines = (int)(lv.cells / lg.len);
  lg.div_inner.init((uint32_t)lg.stride);
  return lg;
}

Stencil7<double> stencil_view64(const rb_op* op) {
  Stencil7<double> v{};
  for (int d = 0; d < 3; ++d) {
    v.n[d] = op->st_n[d];
    v.per[d] = op->st_per[d];
    v.w[d] = static_cast<const double*>(op->st_w[d]);
    v.ic[d] = static_cast<const double*>(op->st_ic[d]);
  }
  v.scale = op->st_scale;
  v.init_div();
  return v;
}

// The line smoother's axis: the wall-bounded axis whose couplings exceed the others' most,
// if by a factor >= 4 somewhere (coupling across a face ~ 1 / width^2 relative to the cell:
// (largest width of the other axes / smallest width of this one)^2); -1 for none
int choose_line_axis(const rb_grid_desc* grid) {
  double mn[3], mx[3];
  for (int d = 0; d < 3; ++d) {
    std::vector<double> h(grid->n[d] + 1);
    if (cudaMemcpy(h.data(), grid->nodes[d], sizeof(double) * h.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    mn[d] = 1e300, mx[d] = 0.0;
    for (int t = 0; t < grid->n[d]; ++t) {
      const double w = h[t + 1] - h[t];
      mn[d] = std::min(mn[d], w), mx[d] = std::max(mx[d], w);
    }
  }
  int best = -1;
  double worst = 1.0;
  for (int d = 0; d < 3; ++d) {
    if (grid->periodic[d]) continue;
    double other = 0.0;
    for (int e = 0; e < 3; ++e)
      if (e != d) other = std::max(other, mx[e]);
    const double r = (other / mn[d]) * (other / mn[d]);
    if (r > worst) best = d, worst = r;
  }
  return worst >= 4.0 ? best : -1;
}

rb_status build_hierarchy(rb_mg* g, const rb_grid_desc* grid, cudaStream_t s) {
  std::vector<std::vector<double*>> nodes;  // per level, per axis (level 0: the caller's)
  struct NodeGuard {
    std::vector<double*> own;
    ~NodeGuard() {
      for (double* p : own) cudaFree(p);
    }
  } guard;
  rb_grid_desc cur = *grid;
  const int mc = g->prm.min_cells;
  for (int l = 0;; ++l) {
    rb_mg_level lv;
    for (int d = 0; d < 3; ++d) lv.n[d] = cur.n[d];
    lv.cells = (int64_t)cur.n[0] * cur.n[1] * cur.n[2];
    // -L on this level, both precisions
    int32_t nr = 0, ncol = 0;
    int64_t nnz = 0;
    RB_TRY(rb_fvm_csr_size(&cur, RB_FVM_LAPLACIAN, &nr, &ncol, &nnz));
    {
      DevCsr t;
      RB_TRY(t.alloc(nr, nnz));
      RB_TRY(rb_fvm_assemble(&cur, RB_FVM_LAPLACIAN, -1.0, t.rp, t.ci, t.va, reinterpret_cast<rb_stream_t>(s)));
      RB_TRY(make_ops(nr, ncol, nnz, t.rp, t.ci, t.va, g->k_max, s, lv.A));
    }
    RB_TRY(rb_fvm_stencil_create(&cur, -1.0, RB_F32, g->k_max, reinterpret_cast<rb_stream_t>(s), &lv.S32));
    if (g->line_axis >= 0) {  // the line smoother's factors (every level but a one-cell line)
      RB_TRY(rb_fvm_stencil_create(&cur, -1.0, RB_F64, g->k_max, reinterpret_cast<rb_stream_t>(s), &lv.S64));
      const size_t cells = (size_t)lv.cells;
      RB_TRY(mg_alloc(g, reinterpret_cast<char**>(&lv.line_mem), cells * 36 + 256));
      char* q = static_cast<char*>(lv.line_mem);
      lv.lc64 = reinterpret_cast<double*>(q);
      lv.lid64 = lv.lc64 + cells;
      lv.la64 = lv.lid64 + cells;
      lv.lc32 = reinterpret_cast<float*>(lv.la64 + cells);
      lv.lid32 = lv.lc32 + cells;
      lv.la32 = lv.lid32 + cells;
      const LineGeom lg = line_geom(lv, g->line_axis);
      Stencil7<double> v = stencil_view64(lv.S64);
      k_line_factors<<<std::max(1, std::min((lg.nlines + 127) / 128, kMaxGrid)), 128, 0, s>>>(
          v, lg, lv.lc64, lv.lid64, lv.la64, lv.lc32, lv.lid32, lv.la32);
      RB_CUDA(cudaGetLastError());
    }
    bool coarsen = l + 1 < kMgMaxLevels;
    for (int d = 0; d < 3; ++d) coarsen = coarsen && cur.n[d] % 2 == 0 && cur.n[d] / 2 >= mc;
    if (coarsen) {
      const int64_t nf = lv.cells, ncoarse = nf / 8;
      DevCsr t;
      RB_TRY(t.alloc(nf, 8 * nf));
      RB_TRY(rb_refine_assemble(&cur, RB_REFINE_PROLONG, t.rp, t.ci, t.va, reinterpret_cast<rb_stream_t>(s)));
      RB_TRY(make_ops((int)nf, (int)ncoarse, 8 * nf, t.rp, t.ci, t.va, g->k_max, s, lv.P));
      RB_TRY(rb_refine_assemble(&cur, RB_REFINE_PROLONG_T, t.rp, t.ci, t.va, reinterpret_cast<rb_stream_t>(s)));
      RB_TRY(make_ops((int)ncoarse, (int)nf, 8 * nf, t.rp, t.ci, t.va, g->k_max, s, lv.PT));
      // per-axis transfer tables, FP64 and FP32, in one allocation
      size_t bytes = 0;
      for (int d = 0; d < 3; ++d)
        bytes += (sizeof(PAxis<double>) + sizeof(PAxis<float>)) * cur.n[d] +
                 (sizeof(TAxisTab<double>) + sizeof(TAxisTab<float>)) * (cur.n[d] / 2) + 64;
      RB_TRY(mg_alloc(g, reinterpret_cast<char**>(&lv.tab_mem), bytes));
      char* q = static_cast<char*>(lv.tab_mem);
      PAxis<double>* pa64[3];
      TAxisTab<double>* ta64[3];
      auto carve = [&q](size_t b) {
        char* r = q;
        q += (b + 15) & ~(size_t)15;
        return r;
      };
      for (int d = 0; d < 3; ++d) {
        pa64[d] = reinterpret_cast<PAxis<double>*>(carve(sizeof(PAxis<double>) * cur.n[d]));
        ta64[d] = reinterpret_cast<TAxisTab<double>*>(carve(sizeof(TAxisTab<double>) * (cur.n[d] / 2)));
        lv.pa32[d] = reinterpret_cast<PAxis<float>*>(carve(sizeof(PAxis<float>) * cur.n[d]));
        lv.ta32[d] = reinterpret_cast<TAxisTab<float>*>(carve(sizeof(TAxisTab<float>) * (cur.n[d] / 2)));
      }
      RB_TRY(transfer_tables(&cur, pa64, ta64, lv.pa32, lv.ta32, s));
    }
    // level vectors (the finest level's right-hand side and output are the solve's r and z)
    const size_t cnt = (size_t)lv.cells * g->k_max;
    RB_TRY(mg_alloc(g, reinterpret_cast<double**>(&lv.ea), cnt));
    RB_TRY(mg_alloc(g, reinterpret_cast<double**>(&lv.eb), cnt));
    RB_TRY(mg_alloc(g, reinterpret_cast<double**>(&lv.res), cnt));
    RB_TRY(mg_alloc(g, reinterpret_cast<double**>(&lv.rhs), cnt));
    RB_TRY(mg_alloc(g, reinterpret_cast<double**>(&lv.out), cnt));
    g->lv.push_back(lv);
    if (!coarsen) break;
    rb_grid_desc nxt = cur;
    for (int d = 0; d < 3; ++d) {
      nxt.n[d] = cur.n[d] / 2;
      double* p = nullptr;
      RB_CUDA(cudaMalloc(&p, sizeof(double) * (nxt.n[d] + 1)));
      guard.own.push_back(p);
      k_every_other<<<(nxt.n[d] + 1 + 127) / 128, 128, 0, s>>>(nxt.n[d] + 1, cur.nodes[d], p);
      RB_CUDA(cudaGetLastError());
      nxt.nodes[d] = p;
    }
    cur = nxt;
  }
  g->L = (int)g->lv.size();
  // the coarsest level's dense inverse
  const rb_mg_level& co = g->lv.back();
  g->nc = (int)co.cells;
  RB_REQUIRE(g->nc <= kMgMaxCoarse,
             "rb_mg_create: the coarsest level has %d cells (more than %d): an axis of the grid does not halve to "
             "an even count >= 2 min_cells often enough", g->nc, kMgMaxCoarse);
  RB_TRY(mg_alloc(g, &g->ainv, (size_t)g->nc * g->nc));
  double* col = nullptr;
  RB_CUDA(cudaMalloc(&col, sizeof(double) * g->nc));
  const rb_op* A0 = co.A[0];
  k_dense_from_csr<<<std::min(g->nc, 1024), 128, 0, s>>>(g->nc, A0->row_ptr, A0->col_idx,
                                                         static_cast<const double*>(A0->vals), g->ainv);
  k_dense_shift<<<1, kThreads, 0, s>>>(g->nc, g->ainv);
  const int ug = (int)std::min<int64_t>(((int64_t)g->nc * g->nc + kThreads - 1) / kThreads, kMaxGrid);
  for (int p = 0; p < g->nc; ++p) {
    k_gj_pivot<<<1, kThreads, 0, s>>>(g->nc, p, g->ainv, col);
    k_gj_update<<<ug, kThreads, 0, s>>>(g->nc, p, g->ainv, col);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(col);
  if (e != cudaSuccess) return cuda_fail(e, "coarsest-level inverse", __FILE__, __LINE__);
  return RB_OK;
}

// ------------------------------------------------------------------------ the cycle

template <typename T>
CsrArgs<T> csr_args(const rb_op* op, const void* X, void* Y, int k, int kp) {
  CsrArgs<T> a;
  a.n_rows = op->n_rows;
  a.rp = op->row_ptr;
  a.ci = op->col_idx;
  a.va = static_cast<const T*>(op->vals);
  a.X = static_cast<const T*>(X);
  a.ldx = k;
  a.Y = static_cast<T*>(Y);
  a.ldy = k;
  a.k = k;
  a.kp = kp;
  return a;
}

template <typename T>
const T* dinv_of(const rb_op* op) {
  if constexpr (sizeof(T) == 8) return op->dinv64;
  else return op->dinv32;
}

template <typename T, int VEC>
struct Cycle {
  const rb_mg* g;
  int k, kp;
  cudaStream_t s;
  const int* gate = nullptr;  // the solve's count of iterating columns (kernels skip at 0)
  int ti() const { return sizeof(T) == 8 ? 0 : 1; }

  template <typename Kern>
  int grid(Kern* kern, int64_t rows) const {
    return wave_grid(kern, (rows + kThreads / kp - 1) / (kThreads / kp));
  }

  // the FP32 cycle runs matrix-free (stencil7.cuh) unless the hierarchy was built otherwise
  bool mf() const { return sizeof(T) == 4 && g->prm.matrix_free; }

  static Stencil7<T> st_view(const rb_op* op) {
    Stencil7<T> v{};
    if (op) {
      for (int d = 0; d < 3; ++d) {
        v.n[d] = op->st_n[d];
        v.per[d] = op->st_per[d];
        v.w[d] = static_cast<const T*>(op->st_w[d]);
        v.ic[d] = static_cast<const T*>(op->st_ic[d]);
      }
      v.scale = (T)op->st_scale;
      v.init_div();
    }
    return v;
  }

  Transfer3<T> tr_view(const rb_mg_level& lv) const {
    Transfer3<T> t{};
    if constexpr (sizeof(T) == 4) {
      for (int d = 0; d < 3; ++d) {
        t.nf[d] = lv.n[d];
        t.pa[d] = lv.pa32[d];
        t.ta[d] = lv.ta32[d];
      }
      t.init_div();
    }
    return t;
  }

  // one product-shaped pass over a level (CSR or matrix-free)
  template <int MODE, bool DOTS>
  void sweep(const rb_mg_level& lv, const T* e, const T* r, const T* dinv, T* out, const MgDots& dd) const {
    const T omega = (T)g->prm.omega;
    if (mf()) {
      auto* kern = &k_mg_sweep<T, VEC, MODE, DOTS, true>;
      kern<<<grid(kern, lv.cells), kThreads, 0, s>>>(csr_args<T>(lv.S32, e, nullptr, k, kp), st_view(lv.S32), r, dinv,
                                                     omega, out, dd, gate);
    } else {
      auto* kern = &k_mg_sweep<T, VEC, MODE, DOTS, false>;
      kern<<<grid(kern, lv.cells), kThreads, 0, s>>>(csr_args<T>(lv.A[ti()], e, nullptr, k, kp), st_view(nullptr), r,
                                                     dinv, omega, out, dd, gate);
    }
  }

  // one line sweep over a level (the FP32 or FP64 tables of its operator)
  template <int MODE, bool DOTS>
  void line(const rb_mg_level& lv, const T* e, const T* r, T* out, const MgDots& dd) const {
    const LineGeom lg = line_geom(lv, g->line_axis);
    const T* cf;
    const T* id;
    const T* ac;
    const rb_op* op;
    if constexpr (sizeof(T) == 4) cf = lv.lc32, id = lv.lid32, ac = lv.la32, op = lv.S32;
    else cf = lv.lc64, id = lv.lid64, ac = lv.la64, op = lv.S64;
    auto* kern = &k_mg_line<T, VEC, MODE, DOTS>;
    const int lines_per_block = 32 / kp;
    const int blocks = wave_grid(kern, (lg.nlines + lines_per_block - 1) / lines_per_block);
    kern<<<blocks, kThreads, 0, s>>>(st_view(op), lg, k, kp, e, r, cf, id, ac, (T)g->prm.omega, out, dd, gate);
  }

  // z = B r on level l (r, z: n_l x k blocks of T, ld = k); dd: dots of the last sweep
  rb_status run(int l, const T* r, T* z, const MgDots* dd) const {
    const rb_mg_level& lv = g->lv[l];
    const T omega = (T)g->prm.omega;
    const int nu = g->prm.nu;
    if (l == g->L - 1) {
      k_mg_coarse<T><<<g->nc, kThreads, 0, s>>>(g->nc, k, g->ainv, r, z, gate);
      RB_CUDA(cudaGetLastError());
      RB_REQUIRE(dd == nullptr, "rb_mg: a one-level hierarchy cannot precondition CG (the grid does not coarsen)");
      return RB_OK;
    }
    const T* dinv = dinv_of<T>(mf() ? lv.S32 : lv.A[ti()]);
    T* bufs[2] = {static_cast<T*>(lv.ea), static_cast<T*>(lv.eb)};
    int c = 0;
    MgDots none;
    if (g->line_axis >= 0) {
      line<LN_ZERO, false>(lv, nullptr, r, bufs[0], none);
      for (int it = 1; it < nu; ++it, c ^= 1) line<LN_JACOBI, false>(lv, bufs[c], r, bufs[c ^ 1], none);
    } else {
      k_mg_smooth0<T, VEC><<<grid(&k_mg_smooth0<T, VEC>, lv.cells), kThreads, 0, s>>>(lv.cells, k, kp, r, dinv, omega,
                                                                                       bufs[0], gate);
      for (int it = 1; it < nu; ++it, c ^= 1) sweep<SW_JACOBI, false>(lv, bufs[c], r, dinv, bufs[c ^ 1], none);
    }
    // residual, restriction, the next level, prolongation-add
    sweep<SW_RESID, false>(lv, bufs[c], r, dinv, static_cast<T*>(lv.res), none);
    const rb_mg_level& nx = g->lv[l + 1];
    if (mf()) {
      auto* rk = &k_mg_restrict_st<T, VEC>;
      rk<<<grid(rk, nx.cells), kThreads, 0, s>>>(tr_view(lv), nx.cells, k, kp, static_cast<const T*>(lv.res),
                                                static_cast<T*>(nx.rhs), gate);
    } else {
      const rb_op* PT = lv.PT[ti()];
      RB_TRY(spmm_launch(PT, pick_sched(PT, k, k, k, lv.res, nx.rhs), lv.res, k, nx.rhs, k, k, nullptr, s));
    }
    RB_TRY(run(l + 1, static_cast<const T*>(nx.rhs), static_cast<T*>(nx.out), nullptr));
    if (mf()) {
      auto* pk = &k_mg_prolong_st<T, VEC>;
      pk<<<grid(pk, lv.cells), kThreads, 0, s>>>(tr_view(lv), lv.cells, k, kp, static_cast<const T*>(nx.out), bufs[c],
                                                gate);
    } else {
      auto* pk = &k_mg_prolong_add<T, VEC>;
      pk<<<grid(pk, lv.cells), kThreads, 0, s>>>(csr_args<T>(lv.P[ti()], nx.out, bufs[c], k, kp), gate);
    }
    for (int it = 1; it <= nu; ++it, c ^= 1) {
      T* dst = (it == nu) ? z : bufs[c ^ 1];
      if (g->line_axis >= 0) {
        if (it == nu && dd) line<LN_JACOBI, true>(lv, bufs[c], r, dst, *dd);
        else line<LN_JACOBI, false>(lv, bufs[c], r, dst, none);
      } else {
        if (it == nu && dd) sweep<SW_JACOBI, true>(lv, bufs[c], r, dinv, dst, *dd);
        else sweep<SW_JACOBI, false>(lv, bufs[c], r, dinv, dst, none);
      }
    }
    RB_CUDA(cudaGetLastError());
    return RB_OK;
  }
};

// One CG iteration (after the initial z and p): q = A p, x, r update, z = B r, p = z + beta p
template <typename T, int VEC>
rb_status cg_iteration(const rb_mg* g, const Cycle<T, VEC>& cy, bool inner, int flexible) {
  const int k = cy.k, kp = cy.kp;
  const rb_mg_level& l0 = g->lv[0];
  const int64_t n = l0.cells;
  const rb_op* A = l0.A[cy.ti()];
  T* x = static_cast<T*>(g->x);
  T* r = static_cast<T*>(g->r);
  T* p = static_cast<T*>(g->p);
  T* q = static_cast<T*>(g->q);
  T* z = static_cast<T*>(g->z);
  cudaStream_t s = cy.s;
  if (cy.mf()) {
    auto* kq = &k_mgcg_q<T, VEC, true>;
    kq<<<cy.grid(kq, n), kThreads, 0, s>>>(csr_args<T>(l0.S32, p, q, k, kp), Cycle<T, VEC>::st_view(l0.S32), g->sc,
                                           g->partials);
  } else {
    auto* kq = &k_mgcg_q<T, VEC, false>;
    kq<<<cy.grid(kq, n), kThreads, 0, s>>>(csr_args<T>(A, p, q, k, kp), Cycle<T, VEC>::st_view(nullptr), g->sc,
                                           g->partials);
  }
  if (inner) {
    auto* kx = &k_mgcg_xr<T, VEC, true>;
    kx<<<cy.grid(kx, n), kThreads, 0, s>>>(n, k, kp, x, r, p, q, g->sc, g->partials);
  } else {
    auto* kx = &k_mgcg_xr<T, VEC, false>;
    kx<<<cy.grid(kx, n), kThreads, 0, s>>>(n, k, kp, x, r, p, q, g->sc, g->partials);
  }
  MgDots dd;
  dd.sc = g->sc;
  dd.partials = g->partials;
  dd.q = q;
  dd.init = 0;
  dd.flexible = flexible;
  RB_TRY(cy.run(0, r, z, &dd));
  auto* kp_ = &k_mgcg_p<T, VEC, false>;
  kp_<<<cy.grid(kp_, n), kThreads, 0, s>>>(n, k, kp, z, p, g->sc);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

// z = B r and p = z (the start of a solve or of a refinement sweep)
template <typename T, int VEC>
rb_status cg_start(const rb_mg* g, const Cycle<T, VEC>& cy) {
  MgDots dd;
  dd.sc = g->sc;
  dd.partials = g->partials;
  dd.init = 1;
  RB_TRY(cy.run(0, static_cast<const T*>(g->r), static_cast<T*>(g->z), &dd));
  const int64_t n = g->lv[0].cells;
  auto* kp_ = &k_mgcg_p<T, VEC, true>;
  kp_<<<cy.grid(kp_, n), kThreads, 0, cy.s>>>(n, cy.k, cy.kp, static_cast<const T*>(g->z), static_cast<T*>(g->p),
                                             g->sc);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

struct MgHost {
  int n_active = 0, n_oactive = 0;
};

rb_status mg_read(rb_mg* g, MgHost& h, cudaStream_t s) {
  RB_CUDA(cudaMemcpyAsync(&h.n_active, &g->sc->n_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  return RB_OK;
}

// `chunk` CG iterations, recorded once per shape as a CUDA graph and replayed
template <typename T, int VEC>
rb_status run_iterations(rb_mg* g, const Cycle<T, VEC>& cy, bool inner, int flexible, int chunk, int& uses) {
  const std::vector<int> key = {(int)sizeof(T), cy.k, chunk, flexible, inner ? 1 : 0};
  auto it = g->graphs.find(key);
  if (it == g->graphs.end() && uses == 0) {  // the first chunk runs eagerly (launch caches fill)
    for (int i = 0; i < chunk; ++i) RB_TRY((cg_iteration<T, VEC>(g, cy, inner, flexible)));
    ++uses;
    return RB_OK;
  }
  if (it == g->graphs.end()) {
    if (!g->cap) RB_CUDA(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
    Cycle<T, VEC> cc = cy;
    cc.s = g->cap;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    RB_CUDA(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    rb_status st = RB_OK;
    for (int i = 0; i < chunk && st == RB_OK; ++i) st = cg_iteration<T, VEC>(g, cc, inner, flexible);
    cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
    if (st != RB_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "CUDA graph of the multigrid CG iterations", __FILE__, __LINE__);
    it = g->graphs.emplace(key, exec).first;
  }
  RB_CUDA(cudaGraphLaunch(it->second, cy.s));
  ++uses;
  return RB_OK;
}

template <int VEC>
rb_status true_resid(rb_mg* g, const double* B, int64_t ldb, const double* X, double* out, int kind, int k, int kp,
                     const rb_cg_params& prm, cudaStream_t s) {
  const rb_op* A = g->lv[0].A[0];
  auto* kern = &k_mg_true_resid<VEC>;
  const int64_t n = g->lv[0].cells;
  const int grid = wave_grid(kern, (n + kThreads / kp - 1) / (kThreads / kp));
  kern<<<grid, kThreads, 0, s>>>(csr_args<double>(A, X, nullptr, k, kp), B, ldb, out, kind, prm.project_mean,
                                 prm.rtol * prm.rtol, g->sc, g->partials);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <int VEC64, int VEC32>
rb_status mg_solve_vec(rb_mg* g, const rb_cg_params& prm, const double* B, int64_t ldb, double* X, int64_t ldx, int k,
                       rb_cg_report& rep, cudaStream_t s) {
  const rb_mg_level& l0 = g->lv[0];
  const int64_t n = l0.cells;
  const int kp64 = next_pow2(k / VEC64), kp32 = next_pow2(k / VEC32);
  const int flexible = g->prm.flexible;
  const int cg = (int)std::min<int64_t>((n * k + 255) / 256, kMaxGrid);
  int syncs = 0, spmm64 = 0, sweeps = 0, uses = 0;
  MgHost h;
  const int check = std::max(1, prm.check_every);
  if (!prm.mixed) {
    Cycle<double, VEC64> cy{g, k, kp64, s, &g->sc->n_active};
    double* x = static_cast<double*>(g->x);
    k_mg_copy<double, double><<<cg, 256, 0, s>>>(n, k, X, ldx, x, k);
    RB_TRY(true_resid<VEC64>(g, B, ldb, x, g->rt, TR_INIT, k, kp64, prm, s));
    ++spmm64;
    auto* kr = &k_mg_rhs<double, VEC64, 0>;
    kr<<<cy.grid(kr, n), kThreads, 0, s>>>(n, k, kp64, g->rt, static_cast<double*>(g->r), g->sc, 0.0, prm.rtol);
    RB_TRY((cg_start<double, VEC64>(g, cy)));
    int it = 0;
    for (;;) {
      RB_TRY(mg_read(g, h, s));
      ++syncs;
      if (h.n_oactive == 0) break;
      if (it >= prm.max_iter) {
        k_mg_mark_noconv<<<1, K, 0, s>>>(g->sc, k);
        break;
      }
      const int chunk = std::min(check, prm.max_iter - it);
      RB_TRY((run_iterations<double, VEC64>(g, cy, false, flexible, chunk, uses)));
      it += chunk;
      RB_TRY(true_resid<VEC64>(g, B, ldb, x, g->rt, TR_CHECK, k, kp64, prm, s));
      ++spmm64;
    }
    if (prm.project_mean) {
      k_mg_colsum<VEC64><<<cy.grid(&k_mg_colsum<VEC64>, n), kThreads, 0, s>>>(n, k, kp64, x, g->sc, g->partials);
      k_mg_submean<VEC64><<<cy.grid(&k_mg_submean<VEC64>, n), kThreads, 0, s>>>(n, k, kp64, x, g->sc);
    }
    k_mg_copy<double, double><<<cg, 256, 0, s>>>(n, k, x, k, X, ldx);
  } else {
    Cycle<float, VEC32> cy{g, k, kp32, s, &g->sc->n_active};
    double* x64 = g->x64;
    k_mg_copy<double, double><<<cg, 256, 0, s>>>(n, k, X, ldx, x64, k);
    int total_inner = 0;
    for (;; ++sweeps) {
      RB_TRY(true_resid<VEC64>(g, B, ldb, x64, g->rt, sweeps == 0 ? TR_INIT : TR_CHECK, k, kp64, prm, s));
      ++spmm64;
      RB_TRY(mg_read(g, h, s));
      ++syncs;
      if (h.n_oactive == 0) break;
      if (sweeps >= prm.max_sweeps || total_inner >= prm.max_iter) {
        k_mg_mark_noconv<<<1, K, 0, s>>>(g->sc, k);
        break;
      }
      RB_CUDA(cudaMemsetAsync(g->x, 0, sizeof(float) * (size_t)n * k, s));
      auto* kr = &k_mg_rhs<float, VEC32, 1>;
      kr<<<cy.grid(kr, n), kThreads, 0, s>>>(n, k, kp32, g->rt, static_cast<float*>(g->r), g->sc, prm.inner_rtol,
                                            prm.rtol);
      RB_TRY((cg_start<float, VEC32>(g, cy)));
      int it = 0;
      for (;;) {
        RB_TRY(mg_read(g, h, s));
        ++syncs;
        if (h.n_active == 0 || total_inner + it >= prm.max_iter) break;
        const int chunk = std::min(check, prm.max_iter - total_inner - it);
        RB_TRY((run_iterations<float, VEC32>(g, cy, true, flexible, chunk, uses)));
        it += chunk;
      }
      total_inner += it;
      auto* ka = &k_mg_refine_add<VEC32>;
      ka<<<cy.grid(ka, n), kThreads, 0, s>>>(n, k, kp32, x64, static_cast<const float*>(g->x), g->sc);
      RB_CUDA(cudaGetLastError());
    }
    if (prm.project_mean) {
      auto* kc = &k_mg_colsum<VEC64>;
      kc<<<wave_grid(kc, (n + kThreads / kp64 - 1) / (kThreads / kp64)), kThreads, 0, s>>>(n, k, kp64, x64, g->sc,
                                                                                           g->partials);
      auto* km = &k_mg_submean<VEC64>;
      km<<<wave_grid(km, (n + kThreads / kp64 - 1) / (kThreads / kp64)), kThreads, 0, s>>>(n, k, kp64, x64, g->sc);
    }
    k_mg_copy<double, double><<<cg, 256, 0, s>>>(n, k, x64, k, X, ldx);
  }
  RB_CUDA(cudaGetLastError());
  // report
  MgScal hs;
  RB_CUDA(cudaMemcpyAsync(&hs, g->sc, sizeof(MgScal), cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  ++syncs;
  rb_status worst = RB_OK;
  for (int j = 0; j < k; ++j) {
    rep.iters[j] = hs.iters[j];
    rep.true_rel_res[j] = hs.bb[j] > 0 ? std::sqrt(hs.rr_true[j] / hs.bb[j]) : 0.0;
    int st = RB_OK;
    if (hs.ostate[j] == MG_BREAKDOWN || hs.state[j] == MG_BREAKDOWN) st = RB_EBREAKDOWN;
    else if (hs.ostate[j] != MG_DONE) st = RB_ENOCONV;
    rep.status[j] = st;
    if (st == RB_EBREAKDOWN || (st == RB_ENOCONV && worst == RB_OK)) worst = (rb_status)st;
  }
  rep.spmm_calls = spmm64;
  rep.sweeps = sweeps;
  rep.host_syncs = syncs;
  if (worst != RB_OK) set_error("rb_mg_solve: a column did not converge (see the report's per-column status)");
  return worst;
}

template <int V64>
rb_status mg_solve_v32(rb_mg* g, int v32, const rb_cg_params& prm, const double* B, int64_t ldb, double* X, int64_t ldx,
                       int k, rb_cg_report& rep, cudaStream_t s) {
  switch (v32) {
    case 1: return mg_solve_vec<V64, 1>(g, prm, B, ldb, X, ldx, k, rep, s);
    case 2: return mg_solve_vec<V64, 2>(g, prm, B, ldb, X, ldx, k, rep, s);
    case 3: return mg_solve_vec<V64, 3>(g, prm, B, ldb, X, ldx, k, rep, s);
    case 4: return mg_solve_vec<V64, 4>(g, prm, B, ldb, X, ldx, k, rep, s);
  }
  set_error("rb_mg_solve: unsupported vector width");
  return RB_EUNSUPPORTED;
}

template <typename T, int VEC>
rb_status vcycle_vec(rb_mg* g, int level, const double* R, int64_t ldr, double* Z, int64_t ldz, int k, cudaStream_t s) {
  const rb_mg_level& lv = g->lv[level];
  const int64_t n = lv.cells;
  const int cg = (int)std::min<int64_t>((n * k + 255) / 256, kMaxGrid);
  // the level's right-hand side and output in the library's layout and the cycle's type
  T* r = static_cast<T*>(level == 0 ? g->r : lv.rhs);
  T* z = static_cast<T*>(level == 0 ? g->z : lv.out);
  k_mg_copy<double, T><<<cg, 256, 0, s>>>(n, k, R, ldr, r, k);
  Cycle<T, VEC> cy{g, k, next_pow2(k / VEC), s};
  RB_TRY(cy.run(level, r, z, nullptr));
  k_mg_copy<T, double><<<cg, 256, 0, s>>>(n, k, z, k, Z, ldz);
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

template <typename T>
rb_status vcycle_t(rb_mg* g, int level, const double* R, int64_t ldr, double* Z, int64_t ldz, int k, cudaStream_t s) {
  switch (mg_vec(sizeof(T), k)) {
    case 1: return vcycle_vec<T, 1>(g, level, R, ldr, Z, ldz, k, s);
    case 2: return vcycle_vec<T, 2>(g, level, R, ldr, Z, ldz, k, s);
    case 3: return vcycle_vec<T, 3>(g, level, R, ldr, Z, ldz, k, s);
    case 4: return vcycle_vec<T, 4>(g, level, R, ldr, Z, ldz, k, s);
  }
  set_error("rb_mg_vcycle: unsupported vector width");
  return RB_EUNSUPPORTED;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_mg_create(const rb_grid_desc* grid, int32_t k_max, const rb_mg_params* params,
                                  rb_stream_t stream, rb_mg_t* out) {
  clear_error();
  RB_REQUIRE(grid && out, "rb_mg_create: null argument");
  *out = nullptr;
  RB_REQUIRE(k_max >= 1 && k_max <= RB_MAX_K, "rb_mg_create: k_max %d outside [1, %d]", k_max, RB_MAX_K);
  rb_mg_params prm{2, 0.8, 4, 1, 1, 1};
  if (params) prm = *params;
  RB_REQUIRE(prm.nu >= 1 && prm.nu <= 16, "rb_mg_create: nu = %d outside [1, 16]", prm.nu);
  RB_REQUIRE(prm.omega > 0.0 && prm.omega <= 1.0, "rb_mg_create: omega = %g outside (0, 1]", prm.omega);
  RB_REQUIRE(prm.min_cells >= 2, "rb_mg_create: min_cells = %d (at least 2)", prm.min_cells);
  RB_REQUIRE(prm.smoother == 0 || prm.smoother == 1, "rb_mg_create: smoother = %d (0 or 1)", prm.smoother);
  for (int d = 0; d < 3; ++d) {
    RB_REQUIRE(grid->nodes[d] != nullptr, "rb_mg_create: null nodes[%d]", d);
    RB_REQUIRE(grid->n[d] >= (grid->periodic[d] ? 3 : 2), "rb_mg_create: axis %d has %d cells", d, grid->n[d]);
  }
  const int64_t n0 = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
  RB_REQUIRE(8 * n0 <= INT32_MAX, "rb_mg_create: grid too large for int32 CSR indexing");
  rb_mg* g = new rb_mg();
  g->k_max = k_max;
  g->prm = prm;
  cudaStream_t s = S(stream);
  g->line_axis = prm.smoother ? choose_line_axis(grid) : -1;
  rb_status st = build_hierarchy(g, grid, s);
  if (st == RB_OK) {
    const size_t cnt = (size_t)n0 * k_max;
    for (void** p : {&g->x, &g->r, &g->p, &g->q, &g->z})
      if (st == RB_OK) st = mg_alloc(g, reinterpret_cast<double**>(p), cnt);
    if (st == RB_OK) st = mg_alloc(g, &g->x64, cnt);
    if (st == RB_OK) st = mg_alloc(g, &g->rt, cnt);
    if (st == RB_OK) st = mg_alloc(g, &g->sc, 1);
    if (st == RB_OK) st = mg_alloc(g, &g->partials, (size_t)kMgPartials);
  }
  if (st != RB_OK) {
    const std::string msg = rb_last_error();
    mg_free(g);
    set_error("%s", msg.c_str());
    return st;
  }
  for (auto& l : g->lv)
    for (int d = 0; d < 2; ++d) {
      if (l.A[d]) g->device_bytes += l.A[d]->device_bytes;
      if (l.P[d]) g->device_bytes += l.P[d]->device_bytes;
      if (l.PT[d]) g->device_bytes += l.PT[d]->device_bytes;
    }
  *out = g;
  return RB_OK;
}

extern "C" rb_status rb_mg_destroy(rb_mg_t mg) {
  clear_error();
  mg_free(mg);
  return RB_OK;
}

extern "C" rb_status rb_mg_info(rb_mg_t mg, rb_mg_info_t* info) {
  clear_error();
  RB_REQUIRE(mg && info, "rb_mg_info: null argument");
  std::memset(info, 0, sizeof(*info));
  info->levels = mg->L;
  for (int l = 0; l < mg->L && l < RB_MG_MAX_LEVELS; ++l) {
    for (int d = 0; d < 3; ++d) info->n[l][d] = mg->lv[l].n[d];
    info->nnz_A[l] = mg->lv[l].A[0]->nnz;
    info->nnz_P[l] = mg->lv[l].P[0] ? mg->lv[l].P[0]->nnz : 0;
  }
  info->device_bytes = mg->device_bytes;
  info->line_axis = mg->line_axis;
  return RB_OK;
}

extern "C" rb_status rb_mg_vcycle(rb_mg_t mg, int32_t level, rb_dtype dtype, const double* R, int64_t ldr, double* Z,
                                  int64_t ldz, int32_t k, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(mg, "rb_mg_vcycle: null hierarchy");
  RB_REQUIRE(level >= 0 && level < mg->L, "rb_mg_vcycle: level %d outside [0, %d)", level, mg->L);
  RB_REQUIRE(dtype == RB_F64 || dtype == RB_F32, "rb_mg_vcycle: unknown dtype %d", (int)dtype);
  RB_REQUIRE(k >= 1 && k <= mg->k_max, "rb_mg_vcycle: k = %d outside [1, k_max = %d]", k, mg->k_max);
  RB_REQUIRE(ldr >= k && ldz >= k, "rb_mg_vcycle: leading dimension smaller than k");
  RB_REQUIRE(R && Z, "rb_mg_vcycle: null R or Z");
  RB_REQUIRE(next_pow2(k / mg_vec(dtype == RB_F64 ? 8 : 4, k)) <= 32, "rb_mg_vcycle: k = %d needs a wider vector", k);
  if (dtype == RB_F64) return vcycle_t<double>(mg, level, R, ldr, Z, ldz, k, S(stream));
  return vcycle_t<float>(mg, level, R, ldr, Z, ldz, k, S(stream));
}

extern "C" rb_status rb_mg_solve(rb_mg_t mg, const rb_cg_params* params, const double* B, int64_t ldb, double* X,
                                 int64_t ldx, int32_t k, rb_cg_report* report, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(mg && params, "rb_mg_solve: null argument");
  RB_REQUIRE(k >= 1 && k <= mg->k_max, "rb_mg_solve: k = %d outside [1, k_max = %d]", k, mg->k_max);
  RB_REQUIRE(ldb >= k && ldx >= k, "rb_mg_solve: leading dimension smaller than k");
  RB_REQUIRE(B && X, "rb_mg_solve: null B or X");
  RB_REQUIRE(mg->L >= 2, "rb_mg_solve: the grid does not coarsen (a one-level hierarchy)");
  RB_REQUIRE(params->rtol > 0 && params->max_iter >= 0, "rb_mg_solve: rtol must be positive, max_iter >= 0");
  const int v64 = mg_vec(8, k), v32 = mg_vec(4, k);
  RB_REQUIRE(next_pow2(k / v64) <= 32 && next_pow2(k / v32) <= 32, "rb_mg_solve: k = %d needs a wider vector", k);
  rb_cg_report rep{};
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = S(stream);
  rb_status st;
  switch (v64) {
    case 1: st = mg_solve_v32<1>(mg, v32, *params, B, ldb, X, ldx, k, rep, s); break;
    case 2: st = mg_solve_v32<2>(mg, v32, *params, B, ldb, X, ldx, k, rep, s); break;
    case 3: st = mg_solve_v32<3>(mg, v32, *params, B, ldb, X, ldx, k, rep, s); break;
    default: set_error("rb_mg_solve: unsupported vector width"); st = RB_EUNSUPPORTED;
  }
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (report) *report = rep;
  return st;
}
