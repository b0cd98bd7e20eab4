// Poisson solve on k columns that share one operator: Jacobi-preconditioned CG per column
// (the pressure solve of the projection method, Sec. 4; k flow states or parameters, Sec. 3),
// and FP32-inner CG inside FP64 iterative refinement.
//
// One FP64 CG iteration is three kernels, each streaming the k interleaved columns once:
//   q  = A p            (SpMM, Algorithm 1)   fused with  pq_j = p_j . q_j
//   x += a p, r -= a q, z = D^-1 r            fused with  rz_j = r_j . z_j,  rr_j = r_j . r_j
//   p  = z + b p        (z recomputed from r; never stored)
// (the inner FP32 solve of the refinement runs a two-kernel form of the same recurrence,
// described at k_cg_q2).  The per-column scalars (alpha = rz/pq, beta = rz_new/rz) are formed
// on the device by the last block of the reducing kernel, so the host only reads the
// per-column state every check_every iterations.  A column whose recurrence residual passes the tolerance is
// checked against its true residual b - A x in FP64; if that fails it restarts from the
// true residual (residual replacement).  Converged columns stop changing.
//
// Mixed precision: the outer loop forms r = b - A x with the FP64 operator, the inner CG
// runs on the FP32 copy of the operator with FP32 vectors (dot products accumulated in
// FP64) on r / ||r||, and x += ||r|| d is applied in FP64.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "reduce.cuh"
#include "spmm_impl.cuh"
#include "stencil7.cuh"

namespace rb {

SpmmSched default_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y);
SpmmSched pick_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y);

namespace {

enum ColState : int {
  ST_ACTIVE = 0,     // iterating
  ST_CHECK = 1,      // recurrence residual passed: true residual pending
  ST_DONE = 2,       // converged (or, for an inner solve, finished)
  ST_BREAKDOWN = 3,  // p.q <= 0 or not finite
  ST_NOCONV = 4,     // iteration budget exhausted
  ST_RESTART = 5,    // restart from the freshly computed true residual
  ST_IDLE = 6        // column takes no part (inner solve of a converged outer column)
};

enum ResidMode : int { RM_INIT = 0, RM_CHECK = 1, RM_REPORT = 2, RM_OUTER = 3 };

constexpr int K = RB_MAX_K;
constexpr int kGridMax = 152 * 8;

struct CgScal {
  double rz[K], pq[K], rr[K], tol2[K], alpha[K], beta[K], mean[K];
  double bb[K], rr_true[K];
  // outer refinement (oprev: the previous sweep's residual norm, 0 before the first sweep)
  double otol2[K], omean[K], oscale[K], oprev[K];
  int ostate[K];
  int state[K], iters[K];
  int n_active, n_check, n_oactive, n_orun;  // n_orun: outer columns not finished (incl. first sweep)
  unsigned counter[8];   // last-block tickets, one per reducing kernel
  unsigned pbar[4];      // persistent solve: barrier arrivals, generation, error word
  int pact[2];           // persistent solve: system still active after iteration it (slot it & 1)
  int met[K];            // inner solve: the column has reached its sweep's target
};

struct CgCtl {
  int k, kp;
  int64_t n;
  int inner;         // 1: inner FP32 solve of the refinement
  int reliable;      // refinement keeps the search direction across sweeps (mixed == 2)
  int project;       // remove column means of true residuals
  double rtol2;      // rtol^2
  double inner_rtol2;
};

// ---------------------------------------------------------------------------------- helpers

// N running dot products in the arithmetic of the solve: FP64 products and sums for the FP64
// solve; for the FP32 inner solve, FP32 products summed in FP32 over the thread's rows (a
// few dozen) and, in block_reduce, over the lanes of a warp, then in FP64 across warps and
// blocks.  FP64 instructions are scarce on this GPU (one warp-wide FP64 instruction holds an
// SM for about 16 cycles), so the FP32 solve keeps them out of its per-row work.
template <typename T, int N>
struct DotAccN {
  T s[N];
  __device__ __forceinline__ DotAccN() {
#pragma unroll
    for (int i = 0; i < N; ++i) s[i] = T(0);
  }
  __device__ __forceinline__ void add(int i, T a, T b) { s[i] = fma(a, b, s[i]); }
  __device__ __forceinline__ void step() {}
  __device__ __forceinline__ T get(int i) const { return s[i]; }
};

__device__ __forceinline__ void recount(CgScal* sc, int k) {
  int na = 0, nc = 0, no = 0, nr = 0;
  for (int j = 0; j < k; ++j) {
    na += sc->state[j] == ST_ACTIVE;
    nc += sc->state[j] == ST_CHECK;
    no += sc->ostate[j] == ST_ACTIVE;
    nr += sc->ostate[j] == ST_ACTIVE || sc->ostate[j] == ST_RESTART;
  }
  sc->n_active = na;
  sc->n_check = nc;
  sc->n_oactive = no;
  sc->n_orun = nr;
}

// ------------------------------------------------------------------------- q = A p, p . q

template <typename T, int VEC, int LPR>
__global__ void __launch_bounds__(kThreads) k_cg_q(CsrArgs<T> a, CgCtl ctl, CgScal* __restrict__ sc,
                                                    double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<1> red;
  const int R = kThreads / (a.kp * LPR);
  const int t = threadIdx.x;
  const int sub = t % LPR, rc = t / LPR, chunk = rc % a.kp, rloc = rc / a.kp;
  DotAccN<T, VEC> dacc;
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
    row_accumulate_direct<T, VEC, LPR, false, true>(a, row, chunk, sub, active, acc);
    if (active && sub == 0) {
      const Vec<T, VEC> p = ldv<T, VEC>(a.X + row * a.ldx + chunk * VEC);
      Vec<T, VEC> q;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        q.v[e] = acc[e];
        dacc.add(e, p.v[e], acc[e]);
      }
      dacc.step();
      stv<T, VEC>(a.Y + row * a.ldy + chunk * VEC, q);
    }
  }
  T part[1][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = (sub == 0) ? dacc.get(e) : T(0);
  const double v = block_reduce<1, VEC>(part, a.kp, LPR, a.k, red);
  if (!publish_partials<1>(v, a.k, partials, &sc->counter[0], red)) return;
  const double tot = final_sum<1>(partials, a.k, gridDim.x, red);
  const int j = threadIdx.x;
  if (j < a.k) {
    sc->pq[j] = tot;
    double al = 0.0;
    if (sc->state[j] == ST_ACTIVE) {
      if (!(tot > 0.0) || !isfinite(tot)) {
        sc->state[j] = ctl.inner ? ST_DONE : ST_BREAKDOWN;
      } else {
        al = sc->rz[j] / tot;
      }
    }
    sc->alpha[j] = al;
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, a.k);
}

// ------------------------------------------- x += a p, r -= a q, rz = r.D^-1 r, rr = r.r

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_cg_update(CgCtl ctl, T* __restrict__ x, int64_t ldx,
                                                         T* __restrict__ r, const T* __restrict__ p,
                                                         const T* __restrict__ q, const T* __restrict__ dinv,
                                                         CgScal* __restrict__ sc, double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const bool col_ok = chunk * VEC < k;
  T al[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) al[e] = col_ok ? (T)sc->alpha[chunk * VEC + e] : T(0);
  DotAccN<T, 2 * VEC> dots;  // [0, VEC): r . D^-1 r, [VEC, 2 VEC): r . r
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
      const int64_t o = row * k + chunk * VEC;
      const Vec<T, VEC> pv = ldv_rw<T, VEC>(p + o);
      const Vec<T, VEC> qv = ldv_rw<T, VEC>(q + o);
      Vec<T, VEC> rv = ldv_rw<T, VEC>(r + o);
      Vec<T, VEC> xv = ldv_rw<T, VEC>(x + row * ldx + chunk * VEC);
      const T d = dinv ? dinv[row] : T(1);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        xv.v[e] = fma(al[e], pv.v[e], xv.v[e]);
        rv.v[e] = fma(-al[e], qv.v[e], rv.v[e]);
        dots.add(e, rv.v[e], d * rv.v[e]);
        dots.add(VEC + e, rv.v[e], rv.v[e]);
      }
      dots.step();
      stv<T, VEC>(x + row * ldx + chunk * VEC, xv);
      stv<T, VEC>(r + o, rv);
    }
  }
  T part[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = dots.get(e), part[1][e] = dots.get(VEC + e);
  const double v = block_reduce<2, VEC>(part, kp, 1, k, red);
  if (!publish_partials<2>(v, 2 * k, partials, &sc->counter[1], red)) return;
  const double tot = final_sum<2>(partials, 2 * k, gridDim.x, red);
  __shared__ double totals[2 * K];
  if ((int)threadIdx.x < 2 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k) {
    const double rz_new = totals[j], rr_new = totals[k + j];
    double be = 0.0;
    if (sc->state[j] == ST_ACTIVE) {
      sc->iters[j] += 1;
      sc->rr[j] = rr_new;
      if (!isfinite(rr_new) || !isfinite(rz_new)) {
        sc->state[j] = ctl.inner ? ST_DONE : ST_BREAKDOWN;
      } else if (rr_new <= sc->tol2[j]) {
        sc->state[j] = ctl.inner ? ST_DONE : ST_CHECK;
      } else {
        be = rz_new / sc->rz[j];
        sc->rz[j] = rz_new;
      }
    }
    sc->beta[j] = be;
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, k);
}

// ------------------------------------------------------------------------ p = D^-1 r + b p

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_cg_p(CgCtl ctl, const T* __restrict__ r, T* __restrict__ p,
                                                    const T* __restrict__ dinv, const CgScal* __restrict__ sc) {
  if (sc->n_active == 0) return;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  T be[VEC];
  bool on[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    be[e] = (T)sc->beta[chunk * VEC + e];
    on[e] = sc->state[chunk * VEC + e] == ST_ACTIVE;
  }
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
    const int64_t o = row * k + chunk * VEC;
    const Vec<T, VEC> rv = ldv_rw<T, VEC>(r + o);
    Vec<T, VEC> pv = ldv_rw<T, VEC>(p + o);
    const T d = dinv ? dinv[row] : T(1);
#pragma unroll
    for (int e = 0; e < VEC; ++e) pv.v[e] = on[e] ? fma(be[e], pv.v[e], d * rv.v[e]) : pv.v[e];
    stv<T, VEC>(p + o, pv);
  }
}

// --------------------------------------------- two-kernel iteration of the inner FP32 solve
//
// The inner solve folds the p update into the x, r update by forming beta before r is
// updated.  With z = D^-1 r and p = z + beta_old p_old (p_old A-conjugate to p, so
// (A p, z) = p . q), the next preconditioned residual product is
//   r_new . z_new = (r - alpha q) . D^-1 (r - alpha q) = alpha^2 q . D^-1 q - r . z,
// so beta = r_new . z_new / r . z = (r . z)(q . D^-1 q) / (p . q)^2 - 1 follows from the two
// sums the q = A p kernel can form.  Per iteration:
//   q = A p                                 fused with  pq_j = p_j . q_j, qdq_j = q_j . D^-1 q_j
//   x += a p, r -= a q, p = D^-1 r + b p    fused with  rz_j = r_j . D^-1 r_j, rr_j = r_j . r_j
// alpha uses the exact r . z of the previous update; only beta uses the identity (the
// single-reduction recurrence of pipelined CG on GPUs, e.g. Rupp et al.'s fused CG).

// The q = A p kernels' common end: the block's sums of p . q and q . D^-1 q per column, then,
// in the last block, alpha and beta per column from the totals (see above)
template <typename T, int VEC, int LPR>
__device__ __forceinline__ void q2_tail(DotAccN<T, 2 * VEC>& dacc, bool lead, int kp, int k, const CgCtl& ctl,
                                        CgScal* __restrict__ sc, double* __restrict__ partials, RedSmem<2>& red) {
  T part[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    part[0][e] = lead ? dacc.get(e) : T(0);
    part[1][e] = lead ? dacc.get(VEC + e) : T(0);
  }
  const double v = block_reduce<2, VEC>(part, kp, LPR, k, red);
  if (!publish_partials<2>(v, 2 * k, partials, &sc->counter[6], red)) return;
  const double tot = final_sum<2>(partials, 2 * k, gridDim.x, red);
  __shared__ double totals[2 * K];
  if ((int)threadIdx.x < 2 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k) {
    const double pq = totals[j], qdq = totals[k + j];
    sc->pq[j] = pq;
    double al = 0.0, be = 0.0;
    if (sc->state[j] == ST_ACTIVE) {
      if (!(pq > 0.0) || !isfinite(pq) || !isfinite(qdq)) {
        sc->state[j] = ctl.inner ? ST_DONE : ST_BREAKDOWN;
      } else {
        al = sc->rz[j] / pq;
        const double b = sc->rz[j] * qdq / (pq * pq) - 1.0;
        be = (b > 0.0 && isfinite(b)) ? b : 0.0;
      }
    }
    sc->alpha[j] = al;
    sc->beta[j] = be;
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, k);
}

template <typename T, int VEC, int LPR>
__global__ void __launch_bounds__(kThreads) k_cg_q2(CsrArgs<T> a, CgCtl ctl, const T* __restrict__ dinv,
                                                     CgScal* __restrict__ sc, double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<2> red;
  const int R = kThreads / (a.kp * LPR);
  const int t = threadIdx.x;
  const int sub = t % LPR, rc = t / LPR, chunk = rc % a.kp, rloc = rc / a.kp;
  DotAccN<T, 2 * VEC> dacc;  // [0, VEC): p . q, [VEC, 2 VEC): q . D^-1 q
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < a.k;
    T acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = T(0);
    row_accumulate_direct<T, VEC, LPR, false, true>(a, row, chunk, sub, active, acc);
    if (active && sub == 0) {
      const Vec<T, VEC> p = ldv<T, VEC>(a.X + row * a.ldx + chunk * VEC);
      const T d = dinv ? dinv[row] : T(1);
      Vec<T, VEC> q;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        q.v[e] = acc[e];
        dacc.add(e, p.v[e], acc[e]);
        dacc.add(VEC + e, acc[e], d * acc[e]);
      }
      stv<T, VEC>(a.Y + row * a.ldy + chunk * VEC, q);
    }
  }
  q2_tail<T, VEC, LPR>(dacc, sub == 0, a.kp, a.k, ctl, sc, partials, red);
}

// The same on runs of RUN consecutive cells along x (n_x a multiple of RUN; stencil7_apply_run):
// the y and z factors once per run, the centre values of p reused for p . q.  CONTIG: p and q
// rows hold exactly VEC columns (k = VEC), moved as 16-byte vectors.
template <typename T, int VEC, int RUN, bool CONTIG>
__global__ void __launch_bounds__(kThreads) k_cg_q2_run(Stencil7<T> st, FastDiv drun, FastDiv drow, int64_t n_runs,
                                                         CgCtl ctl, const T* __restrict__ p, T* __restrict__ q,
                                                         const T* __restrict__ dinv, CgScal* __restrict__ sc,
                                                         double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  DotAccN<T, 2 * VEC> dacc;  // [0, VEC): p . q, [VEC, 2 VEC): q . D^-1 q
  if (chunk * VEC < k) {
    for (int64_t u = (int64_t)blockIdx.x * R + threadIdx.x / kp; u < n_runs; u += (int64_t)gridDim.x * R) {
      Vec<T, VEC> pv[RUN], qv[RUN];
      const int64_t row0 = stencil7_apply_run<T, VEC, RUN, CONTIG>(st, drun, drow, u, p + chunk * VEC, k, pv, qv);
#pragma unroll
      for (int c = 0; c < RUN; ++c) {
        const T d = dinv ? dinv[row0 + c] : T(1);
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          dacc.add(e, pv[c].v[e], qv[c].v[e]);
          dacc.add(VEC + e, qv[c].v[e], d * qv[c].v[e]);
        }
      }
      store_run<T, VEC, RUN, CONTIG>(q + row0 * k + chunk * VEC, k, qv);
    }
  }
  q2_tail<T, VEC, 1>(dacc, true, kp, k, ctl, sc, partials, red);
}

// q = A p with the matrix-free FP32 Laplacian (stencil7.cuh: no index or value streams) and
// the same sums as k_cg_q2; p and q have leading dimension k
template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_cg_q2_st(Stencil7<T> st, CgCtl ctl, const T* __restrict__ p,
                                                        T* __restrict__ q, const T* __restrict__ dinv,
                                                        CgScal* __restrict__ sc, double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp, rloc = threadIdx.x / kp;
  DotAccN<T, 2 * VEC> dacc;  // [0, VEC): p . q, [VEC, 2 VEC): q . D^-1 q
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < ctl.n; base += stride) {
    const int64_t row = base + rloc;
    if (row < ctl.n && chunk * VEC < k) {
      T acc[VEC], unused;
      stencil7_apply<T, VEC>(st, p, k, row, chunk * VEC, acc, unused);
      const Vec<T, VEC> pv = ldv<T, VEC>(p + row * k + chunk * VEC);
      const T d = dinv ? dinv[row] : T(1);
      Vec<T, VEC> qv;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        qv.v[e] = acc[e];
        dacc.add(e, pv.v[e], acc[e]);
        dacc.add(VEC + e, acc[e], d * acc[e]);
      }
      stv<T, VEC>(q + row * k + chunk * VEC, qv);
    }
  }
  q2_tail<T, VEC, 1>(dacc, true, kp, k, ctl, sc, partials, red);
}

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_cg_xrp(CgCtl ctl, T* __restrict__ x, int64_t ldx, T* __restrict__ r,
                                                      T* __restrict__ p, const T* __restrict__ q,
                                                      const T* __restrict__ dinv, CgScal* __restrict__ sc,
                                                      double* __restrict__ partials) {
  if (sc->n_active == 0) return;
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const bool col_ok = chunk * VEC < k;
  T al[VEC], be[VEC];
  bool on[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int j = chunk * VEC + e;
    on[e] = col_ok && sc->state[j] == ST_ACTIVE;
    al[e] = on[e] ? (T)sc->alpha[j] : T(0);
    be[e] = on[e] ? (T)sc->beta[j] : T(0);
  }
  DotAccN<T, 2 * VEC> dots;  // [0, VEC): r . D^-1 r, [VEC, 2 VEC): r . r
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
      const int64_t o = row * k + chunk * VEC;
      Vec<T, VEC> pv = ldv_rw<T, VEC>(p + o);
      const Vec<T, VEC> qv = ldv_rw<T, VEC>(q + o);
      Vec<T, VEC> rv = ldv_rw<T, VEC>(r + o);
      Vec<T, VEC> xv = ldv_rw<T, VEC>(x + row * ldx + chunk * VEC);
      const T d = dinv ? dinv[row] : T(1);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        xv.v[e] = fma(al[e], pv.v[e], xv.v[e]);
        rv.v[e] = fma(-al[e], qv.v[e], rv.v[e]);
        const T z = d * rv.v[e];
        pv.v[e] = on[e] ? fma(be[e], pv.v[e], z) : pv.v[e];
        dots.add(e, rv.v[e], z);
        dots.add(VEC + e, rv.v[e], rv.v[e]);
      }
      stv<T, VEC>(x + row * ldx + chunk * VEC, xv);
      stv<T, VEC>(r + o, rv);
      stv<T, VEC>(p + o, pv);
    }
  }
  T part[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = dots.get(e), part[1][e] = dots.get(VEC + e);
  const double v = block_reduce<2, VEC>(part, kp, 1, k, red);
  if (!publish_partials<2>(v, 2 * k, partials, &sc->counter[7], red)) return;
  const double tot = final_sum<2>(partials, 2 * k, gridDim.x, red);
  __shared__ double totals[2 * K];
  if ((int)threadIdx.x < 2 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k && sc->state[j] == ST_ACTIVE) {
    const double rz_new = totals[j], rr_new = totals[k + j];
    sc->iters[j] += 1;
    sc->rr[j] = rr_new;
    sc->rz[j] = rz_new;
    if (!isfinite(rr_new) || !isfinite(rz_new)) sc->state[j] = ctl.inner ? ST_DONE : ST_BREAKDOWN;
    else if (rr_new <= sc->tol2[j]) {
      if (ctl.inner) sc->met[j] = 1;
      else sc->state[j] = ST_CHECK;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // inner solve: a column that has met its target keeps iterating (its share of the SpMM
    // is paid anyway) until every active column has; then the sweep ends for all of them
    if (ctl.inner) {
      bool all = true;
      for (int c = 0; c < k; ++c) all &= sc->state[c] != ST_ACTIVE || sc->met[c] != 0;
      if (all)
        for (int c = 0; c < k; ++c)
          if (sc->state[c] == ST_ACTIVE) sc->state[c] = ST_DONE;
    }
    recount(sc, k);
  }
}

// ------------------------------------------------ true residual r = b - A x (FP64 operator)

template <int VEC, int LPR>
__global__ void __launch_bounds__(kThreads) k_cg_resid(CsrArgs<double> a, CgCtl ctl, int mode,
                                                        const double* __restrict__ B, int64_t ldb,
                                                        double* __restrict__ rout, CgScal* __restrict__ sc,
                                                        double* __restrict__ partials) {
  if (mode == RM_OUTER && sc->n_orun == 0) return;  // every column of this system has finished
  __shared__ RedSmem<3> red;
  __shared__ bool wmask[K];
  const int k = a.k;
  const int R = kThreads / (a.kp * LPR);
  if ((int)threadIdx.x < k) {
    const int st = sc->state[threadIdx.x];
    bool w = false;
    if (mode == RM_INIT) w = true;
    else if (mode == RM_CHECK) w = (st == ST_CHECK);
    else if (mode == RM_OUTER) w = (sc->ostate[threadIdx.x] == ST_ACTIVE || sc->ostate[threadIdx.x] == ST_RESTART);
    wmask[threadIdx.x] = w;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int sub = t % LPR, rc = t / LPR, chunk = rc % a.kp, rloc = rc / a.kp;
  double acc_rr[VEC], acc_s[VEC], acc_bb[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc_rr[e] = acc_s[e] = acc_bb[e] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * R;
  for (int64_t base = (int64_t)blockIdx.x * R; base < a.n_rows; base += stride) {
    const int64_t row = base + rloc;
    const bool active = row < a.n_rows && chunk * VEC < k;
    double acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.0;
    row_accumulate_direct<double, VEC, LPR>(a, row, chunk, sub, active, acc);
    if (active && sub == 0) {
      const Vec<double, VEC> b = ldv<double, VEC>(B + row * ldb + chunk * VEC);
      Vec<double, VEC> rt;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        rt.v[e] = b.v[e] - acc[e];
        acc_rr[e] = fma(rt.v[e], rt.v[e], acc_rr[e]);
        acc_s[e] += rt.v[e];
        acc_bb[e] = fma(b.v[e], b.v[e], acc_bb[e]);
      }
      if (mode != RM_REPORT) {
        double* dst = rout + row * k + chunk * VEC;
        bool all = true;
#pragma unroll
        for (int e = 0; e < VEC; ++e) all &= wmask[chunk * VEC + e];
        if (all) {
          stv<double, VEC>(dst, rt);
        } else {
#pragma unroll
          for (int e = 0; e < VEC; ++e)
            if (wmask[chunk * VEC + e]) dst[e] = rt.v[e];
        }
      }
    }
  }
  double part[3][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    part[0][e] = sub == 0 ? acc_rr[e] : 0.0;
    part[1][e] = sub == 0 ? acc_s[e] : 0.0;
    part[2][e] = sub == 0 ? acc_bb[e] : 0.0;
  }
  const double v = block_reduce<3, VEC>(part, a.kp, LPR, k, red);
  if (!publish_partials<3>(v, 3 * k, partials, &sc->counter[2], red)) return;
  const double tot = final_sum<3>(partials, 3 * k, gridDim.x, red);
  __shared__ double totals[3 * K];
  if ((int)threadIdx.x < 3 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k) {
    const double rr = totals[j], s = totals[k + j], bb = totals[2 * k + j];
    const double nrow = (double)ctl.n;
    const double mean = ctl.project ? s / nrow : 0.0;
    const double rrp = ctl.project ? fmax(rr - nrow * mean * mean, 0.0) : rr;
    if (mode == RM_INIT) {
      sc->bb[j] = bb;
      sc->tol2[j] = ctl.rtol2 * bb;
      sc->mean[j] = mean;
      sc->iters[j] = 0;
      sc->state[j] = (bb == 0.0) ? ST_DONE : ST_RESTART;
    } else if (mode == RM_CHECK) {
      if (sc->state[j] == ST_CHECK) {
        sc->mean[j] = mean;
        sc->state[j] = (rrp <= sc->tol2[j]) ? ST_DONE : ST_RESTART;
      }
    } else if (mode == RM_REPORT) {
      sc->rr_true[j] = rrp;
    } else {  // RM_OUTER: one refinement sweep's residual
      if (sc->ostate[j] == ST_RESTART) {  // first sweep: record ||b||
        sc->bb[j] = bb;
        sc->otol2[j] = ctl.rtol2 * bb;
        sc->ostate[j] = ST_ACTIVE;
        sc->iters[j] = 0;
      }
      if (sc->ostate[j] == ST_ACTIVE) {
        sc->omean[j] = mean;
        if (sc->bb[j] == 0.0 || rrp <= sc->otol2[j]) {
          sc->ostate[j] = ST_DONE;
        } else if (!isfinite(rrp)) {
          sc->ostate[j] = ST_BREAKDOWN;
        } else {
          sc->oprev[j] = sc->oscale[j];
          sc->oscale[j] = sqrt(rrp);
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, k);
}

// ------------------------------------- restart: r -= mean, p = D^-1 r, rz, rr (RESTART columns)

template <typename T, int VEC>
__global__ void __launch_bounds__(kThreads) k_cg_restart(CgCtl ctl, T* __restrict__ r, T* __restrict__ p,
                                                          const T* __restrict__ dinv, CgScal* __restrict__ sc,
                                                          double* __restrict__ partials) {
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const bool col_ok = chunk * VEC < k;
  bool on[VEC];
  T mu[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    on[e] = col_ok && sc->state[chunk * VEC + e] == ST_RESTART;
    mu[e] = col_ok ? (T)sc->mean[chunk * VEC + e] : T(0);
  }
  DotAccN<T, 2 * VEC> dots;
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
      const int64_t o = row * k + chunk * VEC;
      Vec<T, VEC> rv = ldv_rw<T, VEC>(r + o);
      Vec<T, VEC> pv = ldv_rw<T, VEC>(p + o);
      const T d = dinv ? dinv[row] : T(1);
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        if (on[e]) {
          rv.v[e] = rv.v[e] - mu[e];
          pv.v[e] = d * rv.v[e];
          dots.add(e, rv.v[e], pv.v[e]);
          dots.add(VEC + e, rv.v[e], rv.v[e]);
        }
      }
      dots.step();
      stv<T, VEC>(r + o, rv);
      stv<T, VEC>(p + o, pv);
    }
  }
  T part[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = dots.get(e), part[1][e] = dots.get(VEC + e);
  const double v = block_reduce<2, VEC>(part, kp, 1, k, red);
  if (!publish_partials<2>(v, 2 * k, partials, &sc->counter[3], red)) return;
  const double tot = final_sum<2>(partials, 2 * k, gridDim.x, red);
  __shared__ double totals[2 * K];
  if ((int)threadIdx.x < 2 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k && sc->state[j] == ST_RESTART) {
    sc->rz[j] = totals[j];
    sc->rr[j] = totals[k + j];
    sc->state[j] = (totals[k + j] <= sc->tol2[j]) ? ST_DONE : ST_ACTIVE;
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, k);
}

// ---------------------------------- refinement: inner right-hand side and solution update

// r32 = (r64 - mean) / scale and d32 = 0 on outer-active columns (zero elsewhere).  A column
// that starts its recurrence here gets p32 = D^-1 r32.  With reliable updates a column that
// already has a direction continues it: the previous sweep's last update left
// p_old = D^-1 r_old + beta p_prev (old normalisation), and the continued direction is
// p = D^-1 r32 + ratio (p_old - D^-1 r_old) with ratio = s_prev / s, i.e. the recurrence
// residual's share replaced by the new true residual (a reliable update) in the new scale.
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_ir_init(CgCtl ctl, const double* __restrict__ r64,
                                                       float* __restrict__ r32, float* __restrict__ p32,
                                                       float* __restrict__ d32, const float* __restrict__ dinv,
                                                       CgScal* __restrict__ sc, double* __restrict__ partials) {
  __shared__ RedSmem<2> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  const bool col_ok = chunk * VEC < k;
  bool on[VEC], fresh[VEC];
  bool any_kept = false;
  double mu[VEC], inv[VEC];
  float ratio[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int j = chunk * VEC + e;
    on[e] = col_ok && sc->ostate[j] == ST_ACTIVE;
    fresh[e] = !(ctl.reliable && on[e] && sc->oprev[j] > 0.0);
    any_kept |= !fresh[e];
    mu[e] = on[e] ? sc->omean[j] : 0.0;
    inv[e] = on[e] ? 1.0 / sc->oscale[j] : 0.0;
    ratio[e] = fresh[e] ? 0.0f : (float)(sc->oprev[j] / sc->oscale[j]);
  }
  DotAccN<float, 2 * VEC> dots;
  if (col_ok) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
      const int64_t o = row * k + chunk * VEC;
      const Vec<double, VEC> rv = ldv_rw<double, VEC>(r64 + o);
      const float d = dinv ? dinv[row] : 1.0f;
      Vec<float, VEC> r, p, z, rold;
      if (any_kept) {
        p = ldv_rw<float, VEC>(p32 + o);
        rold = ldv_rw<float, VEC>(r32 + o);
      }
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        r.v[e] = on[e] ? (float)((rv.v[e] - mu[e]) * inv[e]) : 0.0f;
        const float zz = d * r.v[e];
        p.v[e] = fresh[e] ? zz : fmaf(ratio[e], fmaf(-d, rold.v[e], p.v[e]), zz);
        z.v[e] = 0.0f;
        dots.add(e, r.v[e], zz);
        dots.add(VEC + e, r.v[e], r.v[e]);
      }
      stv<float, VEC>(r32 + o, r);
      stv<float, VEC>(p32 + o, p);
      stv<float, VEC>(d32 + o, z);
    }
  }
  float part[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = dots.get(e), part[1][e] = dots.get(VEC + e);
  const double v = block_reduce<2, VEC>(part, kp, 1, k, red);
  if (!publish_partials<2>(v, 2 * k, partials, &sc->counter[4], red)) return;
  const double tot = final_sum<2>(partials, 2 * k, gridDim.x, red);
  __shared__ double totals[2 * K];
  if ((int)threadIdx.x < 2 * k) totals[threadIdx.x] = tot;
  __syncthreads();
  const int j = threadIdx.x;
  if (j < k) {
    sc->met[j] = 0;
    if (sc->ostate[j] == ST_ACTIVE && totals[k + j] > 0.0) {
      sc->rz[j] = totals[j];
      sc->rr[j] = totals[k + j];
      // inner target: inner_rtol of the sweep's residual, but never past what the outer
      // tolerance still needs (half of it, in the inner scale r / s), so that the last sweep
      // does not overshoot
      const double s2 = sc->oscale[j] * sc->oscale[j];
      sc->tol2[j] = fmax(ctl.inner_rtol2 * totals[k + j], 0.25 * sc->otol2[j] / s2);
      sc->state[j] = ST_ACTIVE;
    } else {
      sc->state[j] = ST_IDLE;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) recount(sc, k);
}

// x64 += scale * d32 on outer-active columns
template <int VEC>
__global__ void __launch_bounds__(kThreads) k_ir_update(CgCtl ctl, double* __restrict__ x, int64_t ldx,
                                                         const float* __restrict__ d32,
                                                         const CgScal* __restrict__ sc) {
  if (sc->n_oactive == 0) return;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  double s[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int j = chunk * VEC + e;
    s[e] = (sc->ostate[j] == ST_ACTIVE) ? sc->oscale[j] : 0.0;
  }
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
    const Vec<float, VEC> d = ldv_rw<float, VEC>(d32 + row * k + chunk * VEC);
    Vec<double, VEC> xv = ldv_rw<double, VEC>(x + row * ldx + chunk * VEC);
#pragma unroll
    for (int e = 0; e < VEC; ++e) xv.v[e] = fma(s[e], (double)d.v[e], xv.v[e]);
    stv<double, VEC>(x + row * ldx + chunk * VEC, xv);
  }
}

// ------------------------------------------------------- final projection x -= mean(x)

template <int VEC>
__global__ void __launch_bounds__(kThreads) k_colsum(CgCtl ctl, const double* __restrict__ x, int64_t ldx,
                                                      CgScal* __restrict__ sc, double* __restrict__ partials) {
  __shared__ RedSmem<1> red;
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  double part[1][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) part[0][e] = 0.0;
  if (chunk * VEC < k) {
    for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
      const Vec<double, VEC> xv = ldv_rw<double, VEC>(x + row * ldx + chunk * VEC);
#pragma unroll
      for (int e = 0; e < VEC; ++e) part[0][e] += xv.v[e];
    }
  }
  const double v = block_reduce<1, VEC>(part, kp, 1, k, red);
  if (!publish_partials<1>(v, k, partials, &sc->counter[5], red)) return;
  const double tot = final_sum<1>(partials, k, gridDim.x, red);
  if ((int)threadIdx.x < k) sc->mean[threadIdx.x] = tot / (double)ctl.n;
}

template <int VEC>
__global__ void __launch_bounds__(kThreads) k_submean(CgCtl ctl, double* __restrict__ x, int64_t ldx,
                                                       const CgScal* __restrict__ sc) {
  const int k = ctl.k, kp = ctl.kp;
  const int R = kThreads / kp;
  const int chunk = threadIdx.x % kp;
  if (chunk * VEC >= k) return;
  double mu[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) mu[e] = sc->mean[chunk * VEC + e];
  for (int64_t row = (int64_t)blockIdx.x * R + threadIdx.x / kp; row < ctl.n; row += (int64_t)gridDim.x * R) {
    Vec<double, VEC> xv = ldv_rw<double, VEC>(x + row * ldx + chunk * VEC);
#pragma unroll
    for (int e = 0; e < VEC; ++e) xv.v[e] -= mu[e];
    stv<double, VEC>(x + row * ldx + chunk * VEC, xv);
  }
}

__global__ void k_init_outer(CgScal* sc, int k) {
  const int j = threadIdx.x;
  if (j < k) {
    sc->ostate[j] = ST_RESTART;
    sc->state[j] = ST_IDLE;
    sc->iters[j] = 0;
  }
  if (j == 0) recount(sc, k);
}

__global__ void k_mark_noconv(CgScal* sc, int k, int outer) {
  const int j = threadIdx.x;
  if (j < k) {
    if (outer) {
      if (sc->ostate[j] == ST_ACTIVE) sc->ostate[j] = ST_NOCONV;
    } else if (sc->state[j] == ST_ACTIVE || sc->state[j] == ST_CHECK || sc->state[j] == ST_RESTART) {
      sc->state[j] = ST_NOCONV;
    }
  }
  if (j == 0) recount(sc, k);
}

// ------------------------------------------------------------------------------- host side

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
  size_t scal = 0, partials = 0, r = 0, p = 0, q = 0, r64 = 0, r32 = 0, p32 = 0, q32 = 0, d32 = 0, total = 0;
};

Layout layout(int64_t n, int k, bool mixed) {
  Layout L;
  size_t off = 0;
  L.scal = off;
  off += align256(sizeof(CgScal));
  L.partials = off;
  off += align256((size_t)kGridMax * 3 * K * sizeof(double));
  const size_t v64 = align256((size_t)n * k * sizeof(double));
  const size_t v32 = align256((size_t)n * k * sizeof(float));
  if (!mixed) {
    L.r = off, off += v64;
    L.p = off, off += v64;
    L.q = off, off += v64;
  } else {
    L.r64 = off, off += v64;
    L.r32 = off, off += v32;
    L.p32 = off, off += v32;
    L.q32 = off, off += v32;
    L.d32 = off, off += v32;
  }
  L.total = off;
  return L;
}

// Shared launch plumbing for one solve.
struct Solver {
  const rb_op* A;
  const rb_op* A32;
  int k, vec, kp;
  int64_t n;
  CgCtl ctl;
  CgScal* sc;
  double* partials;
  cudaStream_t s;
  SpmmSched sched64, sched32;
  // One resident wave of `kern`, never more blocks than there are row blocks.  Also when the
  // plain SpMM's tuned schedule launches one block per row block: for these reducing kernels
  // the last block's sum over ~9000 block partials costs more than the wave's grid stride
  // (channel Poisson solve, k = 3: FP64 CG 253 -> 341 ms, refinement 129 -> 218 ms).
  template <typename K_>
  int spmm_grid(K_* kern, const SpmmSched& sc) const {
    const int R = sc.rows_per_block();
    return wave_grid(kern, (n + R - 1) / R);
  }
  template <typename K_>
  int vg(K_* kern) const {
    const int R = kThreads / kp;
    return wave_grid(kern, (n + R - 1) / R);
  }

  template <typename T>
  CsrArgs<T> args(const rb_op* op, const SpmmSched& ss, const T* X, int64_t ldx, T* Y, int64_t ldy) const {
    CsrArgs<T> a;
    fill_csr_args(op, ss, a, 0);
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    a.k = k;
    a.cs = nullptr;
    return a;
  }

  template <typename T, int VEC, int LPR>
  void launch_q(const rb_op* op, const SpmmSched& ss, const T* p, T* q, CgCtl c) const {
    CsrArgs<T> a = args<T>(op, ss, p, k, q, k);
    k_cg_q<T, VEC, LPR><<<spmm_grid(&k_cg_q<T, VEC, LPR>, ss), kThreads, 0, s>>>(a, c, sc, partials);
  }

  template <typename T, int VEC>
  void launch_q_lpr(const rb_op* op, const SpmmSched& ss, const T* p, T* q, CgCtl c) const {
    switch (ss.lpr) {
      case 2: launch_q<T, VEC, 2>(op, ss, p, q, c); break;
      case 4: launch_q<T, VEC, 4>(op, ss, p, q, c); break;
      case 8: launch_q<T, VEC, 8>(op, ss, p, q, c); break;
      default: launch_q<T, VEC, 1>(op, ss, p, q, c); break;
    }
  }

  template <typename T, int VEC, int LPR>
  void launch_q2(const rb_op* op, const SpmmSched& ss, const T* p, T* q, const T* dinv, CgCtl c) const {
    CsrArgs<T> a = args<T>(op, ss, p, k, q, k);
    k_cg_q2<T, VEC, LPR><<<spmm_grid(&k_cg_q2<T, VEC, LPR>, ss), kThreads, 0, s>>>(a, c, dinv, sc,
                                                                                          partials);
  }

  template <typename T, int VEC>
  void launch_q2_lpr(const rb_op* op, const SpmmSched& ss, const T* p, T* q, const T* dinv, CgCtl c) const {
    if constexpr (sizeof(T) == 4) {
      if (op->format == RB_STENCIL) {  // the matrix-free inner operator
        Stencil7<float> st{};
        for (int d = 0; d < 3; ++d) {
          st.n[d] = op->st_n[d];
          st.per[d] = op->st_per[d];
          st.w[d] = static_cast<const float*>(op->st_w[d]);
          st.ic[d] = static_cast<const float*>(op->st_ic[d]);
        }
        st.scale = (float)op->st_scale;
        st.init_div();
        constexpr int RUN = 4;
        if (op->st_n[0] % RUN == 0) {  // runs of four cells along x
          const int64_t n_runs = n / RUN;
          FastDiv drun, drow;
          drun.init((uint32_t)(op->st_n[0] / RUN));
          drow.init((uint32_t)op->st_n[1]);
          const bool contig = kp == 1 && k == VEC && ((uintptr_t)p % 16) == 0 && ((uintptr_t)q % 16) == 0;
          auto go = [&](auto kern) {
            kern<<<wave_grid(kern, (n_runs + kThreads / kp - 1) / (kThreads / kp)), kThreads, 0, s>>>(
                st, drun, drow, n_runs, c, p, q, dinv, sc, partials);
          };
          if (contig) go(&k_cg_q2_run<T, VEC, RUN, true>);
          else go(&k_cg_q2_run<T, VEC, RUN, false>);
          return;
        }
        k_cg_q2_st<T, VEC><<<vg(&k_cg_q2_st<T, VEC>), kThreads, 0, s>>>(st, c, p, q, dinv, sc, partials);
        return;
      }
    }
    switch (ss.lpr) {
      case 2: launch_q2<T, VEC, 2>(op, ss, p, q, dinv, c); break;
      case 4: launch_q2<T, VEC, 4>(op, ss, p, q, dinv, c); break;
      case 8: launch_q2<T, VEC, 8>(op, ss, p, q, dinv, c); break;
      default: launch_q2<T, VEC, 1>(op, ss, p, q, dinv, c); break;
    }
  }

  template <int VEC, int LPR>
  void launch_resid_t(int mode, const double* B, int64_t ldb, const double* X, int64_t ldx, double* r) const {
    CsrArgs<double> a = args<double>(A, sched64, X, ldx, nullptr, 0);
    k_cg_resid<VEC, LPR><<<spmm_grid(&k_cg_resid<VEC, LPR>, sched64), kThreads, 0, s>>>(a, ctl, mode, B, ldb,
                                                                                              r, sc, partials);
  }

  template <int VEC>
  void launch_resid_v(int mode, const double* B, int64_t ldb, const double* X, int64_t ldx, double* r) const {
    switch (sched64.lpr) {
      case 2: launch_resid_t<VEC, 2>(mode, B, ldb, X, ldx, r); break;
      case 4: launch_resid_t<VEC, 4>(mode, B, ldb, X, ldx, r); break;
      case 8: launch_resid_t<VEC, 8>(mode, B, ldb, X, ldx, r); break;
      default: launch_resid_t<VEC, 1>(mode, B, ldb, X, ldx, r); break;
    }
  }
};

template <int VEC>
struct Iter {
  // one CG iteration in precision T on operator op
  template <typename T>
  static void step(const Solver& S_, const rb_op* op, const SpmmSched& ss, CgCtl c, T* x, int64_t ldx, T* r, T* p,
                   T* q, const T* dinv) {
    S_.launch_q_lpr<T, VEC>(op, ss, p, q, c);
    k_cg_update<T, VEC><<<S_.vg(&k_cg_update<T, VEC>), kThreads, 0, S_.s>>>(c, x, ldx, r, p, q, dinv, S_.sc,
                                                                            S_.partials);
    k_cg_p<T, VEC><<<S_.vg(&k_cg_p<T, VEC>), kThreads, 0, S_.s>>>(c, r, p, dinv, S_.sc);
  }
  // one iteration of the two-kernel recurrence (beta from the q = A p kernel's sums)
  template <typename T>
  static void step2(const Solver& S_, const rb_op* op, const SpmmSched& ss, CgCtl c, T* x, int64_t ldx, T* r, T* p,
                    T* q, const T* dinv) {
    S_.launch_q2_lpr<T, VEC>(op, ss, p, q, dinv, c);
    k_cg_xrp<T, VEC><<<S_.vg(&k_cg_xrp<T, VEC>), kThreads, 0, S_.s>>>(c, x, ldx, r, p, q, dinv, S_.sc, S_.partials);
  }
};

struct HostState {
  int state[K], ostate[K];
  int n_active, n_check, n_oactive;
};

// A run of check_every CG iterations recorded once as a CUDA graph and replayed, which
// removes the per-kernel launch cost from the host side of the loop.  Recording happens on
// a private stream of this thread (the legacy default stream cannot be captured); the
// replay goes to the caller's stream.  Kernels whose columns have all finished return at
// once, so a replay past convergence costs only the empty launches.
struct ChunkGraph {
  cudaGraphExec_t exec = nullptr;
  int len = 0;
  ChunkGraph() = default;
  ChunkGraph(const ChunkGraph&) = delete;
  ChunkGraph& operator=(const ChunkGraph&) = delete;
  ~ChunkGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

cudaStream_t capture_stream() {
  static thread_local cudaStream_t cs = nullptr;
  if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cs = nullptr;
  }
  return cs;
}

template <class F>
rb_status run_chunk(Solver& S_, ChunkGraph& g, int chunk, int full, int& uses, F&& one_iteration) {
  // the first full chunk runs eagerly (it also fills the launch-shape caches); later full
  // chunks replay the recorded graph
  cudaStream_t cs = capture_stream();
  if (chunk == full && uses > 0 && cs) {
    if (!g.exec) {
      cudaStream_t user = S_.s;
      S_.s = cs;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int i = 0; i < chunk; ++i) one_iteration();
        e = cudaStreamEndCapture(cs, &graph);
      }
      S_.s = user;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(e, "CUDA graph capture of the CG iterations", __FILE__, __LINE__);
      g.len = chunk;
    }
    RB_CUDA(cudaGraphLaunch(g.exec, S_.s));
  } else {
    for (int i = 0; i < chunk; ++i) one_iteration();
  }
  ++uses;
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

rb_status read_state(const Solver& S_, HostState& h) {
  RB_CUDA(cudaMemcpyAsync(h.state, S_.sc->state, sizeof(int) * K, cudaMemcpyDeviceToHost, S_.s));
  RB_CUDA(cudaMemcpyAsync(h.ostate, S_.sc->ostate, sizeof(int) * K, cudaMemcpyDeviceToHost, S_.s));
  RB_CUDA(cudaMemcpyAsync(&h.n_active, &S_.sc->n_active, sizeof(int) * 3, cudaMemcpyDeviceToHost, S_.s));
  RB_CUDA(cudaStreamSynchronize(S_.s));
  return RB_OK;
}

// one sweep's inner iterations of a single system in one cooperative launch (defined below)
rb_status persistent_inner(Solver& S_, const rb_cg_params& prm, const Layout& L, char* base);

template <int VEC>
rb_status solve_vec(Solver& S_, const rb_cg_params& prm, const double* B, int64_t ldb, double* X, int64_t ldx,
                    const Layout& L, char* base, rb_cg_report& rep) {
  const int k = S_.k;
  HostState h;
  int syncs = 0, spmms = 0;
  if (!prm.mixed) {
    double* r = reinterpret_cast<double*>(base + L.r);
    double* p = reinterpret_cast<double*>(base + L.p);
    double* q = reinterpret_cast<double*>(base + L.q);
    const double* dinv = prm.precond ? S_.A->dinv64 : nullptr;
    CgCtl c = S_.ctl;
    c.inner = 0;
    S_.launch_resid_v<VEC>(RM_INIT, B, ldb, X, ldx, r);
    ++spmms;
    k_cg_restart<double, VEC><<<S_.vg(&k_cg_restart<double, VEC>), kThreads, 0, S_.s>>>(c, r, p, dinv, S_.sc, S_.partials);
    RB_CUDA(cudaGetLastError());
    int it = 0;
    ChunkGraph graph;
    int uses = 0;
    while (true) {
      RB_TRY(read_state(S_, h));
      ++syncs;
      if (h.n_check > 0) {
        S_.launch_resid_v<VEC>(RM_CHECK, B, ldb, X, ldx, r);
        ++spmms;
        k_cg_restart<double, VEC><<<S_.vg(&k_cg_restart<double, VEC>), kThreads, 0, S_.s>>>(c, r, p, dinv, S_.sc, S_.partials);
        RB_CUDA(cudaGetLastError());
        continue;
      }
      if (h.n_active == 0) break;
      if (it >= prm.max_iter) {
        k_mark_noconv<<<1, K, 0, S_.s>>>(S_.sc, k, 0);
        break;
      }
      const int chunk = std::min(prm.check_every, prm.max_iter - it);
      RB_TRY(run_chunk(S_, graph, chunk, prm.check_every, uses, [&] {
        Iter<VEC>::template step<double>(S_, S_.A, S_.sched64, c, X, ldx, r, p, q, dinv);
      }));
      it += chunk;
      spmms += chunk;
    }
  } else {
    double* r64 = reinterpret_cast<double*>(base + L.r64);
    float* r32 = reinterpret_cast<float*>(base + L.r32);
    float* p32 = reinterpret_cast<float*>(base + L.p32);
    float* q32 = reinterpret_cast<float*>(base + L.q32);
    float* d32 = reinterpret_cast<float*>(base + L.d32);
    const float* dinv32 = prm.precond ? S_.A32->dinv32 : nullptr;
    CgCtl c = S_.ctl;
    c.inner = 1;
    k_init_outer<<<1, K, 0, S_.s>>>(S_.sc, k);
    int total_inner = 0;
    int sweep = 0;
    ChunkGraph graph;
    int uses = 0;
    for (;; ++sweep) {
      S_.launch_resid_v<VEC>(RM_OUTER, B, ldb, X, ldx, r64);
      ++spmms;
      RB_CUDA(cudaGetLastError());
      RB_TRY(read_state(S_, h));
      ++syncs;
      if (h.n_oactive == 0) break;
      if (sweep >= prm.max_sweeps || total_inner >= prm.max_iter) {
        k_mark_noconv<<<1, K, 0, S_.s>>>(S_.sc, k, 1);
        break;
      }
      k_ir_init<VEC><<<S_.vg(&k_ir_init<VEC>), kThreads, 0, S_.s>>>(c, r64, r32, p32, d32, dinv32, S_.sc, S_.partials);
      RB_CUDA(cudaGetLastError());
      int it = 0;
      if (prm.persistent) {
        // all of this sweep's inner iterations in one cooperative launch
        rb_cg_params p2 = prm;
        p2.max_iter = prm.max_iter - total_inner;
        RB_TRY(persistent_inner(S_, p2, L, base));
        unsigned pb[2] = {0, 0};  // pbar[2]: barrier error word, pbar[3]: iterations done
        RB_CUDA(cudaMemcpyAsync(pb, &S_.sc->pbar[2], 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, S_.s));
        RB_CUDA(cudaStreamSynchronize(S_.s));
        ++syncs;
        const unsigned err = pb[0], done = pb[1];
        if (err) {
          set_error("rb_cg_solve: a grid barrier wait of the persistent inner solve gave up");
          return RB_ETIMEOUT;
        }
        it = (int)done;
        spmms += it;
      }
      while (!prm.persistent) {
        RB_TRY(read_state(S_, h));
        ++syncs;
        if (h.n_active == 0 || total_inner + it >= prm.max_iter) break;
        const int chunk = std::min(prm.check_every, prm.max_iter - total_inner - it);
        RB_TRY(run_chunk(S_, graph, chunk, prm.check_every, uses, [&] {
          Iter<VEC>::template step2<float>(S_, S_.A32, S_.sched32, c, d32, k, r32, p32, q32, dinv32);
        }));
        it += chunk;
        spmms += chunk;
      }
      total_inner += it;
      k_ir_update<VEC><<<S_.vg(&k_ir_update<VEC>), kThreads, 0, S_.s>>>(c, X, ldx, d32, S_.sc);
      RB_CUDA(cudaGetLastError());
    }
    rep.sweeps = sweep;
  }
  // final projection and report
  if (prm.project_mean) {
    k_colsum<VEC><<<S_.vg(&k_colsum<VEC>), kThreads, 0, S_.s>>>(S_.ctl, X, ldx, S_.sc, S_.partials);
    k_submean<VEC><<<S_.vg(&k_submean<VEC>), kThreads, 0, S_.s>>>(S_.ctl, X, ldx, S_.sc);
  }
  S_.launch_resid_v<VEC>(RM_REPORT, B, ldb, X, ldx, nullptr);
  ++spmms;
  RB_CUDA(cudaGetLastError());
  CgScal hs;
  RB_CUDA(cudaMemcpyAsync(&hs, S_.sc, sizeof(CgScal), cudaMemcpyDeviceToHost, S_.s));
  RB_CUDA(cudaStreamSynchronize(S_.s));
  ++syncs;
  rb_status worst = RB_OK;
  for (int j = 0; j < k; ++j) {
    rep.iters[j] = hs.iters[j];
    rep.true_rel_res[j] = hs.bb[j] > 0 ? sqrt(hs.rr_true[j] / hs.bb[j]) : 0.0;
    const int st = prm.mixed ? hs.ostate[j] : hs.state[j];
    rb_status cs = RB_OK;
    if (st == ST_BREAKDOWN) cs = RB_EBREAKDOWN;
    else if (st == ST_NOCONV || st == ST_ACTIVE) cs = RB_ENOCONV;
    rep.status[j] = cs;
    if (cs == RB_EBREAKDOWN || (cs == RB_ENOCONV && worst == RB_OK)) worst = cs;
  }
  rep.spmm_calls = spmms;
  rep.host_syncs = syncs;
  return worst;
}

// ===================================================================================
// Persistent batched inner solve: every inner FP32 CG iteration of every system of a batch
// in ONE cooperative launch.  Blocks are partitioned among the systems in proportion to
// their work; each iteration runs the two phases of the two-kernel inner loop (q = A p with
// p.q and q.D^-1 q; x, r, p update with r.D^-1 r and r.r) separated by grid-wide barriers,
// and every block of a system reduces the system's per-column sums after each barrier.  The
// barrier waits are bounded (globaltimer): past the limit a block records an error and
// every block leaves.
// ===================================================================================

constexpr int kMaxSys = 8;
constexpr int kPThreads = 512;
constexpr int kPWarps = kPThreads / 32;

struct PSys {
  const int32_t* rp;  // CSR inner operator, or
  const int32_t* ci;
  const float* va;
  Stencil7<float> st;  // the matrix-free one (mf = 1)
  int mf;
  const float* dinv;
  float* r;
  float* p;
  float* q;
  float* d;
  CgScal* sc;
  int n, k, vec, kp;
  int blk0, nblk;  // blocks [blk0, blk0 + nblk) work on this system
  int col0;        // first column of this system in the batch numbering
};

struct PBatch {
  PSys sys[kMaxSys];
  int n_sys, total_cols;
  double* partials;  // [gridDim.x][4][K]: p.q, q.D^-1 q, r.D^-1 r, r.r per block and batch column
  unsigned* bar;     // [0] arrivals, [1] generation (zeroed before every launch)
  int* err;          // 0, or the code of the first wait that gave up
  int max_iter;      // iteration cap of this launch
  int extra_arrivals;  // failure-detection tests only: arrivals the barrier waits for beyond the grid
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch.  Returns false in every thread of the block when
// this block's wait ran past timeout_ns or another block has recorded an error.
__device__ bool grid_barrier(const PBatch& b) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned* gen = b.bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned expected = gridDim.x + (unsigned)b.extra_arrivals;
    if (atomicAdd(b.bar, 1u) == expected - 1u) {
      b.bar[0] = 0u;
      __threadfence();
      atomicAdd(b.bar + 1, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*gen == g) {
        if (*(volatile int*)b.err) {
          ok = 0;
          break;
        }
        if (globaltimer_ns() - t0 > b.timeout_ns) {
          atomicCAS(b.err, 0, 1);
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Sum over the block of acc[q][e] per column (threads laid out (row, chunk), KP chunks per
// row): warp fold in FP32, warps summed in FP64 in order; column totals land in out[q * k + j].
template <int NQ, int VEC>
__device__ __forceinline__ void pblock_reduce(float (&acc)[NQ][VEC], int kp, int k, double* red, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) warp_fold<float, VEC>(acc[q], kp);
  if (lane < kp) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int e = 0; e < VEC; ++e) red[(w * NQ + q) * 64 + lane * VEC + e] = (double)acc[q][e];
  }
  __syncthreads();
  if ((int)threadIdx.x < NQ * k) {
    const int q = threadIdx.x / k, j = threadIdx.x % k;
    double s = 0.0;
    for (int ww = 0; ww < kPWarps; ++ww) s += red[(ww * NQ + q) * 64 + j];
    out[q * k + j] = s;
  }
  __syncthreads();
}

// phase A: q = A p on the block's system; p . q and q . D^-1 q per column into partial slots
// 0 and 1
template <int VEC>
__device__ void pphase_q(const PBatch& b, const PSys& S, double* red, double* out) {
  const int R = kPThreads / S.kp;
  const int chunk = threadIdx.x % S.kp, rloc = threadIdx.x / S.kp;
  CsrArgs<float> a;
  a.n_rows = S.n;
  a.rp = S.rp;
  a.ci = S.ci;
  a.va = S.va;
  a.X = S.p;
  a.ldx = S.k;
  a.k = S.k;
  a.kp = S.kp;
  float acc2[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc2[0][e] = acc2[1][e] = 0.f;
  for (int64_t base = (int64_t)(blockIdx.x - S.blk0) * R; base < S.n; base += (int64_t)S.nblk * R) {
    const int64_t row = base + rloc;
    const bool active = row < S.n && chunk * VEC < S.k;
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = 0.f;
    if (S.mf) {  // p is written by other blocks of this launch: coherent loads
      float unused;
      if (active) stencil7_apply<float, VEC, true>(S.st, S.p, S.k, row, chunk * VEC, acc, unused);
    } else {
      row_accumulate_direct<float, VEC, 1, true>(a, row, chunk, 0, active, acc);
    }
    if (active) {
      const Vec<float, VEC> p = ldv_cg<float, VEC>(S.p + row * S.k + chunk * VEC);
      const float dg = S.dinv ? S.dinv[row] : 1.f;
      Vec<float, VEC> qv;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        qv.v[e] = acc[e];
        acc2[0][e] = fmaf(p.v[e], acc[e], acc2[0][e]);
        acc2[1][e] = fmaf(acc[e], dg * acc[e], acc2[1][e]);
      }
      stv<float, VEC>(S.q + row * S.k + chunk * VEC, qv);
    }
  }
  pblock_reduce<2, VEC>(acc2, S.kp, S.k, red, out);
  if ((int)threadIdx.x < 2 * S.k) {
    const int q = threadIdx.x / S.k, j = threadIdx.x % S.k;
    b.partials[((size_t)blockIdx.x * 4 + q) * K + S.col0 + j] = out[threadIdx.x];
  }
}

// phase B: d += alpha p, r -= alpha q, p = D^-1 r + beta p on active columns; r . D^-1 r and
// r . r per column into partial slots 2 and 3 (slots apart from phase A's, which slower blocks
// may still be reading)
template <int VEC>
__device__ void pphase_xrp(const PBatch& b, const PSys& S, const double* alpha, const double* beta,
                           const int* state, double* red, double* out) {
  const int R = kPThreads / S.kp;
  const int chunk = threadIdx.x % S.kp;
  const bool col_ok = chunk * VEC < S.k;
  float al[VEC], be[VEC];
  bool on[VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    on[e] = col_ok && state[chunk * VEC + e] == ST_ACTIVE;
    al[e] = on[e] ? (float)alpha[chunk * VEC + e] : 0.f;
    be[e] = on[e] ? (float)beta[chunk * VEC + e] : 0.f;
  }
  float acc[2][VEC];
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc[0][e] = acc[1][e] = 0.f;
  if (col_ok) {
    for (int64_t row = (int64_t)(blockIdx.x - S.blk0) * R + threadIdx.x / S.kp; row < S.n;
         row += (int64_t)S.nblk * R) {
      const int64_t o = row * S.k + chunk * VEC;
      Vec<float, VEC> pv = ldv_cg<float, VEC>(S.p + o);
      const Vec<float, VEC> qv = ldv_cg<float, VEC>(S.q + o);
      Vec<float, VEC> rv = ldv_cg<float, VEC>(S.r + o);
      Vec<float, VEC> xv = ldv_cg<float, VEC>(S.d + o);
      const float dg = S.dinv ? S.dinv[row] : 1.f;
#pragma unroll
      for (int e = 0; e < VEC; ++e) {
        xv.v[e] = fmaf(al[e], pv.v[e], xv.v[e]);
        rv.v[e] = fmaf(-al[e], qv.v[e], rv.v[e]);
        const float z = dg * rv.v[e];
        pv.v[e] = on[e] ? fmaf(be[e], pv.v[e], z) : pv.v[e];
        acc[0][e] = fmaf(rv.v[e], z, acc[0][e]);
        acc[1][e] = fmaf(rv.v[e], rv.v[e], acc[1][e]);
      }
      stv<float, VEC>(S.d + o, xv);
      stv<float, VEC>(S.r + o, rv);
      stv<float, VEC>(S.p + o, pv);
    }
  }
  pblock_reduce<2, VEC>(acc, S.kp, S.k, red, out);
  if ((int)threadIdx.x < 2 * S.k) {
    const int q = threadIdx.x / S.k, j = threadIdx.x % S.k;
    b.partials[((size_t)blockIdx.x * 4 + 2 + q) * K + S.col0 + j] = out[threadIdx.x];
  }
}

// Totals over the blocks of system S of nq partial quantities (slots q0 .. q0 + nq/k - 1 of its
// k columns): warp w sums quantities w, w + 16, ... over the system's blocks in a fixed order
// (lanes strided, then a shuffle tree); every block of S computes the same totals, so the
// per-column scalars need no broadcast.  Results land in out[i] for i < nq (nq <= 2 K);
// whole block calls.
__device__ void psys_totals(const PBatch& b, const PSys& S, int q0, int nq, double* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = w; i < nq; i += kPWarps) {
    const int q = q0 + i / S.k, c = S.col0 + i % S.k;
    double s = 0.0;
    for (int bb = lane; bb < S.nblk; bb += 32) s += __ldcg(&b.partials[((size_t)(S.blk0 + bb) * 4 + q) * K + c]);
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ bool pany_active(const PBatch& b) {
  for (int s = 0; s < b.n_sys; ++s)
    for (int j = 0; j < b.sys[s].k; ++j)
      if (__ldcg(&b.sys[s].sc->state[j]) == ST_ACTIVE) return true;
  return false;
}

// Two grid barriers per iteration (the two-kernel recurrence above): after q = A p every block
// reduces its own system's p.q and q.D^-1 q and forms alpha and beta; after the x, r, p update
// every block reduces r.D^-1 r and r.r and forms the convergence test.  Every block keeps its
// system's column scalars (state, r.D^-1 r, iterations) in shared memory, computed
// identically in all of the system's blocks; the system's first block writes them back for
// the host and the next kernel.
__global__ void __launch_bounds__(kPThreads) k_pcg_batch(PBatch b) {
  __shared__ double red[kPWarps * 2 * 64];
  __shared__ double out[2 * K];
  __shared__ double tot[2 * K];
  __shared__ double l_rz[K], l_alpha[K], l_beta[K];
  __shared__ int l_state[K], l_iters[K], l_met[K];
  __shared__ int go, mine;
  int my = -1;
  for (int s = 0; s < b.n_sys; ++s)
    if ((int)blockIdx.x >= b.sys[s].blk0 && (int)blockIdx.x < b.sys[s].blk0 + b.sys[s].nblk) my = s;
  const bool lead = my >= 0 && (int)blockIdx.x == b.sys[my].blk0;
  if (my >= 0 && (int)threadIdx.x < b.sys[my].k) {
    const CgScal* sc = b.sys[my].sc;
    l_state[threadIdx.x] = __ldcg(&sc->state[threadIdx.x]);
    l_rz[threadIdx.x] = __ldcg(&sc->rz[threadIdx.x]);
    l_iters[threadIdx.x] = __ldcg(&sc->iters[threadIdx.x]);
    l_met[threadIdx.x] = 0;
  }
  // Every block must leave the loop in the same iteration.  The states at entry are the same
  // for all blocks; later, the leads publish after each iteration whether their system is
  // still active (pact[it & 1]), and the decision at the top of iteration it reads what was
  // published after iteration it - 2, which the barriers of iteration it - 1 made visible to
  // every block (iteration it - 1's flags may still be in flight).  So the loop runs up to two
  // iterations of bare barriers past the last active column.
  const int entry_go = pany_active(b) ? 1 : 0;
  for (int it = 0; it < b.max_iter; ++it) {
    if (threadIdx.x == 0) {
      int g = entry_go;
      if (it >= 2) {
        g = 0;
        for (int s = 0; s < b.n_sys; ++s) g |= __ldcg(&b.sys[s].sc->pact[it & 1]);
      }
      go = g;
      int m = 0;
      if (my >= 0)
        for (int j = 0; j < b.sys[my].k; ++j) m |= l_state[j] == ST_ACTIVE;
      mine = m;
    }
    __syncthreads();
    if (!go) break;
    if (lead && mine && threadIdx.x == 0) atomicMax(b.bar + 3, (unsigned)(it + 1));  // iterations with work
    // ---- phase A: q = A p, p.q, q.D^-1 q
    if (mine) {
      const PSys& S = b.sys[my];
      switch (S.vec) {
        case 1: pphase_q<1>(b, S, red, out); break;
        case 2: pphase_q<2>(b, S, red, out); break;
        case 3: pphase_q<3>(b, S, red, out); break;
        case 4: pphase_q<4>(b, S, red, out); break;
      }
    }
    if (!grid_barrier(b)) return;
    // ---- phase B: alpha and beta from the system's sums, then x, r, p and the new products
    if (mine) {
      const PSys& S = b.sys[my];
      psys_totals(b, S, 0, 2 * S.k, tot);
      const int j = threadIdx.x;
      if (j < S.k) {
        const double pq = tot[j], qdq = tot[S.k + j];
        double al = 0.0, be = 0.0;
        if (l_state[j] == ST_ACTIVE) {
          if (!(pq > 0.0) || !isfinite(pq) || !isfinite(qdq)) {
            l_state[j] = ST_DONE;
          } else {
            al = l_rz[j] / pq;
            const double bb = l_rz[j] * qdq / (pq * pq) - 1.0;
            be = (bb > 0.0 && isfinite(bb)) ? bb : 0.0;
          }
        }
        l_alpha[j] = al;
        l_beta[j] = be;
        if (lead) {
          S.sc->pq[j] = pq;
          S.sc->alpha[j] = al;
          S.sc->beta[j] = be;
        }
      }
      __syncthreads();
      switch (S.vec) {
        case 1: pphase_xrp<1>(b, S, l_alpha, l_beta, l_state, red, out); break;
        case 2: pphase_xrp<2>(b, S, l_alpha, l_beta, l_state, red, out); break;
        case 3: pphase_xrp<3>(b, S, l_alpha, l_beta, l_state, red, out); break;
        case 4: pphase_xrp<4>(b, S, l_alpha, l_beta, l_state, red, out); break;
      }
    }
    if (!grid_barrier(b)) return;
    // ---- convergence from r.D^-1 r and r.r (every block of the system, identically)
    if (mine) {
      const PSys& S = b.sys[my];
      psys_totals(b, S, 2, 2 * S.k, tot);
      const int j = threadIdx.x;
      if (j < S.k) {
        const double rz_new = tot[j], rr_new = tot[S.k + j];
        if (l_state[j] == ST_ACTIVE) {
          l_iters[j] += 1;
          l_rz[j] = rz_new;
          if (!isfinite(rr_new) || !isfinite(rz_new)) l_state[j] = ST_DONE;
          else if (rr_new <= S.sc->tol2[j]) l_met[j] = 1;
          if (lead) S.sc->rr[j] = rr_new;
        }
      }
      __syncthreads();
      // as in the two-kernel loop: columns that met their target keep iterating until every
      // active column of the system has
      if (threadIdx.x == 0) {
        bool all = true;
        for (int c = 0; c < S.k; ++c) all &= l_state[c] != ST_ACTIVE || l_met[c] != 0;
        if (all)
          for (int c = 0; c < S.k; ++c)
            if (l_state[c] == ST_ACTIVE) l_state[c] = ST_DONE;
      }
      __syncthreads();
      if (lead && j < S.k) {
        S.sc->iters[j] = l_iters[j];
        S.sc->state[j] = l_state[j];
        S.sc->rz[j] = l_rz[j];
      }
      __syncthreads();
      if (lead && threadIdx.x == 0) recount(S.sc, S.k);
    }
    if (lead && threadIdx.x == 0) {
      int m = 0;
      for (int j = 0; j < b.sys[my].k; ++j) m |= l_state[j] == ST_ACTIVE;
      b.sys[my].sc->pact[it & 1] = m;
      __threadfence();
    }
  }
  if (lead && threadIdx.x == 0) recount(b.sys[my].sc, b.sys[my].k);
}

// ------------------------------------------------------------------ host side of the batch

int sm_count() {
  thread_local int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
      sms = 152;
  }
  return sms;
}

// Resident blocks of k_pcg_batch per multiprocessor (the cooperative-launch limit).
int pcg_blocks_per_sm() {
  thread_local int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batch, kPThreads, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  return per_sm;
}

constexpr int kPGridMax = 152 * 4;  // partials capacity: 4 resident blocks of 512 threads per SM

// Blocks per system in proportion to the bytes one iteration streams (rows x (2 + k)), at
// least one each; the first total_cols blocks double as the column reducers.
void partition_blocks(PBatch& pb, int grid) {
  double W = 0.0;
  for (int s = 0; s < pb.n_sys; ++s) W += (double)pb.sys[s].n * (2 + pb.sys[s].k);
  int used = 0;
  for (int s = 0; s < pb.n_sys; ++s) {
    int nb = (int)std::floor(grid * ((double)pb.sys[s].n * (2 + pb.sys[s].k)) / std::max(W, 1.0));
    nb = std::max(1, nb);
    pb.sys[s].nblk = nb;
    used += nb;
  }
  while (used > grid) {  // trim the largest share
    int big = 0;
    for (int s = 1; s < pb.n_sys; ++s)
      if (pb.sys[s].nblk > pb.sys[big].nblk) big = s;
    --pb.sys[big].nblk;
    --used;
  }
  while (used < grid) {  // give the rest to the heaviest per block
    int best = 0;
    double wb = -1.0;
    for (int s = 0; s < pb.n_sys; ++s) {
      const double w = (double)pb.sys[s].n * (2 + pb.sys[s].k) / pb.sys[s].nblk;
      if (w > wb) wb = w, best = s;
    }
    ++pb.sys[best].nblk;
    ++used;
  }
  int b0 = 0;
  for (int s = 0; s < pb.n_sys; ++s) {
    pb.sys[s].blk0 = b0;
    b0 += pb.sys[s].nblk;
  }
}

rb_status launch_pcg(const PBatch& pb, int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RB_CUDA(cudaLaunchKernelEx(&cfg, k_pcg_batch, pb));
  return RB_OK;
}

// Column layout of the vector kernels for k columns and this B / X.
int solver_vec(int k, int64_t ldx, int64_t ldb, const void* X, const void* B) {
  int vec = 1;
  if (k <= 4 && (k != 2 || vec_ok(8, 2, k, ldx, ldb, X, B))) vec = k;
  else if (k % 4 == 0) vec = 4;
  else if (k % 3 == 0) vec = 3;
  else if (vec_ok(8, 2, k, ldx, ldb, X, B)) vec = 2;
  return vec;
}

rb_status validate_solve(const char* fn, rb_op_t A, rb_op_t A_inner, const rb_cg_params& prm, const double* B,
                         int64_t ldb, const double* X, int64_t ldx, int32_t k) {
  RB_REQUIRE(A, "%s: null operator", fn);
  RB_REQUIRE(A->dtype == RB_F64, "%s: the operator must be RB_F64", fn);
  RB_REQUIRE(A->n_rows == A->n_cols, "%s: the operator must be square", fn);
  RB_REQUIRE(A->ext_nz == 0, "%s: extruded operators are not supported by the solver", fn);
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "%s: k = %d outside [1, %d]", fn, k, RB_MAX_K);
  RB_REQUIRE(ldb >= k && ldx >= k, "%s: leading dimension smaller than k", fn);
  RB_REQUIRE(A->n_rows == 0 || (B && X), "%s: null B or X", fn);
  RB_REQUIRE(prm.rtol > 0 && std::isfinite(prm.rtol), "%s: rtol must be positive", fn);
  RB_REQUIRE(prm.max_iter >= 0 && prm.check_every >= 1, "%s: max_iter >= 0 and check_every >= 1 required", fn);
  RB_REQUIRE(!prm.precond || A->has_diag, "%s: Jacobi needs a nonzero diagonal in every row", fn);
  RB_REQUIRE(prm.mixed >= 0 && prm.mixed <= 2, "%s: mixed must be 0, 1 or 2", fn);
  if (prm.mixed) {
    RB_REQUIRE(A_inner && A_inner->dtype == RB_F32 && A_inner->n_rows == A->n_rows && A_inner->nnz == A->nnz,
               "%s: mixed precision needs A_inner, the same matrix stored as RB_F32", fn);
    RB_REQUIRE(A_inner->format == RB_CSR || A_inner->format == RB_STENCIL,
               "%s: the inner operator must be CSR or matrix-free (RB_STENCIL)", fn);
    RB_REQUIRE(prm.inner_rtol > 0 && prm.inner_rtol < 1, "%s: inner_rtol must be in (0, 1)", fn);
    RB_REQUIRE(prm.max_sweeps >= 1, "%s: max_sweeps >= 1 required", fn);
  }
  RB_REQUIRE(A->format == RB_CSR, "%s: the operator must be CSR", fn);
  RB_REQUIRE((uintptr_t)B % 8 == 0 && (uintptr_t)X % 8 == 0, "%s: B or X not 8-byte aligned", fn);
  return RB_OK;
}

// Launch shapes, scalars and controls of one solve whose workspace starts at `base`.
rb_status init_solver(Solver& S_, rb_op_t A, rb_op_t A_inner, const rb_cg_params& prm, int32_t k, const double* B,
                      int64_t ldb, const double* X, int64_t ldx, char* base, const Layout& L, cudaStream_t s) {
  S_.A = A;
  S_.A32 = A_inner;
  S_.k = k;
  S_.n = A->n_rows;
  S_.s = s;
  const int vec = solver_vec(k, ldx, ldb, X, B);
  S_.vec = vec;
  S_.kp = next_pow2(k / vec);
  RB_REQUIRE(S_.kp <= 32, "solve: k = %d needs 16-byte aligned B and X rows", k);
  S_.sched64 = pick_sched(A, k, k, k, base + L.r, base + L.p);
  S_.sched64.vec = vec;
  S_.sched64.kp = S_.kp;
  if (S_.sched64.kp * S_.sched64.lpr > 32) S_.sched64.lpr = 1;
  if (prm.mixed) {
    S_.sched32 = pick_sched(A_inner, k, k, k, base + L.p32, base + L.q32);
    S_.sched32.vec = vec;  // the same (row, chunk) layout as the vector kernels
    S_.sched32.kp = S_.kp;
    if (S_.sched32.kp * S_.sched32.lpr > 32) S_.sched32.lpr = 1;
  }
  S_.sc = reinterpret_cast<CgScal*>(base + L.scal);
  S_.partials = reinterpret_cast<double*>(base + L.partials);
  S_.ctl.k = k;
  S_.ctl.kp = S_.kp;
  S_.ctl.n = S_.n;
  S_.ctl.inner = 0;
  S_.ctl.project = prm.project_mean ? 1 : 0;
  S_.ctl.reliable = prm.mixed == 2 ? 1 : 0;
  S_.ctl.rtol2 = prm.rtol * prm.rtol;
  S_.ctl.inner_rtol2 = prm.inner_rtol * prm.inner_rtol;
  return RB_OK;
}

PSys make_psys(const Solver& S_, const Layout& L, char* base, bool precond) {
  PSys p{};
  p.rp = S_.A32->row_ptr;
  p.ci = S_.A32->col_idx;
  p.va = static_cast<const float*>(S_.A32->vals);
  p.mf = S_.A32->format == RB_STENCIL ? 1 : 0;
  if (p.mf) {
    for (int d = 0; d < 3; ++d) {
      p.st.n[d] = S_.A32->st_n[d];
      p.st.per[d] = S_.A32->st_per[d];
      p.st.w[d] = static_cast<const float*>(S_.A32->st_w[d]);
      p.st.ic[d] = static_cast<const float*>(S_.A32->st_ic[d]);
    }
    p.st.scale = (float)S_.A32->st_scale;
    p.st.init_div();
  }
  p.dinv = precond ? S_.A32->dinv32 : nullptr;
  p.r = reinterpret_cast<float*>(base + L.r32);
  p.p = reinterpret_cast<float*>(base + L.p32);
  p.q = reinterpret_cast<float*>(base + L.q32);
  p.d = reinterpret_cast<float*>(base + L.d32);
  p.sc = S_.sc;
  p.n = (int)S_.n;
  p.k = S_.k;
  p.vec = S_.vec;
  p.kp = S_.kp;
  p.blk0 = 0;
  p.nblk = 1;
  p.col0 = 0;
  return p;
}

// The per-system kernels of one refinement sweep, before and after the inner solve.
template <int VEC>
void sweep_head(Solver& S_, const rb_cg_params& prm, const double* B, int64_t ldb, const double* X, int64_t ldx,
                const Layout& L, char* base) {
  double* r64 = reinterpret_cast<double*>(base + L.r64);
  float* r32 = reinterpret_cast<float*>(base + L.r32);
  float* p32 = reinterpret_cast<float*>(base + L.p32);
  float* d32 = reinterpret_cast<float*>(base + L.d32);
  const float* dinv32 = prm.precond ? S_.A32->dinv32 : nullptr;
  CgCtl c = S_.ctl;
  c.inner = 1;
  S_.launch_resid_v<VEC>(RM_OUTER, B, ldb, X, ldx, r64);
  k_ir_init<VEC><<<S_.vg(&k_ir_init<VEC>), kThreads, 0, S_.s>>>(c, r64, r32, p32, d32, dinv32, S_.sc, S_.partials);
}

template <int VEC>
void sweep_tail(Solver& S_, double* X, int64_t ldx, const Layout& L, char* base) {
  float* d32 = reinterpret_cast<float*>(base + L.d32);
  CgCtl c = S_.ctl;
  c.inner = 1;
  k_ir_update<VEC><<<S_.vg(&k_ir_update<VEC>), kThreads, 0, S_.s>>>(c, X, ldx, d32, S_.sc);
}

template <int VEC>
void solve_tail(Solver& S_, const rb_cg_params& prm, const double* B, int64_t ldb, double* X, int64_t ldx) {
  if (prm.project_mean) {
    k_colsum<VEC><<<S_.vg(&k_colsum<VEC>), kThreads, 0, S_.s>>>(S_.ctl, X, ldx, S_.sc, S_.partials);
    k_submean<VEC><<<S_.vg(&k_submean<VEC>), kThreads, 0, S_.s>>>(S_.ctl, X, ldx, S_.sc);
  }
  S_.launch_resid_v<VEC>(RM_REPORT, B, ldb, X, ldx, nullptr);
}

#define RB_VEC_SWITCH(vec, CALL) \
  switch (vec) {                 \
    case 2: CALL(2); break;      \
    case 3: CALL(3); break;      \
    case 4: CALL(4); break;      \
    default: CALL(1); break;     \
  }

rb_status persistent_inner(Solver& S_, const rb_cg_params& prm, const Layout& L, char* base) {
  PBatch pb;
  pb.n_sys = 1;
  pb.sys[0] = make_psys(S_, L, base, prm.precond != 0);
  pb.total_cols = S_.k;
  pb.partials = S_.partials;  // the workspace's partials hold kGridMax x 3 x K >= kPGridMax x 4 x K
  pb.bar = S_.sc->pbar;
  pb.err = reinterpret_cast<int*>(&S_.sc->pbar[2]);
  pb.max_iter = prm.max_iter;
  pb.extra_arrivals = 0;
  pb.timeout_ns = 2000000000ull;
  const int grid = std::min(kPGridMax, pcg_blocks_per_sm() * sm_count());
  partition_blocks(pb, grid);
  RB_CUDA(cudaMemsetAsync(S_.sc->pbar, 0, 4 * sizeof(unsigned), S_.s));
  return launch_pcg(pb, grid, S_.s);
}

void fill_report(const CgScal& hs, int k, int mixed, rb_cg_report& rep, rb_status& worst) {
  for (int j = 0; j < k; ++j) {
    rep.iters[j] = hs.iters[j];
    rep.true_rel_res[j] = hs.bb[j] > 0 ? sqrt(hs.rr_true[j] / hs.bb[j]) : 0.0;
    const int st = mixed ? hs.ostate[j] : hs.state[j];
    // the recorded batch sequence ends after its last sweep without another outer check: a
    // column whose final true residual (just computed in FP64) meets the tolerance has converged
    const double tol2 = mixed ? hs.otol2[j] : hs.tol2[j];
    const bool met = hs.bb[j] > 0 && hs.rr_true[j] <= tol2;
    rb_status cs = RB_OK;
    if (st == ST_BREAKDOWN) cs = RB_EBREAKDOWN;
    else if ((st == ST_NOCONV || st == ST_ACTIVE || st == ST_RESTART) && !met) cs = RB_ENOCONV;
    rep.status[j] = cs;
    if (cs == RB_EBREAKDOWN || (cs == RB_ENOCONV && worst == RB_OK)) worst = cs;
  }
}

}  // namespace
}  // namespace rb

// --------------------------------------------------------------------------- batch object
struct rb_batch {
  int n_sys = 0;
  rb_op_t A[rb::kMaxSys] = {}, A32[rb::kMaxSys] = {};
  int k[rb::kMaxSys] = {};
  rb_cg_params prm{};
  void* work[rb::kMaxSys] = {};
  rb::Layout L[rb::kMaxSys];
  double* partials = nullptr;
  unsigned* bar = nullptr;  // [0] arrivals, [1] generation, [2] error word
  int blocks_per_sm = 0;    // 0: as many as fit
  int extra_arrivals = 0;
  double timeout_ms = 2000.0;
  // recorded graph and the pointers it was recorded for
  cudaGraphExec_t exec = nullptr;
  const double* gB[rb::kMaxSys] = {};
  double* gX[rb::kMaxSys] = {};
  int64_t gldb[rb::kMaxSys] = {}, gldx[rb::kMaxSys] = {};
  ~rb_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (int s = 0; s < rb::kMaxSys; ++s)
      if (work[s]) cudaFree(work[s]);
    if (partials) cudaFree(partials);
    if (bar) cudaFree(bar);
  }
};

namespace rb {
namespace {

char* ws_base(void* w) { return reinterpret_cast<char*>(((uintptr_t)w + 255) & ~(uintptr_t)255); }

// Records (eagerly executes when `s` is not capturing) the whole batched solve on stream s.
rb_status batch_sequence(rb_batch* bt, Solver* SV, PBatch& pb, int grid, const double* const* B, const int64_t* ldb,
                         double* const* X, const int64_t* ldx, cudaStream_t s) {
  for (int i = 0; i < bt->n_sys; ++i) {
    SV[i].s = s;
    RB_CUDA(cudaMemsetAsync(SV[i].sc, 0, sizeof(CgScal), s));
    k_init_outer<<<1, K, 0, s>>>(SV[i].sc, bt->k[i]);
  }
  for (int sweep = 0; sweep < bt->prm.max_sweeps; ++sweep) {
    for (int i = 0; i < bt->n_sys; ++i) {
      char* base = ws_base(bt->work[i]);
#define RB_HEAD(V) sweep_head<V>(SV[i], bt->prm, B[i], ldb[i], X[i], ldx[i], bt->L[i], base)
      RB_VEC_SWITCH(SV[i].vec, RB_HEAD)
#undef RB_HEAD
    }
    RB_CUDA(cudaMemsetAsync(bt->bar, 0, 4 * sizeof(unsigned), s));
    RB_TRY(launch_pcg(pb, grid, s));
    for (int i = 0; i < bt->n_sys; ++i) {
      char* base = ws_base(bt->work[i]);
#define RB_TAIL(V) sweep_tail<V>(SV[i], X[i], ldx[i], bt->L[i], base)
      RB_VEC_SWITCH(SV[i].vec, RB_TAIL)
#undef RB_TAIL
    }
  }
  for (int i = 0; i < bt->n_sys; ++i) {
#define RB_STAIL(V) solve_tail<V>(SV[i], bt->prm, B[i], ldb[i], X[i], ldx[i])
    RB_VEC_SWITCH(SV[i].vec, RB_STAIL)
#undef RB_STAIL
  }
  RB_CUDA(cudaGetLastError());
  return RB_OK;
}

rb_status batch_prepare(rb_batch* bt, Solver* SV, PBatch& pb, int& grid, const double* const* B, const int64_t* ldb,
                        double* const* X, const int64_t* ldx, cudaStream_t s) {
  pb = PBatch();
  pb.n_sys = bt->n_sys;
  int col = 0;
  for (int i = 0; i < bt->n_sys; ++i) {
    char* base = ws_base(bt->work[i]);
    RB_TRY(init_solver(SV[i], bt->A[i], bt->A32[i], bt->prm, bt->k[i], B[i], ldb[i], X[i], ldx[i], base, bt->L[i], s));
    pb.sys[i] = make_psys(SV[i], bt->L[i], base, bt->prm.precond != 0);
    pb.sys[i].col0 = col;
    col += bt->k[i];
  }
  pb.total_cols = col;
  pb.partials = bt->partials;
  pb.bar = bt->bar;
  pb.err = reinterpret_cast<int*>(bt->bar + 2);
  pb.max_iter = bt->prm.max_iter;
  pb.extra_arrivals = bt->extra_arrivals;
  pb.timeout_ns = (unsigned long long)(bt->timeout_ms * 1e6);
  const int cap = pcg_blocks_per_sm();
  const int bps = bt->blocks_per_sm > 0 ? std::min(bt->blocks_per_sm, cap) : cap;
  grid = std::min(kPGridMax, bps * sm_count());
  grid = std::max(grid, pb.total_cols);
  RB_REQUIRE(grid <= cap * sm_count(), "batch: %d columns need more co-resident blocks than fit", pb.total_cols);
  partition_blocks(pb, grid);
  return RB_OK;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_batch_create(int32_t n_sys, const rb_op_t* ops, const rb_op_t* ops_inner, const int32_t* k,
                                     const rb_cg_params* params, rb_batch_t* out) {
  clear_error();
  RB_REQUIRE(out && ops && ops_inner && k && params, "rb_batch_create: null argument");
  *out = nullptr;
  RB_REQUIRE(n_sys >= 1 && n_sys <= kMaxSys, "rb_batch_create: n_sys = %d outside [1, %d]", n_sys, kMaxSys);
  RB_REQUIRE(params->mixed == 1 || params->mixed == 2, "rb_batch_create: the batch runs the FP32-inner refinement "
             "(params->mixed 1 or 2)");
  int cols = 0;
  for (int i = 0; i < n_sys; ++i) {
    RB_TRY(validate_solve("rb_batch_create", ops[i], ops_inner[i], *params, reinterpret_cast<const double*>(8),
                          k[i], reinterpret_cast<const double*>(8), k[i], k[i]));
    RB_REQUIRE(ops[i]->n_rows > 0, "rb_batch_create: system %d is empty", i);
    cols += k[i];
  }
  RB_REQUIRE(cols <= RB_MAX_K, "rb_batch_create: %d columns in total exceed %d", cols, RB_MAX_K);
  rb_batch* bt = new rb_batch();
  bt->n_sys = n_sys;
  bt->prm = *params;
  for (int i = 0; i < n_sys; ++i) {
    bt->A[i] = ops[i];
    bt->A32[i] = ops_inner[i];
    bt->k[i] = k[i];
    bt->L[i] = layout(ops[i]->n_rows, k[i], true);
    cudaError_t e = cudaMalloc(&bt->work[i], bt->L[i].total + 256);
    if (e != cudaSuccess) {
      delete bt;
      return cuda_fail(e, "cudaMalloc (batch workspace)", __FILE__, __LINE__);
    }
  }
  cudaError_t e = cudaMalloc(&bt->partials, (size_t)kPGridMax * 4 * K * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&bt->bar, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(bt->bar, 0, 4 * sizeof(unsigned));
  if (e != cudaSuccess) {
    delete bt;
    return cuda_fail(e, "cudaMalloc (batch state)", __FILE__, __LINE__);
  }
  *out = bt;
  return RB_OK;
}

extern "C" rb_status rb_batch_destroy(rb_batch_t batch) {
  clear_error();
  delete batch;
  return RB_OK;
}

extern "C" rb_status rb_batch_set_barrier(rb_batch_t batch, double timeout_ms, int32_t extra_arrivals) {
  clear_error();
  RB_REQUIRE(batch, "rb_batch_set_barrier: null batch");
  RB_REQUIRE(timeout_ms > 0 && extra_arrivals >= 0, "rb_batch_set_barrier: invalid knob");
  batch->timeout_ms = timeout_ms;
  batch->extra_arrivals = extra_arrivals;
  if (batch->exec) {
    cudaGraphExecDestroy(batch->exec);
    batch->exec = nullptr;
  }
  return RB_OK;
}

extern "C" rb_status rb_batch_solve(rb_batch_t bt, const double* const* B, const int64_t* ldb, double* const* X,
                                    const int64_t* ldx, rb_cg_report* reports, rb_stream_t stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  RB_REQUIRE(bt && B && ldb && X && ldx, "rb_batch_solve: null argument");
  for (int i = 0; i < bt->n_sys; ++i)
    RB_TRY(validate_solve("rb_batch_solve", bt->A[i], bt->A32[i], bt->prm, B[i], ldb[i], X[i], ldx[i], bt->k[i]));
  cudaStream_t s = S(stream);
  Solver SV[kMaxSys];
  PBatch pb;
  int grid = 0;
  RB_TRY(batch_prepare(bt, SV, pb, grid, B, ldb, X, ldx, s));
  bool same = bt->exec != nullptr;
  for (int i = 0; i < bt->n_sys && same; ++i)
    same = bt->gB[i] == B[i] && bt->gX[i] == X[i] && bt->gldb[i] == ldb[i] && bt->gldx[i] == ldx[i];
  if (!same) {
    if (bt->exec) {
      cudaGraphExecDestroy(bt->exec);
      bt->exec = nullptr;
    }
    // warm the launch-shape caches outside the capture
    for (int i = 0; i < bt->n_sys; ++i) {
#define RB_WARM(V) (void)SV[i].vg(&k_ir_init<V>), (void)SV[i].vg(&k_ir_update<V>), \
                   (void)SV[i].vg(&k_colsum<V>), (void)SV[i].vg(&k_submean<V>)
      RB_VEC_SWITCH(SV[i].vec, RB_WARM)
#undef RB_WARM
    }
    cudaStream_t cs = capture_stream();
    cudaGraph_t graph = nullptr;
    cudaError_t e = cs ? cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) : cudaErrorNotSupported;
    rb_status st = RB_OK;
    if (e == cudaSuccess) {
      st = batch_sequence(bt, SV, pb, grid, B, ldb, X, ldx, cs);
      e = cudaStreamEndCapture(cs, &graph);
    }
    if (st == RB_OK && e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != RB_OK) return st;
    if (e == cudaSuccess) {
      for (int i = 0; i < bt->n_sys; ++i) {
        bt->gB[i] = B[i];
        bt->gX[i] = X[i];
        bt->gldb[i] = ldb[i];
        bt->gldx[i] = ldx[i];
      }
    } else {
      cudaGetLastError();  // this runtime cannot record the sequence: run it eagerly
      bt->exec = nullptr;
    }
  }
  if (bt->exec) {
    RB_CUDA(cudaGraphLaunch(bt->exec, s));
  } else {
    RB_TRY(batch_sequence(bt, SV, pb, grid, B, ldb, X, ldx, s));
  }
  CgScal hs[kMaxSys];
  unsigned hb[4];
  for (int i = 0; i < bt->n_sys; ++i)
    RB_CUDA(cudaMemcpyAsync(&hs[i], SV[i].sc, sizeof(CgScal), cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaMemcpyAsync(hb, bt->bar, sizeof(hb), cudaMemcpyDeviceToHost, s));
  RB_CUDA(cudaStreamSynchronize(s));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  rb_status worst = RB_OK;
  for (int i = 0; i < bt->n_sys; ++i) {
    rb_cg_report rep;
    std::memset(&rep, 0, sizeof(rep));
    fill_report(hs[i], bt->k[i], 1, rep, worst);
    rep.sweeps = bt->prm.max_sweeps;
    rep.host_syncs = 1;
    rep.ms = ms;
    if (reports) reports[i] = rep;
  }
  if (hb[2] != 0) {
    set_error("rb_batch_solve: a grid barrier wait gave up (timeout %.1f ms); the solutions are invalid",
              bt->timeout_ms);
    return RB_ETIMEOUT;
  }
  if (worst == RB_ENOCONV) set_error("rb_batch_solve: a column did not converge within max_sweeps / max_iter");
  if (worst == RB_EBREAKDOWN) set_error("rb_batch_solve: breakdown in a column");
  return worst;
}

extern "C" rb_status rb_batch_tune(rb_batch_t bt, const double* const* B, const int64_t* ldb, double* const* X,
                                   const int64_t* ldx, double* best_ms, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(bt && B && ldb && X && ldx, "rb_batch_tune: null argument");
  cudaStream_t s = S(stream);
  const int cap = pcg_blocks_per_sm();
  const double rtols[] = {1e-1, 5e-2, 3e-2, 1e-2};
  double best = 1e30;
  int best_bps = 0;
  double best_rtol = bt->prm.inner_rtol;
  for (int bps = 1; bps <= cap; ++bps) {
    for (double it : rtols) {
      if (bt->prm.mixed == 1 && it > 1e-2) continue;  // restarted refinement wants tighter inner solves
      bt->blocks_per_sm = bps;
      bt->prm.inner_rtol = it;
      if (bt->exec) {
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
      }
      double t = 0.0;
      rb_status st = RB_OK;
      for (int rep = 0; rep < 2 && st == RB_OK; ++rep) {
        for (int i = 0; i < bt->n_sys; ++i)
          RB_CUDA(cudaMemset2DAsync(X[i], ldx[i] * sizeof(double), 0, bt->k[i] * sizeof(double), bt->A[i]->n_rows, s));
        RB_CUDA(cudaStreamSynchronize(s));
        const auto t0 = std::chrono::steady_clock::now();
        st = rb_batch_solve(bt, B, ldb, X, ldx, nullptr, stream);
        t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      }
      if (st == RB_OK && t < best) {
        best = t;
        best_bps = bps;
        best_rtol = it;
      }
    }
  }
  bt->blocks_per_sm = best_bps;
  bt->prm.inner_rtol = best_rtol;
  if (bt->exec) {
    cudaGraphExecDestroy(bt->exec);
    bt->exec = nullptr;
  }
  if (best_ms) *best_ms = best;
  clear_error();
  return best < 1e30 ? RB_OK : RB_ENOCONV;
}

extern "C" size_t rb_cg_workspace_bytes(rb_op_t A, int32_t k, const rb_cg_params* params) {
  if (!A || !params || k < 1 || k > RB_MAX_K) return 0;
  return layout(A->n_rows, k, params->mixed != 0).total + 256;
}

extern "C" rb_status rb_cg_solve(rb_op_t A, rb_op_t A_inner, const rb_cg_params* params, const double* B,
                                 int64_t ldb, double* X, int64_t ldx, int32_t k, void* work, size_t work_bytes,
                                 rb_cg_report* report, rb_stream_t stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  RB_REQUIRE(A && params, "rb_cg_solve: null operator or params");
  const rb_cg_params& prm = *params;
  RB_TRY(validate_solve("rb_cg_solve", A, A_inner, prm, B, ldb, X, ldx, k));
  RB_REQUIRE(!prm.persistent || prm.mixed, "rb_cg_solve: the persistent launch serves the refinement (mixed 1 or 2)");
  const Layout L = layout(A->n_rows, k, prm.mixed != 0);
  RB_REQUIRE(work && work_bytes >= L.total + 256, "rb_cg_solve: workspace too small (%zu < %zu)", work_bytes,
             L.total + 256);
  rb_cg_report rep;
  std::memset(&rep, 0, sizeof(rep));
  if (A->n_rows == 0) {
    if (report) *report = rep;
    return RB_OK;
  }
  char* base = reinterpret_cast<char*>(((uintptr_t)work + 255) & ~(uintptr_t)255);
  // columns per thread: all k for k <= 4 (one thread per row; 4 doubles as scalar loads), 3
  // for multiples of 3, else 2 when the FP64 rows of B and X are 16-byte aligned, else 1.
  // Internal vectors have ld = k and 256-byte aligned bases.
  Solver S_;
  RB_TRY(init_solver(S_, A, A_inner, prm, k, B, ldb, X, ldx, base, L, S(stream)));
  RB_CUDA(cudaMemsetAsync(S_.sc, 0, sizeof(CgScal), S_.s));
  rb_status st;
  switch (S_.vec) {
    case 2: st = solve_vec<2>(S_, prm, B, ldb, X, ldx, L, base, rep); break;
    case 3: st = solve_vec<3>(S_, prm, B, ldb, X, ldx, L, base, rep); break;
    case 4: st = solve_vec<4>(S_, prm, B, ldb, X, ldx, L, base, rep); break;
    default: st = solve_vec<1>(S_, prm, B, ldb, X, ldx, L, base, rep); break;
  }
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (report) *report = rep;
  if (st != RB_OK && st != RB_ENOCONV && st != RB_EBREAKDOWN) return st;
  if (st == RB_ENOCONV) set_error("rb_cg_solve: a column did not converge in max_iter iterations");
  if (st == RB_EBREAKDOWN) set_error("rb_cg_solve: breakdown (p.q <= 0 or not finite) in a column");
  return st;
}
