// The projection step on m stacked flow states (Sec. 3, Eq. (ns) and Eq. (ns-nrhs); Sec. 4:
// Heun's third-order Runge-Kutta scheme with a projection at every stage), sequenced in the
// library on its own calls: every operator application is one SpMM over the states' columns
// (I_m (x) A), the convective term is the divergence SpMM of an axty of the face velocities
// with the face-interpolated cell velocities, and each projection is a Poisson solve by
// rb_cg_solve or rb_mg_solve.
//
// Layout: u_c is n x 3 m with column i m + s for component i of state s; u_s is n_faces x m,
// the x faces first, then y, then z (on a periodic axis a direction has n faces).  The grid is
// uniform and periodic along every axis, so the cell volume is one number and the
// face-to-cell interpolator is the transpose of the cell-to-face one.
//
//   derivative:  F = Omega^{-1} (nu L u - M (u_s * Gamma u))       (Omega = V I)
//   projection:  u~_s = the face-normal components of Gamma u~, -L p = -M u~_s / (c dt)
//                (zero-mean p), u_s = u~_s - c dt G p, u_c = u~ - c dt G_c p, G_c p's
//                component d being Gamma^T applied to G p on the faces of direction d
//   Heun RK3:    c = (0, 1/3, 2/3), a_21 = 1/3, a_32 = 2/3, b = (1/4, 0, 3/4)
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

struct rb_projection {
  int n = 0, nf = 0, m = 0, m3 = 0;
  double nu = 0.0, dt = 0.0, vol = 0.0;
  int solver = RB_PROJ_JACOBI;
  rb_cg_params prm{};
  rb_op_t M = nullptr, G = nullptr, L = nullptr, A = nullptr, A32 = nullptr, I = nullptr, IT = nullptr;
  rb_mg_t mg = nullptr;
  void* work = nullptr;
  size_t work_bytes = 0;
  double *Y = nullptr, *Gm = nullptr, *ut_s = nullptr, *g = nullptr, *B = nullptr, *ut = nullptr, *tmp = nullptr,
         *us_stage = nullptr;
  double* P[3] = {nullptr, nullptr, nullptr};
  double* F[3] = {nullptr, nullptr, nullptr};
  // column scales: 1 (m and 3 m), nu / V and -1 / V (3 m), the stage combinations dt a
  // (1/3, 2/3, 1/4, 3/4; 3 m), and a projection's -1 / (c dt) (m), -c dt (m) and -c dt (3 m)
  double *one_m = nullptr, *one_m3 = nullptr, *c_diff = nullptr, *c_conv = nullptr;
  double* c_comb[4] = {nullptr, nullptr, nullptr, nullptr};
  double *c_rhs = nullptr, *c_gm = nullptr, *c_gm3 = nullptr;
  std::vector<void*> allocs;
};

namespace rb {
namespace {

constexpr double kHeunC[3] = {0.0, 1.0 / 3.0, 2.0 / 3.0};
constexpr double kComb[4] = {1.0 / 3.0, 2.0 / 3.0, 0.25, 0.75};  // dt a_21, dt a_32, dt b_1, dt b_3

__global__ void k_fill3(double* a, int ka, double va, double* b, int kb, double vb, double* c, int kc, double vc) {
  const int t = threadIdx.x;
  if (t < ka) a[t] = va;
  if (t < kb) b[t] = vb;
  if (t < kc) c[t] = vc;
}

rb_status palloc(rb_projection* p, double** out, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("rb_projection_create: device allocation of %zu bytes failed", count * sizeof(double));
    return RB_ENOMEM;
  }
  p->allocs.push_back(q);
  *out = static_cast<double*>(q);
  return RB_OK;
}

void release(rb_projection* p) {
  for (rb_op_t o : {p->M, p->G, p->L, p->A, p->A32, p->I, p->IT})
    if (o) rb_operator_destroy(o);
  if (p->mg) rb_mg_destroy(p->mg);
  for (void* q : p->allocs) cudaFree(q);
  if (p->work) cudaFree(p->work);
  delete p;
}

// operator `kind` times `scale` on the grid, stored in `dtype` for up to k columns
rb_status make_op(const rb_grid_desc* grid, rb_fvm_kind kind, double scale, rb_dtype dtype, int k, cudaStream_t s,
                  rb_op_t* out) {
  int32_t nr = 0, nc = 0;
  int64_t nnz = 0;
  RB_TRY(rb_fvm_csr_size(grid, kind, &nr, &nc, &nnz));
  int32_t *rp = nullptr, *ci = nullptr;
  double* va = nullptr;
  rb_status st = RB_OK;
  if (cudaMalloc(&rp, sizeof(int32_t) * (nr + 1)) != cudaSuccess || cudaMalloc(&ci, sizeof(int32_t) * nnz) != cudaSuccess ||
      cudaMalloc(&va, sizeof(double) * nnz) != cudaSuccess) {
    cudaGetLastError();
    set_error("rb_projection_create: device allocation for an operator failed");
    st = RB_ENOMEM;
  }
  if (st == RB_OK) st = rb_fvm_assemble(grid, kind, scale, rp, ci, va, reinterpret_cast<rb_stream_t>(s));
  if (st == RB_OK) {
    rb_csr_desc d{nr, nc, nnz, rp, ci, va, 1};
    rb_block_desc b{k, 0, nullptr, 0.0};
    st = rb_operator_create(&d, &b, dtype, RB_CSR, reinterpret_cast<rb_stream_t>(s), out);
  }
  cudaFree(rp);
  cudaFree(ci);
  cudaFree(va);
  return st;
}

rb_status spmm(rb_op_t op, const double* X, int64_t ldx, double* Y, int64_t ldy, int k, const double* c,
               cudaStream_t s) {
  return rb_spmm(op, X, ldx, Y, ldy, k, c, reinterpret_cast<rb_stream_t>(s));
}
rb_status axpy(int64_t n, int k, const double* alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
               cudaStream_t s) {
  return rb_axpy(n, k, RB_F64, alpha, X, ldx, Y, ldy, reinterpret_cast<rb_stream_t>(s));
}
rb_status copy2d(double* dst, int64_t ldd, const double* src, int64_t lds, int64_t rows, int cols, cudaStream_t s) {
  RB_CUDA(cudaMemcpy2DAsync(dst, (size_t)ldd * 8, src, (size_t)lds * 8, (size_t)cols * 8, (size_t)rows,
                            cudaMemcpyDeviceToDevice, s));
  return RB_OK;
}

// F = Omega^{-1} (nu L u - M (u_s * Gamma u)); u: n x 3 m (ldu), us: nf x m (contiguous)
rb_status derivative(rb_projection* p, const double* u, int64_t ldu, const double* us, double* F, cudaStream_t s) {
  const int m = p->m, m3 = p->m3;
  RB_TRY(spmm(p->I, u, ldu, p->Y, m3, m3, nullptr, s));
  for (int i = 0; i < 3; ++i)
    RB_TRY(rb_axty(p->nf, m, RB_F64, 1.0, us, m, p->Y + i * m, m3, reinterpret_cast<rb_stream_t>(s)));
  RB_TRY(spmm(p->M, p->Y, m3, p->tmp, m3, m3, p->c_conv, s));
  RB_TRY(spmm(p->L, u, ldu, F, m3, m3, p->c_diff, s));
  return axpy(p->n, m3, p->one_m3, p->tmp, m3, F, m3, s);
}

// In place: ut (n x 3 m, contiguous) becomes u_c; p->ut_s the face velocities, after the
// projection with time cdt whose pressure (initial guess in, solution out) is P[slot]
rb_status project(rb_projection* p, double* ut, double cdt, int slot, int* iters, double* ms, int* worst,
                  cudaStream_t s) {
  const int m = p->m, m3 = p->m3, n = p->n;
  k_fill3<<<1, 64, 0, s>>>(p->c_rhs, m, -1.0 / cdt, p->c_gm, m, -cdt, p->c_gm3, m3, -cdt);
  RB_CUDA(cudaGetLastError());
  RB_TRY(spmm(p->I, ut, m3, p->Y, m3, m3, nullptr, s));
  // u~_s: component d of Gamma u~ on the faces of direction d
  for (int d = 0; d < 3; ++d) RB_TRY(copy2d(p->ut_s + (size_t)d * n * m, m, p->Y + (size_t)d * n * m3 + d * m, m3, n, m, s));
  RB_TRY(spmm(p->M, p->ut_s, m, p->B, m, m, p->c_rhs, s));
  rb_cg_report rep{};
  const auto t0 = std::chrono::steady_clock::now();
  rb_status st;
  if (p->mg)
    st = rb_mg_solve(p->mg, &p->prm, p->B, m, p->P[slot], m, m, &rep, reinterpret_cast<rb_stream_t>(s));
  else
    st = rb_cg_solve(p->A, p->A32, &p->prm, p->B, m, p->P[slot], m, m, p->work, p->work_bytes, &rep,
                     reinterpret_cast<rb_stream_t>(s));
  *ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  int it = 0;
  for (int j = 0; j < m; ++j) it = std::max(it, rep.iters[j]);
  *iters = it;
  if (st != RB_OK && st != RB_ENOCONV && st != RB_EBREAKDOWN) return st;  // an argument or CUDA error
  if (st != RB_OK) *worst = std::max(*worst, (int)st);
  RB_TRY(spmm(p->G, p->P[slot], m, p->g, m, m, nullptr, s));
  RB_TRY(axpy(p->nf, m, p->c_gm, p->g, m, p->ut_s, m, s));
  // G_c p: component d = Gamma^T of G p on the faces of direction d (zero elsewhere)
  RB_CUDA(cudaMemsetAsync(p->Gm, 0, sizeof(double) * p->nf * m3, s));
  for (int d = 0; d < 3; ++d) RB_TRY(copy2d(p->Gm + (size_t)d * n * m3 + d * m, m3, p->g + (size_t)d * n * m, m, n, m, s));
  RB_TRY(spmm(p->IT, p->Gm, m3, p->tmp, m3, m3, nullptr, s));
  return axpy(n, m3, p->c_gm3, p->tmp, m3, ut, m3, s);
}

// ut = u + sum_j (dt a_j) F_j over the given combination slots (-1: none)
rb_status combine(rb_projection* p, const double* u, int64_t ldu, const int (&comb)[3], cudaStream_t s) {
  RB_TRY(copy2d(p->ut, p->m3, u, ldu, p->n, p->m3, s));
  for (int j = 0; j < 3; ++j)
    if (comb[j] >= 0) RB_TRY(axpy(p->n, p->m3, p->c_comb[comb[j]], p->F[j], p->m3, p->ut, p->m3, s));
  return RB_OK;
}

rb_status check_blocks(const rb_projection* p, const double* u_c, int64_t ldu, const double* u_s, int64_t lds,
                       const char* fn) {
  RB_REQUIRE(p, "%s: null handle", fn);
  RB_REQUIRE(u_c && u_s, "%s: null u_c or u_s", fn);
  RB_REQUIRE(ldu >= p->m3 && lds >= p->m, "%s: leading dimensions (%lld, %lld) below (3 m, m) = (%d, %d)", fn,
             (long long)ldu, (long long)lds, p->m3, p->m);
  RB_REQUIRE((uintptr_t)u_c % 8 == 0 && (uintptr_t)u_s % 8 == 0, "%s: u_c or u_s not 8-byte aligned", fn);
  // the bytes the blocks span: the last row ends after its 3 m (m) used columns
  const uintptr_t cb = (uintptr_t)u_c, ce = cb + (uintptr_t)(((int64_t)(p->n - 1) * ldu + p->m3) * 8);
  const uintptr_t sb = (uintptr_t)u_s, se = sb + (uintptr_t)(((int64_t)(p->nf - 1) * lds + p->m) * 8);
  RB_REQUIRE(ce <= sb || se <= cb, "%s: u_c and u_s overlap", fn);
  return RB_OK;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_projection_create(const rb_grid_desc* grid, const rb_projection_params* params,
                                          rb_stream_t stream, rb_projection_t* out) {
  clear_error();
  RB_REQUIRE(grid && params && out, "rb_projection_create: null argument");
  *out = nullptr;
  const int m = params->m;
  RB_REQUIRE(m >= 1 && 3 * m <= RB_MAX_K, "rb_projection_create: m = %d outside [1, %d]", m, RB_MAX_K / 3);
  RB_REQUIRE(std::isfinite(params->nu) && params->nu >= 0.0, "rb_projection_create: nu must be finite and >= 0");
  RB_REQUIRE(std::isfinite(params->dt) && params->dt > 0.0, "rb_projection_create: dt must be positive");
  RB_REQUIRE(params->solver == RB_PROJ_JACOBI || params->solver == RB_PROJ_MG, "rb_projection_create: unknown solver %d",
             params->solver);
  RB_REQUIRE(params->cg.project_mean == 1, "rb_projection_create: the periodic pressure needs project_mean = 1");
  RB_REQUIRE(params->cg.mixed >= 0 && params->cg.mixed <= 2, "rb_projection_create: mixed must be 0, 1 or 2");
  for (int d = 0; d < 3; ++d) RB_REQUIRE(grid->periodic[d] == 1, "rb_projection_create: every axis must be periodic");
  double h[3];
  int64_t n = 1;
  for (int d = 0; d < 3; ++d) {
    RB_REQUIRE(grid->n[d] >= 3 && grid->nodes[d], "rb_projection_create: axis %d needs >= 3 cells and its nodes", d);
    std::vector<double> x((size_t)grid->n[d] + 1);
    RB_CUDA(cudaMemcpy(x.data(), grid->nodes[d], x.size() * sizeof(double), cudaMemcpyDeviceToHost));
    double wmin = INFINITY, wmax = -INFINITY;
    for (int i = 0; i < grid->n[d]; ++i) {
      wmin = std::min(wmin, x[i + 1] - x[i]);
      wmax = std::max(wmax, x[i + 1] - x[i]);
    }
    RB_REQUIRE(wmin > 0.0 && wmax - wmin <= 1e-12 * wmax, "rb_projection_create: axis %d is not uniform", d);
    h[d] = x[1] - x[0];
    n *= grid->n[d];
  }
  RB_REQUIRE(3 * n <= INT32_MAX, "rb_projection_create: grid beyond int32 indexing");
  cudaStream_t s = S(stream);
  rb_projection* p = new rb_projection();
  p->n = (int)n;
  p->nf = (int)(3 * n);
  p->m = m;
  p->m3 = 3 * m;
  p->nu = params->nu;
  p->dt = params->dt;
  p->vol = h[0] * h[1] * h[2];
  p->solver = params->solver;
  p->prm = params->cg;
  const int m3 = p->m3;
  rb_status st = RB_OK;
  auto T = [&](rb_status r) {
    if (st == RB_OK) st = r;
    return st == RB_OK;
  };
  T(make_op(grid, RB_FVM_DIVERGENCE, 1.0, RB_F64, m3, s, &p->M)) &&
      T(make_op(grid, RB_FVM_GRADIENT, 1.0, RB_F64, m, s, &p->G)) &&
      T(make_op(grid, RB_FVM_LAPLACIAN, 1.0, RB_F64, m3, s, &p->L)) &&
      T(make_op(grid, RB_FVM_INTERP_C2S, 1.0, RB_F64, m3, s, &p->I)) &&
      T(make_op(grid, RB_FVM_INTERP_S2C, 1.0, RB_F64, m3, s, &p->IT));
  if (st == RB_OK && p->solver == RB_PROJ_MG) {
    rb_mg_info_t inf{};
    if (T(rb_mg_create(grid, m, nullptr, stream, &p->mg)) && T(rb_mg_info(p->mg, &inf)) && inf.levels < 2) {
      set_error("rb_projection_create: the grid does not coarsen, so the multigrid solver has one level");
      st = RB_EINVAL;
    }
  } else if (st == RB_OK) {
    T(make_op(grid, RB_FVM_LAPLACIAN, -1.0, RB_F64, m, s, &p->A));
    // the inner FP32 solve on the matrix-free Laplacian (no matrix streams in its iterations)
    if (st == RB_OK && p->prm.mixed) T(rb_fvm_stencil_create(grid, -1.0, RB_F32, m, stream, &p->A32));
    if (st == RB_OK) {
      p->work_bytes = rb_cg_workspace_bytes(p->A, m, &p->prm);
      if (p->work_bytes && cudaMalloc(&p->work, p->work_bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("rb_projection_create: CG workspace allocation failed");
        st = RB_ENOMEM;
      }
    }
  }
  const size_t nf = (size_t)p->nf, nc = (size_t)p->n;
  if (st == RB_OK)
    T(palloc(p, &p->Y, nf * m3)) && T(palloc(p, &p->Gm, nf * m3)) && T(palloc(p, &p->ut_s, nf * m)) &&
        T(palloc(p, &p->g, nf * m)) && T(palloc(p, &p->B, nc * m)) && T(palloc(p, &p->ut, nc * m3)) &&
        T(palloc(p, &p->tmp, nc * m3)) && T(palloc(p, &p->us_stage, nf * m)) && T(palloc(p, &p->P[0], nc * m)) &&
        T(palloc(p, &p->P[1], nc * m)) && T(palloc(p, &p->P[2], nc * m)) && T(palloc(p, &p->F[0], nc * m3)) &&
        T(palloc(p, &p->F[1], nc * m3)) && T(palloc(p, &p->F[2], nc * m3)) && T(palloc(p, &p->one_m, m)) &&
        T(palloc(p, &p->one_m3, m3)) && T(palloc(p, &p->c_diff, m3)) && T(palloc(p, &p->c_conv, m3)) &&
        T(palloc(p, &p->c_comb[0], m3)) && T(palloc(p, &p->c_comb[1], m3)) && T(palloc(p, &p->c_comb[2], m3)) &&
        T(palloc(p, &p->c_comb[3], m3)) && T(palloc(p, &p->c_rhs, m)) && T(palloc(p, &p->c_gm, m)) &&
        T(palloc(p, &p->c_gm3, m3));
  if (st == RB_OK) {
    for (int i = 0; i < 3; ++i)
      if (cudaMemsetAsync(p->P[i], 0, sizeof(double) * nc * m, s) != cudaSuccess) st = RB_ECUDA;
    k_fill3<<<1, 64, 0, s>>>(p->one_m, m, 1.0, p->one_m3, m3, 1.0, p->c_diff, m3, p->nu / p->vol);
    k_fill3<<<1, 64, 0, s>>>(p->c_conv, m3, -1.0 / p->vol, p->c_comb[0], m3, p->dt * kComb[0], p->c_comb[1], m3,
                             p->dt * kComb[1]);
    k_fill3<<<1, 64, 0, s>>>(p->c_comb[2], m3, p->dt * kComb[2], p->c_comb[3], m3, p->dt * kComb[3], nullptr, 0, 0.0);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("rb_projection_create: initialising the buffers failed");
      st = RB_ECUDA;
    }
  }
  if (st != RB_OK) {
    const std::string msg = rb_last_error();  // the destroy calls of the cleanup clear it
    release(p);
    set_error("%s", msg.c_str());
    return st;
  }
  *out = p;
  return RB_OK;
}

extern "C" rb_status rb_projection_destroy(rb_projection_t p) {
  clear_error();
  if (p) release(p);
  return RB_OK;
}

extern "C" rb_status rb_projection_step(rb_projection_t p, double* u_c, int64_t ldu, double* u_s, int64_t lds,
                                        rb_projection_report* report, rb_stream_t stream) {
  clear_error();
  RB_TRY(check_blocks(p, u_c, ldu, u_s, lds, "rb_projection_step"));
  cudaStream_t s = S(stream);
  rb_projection_report rep{};
  int worst = RB_OK;
  const int m = p->m, m3 = p->m3;
  // stage 1: F_0 at (u_c, u_s); the stage slots of HEUN's combinations (-1: coefficient 0)
  RB_TRY(copy2d(p->us_stage, m, u_s, lds, p->nf, m, s));
  RB_TRY(derivative(p, u_c, ldu, p->us_stage, p->F[0], s));
  const int comb2[3] = {0, -1, -1};  // u + dt/3 F_0
  const int comb3[3] = {-1, 1, -1};  // u + 2 dt/3 F_1
  const int combf[3] = {2, -1, 3};   // u + dt/4 F_0 + 3 dt/4 F_2
  for (int i = 1; i <= 2; ++i) {
    RB_TRY(combine(p, u_c, ldu, i == 1 ? comb2 : comb3, s));
    RB_TRY(project(p, p->ut, kHeunC[i] * p->dt, i - 1, &rep.iters[i - 1], &rep.poisson_ms, &worst, s));
    RB_TRY(copy2d(p->us_stage, m, p->ut_s, m, p->nf, m, s));
    RB_TRY(derivative(p, p->ut, m3, p->us_stage, p->F[i], s));
  }
  RB_TRY(combine(p, u_c, ldu, combf, s));
  RB_TRY(project(p, p->ut, p->dt, 2, &rep.iters[2], &rep.poisson_ms, &worst, s));
  RB_TRY(copy2d(u_c, ldu, p->ut, m3, p->n, m3, s));
  RB_TRY(copy2d(u_s, lds, p->ut_s, m, p->nf, m, s));
  rep.status = worst;
  if (report) *report = rep;
  return (rb_status)worst;
}

extern "C" rb_status rb_projection_project(rb_projection_t p, double cdt, double* u_c, int64_t ldu, double* u_s,
                                           int64_t lds, rb_projection_report* report, rb_stream_t stream) {
  clear_error();
  RB_TRY(check_blocks(p, u_c, ldu, u_s, lds, "rb_projection_project"));
  RB_REQUIRE(std::isfinite(cdt) && cdt > 0.0, "rb_projection_project: the projection time must be positive");
  cudaStream_t s = S(stream);
  rb_projection_report rep{};
  int worst = RB_OK;
  RB_TRY(copy2d(p->ut, p->m3, u_c, ldu, p->n, p->m3, s));
  RB_TRY(project(p, p->ut, cdt, 2, &rep.iters[0], &rep.poisson_ms, &worst, s));
  RB_TRY(copy2d(u_c, ldu, p->ut, p->m3, p->n, p->m3, s));
  RB_TRY(copy2d(u_s, lds, p->ut_s, p->m, p->nf, p->m, s));
  rep.status = worst;
  if (report) *report = rep;
  return (rb_status)worst;
}
