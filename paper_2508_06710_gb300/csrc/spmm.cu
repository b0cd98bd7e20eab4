// SpMM over k interleaved right-hand sides (Sec. 2, Eq. (1), Algorithm 1), for CSR and
// sliced-ELL operators, plus the extruded-plane form (Sec. 2, repeated geometries):
//
//   Y[i, j] = c[j] * sum_p val[p] * X[idx[p], j]
//   extruded: Y[i, z] = c[z] * ( dz * sum_p val[p] X[idx[p], z] + w_i (X[i, z-1] - 2 X[i, z] + X[i, z+1]) )
//
// Each matrix coefficient and column index is read from HBM once and used for all k
// columns.  Threads are laid out as (row, chunk of VEC columns, lane within row): the KP
// chunks of a row sit in adjacent lanes, so the X rows they gather (k * sizeof(T) bytes)
// are read with coalesced 16-byte loads, and Y is written the same way.  The block's
// contiguous range of nonzeros (column indices and values) is staged in shared memory with
// coalesced loads before use, and broadcast from there to the KP chunk lanes of each row.
// With LPR > 1 several lanes split one row's nonzeros and are reduced with warp shuffles.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rb {

rb_status spmm_launch_f64(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                          int k, const double* cs, cudaStream_t s);
rb_status spmm_launch_f32(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                          int k, const double* cs, cudaStream_t s);
rb_status stencil_spmm_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                              int k, const double* cs, cudaStream_t s);
rb_status spmm_launch_df(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                         int k, const double* cs, cudaStream_t s);

namespace {

bool sched_valid(const rb_op* op, const SpmmSched& sc, int k, int64_t ldx, int64_t ldy, const void* X,
                 const void* Y) {
  const int eb = op->dtype == RB_F32 ? 4 : 8;
  if (sc.vec < 1 || sc.vec > 4 || !vec_ok(eb, sc.vec, k, ldx, ldy, X, Y)) return false;
  if (sc.kp != next_pow2(k / sc.vec) || sc.kp > 32) return false;
  if (sc.kp * sc.lpr > 32) return false;
  if ((op->format == RB_SELL || op->format == RB_STENCIL) && (sc.lpr != 1 || sc.stage)) return false;
  if (sc.stage == 2 && sc.lpr != 1) return false;
  if (op->dtype == RB_DF64 && sc.stage) return false;  // double-float: the direct kernel only
  if (op->ext_nz > 0 && sc.vec == 3) return false;  // the spanwise epilogue takes widths dividing Nz only
  if (op->ext_nz > 0 && (op->ext_nz % sc.vec)) return false;
  return true;
}

// Widths worth trying for k columns, best first: one thread per row for k <= 4 (3-wide
// scalar loads for k = 3), else the widest aligned vector.
std::vector<int> vec_candidates(int eb, int k) {
  std::vector<int> v;
  if (k == 3 || (k % 3 == 0 && k <= 96)) v.push_back(3);
  for (int w = 4; w >= 1; w >>= 1)
    if (k % w == 0 && !(eb == 8 && w == 4 && k > 4)) v.push_back(w);
  return v;
}

}  // namespace

SpmmSched default_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  const int eb = op->dtype == RB_F32 ? 4 : 8;
  SpmmSched sc;
  sc.lpr = 1;
  sc.stage = 0;
  sc.grid_cap = -1;
  // preference: 16-byte vectors with one thread per row, then 3-wide, then the widest aligned vector
  std::vector<int> order;
  if (k * eb == 16 || k * eb == 8) order.push_back(k);
  if (k % 3 == 0 && k <= 12) order.push_back(3);
  for (int w = 16 / eb; w >= 1; w >>= 1) order.push_back(w);
  if (eb == 8 && k == 4) order.insert(order.begin(), 2);
  for (int w : order) {
    SpmmSched t = sc;
    t.vec = w;
    if (k % w) continue;
    t.kp = next_pow2(k / w);
    if (sched_valid(op, t, k, ldx, ldy, X, Y)) {
      if (op->format != RB_SELL && op->avg_row_len >= 12.0) t.lpr = std::max(1, std::min(8, 32 / t.kp / 4));
      if (!sched_valid(op, t, k, ldx, ldy, X, Y)) t.lpr = 1;
      return t;
    }
  }
  sc.vec = 1;
  sc.kp = next_pow2(k);
  return sc;
}

rb_status spmm_launch(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy, int k,
                      const double* cs, cudaStream_t s) {
  if (op->format == RB_STENCIL) return stencil_spmm_launch(op, sc, X, ldx, Y, ldy, k, cs, s);
  if (op->dtype == RB_F64) return spmm_launch_f64(op, sc, X, ldx, Y, ldy, k, cs, s);
  if (op->dtype == RB_DF64) return spmm_launch_df(op, sc, X, ldx, Y, ldy, k, cs, s);
  return spmm_launch_f32(op, sc, X, ldx, Y, ldy, k, cs, s);
}

rb_status spmm_validate(const rb_op* op, const void* X, int64_t ldx, const void* Y, int64_t ldy, int k) {
  RB_REQUIRE(op != nullptr, "spmm: null operator");
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "spmm: k = %d outside [1, %d]", k, RB_MAX_K);
  RB_REQUIRE(ldx >= k && ldy >= k, "spmm: leading dimensions (%lld, %lld) smaller than k = %d", (long long)ldx,
             (long long)ldy, k);
  RB_REQUIRE((op->n_cols == 0 || X) && (op->n_rows == 0 || Y), "spmm: null X or Y");
  RB_REQUIRE(op->ext_nz == 0 || k == op->ext_nz, "spmm: extruded operator needs k == extruded_nz (%d), got %d",
             op->ext_nz, k);
  const int eb = op->dtype == RB_F32 ? 4 : 8;
  RB_REQUIRE((uintptr_t)X % eb == 0 && (uintptr_t)Y % eb == 0, "spmm: X or Y not aligned to the element size");
  const SpmmSched sc = default_sched(op, k, ldx, ldy, X, Y);
  if (!sched_valid(op, sc, k, ldx, ldy, X, Y)) {
    set_error("spmm: no schedule for k = %d with these leading dimensions and alignments (k > 32 needs "
              "8- or 16-byte aligned rows)", k);
    return RB_EUNSUPPORTED;
  }
  // X and Y must not overlap (the bytes each spans: its last row ends after k columns)
  const uintptr_t xb = (uintptr_t)X, xe = xb + (uintptr_t)(((int64_t)(op->n_cols - 1) * ldx + k) * eb);
  const uintptr_t yb = (uintptr_t)Y, ye = yb + (uintptr_t)(((int64_t)(op->n_rows - 1) * ldy + k) * eb);
  RB_REQUIRE(op->n_rows == 0 || op->n_cols == 0 || xe <= yb || ye <= xb, "spmm: X and Y overlap");
  return RB_OK;
}

SpmmSched pick_sched(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X, const void* Y) {
  auto it = op->tuned.find(k);
  if (it != op->tuned.end() && sched_valid(op, it->second, k, ldx, ldy, X, Y)) return it->second;
  return default_sched(op, k, ldx, ldy, X, Y);
}

std::vector<SpmmSched> tune_candidates(const rb_op* op, int k, int64_t ldx, int64_t ldy, const void* X,
                                       const void* Y) {
  std::vector<SpmmSched> cands;
  const int eb = op->dtype == RB_F32 ? 4 : 8;
  for (int vec : vec_candidates(eb, k)) {
    for (int lpr = 1; lpr <= 8; lpr <<= 1) {
      if (lpr > 1 && op->avg_row_len < 2.0 * lpr) continue;  // lanes would idle on short rows
      for (int stage = 0; stage <= 2; ++stage) {
        for (int gc : {-1, 0}) {
          if (stage && gc != 0) continue;
          SpmmSched sc;
          sc.vec = vec;
          sc.kp = next_pow2(k / vec);
          sc.lpr = lpr;
          sc.stage = stage;
          sc.grid_cap = gc;
          if (!sched_valid(op, sc, k, ldx, ldy, X, Y)) continue;
          if (op->format == RB_SELL && gc != -1) continue;
          cands.push_back(sc);
        }
      }
    }
  }
  return cands;
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_spmm(rb_op_t A, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t k, const double* c,
                             rb_stream_t stream) {
  clear_error();
  RB_TRY(spmm_validate(A, X, ldx, Y, ldy, k));
  if (A->n_rows == 0) return RB_OK;
  const SpmmSched sc = pick_sched(A, k, ldx, ldy, X, Y);
  return spmm_launch(A, sc, X, ldx, Y, ldy, k, c, S(stream));
}

extern "C" rb_status rb_tune_spmm(rb_op_t A, const void* X, int64_t ldx, void* Y, int64_t ldy, int32_t k,
                                  rb_stream_t stream) {
  clear_error();
  RB_TRY(spmm_validate(A, X, ldx, Y, ldy, k));
  if (A->n_rows == 0) return RB_OK;
  cudaStream_t s = S(stream);
  const std::vector<SpmmSched> cands = tune_candidates(A, k, ldx, ldy, X, Y);
  if (cands.empty()) {
    set_error("rb_tune_spmm: no valid schedule for k = %d", k);
    return RB_EUNSUPPORTED;
  }
  cudaEvent_t e0, e1;
  RB_CUDA(cudaEventCreate(&e0));
  RB_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  SpmmSched best_sc = cands[0];
  for (const SpmmSched& sc : cands) {
    rb_status st = RB_OK;
    for (int w = 0; w < 2 && st == RB_OK; ++w) st = spmm_launch(A, sc, X, ldx, Y, ldy, k, nullptr, s);
    if (st != RB_OK) continue;
    float times[5];
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0, s);
      spmm_launch(A, sc, X, ldx, Y, ldy, k, nullptr, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&times[r], e0, e1);
    }
    std::sort(times, times + 5);
    if (times[2] < best) {
      best = times[2];
      best_sc = sc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RB_CUDA(cudaGetLastError());
  A->tuned[k] = best_sc;
  return RB_OK;
}

extern "C" rb_status rb_set_spmm_schedule(rb_op_t A, int32_t k, const rb_spmm_schedule* sched) {
  clear_error();
  RB_REQUIRE(A && sched, "rb_set_spmm_schedule: null argument");
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "rb_set_spmm_schedule: k = %d outside [1, %d]", k, RB_MAX_K);
  SpmmSched sc;
  sc.vec = sched->vec;
  sc.lpr = sched->lpr;
  sc.stage = sched->stage;
  sc.grid_cap = sched->grid_cap;
  RB_REQUIRE(sc.vec >= 1 && sc.vec <= 4 && k % sc.vec == 0, "rb_set_spmm_schedule: vec %d does not divide k", sc.vec);
  sc.kp = next_pow2(k / sc.vec);
  RB_REQUIRE(sc.lpr == 1 || sc.lpr == 2 || sc.lpr == 4 || sc.lpr == 8, "rb_set_spmm_schedule: lpr must be 1, 2, 4 or 8");
  RB_REQUIRE(sc.stage >= 0 && sc.stage <= 2, "rb_set_spmm_schedule: stage must be 0, 1 or 2");
  RB_REQUIRE(sc.kp * sc.lpr <= 32, "rb_set_spmm_schedule: (k / vec) * lpr exceeds a warp");
  RB_REQUIRE(!(A->format == RB_SELL && (sc.lpr != 1 || sc.stage)), "rb_set_spmm_schedule: sliced ELL takes lpr 1, stage 0");
  RB_REQUIRE(!(A->format == RB_STENCIL && (sc.lpr != 1 || sc.stage)),
             "rb_set_spmm_schedule: a stencil operator takes lpr 1, stage 0");
  RB_REQUIRE(!(sc.stage == 2 && sc.lpr != 1), "rb_set_spmm_schedule: the TMA pipeline takes lpr 1");
  RB_REQUIRE(!(A->dtype == RB_DF64 && sc.stage), "rb_set_spmm_schedule: a double-float operator takes stage 0");
  RB_REQUIRE(!(A->ext_nz > 0 && (sc.vec == 3 || A->ext_nz % sc.vec)), "rb_set_spmm_schedule: vec must divide Nz");
  A->tuned[k] = sc;
  return RB_OK;
}

extern "C" rb_status rb_get_spmm_schedule(rb_op_t A, int32_t k, int64_t ldx, int64_t ldy, const void* X,
                                          const void* Y, rb_spmm_schedule* sched) {
  clear_error();
  RB_REQUIRE(A && sched, "rb_get_spmm_schedule: null argument");
  RB_REQUIRE(k >= 1 && k <= RB_MAX_K, "rb_get_spmm_schedule: k = %d outside [1, %d]", k, RB_MAX_K);
  const SpmmSched sc = pick_sched(A, k, ldx, ldy, X, Y);
  sched->vec = sc.vec;
  sched->lpr = sc.lpr;
  sched->stage = sc.stage;
  sched->grid_cap = sc.grid_cap;
  return RB_OK;
}
