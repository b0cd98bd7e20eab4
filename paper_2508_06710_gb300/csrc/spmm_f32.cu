// SpMM kernels (Sec. 2, Eq. (1), Algorithm 1) instantiated for float values and vectors.
#include "spmm_kernels.cuh"

namespace rb {

rb_status spmm_launch_f32(const rb_op* op, const SpmmSched& sc, const void* X, int64_t ldx, void* Y, int64_t ldy,
                         int k, const double* cs, cudaStream_t s) {
  return dispatch_vec<float>(op, sc, X, ldx, Y, ldy, k, cs, s);
}

}  // namespace rb
