// C ABI: error state, operator creation (validation, format conversion, Jacobi diagonal),
// destruction and introspection.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace rb {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

void clear_error() { g_err.clear(); }

int resident_blocks(const void* kernel, size_t smem, int threads) {
  static std::mutex mu;
  static std::map<std::pair<int, std::pair<const void*, size_t>>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(dev, std::make_pair(kernel, smem * 4096 + (size_t)threads));
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int v = std::min(kPersistentGrid, std::max(1, per_sm * sms));
  cache[key] = v;
  return v;
}

rb_status opt_in_smem(const void* kernel, size_t bytes) {
  if (bytes == 0) return RB_OK;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> opted;
  int dev = 0;
  RB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = opted[std::make_pair(dev, kernel)];
  if (bytes > cur) {
    // without the attribute, static and dynamic shared memory together stay within 48 KB
    cudaFuncAttributes fa{};
    RB_CUDA(cudaFuncGetAttributes(&fa, kernel));
    if (fa.sharedSizeBytes + bytes > 48 * 1024)
      RB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    cur = bytes;
  }
  return RB_OK;
}

rb_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  return e == cudaErrorMemoryAllocation ? RB_ENOMEM : RB_ECUDA;
}

namespace {

// Device allocation owned by an operator; every array gets 64 bytes of slack so that
// 16-byte vector loads of an aligned-down range may run past the last element.
template <typename T>
rb_status dalloc(rb_op* op, T** p, size_t count) {
  const size_t bytes = count * sizeof(T) + 64;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  e = cudaMemset(q, 0, bytes);
  if (e != cudaSuccess) {
    cudaFree(q);
    return cuda_fail(e, "cudaMemset", __FILE__, __LINE__);
  }
  *p = static_cast<T*>(q);
  op->device_bytes += (int64_t)bytes;
  return RB_OK;
}

void free_op(rb_op* op) {
  if (!op) return;
  void* ptrs[] = {op->row_ptr, op->col_idx, op->vals,    op->sell_ptr, op->sell_width, op->sell_row,
                  op->sell_col, op->sell_val, op->dinv64, op->dinv32,  op->zw64,       op->zw32, op->err,
                  op->st_w[0],  op->st_w[1],  op->st_w[2],  op->st_ic[0], op->st_ic[1],  op->st_ic[2]};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete op;
}

template <typename T>
rb_status fetch(std::vector<T>& dst, const T* src, size_t count, bool on_device) {
  dst.resize(count);
  if (count == 0) return RB_OK;
  if (on_device) {
    RB_CUDA(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst.data(), src, count * sizeof(T));
  }
  return RB_OK;
}

template <typename T>
rb_status upload(T* dst, const T* src, size_t count, cudaStream_t s) {
  if (count == 0) return RB_OK;
  RB_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  return RB_OK;
}

rb_status upload_values(rb_op* op, void** dst, const std::vector<double>& v, cudaStream_t s) {
  if (op->dtype == RB_F64) {
    double* p = nullptr;
    RB_TRY(dalloc(op, &p, v.size()));
    RB_TRY(upload(p, v.data(), v.size(), s));
    RB_CUDA(cudaStreamSynchronize(s));
    *dst = p;
  } else if (op->dtype == RB_DF64) {
    // pairs (hi, lo) = (RN32(v), RN32(v - hi)); v - hi is exact in FP64
    std::vector<float> f(2 * v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float hi = (float)v[i];
      f[2 * i] = hi;
      f[2 * i + 1] = (float)(v[i] - (double)hi);
    }
    float* p = nullptr;
    RB_TRY(dalloc(op, &p, f.size()));
    RB_TRY(upload(p, f.data(), f.size(), s));
    RB_CUDA(cudaStreamSynchronize(s));
    *dst = p;
  } else {
    std::vector<float> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];  // round to nearest even
    float* p = nullptr;
    RB_TRY(dalloc(op, &p, f.size()));
    RB_TRY(upload(p, f.data(), f.size(), s));
    RB_CUDA(cudaStreamSynchronize(s));
    *dst = p;
  }
  return RB_OK;
}

// Sliced ELL with C rows per slice: rows are sorted by decreasing length inside windows of
// sigma rows (stable), grouped C at a time; a slice is stored column-major (entry j of
// slot r at offset ptr + j * C + r), padded with (column 0, value 0).
rb_status build_sell(rb_op* op, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                     const std::vector<double>& va, cudaStream_t s) {
  const int C = 32, sigma = 256;
  const int n = op->n_rows;
  std::vector<int32_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  for (int w0 = 0; w0 < n; w0 += sigma) {
    const int w1 = std::min(n, w0 + sigma);
    std::stable_sort(order.begin() + w0, order.begin() + w1,
                     [&](int a, int b) { return (rp[a + 1] - rp[a]) > (rp[b + 1] - rp[b]); });
  }
  const int ns = (n + C - 1) / C;
  std::vector<int32_t> sptr(ns + 1, 0), swidth(ns, 0), srow((size_t)ns * C, -1);
  int64_t total = 0;
  for (int sl = 0; sl < ns; ++sl) {
    int w = 0;
    for (int r = 0; r < C; ++r) {
      const int idx = sl * C + r;
      if (idx < n) {
        srow[(size_t)sl * C + r] = order[idx];
        w = std::max(w, rp[order[idx] + 1] - rp[order[idx]]);
      }
    }
    swidth[sl] = w;
    sptr[sl] = (int32_t)total;
    total += (int64_t)w * C;
    if (total > INT32_MAX) {
      set_error("sliced ELL needs more than 2^31 entries");
      return RB_EUNSUPPORTED;
    }
  }
  sptr[ns] = (int32_t)total;
  std::vector<int32_t> scol((size_t)total, 0);
  std::vector<double> sval((size_t)total, 0.0);
  for (int sl = 0; sl < ns; ++sl) {
    for (int r = 0; r < C; ++r) {
      const int row = srow[(size_t)sl * C + r];
      if (row < 0) continue;
      int j = 0;
      for (int p = rp[row]; p < rp[row + 1]; ++p, ++j) {
        scol[(size_t)sptr[sl] + (size_t)j * C + r] = ci[p];
        sval[(size_t)sptr[sl] + (size_t)j * C + r] = va[p];
      }
    }
  }
  op->sell_c = C;
  op->sell_sigma = sigma;
  op->n_slices = ns;
  op->sell_nnz = total;
  RB_TRY(dalloc(op, &op->sell_ptr, sptr.size()));
  RB_TRY(dalloc(op, &op->sell_width, swidth.size()));
  RB_TRY(dalloc(op, &op->sell_row, srow.size()));
  RB_TRY(dalloc(op, &op->sell_col, scol.size()));
  RB_TRY(upload(op->sell_ptr, sptr.data(), sptr.size(), s));
  RB_TRY(upload(op->sell_width, swidth.data(), swidth.size(), s));
  RB_TRY(upload(op->sell_row, srow.data(), srow.size(), s));
  RB_TRY(upload(op->sell_col, scol.data(), scol.size(), s));
  RB_CUDA(cudaStreamSynchronize(s));
  return upload_values(op, &op->sell_val, sval, s);
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" const char* rb_last_error(void) { return g_err.c_str(); }
extern "C" const char* rb_version(void) { return "0.1.0"; }

extern "C" rb_status rb_operator_create(const rb_csr_desc* csr, const rb_block_desc* block, rb_dtype dtype,
                                        rb_format format, rb_stream_t stream, rb_op_t* out) {
  clear_error();
  RB_REQUIRE(csr && out, "rb_operator_create: null descriptor or output");
  *out = nullptr;
  RB_REQUIRE(dtype == RB_F64 || dtype == RB_F32 || dtype == RB_DF64, "rb_operator_create: unknown dtype %d",
             (int)dtype);
  RB_REQUIRE(dtype != RB_DF64 || format != RB_SELL, "rb_operator_create: RB_DF64 takes the CSR layout only");
  RB_REQUIRE(dtype != RB_DF64 || !block || block->extruded_nz == 0,
             "rb_operator_create: RB_DF64 operators cannot be extruded");
  RB_REQUIRE(format == RB_CSR || format == RB_SELL || format == RB_AUTO, "rb_operator_create: unknown format %d",
             (int)format);
  RB_REQUIRE(csr->n_rows >= 0 && csr->n_cols >= 0 && csr->nnz >= 0, "rb_operator_create: negative size");
  RB_REQUIRE(csr->nnz <= INT32_MAX, "rb_operator_create: nnz %lld exceeds int32 indexing", (long long)csr->nnz);
  RB_REQUIRE(csr->row_ptr != nullptr, "rb_operator_create: null row_ptr");
  RB_REQUIRE(csr->nnz == 0 || (csr->col_idx && csr->vals), "rb_operator_create: null col_idx or vals");
  const int k_max = block ? block->k_max : 1;
  RB_REQUIRE(k_max >= 1 && k_max <= RB_MAX_K, "rb_operator_create: k_max %d outside [1, %d]", k_max, RB_MAX_K);
  const int ext_nz = block ? block->extruded_nz : 0;
  RB_REQUIRE(ext_nz >= 0 && ext_nz <= RB_MAX_K, "rb_operator_create: extruded_nz %d outside [0, %d]", ext_nz,
             RB_MAX_K);
  if (ext_nz > 0) {
    RB_REQUIRE(block->z_weight != nullptr, "rb_operator_create: extruded operator without z_weight");
    RB_REQUIRE(csr->n_rows == csr->n_cols, "rb_operator_create: an extruded operator must be square");
    RB_REQUIRE(ext_nz >= 3, "rb_operator_create: extruded_nz must be >= 3 (distinct periodic neighbours)");
    RB_REQUIRE(std::isfinite(block->dz) && block->dz > 0, "rb_operator_create: dz must be positive");
  }
  cudaStream_t s = S(stream);
  const bool dev = csr->on_device != 0;
  std::vector<int32_t> rp, ci;
  std::vector<double> va;
  RB_TRY(fetch(rp, csr->row_ptr, (size_t)csr->n_rows + 1, dev));
  RB_TRY(fetch(ci, csr->col_idx, (size_t)csr->nnz, dev));
  RB_TRY(fetch(va, csr->vals, (size_t)csr->nnz, dev));
  // validation
  RB_REQUIRE(rp[0] == 0, "rb_operator_create: row_ptr[0] = %d, expected 0", rp[0]);
  RB_REQUIRE((int64_t)rp[csr->n_rows] == csr->nnz, "rb_operator_create: row_ptr[n_rows] = %d, nnz = %lld",
             rp[csr->n_rows], (long long)csr->nnz);
  int max_len = 0;
  for (int i = 0; i < csr->n_rows; ++i) {
    RB_REQUIRE(rp[i + 1] >= rp[i], "rb_operator_create: row_ptr decreases at row %d", i);
    max_len = std::max(max_len, rp[i + 1] - rp[i]);
  }
  for (int64_t p = 0; p < csr->nnz; ++p) {
    RB_REQUIRE(ci[p] >= 0 && ci[p] < csr->n_cols, "rb_operator_create: col_idx[%lld] = %d outside [0, %d)",
               (long long)p, ci[p], csr->n_cols);
    RB_REQUIRE(std::isfinite(va[p]), "rb_operator_create: vals[%lld] is not finite", (long long)p);
    RB_REQUIRE(dtype != RB_DF64 || std::fabs(va[p]) <= 3.4028234663852886e38,
               "rb_operator_create: vals[%lld] = %g outside the FP32 range of RB_DF64 pairs", (long long)p, va[p]);
  }
  // Extruded operator: the spanwise weights are checked, and dz and the -2 w_i of the periodic
  // second difference are folded into the library's copy of the values (dz a_ij off the
  // diagonal, dz a_ii - 2 w_i on it), so that the kernels add only w_i (x_{z-1} + x_{z+1}).
  std::vector<double> w;
  if (ext_nz > 0) {
    RB_TRY(fetch(w, block->z_weight, (size_t)csr->n_rows, dev));
    for (size_t i = 0; i < w.size(); ++i)
      RB_REQUIRE(std::isfinite(w[i]), "rb_operator_create: z_weight[%zu] is not finite", i);
    for (int i = 0; i < csr->n_rows; ++i) {
      int diag = -1;
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        va[p] *= block->dz;
        if (ci[p] == i) diag = p;
      }
      RB_REQUIRE(diag >= 0, "rb_operator_create: row %d of an extruded operator stores no diagonal entry", i);
      va[diag] -= 2.0 * w[i];
    }
  }
  rb_op* op = new rb_op();
  op->n_rows = csr->n_rows;
  op->n_cols = csr->n_cols;
  op->nnz = csr->nnz;
  op->dtype = dtype;
  op->format = (format == RB_SELL) ? RB_SELL : RB_CSR;
  op->k_max = k_max;
  op->max_row_len = max_len;
  op->avg_row_len = op->n_rows ? (double)op->nnz / op->n_rows : 0.0;
  rb_status st = RB_OK;
  do {
    if ((st = dalloc(op, &op->err, 1)) != RB_OK) break;
    if ((st = dalloc(op, &op->row_ptr, rp.size())) != RB_OK) break;
    if ((st = dalloc(op, &op->col_idx, ci.size())) != RB_OK) break;
    if ((st = upload(op->row_ptr, rp.data(), rp.size(), s)) != RB_OK) break;
    if ((st = upload(op->col_idx, ci.data(), ci.size(), s)) != RB_OK) break;
    if ((st = upload_values(op, &op->vals, va, s)) != RB_OK) break;
    // Jacobi diagonal (square operators): 1 / a_ii, zero where a row has no diagonal
    if (op->n_rows == op->n_cols && op->n_rows > 0) {
      std::vector<double> d64(op->n_rows, 0.0);
      std::vector<float> d32(op->n_rows, 0.0f);
      int with_diag = 0;
      for (int i = 0; i < op->n_rows; ++i) {
        for (int p = rp[i]; p < rp[i + 1]; ++p) {
          if (ci[p] == i && va[p] != 0.0) {
            d64[i] = 1.0 / va[p];
            d32[i] = (float)(1.0 / (double)(float)va[p]);
            ++with_diag;
            break;
          }
        }
      }
      op->has_diag = (with_diag == op->n_rows);
      if ((st = dalloc(op, &op->dinv64, d64.size())) != RB_OK) break;
      if ((st = dalloc(op, &op->dinv32, d32.size())) != RB_OK) break;
      if ((st = upload(op->dinv64, d64.data(), d64.size(), s)) != RB_OK) break;
      if ((st = upload(op->dinv32, d32.data(), d32.size(), s)) != RB_OK) break;
    }
    if (ext_nz > 0) {
      std::vector<float> w32(w.size());
      for (size_t i = 0; i < w.size(); ++i) w32[i] = (float)w[i];
      op->ext_nz = ext_nz;
      op->dz = block->dz;
      if ((st = dalloc(op, &op->zw64, w.size())) != RB_OK) break;
      if ((st = dalloc(op, &op->zw32, w32.size())) != RB_OK) break;
      if ((st = upload(op->zw64, w.data(), w.size(), s)) != RB_OK) break;
      if ((st = upload(op->zw32, w32.data(), w32.size(), s)) != RB_OK) break;
    }
    if (op->format == RB_SELL) {
      if ((st = build_sell(op, rp, ci, va, s)) != RB_OK) break;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "cudaStreamSynchronize", __FILE__, __LINE__);
      break;
    }
  } while (0);
  if (st != RB_OK) {
    free_op(op);
    return st;
  }
  *out = op;
  return RB_OK;
}

extern "C" rb_status rb_operator_destroy(rb_op_t op) {
  clear_error();
  if (!op) return RB_OK;
  free_op(op);
  return RB_OK;
}

extern "C" rb_status rb_operator_check(rb_op_t op, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(op != nullptr, "rb_operator_check: null operator");
  int h = 0;
  RB_CUDA(cudaMemcpyAsync(&h, op->err, sizeof(int), cudaMemcpyDeviceToHost, S(stream)));
  RB_CUDA(cudaStreamSynchronize(S(stream)));
  if (h != 0) {
    RB_CUDA(cudaMemsetAsync(op->err, 0, sizeof(int), S(stream)));
    RB_CUDA(cudaStreamSynchronize(S(stream)));
    set_error("a bounded wait in an SpMM kernel gave up (code %d); its output is invalid", h);
    return RB_ETIMEOUT;
  }
  return RB_OK;
}

extern "C" rb_status rb_operator_set_row_blocks(rb_op_t op, int32_t n_blocks, const int32_t* starts) {
  clear_error();
  RB_REQUIRE(op != nullptr, "rb_operator_set_row_blocks: null operator");
  RB_REQUIRE(n_blocks >= 1 && n_blocks <= 3, "rb_operator_set_row_blocks: n_blocks = %d outside [1, 3]", n_blocks);
  RB_REQUIRE(op->format == RB_CSR, "rb_operator_set_row_blocks: CSR operators only");
  RB_REQUIRE(n_blocks == 1 || starts != nullptr, "rb_operator_set_row_blocks: null starts");
  if (n_blocks > 1) {
    RB_REQUIRE(starts[0] == 0, "rb_operator_set_row_blocks: the first block must start at row 0");
    for (int b = 1; b < n_blocks; ++b)
      RB_REQUIRE(starts[b] > starts[b - 1] && starts[b] < op->n_rows,
                 "rb_operator_set_row_blocks: block starts must increase within [0, n_rows)");
  }
  op->n_rblk = n_blocks;
  for (int b = 0; b < n_blocks; ++b) op->rblk_off[b] = n_blocks > 1 ? starts[b] : 0;
  op->rblk_off[n_blocks] = op->n_rows;
  return RB_OK;
}

extern "C" rb_status rb_operator_info(rb_op_t op, rb_op_info* info) {
  clear_error();
  RB_REQUIRE(op && info, "rb_operator_info: null argument");
  info->n_rows = op->n_rows;
  info->n_cols = op->n_cols;
  info->nnz = op->nnz;
  info->dtype = op->dtype;
  info->format = op->format;
  info->sell_c = op->sell_c;
  info->sell_sigma = op->sell_sigma;
  info->sell_padded_nnz = op->sell_nnz;
  info->device_bytes = op->device_bytes;
  info->has_diag = op->has_diag;
  info->extruded_nz = op->ext_nz;
  return RB_OK;
}
