// Measured FMA throughput of the GPU (FP64 and FP32): the arithmetic roof of the FP64 SpMM
// and CG kernels, which GB300's FP64 rate bounds before HBM does.  Every thread runs eight
// independent FMA chains on values the compiler cannot fold, a full-occupancy grid keeps every
// pipe busy, and CUDA events time the launch.  The multiplier and addend are per-thread
// register values: taken straight from the kernel's parameters (constant-bank operands), the
// FP64 FMAs of GB300 issue at about 0.81 of their rate with register operands.
#include "common.cuh"

namespace rb {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

// sinks that keep the chains live (written only if the chains' sum took a value it never takes
// for the inputs below), so that the measurement allocates nothing
__device__ double g_fma_sink64;
__device__ float g_fma_sink32;
__device__ __forceinline__ void fma_sink(double v) { g_fma_sink64 = v; }
__device__ __forceinline__ void fma_sink(float v) { g_fma_sink32 = v; }

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(int iters, T a0, T b0) {
  const T a = a0 + (T)threadIdx.x * (T)1e-15, b = b0 + (T)threadIdx.x * (T)1e-17;  // in registers
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = a + (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  if (s == T(12345)) fma_sink(s);  // the chains tend to b / (1 - a) = 0.1 each: never taken
}

template <typename T>
rb_status measure(double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  RB_CUDA(cudaGetDevice(&dev));
  RB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kPeakThreads, 0));
  const int grid = std::max(1, per_sm) * sms;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  cudaEvent_t e0, e1;
  RB_CUDA(cudaEventCreate(&e0));
  RB_CUDA(cudaEventCreate(&e1));
  const T a = (T)0.999999, b = (T)1e-7;
  k_fma_peak<T><<<grid, kPeakThreads, 0, s>>>(iters / 16, a, b);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<grid, kPeakThreads, 0, s>>>(iters, a, b);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::min(best, ms);
  }
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RB_CUDA(err);
  RB_CUDA(cudaStreamSynchronize(s));
  const double flops = 2.0 * kChains * (double)iters * grid * kPeakThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return RB_OK;
}

}  // namespace
}  // namespace rb

using namespace rb;

extern "C" rb_status rb_fma_peak(rb_dtype dtype, double* tflops, rb_stream_t stream) {
  clear_error();
  RB_REQUIRE(tflops != nullptr, "rb_fma_peak: null output");
  RB_REQUIRE(dtype == RB_F64 || dtype == RB_F32, "rb_fma_peak: unknown dtype %d", (int)dtype);
  cudaStream_t s = S(stream);
  return dtype == RB_F64 ? measure<double>(tflops, s) : measure<float>(tflops, s);
}
