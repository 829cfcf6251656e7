// Arithmetic peak of the device, measured: the roofline denominator of the
// FP64-bound stepping kernels (and the FP32 rate, for the mixed forms).  Every
// thread runs kChains independent fused multiply-add chains, so the pipes see
// enough independent instructions to stay full; the grid is several CTAs per
// SM.  Timed with CUDA events on the caller's stream after one warm-up launch.
#include "mqs_internal.cuh"

namespace mqs {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) k_fma_chains(int iters, T x, T y, T* sink) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == (T)12345.678) sink[0] = s;   // keeps the chains live; never true for these inputs
}

template <typename T>
int measure(cudaStream_t st, int n_sm, int iters, double* tflops) {
  T* sink = nullptr;
  MQS_CUDA_TRY(cudaMalloc(&sink, sizeof(T)));
  cudaEvent_t e0, e1;
  MQS_CUDA_TRY(cudaEventCreate(&e0));
  MQS_CUDA_TRY(cudaEventCreate(&e1));
  const int blocks = n_sm * 8;
  // x slightly below 1 and y small keep every value finite
  k_fma_chains<T><<<blocks, kPeakThreads, 0, st>>>(iters / 8, (T)0.999999, (T)1e-7, sink);
  MQS_CUDA_TRY(cudaGetLastError());
  MQS_CUDA_TRY(cudaEventRecord(e0, st));
  k_fma_chains<T><<<blocks, kPeakThreads, 0, st>>>(iters, (T)0.999999, (T)1e-7, sink);
  MQS_CUDA_TRY(cudaGetLastError());
  MQS_CUDA_TRY(cudaEventRecord(e1, st));
  MQS_CUDA_TRY(cudaEventSynchronize(e1));
  float ms = 0.0f;
  MQS_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
  count_launch(2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flops = 2.0 * kChains * (double)iters * blocks * kPeakThreads;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return MQS_OK;
}

}  // namespace
}  // namespace mqs

using namespace mqs;

extern "C" int mqs_measure_peak(int32_t device, void* cuda_stream, int32_t precision,
                                double* tflops) {
  clear_error();
  if (!tflops || (precision != MQS_FP64 && precision != MQS_MIXED)) {
    set_error("bad arguments to mqs_measure_peak");
    return MQS_EINVAL;
  }
  int saved = 0;
  MQS_CUDA_TRY(cudaGetDevice(&saved));
  MQS_CUDA_TRY(cudaSetDevice(device));
  int n_sm = 0;
  MQS_CUDA_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device));
  const cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // about 50 ms of FP64 work at 1.25 TFLOP/s; the FP32 run is sized alike
  const int rc = precision == MQS_FP64 ? measure<double>(st, n_sm, 1 << 14, tflops)
                                       : measure<float>(st, n_sm, 1 << 18, tflops);
  cudaSetDevice(saved);
  return rc;
}
