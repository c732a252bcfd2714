// Arithmetic-throughput probe: the FP64 and FP32 fused multiply-add rate of
// the current GPU, measured rather than taken from a data sheet.  It gives
// the ALU roofline of the FP64 pencil solves and of the FP32 transforms a
// measured denominator (the FP64 rate of this part is a small fraction of
// its FP32 rate and is not among the copy-bandwidth and GEMM peaks that are
// measured elsewhere).  The paper has no counterpart; it is a measurement
// utility and changes no device setting.
#include <cstdio>

#include "internal.h"

namespace spectau {

constexpr int PEAK_CHAINS = 8;      // independent FMA chains per thread
constexpr int PEAK_THREADS = 256;

// Every thread runs PEAK_CHAINS independent chains x <- x a + b for `iters`
// rounds; a = 1 - 2^-20 and b small keep the values bounded and normal.  The
// store under a never-true condition keeps the compiler from removing them.
template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T* sink, int iters, T a, T b) {
  T x[PEAK_CHAINS];
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PEAK_CHAINS; ++k) s += x[k];
  if (s == (T)-1.2345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace spectau

using namespace spectau;

extern "C" sp_status sp_measure_fma_peak(int device, int precision, double* tflops) {
  if (!tflops || (precision != 0 && precision != 1)) return SP_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return SP_ERR_CUDA;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SP_ERR_CUDA;
  const int blocks = prop.multiProcessorCount * (prop.maxThreadsPerMultiProcessor / PEAK_THREADS);
  // ~10 ms per launch at the nominal rates (FP64 ~1.2 TFLOP/s, FP32 ~75)
  const int iters = precision == 0 ? 2048 : 131072;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return SP_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  void* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, (size_t)blocks * PEAK_THREADS * sizeof(double));
  float best = 1e30f;
  for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    if (precision == 0)
      k_fma_peak<double><<<blocks, PEAK_THREADS, 0, s>>>((double*)sink, iters, 1.0 - 0x1p-20, 0x1p-30);
    else
      k_fma_peak<float><<<blocks, PEAK_THREADS, 0, s>>>((float*)sink, iters, 1.0f - 0x1p-20f, 0x1p-30f);
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms < best) best = ms;   // the first launch warms up
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(sink);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return SP_ERR_CUDA;
  const double flops = 2.0 * PEAK_CHAINS * (double)iters * blocks * PEAK_THREADS;
  *tflops = flops / (best * 1e-3) / 1e12;
  return SP_OK;
}
