// Measured arithmetic peaks of the GPU the library runs on: FP64 and FP32 fused
// multiply-add throughput, timed with CUDA events.  The step's truncation solves
// run on the FP64 pipe (or on the FP32 pipe in double-float), so these are the
// denominators of their roofline fractions.
//
// Each thread runs eight independent FMA chains (enough to cover the pipe latency
// at eight CTAs of 256 threads per SM); the result is kept live through a store
// that the compiler cannot prove dead.  flops = 2 x chains x iterations x threads.

#include <algorithm>

#include "qlb_internal.cuh"

#define QLB_API extern "C" __attribute__((visibility("default")))

namespace qlb {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* out, int iters, T seed) {
  const T m = (T)0.9999999, c = (T)1e-7;
  T a0 = seed + (T)threadIdx.x, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int i = 0; i < iters; i++) {
    a0 = fma(a0, m, c);
    a1 = fma(a1, m, c);
    a2 = fma(a2, m, c);
    a3 = fma(a3, m, c);
    a4 = fma(a4, m, c);
    a5 = fma(a5, m, c);
    a6 = fma(a6, m, c);
    a7 = fma(a7, m, c);
  }
  T r = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (r == (T)-12345.0) out[blockIdx.x] = r;
}

template <typename T>
qlb_status time_peak(int iters, int blocks, T* out, cudaEvent_t a, cudaEvent_t b, double* ms) {
  QLB_CUDA_TRY(cudaEventRecord(a, 0));
  k_fma_peak<T><<<blocks, 256>>>(out, iters, (T)1.0);
  QLB_CUDA_TRY(cudaGetLastError());
  QLB_CUDA_TRY(cudaEventRecord(b, 0));
  QLB_CUDA_TRY(cudaEventSynchronize(b));
  float f = 0;
  QLB_CUDA_TRY(cudaEventElapsedTime(&f, a, b));
  *ms = f;
  return QLB_OK;
}

template <typename T>
qlb_status measure(double* tflops) {
  int dev = 0, sms = 0;
  QLB_CUDA_TRY(cudaGetDevice(&dev));
  QLB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;
  T* out = nullptr;
  QLB_CUDA_TRY(cudaMalloc(&out, sizeof(T) * blocks));
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  qlb_status s = QLB_OK;
  double ms = 0, best = 0;
  int iters = 256;
  // grow the loop until one launch lasts about 20 ms, then keep the best of three
  for (int g = 0; g < 16 && !s; g++) {
    s = time_peak<T>(iters, blocks, out, a, b, &ms);
    if (s || ms > 20.0) break;
    iters = (int)std::min<double>(2.0e9, iters * std::max(2.0, 25.0 / std::max(ms, 0.01)));
  }
  for (int r = 0; r < 3 && !s; r++) {
    s = time_peak<T>(iters, blocks, out, a, b, &ms);
    double fl = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0;
    best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (!s) *tflops = best;
  return s;
}

}  // namespace
}  // namespace qlb

using namespace qlb;

QLB_API qlb_status qlb_measure_peak(int device, int kind, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) {
    set_error("qlb_measure_peak: kind must be 0 (FP64) or 1 (FP32) and tflops non-null");
    return QLB_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    set_error("qlb_measure_peak: no such CUDA device");
    return QLB_EDEVICE;
  }
  int prev = -1;
  QLB_CUDA_TRY(cudaGetDevice(&prev));
  QLB_CUDA_TRY(cudaSetDevice(device));
  qlb_status s = kind == 0 ? measure<double>(tflops) : measure<float>(tflops);
  cudaSetDevice(prev);
  return s;
}
