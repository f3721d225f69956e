// peak.cu -- arithmetic peaks of the GPU the library runs on, measured with
// an FMA loop (no counterpart in the paper; used to state the roofline of the
// transforms that the FP64 units bound, complex128 on this part).
//
// Every thread runs kChains independent multiply-add chains for `iters`
// iterations: x <- x * a + b with |a| < 1, so nothing overflows and no chain
// waits on another.  Flops counted: 2 per FMA.  The result is written out so
// the loop is not removed.
#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tfft_internal.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void fma_loop_kernel(T* out, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int measure(double* tflops, int iters) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
  const int threads = 256, blocks = sms * 8;
  T* out = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(T) * (size_t)blocks * threads);
  if (e != cudaSuccess) return tfft::record_cuda_error(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T a = (T)0.999999, b = (T)1e-7;
  fma_loop_kernel<T><<<blocks, threads>>>(out, iters / 8, a, b);     // warm-up
  cudaEventRecord(e0);
  fma_loop_kernel<T><<<blocks, threads>>>(out, iters, a, b);
  cudaEventRecord(e1);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return tfft::record_cuda_error(e);
  const double flops = 2.0 * kChains * (double)iters * (double)blocks * threads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return TFFT_SUCCESS;
}

}  // namespace

extern "C" int tfft_measure_fma_peak(int fp64, int iters, double* tflops) {
  if (!tflops || iters < 8 || (fp64 != 0 && fp64 != 1)) return TFFT_ERR_INVALID_ARG;
  return fp64 ? measure<double>(tflops, iters) : measure<float>(tflops, iters);
}
