// v3_f32_last.cu -- instantiations of the v3 pass kernel: float values, role last.
#include "fft_v3.cuh"

namespace tfft {

cudaError_t v3_launch_f32_last(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (nsub) {
    case 32: fft_v3_kernel<float, 32, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    case 64: fft_v3_kernel<float, 64, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    case 128: fft_v3_kernel<float, 128, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    case 256: fft_v3_kernel<float, 256, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    case 512: fft_v3_kernel<float, 512, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    case 1024: fft_v3_kernel<float, 1024, 16, 2><<<grid, 256, smem, s>>>(p); return cudaGetLastError();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t v3_attrs_f32_last(int nsub, size_t smem, int* bps) {
  const void* f = nullptr;
  switch (nsub) {
    case 32: f = (const void*)fft_v3_kernel<float, 32, 16, 2>; break;
    case 64: f = (const void*)fft_v3_kernel<float, 64, 16, 2>; break;
    case 128: f = (const void*)fft_v3_kernel<float, 128, 16, 2>; break;
    case 256: f = (const void*)fft_v3_kernel<float, 256, 16, 2>; break;
    case 512: f = (const void*)fft_v3_kernel<float, 512, 16, 2>; break;
    case 1024: f = (const void*)fft_v3_kernel<float, 1024, 16, 2>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, f, 256, smem);
}

}  // namespace tfft
