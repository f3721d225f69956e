// v3_f32_single.cu -- instantiations of the v3 pass kernel: float values, role single.
#include "fft_v3.cuh"

namespace tfft {

cudaError_t v3_launch_f32_single(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  switch (nsub) {
    case 256: return launch_v3_kernel(fft_v3_kernel<float, 256, 16, 0>, grid, 256, smem, s, p);
    case 512: return launch_v3_kernel(fft_v3_kernel<float, 512, 16, 0>, grid, 256, smem, s, p);
    case 1024: return launch_v3_kernel(fft_v3_kernel<float, 1024, 16, 0>, grid, 256, smem, s, p);
    case 2048: return launch_v3_kernel(fft_v3_kernel<float, 2048, 16, 0>, grid, 256, smem, s, p);
    case 4096: return launch_v3_kernel(fft_v3_kernel<float, 4096, 16, 0>, grid, 256, smem, s, p);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t v3_attrs_f32_single(int nsub, size_t smem, int* bps) {
  const void* f = nullptr;
  switch (nsub) {
    case 256: f = (const void*)fft_v3_kernel<float, 256, 16, 0>; break;
    case 512: f = (const void*)fft_v3_kernel<float, 512, 16, 0>; break;
    case 1024: f = (const void*)fft_v3_kernel<float, 1024, 16, 0>; break;
    case 2048: f = (const void*)fft_v3_kernel<float, 2048, 16, 0>; break;
    case 4096: f = (const void*)fft_v3_kernel<float, 4096, 16, 0>; break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, f, 256, smem);
}

}  // namespace tfft
