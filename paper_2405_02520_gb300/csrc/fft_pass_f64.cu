// fft_pass_f64.cu -- instantiations and launchers of the pass kernel for
// complex128 elements (double real and imaginary parts).
#include "fft_tile.cuh"

namespace tfft {

template <int E>
static cudaError_t launch_E(const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  fft_pass_kernel<double, E><<<grid, p.nthreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int E>
static cudaError_t attrs_E(size_t smem, int block, int* bps) {
  // a fixed cap well above any tile, so that plans with smaller tiles never
  // lower the limit another plan relies on
  (void)smem;
  cudaError_t e = cudaFuncSetAttribute(fft_pass_kernel<double, E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fft_pass_kernel<double, E>, block, smem);
}

cudaError_t launch_pass_f64(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s) {
  switch (E) {
    case 1: return launch_E<1>(p, grid, smem, s);
    case 2: return launch_E<2>(p, grid, smem, s);
    case 4: return launch_E<4>(p, grid, smem, s);
    case 8: return launch_E<8>(p, grid, smem, s);
    case 16: return launch_E<16>(p, grid, smem, s);     // 4096-point single pass
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t pass_func_attrs_f64(int E, size_t smem, int block, int* blocks_per_sm) {
  switch (E) {
    case 1: return attrs_E<1>(smem, block, blocks_per_sm);
    case 2: return attrs_E<2>(smem, block, blocks_per_sm);
    case 4: return attrs_E<4>(smem, block, blocks_per_sm);
    case 8: return attrs_E<8>(smem, block, blocks_per_sm);
    case 16: return attrs_E<16>(smem, block, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

template <int E>
static cudaError_t tile_launch_E(const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  fft_tile_kernel<double, E><<<grid, p.nthreads, smem, s>>>(p);
  return cudaGetLastError();
}

template <int E>
static cudaError_t tile_attrs_E(size_t smem, int block, int* bps) {
  cudaError_t e = cudaFuncSetAttribute(fft_tile_kernel<double, E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fft_tile_kernel<double, E>, block, smem);
}

cudaError_t launch_tile_f64(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s) {
  switch (E) {
    case 1: return tile_launch_E<1>(p, grid, smem, s);
    case 2: return tile_launch_E<2>(p, grid, smem, s);
    case 4: return tile_launch_E<4>(p, grid, smem, s);
    case 8: return tile_launch_E<8>(p, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t tile_func_attrs_f64(int E, size_t smem, int block, int* blocks_per_sm) {
  switch (E) {
    case 1: return tile_attrs_E<1>(smem, block, blocks_per_sm);
    case 2: return tile_attrs_E<2>(smem, block, blocks_per_sm);
    case 4: return tile_attrs_E<4>(smem, block, blocks_per_sm);
    case 8: return tile_attrs_E<8>(smem, block, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tfft
