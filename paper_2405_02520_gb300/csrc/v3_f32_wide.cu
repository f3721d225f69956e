// v3_f32_wide.cu -- instantiations of the v3 pass kernel with 512 threads
// (tiles of 8192 complex64 values, one block per SM): the column and last
// passes of 512, 1024 and 2048 points, whose tiles then hold 16, 8 and 4
// lines (128-, 64- and 32-byte rows of the element-major boxes).
#include "fft_v3.cuh"

namespace tfft {

namespace {
template <int NSUB, int ROLE>
const void* wide_fn() { return (const void*)fft_v3_kernel<float, NSUB, 16, ROLE, 0, 512>; }
}  // namespace

cudaError_t launch_v3_wide(int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s) {
#define TFFT_WIDE(NS, R)                                                           \
  if (nsub == NS && role == R) {                                                   \
    fft_v3_kernel<float, NS, 16, R, 0, 512><<<grid, 512, smem, s>>>(p);           \
    return cudaGetLastError();                                                     \
  }
  TFFT_WIDE(512, 1) TFFT_WIDE(1024, 1) TFFT_WIDE(2048, 1)
  TFFT_WIDE(512, 2) TFFT_WIDE(1024, 2) TFFT_WIDE(2048, 2)
#undef TFFT_WIDE
  return cudaErrorInvalidValue;
}

cudaError_t v3_attrs_wide(int role, int nsub, size_t smem, int* bps) {
  const void* f = nullptr;
  if (role == 1) f = nsub == 512 ? wide_fn<512, 1>() : nsub == 1024 ? wide_fn<1024, 1>() : nsub == 2048 ? wide_fn<2048, 1>() : nullptr;
  if (role == 2) f = nsub == 512 ? wide_fn<512, 2>() : nsub == 1024 ? wide_fn<1024, 2>() : nsub == 2048 ? wide_fn<2048, 2>() : nullptr;
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, f, 512, smem);
}

// Bytes of the padded line scratch of a 512-thread kernel.
int v3_wide_scratch_bytes(int nsub) {
  const int c = 8192 / nsub, pitch = nsub + nsub / 16;
  return c * pitch * 8;
}

}  // namespace tfft
