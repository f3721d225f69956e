// v3_tc.cu -- instantiations of the v3 pass kernel with the tensor-core
// radix-16 DFT (complex64): TC = 3 three-term split TF32, TC = 2 three-term
// split BF16, TC = 1 plain TF32;
// single pass 256..4096 points, column and last passes of 256 points.
#include "fft_v3.cuh"

namespace tfft {

namespace {
template <int TC>
const void* tc_kernel(int role, int nsub) {
  if (role == 0) {
    switch (nsub) {
      case 256: return (const void*)fft_v3_kernel<float, 256, 16, 0, TC>;
      case 512: return (const void*)fft_v3_kernel<float, 512, 16, 0, TC>;
      case 1024: return (const void*)fft_v3_kernel<float, 1024, 16, 0, TC>;
      case 2048: return (const void*)fft_v3_kernel<float, 2048, 16, 0, TC>;
      case 4096: return (const void*)fft_v3_kernel<float, 4096, 16, 0, TC>;
      default: return nullptr;
    }
  }
  if (nsub != 256) return nullptr;
  return role == 1 ? (const void*)fft_v3_kernel<float, 256, 16, 1, TC>
                   : (const void*)fft_v3_kernel<float, 256, 16, 2, TC>;
}
}  // namespace

cudaError_t launch_v3_tc(int tc, int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  const void* f = tc == 3 ? tc_kernel<3>(role, nsub)
                : tc == 2 ? tc_kernel<2>(role, nsub) : (tc == 1 ? tc_kernel<1>(role, nsub) : nullptr);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<PassParams*>(&p)};
  return cudaLaunchKernel(f, dim3(grid), dim3(256), args, smem, s);
}

cudaError_t v3_attrs_tc(int tc, int role, int nsub, size_t smem, int* bps) {
  const void* f = tc == 3 ? tc_kernel<3>(role, nsub)
                : tc == 2 ? tc_kernel<2>(role, nsub) : (tc == 1 ? tc_kernel<1>(role, nsub) : nullptr);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
  if (e != cudaSuccess) return e;
  // all of the unified L1 / shared storage as shared memory, so that two
  // blocks of the scratch-aliased forms fit
  e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, f, 256, smem);
}

int v3_tc_bytes(int tc) { return v3_tc_smem_bytes(tc); }
bool v3_tc_two_blocks(int tc) { return v3_tc_aliased(tc); }

}  // namespace tfft
