// v3_ragged.cu -- host side of the persistent ragged kernels: the families
// they cover, their launch attributes and launches.
#include "tfft_internal.h"

namespace tfft {

const void* ragged_single_fn(int nsub);
const void* ragged_cols_fn(int nsub);
const void* ragged_last_fn(int nsub);

namespace {
const void* ragged_fn(int role, int nsub) {
  return role == 0 ? ragged_single_fn(nsub) : role == 1 ? ragged_cols_fn(nsub) : role == 2 ? ragged_last_fn(nsub)
                                                                                          : nullptr;
}
}  // namespace

bool v3_ragged_has(int role, int nsub) { return ragged_fn(role, nsub) != nullptr; }

cudaError_t v3_ragged_attrs(int role, int nsub, size_t smem, int* bps) {
  const void* f = ragged_fn(role, nsub);
  if (!f) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, f, 256, smem);
}

cudaError_t launch_v3_ragged(int role, int nsub, const RaggedParams& r, int grid, size_t smem, cudaStream_t s) {
  const void* f = ragged_fn(role, nsub);
  if (!f) return cudaErrorInvalidValue;
  void* args[1] = {const_cast<RaggedParams*>(&r)};
  return cudaLaunchKernel(f, dim3((unsigned)grid), dim3(256), args, smem, s);
}

}  // namespace tfft
