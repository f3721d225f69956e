// v3_ragged_single.cu -- the persistent ragged kernels of the single-pass
// families (one pass of 256 to 4096 points).
#include "v3_ragged.cuh"

namespace tfft {

const void* ragged_single_fn(int nsub) {
  switch (nsub) {
    case 256: return (const void*)ragged_v3_kernel<V3_SINGLE, 256>;
    case 512: return (const void*)ragged_v3_kernel<V3_SINGLE, 512>;
    case 1024: return (const void*)ragged_v3_kernel<V3_SINGLE, 1024>;
    case 2048: return (const void*)ragged_v3_kernel<V3_SINGLE, 2048>;
    case 4096: return (const void*)ragged_v3_kernel<V3_SINGLE, 4096>;
    default: return nullptr;
  }
}

}  // namespace tfft
