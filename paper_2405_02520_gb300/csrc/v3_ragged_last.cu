// v3_ragged_last.cu -- the persistent ragged kernels of the last-pass
// families (32 to 1024 points).
#include "v3_ragged.cuh"

namespace tfft {

const void* ragged_last_fn(int nsub) {
  switch (nsub) {
    case 32: return (const void*)ragged_v3_kernel<V3_LAST, 32>;
    case 64: return (const void*)ragged_v3_kernel<V3_LAST, 64>;
    case 128: return (const void*)ragged_v3_kernel<V3_LAST, 128>;
    case 256: return (const void*)ragged_v3_kernel<V3_LAST, 256>;
    case 512: return (const void*)ragged_v3_kernel<V3_LAST, 512>;
    case 1024: return (const void*)ragged_v3_kernel<V3_LAST, 1024>;
    default: return nullptr;
  }
}

}  // namespace tfft
