// v3_ragged_cols.cu -- the persistent ragged kernels of the column-pass
// families (first and middle passes of 32 to 512 points).
#include "v3_ragged.cuh"

namespace tfft {

const void* ragged_cols_fn(int nsub) {
  switch (nsub) {
    case 32: return (const void*)ragged_v3_kernel<V3_COLS, 32>;
    case 64: return (const void*)ragged_v3_kernel<V3_COLS, 64>;
    case 128: return (const void*)ragged_v3_kernel<V3_COLS, 128>;
    case 256: return (const void*)ragged_v3_kernel<V3_COLS, 256>;
    case 512: return (const void*)ragged_v3_kernel<V3_COLS, 512>;
    default: return nullptr;
  }
}

}  // namespace tfft
