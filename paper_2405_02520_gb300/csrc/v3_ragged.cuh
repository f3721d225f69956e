// v3_ragged.cuh -- the persistent tile kernel of one pass family for ragged
// batches.  A ragged batch sorts its signals into buckets of one length, each
// an ordinary batched plan.  A pass family is the passes of every bucket that
// run the same tile kernel (pass role and sub-transform length): one
// persistent launch runs them all.  Its blocks take work items -- a range of
// chunks of one bucket's pass -- from a list sorted by work, largest first,
// through an atomic counter (no block waits for another), and run each with
// that bucket's own pass parameters (in the launch's parameter block, as for
// the batched launches) through the same tile-kernel body.  (One kernel per family rather than per role: a kernel
// that switches among sub-transform lengths does not keep each length's body
// within the registers of two blocks per SM.)
#pragma once
#include "fft_v3.cuh"

namespace tfft {

template <int ROLE, int N>
__global__ void __launch_bounds__(256, 2) ragged_v3_kernel(const __grid_constant__ RaggedParams r) {
  __shared__ RaggedItem s_w;
  __shared__ int s_done;
  __shared__ V3Smem<8> vs;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(r.head, 1ull);
      s_done = it >= r.nitems;
      if (it < r.nitems) s_w = r.items[it];
    }
    __syncthreads();
    if (s_done) return;
    // the item holding chunk 0 of a bucket's first pass resets the bucket's
    // per-exec lists (the pass parameters carry them only for that pass)
    const bool gave_up = v3_body<float, N, 16, ROLE, 0, 256>(r.pp[s_w.bucket], s_w.c0, 1, s_w.c1, s_w.c0 == 0, vs);
    __syncthreads();                     // every thread has read s_w before the next item lands
    if (gave_up) return;                 // a copy may still be in flight into the buffers
  }
}

}  // namespace tfft
