// fusedfix.cuh -- the correction of a single-pass exec inside the pass
// kernel's last block (TurboFFT Section III-B, the one-pass case: the
// correction stays in the thread block instead of a separate launch).
//
// After the fused verification (sigverify.cuh) has queued the groups of this
// exec, the same block corrects them with no further launch:
//   located group g, faulty signal b*:
//     c1 = sum_{b in g} x_b                  (FP64 sums, rounded to the element type)
//     y_{b*} = W c1 - sum_{b in g, b != b*} y'_b
//   group that could not be located: y_b = W x_b for every b in g.
// W is one N-point transform (N <= 4096, a power of two) in shared memory:
// radix-2 decimation in time over the bit-reversed input, the stage roots
// read from the plan's table omega_N^m.  The outputs the other blocks wrote
// are read through the L2 (they counted themselves done after their stores
// completed).  Both kinds are counted once applied, as the separate
// correction kernels count them.
#pragma once

#include "fft_pass.cuh"
#include "tfft_internal.h"

namespace tfft {

// In-place forward transform of the n = 2^lg values in a[] (bit-reversed
// order in, natural order out), by the whole block.
template <typename cT>
__device__ void block_dit(cT* a, int n, int lg, const cT* tw, int tw_stride) {
  for (int s = 1; s <= lg; s++) {
    const int half = 1 << (s - 1), step = n >> s;       // omega_{2 half}^j = omega_n^(j step)
    for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
      const int pos = j & (half - 1);
      const int i0 = ((j >> (s - 1)) << s) + pos, i1 = i0 + half;
      const cT w = tw[(int64_t)pos * step * tw_stride];
      const cT u = a[i0], v = c_mul(a[i1], w);
      a[i0] = c_add(u, v);
      a[i1] = c_sub(u, v);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bit_reverse(int k, int lg) {
  return lg == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - lg));
}

template <typename real>
__device__ __noinline__ void fused_correct(const PassParams& p, const VerifyParams& v, unsigned char* work,
                                           size_t work_bytes) {
  using cT = typename Cplx<real>::T;
  const long long nfix = min(__ldcg(v.lists.fix), (long long)v.lists.cap_fix);
  const long long nrec = min(__ldcg(v.lists.rec), (long long)v.lists.cap_rec);
  if (nfix <= 0 && nrec <= 0) return;
  // a tile wait that gave up leaves loads that may still land in the
  // buffers this block would work in: the exec reports the timeout instead
  if (p.err_flag && *(volatile int*)p.err_flag) return;
  const int n = (int)p.n, lg = p.log2nsub;
  if ((size_t)n * sizeof(cT) > work_bytes) {         // the plan only fuses what fits
    if (threadIdx.x == 0 && p.err_flag) atomicExch(p.err_flag, 1);
    return;
  }
  cT* a = reinterpret_cast<cT*>(work);
  const cT* x = reinterpret_cast<const cT*>(p.in);
  cT* y = reinterpret_cast<cT*>(p.out);
  const cT* tw = reinterpret_cast<const cT*>(p.tw_sub);
  auto in_at = [&](int64_t b) { return p.soff_in ? (int64_t)p.soff_in[b] : b * (int64_t)n; };
  auto out_at = [&](int64_t b) { return p.soff_out ? (int64_t)p.soff_out[b] : b * (int64_t)n; };
  auto load = [&](cT c, int k) {
    if (p.conj_in) c.y = -c.y;
    a[bit_reverse(k, lg)] = c;
  };

  for (long long e = 0; e < nfix; e++) {
    const int64_t g = __ldcg(v.lists.fix + 1 + e), bstar = __ldcg(v.lists.fix_signal + e);
    const int64_t gb = g * v.group, ge = min(v.batch, gb + (int64_t)v.group);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double sr = 0, si = 0;
      for (int64_t b = gb; b < ge; b++) {
        const cT xv = x[in_at(b) + k];
        sr += (double)xv.x; si += (double)xv.y;
      }
      load(cT{(real)sr, (real)si}, k);
    }
    __syncthreads();
    block_dit(a, n, lg, tw, p.tw_sub_stride);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      double sr = 0, si = 0;
      for (int64_t b = gb; b < ge; b++) {
        if (b == bstar) continue;
        const cT yv = __ldcg(y + out_at(b) + k);
        sr += (double)yv.x; si += (double)yv.y;
      }
      const cT fc = out_xform(a[k], p);
      y[out_at(bstar) + k] = cT{fc.x - (real)sr, fc.y - (real)si};
    }
    __syncthreads();
  }
  for (long long e = 0; e < nrec; e++) {
    const int64_t g = __ldcg(v.lists.rec + 1 + e);
    const int64_t gb = g * v.group, ge = min(v.batch, gb + (int64_t)v.group);
    for (int64_t b = gb; b < ge; b++) {
      for (int k = threadIdx.x; k < n; k += blockDim.x) load(x[in_at(b) + k], k);
      __syncthreads();
      block_dit(a, n, lg, tw, p.tw_sub_stride);
      for (int k = threadIdx.x; k < n; k += blockDim.x) y[out_at(b) + k] = out_xform(a[k], p);
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && !(p.err_flag && *(volatile int*)p.err_flag)) {
    if (nfix > 0) atomicAdd(&v.counters->corrected, (unsigned long long)nfix);
    if (nrec > 0) atomicAdd(&v.counters->recomputed, (unsigned long long)nrec);
  }
}

}  // namespace tfft
