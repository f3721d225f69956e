// abft_fix.cu -- group verification and the delayed batched correction of the
// two-sided ABFT (TurboFFT Section III-A "Error Detection" and Section III-B
// "Delayed Batched Correction").
//
//  verify   : one warp per checksum group combines the chunk records in FP64,
//             compares |T1 - S1| with the threshold, names the faulty signal
//             b* from the quotient (T2 - S2)/(T1 - S1) = b* + 1, and queues the
//             group on the correction list (b* named with confidence) or on the
//             recompute list (not locatable, e.g. more than one fault).
//  gather   : for each queued group, c1 = sum_b x_b (the batch checksum X e_1)
//             and the partial output sum sum_{b != b*} y'_b.
//  (the pass kernels then transform c1 in place: W X e_1)
//  apply    : y_{b*} = W X e_1 - sum_{b != b*} y'_b, which equals
//             y'_{b*} - (Y' e_1 - W X e_1) but never subtracts the faulty value
//             from itself, so a huge or non-finite fault is removed exactly.
// Every kernel here is launched on every exec and returns at once when the
// lists are empty, so an exec never waits on the host.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "tfft_internal.h"

namespace tfft {

// Each group is reduced by `lanes_per_group` threads (one thread when a group
// holds few records -- FP64 adds are scarce on this part, so a 32-lane
// shuffle tree over a handful of records costs more than a serial sum --,
// one warp, or a whole block of 256 when a group holds many records); lane 0
// of the group decides.
// Blocks stride over the groups; the largest clean residual ratio is kept per
// thread and folded into the counter with one atomic per block.
__global__ void verify_kernel(const VerifyParams v, int lanes_per_group) {
  __shared__ double sred[8][11];
  __shared__ unsigned long long smax[8];
  const int lane = threadIdx.x % lanes_per_group;
  const int64_t per_block = blockDim.x / lanes_per_group;
  unsigned long long clean_max = 0;   // bits of the largest clean ratio (a nonnegative double)
  for (int64_t g0 = (int64_t)blockIdx.x * per_block; g0 < v.ngroups; g0 += (int64_t)gridDim.x * per_block) {
    const int64_t g = g0 + threadIdx.x / lanes_per_group;
    const bool active = g < v.ngroups;
    double s1r = 0, s1i = 0, s2r = 0, s2i = 0, en = 0, t1r = 0, t1i = 0, t2r = 0, t2i = 0;
    long long nfmin = 0x7fffffffffffffffLL, nfmax = -1;
    if (active) {
      for (int64_t k = lane; k < v.slots_in; k += lanes_per_group) {
        const RecIn r = v.rec_in[g * v.slots_in + k];
        s1r += r.s1r; s1i += r.s1i; s2r += r.s2r; s2i += r.s2i; en += r.energy;
      }
      for (int64_t k = lane; k < v.slots_out; k += lanes_per_group) {
        const RecOut r = v.rec_out[g * v.slots_out + k];
        t1r += r.t1r; t1i += r.t1i; t2r += r.t2r; t2i += r.t2i;
        nfmin = min(nfmin, r.nf_min); nfmax = max(nfmax, r.nf_max);
      }
    }
    for (int off = 16; off > 0 && lanes_per_group >= 32; off >>= 1) {
      s1r += __shfl_xor_sync(0xffffffffu, s1r, off); s1i += __shfl_xor_sync(0xffffffffu, s1i, off);
      s2r += __shfl_xor_sync(0xffffffffu, s2r, off); s2i += __shfl_xor_sync(0xffffffffu, s2i, off);
      en += __shfl_xor_sync(0xffffffffu, en, off);
      t1r += __shfl_xor_sync(0xffffffffu, t1r, off); t1i += __shfl_xor_sync(0xffffffffu, t1i, off);
      t2r += __shfl_xor_sync(0xffffffffu, t2r, off); t2i += __shfl_xor_sync(0xffffffffu, t2i, off);
      nfmin = min(nfmin, __shfl_xor_sync(0xffffffffu, nfmin, off));
      nfmax = max(nfmax, __shfl_xor_sync(0xffffffffu, nfmax, off));
    }
    if (lanes_per_group > 32) {          // combine the warps of the block
      const int w = threadIdx.x >> 5;
      if ((threadIdx.x & 31) == 0) {
        sred[w][0] = s1r; sred[w][1] = s1i; sred[w][2] = s2r; sred[w][3] = s2i; sred[w][4] = en;
        sred[w][5] = t1r; sred[w][6] = t1i; sred[w][7] = t2r; sred[w][8] = t2i;
        sred[w][9] = __longlong_as_double(nfmin); sred[w][10] = __longlong_as_double(nfmax);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int q = 1; q < lanes_per_group / 32; q++) {
          s1r += sred[q][0]; s1i += sred[q][1]; s2r += sred[q][2]; s2i += sred[q][3]; en += sred[q][4];
          t1r += sred[q][5]; t1i += sred[q][6]; t2r += sred[q][7]; t2i += sred[q][8];
          nfmin = min(nfmin, __double_as_longlong(sred[q][9]));
          nfmax = max(nfmax, __double_as_longlong(sred[q][10]));
        }
      }
      __syncthreads();
    }
    if (!active || lane != 0) continue;

    const int64_t gb = g * v.group;
    const int64_t gsize = min((int64_t)v.group, v.batch - gb);
    const double d1r = t1r - s1r, d1i = t1i - s1i;
    const double d2r = t2r - s2r, d2i = t2i - s2i;
    const double res = sqrt(d1r * d1r + d1i * d1i);
    const double tau = v.kappa_u_log2n_sqrtn * sqrt(en);
    const bool finite = isfinite(res) && isfinite(d2r) && isfinite(d2i);
    const bool nonfinite = !finite || nfmax >= 0;
    if (!(nonfinite || res > tau)) {
      // calibration record: the largest clean residual relative to the threshold
      const double ratio = tau > 0 ? res / tau : 0.0;
      clean_max = max(clean_max, (unsigned long long)__double_as_longlong(ratio));
      continue;
    }

    atomicAdd(&v.counters->detected, 1ull);
    // ---- locate ----
    int64_t bstar = -1;
    double qr = NAN, qi = NAN;
    if (nfmax >= 0) {
      if (nfmin == nfmax) bstar = nfmax - gb;          // the one signal whose sum overflowed
    } else if (finite && res > 0) {
      const double den = d1r * d1r + d1i * d1i;
      qr = (d2r * d1r + d2i * d1i) / den;
      qi = (d2i * d1r - d2r * d1i) / den;
      const double m = rint(qr);
      if (fabs(qr - m) < 0.25 && fabs(qi) < 0.25 && m >= 1.0 && m <= (double)gsize)
        bstar = (int64_t)m - 1;
    }
    // ---- decide ----
    int action = 3;
    if (!v.detect_only) {
      if (bstar >= 0) {
        const long long e = (long long)atomicAdd((unsigned long long*)&v.lists.fix[0], 1ull);
        if (e < v.lists.cap_fix) {
          v.lists.fix[1 + e] = g;
          v.lists.fix_signal[e] = gb + bstar;
          action = 1;
        }
      } else {
        const long long e = (long long)atomicAdd((unsigned long long*)&v.lists.rec[0], 1ull);
        if (e < v.lists.cap_rec) {
          v.lists.rec[1 + e] = g;
          action = 2;
        }
      }
    }
    if (action == 1) atomicAdd(&v.counters->corrected, 1ull);
    else if (action == 2) atomicAdd(&v.counters->recomputed, 1ull);
    else atomicAdd(&v.counters->uncorrectable, 1ull);
    const unsigned long long slot = atomicAdd(&v.counters->log_total, 1ull);
    LogEvent ev;
    ev.exec_index = v.exec_index;
    ev.group = g;
    ev.signal = bstar >= 0 ? gb + bstar : -1;
    ev.action = action;
    ev.nonfinite = nonfinite ? 1 : 0;
    ev.residual = res;
    ev.tau = tau;
    ev.q_re = qr;
    ev.q_im = qi;
    v.log[slot % kLogRing] = ev;
  }
  // one atomic per block for the calibration maximum
  for (int off = 16; off > 0; off >>= 1) clean_max = max(clean_max, __shfl_xor_sync(0xffffffffu, clean_max, off));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = clean_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, smax[w]);
    if (m) atomicMax(&v.counters->max_clean_ratio_bits, m);
  }
}

cudaError_t launch_verify(const VerifyParams& v, cudaStream_t s) {
  const int threads = 256;
  const int64_t recs = v.slots_in + v.slots_out;
  const int lanes = recs > 512 ? 256 : (recs > 64 ? 32 : 1);
  const int64_t need = (v.ngroups * lanes + threads - 1) / threads;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)v.max_blocks));
  verify_kernel<<<(unsigned)blocks, threads, 0, s>>>(v, lanes);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- gather
template <typename cT, typename acc_t>
__global__ void fix_gather_kernel(const FixParams f) {
  const long long count = min((long long)f.lists.fix[0], (long long)f.lists.cap_fix);
  const int64_t total = count * f.n;
  const cT* x = reinterpret_cast<const cT*>(f.in);
  const cT* y = reinterpret_cast<const cT*>(f.out);
  cT* c1 = reinterpret_cast<cT*>(f.ws_c1);
  cT* ac = reinterpret_cast<cT*>(f.ws_acc);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / f.n, k = idx % f.n;
    const int64_t g = f.lists.fix[1 + e];
    const int64_t bstar = f.lists.fix_signal[e];
    const int64_t gb = g * f.group, ge = min(f.batch, gb + (int64_t)f.group);
    acc_t sxr = 0, sxi = 0, syr = 0, syi = 0;
    for (int64_t b = gb; b < ge; b++) {
      const int64_t o = f.soff ? f.soff[b] : b * f.n;
      const cT xv = x[o + k];
      sxr += (acc_t)xv.x; sxi += (acc_t)xv.y;
      if (b != bstar) {
        const cT yv = y[o + k];
        syr += (acc_t)yv.x; syi += (acc_t)yv.y;
      }
    }
    c1[idx] = cT{(decltype(cT{}.x))sxr, (decltype(cT{}.x))sxi};
    ac[idx] = cT{(decltype(cT{}.x))syr, (decltype(cT{}.x))syi};
  }
}

template <typename cT>
__global__ void fix_apply_kernel(const FixParams f) {
  const long long count = min((long long)f.lists.fix[0], (long long)f.lists.cap_fix);
  const int64_t total = count * f.n;
  cT* y = reinterpret_cast<cT*>(f.out);
  const cT* fc1 = reinterpret_cast<const cT*>(f.ws_c1);
  const cT* ac = reinterpret_cast<const cT*>(f.ws_acc);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / f.n, k = idx % f.n;
    const int64_t bstar = f.lists.fix_signal[e];
    const cT a = fc1[idx], b = ac[idx];
    y[(f.soff ? f.soff[bstar] : bstar * f.n) + k] = cT{a.x - b.x, a.y - b.y};
  }
}

static int fix_grid(int64_t n, int cap) {
  int64_t blocks = ((int64_t)cap * n + 255) / 256;
  if (blocks > 1184) blocks = 1184;     // grid-stride beyond this
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

cudaError_t launch_fix_gather(const FixParams& f, cudaStream_t s) {
  const int grid = fix_grid(f.n, f.lists.cap_fix);
  if (f.dtype == 0) fix_gather_kernel<float2, double><<<grid, 256, 0, s>>>(f);
  else fix_gather_kernel<double2, double><<<grid, 256, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_fix_apply(const FixParams& f, cudaStream_t s) {
  const int grid = fix_grid(f.n, f.lists.cap_fix);
  if (f.dtype == 0) fix_apply_kernel<float2><<<grid, 256, 0, s>>>(f);
  else fix_apply_kernel<double2><<<grid, 256, 0, s>>>(f);
  return cudaGetLastError();
}

// ------------------------------------------------ random checksum vector
__global__ void gen_signs_kernel(double2* r, int64_t n, unsigned long long seed) {
  const double h = 0.86602540378443864676;   // sqrt(3)/2: w3 = -1/2 - i h
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double s = (splitmix64_at(seed, (unsigned long long)k) >> 63) ? -1.0 : 1.0;
    const int m = (int)(k % 3);
    const double re = m == 0 ? 1.0 : -0.5, im = m == 0 ? 0.0 : (m == 1 ? -h : h);
    r[k] = double2{s * re, s * im};
  }
}

__global__ void c128_to_c64_kernel(const double2* a, float2* b, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = float2{(float)a[k].x, (float)a[k].y};
}

cudaError_t launch_gen_signs(void* r, int64_t n, unsigned long long seed, cudaStream_t s) {
  gen_signs_kernel<<<fix_grid(n, 1), 256, 0, s>>>(reinterpret_cast<double2*>(r), n, seed);
  return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const void* src, void* dst, int64_t n, cudaStream_t s) {
  c128_to_c64_kernel<<<fix_grid(n, 1), 256, 0, s>>>(reinterpret_cast<const double2*>(src),
                                                    reinterpret_cast<float2*>(dst), n);
  return cudaGetLastError();
}

}  // namespace tfft
