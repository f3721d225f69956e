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

#include "sigverify.cuh"
#include "tfft_internal.h"

namespace tfft {

// Each group is reduced by `lanes_per_group` threads (one thread when a group
// holds few records -- FP64 adds are scarce on this part, so a 32-lane
// shuffle tree over a handful of records costs more than a serial sum --,
// one warp, or a whole block of 256 when a group holds many records); lane 0
// of the group decides.
// Blocks stride over the groups; the largest clean residual ratio is kept per
// thread and folded into the counter with one atomic per block.
// The decision for group g from its combined sums (lane 0 of the group):
// detection against the threshold, location by the quotient, the work lists,
// the counters and the fault log.  Clean groups update the calibration
// maximum `clean_max` (the bits of a nonnegative double).
struct GroupSums {
  double s1r, s1i, s2r, s2i, en, t1r, t1i, t2r, t2i;
  long long nfmin, nfmax;
};

__device__ void decide_group(const VerifyParams& v, int64_t g, const GroupSums& c,
                             unsigned long long& clean_max) {
  const int64_t gb = g * v.group;
  const int64_t gsize = min((int64_t)v.group, v.batch - gb);
  const double d1r = c.t1r - c.s1r, d1i = c.t1i - c.s1i;
  const double d2r = c.t2r - c.s2r, d2i = c.t2i - c.s2i;
  const double res = sqrt(d1r * d1r + d1i * d1i);
  const double tau = v.kappa_u_log2n_sqrtn * sqrt(c.en);
  const bool finite = isfinite(res) && isfinite(d2r) && isfinite(d2i);
  const bool nonfinite = !finite || c.nfmax >= 0;
  if (!(nonfinite || res > tau)) {
    // calibration record: the largest clean residual relative to the threshold
    const double ratio = tau > 0 ? res / tau : 0.0;
    clean_max = max(clean_max, (unsigned long long)__double_as_longlong(ratio));
    return;
  }

  atomicAdd(&v.counters->detected, 1ull);
  // ---- locate ----
  int64_t bstar = -1;
  double qr = NAN, qi = NAN;
  if (c.nfmax >= 0) {
    if (c.nfmin == c.nfmax) bstar = c.nfmax - gb;          // the one signal whose sum overflowed
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
  if ((action == 1 || action == 2) && v.cond_flag &&
      atomicExch(reinterpret_cast<unsigned long long*>(v.cond_flag), 1ull) == 0ull)
    cudaGraphSetConditional(v.cond, 1u);      // run the correction body of this exec's graph
  // corrected and recomputed groups are counted by fix_apply, after the
  // correction has run; a group left as it is is counted here
  if (action == 3) atomicAdd(&v.counters->uncorrectable, 1ull);
  const unsigned long long slot = atomicAdd(&v.counters->log_total, 1ull);
  LogEvent ev;
  ev.exec_index = v.exec_index;
  ev.group = v.group_base + g;
  ev.signal = bstar >= 0 ? v.group_base * v.group + gb + bstar : -1;
  ev.action = action;
  ev.nonfinite = nonfinite ? 1 : 0;
  ev.residual = res;
  ev.tau = tau;
  ev.q_re = qr;
  ev.q_im = qi;
  v.log[slot % kLogRing] = ev;
}

// Each group is reduced by `lanes_per_group` threads (one thread when a group
// holds few records -- FP64 adds are scarce on this part, so a 32-lane
// shuffle tree over a handful of records costs more than a serial sum --,
// one warp, or a whole block of 256 when a group holds many records); lane 0
// of the group decides.  With v.split > 1 several blocks share a group
// (lanes_per_group = 256) and the last of them decides.
// Blocks stride over the groups; the largest clean residual ratio is kept per
// thread and folded into the counter with one atomic per block.
__global__ void verify_kernel(const VerifyParams v, int lanes_per_group) {
  __shared__ double sred[8][11];
  __shared__ unsigned long long smax[8];
  __shared__ int s_last;
  const int lane = threadIdx.x % lanes_per_group;
  const int64_t per_block = v.split > 1 ? 1 : blockDim.x / lanes_per_group;
  const int64_t nunits = v.ngroups * v.split;           // (group, slice) units
  unsigned long long clean_max = 0;   // bits of the largest clean ratio (a nonnegative double)
  for (int64_t u0 = (int64_t)blockIdx.x * per_block; u0 < nunits; u0 += (int64_t)gridDim.x * per_block) {
    const int64_t unit = u0 + (v.split > 1 ? 0 : threadIdx.x / lanes_per_group);
    const int64_t g = unit / v.split;
    const int64_t slice = unit - g * v.split;
    const bool active = unit < nunits;
    GroupSums c{0, 0, 0, 0, 0, 0, 0, 0, 0, 0x7fffffffffffffffLL, -1};
    if (active) {
      // this slice's records: [k0, k1) of the inputs and of the outputs
      const int64_t ki0 = v.slots_in * slice / v.split, ki1 = v.slots_in * (slice + 1) / v.split;
      const int64_t ko0 = v.slots_out * slice / v.split, ko1 = v.slots_out * (slice + 1) / v.split;
      for (int64_t k = ki0 + lane; k < ki1; k += lanes_per_group) {
        const RecIn r = v.rec_in[g * v.slots_in + k];
        c.s1r += r.s1r; c.s1i += r.s1i; c.s2r += r.s2r; c.s2i += r.s2i; c.en += r.energy;
      }
      for (int64_t k = ko0 + lane; k < ko1; k += lanes_per_group) {
        const RecOut r = v.rec_out[g * v.slots_out + k];
        c.t1r += r.t1r; c.t1i += r.t1i; c.t2r += r.t2r; c.t2i += r.t2i;
        c.nfmin = min(c.nfmin, r.nf_min); c.nfmax = max(c.nfmax, r.nf_max);
      }
    }
    for (int off = 16; off > 0 && lanes_per_group >= 32; off >>= 1) {
      c.s1r += __shfl_xor_sync(0xffffffffu, c.s1r, off); c.s1i += __shfl_xor_sync(0xffffffffu, c.s1i, off);
      c.s2r += __shfl_xor_sync(0xffffffffu, c.s2r, off); c.s2i += __shfl_xor_sync(0xffffffffu, c.s2i, off);
      c.en += __shfl_xor_sync(0xffffffffu, c.en, off);
      c.t1r += __shfl_xor_sync(0xffffffffu, c.t1r, off); c.t1i += __shfl_xor_sync(0xffffffffu, c.t1i, off);
      c.t2r += __shfl_xor_sync(0xffffffffu, c.t2r, off); c.t2i += __shfl_xor_sync(0xffffffffu, c.t2i, off);
      c.nfmin = min(c.nfmin, __shfl_xor_sync(0xffffffffu, c.nfmin, off));
      c.nfmax = max(c.nfmax, __shfl_xor_sync(0xffffffffu, c.nfmax, off));
    }
    if (lanes_per_group > 32) {          // combine the warps of the block
      const int w = threadIdx.x >> 5;
      if ((threadIdx.x & 31) == 0) {
        sred[w][0] = c.s1r; sred[w][1] = c.s1i; sred[w][2] = c.s2r; sred[w][3] = c.s2i; sred[w][4] = c.en;
        sred[w][5] = c.t1r; sred[w][6] = c.t1i; sred[w][7] = c.t2r; sred[w][8] = c.t2i;
        sred[w][9] = __longlong_as_double(c.nfmin); sred[w][10] = __longlong_as_double(c.nfmax);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int q = 1; q < lanes_per_group / 32; q++) {
          c.s1r += sred[q][0]; c.s1i += sred[q][1]; c.s2r += sred[q][2]; c.s2i += sred[q][3];
          c.en += sred[q][4];
          c.t1r += sred[q][5]; c.t1i += sred[q][6]; c.t2r += sred[q][7]; c.t2i += sred[q][8];
          c.nfmin = min(c.nfmin, __double_as_longlong(sred[q][9]));
          c.nfmax = max(c.nfmax, __double_as_longlong(sred[q][10]));
        }
      }
      __syncthreads();
    }
    if (v.split > 1) {
      // add this slice into the group's accumulators; the last slice decides
      if (threadIdx.x == 0) {
        double* a = v.part_acc + g * kVerifyAcc;
        const double add[9] = {c.s1r, c.s1i, c.s2r, c.s2i, c.en, c.t1r, c.t1i, c.t2r, c.t2i};
        for (int q = 0; q < 9; q++) atomicAdd(a + q, add[q]);
        long long* nf = reinterpret_cast<long long*>(a + 9);
        atomicMin(nf, c.nfmin);
        atomicMax(nf + 1, c.nfmax);
        __threadfence();
        s_last = atomicAdd(v.part_cnt + g, 1u) == (unsigned)(v.split - 1);
        if (s_last) {
          __threadfence();
          c.s1r = __ldcg(a + 0); c.s1i = __ldcg(a + 1); c.s2r = __ldcg(a + 2); c.s2i = __ldcg(a + 3);
          c.en = __ldcg(a + 4);
          c.t1r = __ldcg(a + 5); c.t1i = __ldcg(a + 6); c.t2r = __ldcg(a + 7); c.t2i = __ldcg(a + 8);
          c.nfmin = __ldcg(nf); c.nfmax = __ldcg(nf + 1);
          for (int q = 0; q < 9; q++) a[q] = 0.0;
          nf[0] = 0x7fffffffffffffffLL;
          nf[1] = -1;
          v.part_cnt[g] = 0u;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0 && s_last) decide_group(v, g, c, clean_max);
      __syncthreads();
      continue;
    }
    if (!active || lane != 0) continue;
    decide_group(v, g, c, clean_max);
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

// ------------------------------------------------ per-signal verification
// Per-signal records (written by the tile kernels): every signal is tested on
// its own -- d_b = r^T y'_b - w^T x_b against tau_b = kappa u (log2 N + 4)
// sqrt(N) ||x_b|| -- and the group's two-sided checksums of Section III are
// formed from the same sums: D1 = sum_b d_b = T1 - S1 (right-side vector
// e_1) and D2 = sum_b (b+1) d_b = T2 - S2 (e_3), tested against the group
// threshold.  Multi-pass plans add a second per-signal test across their
// last pass (second left vector r2, threshold with log2 n_last).  A group is
// flagged when a signal or the group sum exceeds its threshold (or is not
// finite).  Location: the one flagged signal; with none flagged (a group-level
// detection) the quotient D2 / D1 = b* + 1; with several flagged the group is
// recomputed (outside the single-event model).  The quotient is logged in
// every case.
//
// Many records per signal: warp u takes slice u % sig_split of signal
// u / sig_split (its lanes stride over the slice), adds its compensated sums
// into the FP64 accumulators sig_acc[b] and counts itself in part_cnt[g]; the
// warp that completes group g tests its signals (one lane per signal) and
// decides it -- no warp waits on another -- and restores sig_acc and the count.
template <typename real>
__device__ void verify_sig_split(const VerifyParams& v, unsigned long long& clean_max) {
  const int64_t split = v.sig_split;
  const int64_t nunits = v.batch * split;
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t u = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); u < nunits; u += (int64_t)gridDim.x * wpb) {
    const int64_t b = u / split, sl = u - b * split;
    const int64_t i0 = v.sig_slots_in * sl / split, i1 = v.sig_slots_in * (sl + 1) / split;
    const int64_t o0 = v.sig_slots_out * sl / split, o1 = v.sig_slots_out * (sl + 1) / split;
    SigSums<real> a;
    sig_add_records(v, b, i0 + lane, i1, o0 + lane, o1, 32, a);
    for (int off = 16; off > 0; off >>= 1) a.merge(a.shfl(off));
    const int64_t g = b / v.group;
    const int64_t gsize = min((int64_t)v.group, v.batch - g * v.group);
    int last = 0;
    if (lane == 0) {
      double* acc = v.sig_acc + b * kSigAcc;
      for (int k = 0; k < kSigQ; k++) atomicAdd(acc + k, (double)a.q[k].s + (double)a.q[k].c);
      __threadfence();
      last = atomicAdd(v.part_cnt + g, 1u) == (unsigned)(gsize * split - 1);
      if (last) __threadfence();
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) continue;
    SigGroup<real> c;
    c.zero();
    for (int64_t j = lane; j < gsize; j += 32) {
      double* aj = v.sig_acc + (g * v.group + j) * kSigAcc;
      double q[kSigQ];
      for (int k = 0; k < kSigQ; k++) { q[k] = __ldcg(aj + k); aj[k] = 0.0; }
      real hi[kSigQ], lo[kSigQ];
      for (int k = 0; k < kSigQ; k++) { hi[k] = (real)q[k]; lo[k] = (real)(q[k] - (double)hi[k]); }
      sig_test(v, c, (int)j, hi, lo);
    }
    for (int off = 16; off > 0; off >>= 1) c.merge(c.shfl(off));
    if (lane == 0) {
      v.part_cnt[g] = 0u;
      decide_sig_group(v, g, gsize, c, clean_max);
    }
  }
}

template <typename real>
__global__ void verify_sig_kernel(const VerifyParams v, int lanes) {
  __shared__ unsigned long long smax[8];
  unsigned long long clean_max = 0;   // bits of the largest clean ratio (a nonnegative double)
  if (v.sig_split > 0) verify_sig_split<real>(v, clean_max);
  else verify_sig_serial<real>(v, lanes, clean_max, blockIdx.x, gridDim.x);
  for (int off = 16; off > 0; off >>= 1) clean_max = max(clean_max, __shfl_xor_sync(0xffffffffu, clean_max, off));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = clean_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, smax[w]);
    if (m) atomicMax(&v.counters->max_clean_ratio_bits, m);
  }
}

// Many signals with a few dozen to a few hundred records each: one block of
// kVT threads per unit of `gpb` consecutive groups (or one group in rounds
// of kVT / L signals when a group has more).  L consecutive lanes add one
// signal's records (lane l takes records l, l + L, ...; L a power of two
// near the record count, at most 32) and combine by shuffles; the signal
// sums go to shared memory and the unit's groups are decided there.  No
// atomics and no cross-block accumulators: the split mode's per-signal
// FP64 atomics and fences cost more than the records themselves here.
constexpr int kVT = 256;

// Groups [0, ng) of a one-round unit, signal j of the unit's sums at
// sm[j 2 kSigQ]: Dl lanes per group (a power of two, at most 32), lane d its
// signals d, d + Dl, ...; the group's first lane decides.
template <typename real>
__device__ void decide_unit(const VerifyParams& v, int64_t g0, int ng, const real* sm,
                            unsigned long long& clean_max) {
  int Dl = 1;
  while (Dl < v.group && Dl < 32) Dl <<= 1;
  const int per_warp = 32 / Dl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / Dl, d = lane % Dl;
  for (int q0 = warp * per_warp; q0 < ng; q0 += (kVT / 32) * per_warp) {
    const int q = q0 + sub;
    SigGroup<real> c;
    c.zero();
    int64_t gsize = 0;
    if (q < ng) {
      gsize = min((int64_t)v.group, v.batch - (g0 + q) * v.group);
      for (int64_t j = d; j < gsize; j += Dl) {
        const real* sj = sm + ((int64_t)q * v.group + j) * 2 * kSigQ;
        sig_test(v, c, (int)j, sj, sj + kSigQ);
      }
    }
    for (int off = Dl >> 1; off > 0; off >>= 1) c.merge(c.shfl(off));
    if (q < ng && d == 0) decide_sig_group(v, g0 + q, gsize, c, clean_max);
  }
}

template <typename real>
__global__ void __launch_bounds__(kVT, 2) verify_sig_blocks(const VerifyParams v, int lanes) {
  __shared__ real sm[kVT * 2 * kSigQ];
  __shared__ unsigned long long smax[kVT / 32];
  unsigned long long clean_max = 0;   // bits of the largest clean ratio (a nonnegative double)
  const int L = lanes, spb = kVT / L, gpb = v.sig_gpb;
  const int t = threadIdx.x, jj = t / L, l = t % L, warp = t >> 5, lane = t & 31;
  const int64_t nunits = (v.ngroups + gpb - 1) / gpb;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int64_t g0 = u * gpb;
    const int ng = (int)min((int64_t)gpb, v.ngroups - g0);
    const int64_t bfirst = g0 * v.group;
    const int64_t nsig = min(v.batch, (g0 + ng) * v.group) - bfirst;
    const int64_t rounds = (nsig + spb - 1) / spb;
    SigGroup<real> c;                 // a unit of one group in rounds: warp 0 tests, round by round
    c.zero();
    for (int64_t r = 0; r < rounds; r++) {
      const int64_t j = r * spb + jj;
      SigSums<real> a;
      if (j < nsig) sig_add_records(v, bfirst + j, l, v.sig_slots_in, l, v.sig_slots_out, L, a);
      for (int off = L >> 1; off > 0; off >>= 1) a.merge(a.shfl(off));
      if (l == 0 && j < nsig) {
        real* dst = sm + (int64_t)jj * 2 * kSigQ;
#pragma unroll
        for (int k = 0; k < kSigQ; k++) { dst[k] = a.q[k].s; dst[kSigQ + k] = a.q[k].c; }
      }
      __syncthreads();
      if (rounds == 1) {
        decide_unit(v, g0, ng, sm, clean_max);
      } else if (warp == 0) {
        const int64_t jend = min(nsig, (r + 1) * spb);
        for (int64_t jx = r * spb + lane; jx < jend; jx += 32) {
          const real* sj = sm + (jx - r * spb) * 2 * kSigQ;
          sig_test(v, c, (int)jx, sj, sj + kSigQ);
        }
      }
      __syncthreads();
    }
    if (rounds > 1 && warp == 0) {
      const int64_t gsize = min((int64_t)v.group, v.batch - g0 * v.group);
      for (int off = 16; off > 0; off >>= 1) c.merge(c.shfl(off));
      if (lane == 0) decide_sig_group(v, g0, gsize, c, clean_max);
    }
  }
  for (int off = 16; off > 0; off >>= 1) clean_max = max(clean_max, __shfl_xor_sync(0xffffffffu, clean_max, off));
  if (lane == 0) smax[warp] = clean_max;
  __syncthreads();
  if (t == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < kVT / 32; w++) m = max(m, smax[w]);
    if (m) atomicMax(&v.counters->max_clean_ratio_bits, m);
  }
}

int sig_split_of(int64_t recs, int64_t batch, int sms) {
  if (recs <= kSigSerialMax) return 0;               // one lane per signal
  // warps of at most 1024 records, and at least 16 warps per SM in all
  int64_t want = (recs + 1023) / 1024;
  const int64_t cover = (16 * (int64_t)sms + batch - 1) / batch;
  want = std::max(want, std::min(cover, (recs + 127) / 128));
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 1 << 16));
}

int sig_block_geom(int64_t rin, int64_t rout, int64_t group, int64_t ngroups, int sms, int* gpb) {
  const int64_t rmax = std::max<int64_t>(1, std::max(rin, rout));
  int L = 1;
  while (L < 32 && L < rmax) L <<= 1;
  const int64_t spb = kVT / L;
  *gpb = group <= spb ? (int)(spb / group) : 1;
  const int64_t units = (ngroups + *gpb - 1) / *gpb;
  return units >= sms ? L : 0;
}

int verify_split(int64_t recs, int64_t ngroups, int sms) {
  // about 2048 records per block, and no more blocks in total than 4 per SM
  if (recs <= 4096 || ngroups >= sms) return 1;
  const int64_t want = (recs + 2047) / 2048;
  const int64_t cap = std::max<int64_t>(1, (int64_t)4 * sms / ngroups);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(cap, 256)));
}

cudaError_t launch_verify(const VerifyParams& vin, cudaStream_t s) {
  const int threads = 256;
  VerifyParams v = vin;
  if (v.sigrec && v.sig_blk_lanes > 0) {
    const int64_t units = (v.ngroups + v.sig_gpb - 1) / v.sig_gpb;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(units, (int64_t)v.max_blocks));
    if (v.dtype == 0) verify_sig_blocks<float><<<(unsigned)blocks, kVT, 0, s>>>(v, v.sig_blk_lanes);
    else verify_sig_blocks<double><<<(unsigned)blocks, kVT, 0, s>>>(v, v.sig_blk_lanes);
    return cudaGetLastError();
  }
  if (v.sigrec) {
    int lanes = 1;
    while (lanes < v.group && lanes < 32) lanes <<= 1;
    int64_t blocks;
    if (v.sig_split > 0) blocks = (v.batch * v.sig_split + threads / 32 - 1) / (threads / 32);
    else blocks = (v.ngroups * lanes + threads - 1) / threads;
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)v.max_blocks));
    if (v.dtype == 0) verify_sig_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(v, lanes);
    else verify_sig_kernel<double><<<(unsigned)blocks, threads, 0, s>>>(v, lanes);
    return cudaGetLastError();
  }
  if (v.split < 1 || !v.part_acc || !v.part_cnt) v.split = 1;
  const int64_t recs = v.slots_in + v.slots_out;
  if (v.split > 1) {
    const int64_t blocks = std::min<int64_t>(v.ngroups * v.split, (int64_t)v.max_blocks);
    verify_kernel<<<(unsigned)blocks, threads, 0, s>>>(v, threads);
    return cudaGetLastError();
  }
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
  if (blockIdx.x == 0 && threadIdx.x == 0 && f.counters && !(f.err_flag && *f.err_flag)) {
    // this launch follows the transform of the checksums and the group
    // recomputes in stream order: both are done
    const long long nrec = min((long long)f.lists.rec[0], (long long)f.lists.cap_rec);
    if (count > 0) atomicAdd(&f.counters->corrected, (unsigned long long)count);
    if (nrec > 0) atomicAdd(&f.counters->recomputed, (unsigned long long)nrec);
  }
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
__global__ void gen_signs_kernel(double2* r, int64_t n, unsigned long long seed, int qdiv, int sign) {
  const double h = 0.86602540378443864676;   // sqrt(3)/2: w3 = -1/2 - i h
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double s = (sign && (splitmix64_at(seed, (unsigned long long)k) >> 63)) ? -1.0 : 1.0;
    // w3^k, times w3^floor(qdiv k / n) for the second left vector
    const int m = (int)((k + (qdiv ? ((int64_t)qdiv * k) / n : 0)) % 3);
    const double re = m == 0 ? 1.0 : -0.5, im = m == 0 ? 0.0 : (m == 1 ? -h : h);
    r[k] = double2{s * re, s * im};
  }
}

__global__ void c128_to_c64_kernel(const double2* a, float2* b, int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    b[k] = float2{(float)a[k].x, (float)a[k].y};
}

__global__ void gather_classes_kernel(const double2* src, double2* dst, int64_t M, int64_t nl) {
  const int64_t n = M * nl;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t L = i / nl, k = i - L * nl;
    dst[i] = src[L + M * k];
  }
}

cudaError_t launch_gather_classes(const void* src, void* dst, int64_t M, int64_t nl, cudaStream_t s) {
  gather_classes_kernel<<<fix_grid(M * nl, 1), 256, 0, s>>>(reinterpret_cast<const double2*>(src),
                                                          reinterpret_cast<double2*>(dst), M, nl);
  return cudaGetLastError();
}

cudaError_t launch_gen_signs(void* r, int64_t n, unsigned long long seed, cudaStream_t s, int qdiv, int sign) {
  gen_signs_kernel<<<fix_grid(n, 1), 256, 0, s>>>(reinterpret_cast<double2*>(r), n, seed, qdiv, sign);
  return cudaGetLastError();
}

cudaError_t launch_c128_to_c64(const void* src, void* dst, int64_t n, cudaStream_t s) {
  c128_to_c64_kernel<<<fix_grid(n, 1), 256, 0, s>>>(reinterpret_cast<const double2*>(src),
                                                    reinterpret_cast<float2*>(dst), n);
  return cudaGetLastError();
}

}  // namespace tfft
