// sigverify.cuh -- the per-signal checksum verification of the two-sided
// ABFT (Section III-A "Error Detection"): the device code shared by the
// verification kernels (abft_fix.cu) and the single-pass tile kernel, whose
// last block verifies small plans itself (fused verification).
#pragma once
#include <cmath>
#include <cstdint>

#include "tfft_internal.h"

namespace tfft {

// An exec's own fields, given apart from the plan's verification parameters.
struct ExecFields {
  long long exec_index;
  long long* cond_flag;
  cudaGraphConditionalHandle cond;
  int* queued = nullptr;        // set (shared memory) when a group is queued for correction
};

// A record, read through the L2 (the fused verification reads records that
// other blocks of the same launch wrote).
template <typename T>
__device__ __forceinline__ T ld_rec(const T* p) {
  static_assert(sizeof(T) % 8 == 0, "records are whole 8-byte words");
  T r;
  if constexpr (sizeof(T) % 16 == 0) {
    const uint4* s = reinterpret_cast<const uint4*>(p);
    uint4* d = reinterpret_cast<uint4*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 16); i++) d[i] = __ldcg(s + i);
  } else {
    const uint2* s = reinterpret_cast<const uint2*>(p);
    uint2* d = reinterpret_cast<uint2*>(&r);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 8); i++) d[i] = __ldcg(s + i);
  }
  return r;
}

// Numerics: a signal's records are added with compensated sums in the
// element type (Neumaier's variant of Kahan summation for complex64), so the
// sums carry a few units of rounding whatever their length, and the
// residual is formed from the compensated parts; the tests and the group
// sums then run in the element type.  Only the cross-block accumulators of
// the split mode are FP64 (atomics in the L2), and the group's decision
// converts to FP64 for its log entry.  GB300's FP64 rate is a small fraction
// of its FP32 rate, and a batch of short signals has a million of them.

template <typename real> struct CSum;
template <> struct CSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ void merge(const CSum& o) { add(o.s); c += o.c; }
  __device__ __forceinline__ CSum shfl(int off) const {
    CSum r;
    r.s = __shfl_xor_sync(0xffffffffu, s, off);
    r.c = __shfl_xor_sync(0xffffffffu, c, off);
    return r;
  }
};
template <> struct CSum<double> {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void merge(const CSum& o) { s += o.s; }
  __device__ __forceinline__ CSum shfl(int off) const {
    CSum r;
    r.s = __shfl_xor_sync(0xffffffffu, s, off);
    return r;
  }
};

// The nine sums of one signal: w^T x (re, im), ||x||^2, r^T y (re, im), and
// for the second check r2^T y and u2^T z (re, im each).
constexpr int kSigQ = 9;
template <typename real>
struct SigSums {
  CSum<real> q[kSigQ];
  __device__ __forceinline__ void merge(const SigSums& o) {
#pragma unroll
    for (int k = 0; k < kSigQ; k++) q[k].merge(o.q[k]);
  }
  __device__ __forceinline__ SigSums shfl(int off) const {
    SigSums r;
#pragma unroll
    for (int k = 0; k < kSigQ; k++) r.q[k] = q[k].shfl(off);
    return r;
  }
};

// Adds records [k0, k1) of signal b (SigIn / SigOut / SigChk slots k).
template <typename real>
__device__ __forceinline__ void sig_add_records(const VerifyParams& v, int64_t b, int64_t i0, int64_t i1,
                                                int64_t o0, int64_t o1, int64_t step, SigSums<real>& a) {
  const SigIn<real>* rin = reinterpret_cast<const SigIn<real>*>(v.sig_in) + b * v.sig_slots_in;
  const SigOut<real>* rout = reinterpret_cast<const SigOut<real>*>(v.sig_out) + b * v.sig_slots_out;
  // two input and two output records are loaded before any is added (four
  // loads in flight; each sum still adds its records in slot order)
  for (int64_t ki = i0, ko = o0; ki < i1 || ko < o1; ki += 2 * step, ko += 2 * step) {
    const bool ia = ki < i1, ib = ki + step < i1, oa = ko < o1, ob = ko + step < o1;
    SigIn<real> r0{}, r1{};
    SigOut<real> u0{}, u1{};
    if (ia) r0 = ld_rec(rin + ki);
    if (ib) r1 = ld_rec(rin + ki + step);
    if (oa) u0 = ld_rec(rout + ko);
    if (ob) u1 = ld_rec(rout + ko + step);
    if (ia) { a.q[0].add(r0.sr); a.q[1].add(r0.si); a.q[2].add(r0.en); }
    if (ib) { a.q[0].add(r1.sr); a.q[1].add(r1.si); a.q[2].add(r1.en); }
    if (oa) { a.q[3].add(u0.tr); a.q[4].add(u0.ti); }
    if (ob) { a.q[3].add(u1.tr); a.q[4].add(u1.ti); }
  }
  if (v.chk2) {
    const SigChk<real>* rc = reinterpret_cast<const SigChk<real>*>(v.sig_chk) + b * v.sig_slots_out;
    for (int64_t k = o0; k < o1; k += 2 * step) {
      const bool two = k + step < o1;
      const SigChk<real> r0 = ld_rec(rc + k);
      SigChk<real> r1{};
      if (two) r1 = ld_rec(rc + k + step);
      a.q[5].add(r0.tr); a.q[6].add(r0.ti); a.q[7].add(r0.sr); a.q[8].add(r0.si);
      if (two) { a.q[5].add(r1.tr); a.q[6].add(r1.ti); a.q[7].add(r1.sr); a.q[8].add(r1.si); }
    }
  }
}

// The group state, merged over its signals.
template <typename real>
struct SigGroup {
  real d1r, d1i, d2r, d2i, en;   // group sums (finite signals only)
  int nflag, flagj, nonf;        // flagged signals, the lowest flagged index, non-finite ones
  real cmax;                     // largest clean |d| / tau of the signal tests
  real fres, ftau;               // residual and threshold of the lowest flagged signal
  __device__ __forceinline__ void zero() {
    d1r = d1i = d2r = d2i = en = (real)0;
    nflag = 0; flagj = 0x7fffffff; nonf = 0;
    cmax = fres = ftau = (real)0;
  }
  __device__ __forceinline__ void merge(const SigGroup& b) {
    d1r += b.d1r; d1i += b.d1i; d2r += b.d2r; d2i += b.d2i; en += b.en;
    if (b.nflag > 0 && (nflag == 0 || b.flagj < flagj)) { flagj = b.flagj; fres = b.fres; ftau = b.ftau; }
    nflag += b.nflag; nonf += b.nonf;
    cmax = cmax > b.cmax ? cmax : b.cmax;
  }
  __device__ __forceinline__ SigGroup shfl(int off) const {
    SigGroup o;
    const unsigned m = 0xffffffffu;
    o.d1r = __shfl_xor_sync(m, d1r, off); o.d1i = __shfl_xor_sync(m, d1i, off);
    o.d2r = __shfl_xor_sync(m, d2r, off); o.d2i = __shfl_xor_sync(m, d2i, off);
    o.en = __shfl_xor_sync(m, en, off);
    o.nflag = __shfl_xor_sync(m, nflag, off); o.flagj = __shfl_xor_sync(m, flagj, off);
    o.nonf = __shfl_xor_sync(m, nonf, off);
    o.cmax = __shfl_xor_sync(m, cmax, off);
    o.fres = __shfl_xor_sync(m, fres, off); o.ftau = __shfl_xor_sync(m, ftau, off);
    return o;
  }
};

// Signal j's (0-based within its group) tests from its sums s[0..8] (value
// and compensation per sum), added to the group state.
template <typename real>
__device__ __forceinline__ void sig_test(const VerifyParams& v, SigGroup<real>& c, int j, const real* hi,
                                         const real* lo) {
  // the residual from the compensated parts: (t - s) = (t_hi - s_hi) + (t_lo - s_lo)
  const real dr = (hi[3] - hi[0]) + (lo[3] - lo[0]);
  const real di = (hi[4] - hi[1]) + (lo[4] - lo[1]);
  const real en = hi[2] > (real)0 ? hi[2] : (real)0;
  const real se = sqrt(en);
  const real d = sqrt(dr * dr + di * di);
  real tb = (real)v.kappa_u_log2n_sqrtn * se;
  if (tb < (real)v.tau_floor) tb = (real)v.tau_floor;
  const bool fin = isfinite(d);
  bool fail = !fin || d > tb;
  real fres = d, ftau = tb, ratio = tb > (real)0 ? d / tb : (real)0;
  bool nonfin = !fin;
  if (v.chk2) {
    // the last pass on its own, against the second left vector
    const real er = (hi[5] - hi[7]) + (lo[5] - lo[7]);
    const real ei = (hi[6] - hi[8]) + (lo[6] - lo[8]);
    const real d2 = sqrt(er * er + ei * ei);
    real t2 = (real)v.kappa_u_chk2 * se;
    if (t2 < (real)v.tau_floor) t2 = (real)v.tau_floor;
    const bool fin2 = isfinite(d2);
    nonfin = nonfin || !fin2;
    if (!fail && (!fin2 || d2 > t2)) { fail = true; fres = d2; ftau = t2; }
    const real r2 = t2 > (real)0 ? d2 / t2 : (real)0;
    if (r2 > ratio) ratio = r2;
  }
  if (fin) {
    c.en += en;
    c.d1r += dr; c.d1i += di;
    c.d2r += (real)(j + 1) * dr;
    c.d2i += (real)(j + 1) * di;
  }
  if (fail) {
    if (c.nflag == 0 || j < c.flagj) { c.flagj = j; c.fres = fres; c.ftau = ftau; }
    c.nflag++;
    c.nonf += nonfin ? 1 : 0;
  } else if (ratio > c.cmax) {
    c.cmax = ratio;
  }
}

// The decision for group g (one thread): detection, location, work lists,
// counters and the fault log.
template <typename real>
__device__ void decide_sig_group(const VerifyParams& v, int64_t g, int64_t gsize, const SigGroup<real>& c,
                                 unsigned long long& clean_max, const ExecFields* ex = nullptr);

// (ex: this exec's index and graph conditional in place of v's -- the fused
// verification reads the plan's parameters where they lie)
template <typename real>
__device__ void decide_sig_group(const VerifyParams& v, int64_t g, int64_t gsize, const SigGroup<real>& c,
                                 unsigned long long& clean_max, const ExecFields* ex) {
  const real res = sqrt(c.d1r * c.d1r + c.d1i * c.d1i);
  real tau = (real)v.kappa_u_log2n_sqrtn * sqrt(c.en > (real)0 ? c.en : (real)0);
  if (tau < (real)v.tau_floor) tau = (real)v.tau_floor;
  const bool gfin = isfinite(res) && isfinite(c.d2r) && isfinite(c.d2i);
  if (c.nflag == 0 && gfin && !(res > tau)) {
    real ratio = tau > (real)0 ? res / tau : (real)0;
    if (c.cmax > ratio) ratio = c.cmax;
    clean_max = max(clean_max, (unsigned long long)__double_as_longlong((double)ratio));
    return;
  }
  atomicAdd(&v.counters->detected, 1ull);
  const int64_t gb = g * v.group;
  double qr = NAN, qi = NAN;
  if (gfin && res > (real)0) {
    const double a = c.d1r, bb = c.d1i, e = c.d2r, f = c.d2i;
    const double den = a * a + bb * bb;
    qr = (e * a + f * bb) / den;
    qi = (f * a - e * bb) / den;
  }
  int64_t bstar = -1;
  if (c.nflag == 1) {
    bstar = c.flagj;                                     // the one signal whose own test failed
  } else if (c.nflag == 0 && gfin && res > (real)0) {
    const double m = rint(qr);
    if (fabs(qr - m) < 0.25 && fabs(qi) < 0.25 && m >= 1.0 && m <= (double)gsize) bstar = (int64_t)m - 1;
  }
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
  if ((action == 1 || action == 2) && ex && ex->queued) *ex->queued = 1;
  long long* const cond_flag = ex ? ex->cond_flag : v.cond_flag;
  if ((action == 1 || action == 2) && cond_flag &&
      atomicExch(reinterpret_cast<unsigned long long*>(cond_flag), 1ull) == 0ull)
    cudaGraphSetConditional(ex ? ex->cond : v.cond, 1u);      // run the correction body of this exec's graph
  if (action == 3) atomicAdd(&v.counters->uncorrectable, 1ull);
  const unsigned long long slot = atomicAdd(&v.counters->log_total, 1ull);
  LogEvent ev;
  ev.exec_index = ex ? ex->exec_index : v.exec_index;
  ev.group = v.group_base + g;
  ev.signal = bstar >= 0 ? v.group_base * v.group + gb + bstar : -1;
  ev.action = action;
  ev.nonfinite = (c.nonf > 0 || !gfin) ? 1 : 0;
  // the located signal's own residual and threshold when one signal failed,
  // else the group's
  ev.residual = (double)(c.nflag == 1 ? c.fres : res);
  ev.tau = (double)(c.nflag == 1 ? c.ftau : tau);
  ev.q_re = qr;
  ev.q_im = qi;
  v.log[slot % kLogRing] = ev;
}

// Few records per signal: `lanes` (a power of two <= 32) consecutive lanes
// take one group, lane j its signals j, j + lanes, ...; each adds its
// records, tests the signal, the lanes combine by shuffles and the group's
// first lane decides.
// The block takes groups first, first + step, ... in units of blockDim.x /
// lanes groups (the kernel: its grid-stride share; the fused verification of
// a single-pass kernel: all of them in one block).
template <typename real>
__device__ void verify_sig_serial(const VerifyParams& v, int lanes, unsigned long long& clean_max,
                                  int64_t first_unit, int64_t unit_step, const ExecFields* ex = nullptr) {
  const int lane = threadIdx.x % lanes;
  const int64_t per_block = blockDim.x / lanes;
  for (int64_t g0 = first_unit * per_block; g0 < v.ngroups; g0 += unit_step * per_block) {
    const int64_t g = g0 + threadIdx.x / lanes;
    SigGroup<real> c;
    c.zero();
    int64_t gsize = 0;
    if (g < v.ngroups) {
      const int64_t gb = g * v.group;
      gsize = min((int64_t)v.group, v.batch - gb);
      for (int64_t j = lane; j < gsize; j += lanes) {
        SigSums<real> a;
        sig_add_records(v, gb + j, 0, v.sig_slots_in, 0, v.sig_slots_out, 1, a);
        real hi[kSigQ], lo[kSigQ];
#pragma unroll
        for (int k = 0; k < kSigQ; k++) { hi[k] = a.q[k].s; lo[k] = a.q[k].c; }
        sig_test(v, c, (int)j, hi, lo);
      }
    }
    for (int off = lanes >> 1; off > 0; off >>= 1) c.merge(c.shfl(off));
    if (g < v.ngroups && lane == 0) decide_sig_group(v, g, gsize, c, clean_max, ex);
  }
}

// The fused verification, at the end of a single-pass tile kernel: each
// block's threads fence their record stores (and the tile stores their
// block's bulk copies completed) and the block counts itself; the last block
// (no block waits for another) fences again, verifies every group, adds its
// largest clean ratio and resets the count.  Returns 0 in the other blocks,
// 1 in that block when the exec is clean, 2 when it queued a group.
template <typename real>
__device__ __noinline__ int fused_verify(const PassParams* pp) {
  __shared__ int s_last, s_queued;
  __shared__ unsigned long long s_max[32];
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __threadfence();                       // this thread's records and stores before the count
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(pp->fdone, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (!s_last) return 0;
  __threadfence();                       // every block's records before they are read
  const VerifyParams& v = *pp->fverify;
  if (threadIdx.x == 0) s_queued = 0;
  __syncthreads();
  const ExecFields ex{pp->exec_index, nullptr, cudaGraphConditionalHandle{}, &s_queued};
  int lanes = 1;
  while (lanes < v.group && lanes < 32) lanes <<= 1;
  unsigned long long clean_max = 0;
  verify_sig_serial<real>(v, lanes, clean_max, 0, 1, &ex);
  for (int off = 16; off > 0; off >>= 1) clean_max = max(clean_max, __shfl_xor_sync(0xffffffffu, clean_max, off));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = clean_max;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = max(m, s_max[w]);
    if (m) atomicMax(&v.counters->max_clean_ratio_bits, m);
    *pp->fdone = 0u;
  }
  __syncthreads();                       // the groups this block queued are in the lists
  return s_queued ? 2 : 1;
}

}  // namespace tfft
