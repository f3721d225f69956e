// fft_pass.cuh -- the batched Stockham sub-transform kernel with the fused
// two-sided checksum encode (TurboFFT Sections III and IV).
//
// One launch performs one "pass": a batch of independent sub-DFTs of length
// nsub along the lines of a strided view of the data (Section IV-A, tiled FFT:
// the signal of length N is viewed as an N1 x N2 (x N3) array and each launch
// transforms along one axis).  A thread block takes a tile of C lines x nsub
// elements; every thread holds E complex values in registers and performs
// radix-E butterflies ("thread-level workload", Section IV-A: 8, 16 or 32
// elements per thread); the tile is exchanged between radix stages through
// shared memory in Stockham (autosort) order, so the result comes out in
// natural order with no bit reversal.
//
// Fused two-sided ABFT (Section III, Eqs. two_side_X and two_side_Y, and the
// threadblock-level scheme of Section IV-B):
//   * first pass, as values are loaded: each thread adds w_n x_n over its
//     elements (w = W^T r, r_j = e^{-2 pi i j/3}) and accumulates the signal's
//     partial into S1 (weight 1) and S2 (weight b+1) of the group, plus the
//     input energy for the threshold -- registers only, no extra memory pass;
//   * last pass, as values are stored: each thread adds r_k y_k over its
//     outputs into T1 and T2 the same way;
//   * once per chunk (a share of one group) the block reduces its partials and
//     writes one record; the verify kernel combines records per group.
// Fault injection (Section II-A) perturbs one register value at a chosen
// (pass, stage, signal, line, index) before it is checksummed or stored.
#pragma once

#include <cstdint>
#include <utility>

#include "tfft_internal.h"

namespace tfft {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename cT> __device__ __forceinline__ cT c_add(cT a, cT b) { return {a.x + b.x, a.y + b.y}; }
template <typename cT> __device__ __forceinline__ cT c_sub(cT a, cT b) { return {a.x - b.x, a.y - b.y}; }
template <typename cT> __device__ __forceinline__ cT c_mul(cT a, cT b) {
  return {fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return {fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}


// cos(pi m / 8) and sin(pi m / 8) for m = 0..15: the only angles a radix-2^k
// butterfly with k <= 4 needs.  Values of the trigonometric functions at
// multiples of pi/8 (cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2).
struct Eighths {
  static constexpr double c4 = 0.70710678118654752440084436210484904;   // cos(pi/4)
  static constexpr double c1 = 0.92387953251128675612818318939678829;   // cos(pi/8)
  static constexpr double s1 = 0.38268343236508977172845998403039887;   // sin(pi/8)
  __host__ __device__ static constexpr double cosv(int m) {
    switch (m & 15) {
      case 0: return 1.0;   case 1: return c1;    case 2: return c4;    case 3: return s1;
      case 4: return 0.0;   case 5: return -s1;   case 6: return -c4;   case 7: return -c1;
      case 8: return -1.0;  case 9: return -c1;   case 10: return -c4;  case 11: return -s1;
      case 12: return 0.0;  case 13: return s1;   case 14: return c4;   default: return c1;
    }
  }
  // sin x = cos(x - pi/2)
  __host__ __device__ static constexpr double sinv(int m) { return cosv(m + 12); }
};

// v * omega_R^k, omega_R = e^{-2 pi i / R}, R <= 16, with the trivial angles
// special-cased (no multiply by 0 or 1).
template <int R, int k, typename cT>
__device__ __forceinline__ cT mul_root(cT a) {
  using real = decltype(a.x);
  constexpr int m = (k * (16 / R)) & 15;   // angle 2 pi k / R = pi m / 8
  if constexpr (m == 0) return a;
  else if constexpr (m == 4) return {a.y, -a.x};
  else if constexpr (m == 8) return {-a.x, -a.y};
  else if constexpr (m == 12) return {-a.y, a.x};
  else if constexpr (m == 2) {
    const real h = (real)Eighths::c4;
    return {(a.x + a.y) * h, (a.y - a.x) * h};
  } else if constexpr (m == 6) {
    const real h = (real)Eighths::c4;
    return {(a.y - a.x) * h, -(a.x + a.y) * h};
  } else if constexpr (m == 10) {
    const real h = (real)Eighths::c4;
    return {-(a.x + a.y) * h, (a.x - a.y) * h};
  } else if constexpr (m == 14) {
    const real h = (real)Eighths::c4;
    return {(a.x - a.y) * h, (a.x + a.y) * h};
  } else {
    // (a.x + i a.y)(c - i s) = (a.x c + a.y s) + i (a.y c - a.x s)
    constexpr real c = (real)Eighths::cosv(m), s = (real)Eighths::sinv(m);
    return {fma(a.x, c, a.y * s), fma(a.y, c, -(a.x * s))};
  }
}

// In-register DFT of length R (natural order in and out), recursive radix-2
// decimation in time with compile-time twiddles.
template <int R> struct Dft {
  template <typename cT, int... ks>
  __device__ __forceinline__ static void combine(cT* v, const cT* e, const cT* o,
                                                 std::integer_sequence<int, ks...>) {
    constexpr int H = R / 2;
    ((v[ks] = c_add(e[ks], mul_root<R, ks>(o[ks])),
      v[ks + H] = c_sub(e[ks], mul_root<R, ks>(o[ks]))), ...);
  }
  template <typename cT> __device__ __forceinline__ static void run(cT* v) {
    constexpr int H = R / 2;
    cT e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; i++) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    Dft<H>::run(e);
    Dft<H>::run(o);
    combine(v, e, o, std::make_integer_sequence<int, H>{});
  }
};
template <> struct Dft<1> {
  template <typename cT> __device__ __forceinline__ static void run(cT*) {}
};

template <typename cT>
__device__ __forceinline__ cT ldg_c(const cT* p) { return __ldg(p); }

// The stored form of an output value: conjugated for the inverse transform,
// scaled by 1/N when normalising (the checksums use the value before this).
template <typename cT>
__device__ __forceinline__ cT out_xform(cT v, const PassParams& p) {
  using real = decltype(v.x);
  if (p.conj_out || p.out_scale != 1.0) {
    const real sc = (real)p.out_scale;
    v.x *= sc;
    v.y *= p.conj_out ? -sc : sc;
  }
  return v;
}

// Multiply v[1..R-1] by omega_{Ns R}^{r k}.  tab holds omega_T^m, T = the
// table length; m1 = k * nsub / (Ns R), scaled by `stride` = T / nsub.
// Four table reads (r = 1, 2, 4, 8); the other powers are products of at
// most three table values, so the error stays a few units in the last place.
template <int R, typename cT>
__device__ __forceinline__ void stage_twiddle(cT* v, const cT* tab, int m1s) {
  if (m1s == 0) return;
  if constexpr (R == 2) {
    v[1] = c_mul(v[1], ldg_c(tab + m1s));
  } else if constexpr (R == 4) {
    cT w1 = ldg_c(tab + m1s), w2 = ldg_c(tab + 2 * m1s);
    cT w3 = c_mul(w2, w1);
    v[1] = c_mul(v[1], w1); v[2] = c_mul(v[2], w2); v[3] = c_mul(v[3], w3);
  } else if constexpr (R == 8) {
    cT w[8];
    w[1] = ldg_c(tab + m1s); w[2] = ldg_c(tab + 2 * m1s); w[4] = ldg_c(tab + 4 * m1s);
    w[3] = c_mul(w[2], w[1]); w[5] = c_mul(w[4], w[1]); w[6] = c_mul(w[4], w[2]);
    w[7] = c_mul(w[4], w[3]);
#pragma unroll
    for (int r = 1; r < 8; r++) v[r] = c_mul(v[r], w[r]);
  } else if constexpr (R == 16) {
    cT w[16];
    w[1] = ldg_c(tab + m1s); w[2] = ldg_c(tab + 2 * m1s); w[4] = ldg_c(tab + 4 * m1s);
    w[8] = ldg_c(tab + 8 * m1s);
    w[3] = c_mul(w[2], w[1]); w[5] = c_mul(w[4], w[1]); w[6] = c_mul(w[4], w[2]);
    w[7] = c_mul(w[4], w[3]);
#pragma unroll
    for (int r = 1; r < 8; r++) w[8 + r] = c_mul(w[8], w[r]);
#pragma unroll
    for (int r = 1; r < 16; r++) v[r] = c_mul(v[r], w[r]);
  }
}

// Swizzled shared-memory index of element i of tile line c: the low bits of
// i are XORed with the next bits so that strided Stockham writes and unit-
// stride reads both spread over the banks; `pitch` separates the lines.
template <typename cT>
__device__ __forceinline__ int sm_index(int c, int i, int pitch) {
  constexpr int S = 128 / sizeof(cT);          // elements per 128-byte row
  constexpr int lgS = (S == 16) ? 4 : 3;
  return c * pitch + (i ^ ((i >> lgS) & (S - 1)));
}

// omega_N^m from the two-level table (m < N).
template <typename cT>
__device__ __forceinline__ cT twN(const PassParams& p, int64_t m) {
  const cT* lo = reinterpret_cast<const cT*>(p.twN_lo);
  const cT* hi = reinterpret_cast<const cT*>(p.twN_hi);
  return c_mul(ldg_c(hi + (m >> p.twN_lbits)), ldg_c(lo + (m & ((int64_t(1) << p.twN_lbits) - 1))));
}

// Checksum weight w_n = (W^T r)_n = K / (1 - w3 wN^n), K = 1 - w3^N, evaluated
// without cancellation: w3 wN^n = e^{-i theta}, theta = 2 pi m / (3N),
// m = (N + 3n) mod 3N, and 1/(1 - e^{-i theta}) = 1/2 - (i/2) cot(theta/2);
// theta/2 is folded into [0, pi/2] and e^{i theta/2} read from a two-level table.
template <typename cT>
__device__ __forceinline__ cT checksum_weight(const PassParams& p, int64_t npos) {
  using real = decltype(cT{}.x);
  const int64_t N3 = 3 * p.n;
  int64_t m = p.n + 3 * npos;
  if (m >= N3) m -= N3;
  const bool up = 2 * m > N3;
  const int64_t mm = up ? N3 - m : m;
  const cT* lo = reinterpret_cast<const cT*>(p.wt_lo);
  const cT* hi = reinterpret_cast<const cT*>(p.wt_hi);
  const cT h = ldg_c(hi + (mm >> p.wt_lbits));
  const cT l = ldg_c(lo + (mm & ((int64_t(1) << p.wt_lbits) - 1)));
  const real s = fma(h.y, l.x, h.x * l.y);     // sin: both terms >= 0
  real c = fma(h.x, l.x, -(h.y * l.y));        // cos
  if (up) c = -c;
  const real rho = c / s;
  const real kr = (real)p.wk_re, ki = (real)p.wk_im;
  return {(real)0.5 * fma(rho, ki, kr), (real)0.5 * fma(-rho, kr, ki)};
}

// The value with the armed fault applied (returned by value so that no
// register array is ever addressed through a pointer).
template <typename cT>
__device__ __forceinline__ cT faulted(cT v, const FaultSite& f) {
  using real = decltype(v.x);
  if (f.mode == 1) {
    constexpr int W = 8 * sizeof(real);
    if constexpr (sizeof(real) == 4) {
      if (f.bit < W) v.x = __int_as_float(__float_as_int(v.x) ^ (int)(1u << f.bit));
      else v.y = __int_as_float(__float_as_int(v.y) ^ (int)(1u << (f.bit - W)));
    } else {
      if (f.bit < W) v.x = __longlong_as_double(__double_as_longlong(v.x) ^ (long long)(1ull << f.bit));
      else v.y = __longlong_as_double(__double_as_longlong(v.y) ^ (long long)(1ull << (f.bit - W)));
    }
  } else if (f.mode == 2) {
    v.x *= (real)f.factor;
    v.y *= (real)f.factor;
  } else if (f.mode == 3 || f.mode == 4) {
    v.x += (real)f.factor;
  }
  return v;
}

// Signal b carries the armed fault (mode 4 arms signals s and s + 1).
__device__ __forceinline__ bool fault_signal(const FaultSite& f, int64_t b) {
  return f.signal == b || (f.mode == 4 && f.signal + 1 == b);
}

// (c, j) of butterfly f in a stage of radix R.
__device__ __forceinline__ void map_bfly(int f, int mode, int C, int nb, int& c, int& j) {
  if (mode == MAP_COL) { c = f & (C - 1); j = f / C; }
  else { j = f & (nb - 1); c = f / nb; }
}

// Per-thread ABFT partials.
template <typename real>
struct Partials {
  real s1r, s1i, s2r, s2i, en, t1r, t1i, t2r, t2i;
  long long nf_min, nf_max;
  __device__ __forceinline__ void zero() {
    s1r = s1i = s2r = s2i = en = t1r = t1i = t2r = t2i = (real)0;
    nf_min = 0x7fffffffffffffffLL; nf_max = -1;
  }
};

// Block-wide reduction of the partials; thread 0 writes the records.
template <typename real>
__device__ void reduce_and_store(Partials<real>& a, const PassParams& p, int64_t g,
                                 int64_t slot, double* red) {
  const unsigned full = 0xffffffffu;
  real v[9] = {a.s1r, a.s1i, a.s2r, a.s2i, a.en, a.t1r, a.t1i, a.t2r, a.t2i};
  long long mn = a.nf_min, mx = a.nf_max;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < 9; q++) v[q] += __shfl_xor_sync(full, v[q], off);
    mn = min(mn, __shfl_xor_sync(full, mn, off));
    mx = max(mx, __shfl_xor_sync(full, mx, off));
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = (blockDim.x + 31) >> 5;
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 9; q++) red[warp * 12 + q] = (double)v[q];
    reinterpret_cast<long long*>(red)[warp * 12 + 9] = mn;
    reinterpret_cast<long long*>(red)[warp * 12 + 10] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    long long m0 = 0x7fffffffffffffffLL, m1 = -1;
    for (int w = 0; w < nwarps; w++) {
      for (int q = 0; q < 9; q++) s[q] += red[w * 12 + q];
      m0 = min(m0, reinterpret_cast<long long*>(red)[w * 12 + 9]);
      m1 = max(m1, reinterpret_cast<long long*>(red)[w * 12 + 10]);
    }
    if (p.abft_in) {
      RecIn r;
      r.s1r = s[0]; r.s1i = s[1]; r.s2r = s[2]; r.s2i = s[3]; r.energy = s[4];
      r.pad0 = r.pad1 = r.pad2 = 0.0;
      p.rec_in[g * p.slots + slot] = r;
    }
    if (p.abft_out) {
      RecOut r;
      r.t1r = s[5]; r.t1i = s[6]; r.t2r = s[7]; r.t2i = s[8];
      r.nf_min = m0; r.nf_max = m1; r.pad0 = r.pad1 = 0.0;
      p.rec_out[g * p.slots + slot] = r;
    }
  }
  __syncthreads();
}

// Threads per block are capped so that the widest per-thread state (E complex
// values of data and of checksum weights) fits in registers without spilling.
// Warp-wide reduction of the partials; lane 0 writes the warp's records at
// slot `slot` of group g (no block-wide synchronisation).
template <typename real>
__device__ void reduce_warp_and_store(Partials<real>& a, const PassParams& p, long long g, long long slot) {
  const unsigned full = 0xffffffffu;
  real v[9] = {a.s1r, a.s1i, a.s2r, a.s2i, a.en, a.t1r, a.t1i, a.t2r, a.t2i};
  long long mn = a.nf_min, mx = a.nf_max;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int q = 0; q < 9; q++) v[q] += __shfl_xor_sync(full, v[q], off);
    mn = min(mn, __shfl_xor_sync(full, mn, off));
    mx = max(mx, __shfl_xor_sync(full, mx, off));
  }
  if ((threadIdx.x & 31) == 0) {
    if (p.abft_in) {
      RecIn r;
      r.s1r = v[0]; r.s1i = v[1]; r.s2r = v[2]; r.s2i = v[3]; r.energy = v[4];
      r.pad0 = r.pad1 = r.pad2 = 0.0;
      p.rec_in[g * p.slots + slot] = r;
    }
    if (p.abft_out) {
      RecOut r;
      r.t1r = v[5]; r.t1i = v[6]; r.t2r = v[7]; r.t2i = v[8];
      r.nf_min = mn; r.nf_max = mx; r.pad0 = r.pad1 = 0.0;
      p.rec_out[g * p.slots + slot] = r;
    }
  }
}

template <typename real, int E>
constexpr int max_threads() { return sizeof(real) * E >= 64 ? 256 : 512; }

template <typename real, int E>
__global__ void __launch_bounds__(max_threads<real, E>())
fft_pass_kernel(const __grid_constant__ PassParams p) {
  using cT = typename Cplx<real>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cT* sm = reinterpret_cast<cT*>(smem_raw);
  __shared__ double red[32 * 12];

  const int t = threadIdx.x;
  const int nsub = p.nsub;
  const int C = p.C;
  const cT* __restrict__ gin = reinterpret_cast<const cT*>(p.in);
  cT* __restrict__ gout = reinterpret_cast<cT*>(p.out);
  const cT* tws = reinterpret_cast<const cT*>(p.tw_sub);
  const bool abft = p.abft_in || p.abft_out;
  const bool inject = p.fault.mode != 0 && p.fault.pass == p.pass_index;

  if (blockIdx.x == 0 && t == 0) {
    if (p.zero_on_entry[0]) *p.zero_on_entry[0] = 0;
    if (p.zero_on_entry[1]) *p.zero_on_entry[1] = 0;
    if (p.zero_on_entry[2]) *p.zero_on_entry[2] = 0;
  }

  // stage-0 butterfly of this thread (radix E, one per thread)
  int c0, j0;
  map_bfly(t, p.in_map, C, nsub / E, c0, j0);
  const int R_last = nsub >> (__ffs(E) - 1) * (p.nstages - 1);   // nsub / E^(nstages-1)

  cT wv[E];             // checksum weights of this thread's input positions
  unsigned smask = 0;   // signs s_k of r at this thread's outputs, bit u*RL+q
  Partials<real> acc;
  bool setup_done = false;
  auto setup_positions = [&](int64_t hi, int64_t lo0) {
      if (p.abft_in) {
      const cT* wtab = reinterpret_cast<const cT*>(p.wtab);
#pragma unroll
      for (int r = 0; r < E; r++) {
        const int i = j0 + r * (nsub / E);
        const int64_t npos = p.lines_are_signals ? (int64_t)i * p.in_es
                                                 : hi * p.in_hi + (lo0 + c0) * p.in_lo + (int64_t)i * p.in_es;
        wv[r] = (p.rvec == RVEC_WANG) ? checksum_weight<cT>(p, npos) : ldg_c(wtab + npos);
      }
    }
    // signs s_k of r at this thread's output positions, bit u*RL+q
    smask = 0;
    if (p.abft_out && p.rvec == RVEC_SIGNED_WANG) {
      const int RL = p.nstages > 1 ? R_last : E;
      const int nb = nsub / RL;
      for (int ub = 0; ub < E / RL; ub++) {
        int c, j;
        if (p.nstages > 1) map_bfly(t + ub * p.nthreads, p.out_map, C, nb, c, j);
        else { c = c0; j = j0; }
        const int64_t lo = p.lines_are_signals ? 0 : lo0 + c;
        const int64_t kb = hi * p.out_hi + lo * p.out_lo;
        for (int q = 0; q < RL; q++) {
          const int64_t kpos = kb + (int64_t)(j + q * nb) * p.out_es;
          smask |= (unsigned)(splitmix64_at(p.rseed, (unsigned long long)kpos) >> 63) << (ub * RL + q);
        }
      }
    }
  };

  // a work list holds list[0] entries (often none): only their chunks are visited
  const int64_t nchunks =
      p.list ? min(p.nchunks, min((int64_t)p.list[0], (int64_t)p.list_cap) * p.parts * p.line_blocks) : p.nchunks;
  for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
    // ---- decode chunk -> (group, part, line block) and its signal range ----
    const int64_t lb = chunk % p.line_blocks;
    const int64_t rest = chunk / p.line_blocks;
    const int part = (int)(rest % p.parts);
    const int64_t g = rest / p.parts;
    int64_t gb, ge;
    if (p.list) {
      if (g >= p.list[0] || g >= p.list_cap) continue;
      const int64_t blk = p.list_identity ? g : p.list[1 + g];
      gb = blk * p.list_block;
      ge = min(p.batch, gb + p.list_block);
    } else {
      gb = g * p.group;
      ge = min(p.batch, gb + (int64_t)p.group);
    }
    const int64_t unit = p.lines_are_signals ? C : 1;          // signals per tile
    const int64_t ntiles = (ge - gb + unit - 1) / unit;
    const int64_t per = (ntiles + p.parts - 1) / p.parts;
    const int64_t sb = gb + (int64_t)part * per * unit;
    const int64_t se = min(ge, sb + per * unit);
    if (sb >= se) {
      if (abft) {   // keep the record well defined
        acc.zero();
        reduce_and_store(acc, p, g, part * p.line_blocks + lb, red);
      }
      continue;
    }
    // line block -> (hi, lo0) for multi-pass
    const int64_t L0 = lb * C;
    const int64_t hi = p.lines_are_signals ? 0 : L0 / p.LO;
    const int64_t lo0 = p.lines_are_signals ? 0 : L0 % p.LO;

    // checksum weights of this thread's input positions and signs of r at
    // its output positions: fixed for the whole kernel when lines are
    // signals, else per chunk (line block)
    if (!p.lines_are_signals || !setup_done) {
      setup_positions(hi, lo0);
      setup_done = true;
    }
    if (abft) acc.zero();

    for (int64_t tb = sb; tb < se; tb += unit) {
      // ================= stage 0: global -> registers =================
      cT v[E];
      {
        const int64_t b = p.lines_are_signals ? tb + c0 : tb;
        const int64_t lo = p.lines_are_signals ? 0 : lo0 + c0;
        const bool valid = b < se;
        const int64_t sb = p.soff_in ? (valid ? p.soff_in[b] : 0) : b * p.n;
        const int64_t base = sb + hi * p.in_hi + lo * p.in_lo;
#pragma unroll
        for (int r = 0; r < E; r++) {
          const int i = j0 + r * (nsub / E);
          v[r] = valid ? gin[base + (int64_t)i * p.in_es] : cT{(real)0, (real)0};
        }
        if (p.conj_in) {
#pragma unroll
          for (int r = 0; r < E; r++) v[r].y = -v[r].y;
        }
        if (p.abft_in) {
          real sr = 0, si = 0, en = 0;
#pragma unroll
          for (int r = 0; r < E; r++) {
            sr = fma(wv[r].x, v[r].x, sr); sr = fma(-wv[r].y, v[r].y, sr);
            si = fma(wv[r].x, v[r].y, si); si = fma(wv[r].y, v[r].x, si);
            en = fma(v[r].x, v[r].x, en); en = fma(v[r].y, v[r].y, en);
          }
          const real wgt = (real)(b - gb + 1);
          acc.s1r += sr; acc.s1i += si;
          acc.s2r = fma(wgt, sr, acc.s2r); acc.s2i = fma(wgt, si, acc.s2i);
          acc.en += en;
        }
        if (inject && p.fault.stage == -1 && valid && fault_signal(p.fault, b) &&
            p.fault.line == (p.lines_are_signals ? 0 : hi * p.LO + lo)) {
#pragma unroll
          for (int r = 0; r < E; r++)
            if (p.fault.index == j0 + r * (nsub / E)) v[r] = faulted(v[r], p.fault);
        }
      }

      int Ns = 1;
      if (p.nstages > 1) {
        // first radix-E stage, registers -> shared
        Dft<E>::run(v);
        {
          const int64_t b = p.lines_are_signals ? tb + c0 : tb;
          const int64_t line = p.lines_are_signals ? 0 : hi * p.LO + lo0 + c0;
#pragma unroll
          for (int q = 0; q < E; q++) {
            const int i = j0 * E + q;
            if (inject && p.fault.stage == 0 && fault_signal(p.fault, b) && p.fault.line == line &&
                p.fault.index == i && b < se)
              v[q] = faulted(v[q], p.fault);
            sm[sm_index<cT>(c0, i, p.pitch)] = v[q];
          }
        }
        __syncthreads();
        Ns = E;
        // middle radix-E stages, shared -> shared
        for (int s = 1; s < p.nstages - 1; s++) {
          int c, j;
          map_bfly(t, p.mid_map, C, nsub / E, c, j);
#pragma unroll
          for (int r = 0; r < E; r++) v[r] = sm[sm_index<cT>(c, j + r * (nsub / E), p.pitch)];
          __syncthreads();
          const int k = j & (Ns - 1);
          stage_twiddle<E>(v, tws, k * (nsub / (Ns * E)) * p.tw_sub_stride);
          Dft<E>::run(v);
          const int basei = (j / Ns) * Ns * E + k;
          const int64_t b = p.lines_are_signals ? tb + c : tb;
          const int64_t line = p.lines_are_signals ? 0 : hi * p.LO + lo0 + c;
#pragma unroll
          for (int q = 0; q < E; q++) {
            const int i = basei + q * Ns;
            if (inject && p.fault.stage == s && fault_signal(p.fault, b) && p.fault.line == line &&
                p.fault.index == i && b < se)
              v[q] = faulted(v[q], p.fault);
            sm[sm_index<cT>(c, i, p.pitch)] = v[q];
          }
          __syncthreads();
          Ns *= E;
        }
      }

      // ================= last stage: -> global =================
      auto last_stage = [&](auto RC) {
        constexpr int RL = decltype(RC)::value;
        constexpr int NB = E / RL;              // butterflies per thread
        const int nb = nsub / RL;
        cT u[E];
        int cc[NB], jj[NB];
        if (p.nstages > 1) {
#pragma unroll
          for (int ub = 0; ub < NB; ub++) {
            map_bfly(t + ub * p.nthreads, p.out_map, C, nb, cc[ub], jj[ub]);
#pragma unroll
            for (int r = 0; r < RL; r++)
              u[ub * RL + r] = sm[sm_index<cT>(cc[ub], jj[ub] + r * nb, p.pitch)];
          }
        } else {
          // single-stage transform: the loaded registers are the butterfly
#pragma unroll
          for (int r = 0; r < E; r++) u[r] = v[r];
          cc[0] = c0; jj[0] = j0;
        }
#pragma unroll
        for (int ub = 0; ub < NB; ub++) {
          cT* w = u + ub * RL;
          const int c = cc[ub], j = jj[ub];
          const int k = j & (Ns - 1);            // j < nb == Ns here (or Ns == 1)
          stage_twiddle<RL>(w, tws, k * (nsub / (Ns * RL)) * p.tw_sub_stride);
          Dft<RL>::run(w);
          const int64_t b = p.lines_are_signals ? tb + c : tb;
          const int64_t lo = p.lines_are_signals ? 0 : lo0 + c;
          const bool valid = b < se;
          if (p.twiddle) {
            // inter-pass twiddle omega_{tw_n}^{lo * i}, i = j + q * nb
#pragma unroll
            for (int q = 0; q < RL; q++) {
              const int64_t m = lo * (int64_t)(j + q * nb) * p.tw_scale;
              w[q] = c_mul(w[q], twN<cT>(p, m));
            }
          }
          if (inject && p.fault.stage == p.nstages - 1 && valid && fault_signal(p.fault, b) &&
              p.fault.line == (p.lines_are_signals ? 0 : hi * p.LO + lo)) {
#pragma unroll
            for (int q = 0; q < RL; q++)
              if (p.fault.index == j + q * nb) w[q] = faulted(w[q], p.fault);
          }
          const int64_t osb = p.soff_out ? (valid ? p.soff_out[b] : 0) : b * p.n;
          const int64_t obase = osb + hi * p.out_hi + lo * p.out_lo;
          if (valid) {
#pragma unroll
            for (int q = 0; q < RL; q++) gout[obase + (int64_t)(j + q * nb) * p.out_es] = out_xform(w[q], p);
          }
          if (p.abft_out && valid) {
            // r_k = s_k w3^(k mod 3), k = hi*out_hi + lo*out_lo + (j + q nb) out_es,
            // s_k = -1 where the sign mask has a bit (s = 1 for plain e_Wang):
            // signed sums per residue class of q mod 3, then the w3 powers
            real a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0;
#pragma unroll
            for (int q = 0; q < RL; q++) {
              const bool neg = (smask >> (ub * RL + q)) & 1u;
              const real yr = neg ? -w[q].x : w[q].x, yi = neg ? -w[q].y : w[q].y;
              if (q % 3 == 0) { a0r += yr; a0i += yi; }
              else if (q % 3 == 1) { a1r += yr; a1i += yi; }
              else { a2r += yr; a2i += yi; }
            }
            const int64_t kpos = hi * p.out_hi + lo * p.out_lo + (int64_t)j * p.out_es;
            const int k0 = (int)(kpos % 3);
            const int dl = (int)(((int64_t)nb * p.out_es) % 3);   // 1 or 2
            const real hr = (real)-0.5, hs = (real)0.86602540378443864676;   // w3 = hr - i hs
            // sum_c (w3^dl)^c a_c, w3^1 = (hr, -hs), w3^2 = (hr, +hs)
            const real s1 = (dl == 1) ? -hs : hs;    // imag of w3^dl
            real tr = a0r + (hr * a1r - s1 * a1i) + (hr * a2r + s1 * a2i);
            real ti = a0i + (hr * a1i + s1 * a1r) + (hr * a2i - s1 * a2r);
            // times w3^k0
            if (k0 == 1) { real x = hr * tr + hs * ti; ti = hr * ti - hs * tr; tr = x; }
            else if (k0 == 2) { real x = hr * tr - hs * ti; ti = hr * ti + hs * tr; tr = x; }
            const real wgt = (real)(b - gb + 1);
            acc.t1r += tr; acc.t1i += ti;
            acc.t2r = fma(wgt, tr, acc.t2r); acc.t2i = fma(wgt, ti, acc.t2i);
            if (!(isfinite(tr) && isfinite(ti))) {
              acc.nf_min = min(acc.nf_min, (long long)b);
              acc.nf_max = max(acc.nf_max, (long long)b);
            }
          }
        }
      };
      switch (p.nstages > 1 ? R_last : E) {
        case 1: if constexpr (E == 1) last_stage(std::integral_constant<int, 1>{}); break;
        case 2: if constexpr (E >= 2) last_stage(std::integral_constant<int, 2>{}); break;
        case 4: if constexpr (E >= 4) last_stage(std::integral_constant<int, 4>{}); break;
        case 8: if constexpr (E >= 8) last_stage(std::integral_constant<int, 8>{}); break;
        case 16: if constexpr (E >= 16) last_stage(std::integral_constant<int, 16>{}); break;
        default: break;
      }
      if (p.nstages > 1) __syncthreads();   // shared tile reused by the next tile
    }
    if (abft) reduce_and_store(acc, p, g, part * p.line_blocks + lb, red);
  }
}

}  // namespace tfft
