// fft_v3.cuh -- the pass kernel with compile-time geometry and warp-local lines.
//
// Same transform, twiddles, fused checksum encode and TMA tile ring as
// fft_tile_kernel (fft_tile.cuh), restructured so that almost every issued
// instruction is arithmetic on the data:
//
//   * the sub-transform length NSUB and the pass role are template
//     parameters: every shared-memory offset is a compile-time multiple of a
//     per-thread base, the radix schedule is unrolled;
//   * a tile has 256 threads x E values; when a line (NSUB values) is held by
//     at most one warp, the warp owns whole lines and the radix stages
//     exchange data in place through the line's padded scratch with only
//     __syncwarp; longer lines (NSUB > 32 E) share a named barrier among the
//     warps of the line;
//   * two blocks per SM for complex64 (at most 128 registers a thread, about
//     100 KB of shared memory a block: two tile buffers and one scratch);
//   * no block-wide barrier per tile: thread 0 starts the first tile loads,
//     then each warp counts itself out of a tile with a shared-memory atomic
//     and the last of the eight stores the tile and refills its buffer with
//     the tile nbuf ahead; when the output box layout differs from the input
//     box layout (the last pass), a second counter makes sure every warp has
//     read its input before any output is written over it;
//   * column tiles (element-major boxes) are moved by TMA with its 128-byte /
//     64-byte shared-memory swizzle, which keeps the strided column reads of
//     the first stage within two wavefronts;
//   * the checksum partials are reduced per warp with shuffles and written as
//     one record per warp and chunk in the single pass (a chunk is one or a
//     few tiles there), and by one block reduction per chunk in the multi-pass
//     roles (a chunk spans the sixteen signals of a group).
#pragma once

#include "fft_tile.cuh"

namespace tfft {

enum V3Role : int { V3_SINGLE = 0, V3_COLS = 1, V3_LAST = 2 };

__host__ __device__ constexpr int v3_stages(int nsub, int e) {
  int s = 0;
  long long v = 1;
  while (v < nsub) { v *= e; s++; }
  return s < 1 ? 1 : s;
}
__host__ __device__ constexpr int v3_ipow(int b, int k) { return k == 0 ? 1 : b * v3_ipow(b, k - 1); }

template <typename real, int NSUB, int E, int ROLE>
struct V3 {
  using cT = typename Cplx<real>::T;
  static constexpr int ES = (int)sizeof(cT);                // 8 or 16 bytes
  static constexpr int T = 256;                             // threads per block
  static constexpr int TILE = T * E;                        // values per tile
  static constexpr int C = TILE / NSUB;                     // lines per tile
  static constexpr int TPL = NSUB / E;                      // threads per line
  static constexpr bool WL = TPL <= 32;                     // warp-local lines
  static constexpr int LPW = WL ? 32 / TPL : 1;             // lines per warp
  static constexpr int WPL = WL ? 1 : TPL / 32;             // warps per line
  static constexpr int S = v3_stages(NSUB, E);              // radix stages
  static constexpr int RL = NSUB / v3_ipow(E, S - 1);       // last radix
  static constexpr int NBL = NSUB / RL;                     // last-stage butterflies per line
  static constexpr int BPT = E / RL;                        // last-stage butterflies per thread
  static constexpr bool LM_IN = (ROLE == V3_SINGLE || ROLE == V3_LAST);
  static constexpr bool LM_OUT = (ROLE == V3_SINGLE);
  // element-major boxes: columns in groups of CS (<= 128 bytes per row)
  static constexpr int CS = (C * ES > 128) ? 128 / ES : C;
  static constexpr int ROWB = CS * ES;                      // bytes per box row
  static constexpr int SWZ = ROWB >= 128 ? 7 : (ROWB >= 64 ? 3 : (ROWB >= 32 ? 1 : 0));
  // padded line-major scratch: one pad value per 128 bytes
  static constexpr int PG = 128 / ES;
  static constexpr int PITCH = NSUB + NSUB / PG + (NSUB < PG ? 1 : 0);
  static constexpr int SCR = C * PITCH;                     // scratch values
  static_assert(C >= 1 && TILE % NSUB == 0, "tile must hold whole lines");
  static_assert(WL || TPL % 32 == 0, "a line is held by whole warps");

};

__device__ __forceinline__ uint32_t atom_add_acq_rel(unsigned* a, unsigned v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(a)), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ void red_add_release(unsigned* a, unsigned v) {
  asm volatile("red.release.cta.shared::cta.add.u32 [%0], %1;" ::"r"(smem_u32(a)), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(a)) : "memory");
  return v;
}

// Bounded wait on an mbarrier phase; gives up early once another warp has
// recorded a timeout in *abort.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort) {
  for (long long it = 0; it < kWaitLimit; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 1023) == 1023 && *abort) return false;
  }
  return false;
}

// Block reduction of the partials (256 threads), one record per chunk.
template <typename real>
__device__ void reduce_block_records(Partials<real>& a, const PassParams& p, long long g, long long slot,
                                     double* red) {
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
    for (int w = 0; w < 8; w++) {
#pragma unroll
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

// Shared-memory offsets of the per-thread access patterns.  Every pattern is
// a per-thread base plus a compile-time offset: idx(x) = x + x / PG is
// additive over the (base, offset) splits used below because each base is
// a multiple of PG or each offset keeps the sum inside the base's PG group.
template <typename G>
struct V3Addr {
  __host__ __device__ static constexpr int idx(int x) { return x + x / G::PG; }
  // box byte offset of (c, j + m) for a compile-time m that is a multiple of TPL
  // (base_swz is the swizzled base_lin; an offset that is a multiple of 1024
  // bytes leaves the swizzle bits 7..9 alone)
  template <bool LM>
  __device__ __forceinline__ static uint32_t box(uint32_t base_lin, uint32_t base_swz, int m) {
    if constexpr (LM) {
      return base_lin + (uint32_t)(m * G::ES);
    } else {
      const uint32_t mo = (uint32_t)(m * G::ROWB);
      if ((mo & 1023u) == 0) return base_swz + mo;
      const uint32_t o = base_lin + mo;
      return o ^ (((o >> 7) & G::SWZ) << 4);
    }
  }
};

// Blocks per SM the register budget targets: two for complex64 (at most 128
// registers a thread), one for complex128, whose values take twice the registers.
template <typename real>
constexpr int v3_min_blocks() { return sizeof(real) == 4 ? 2 : 1; }

// 256 threads (eight warps), two blocks per SM for complex64.  Thread 0 starts the first
// nbuf tile loads; afterwards the last warp to finish a tile stores it and
// refills its buffer with the tile nbuf ahead, so no warp waits for another
// except on data that has not arrived yet.
template <typename real, int NSUB, int E, int ROLE>
__global__ void __launch_bounds__(256, (v3_min_blocks<real>())) fft_v3_kernel(const __grid_constant__ PassParams p) {
  using G = V3<real, NSUB, E, ROLE>;
  using A = V3Addr<G>;
  using cT = typename G::cT;
  static_assert(E % G::PG == 0, "a thread's stage-0 values start on a pad group");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8 * 12];
  __shared__ TileCursor ldc[8];
  __shared__ unsigned arrivals[8];   // per buffer: warps done with the tile, cumulative
  __shared__ unsigned readers[8];    // per buffer: warps done reading the input box, cumulative
  __shared__ int s_abort;

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int nbuf = p.nbuf;
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nbuf * p.buf_bytes);
  cT* scr = reinterpret_cast<cT*>(base + (size_t)nbuf * p.buf_bytes + 1024);
  volatile int* abort_flag = &s_abort;

  if (t == 0) {
    for (int s = 0; s < nbuf; s++) {
      mbar_init(&full[s], 1);
      arrivals[s] = 0;
      readers[s] = 0;
    }
    fence_mbar_init();
    s_abort = 0;
    if (blockIdx.x == 0) {
      if (p.zero_on_entry[0]) *p.zero_on_entry[0] = 0;
      if (p.zero_on_entry[1]) *p.zero_on_entry[1] = 0;
    }
  }
  __syncthreads();
  if (t == 0) {
    TileCursor ld;
    ld.start(p);
    for (int s = 0; s < nbuf && ld.valid(p); s++) {
      issue_load(p, ld, reinterpret_cast<cT*>(base + (size_t)s * p.buf_bytes), &full[s]);
      ld.advance(p);
    }
    for (int w = 0; w < 8; w++) ldc[w] = ld;
  }
  __syncthreads();

  const cT* tws = reinterpret_cast<const cT*>(p.tw_sub);
  const bool abft = p.abft_in || p.abft_out;
  const bool inject = p.fault.mode != 0 && p.fault.pass == p.pass_index;

  // this thread's line and butterfly index inside the tile
  const int c0 = G::WL ? warp * G::LPW + lane / G::TPL : warp / G::WPL;
  const int j0 = G::WL ? lane % G::TPL : (warp % G::WPL) * 32 + lane;

  auto line_sync = [&]() {
    if constexpr (G::WL) {
      __syncwarp();
    } else if constexpr (G::WPL * 32 == G::T) {
      asm volatile("bar.sync 1, 256;" ::: "memory");
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(2 + c0), "r"(32 * G::WPL) : "memory");
    }
  };

  // per-thread shared-memory bases
  const int scr_c = c0 * G::PITCH;
  const int s_rd = scr_c + A::idx(j0);            // reads at j0 + m  (m a multiple of TPL)
  const int s_wr0 = scr_c + A::idx(j0 * E);       // stage-0 writes at j0 E + q
  auto lin_base = [&](bool lm) -> uint32_t {
    return lm ? (uint32_t)((c0 * NSUB + j0) * G::ES)
              : (uint32_t)(((c0 / G::CS) * NSUB + j0) * G::ROWB + (c0 % G::CS) * G::ES);
  };
  const uint32_t b_in = lin_base(G::LM_IN), b_out = lin_base(G::LM_OUT);
  const uint32_t z_in = b_in ^ (((b_in >> 7) & G::SWZ) << 4), z_out = b_out ^ (((b_out >> 7) & G::SWZ) << 4);

  cT wv[E];
  unsigned smask = 0;
  unsigned k0mask = 0;          // (k mod 3) of each last-stage butterfly, 2 bits each
  Partials<real> acc;
  bool setup_done = false;
  auto setup_positions = [&](long long hi, long long lo0) {
    if (p.abft_in) {
      const cT* wtab = reinterpret_cast<const cT*>(p.wtab);
      const long long lo = ROLE == V3_SINGLE ? 0 : lo0 + c0;
#pragma unroll
      for (int r = 0; r < E; r++) {
        const int i = j0 + r * G::TPL;
        const long long npos = (ROLE == V3_SINGLE) ? (long long)i
                                                    : hi * p.in_hi + lo * p.in_lo + (long long)i * p.in_es;
        wv[r] = (p.rvec == RVEC_WANG) ? checksum_weight<cT>(p, npos) : ldg_c(wtab + npos);
      }
    }
    smask = 0;
    k0mask = 0;
    if (p.abft_out) {
      const long long lo = (ROLE == V3_SINGLE) ? 0 : lo0 + c0;
      const long long kb = hi * p.out_hi + lo * p.out_lo;
#pragma unroll
      for (int u = 0; u < G::BPT; u++) {
        const int jl = j0 + u * G::TPL;
        const long long kp0 = kb + (long long)jl * p.out_es;
        k0mask |= (unsigned)(kp0 % 3) << (2 * u);
        if (p.rvec == RVEC_SIGNED_WANG) {
#pragma unroll
          for (int q = 0; q < G::RL; q++) {
            const long long kpos = kp0 + (long long)(q * G::NBL) * p.out_es;
            smask |= (unsigned)(splitmix64_at(p.rseed, (unsigned long long)kpos) >> 63) << (u * G::RL + q);
          }
        }
      }
    }
  };
  const int dl = (int)(((long long)G::NBL * p.out_es) % 3);   // 1 or 2
  bool aborted = false;

  int s = 0;             // ring buffer of the current tile
  unsigned wrap = 0;     // completed passes over the ring
  for (long long chunk = blockIdx.x; chunk < p.nchunks; chunk += gridDim.x) {
    TileCursor cur;
    cur.chunk = chunk;
    const bool nonempty = cur.decode(p);
    const long long slot0 = (long long)(cur.part * p.line_blocks + cur.lb) * (ROLE == V3_SINGLE ? 8 : 1);
    if (!nonempty) {
      if (abft && !p.list) {
        acc.zero();
        if constexpr (ROLE == V3_SINGLE) reduce_warp_and_store(acc, p, cur.g, slot0 + warp);
        else reduce_block_records(acc, p, cur.g, slot0, red);
      }
      continue;
    }
    const long long hi = cur.hi(p), lo0 = cur.lo0(p);
    if (ROLE != V3_SINGLE || !setup_done) {
      setup_positions(hi, lo0);
      setup_done = true;
    }
    if (abft) acc.zero();
    const long long se = cur.se;
    const long long lo_c = (ROLE == V3_SINGLE) ? 0 : lo0 + c0;
    const long long line_c = (ROLE == V3_SINGLE) ? 0 : hi * p.LO + lo_c;
    // checksum weight (b - first signal of the group + 1) of this thread's signal
    real wgt = (real)(int)(cur.sb - cur.gb + (ROLE == V3_SINGLE ? c0 : 0) + 1);
    constexpr int BSTEP = ROLE == V3_SINGLE ? G::C : 1;

    for (long long tb = cur.sb; tb < se; tb += BSTEP, wgt += (real)BSTEP) {
      unsigned char* tile = base + (size_t)s * p.buf_bytes;
      if (!aborted && !mbar_wait_bounded(&full[s], wrap & 1u, abort_flag)) {
        aborted = true;
        *abort_flag = 1;
        atomicExch(p.err_flag, 1);
      }
      // after a timeout the warp still runs the tile (on whatever the buffer
      // holds) so that every line barrier is reached; the error flag is set
      const long long b0 = (ROLE == V3_SINGLE) ? tb + c0 : tb;     // this thread's signal
      const bool valid = b0 < se;
      // the stage at which this thread plants the test fault (none: -9)
      const int fst = (inject && valid && fault_signal(p.fault, b0) && p.fault.line == line_c) ? p.fault.stage
                                                                                               : -9;

      // ---------------- stage 0: box -> registers ----------------
      cT v[E];
#pragma unroll
      for (int r = 0; r < E; r++)
        v[r] = *reinterpret_cast<const cT*>(tile + A::template box<G::LM_IN>(b_in, z_in, r * G::TPL));
      if constexpr (G::LM_IN != G::LM_OUT) {
        // the output box overlaps other warps' input lines: announce that
        // this warp's input values are in registers
        __syncwarp();
        if (lane == 0) red_add_release(&readers[s], 1u);
      }
      if (p.abft_in && valid) {
        real sr = 0, si = 0, en = 0;
#pragma unroll
        for (int r = 0; r < E; r++) {
          sr = fma(wv[r].x, v[r].x, sr); sr = fma(-wv[r].y, v[r].y, sr);
          si = fma(wv[r].x, v[r].y, si); si = fma(wv[r].y, v[r].x, si);
          en = fma(v[r].x, v[r].x, en); en = fma(v[r].y, v[r].y, en);
        }
        acc.s1r += sr; acc.s1i += si;
        acc.s2r = fma(wgt, sr, acc.s2r); acc.s2i = fma(wgt, si, acc.s2i);
        acc.en += en;
      }
      if (fst == -1) {
#pragma unroll
        for (int r = 0; r < E; r++)
          if (p.fault.index == j0 + r * G::TPL) v[r] = faulted(v[r], p.fault);
      }

      // ---------------- radix stages 0 .. S-2 (in place in the line scratch) ----------------
      if constexpr (G::S > 1) {
        Dft<E>::run(v);
        if (fst == 0) {
#pragma unroll
          for (int q = 0; q < E; q++)
            if (p.fault.index == j0 * E + q) v[q] = faulted(v[q], p.fault);
        }
        if constexpr (!G::WL) line_sync();   // the previous tile's last-stage reads are done
#pragma unroll
        for (int q = 0; q < E; q++) scr[s_wr0 + A::idx(q)] = v[q];
        line_sync();
#pragma unroll
        for (int st = 1; st < G::S - 1; st++) {
          const int Ns = v3_ipow(E, st);
#pragma unroll
          for (int r = 0; r < E; r++) v[r] = scr[s_rd + A::idx(r * G::TPL)];
          line_sync();                          // the whole line is read before it is overwritten
          const int kk = j0 % Ns;
          stage_twiddle<E>(v, tws, kk * (NSUB / (Ns * E)) * p.tw_sub_stride);
          Dft<E>::run(v);
          const int basei = (j0 / Ns) * Ns * E + kk;
          if (fst == st) {
#pragma unroll
            for (int q = 0; q < E; q++)
              if (p.fault.index == basei + q * Ns) v[q] = faulted(v[q], p.fault);
          }
          const int wb = scr_c + A::idx(basei);
#pragma unroll
          for (int q = 0; q < E; q++) scr[wb + A::idx(q * Ns)] = v[q];
          line_sync();
        }
        // last stage reads
#pragma unroll
        for (int ub = 0; ub < G::BPT; ub++)
#pragma unroll
          for (int r = 0; r < G::RL; r++)
            v[ub * G::RL + r] = scr[s_rd + A::idx(ub * G::TPL + r * G::NBL)];
      }

      // ---------------- last stage -> registers -> output box ----------------
      constexpr int NsL = G::NBL;   // E^(S-1)
#pragma unroll
      for (int ub = 0; ub < G::BPT; ub++) {
        cT* w = v + ub * G::RL;
        const int jl = j0 + ub * G::TPL;
        if constexpr (G::S > 1) stage_twiddle<G::RL>(w, tws, jl * (NSUB / (NsL * G::RL)) * p.tw_sub_stride);
        Dft<G::RL>::run(w);
        if (ROLE == V3_COLS && p.twiddle) {
          const cT base_t = twN<cT>(p, lo_c * (long long)jl * p.tw_scale);
          const cT step = twN<cT>(p, lo_c * (long long)G::NBL * p.tw_scale);
          cT f = base_t;
#pragma unroll
          for (int q = 0; q < G::RL; q++) {
            w[q] = c_mul(w[q], f);
            if (q + 1 < G::RL) f = c_mul(f, step);
          }
        }
        if (fst == G::S - 1) {
#pragma unroll
          for (int q = 0; q < G::RL; q++)
            if (p.fault.index == jl + q * G::NBL) w[q] = faulted(w[q], p.fault);
        }
        if (p.abft_out && valid) {
          real a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0;
#pragma unroll
          for (int q = 0; q < G::RL; q++) {
            const bool neg = (smask >> (ub * G::RL + q)) & 1u;
            const real yr = neg ? -w[q].x : w[q].x, yi = neg ? -w[q].y : w[q].y;
            if (q % 3 == 0) { a0r += yr; a0i += yi; }
            else if (q % 3 == 1) { a1r += yr; a1i += yi; }
            else { a2r += yr; a2i += yi; }
          }
          const int kz = (k0mask >> (2 * ub)) & 3;
          const real hr = (real)-0.5, hs = (real)0.86602540378443864676;
          const real s1 = (dl == 1) ? -hs : hs;
          real tr = a0r + (hr * a1r - s1 * a1i) + (hr * a2r + s1 * a2i);
          real ti = a0i + (hr * a1i + s1 * a1r) + (hr * a2i - s1 * a2r);
          if (kz == 1) { real x = hr * tr + hs * ti; ti = hr * ti - hs * tr; tr = x; }
          else if (kz == 2) { real x = hr * tr - hs * ti; ti = hr * ti + hs * tr; tr = x; }
          acc.t1r += tr; acc.t1i += ti;
          acc.t2r = fma(wgt, tr, acc.t2r); acc.t2i = fma(wgt, ti, acc.t2i);
          if (!(isfinite(tr) && isfinite(ti))) {
            acc.nf_min = min(acc.nf_min, (long long)b0);
            acc.nf_max = max(acc.nf_max, (long long)b0);
          }
        }
      }
      if constexpr (G::S == 1) line_sync();
      if constexpr (G::LM_IN != G::LM_OUT) {
        // every warp has read its input from the box before any output lands there
        if (lane == 0) {
          const unsigned want = 8u * (wrap + 1u);
          long long it = 0;
          while (ld_acquire(&readers[s]) < want) {
            if (++it >= kWaitLimit || ((it & 1023) == 0 && *abort_flag)) {
              *abort_flag = 1;
              atomicExch(p.err_flag, 1);
              break;
            }
          }
        }
        __syncwarp();
      }
#pragma unroll
      for (int ub = 0; ub < G::BPT; ub++)
#pragma unroll
        for (int q = 0; q < G::RL; q++)
          *reinterpret_cast<cT*>(tile + A::template box<G::LM_OUT>(b_out, z_out, ub * G::TPL + q * G::NBL)) =
              v[ub * G::RL + q];

      // hand the tile back: this warp's box writes become visible to the TMA
      // unit, the eighth warp to arrive stores the tile and refills the buffer
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        const unsigned old = atom_add_acq_rel(&arrivals[s], 1u);
        TileCursor& ld = ldc[warp];
        if (old == 8u * wrap + 7u && !*abort_flag) {
          issue_store(p, tb, se, hi, lo0, reinterpret_cast<const cT*>(tile));
          bulk_commit();
          if (ld.valid(p)) {
            bulk_wait_read_0();               // the store has read the buffer
            issue_load(p, ld, reinterpret_cast<cT*>(tile), &full[s]);
          }
        }
        ld.advance(p);
      }
      __syncwarp();
      if (++s == nbuf) { s = 0; wrap++; }
    }
    if (abft) {
      if constexpr (ROLE == V3_SINGLE) reduce_warp_and_store(acc, p, cur.g, slot0 + warp);
      else reduce_block_records(acc, p, cur.g, slot0, red);
    }
  }
  if (lane == 0) bulk_wait_0();
}

}  // namespace tfft
