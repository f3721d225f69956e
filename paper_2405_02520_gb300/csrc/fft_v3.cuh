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
//     exchange data through warp-private, padded ping-pong scratch with only
//     __syncwarp; longer lines (single pass, NSUB > 32 E) share a named
//     barrier among the warps of the line;
//   * one block barrier per tile, before the TMA store of the output box;
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
  static constexpr int SCR = C * PITCH;                     // scratch values per buffer
  static_assert(C >= 1 && TILE % NSUB == 0, "tile must hold whole lines");
  static_assert(WL || TPL % 32 == 0, "a line is held by whole warps");

  // byte offset of value (c, i) in the dense input / output box
  __device__ __forceinline__ static uint32_t box_off(bool lm, int c, int i) {
    if (lm) return (uint32_t)((c * NSUB + i) * ES);
    const uint32_t o = (uint32_t)(((c / CS) * NSUB + i) * ROWB + (c % CS) * ES);
    return o ^ (((o >> 7) & SWZ) << 4);   // TMA 128 / 64 / 32-byte swizzle pattern
  }
  __device__ __forceinline__ static int scr_idx(int c, int i) { return c * PITCH + i + i / PG; }
};

template <typename real, int NSUB, int E, int ROLE>
__global__ void __launch_bounds__(256, 1)
fft_v3_kernel(const __grid_constant__ PassParams p) {
  using G = V3<real, NSUB, E, ROLE>;
  using cT = typename G::cT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32 * 12];

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int nbuf = p.nbuf;
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nbuf * p.buf_bytes);
  cT* scr0 = reinterpret_cast<cT*>(base + (size_t)nbuf * p.buf_bytes + 1024);
  cT* scr1 = scr0 + G::SCR;
  auto box = [&](int s) { return base + (size_t)s * p.buf_bytes; };
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
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(1 + c0), "r"(32 * G::WPL) : "memory");
    }
  };

  if (t == 0) {
    for (int s = 0; s < nbuf; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
    if (blockIdx.x == 0) {
      if (p.zero_on_entry[0]) *p.zero_on_entry[0] = 0;
      if (p.zero_on_entry[1]) *p.zero_on_entry[1] = 0;
    }
  }
  __syncthreads();

  TileCursor prod;
  if (t == 0) {
    prod.start(p);
    for (int s = 0; s < nbuf - 1 && prod.valid(p); s++) {
      issue_load(p, prod, reinterpret_cast<cT*>(box(s)), &full[s]);
      prod.advance(p);
    }
  }

  cT wv[E];
  unsigned smask = 0;
  unsigned k0mask = 0;          // (k mod 3) of each last-stage butterfly, 2 bits each
  Partials<real> acc;
  bool setup_done = false;
  auto setup_positions = [&](long long hi, long long lo0) {
    if (p.abft_in) {
      const cT* wtab = reinterpret_cast<const cT*>(p.wtab);
      const long long lo = G::LM_IN && ROLE == V3_SINGLE ? 0 : lo0 + c0;
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

  int k = 0;
  for (long long chunk = blockIdx.x; chunk < p.nchunks; chunk += gridDim.x) {
    TileCursor cur;
    cur.chunk = chunk;
    const bool nonempty = cur.decode(p);
    const long long slot0 = (long long)(cur.part * p.line_blocks + cur.lb) * (ROLE == V3_SINGLE ? 8 : 1);
    if (!nonempty) {
      if (abft && !p.list) {
        acc.zero();
        if constexpr (ROLE == V3_SINGLE) reduce_warp_and_store(acc, p, cur.g, slot0 + warp);
        else reduce_and_store(acc, p, cur.g, slot0, red);
      }
      continue;
    }
    const long long hi = cur.hi(p), lo0 = cur.lo0(p);
    if (ROLE != V3_SINGLE || !setup_done) {
      setup_positions(hi, lo0);
      setup_done = true;
    }
    if (abft) acc.zero();
    const long long gb = cur.gb, se = cur.se;

    for (long long tb = cur.sb; tb < se; tb += (ROLE == V3_SINGLE ? G::C : 1), k++) {
      const int s = k % nbuf;
      const uint32_t parity = (uint32_t)((k / nbuf) & 1);
      unsigned char* tile = box(s);
      {
        bool ok = false;
        for (long long it = 0; it < kWaitLimit && !ok; it++) ok = mbar_try_wait(&full[s], parity);
        if (__syncthreads_or(!ok)) {
          if (t == 0) {
            atomicExch(p.err_flag, 1);
            bulk_wait_0();
          }
          return;
        }
      }
      const long long b0 = (ROLE == V3_SINGLE) ? tb + c0 : tb;     // this thread's signal
      const bool valid = b0 < se;
      const long long lo_c = (ROLE == V3_SINGLE) ? 0 : lo0 + c0;
      const long long line_c = (ROLE == V3_SINGLE) ? 0 : hi * p.LO + lo_c;

      // ---------------- stage 0: box -> registers ----------------
      cT v[E];
#pragma unroll
      for (int r = 0; r < E; r++)
        v[r] = *reinterpret_cast<const cT*>(tile + G::box_off(G::LM_IN, c0, j0 + r * G::TPL));
      if (p.abft_in && valid) {
        real sr = 0, si = 0, en = 0;
#pragma unroll
        for (int r = 0; r < E; r++) {
          sr = fma(wv[r].x, v[r].x, sr); sr = fma(-wv[r].y, v[r].y, sr);
          si = fma(wv[r].x, v[r].y, si); si = fma(wv[r].y, v[r].x, si);
          en = fma(v[r].x, v[r].x, en); en = fma(v[r].y, v[r].y, en);
        }
        const real wgt = (real)(b0 - gb + 1);
        acc.s1r += sr; acc.s1i += si;
        acc.s2r = fma(wgt, sr, acc.s2r); acc.s2i = fma(wgt, si, acc.s2i);
        acc.en += en;
      }
      if (inject && p.fault.stage == -1 && valid && fault_signal(p.fault, b0) && p.fault.line == line_c) {
#pragma unroll
        for (int r = 0; r < E; r++)
          if (p.fault.index == j0 + r * G::TPL) v[r] = faulted(v[r], p.fault);
      }

      // ---------------- radix stages 0 .. S-2 (shared scratch) ----------------
      if constexpr (G::S > 1) {
        Dft<E>::run(v);
#pragma unroll
        for (int q = 0; q < E; q++) {
          const int i = j0 * E + q;
          if (inject && p.fault.stage == 0 && valid && fault_signal(p.fault, b0) && p.fault.line == line_c &&
              p.fault.index == i)
            v[q] = faulted(v[q], p.fault);
          scr0[G::scr_idx(c0, i)] = v[q];
        }
        line_sync();
#pragma unroll
        for (int st = 1; st < G::S - 1; st++) {
          const int Ns = v3_ipow(E, st);
          const cT* src = (st & 1) ? scr0 : scr1;
          cT* dst = (st & 1) ? scr1 : scr0;
#pragma unroll
          for (int r = 0; r < E; r++) v[r] = src[G::scr_idx(c0, j0 + r * G::TPL)];
          const int kk = j0 % Ns;
          stage_twiddle<E>(v, tws, kk * (NSUB / (Ns * E)) * p.tw_sub_stride);
          Dft<E>::run(v);
          const int basei = (j0 / Ns) * Ns * E + kk;
#pragma unroll
          for (int q = 0; q < E; q++) {
            const int i = basei + q * Ns;
            if (inject && p.fault.stage == st && valid && fault_signal(p.fault, b0) && p.fault.line == line_c &&
                p.fault.index == i)
              v[q] = faulted(v[q], p.fault);
            dst[G::scr_idx(c0, i)] = v[q];
          }
          line_sync();
        }
      }

      // ---------------- last stage -> registers -> output box ----------------
      cT u[E];
      if constexpr (G::S > 1) {
        const cT* src = ((G::S - 1) & 1) ? scr0 : scr1;
#pragma unroll
        for (int ub = 0; ub < G::BPT; ub++)
#pragma unroll
          for (int r = 0; r < G::RL; r++)
            u[ub * G::RL + r] = src[G::scr_idx(c0, j0 + ub * G::TPL + r * G::NBL)];
      } else {
#pragma unroll
        for (int r = 0; r < E; r++) u[r] = v[r];
      }
      constexpr int NsL = G::NBL;   // E^(S-1)
#pragma unroll
      for (int ub = 0; ub < G::BPT; ub++) {
        cT* w = u + ub * G::RL;
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
        if (inject && p.fault.stage == G::S - 1 && valid && fault_signal(p.fault, b0) && p.fault.line == line_c) {
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
          const real wgt = (real)(b0 - gb + 1);
          acc.t1r += tr; acc.t1i += ti;
          acc.t2r = fma(wgt, tr, acc.t2r); acc.t2i = fma(wgt, ti, acc.t2i);
          if (!(isfinite(tr) && isfinite(ti))) {
            acc.nf_min = min(acc.nf_min, (long long)b0);
            acc.nf_max = max(acc.nf_max, (long long)b0);
          }
        }
      }
      if constexpr (G::S == 1 || !G::WL) line_sync();   // the box is still read by this line's threads
#pragma unroll
      for (int ub = 0; ub < G::BPT; ub++)
#pragma unroll
        for (int q = 0; q < G::RL; q++)
          *reinterpret_cast<cT*>(tile + G::box_off(G::LM_OUT, c0, j0 + ub * G::TPL + q * G::NBL)) =
              u[ub * G::RL + q];
      fence_proxy_async();
      __syncthreads();
      if (t == 0) {
        issue_store(p, tb, se, hi, lo0, reinterpret_cast<const cT*>(tile));
        bulk_commit();
        bulk_wait_read_1();
        if (prod.valid(p)) {
          const int sp = (k + nbuf - 1) % nbuf;
          issue_load(p, prod, reinterpret_cast<cT*>(box(sp)), &full[sp]);
          prod.advance(p);
        }
      }
    }
    if (abft) {
      if constexpr (ROLE == V3_SINGLE) reduce_warp_and_store(acc, p, cur.g, slot0 + warp);
      else reduce_and_store(acc, p, cur.g, slot0, red);
    }
  }
  if (t == 0) bulk_wait_0();
}

}  // namespace tfft
