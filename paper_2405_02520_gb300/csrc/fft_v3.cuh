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
#include "sigverify.cuh"
#include "fusedfix.cuh"
#include "tc.cuh"

namespace tfft {

enum V3Role : int { V3_SINGLE = 0, V3_COLS = 1, V3_LAST = 2 };

__host__ __device__ constexpr int v3_stages(int nsub, int e) {
  int s = 0;
  long long v = 1;
  while (v < nsub) { v *= e; s++; }
  return s < 1 ? 1 : s;
}
__host__ __device__ constexpr int v3_ipow(int b, int k) { return k == 0 ? 1 : b * v3_ipow(b, k - 1); }
// Entries of the stage-twiddle table: stages 1 .. S-1 (radix e, Ns = R0 e^(st-1))
// each hold omega_{Ns e}^(q kk) for q = 1 .. e-1, kk < Ns, as [q-1][kk].
__host__ __device__ constexpr int v3_tw_entries(int nsub, int e) {
  const int s = v3_stages(nsub, e), r0 = nsub / v3_ipow(e, s - 1);
  int n = 0;
  for (int st = 1; st < s; st++) n += (e - 1) * r0 * v3_ipow(e, st - 1);
  return n;
}
__host__ __device__ constexpr int v3_tw_offset(int nsub, int e, int stage) {
  const int s = v3_stages(nsub, e), r0 = nsub / v3_ipow(e, s - 1);
  int n = 0;
  for (int st = 1; st < stage; st++) n += (e - 1) * r0 * v3_ipow(e, st - 1);
  return n;
}
// The table is staged in shared memory when it takes at most this many bytes.
constexpr int kV3TwSmemMax = 8192;

template <typename real, int NSUB, int E, int ROLE, int NT = 256>
struct V3 {
  using cT = typename Cplx<real>::T;
  static constexpr int ES = (int)sizeof(cT);                // 8 or 16 bytes
  static constexpr int NSUBV = NSUB;
  static constexpr int T = NT;                              // threads per block
  static constexpr int NW = NT / 32;                        // warps per block
  static constexpr int TILE = T * E;                        // values per tile
  static constexpr int C = TILE / NSUB;                     // lines per tile
  static constexpr int TPL = NSUB / E;                      // threads per line
  static constexpr bool WL = TPL <= 32;                     // warp-local lines
  static constexpr int LPW = WL ? 32 / TPL : 1;             // lines per warp
  static constexpr int WPL = WL ? 1 : TPL / 32;             // warps per line
  static constexpr int S = v3_stages(NSUB, E);              // radix stages
  static constexpr int R0 = NSUB / v3_ipow(E, S - 1);       // radix of stage 0; later stages radix E
  static constexpr int BPT0 = E / R0;                       // stage-0 butterflies per thread
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
  static constexpr int TWN = v3_tw_entries(NSUB, E);        // stage-twiddle table entries
  static constexpr bool TWS = TWN * ES <= kV3TwSmemMax;     // ... staged in shared memory
  static_assert(C >= 1 && TILE % NSUB == 0, "tile must hold whole lines");
  static_assert(WL || TPL % 32 == 0, "a line is held by whole warps");
  static_assert(S >= 2, "at least two radix stages");
  // scratch offsets split into a per-thread base and a compile-time part
  // (idx(x) = x + x / PG is additive over these splits; see V3Addr)
  static constexpr bool SPLIT0 = (TPL * R0) % PG == 0 && PG % R0 == 0;

};

__device__ __forceinline__ uint32_t atom_add_acq_rel(unsigned* a, unsigned v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(a)), "r"(v)
               : "memory");
  return old;
}


// Bounded wait on an mbarrier phase (at most `limit` polls); gives up early
// once another warp has recorded a timeout in *abort.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort,
                                                  long long limit = kWaitLimit) {
  for (long long it = 0; it < limit; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort && (it & 1023) == 1023 && *abort) return false;
  }
  return false;
}

// One warp's checksum record (single pass): the nine partial sums are
// reduced by recursive halving -- at each of four shuffle rounds a lane keeps
// half of its values and receives its partner's copy of them -- and a last
// exchange completes the sums, so lane L ends with the warp total of value
// idx(L) = 5 b4 + 3 b3 + 2 b2 + b1 (b_k = bit k of L; a few lanes hold a
// padding value).  Twelve shuffles instead of 45; every lane that holds a
// value writes its word of the record.  The nonfinite range is reduced only
// when some lane has one.
template <typename real>
__device__ __forceinline__ void warp_records(const Partials<real>& a, const PassParams& p, long long g,
                                             long long slot) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const real v[10] = {a.s1r, a.s1i, a.s2r, a.s2i, a.en, a.t1r, a.t1i, a.t2r, a.t2i, (real)0};
  const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4, h1 = lane & 2;
  real u[6];
#pragma unroll
  for (int i = 0; i < 5; i++)
    u[i] = (h4 ? v[i + 5] : v[i]) + __shfl_xor_sync(full, h4 ? v[i] : v[i + 5], 16);
  u[5] = (real)0;
  real w[4];
#pragma unroll
  for (int i = 0; i < 3; i++)
    w[i] = (h3 ? u[i + 3] : u[i]) + __shfl_xor_sync(full, h3 ? u[i] : u[i + 3], 8);
  w[3] = (real)0;
  real x[2];
#pragma unroll
  for (int i = 0; i < 2; i++)
    x[i] = (h2 ? w[i + 2] : w[i]) + __shfl_xor_sync(full, h2 ? w[i] : w[i + 2], 4);
  real y = (h1 ? x[1] : x[0]) + __shfl_xor_sync(full, h1 ? x[0] : x[1], 2);
  y += __shfl_xor_sync(full, y, 1);
  const int r1 = (h3 ? 3 : 0) + (h2 ? 2 : 0) + (h1 ? 1 : 0);
  const int idx = (h4 ? 5 : 0) + r1;
  const bool holds = !(lane & 1) && !(h2 && h1) && !(h3 && h2) && idx < 9;

  long long mn = a.nf_min, mx = a.nf_max;
  if (__any_sync(full, mx >= 0)) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      mn = min(mn, __shfl_xor_sync(full, mn, off));
      mx = max(mx, __shfl_xor_sync(full, mx, off));
    }
  }
  if (holds) {
    if (idx < 5) {
      if (p.abft_in) reinterpret_cast<double*>(p.rec_in + g * p.slots + slot)[idx] = (double)y;
    } else if (p.abft_out) {
      reinterpret_cast<double*>(p.rec_out + g * p.slots + slot)[idx - 5] = (double)y;
    }
  }
  if (p.abft_out && lane == 1) {
    RecOut* r = p.rec_out + g * p.slots + slot;
    r->nf_min = mn;
    r->nf_max = mx;
  }
}

// Last-pass records with the second check: [r^T y | r2^T y, u2^T z] of the
// warp's share of the tile, one SigOut and one SigChk record per (signal, slot).
template <typename real>
__device__ __forceinline__ void sig_flush_chk(const Partials<real>& a, const PassParams& p, long long sig,
                                              long long slot);

// Recursive halving over the lanes of a shuffle group: with V values held
// and the next exchange at lane distance OFF, a lane keeps the half of its
// values selected by its bit OFF and adds its partner's copy of that half;
// once one value is left the remaining distances complete its sum.  Every
// lane ends with the group total of value `idx`.
template <typename real, int V, int OFF>
struct Halve {
  __device__ __forceinline__ static void run(real* v, int lane, int& idx) {
    if constexpr (OFF >= 1) {
      if constexpr (V > 1) {
        constexpr int H = V / 2;
        const bool up = lane & OFF;
#pragma unroll
        for (int i = 0; i < H; i++) {
          const real keep = up ? v[i + H] : v[i];
          const real send = up ? v[i] : v[i + H];
          v[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
        }
        if (up) idx += H;
        Halve<real, H, OFF / 2>::run(v, lane, idx);
      } else {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], OFF);
        Halve<real, 1, OFF / 2>::run(v, lane, idx);
      }
    }
  }
};

// Per-signal records of one tile: the W consecutive lanes that hold one
// signal's values in this tile (W = the lanes of a line in the single pass,
// the whole warp otherwise) reduce their partial sums -- w^T x and ||x||^2 on
// the input side, r^T y on the output side -- and write them as the record of
// (signal `sig`, slot `slot`).  Every lane of the warp calls this; only lanes
// of a valid signal write.
template <typename real, int W, bool IN, bool OUT>
__device__ __forceinline__ void sig_flush(const Partials<real>& a, const PassParams& p, long long sig,
                                          long long slot, bool valid) {
  constexpr int V = (IN && OUT) ? 8 : (IN ? 4 : 2);
  static_assert(V <= W, "a record's values fit the lanes that reduce them");
  real v[V];
  if constexpr (IN && OUT) {
    v[0] = a.s1r; v[1] = a.s1i; v[2] = a.en; v[3] = (real)0;
    v[4] = a.t1r; v[5] = a.t1i; v[6] = (real)0; v[7] = (real)0;
  } else if constexpr (IN) {
    v[0] = a.s1r; v[1] = a.s1i; v[2] = a.en; v[3] = (real)0;
  } else {
    v[0] = a.t1r; v[1] = a.t1i;
  }
  const int lane = threadIdx.x & 31;
  int idx = 0;
  Halve<real, V, W / 2>::run(v, lane, idx);
  if (!valid || (lane & (W / V - 1))) return;
  if constexpr (IN) {
    if (idx < 3) reinterpret_cast<real*>(reinterpret_cast<SigIn<real>*>(p.sig_in) + sig * p.sig_slots + slot)[idx] = v[0];
  }
  if constexpr (OUT) {
    constexpr int O = IN ? 4 : 0;
    if (idx >= O && idx < O + 2)
      reinterpret_cast<real*>(reinterpret_cast<SigOut<real>*>(p.sig_out) + sig * p.sig_slots + slot)[idx - O] = v[0];
  }
}

template <typename real>
__device__ __forceinline__ void sig_flush_chk(const Partials<real>& a, const PassParams& p, long long sig,
                                              long long slot) {
  real v[8] = {a.t1r, a.t1i, (real)0, (real)0, a.t2r, a.t2i, a.s2r, a.s2i};
  const int lane = threadIdx.x & 31;
  int idx = 0;
  Halve<real, 8, 16>::run(v, lane, idx);
  if (lane & 3) return;
  if (idx < 2)
    reinterpret_cast<real*>(reinterpret_cast<SigOut<real>*>(p.sig_out) + sig * p.sig_slots + slot)[idx] = v[0];
  else if (idx >= 4)
    reinterpret_cast<real*>(reinterpret_cast<SigChk<real>*>(p.sig_chk) + sig * p.sig_slots + slot)[idx - 4] = v[0];
}

// The chunks of one thread block and their tiles, as TileCursor, for the v3
// kernels (never a work list): C, LO and the line-block count are powers of
// two, so the decomposition is shifts and masks except for the split of a
// group into parts, and the one-part, one-line-block cases skip even that.
struct V3Cursor {
  long long tb, gb, sb, se;
  long long chunk;
  long long cstep, cend;        // the block's chunk schedule: chunk, chunk + cstep, ... below cend
  unsigned lb, part, g;
  __device__ __forceinline__ bool decode(const PassParams& p) {
    const unsigned c = (unsigned)chunk;
    unsigned rest = c;
    lb = 0;
    if (p.log2LB) { rest = c >> p.log2LB; lb = c & ((1u << p.log2LB) - 1u); }
    part = 0;
    g = rest;
    if (p.parts != 1) { g = rest / (unsigned)p.parts; part = rest - g * (unsigned)p.parts; }
    gb = (long long)g * p.group;
    const long long ge = min((long long)p.batch, gb + (long long)p.group);
    if (p.parts == 1) {
      sb = gb;
      se = ge;
    } else {
      const int lu = p.lines_are_signals ? p.log2C : 0;
      const unsigned ntiles = (unsigned)((ge - gb + (1ll << lu) - 1) >> lu);
      const unsigned per = (ntiles + (unsigned)p.parts - 1u) / (unsigned)p.parts;
      sb = gb + ((long long)(part * per) << lu);
      se = min(ge, sb + ((long long)per << lu));
    }
    return sb < se;
  }
  __device__ __forceinline__ void settle(const PassParams& p) {
    while (chunk < cend) {
      if (decode(p)) { tb = sb; return; }
      chunk += cstep;
    }
  }
  __device__ __forceinline__ void start(const PassParams& p, long long first, long long step, long long end) {
    chunk = first;
    cstep = step;
    cend = end;
    settle(p);
  }
  __device__ __forceinline__ bool valid(const PassParams&) const { return chunk < cend; }
  __device__ __forceinline__ void advance(const PassParams& p) {
    tb += p.lines_are_signals ? p.C : 1;
    if (tb >= se) { chunk += cstep; settle(p); }
  }
  __device__ __forceinline__ long long hi(const PassParams& p) const {
    return p.lines_are_signals ? 0 : ((long long)lb << p.log2C) >> p.log2LO;
  }
  __device__ __forceinline__ long long lo0(const PassParams& p) const {
    return p.lines_are_signals ? 0 : ((long long)lb << p.log2C) & ((1ll << p.log2LO) - 1);
  }
};

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

// Copies rows [r_begin, r_end) of a finished last-pass tile from its
// shared-memory box to the output, one warp, 16 bytes a lane per access.  The
// box is laid out as the TMA would store it: element-major rows of ROWB bytes
// in column groups of CS lines with the TMA swizzle (row i of group gx holds
// element i of lines lo0 + gx CS .. + CS - 1, which are adjacent in memory).
// Plain loads and stores leave nothing in flight that still reads the box, so
// the buffer can be refilled right after.  (The single and column passes
// store their tiles by TMA.)
template <typename G, int ROLE>
__device__ __forceinline__ void copy_out(const PassParams& p, long long tb, long long se, long long hi,
                                         long long lo0, const unsigned char* tile, int lane, int r_begin = 0,
                                         int r_end = G::NSUBV) {
  static_assert(ROLE == V3_LAST, "the last pass copies its tiles out");
  (void)se;
  unsigned char* out = reinterpret_cast<unsigned char*>(p.out);
  {
    constexpr int CPR = G::ROWB / 16;           // 16-byte chunks per box row
    constexpr int RPI = 32 / CPR;               // rows per warp access
    static_assert(G::ROWB % 16 == 0 && CPR <= 32, "box rows are whole 16-byte chunks");
    const int j = lane % CPR, rr = lane / CPR;
    const long long row_stride = p.out_es * G::ES;
#pragma unroll 1
    for (int gx = 0; gx < G::C / G::CS; gx++) {
      const long long sbase = p.soff_out ? p.soff_out[tb] : tb * p.n;
      unsigned char* dst = out + (sbase + hi * p.out_hi + (lo0 + gx * G::CS) * p.out_lo) * G::ES +
                           rr * row_stride + 16 * j;
      const uint32_t o0 = (uint32_t)((gx * G::NSUBV + rr) * G::ROWB + 16 * j);
#pragma unroll 4
      for (int r0 = r_begin; r0 < r_end; r0 += RPI) {
        const uint32_t o = o0 + (uint32_t)(r0 * G::ROWB);
        const float4 v = *reinterpret_cast<const float4*>(tile + (o ^ (((o >> 7) & G::SWZ) << 4)));
        __stcs(reinterpret_cast<float4*>(dst + (long long)r0 * row_stride), v);
      }
    }
  }
}

// The tensor-core forms whose A operands (the rows of the butterflies) fit in
// the line scratch and are placed there: split BF16 (64-byte rows, high and
// low, 16 KB a warpgroup) and plain TF32 (128-byte rows, 16 KB a warpgroup).
// Their blocks take no more shared memory than the FP32 kernel, so two run
// per SM; the split-TF32 form keeps separate operands and one block per SM.
__host__ __device__ constexpr bool v3_tc_aliased(int tc) { return tc == 1 || tc == 2; }

// Shared memory of the tensor-core operands: per warpgroup the A rows (high,
// and low for the split form) of its 128 butterflies unless they sit in the
// line scratch, and the DFT-16 matrix (high and low); 1024-byte aligned.
__host__ __device__ constexpr int v3_tc_smem_bytes(int tc) {
  // B: 32 rows of 64 bytes (BF16) or 128 bytes (TF32), high and (split forms) low
  return tc == 0 ? 0 : tc == 2 ? 1024 + 2 * 2048 : tc == 1 ? 1024 + 4096 : 1024 + 2 * 2 * 16384 + 2 * 4096;
}

// Blocks per SM the register budget targets: two for complex64 (at most 128
// registers a thread), one for complex128, whose values take twice the registers.
template <typename real>
constexpr int v3_min_blocks() { return sizeof(real) == 4 ? 2 : 1; }
template <typename real, int TC>
constexpr int v3_min_blocks_tc() { return TC == 0 ? v3_min_blocks<real>() : (v3_tc_aliased(TC) ? 2 : 1); }

// NT = 256 threads (eight warps), two blocks per SM for complex64; the wide
// form, NT = 512 (sixteen warps, one block per SM), takes tiles of 8192
// complex64 values so that column and last passes of 512 to 2048 points keep
// 32- to 128-byte rows.  Thread 0 starts the first
// nbuf tile loads; afterwards the last warp to finish a tile stores it and
// refills its buffer with the tile nbuf ahead, so no warp waits for another
// except on data that has not arrived yet.
//
// TC != 0 (complex64, E = 16): every radix-16 butterfly is a row of a dense
// 128 x 32 x 32 real product on the tensor cores -- the 16 complex inputs of
// a butterfly interleaved (re, im) times the real 32 x 32 form of the DFT-16
// matrix -- one product per warpgroup and stage, the accumulator in tensor
// memory; TC = 1 multiplies TF32-rounded operands, TC = 3 the three-term
// split (x_hi w_hi + x_hi w_lo + x_lo w_hi) that keeps about 21 bits.
//
// The block's own state (load cursors, tile counters, the timeout flag, the
// tensor-core barriers), in static shared memory of the calling kernel: one
// copy per block whatever the bodies it runs.
template <int NW>
struct V3Smem {
  V3Cursor ldc[NW];        // per warp: the next tile to load
  unsigned arrivals[8];    // per buffer: warps done with the tile, cumulative
  unsigned copied[8];      // per buffer: warps done copying the tile out (last pass), cumulative
  unsigned issued[8];      // per buffer: tile loads issued into it, cumulative
  int s_abort;
  uint64_t tcbar[2];
  uint32_t tc_tmem;
};

// The body runs the chunks cfirst, cfirst + cstep, ... below cend of the pass
// (the kernel: the grid-stride share of its block); zero_entry marks the one
// block that resets the plan's per-exec lists.  It may run again in the same
// block for another pass (the persistent ragged kernels): it starts and ends
// at a block barrier, fences generic writes to its buffers before the first
// tile copies into them, and invalidates its tile barriers before it returns.
// Returns true when a bounded wait gave up (the block must not run another
// body then: a copy may still be in flight into its buffers).
template <typename real, int NSUB, int E, int ROLE, int TC = 0, int NT = 256>
__device__ __forceinline__ bool v3_body(const PassParams& p, long long cfirst, long long cstep, long long cend,
                                        bool zero_entry, V3Smem<NT / 32>& vs) {
  static_assert(TC == 0 || (sizeof(real) == 4 && E == 16 && NT == 256), "tensor-core DFT: complex64, radix 16");
  static_assert(NT == 256 || NT == 512, "eight or sixteen warps");
  using G = V3<real, NSUB, E, ROLE, NT>;
  constexpr bool TCA = v3_tc_aliased(TC);
  constexpr bool BOXA = TCA && ROLE == V3_SINGLE && G::C == 1;
  static_assert(!TCA || 2 * 16384 <= G::SCR * G::ES, "tensor-core operands fit in the line scratch");
  static_assert(!TCA || G::C < 2 || ((G::C / 2) * G::PITCH * G::ES >= 16384 && ((G::C / 2) * G::PITCH * G::ES) % 1024 == 0),
                "a warpgroup's operands fit over its own lines' scratch, 1024-byte aligned");
  using A = V3Addr<G>;
  using cT = typename G::cT;
  static_assert(E % G::PG == 0, "a thread's stage-0 values start on a pad group");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V3Cursor* ldc = vs.ldc;
  unsigned* arrivals = vs.arrivals;
  unsigned* copied = vs.copied;
  unsigned* issued = vs.issued;
  int& s_abort = vs.s_abort;

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const int nbuf = p.nbuf;
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nbuf * p.buf_bytes);
  cT* scr = reinterpret_cast<cT*>(base + (size_t)nbuf * p.buf_bytes + 1024);
  volatile int* abort_flag = &s_abort;

  // stage twiddles: from the plan's table, staged next to the scratch when small
  const cT* twt = reinterpret_cast<const cT*>(p.tw_stage);
  auto stage_twiddles = [&] {
    if constexpr (G::TWS) {
      cT* tsm = scr + G::SCR;
      for (int i = t; i < G::TWN; i += G::T) tsm[i] = twt[i];
    }
  };
  if (t == 0) {
    for (int s = 0; s < nbuf; s++) {
      mbar_init(&full[s], 1);
      arrivals[s] = 0;
      copied[s] = 0;
      issued[s] = 0;
    }
    fence_mbar_init();
    s_abort = 0;
  }
  if (p.pdl) {
    // a programmatic dependent: the table (a plan constant) while the kernel
    // before it finishes, then wait for it before any global write or load
    stage_twiddles();
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  if (t == 0 && zero_entry) {
    if (p.zero_on_entry[0]) *p.zero_on_entry[0] = 0;
    if (p.zero_on_entry[1]) *p.zero_on_entry[1] = 0;
    if (p.zero_on_entry[2]) *p.zero_on_entry[2] = 0;
  }
  __syncthreads();
  if (t == 0) {
    V3Cursor ld;
    ld.start(p, cfirst, cstep, cend);
    fence_proxy_async();                // generic writes to the buffers before the tile copies land
    for (int s = 0; s < nbuf && ld.valid(p); s++) {
      issue_load(p, ld, reinterpret_cast<cT*>(base + (size_t)s * p.buf_bytes), &full[s]);
      issued[s]++;
      ld.advance(p);
    }
    for (int w = 0; w < G::NW; w++) ldc[w] = ld;
  }
  if (!p.pdl) stage_twiddles();
  if constexpr (G::TWS) twt = scr + G::SCR;
  // tensor-core operands and accumulator (TC != 0)
  uint64_t* tcbar = vs.tcbar;
  uint32_t& tc_tmem = vs.tc_tmem;
  unsigned char* tc_a = nullptr;      // per warpgroup: A high [, A low], 16 KB in all
  unsigned char* tc_b = nullptr;      // DFT-16 matrix, transposed: high [, low]
  if constexpr (TC != 0) {
    const uintptr_t after = reinterpret_cast<uintptr_t>(scr + G::SCR + (G::TWS ? G::TWN : 0));
    const uintptr_t al = (after + 1023) & ~uintptr_t(1023);
    if constexpr (TCA) {
      tc_a = reinterpret_cast<unsigned char*>(scr);     // 1024-byte aligned (the tile buffers are)
      tc_b = reinterpret_cast<unsigned char*>(al);
    } else {
      tc_a = reinterpret_cast<unsigned char*>(al);
      tc_b = tc_a + 2 * 2 * 16384;
    }
    if (t < 32) {
      // row n of B^T = column n of the real 32 x 32 DFT-16 matrix W:
      // W[2j][2m] = W[2j+1][2m+1] = cos(2 pi jm/16), W[2j][2m+1] = -W[2j+1][2m] = -sin(2 pi jm/16)
      const int m = t >> 1, im = t & 1;
      auto wval = [&](int kk) -> float {
        const int j = kk >> 1, kim = kk & 1;
        const int q = (j * m) & 15;
        const double cs = Eighths::cosv(q), sn = -Eighths::sinv(q);
        return (float)(kim == im ? cs : (kim ? -sn : sn));
      };
      if constexpr (TC == 2) {
        // BF16: 32 values = one 64-byte row (64-byte swizzle), high then low
#pragma unroll
        for (int c = 0; c < 4; c++) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; e++) tc::split_bf16x2(wval(8 * c + 2 * e), wval(8 * c + 2 * e + 1), h[e], l[e]);
          *reinterpret_cast<uint4*>(tc_b + tc::sw64_off(t, c)) = uint4{h[0], h[1], h[2], h[3]};
          *reinterpret_cast<uint4*>(tc_b + 2048 + tc::sw64_off(t, c)) = uint4{l[0], l[1], l[2], l[3]};
        }
      } else {
#pragma unroll
        for (int c = 0; c < 8; c++) {
          float w[4];
#pragma unroll
          for (int e = 0; e < 4; e++) w[e] = wval(4 * c + e);
          const float4 h = {tc::to_tf32(w[0]), tc::to_tf32(w[1]), tc::to_tf32(w[2]), tc::to_tf32(w[3])};
          *reinterpret_cast<float4*>(tc_b + tc::sw128_off(t, c)) = h;
          if constexpr (TC == 3) {
            const float4 l = {tc::to_tf32(w[0] - h.x), tc::to_tf32(w[1] - h.y), tc::to_tf32(w[2] - h.z),
                              tc::to_tf32(w[3] - h.w)};
            *reinterpret_cast<float4*>(tc_b + 4096 + tc::sw128_off(t, c)) = l;
          }
        }
      }
    }
    fence_proxy_async();
    if (warp == 0) tc::tmem_alloc(&tc_tmem, 64);
    if (t == 0) {
      mbar_init(&tcbar[0], 1);
      mbar_init(&tcbar[1], 1);
      fence_mbar_init();
    }
    tc::fence_before_sync();
  }
  __syncthreads();
  if constexpr (TC != 0) tc::fence_after_sync();
  uint32_t tc_phase = 0;

  const bool abft = p.abft_in || p.abft_out;
  bool inject = false;     // a fault site is armed for this pass
  for (int q = 0; q < p.nfault && q < 4; q++) {
    const FaultSite& f = q == 0 ? p.fault : p.fault_more[q - 1];
    inject |= f.mode != 0 && f.pass == p.pass_index;
  }

  // this thread's line and butterfly index inside the tile
  const int c0 = G::WL ? warp * G::LPW + lane / G::TPL : warp / G::WPL;
  const int j0 = G::WL ? lane % G::TPL : (warp % G::WPL) * 32 + lane;

  // All warps of the block at one point of the same tile (the last pass's
  // two box hand-overs): a hardware barrier, on which waiting warps take no
  // issue slots.  Every warp runs the same sequence of tiles, also after a
  // timed-out wait, so each barrier is reached by all of them.
  auto tile_sync = [&]() { asm volatile("bar.sync 15, %0;" ::"n"(G::T) : "memory"); };

  auto line_sync = [&]() {
    if constexpr (G::WL) {
      __syncwarp();
    } else if constexpr (G::WPL * 32 == G::T) {
      asm volatile("bar.sync 1, %0;" ::"n"(G::T) : "memory");
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(2 + c0), "r"(32 * G::WPL) : "memory");
    }
  };

  // The radix-16 DFT of this thread's 16 values: register butterflies, or
  // this thread's row of its warpgroup's tensor-core product.
  // kind: 0 the first stage, 1 a middle stage (its reads ended by a line
  // barrier), 2 the last stage; box: the current tile's buffer
  auto dft16 = [&](cT* v, int kind, unsigned char* box) {
    if constexpr (TC == 0) {
      Dft<E>::run(v);
    } else {
      const int wg = warp >> 2, row = t & 127;
      // split BF16: 8 KB of high and 8 KB of low rows a warpgroup; TF32: 16 KB
      // of rows (plain) or 16 KB high and 16 KB low (split).  In the line
      // scratch, a warpgroup whose lines are its own (two or more lines a
      // tile) puts them over its own lines' scratch; one line a tile (shared
      // by both warpgroups) the two take the first 32 KB.
      // A single-pass tile of one line: after the first stage has read the
      // tile's buffer, the later stages put their operands there (the
      // output is written to it only after the last product), which spares
      // the barriers around the line scratch.
      const bool in_box = BOXA && kind != 0;
      unsigned char* ahi = TCA && G::C >= 2 ? tc_a + wg * (G::C / 2) * G::PITCH * G::ES
                                            : (in_box ? box : tc_a) + wg * (TC == 3 ? 2 : 1) * 16384;
      unsigned char* alo = ahi + (TC == 2 ? 8192 : 16384);
      // the threads that read or write the scratch the operands overlay
      auto overlay_sync = [&]() {
        if constexpr (G::C >= 2) asm volatile("bar.sync %0, 128;" ::"r"(8 + wg) : "memory");
        else asm volatile("bar.sync 1, 256;" ::: "memory");
      };
      if constexpr (TCA) {
        // the operands overwrite the line scratch: every thread that uses it
        // has read its values of this stage (and of the previous tile's last
        // stage) from it
        if (!in_box) overlay_sync();
      }
      if constexpr (TC == 2) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
          uint32_t h[4], l[4];
#pragma unroll
          for (int e = 0; e < 2; e++) {
            tc::split_bf16x2(v[4 * c + 2 * e].x, v[4 * c + 2 * e].y, h[2 * e], l[2 * e]);
            tc::split_bf16x2(v[4 * c + 2 * e + 1].x, v[4 * c + 2 * e + 1].y, h[2 * e + 1], l[2 * e + 1]);
          }
          *reinterpret_cast<uint4*>(ahi + tc::sw64_off(row, c)) = uint4{h[0], h[1], h[2], h[3]};
          *reinterpret_cast<uint4*>(alo + tc::sw64_off(row, c)) = uint4{l[0], l[1], l[2], l[3]};
        }
      } else {
#pragma unroll
        for (int c = 0; c < 8; c++) {
          const float4 q = {v[2 * c].x, v[2 * c].y, v[2 * c + 1].x, v[2 * c + 1].y};
          const float4 h = {tc::to_tf32(q.x), tc::to_tf32(q.y), tc::to_tf32(q.z), tc::to_tf32(q.w)};
          *reinterpret_cast<float4*>(ahi + tc::sw128_off(row, c)) = h;
          if constexpr (TC == 3) {
            const float4 l = {tc::to_tf32(q.x - h.x), tc::to_tf32(q.y - h.y), tc::to_tf32(q.z - h.z),
                              tc::to_tf32(q.w - h.w)};
            *reinterpret_cast<float4*>(alo + tc::sw128_off(row, c)) = l;
          }
        }
      }
      fence_proxy_async();
      tc::fence_before_sync();
      asm volatile("bar.sync %0, 128;" ::"r"(8 + wg) : "memory");
      tc::fence_after_sync();
      const uint32_t d_tmem = tc_tmem + 32u * wg;
      if (row == 0) {
        const unsigned char* as[3] = {ahi, ahi, alo};
        const unsigned char* bs[3] = {tc_b, tc_b + (TC == 2 ? 2048 : 4096), tc_b};
        if constexpr (TC == 2) {
          // BF16: K = 16 values (32 bytes) per product, two products per term
          constexpr uint32_t idesc = tc::instr_desc(1, 128, 32);
#pragma unroll
          for (int term = 0; term < 3; term++)
#pragma unroll
            for (int kq = 0; kq < 2; kq++)
              tc::mma_f16(d_tmem, tc::smem_desc_sw64(smem_u32(as[term]) + 32u * kq),
                          tc::smem_desc_sw64(smem_u32(bs[term]) + 32u * kq), idesc, (term | kq) != 0);
        } else {
          constexpr uint32_t idesc = tc::instr_desc(2, 128, 32);
#pragma unroll
          for (int term = 0; term < (TC == 3 ? 3 : 1); term++)
#pragma unroll
            for (int kq = 0; kq < 4; kq++)
              tc::mma_tf32(d_tmem, tc::smem_desc_sw128(smem_u32(as[term]) + 32u * kq),
                           tc::smem_desc_sw128(smem_u32(bs[term]) + 32u * kq), idesc, (term | kq) != 0);
        }
        tc::mma_commit(&tcbar[wg]);
      }
      if (!mbar_wait_bounded(&tcbar[wg], tc_phase, abort_flag)) {
        *abort_flag = 1;
        atomicExch(p.err_flag, 1);
      }
      tc_phase ^= 1u;
      tc::fence_after_sync();
      float d[32];
      tc::tmem_ld32(d_tmem + ((uint32_t)(32 * (warp & 3)) << 16), d);
#pragma unroll
      for (int m = 0; m < 16; m++) v[m] = cT{d[2 * m], d[2 * m + 1]};
      tc::fence_before_sync();
      if constexpr (TCA) {
        // the products over this scratch (or over the tile buffer, before the
        // last stage writes the output there) are complete before it is written
        if (!in_box || kind == 2) overlay_sync();
      }
    }
  };

  // per-thread shared-memory bases
  const int scr_c = c0 * G::PITCH;
  const int s_rd = scr_c + A::idx(j0);            // reads at j0 + m  (m a multiple of TPL)
  const int s_wr0 = scr_c + A::idx(j0 * G::R0);   // stage-0 writes at j0 R0 + (u TPL R0 + q)
  auto lin_base = [&](bool lm) -> uint32_t {
    return lm ? (uint32_t)((c0 * NSUB + j0) * G::ES)
              : (uint32_t)(((c0 / G::CS) * NSUB + j0) * G::ROWB + (c0 % G::CS) * G::ES);
  };
  const uint32_t b_in = lin_base(G::LM_IN), b_out = lin_base(G::LM_OUT);
  const uint32_t z_in = b_in ^ (((b_in >> 7) & G::SWZ) << 4), z_out = b_out ^ (((b_out >> 7) & G::SWZ) << 4);

  // The output stage is radix E with one butterfly per thread: thread j0 of
  // a line produces the outputs k = j0 + q TPL, q < E, of its line.
  cT wv[E];
  unsigned smask = 0;           // sign bit of r_k for each of the thread's outputs
  int k0 = 0;                   // (k of output q = 0) mod 3
  Partials<real> acc;
  bool setup_done = false;
  long long setup_hi = -1, setup_lo0 = -1;   // the line block the setup was made for
  // the input side of the checksum runs in the first pass (single or
  // column role), the output side in the last (single or last role): the
  // other side is compiled out of each role
  constexpr bool IN_CK = ROLE != V3_LAST, OUT_CK = ROLE != V3_COLS;
  // the last pass of a multi-pass plan may carry a second check across
  // itself: its input z against u2 (held in wv, which the input side of the
  // whole-transform check does not use in this role), its output against
  // r2_k = r_k w3^floor(E k / N).  Output q of this thread (k = L + (N/NSUB)
  // (j0 + q NSUB/E)) has floor(E k / N) = q, so r2 differs from r on the
  // thread's outputs by w3^(q mod 3): the output side is a second
  // combination of the sums over q mod 3 that the first check forms.
  constexpr bool CHK2 = ROLE == V3_LAST;
  auto setup_positions = [&](long long hi, long long lo0) {
    if (CHK2 && p.chk2) {
      const cT* lt = reinterpret_cast<const cT*>(p.ltab);
      const long long L = hi * p.out_hi + (lo0 + c0) * p.out_lo;    // the line's first output
#pragma unroll
      for (int r = 0; r < E; r++) wv[r] = ldg_c(lt + L * NSUB + j0 + r * G::TPL);
    }
    if (IN_CK && p.abft_in) {
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
    k0 = 0;
    if (OUT_CK && p.abft_out) {
      const long long lo = (ROLE == V3_SINGLE) ? 0 : lo0 + c0;
      const long long kp0 = hi * p.out_hi + lo * p.out_lo + (long long)j0 * p.out_es;
      k0 = (int)(kp0 % 3);
      if (p.rvec == RVEC_SIGNED_WANG) {
#pragma unroll
        for (int q = 0; q < E; q++) {
          const long long kpos = kp0 + (long long)(q * G::TPL) * p.out_es;
          smask |= (unsigned)(splitmix64_at(p.rseed, (unsigned long long)kpos) >> 63) << q;
        }
      }
    }
  };
  const int dl = (int)(((long long)G::TPL * p.out_es) % 3);   // 1 or 2: k steps by TPL out_es
  bool aborted = false;

  int s = 0;             // ring buffer of the current tile
  unsigned wrap = 0;     // completed passes over the ring
  for (long long chunk = cfirst; chunk < cend; chunk += cstep) {
    V3Cursor cur;
    cur.chunk = chunk;
    cur.cstep = cstep;
    cur.cend = cend;
    const bool nonempty = cur.decode(p);
    // one checksum record per warp and chunk
    const long long slot = (long long)(cur.part * p.line_blocks + cur.lb) * G::NW + warp;
    if (!nonempty) {
      if (abft && !p.list && !p.sigrec) {
        acc.zero();
        warp_records(acc, p, cur.g, slot);
      }
      continue;
    }
    const long long hi = cur.hi(p), lo0 = cur.lo0(p);
    // the checksum weights, signs and residues of a thread depend only on the
    // line block (hi, lo0) of the chunk (the single pass: on nothing), so a
    // block whose chunks keep their line block -- a grid that is a multiple
    // of the line blocks -- sets them up once
    if (!setup_done || (ROLE != V3_SINGLE && (hi != setup_hi || lo0 != setup_lo0))) {
      setup_hi = hi;
      setup_lo0 = lo0;
      setup_positions(hi, lo0);
      setup_done = true;
    }
    if (abft) acc.zero();
    const long long se = cur.se;
    const long long lo_c = (ROLE == V3_SINGLE) ? 0 : lo0 + c0;
    const long long line_c = (ROLE == V3_SINGLE) ? 0 : hi * p.LO + lo_c;
    // inter-pass twiddles of the column pass: output q of this thread is
    // multiplied by omega^(lo (j0 + q TPL)) = tw_base tw_step^q
    cT tw_base = {(real)1, (real)0}, tw_step = {(real)1, (real)0};
    if (ROLE == V3_COLS && p.twiddle) {
      tw_base = twN<cT>(p, lo_c * (long long)j0 * p.tw_scale);
      tw_step = twN<cT>(p, lo_c * (long long)G::TPL * p.tw_scale);
    }
    // checksum weight (b - first signal of the group + 1) of this thread's signal
    // (one-sided mode: every signal is its own group, weight 1)
    // (per-signal records: the group weights are applied by the verification)
    real wgt = (real)(int)(cur.sb - cur.gb + (ROLE == V3_SINGLE ? c0 : 0) + 1);
    constexpr int BSTEP = ROLE == V3_SINGLE ? G::C : 1;
    const real wstep = (real)BSTEP;

    for (long long tb = cur.sb; tb < se; tb += BSTEP, wgt += wstep) {
      unsigned char* tile = base + (size_t)s * p.buf_bytes;
      if (!aborted && !mbar_wait_bounded(&full[s], wrap & 1u, abort_flag, p.wait_limit)) {
        aborted = true;
        *abort_flag = 1;
        atomicExch(p.err_flag, 1);
      }
      // after a timeout the warp still runs the tile (on whatever the buffer
      // holds) so that every line barrier is reached; the error flag is set
      const long long b0 = (ROLE == V3_SINGLE) ? tb + c0 : tb;     // this thread's signal
      const bool valid = b0 < se;
      // the stage at which this thread plants the test fault (none: -9)
      int fst = -9, fk = 0;
      if (inject && valid) {
        for (int q = 0; q < p.nfault && q < 4; q++) {
          const FaultSite& f = q == 0 ? p.fault : p.fault_more[q - 1];
          if (fst == -9 && f.mode != 0 && f.pass == p.pass_index && fault_signal(f, b0) && f.line == line_c) {
            fst = f.stage;
            fk = q;
          }
        }
      }
      const FaultSite& fs = fk == 0 ? p.fault : p.fault_more[fk - 1];

      // ---------------- stage 0: box -> registers, radix R0 -> scratch ----------------
      cT v[E];
#pragma unroll
      for (int r = 0; r < E; r++)
        v[r] = *reinterpret_cast<const cT*>(tile + A::template box<G::LM_IN>(b_in, z_in, r * G::TPL));
      if (p.conj_in) {
#pragma unroll
        for (int r = 0; r < E; r++) v[r].y = -v[r].y;
      }
      if (IN_CK && p.abft_in && valid) {
        real sr, si, en;
        if constexpr (sizeof(real) == 4) {
          // paired FP32: P = sum (wr xr, wi xi) gives Re = P.x - P.y, and
          // Q = sum (xr^2, xi^2) the energy; Im stays two scalar FMAs
          float2 P = {0.f, 0.f}, Q = {0.f, 0.f};
          float im = 0.f;
#pragma unroll
          for (int r = 0; r < E; r++) {
            P = __ffma2_rn(wv[r], v[r], P);
            Q = __ffma2_rn(v[r], v[r], Q);
            im = fmaf(wv[r].x, v[r].y, im); im = fmaf(wv[r].y, v[r].x, im);
          }
          sr = P.x - P.y; si = im; en = Q.x + Q.y;
        } else {
          sr = 0; si = 0; en = 0;
#pragma unroll
          for (int r = 0; r < E; r++) {
            sr = fma(wv[r].x, v[r].x, sr); sr = fma(-wv[r].y, v[r].y, sr);
            si = fma(wv[r].x, v[r].y, si); si = fma(wv[r].y, v[r].x, si);
            en = fma(v[r].x, v[r].x, en); en = fma(v[r].y, v[r].y, en);
          }
        }
        acc.s1r += sr; acc.s1i += si;
        if (!p.sigrec) { acc.s2r = fma(wgt, sr, acc.s2r); acc.s2i = fma(wgt, si, acc.s2i); }
        acc.en += en;
      }
      if (CHK2 && p.chk2) {
        // u2^T z over this thread's values (the last pass's input)
        real sr, si;
        if constexpr (sizeof(real) == 4) {
          float2 P = {0.f, 0.f};
          float im = 0.f;
#pragma unroll
          for (int r = 0; r < E; r++) {
            P = __ffma2_rn(wv[r], v[r], P);
            im = fmaf(wv[r].x, v[r].y, im); im = fmaf(wv[r].y, v[r].x, im);
          }
          sr = P.x - P.y; si = im;
        } else {
          sr = 0; si = 0;
#pragma unroll
          for (int r = 0; r < E; r++) {
            sr = fma(wv[r].x, v[r].x, sr); sr = fma(-wv[r].y, v[r].y, sr);
            si = fma(wv[r].x, v[r].y, si); si = fma(wv[r].y, v[r].x, si);
          }
        }
        acc.s2r += sr; acc.s2i += si;
      }
      if (fst == -1) {
#pragma unroll
        for (int r = 0; r < E; r++)
          if (fs.index == j0 + r * G::TPL) v[r] = faulted(v[r], fs);
      }
      // butterfly u of stage 0 takes v[u + m BPT0] (inputs j0 + u TPL + m NSUB / R0)
      // and writes its output q to position (j0 + u TPL) R0 + q
      if constexpr (G::R0 == E) {
        dft16(v, 0, tile);
      } else {
#pragma unroll
        for (int u = 0; u < G::BPT0; u++) {
          cT w[G::R0];
#pragma unroll
          for (int m = 0; m < G::R0; m++) w[m] = v[u + m * G::BPT0];
          Dft<G::R0>::run(w);
#pragma unroll
          for (int m = 0; m < G::R0; m++) v[u + m * G::BPT0] = w[m];
        }
      }
      if (fst == 0) {
#pragma unroll
        for (int u = 0; u < G::BPT0; u++)
#pragma unroll
          for (int q = 0; q < G::R0; q++)
            if (fs.index == (j0 + u * G::TPL) * G::R0 + q) v[u + q * G::BPT0] = faulted(v[u + q * G::BPT0], fs);
      }
      if constexpr (!G::WL) line_sync();   // the previous tile's last-stage reads are done
#pragma unroll
      for (int u = 0; u < G::BPT0; u++)
#pragma unroll
        for (int q = 0; q < G::R0; q++) {
          if constexpr (G::SPLIT0)
            scr[s_wr0 + A::idx(u * G::TPL * G::R0 + q)] = v[u + q * G::BPT0];
          else
            scr[scr_c + A::idx((j0 + u * G::TPL) * G::R0 + q)] = v[u + q * G::BPT0];
        }
      line_sync();

      // ---------------- stages 1 .. S-2: radix E, in place in the line scratch ----------------
#pragma unroll
      for (int st = 1; st < G::S - 1; st++) {
        const int Ns = G::R0 * v3_ipow(E, st - 1);
#pragma unroll
        for (int r = 0; r < E; r++) v[r] = scr[s_rd + A::idx(r * G::TPL)];
        line_sync();                          // the whole line is read before it is overwritten
        const int kk = j0 % Ns;
        {
          const cT* tw = twt + v3_tw_offset(NSUB, E, st) + kk;
#pragma unroll
          for (int q = 1; q < E; q++) v[q] = c_mul(v[q], G::TWS ? tw[(q - 1) * Ns] : ldg_c(tw + (q - 1) * Ns));
        }
        dft16(v, 1, tile);
        const int basei = (j0 / Ns) * Ns * E + kk;
        if (fst == st) {
#pragma unroll
          for (int q = 0; q < E; q++)
            if (fs.index == basei + q * Ns) v[q] = faulted(v[q], fs);
        }
        const int wb = scr_c + A::idx(basei);
#pragma unroll
        for (int q = 0; q < E; q++) scr[wb + A::idx(q * Ns)] = v[q];
        line_sync();
      }

      // ---------------- last stage: radix E -> registers -> output box ----------------
#pragma unroll
      for (int r = 0; r < E; r++) v[r] = scr[s_rd + A::idx(r * G::TPL)];
      {
        // Ns = TPL, kk = j0
        const cT* tw = twt + v3_tw_offset(NSUB, E, G::S - 1) + j0;
#pragma unroll
        for (int q = 1; q < E; q++) v[q] = c_mul(v[q], G::TWS ? tw[(q - 1) * G::TPL] : ldg_c(tw + (q - 1) * G::TPL));
      }
      dft16(v, 2, tile);
      if (ROLE == V3_COLS && p.twiddle) {
        cT f = tw_base;
#pragma unroll
        for (int q = 0; q < E; q++) {
          v[q] = c_mul(v[q], f);
          if (q + 1 < E) f = c_mul(f, tw_step);
        }
      }
      if (fst == G::S - 1) {
#pragma unroll
        for (int q = 0; q < E; q++)
          if (fs.index == j0 + q * G::TPL) v[q] = faulted(v[q], fs);
      }
      if (OUT_CK && p.abft_out && valid) {
        // T += r^T y over this thread's outputs: sum_q s_q w3^(k0 + q dl) y_q,
        // the outputs grouped by q mod 3
        real a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0;
        if constexpr (sizeof(real) == 4) {
          // s_q y_q as one paired multiply-add by (s_q, s_q), s_q = +-1 built
          // from bit q of the mask (exact: the same sums as signed adds)
          float2 A0 = {0.f, 0.f}, A1 = {0.f, 0.f}, A2 = {0.f, 0.f};
#pragma unroll
          for (int q = 0; q < E; q++) {
            const float sq = __uint_as_float(0x3f800000u | ((smask << (31 - q)) & 0x80000000u));
            const float2 s2 = {sq, sq};
            if (q % 3 == 0) A0 = __ffma2_rn(s2, v[q], A0);
            else if (q % 3 == 1) A1 = __ffma2_rn(s2, v[q], A1);
            else A2 = __ffma2_rn(s2, v[q], A2);
          }
          a0r = A0.x; a0i = A0.y; a1r = A1.x; a1i = A1.y; a2r = A2.x; a2i = A2.y;
        } else {
#pragma unroll
          for (int q = 0; q < E; q++) {
            const bool neg = (smask >> q) & 1u;
            const real yr = neg ? -v[q].x : v[q].x, yi = neg ? -v[q].y : v[q].y;
            if (q % 3 == 0) { a0r += yr; a0i += yi; }
            else if (q % 3 == 1) { a1r += yr; a1i += yi; }
            else { a2r += yr; a2i += yi; }
          }
        }
        const real hr = (real)-0.5, hs = (real)0.86602540378443864676;
        // rotate (x, y) by w3^k0
        auto rot = [&](real& x, real& y) {
          if (k0 == 1) { const real t = hr * x + hs * y; y = hr * y - hs * x; x = t; }
          else if (k0 == 2) { const real t = hr * x - hs * y; y = hr * y + hs * x; x = t; }
        };
        const real s1 = (dl == 1) ? -hs : hs;
        real tr = a0r + (hr * a1r - s1 * a1i) + (hr * a2r + s1 * a2i);
        real ti = a0i + (hr * a1i + s1 * a1r) + (hr * a2i - s1 * a2r);
        rot(tr, ti);
        if (CHK2 && p.chk2) {
          // r2 on these outputs: w3^(q dl) w3^(q mod 3) -- group q mod 3 = g
          // takes w3^(g (dl + 1)): (w3^2, w3) for dl = 1, (1, 1) for dl = 2
          real ur, ui;
          if (dl == 1) {
            ur = a0r + (hr * a1r - hs * a1i) + (hr * a2r + hs * a2i);
            ui = a0i + (hr * a1i + hs * a1r) + (hr * a2i - hs * a2r);
          } else {
            ur = a0r + a1r + a2r;
            ui = a0i + a1i + a2i;
          }
          rot(ur, ui);
          acc.t2r += ur; acc.t2i += ui;
        }
        acc.t1r += tr; acc.t1i += ti;
        if (!p.sigrec) {
          acc.t2r = fma(wgt, tr, acc.t2r); acc.t2i = fma(wgt, ti, acc.t2i);
          if (!(isfinite(tr) && isfinite(ti))) {
            acc.nf_min = min(acc.nf_min, (long long)b0);
            acc.nf_max = max(acc.nf_max, (long long)b0);
          }
        }
      }
      if (abft && p.sigrec) {
        // this tile's records, one per (signal, slot); a non-finite output
        // makes its signal's r^T y partial non-finite
        if constexpr (ROLE == V3_SINGLE) {
          if constexpr (G::WL) sig_flush<real, G::TPL, IN_CK, OUT_CK>(acc, p, b0, 0, valid);
          else sig_flush<real, 32, IN_CK, OUT_CK>(acc, p, b0, warp % G::WPL, valid);
        } else if (CHK2 && p.chk2) {
          sig_flush_chk<real>(acc, p, tb, (long long)cur.lb * G::NW + warp);
          acc.t2r = acc.t2i = acc.s2r = acc.s2i = (real)0;
        } else {
          sig_flush<real, 32, IN_CK, OUT_CK>(acc, p, tb, (long long)cur.lb * G::NW + warp, true);
        }
        acc.s1r = acc.s1i = acc.en = acc.t1r = acc.t1i = (real)0;
      }
      if constexpr (G::LM_IN != G::LM_OUT) {
        // the output box overlaps other warps' input lines: every warp has
        // its input in registers before any output lands there
        tile_sync();
      }
      if (p.conj_out || p.out_scale != 1.0) {
        const real sc = (real)p.out_scale, si = p.conj_out ? -sc : sc;
#pragma unroll
        for (int q = 0; q < E; q++) { v[q].x *= sc; v[q].y *= si; }
      }
#pragma unroll
      for (int q = 0; q < E; q++)
        *reinterpret_cast<cT*>(tile + A::template box<G::LM_OUT>(b_out, z_out, q * G::TPL)) = v[q];

      if constexpr (ROLE != V3_LAST) {
        // hand the tile back: this warp's box writes become visible to the TMA
        // unit, the eighth warp to arrive stores the tile and refills the buffer
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          const unsigned old = atom_add_acq_rel(&arrivals[s], 1u);
          V3Cursor& ld = ldc[warp];
          if (old == (unsigned)G::NW * wrap + (unsigned)(G::NW - 1) && !*abort_flag) {
            issue_store(p, tb, se, hi, lo0, reinterpret_cast<const cT*>(tile));
            bulk_commit();
            if (ld.valid(p)) {
              bulk_wait_read_0();               // the store has read the buffer
              issue_load(p, ld, reinterpret_cast<cT*>(tile), &full[s]);
              issued[s]++;
            }
          }
          ld.advance(p);
        }
        __syncwarp();
      } else {
        // the last pass's element-major box is written by all warps: once all
        // have written, each copies out its share of the rows with plain
        // stores, and the last to finish refills the buffer (no store in
        // flight holds the box)
        tile_sync();
        copy_out<G, ROLE>(p, tb, se, hi, lo0, tile, lane, warp * (NSUB / G::NW), (warp + 1) * (NSUB / G::NW));
        __syncwarp();
        if (lane == 0) {
          V3Cursor& ld = ldc[warp];
          const unsigned old = atom_add_acq_rel(&copied[s], 1u);
          if (old == (unsigned)G::NW * wrap + (unsigned)(G::NW - 1) && !*abort_flag && ld.valid(p)) {
            fence_proxy_async();
            issue_load(p, ld, reinterpret_cast<cT*>(tile), &full[s]);
            issued[s]++;
          }
          ld.advance(p);
        }
        __syncwarp();
      }
      if (++s == nbuf) { s = 0; wrap++; }
    }
    if (abft && !p.sigrec) warp_records(acc, p, cur.g, slot);
  }
  if (lane == 0) bulk_wait_0();
  // After a timed-out wait the warps skipped waiting for tiles whose loads
  // were already issued (no load is issued after the timeout): before the
  // block's shared memory is released, wait (bounded) for the last load
  // issued into every buffer.  Without a timeout every load has been waited
  // for and each of these waits returns at once.
  __syncthreads();
  if (t == 0 && *abort_flag) {
    for (int b = 0; b < nbuf; b++)
      if (issued[b] > 0u) mbar_wait_bounded(&full[b], (issued[b] - 1u) & 1u, nullptr);
  }
  if constexpr (TC != 0) {
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tc_tmem, 64);
  }
  const bool gave_up = *abort_flag != 0;
  if (t == 0 && !gave_up)
    for (int b = 0; b < nbuf; b++) mbar_inval(&full[b]);
  __syncthreads();
  return gave_up;
}

// Launches `kernel` on `s`; as a programmatic dependent of the kernel before
// it on the stream when p.pdl is set (its blocks may start while that kernel
// finishes and wait for it in griddepcontrol.wait).
template <typename K>
cudaError_t launch_v3_kernel(K kernel, int grid, int threads, size_t smem, cudaStream_t s, const PassParams& p) {
  if (!p.pdl) {
    kernel<<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, p);
}

template <typename real, int NSUB, int E, int ROLE, int TC = 0, int NT = 256>
__global__ void __launch_bounds__(NT, (NT == 256 ? v3_min_blocks_tc<real, TC>() : 1)) fft_v3_kernel(const __grid_constant__ PassParams p) {
  __shared__ V3Smem<NT / 32> vs;
  v3_body<real, NSUB, E, ROLE, TC, NT>(p, blockIdx.x, gridDim.x, p.nchunks, blockIdx.x == 0, vs);
  // this block's tiles are done: a kernel launched as a programmatic
  // dependent of this one may start its set-up (it waits for this grid to
  // complete before it touches global memory)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if constexpr (ROLE == V3_SINGLE) {
    // the last block verifies the exec and corrects what it queued, in the
    // tile ring (free once every tile is done)
    if (p.fverify && fused_verify<real>(&p) == 2) {
      extern __shared__ __align__(16) unsigned char smem_raw[];
      unsigned char* ring = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
      fused_correct<real>(p, *p.fverify, ring, (size_t)p.nbuf * p.buf_bytes);
    }
  }
}

}  // namespace tfft
