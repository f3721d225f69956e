// fft_tile.cuh -- the pass kernel with TMA-streamed tiles (the main exec path).
//
// Same sub-transform, twiddles and fused checksum encode as fft_pass_kernel
// (fft_pass.cuh), but the data move through shared memory by the Tensor
// Memory Accelerator instead of per-thread global loads and stores:
//
//   * a ring of `nbuf` tile buffers in shared memory; thread 0 keeps the
//     loads of the next two tiles in flight (cp.async.bulk for the contiguous
//     rows of a single-pass tile, cp.async.bulk.tensor through a tensor map
//     for the strided column and row tiles of the multi-pass plans), each
//     completing an mbarrier with its byte count;
//   * the block waits on the buffer's mbarrier (bounded: after the limit it
//     records an error and stops), reads its stage-0 values from the dense
//     box, runs the radix stages in place in the same buffer (XOR-swizzled
//     element-major layout between stages), writes the results back as the
//     dense output box, and thread 0 issues the TMA store;
//   * a buffer is reloaded only after its store has finished reading it
//     (cp.async.bulk.wait_group.read).
// No global address is formed per element: the only per-element memory
// operations are shared-memory loads and stores.
#pragma once

#include "fft_pass.cuh"

namespace tfft {

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_bulk(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, const void* src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(map),
               "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Dense box index (the layout TMA reads and writes).
__device__ __forceinline__ int box_index(int layout, int c, int i, int C, int nsub) {
  return layout == 0 ? c * nsub + i : i * C + c;
}
// Exchange index between radix stages: element-major with the low bits of
// the address XORed by two higher nibbles (8-byte elements: 16 per 128-byte
// row; 16-byte elements: 8 per row), so strided and unit-stride accesses
// both spread over the banks.
template <typename cT>
__device__ __forceinline__ int xchg_index(int c, int i, int C) {
  const int a = i * C + c;
  if constexpr (sizeof(cT) == 8) return a ^ (((a >> 4) ^ (a >> 8)) & 15);
  else return a ^ (((a >> 3) ^ (a >> 6)) & 7);
}

// The non-empty tiles of one thread block, in order: chunks blockIdx.x,
// blockIdx.x + gridDim.x, ...; inside a chunk its tiles (one signal, or C
// signals when lines are signals).
struct TileCursor {
  long long chunk, tb, g, lb, gb, sb, se;
  int part;
  __device__ bool decode(const PassParams& p) {
    lb = chunk % p.line_blocks;
    const long long rest = chunk / p.line_blocks;
    part = (int)(rest % p.parts);
    g = rest / p.parts;
    long long ge;
    if (p.list) {
      if (g >= p.list[0] || g >= p.list_cap) return false;
      const long long blk = p.list_identity ? g : p.list[1 + g];
      gb = blk * p.list_block;
      ge = min((long long)p.batch, gb + (long long)p.list_block);
    } else {
      gb = g * p.group;
      ge = min((long long)p.batch, gb + (long long)p.group);
    }
    const long long unit = p.lines_are_signals ? p.C : 1;
    const long long ntiles = (ge - gb + unit - 1) / unit;
    const long long per = (ntiles + p.parts - 1) / p.parts;
    sb = gb + (long long)part * per * unit;
    se = min(ge, sb + per * unit);
    return sb < se;
  }
  __device__ void settle(const PassParams& p) {
    while (chunk < p.nchunks) {
      if (decode(p)) { tb = sb; return; }
      chunk += gridDim.x;
    }
  }
  __device__ void start(const PassParams& p) { chunk = blockIdx.x; settle(p); }
  __device__ bool valid(const PassParams& p) const { return chunk < p.nchunks; }
  __device__ void advance(const PassParams& p) {
    tb += p.lines_are_signals ? p.C : 1;
    if (tb >= se) { chunk += gridDim.x; settle(p); }
  }
  __device__ long long hi(const PassParams& p) const {
    return p.lines_are_signals ? 0 : (lb * p.C) / p.LO;
  }
  __device__ long long lo0(const PassParams& p) const {
    return p.lines_are_signals ? 0 : (lb * p.C) % p.LO;
  }
};

template <typename cT, typename Cursor>
__device__ __forceinline__ void issue_load(const PassParams& p, const Cursor& cur, cT* dst,
                                           uint64_t* bar) {
  const TileMap& m = p.map_in;
  if (m.kind == 1) {
    const long long rows = min((long long)p.C, cur.se - cur.tb);
    const uint32_t bytes = (uint32_t)(rows * p.nsub * (long long)sizeof(cT));
    mbar_expect_tx(bar, bytes);
    if (p.soff_in) {          // one copy per signal (lines are whole signals here)
      const uint32_t sb = (uint32_t)(p.nsub * (long long)sizeof(cT));
      for (long long r = 0; r < rows; r++)
        tma_load_bulk(dst + r * p.nsub, reinterpret_cast<const cT*>(p.in) + p.soff_in[cur.tb + r], sb, bar);
    } else {
      tma_load_bulk(dst, reinterpret_cast<const cT*>(p.in) + cur.tb * p.n, bytes, bar);
    }
    return;
  }
  const long long hi = cur.hi(p), lo0 = cur.lo0(p), b = cur.tb;
  mbar_expect_tx(bar, m.bytes);
  if (p.soff_in) {
    // first pass, 2-D map over the whole packed buffer as rows of M = n / nsub
    // columns: signal b starts at row off / M, column off mod M; a box of
    // columns that runs past M continues on the next row (the plan checked
    // that every offset is a multiple of the box width, so no box straddles)
    const long long M = p.n / p.nsub, off = p.soff_in[b];
    const long long q = off / M, r = off - q * M;
    const int u = m.ax;
    for (int kx = 0; kx < m.nbx; kx++) {
      long long col = r + lo0 + (long long)kx * (m.bx_step / u), row = q;
      if (col >= M) { col -= M; row += 1; }
      for (int k = 0; k < m.nbox; k++)
        tma_load_2d(dst + kx * m.bx_elems + k * m.box_elems, &p.tmap_in, (int)(u * col),
                    (int)(row + (long long)k * m.box_rows), bar);
    }
    return;
  }
  const int x = (int)(m.ax * lo0);
  const int y = (int)(m.ay * hi + m.by * b + m.cy * lo0);
  const int z = (int)(m.az * hi + m.bz * b + m.cz * lo0);
  for (int kx = 0; kx < m.nbx; kx++)
    for (int k = 0; k < m.nbox; k++) {
      cT* d = dst + kx * m.bx_elems + k * m.box_elems;
      if (m.kind == 2) tma_load_2d(d, &p.tmap_in, x + kx * m.bx_step, y + k * m.box_rows, bar);
      else tma_load_3d(d, &p.tmap_in, x + kx * m.bx_step, y + k * m.box_rows, z, bar);
    }
}

template <typename cT>
__device__ __forceinline__ void issue_store(const PassParams& p, long long tb, long long se, long long hi,
                                            long long lo0, const cT* src) {
  const TileMap& m = p.map_out;
  if (m.kind == 1) {
    const long long rows = min((long long)p.C, se - tb);
    if (p.soff_out) {
      const uint32_t sb = (uint32_t)(p.nsub * (long long)sizeof(cT));
      for (long long r = 0; r < rows; r++)
        tma_store_bulk(reinterpret_cast<cT*>(p.out) + p.soff_out[tb + r], src + r * p.nsub, sb);
    } else {
      const uint32_t bytes = (uint32_t)(rows * p.nsub * (long long)sizeof(cT));
      tma_store_bulk(reinterpret_cast<cT*>(p.out) + tb * p.n, src, bytes);
    }
    return;
  }
  const int x = (int)(m.ax * lo0);
  const int y = (int)(m.ay * hi + m.by * tb + m.cy * lo0);
  const int z = (int)(m.az * hi + m.bz * tb + m.cz * lo0);
  for (int kx = 0; kx < m.nbx; kx++)
    for (int k = 0; k < m.nbox; k++) {
      const cT* s = src + kx * m.bx_elems + k * m.box_elems;
      if (m.kind == 2) tma_store_2d(&p.tmap_out, x + kx * m.bx_step, y + k * m.box_rows, s);
      else tma_store_3d(&p.tmap_out, x + kx * m.bx_step, y + k * m.box_rows, z, s);
    }
}

constexpr long long kWaitLimit = 1ll << 20;   // mbarrier polls before giving up (~1 s)

template <typename real, int E>
__global__ void __launch_bounds__(max_threads<real, E>())
fft_tile_kernel(const __grid_constant__ PassParams p) {
  using cT = typename Cplx<real>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32 * 12];

  const int t = threadIdx.x;
  const int nsub = p.nsub;
  const int C = p.C;
  const int nbuf = p.nbuf;
  // tile buffers start on a 1 KiB boundary (the launch adds 1 KiB of slack)
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nbuf * p.buf_bytes);
  auto buffer = [&](int s) { return reinterpret_cast<cT*>(base + (size_t)s * p.buf_bytes); };
  const cT* tws = reinterpret_cast<const cT*>(p.tw_sub);
  const bool abft = p.abft_in || p.abft_out;
  const bool inject = p.fault.mode != 0 && p.fault.pass == p.pass_index;
  const int lin = p.map_in.layout, lout = p.map_out.layout;

  if (t == 0) {
    for (int s = 0; s < nbuf; s++) mbar_init(&full[s], 1);
    fence_mbar_init();
    if (blockIdx.x == 0) {
      if (p.zero_on_entry[0]) *p.zero_on_entry[0] = 0;
      if (p.zero_on_entry[1]) *p.zero_on_entry[1] = 0;
      if (p.zero_on_entry[2]) *p.zero_on_entry[2] = 0;
    }
  }
  __syncthreads();

  // producer: thread 0 keeps the loads of the next tiles in flight
  TileCursor prod;
  int nissued = 0;     // loads issued by thread 0; load j goes to buffer j % nbuf
  if (t == 0) {
    prod.start(p);
    for (int s = 0; s < nbuf - 1 && prod.valid(p); s++) {
      issue_load(p, prod, buffer(s), &full[s]);
      nissued++;
      prod.advance(p);
    }
  }

  int c0, j0;
  map_bfly(t, p.in_map, C, nsub / E, c0, j0);
  const int R_last = nsub >> (__ffs(E) - 1) * (p.nstages - 1);

  cT wv[E];
  unsigned smask = 0;
  Partials<real> acc;
  bool setup_done = false;
  auto setup_positions = [&](long long hi, long long lo0) {
    if (p.abft_in) {
      const cT* wtab = reinterpret_cast<const cT*>(p.wtab);
#pragma unroll
      for (int r = 0; r < E; r++) {
        const int i = j0 + r * (nsub / E);
        const long long npos = p.lines_are_signals ? (long long)i * p.in_es
                                                   : hi * p.in_hi + (lo0 + c0) * p.in_lo + (long long)i * p.in_es;
        wv[r] = (p.rvec == RVEC_WANG) ? checksum_weight<cT>(p, npos) : ldg_c(wtab + npos);
      }
    }
    smask = 0;
    if (p.abft_out && p.rvec == RVEC_SIGNED_WANG) {
      const int RL = p.nstages > 1 ? R_last : E;
      const int nb = nsub / RL;
      for (int ub = 0; ub < E / RL; ub++) {
        int c, j;
        if (p.nstages > 1) map_bfly(t + ub * p.nthreads, p.out_map, C, nb, c, j);
        else { c = c0; j = j0; }
        const long long lo = p.lines_are_signals ? 0 : lo0 + c;
        const long long kb = hi * p.out_hi + lo * p.out_lo;
        for (int q = 0; q < RL; q++) {
          const long long kpos = kb + (long long)(j + q * nb) * p.out_es;
          smask |= (unsigned)(splitmix64_at(p.rseed, (unsigned long long)kpos) >> 63) << (ub * RL + q);
        }
      }
    }
  };

  int k = 0;   // tiles consumed so far (buffer k % nbuf)
  for (long long chunk = blockIdx.x; chunk < p.nchunks; chunk += gridDim.x) {
    TileCursor cur;
    cur.chunk = chunk;
    const bool nonempty = cur.decode(p);
    if (!nonempty) {
      if (abft && !p.list) {    // keep the record of an empty share well defined
        acc.zero();
        reduce_and_store(acc, p, cur.g, cur.part * p.line_blocks + cur.lb, red);
      }
      continue;
    }
    const long long hi = cur.hi(p), lo0 = cur.lo0(p);
    if (!p.lines_are_signals || !setup_done) {
      setup_positions(hi, lo0);
      setup_done = true;
    }
    if (abft) acc.zero();
    const long long gb = cur.gb, se = cur.se;

    for (long long tb = cur.sb; tb < se; tb += (p.lines_are_signals ? C : 1), k++) {
      const int s = k % nbuf;
      const uint32_t parity = (uint32_t)((k / nbuf) & 1);
      cT* tile = buffer(s);
      // ---- wait for the tile (bounded) ----
      {
        bool ok = false;
        for (long long it = 0; it < p.wait_limit && !ok; it++) ok = mbar_try_wait(&full[s], parity);
        if (__syncthreads_or(!ok)) {
          if (t == 0) {
            atomicExch(p.err_flag, 1);
            bulk_wait_0();
            // the loads still in flight (tiles k .. nissued-1, one per
            // buffer) land before the block's shared memory is released
            for (int j = k; j < nissued; j++) {
              bool done = false;
              for (long long it = 0; it < kWaitLimit && !done; it++)
                done = mbar_try_wait(&full[j % nbuf], (uint32_t)((j / nbuf) & 1));
            }
          }
          return;
        }
      }

      // ================= stage 0: shared (dense box) -> registers =================
      cT v[E];
      {
        const long long b = p.lines_are_signals ? tb + c0 : tb;
        const long long lo = p.lines_are_signals ? 0 : lo0 + c0;
        const bool valid = b < se;
#pragma unroll
        for (int r = 0; r < E; r++) v[r] = tile[box_index(lin, c0, j0 + r * (nsub / E), C, nsub)];
        if (p.conj_in) {
#pragma unroll
          for (int r = 0; r < E; r++) v[r].y = -v[r].y;
        }
        if (p.abft_in && valid) {
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
        Dft<E>::run(v);
        __syncthreads();                      // every stage-0 read of the box is done
        {
          const long long b = p.lines_are_signals ? tb + c0 : tb;
          const long long line = p.lines_are_signals ? 0 : hi * p.LO + lo0 + c0;
#pragma unroll
          for (int q = 0; q < E; q++) {
            const int i = j0 * E + q;
            if (inject && p.fault.stage == 0 && fault_signal(p.fault, b) && p.fault.line == line &&
                p.fault.index == i && b < se)
              v[q] = faulted(v[q], p.fault);
            tile[xchg_index<cT>(c0, i, C)] = v[q];
          }
        }
        __syncthreads();
        Ns = E;
        for (int st = 1; st < p.nstages - 1; st++) {
          int c, j;
          map_bfly(t, p.mid_map, C, nsub / E, c, j);
#pragma unroll
          for (int r = 0; r < E; r++) v[r] = tile[xchg_index<cT>(c, j + r * (nsub / E), C)];
          __syncthreads();
          const int kk = j & (Ns - 1);
          stage_twiddle<E>(v, tws, kk * (nsub / (Ns * E)) * p.tw_sub_stride);
          Dft<E>::run(v);
          const int basei = (j / Ns) * Ns * E + kk;
          const long long b = p.lines_are_signals ? tb + c : tb;
          const long long line = p.lines_are_signals ? 0 : hi * p.LO + lo0 + c;
#pragma unroll
          for (int q = 0; q < E; q++) {
            const int i = basei + q * Ns;
            if (inject && p.fault.stage == st && fault_signal(p.fault, b) && p.fault.line == line &&
                p.fault.index == i && b < se)
              v[q] = faulted(v[q], p.fault);
            tile[xchg_index<cT>(c, i, C)] = v[q];
          }
          __syncthreads();
          Ns *= E;
        }
      }

      // ================= last stage: -> shared (dense output box) =================
      auto last_stage = [&](auto RC) {
        constexpr int RL = decltype(RC)::value;
        constexpr int NB = E / RL;
        const int nb = nsub / RL;
        cT u[E];
        int cc[NB], jj[NB];
        if (p.nstages > 1) {
#pragma unroll
          for (int ub = 0; ub < NB; ub++) {
            map_bfly(t + ub * p.nthreads, p.out_map, C, nb, cc[ub], jj[ub]);
#pragma unroll
            for (int r = 0; r < RL; r++) u[ub * RL + r] = tile[xchg_index<cT>(cc[ub], jj[ub] + r * nb, C)];
          }
        } else {
#pragma unroll
          for (int r = 0; r < E; r++) u[r] = v[r];
          cc[0] = c0; jj[0] = j0;
        }
#pragma unroll
        for (int ub = 0; ub < NB; ub++) {
          cT* w = u + ub * RL;
          const int c = cc[ub], j = jj[ub];
          const int kk = j & (Ns - 1);
          stage_twiddle<RL>(w, tws, kk * (nsub / (Ns * RL)) * p.tw_sub_stride);
          Dft<RL>::run(w);
          const long long b = p.lines_are_signals ? tb + c : tb;
          const long long lo = p.lines_are_signals ? 0 : lo0 + c;
          const bool valid = b < se;
          if (p.twiddle) {
            // inter-pass twiddle omega_{tw_n}^{lo i}, i = j + q nb: omega^{lo j} (omega^{lo nb})^q
            const cT base = twN<cT>(p, lo * (long long)j * p.tw_scale);
            const cT step = twN<cT>(p, lo * (long long)nb * p.tw_scale);
            cT f = base;
#pragma unroll
            for (int q = 0; q < RL; q++) {
              w[q] = c_mul(w[q], f);
              if (q + 1 < RL) f = c_mul(f, step);
            }
          }
          if (inject && p.fault.stage == p.nstages - 1 && valid && fault_signal(p.fault, b) &&
              p.fault.line == (p.lines_are_signals ? 0 : hi * p.LO + lo)) {
#pragma unroll
            for (int q = 0; q < RL; q++)
              if (p.fault.index == j + q * nb) w[q] = faulted(w[q], p.fault);
          }
          if (p.abft_out && valid) {
            real a0r = 0, a0i = 0, a1r = 0, a1i = 0, a2r = 0, a2i = 0;
#pragma unroll
            for (int q = 0; q < RL; q++) {
              const bool neg = (smask >> (ub * RL + q)) & 1u;
              const real yr = neg ? -w[q].x : w[q].x, yi = neg ? -w[q].y : w[q].y;
              if (q % 3 == 0) { a0r += yr; a0i += yi; }
              else if (q % 3 == 1) { a1r += yr; a1i += yi; }
              else { a2r += yr; a2i += yi; }
            }
            const long long kpos = hi * p.out_hi + lo * p.out_lo + (long long)j * p.out_es;
            const int k0 = (int)(kpos % 3);
            const int dl = (int)(((long long)nb * p.out_es) % 3);
            const real hr = (real)-0.5, hs = (real)0.86602540378443864676;
            const real s1 = (dl == 1) ? -hs : hs;
            real tr = a0r + (hr * a1r - s1 * a1i) + (hr * a2r + s1 * a2i);
            real ti = a0i + (hr * a1i + s1 * a1r) + (hr * a2i - s1 * a2r);
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
        __syncthreads();                      // every read of the exchange layout is done
#pragma unroll
        for (int ub = 0; ub < NB; ub++)
#pragma unroll
          for (int q = 0; q < RL; q++)
            tile[box_index(lout, cc[ub], jj[ub] + q * nb, C, nsub)] = out_xform(u[ub * RL + q], p);
      };
      switch (p.nstages > 1 ? R_last : E) {
        case 1: if constexpr (E == 1) last_stage(std::integral_constant<int, 1>{}); break;
        case 2: if constexpr (E >= 2) last_stage(std::integral_constant<int, 2>{}); break;
        case 4: if constexpr (E >= 4) last_stage(std::integral_constant<int, 4>{}); break;
        case 8: if constexpr (E >= 8) last_stage(std::integral_constant<int, 8>{}); break;
        case 16: if constexpr (E >= 16) last_stage(std::integral_constant<int, 16>{}); break;
        default: break;
      }
      fence_proxy_async();                    // make the box visible to the TMA unit
      __syncthreads();
      if (t == 0) {
        issue_store(p, tb, se, hi, lo0, tile);
        bulk_commit();
        // the buffer of the previous tile is free once its store has read it
        bulk_wait_read_1();
        if (prod.valid(p)) {
          const int sp = (k + nbuf - 1) % nbuf;
          issue_load(p, prod, buffer(sp), &full[sp]);
          nissued++;
          prod.advance(p);
        }
      }
    }
    if (abft) reduce_and_store(acc, p, cur.g, cur.part * p.line_blocks + cur.lb, red);
  }
  if (t == 0) bulk_wait_0();
}

}  // namespace tfft
