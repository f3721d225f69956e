// plan.cu -- host side of the library: planner, FP64 twiddle and checksum
// tables, workspace, the exec launch sequence and the C ABI of include/tfft.h.
//
// Plan (TurboFFT Section IV-A, "Tiled FFT" and "Kernel Parameters"): a signal
// that fits one thread block's tile is transformed in one launch; a longer one
// is viewed as an N1 x N2 (x N3) array and transformed by two (three)
// launches, one per axis, the first ones writing in place and the last one
// transposing into natural order (the four-step factorisation
//   y[k1 + N1 k2] = sum_{n2} wN2^{n2 k2} wN^{n2 k1} sum_{n1} x[N2 n1 + n2] wN1^{n1 k1}).
// Exec (Section III): pass kernels with the checksum encode fused into the
// first and last pass, then verify, then the correction path, all on the
// caller's stream with no host synchronisation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tfft_internal.h"

using namespace tfft;

namespace {

std::atomic<int> g_last_cuda_error{0};

int cuda_fail(cudaError_t e) {
  g_last_cuda_error.store((int)e);
  return TFFT_ERR_CUDA;
}

}  // namespace

namespace tfft {
int record_cuda_error(cudaError_t e) { return cuda_fail(e); }
}  // namespace tfft

namespace {

#define TFFT_CUDA(call)                       \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

// e^{-2 pi i m / n} in FP64: the integer m is reduced modulo n and split into
// a quarter turn q and a remainder before any rounding, and the remaining
// angle is taken from whichever of r, n - r keeps it below pi/4.
void unit_root(int64_t m, int64_t n, double* re, double* im) {
  m %= n;
  if (m < 0) m += n;
  const int64_t q = (4 * m) / n, r = 4 * m - q * n;       // theta = (pi/2)(q + r/n)
  const double half_pi = 1.57079632679489661923132169163975144;
  double c, s;
  if (2 * r <= n) {
    const double a = half_pi * (double)r / (double)n;
    c = std::cos(a); s = std::sin(a);
  } else {
    const double a = half_pi * (double)(n - r) / (double)n;
    c = std::sin(a); s = std::cos(a);
  }
  double x, y;   // e^{+i theta}
  switch (q & 3) {
    case 0: x = c; y = s; break;
    case 1: x = -s; y = c; break;
    case 2: x = -c; y = -s; break;
    default: x = s; y = -c; break;
  }
  *re = x;
  *im = -y;
}

int ilog2(int64_t v) { int k = 0; while ((int64_t(1) << k) < v) k++; return k; }
bool is_pow2(int64_t v) { return v >= 1 && (v & (v - 1)) == 0; }

// Geometry of one tensor map (in 8-byte units along the innermost dimension).
struct MapGeom {
  int rank = 0;
  int swizzle = 0;                 // CUtensorMapSwizzle
  uint64_t dims[3] = {0, 0, 0};
  uint64_t strides[2] = {0, 0};   // bytes, dimensions 1 and 2
  uint32_t box[3] = {1, 1, 1};
};

struct PassPlan {
  int nsub = 1, E = 1, C = 1, nthreads = 32, nstages = 1, pitch = 1;
  // TMA tile pipeline (fft_tile_kernel) for the main exec
  int tma = 0, nbuf = 0, tbps = 1;
  int v3 = 0, role = 0;            // v3 kernel (compile-time geometry) and its role
  int vC = 0;                      // v3 lines per tile
  int vdt = 0;                     // v3 kernel family (launch_v3 dtype code)
  int vtc = 0;                     // v3 tensor-core variant (3 split TF32, 1 TF32), 0 none
  int vnt = 256;                   // v3 threads per block (256, or 512 for the wide tiles)
  int no_tile = 0;                 // no TMA tile kernel for this pass's E (complex128, E = 16)
  int64_t vLB = 0;                 // v3 line blocks per signal
  unsigned buf_bytes = 0;
  size_t tsmem = 0;
  TileMap map_in{}, map_out{};
  MapGeom gin{}, gout{};
  int in_map = MAP_ROW, mid_map = MAP_ROW, out_map = MAP_ROW;
  int lines_are_signals = 0, twiddle = 0, parts = 1;
  int64_t LO = 1, HI = 1, line_blocks = 1;
  int64_t in_es = 1, in_lo = 0, in_hi = 0, out_es = 1, out_lo = 0, out_hi = 0;
  int64_t tw_scale = 1;
  size_t smem = 0;
  int bps = 1;       // resident blocks per SM
  void* vtw = nullptr;               // v3 stage-twiddle table
};

struct TimedLaunch {
  cudaEvent_t a, b;
  int kind;
};

}  // namespace

struct tfft_plan_s {
  int64_t n = 0, batch = 0;
  int dtype = 0, abft = 0;
  int G = 16;
  double kappa = 2.0;
  int rvec = RVEC_SIGNED_WANG;
  unsigned long long rseed = 20240502ull;
  void* wtab = nullptr;
  int detect_only = 0;
  int inverse = 0, normalize = 0;
  int one_sided = 0;                 // per-signal checksums (verification groups of one)
  int prec = TFFT_PREC_FP32;         // arithmetic of the radix-16 butterflies
  long long wait_limit = 1ll << 20;  // polls of a tile-arrival wait
  int tile_threads = 0;              // column / last passes of 512..2048 points: 0 auto, 256, 512
  int tuned = 0;                     // the pass configuration came from the autotuner's table
  int vG = 16;                       // signals per verification group
  int64_t vgroups = 0;               // verification groups
  int cap_fix = 1, cap_rec = 1;
  int passes = 1;
  PassPlan pp[3];
  int64_t ngroups = 0;
  int device = 0, sms = 1;
  size_t esize = 8;

  void* tw_sub = nullptr; int tw_sub_n = 1;
  void* twN_lo = nullptr; void* twN_hi = nullptr; int twN_lbits = 0;
  void* wt_lo = nullptr; void* wt_hi = nullptr; int wt_lbits = 0;
  void* tmp = nullptr;
  RecIn* rec_in = nullptr; RecOut* rec_out = nullptr;
  // per-signal records (every encoding pass on the tile kernels)
  int sigrec = 0;
  void* sig_in = nullptr; void* sig_out = nullptr;
  int64_t sslots_in = 1, sslots_out = 1;
  int sig_split = 0;
  double* sig_acc = nullptr;
  int sig_blk_lanes = 0, sig_gpb = 1;   // block verification in place of the split mode
  // second check across the last pass (multi-pass plans with per-signal records)
  int chk2 = 0;
  void* ltab = nullptr;             // u2[L][n], N entries
  void* sig_chk = nullptr;
  int vsplit = 1;                   // verification blocks per group
  double* part_acc = nullptr;       // split verification: per-group accumulators
  unsigned* part_cnt = nullptr;
  int64_t slots_in = 1, slots_out = 1;
  long long* lists_mem = nullptr;
  Lists lists{};
  Counters* counters = nullptr;
  LogEvent* log = nullptr;
  void* ws_c1 = nullptr; void* ws_acc = nullptr;
  void* stage_in = nullptr; void* stage_out = nullptr;
  int* err_flag = nullptr;
  const void* enc_ptr[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  const long long* soff = nullptr;   // signal offsets of the exec's input and output (ragged)
  CUtensorMap enc_map[3][2];

  FaultSite pending{};                 // first armed fault site (every kernel)
  FaultSite pending_more[3]{};          // further sites (tile kernels)
  int npending = 0;
  int64_t execs = 0, launches = 0;
  cudaStream_t last_stream = nullptr;
  bool used = false;
  // correction graph: verification, then a conditional node whose body is the
  // correction sequence; built for one (in, out) pair, replayed afterwards
  long long* cond_flag = nullptr;
  cudaStream_t gcap = nullptr;
  cudaGraph_t cg = nullptr;
  cudaGraphExec_t cgx = nullptr;
  cudaGraphNode_t cg_vnode = nullptr;
  cudaKernelNodeParams cg_kp{};
  VerifyParams cg_v{};
  int cg_lanes = 0;
  const void* cg_in = nullptr;
  void* cg_out = nullptr;
  const void* last_in = nullptr;    // the previous whole-batch exec's buffers
  void* last_out = nullptr;
  bool cg_off = false;              // building failed once: stream launches only
  bool cg_full = false;             // the cached graph also holds the passes
  bool cg_armed = false;            // ... with an armed test fault in them (built for one exec)
  // fused verification (single-pass plans of few groups, stream-launched whole-batch execs):
  // the pass kernel's last block verifies, with the parameters in fverify
  int fuse = 0;
  int pdl_now = 0;                   // this exec's fused pass is a programmatic dependent launch
  unsigned* fdone = nullptr;         // blocks done, reset by the last
  VerifyParams* fverify = nullptr;   // without a conditional node

  // tfft_exec_host pipeline: copy streams and per-chunk events, made on first use
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_entry = nullptr, ev_end = nullptr;
  cudaEvent_t ev_in[8] = {}, ev_done[8] = {};
  int timing = 0;
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  int64_t workspace_bytes = 0;
  std::mutex mu;
};

namespace {

template <typename real>
struct HostC { real x, y; };

template <typename real>
int upload_table(void** dst, const std::vector<double>& re, const std::vector<double>& im, int64_t* bytes) {
  std::vector<HostC<real>> h(re.size());
  for (size_t i = 0; i < re.size(); i++) h[i] = HostC<real>{(real)re[i], (real)im[i]};
  const size_t b = h.size() * sizeof(HostC<real>);
  TFFT_CUDA(cudaMalloc(dst, std::max<size_t>(b, 16)));
  TFFT_CUDA(cudaMemcpy(*dst, h.data(), b, cudaMemcpyHostToDevice));
  *bytes += (int64_t)b;
  return 0;
}

int upload(tfft_plan_s* p, void** dst, const std::vector<double>& re, const std::vector<double>& im) {
  return p->dtype == TFFT_C64 ? upload_table<float>(dst, re, im, &p->workspace_bytes)
                              : upload_table<double>(dst, re, im, &p->workspace_bytes);
}

void free_plan(tfft_plan_s* p) {
  if (p->cgx) cudaGraphExecDestroy(p->cgx);
  if (p->cg) cudaGraphDestroy(p->cg);
  if (p->gcap) cudaStreamDestroy(p->gcap);
  for (cudaEvent_t e : p->ev_in) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_done) if (e) cudaEventDestroy(e);
  if (p->ev_entry) cudaEventDestroy(p->ev_entry);
  if (p->ev_end) cudaEventDestroy(p->ev_end);
  if (p->h2d) cudaStreamDestroy(p->h2d);
  if (p->d2h) cudaStreamDestroy(p->d2h);
  void* bufs[] = {p->tw_sub, p->twN_lo, p->twN_hi, p->wt_lo, p->wt_hi, p->wtab, p->tmp, p->rec_in, p->rec_out,
                  p->lists_mem, p->counters, p->log, p->ws_c1, p->ws_acc, p->stage_in, p->stage_out,
                  p->err_flag, p->part_acc, p->part_cnt, p->sig_in, p->sig_out, p->sig_acc, p->ltab,
                  p->sig_chk, p->fdone, p->fverify};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (auto& q : p->pp)
    if (q.vtw) cudaFree(q.vtw);
  for (auto& t : p->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  for (auto e : p->event_pool) cudaEventDestroy(e);
  delete p;
}

int pass_attrs(const tfft_plan_s* p, PassPlan& q) {
  cudaError_t e = p->dtype == TFFT_C64 ? pass_func_attrs_f32(q.E, q.smem, q.nthreads, &q.bps)
                                       : pass_func_attrs_f64(q.E, q.smem, q.nthreads, &q.bps);
  if (e != cudaSuccess) return cuda_fail(e);
  if (q.bps < 1) return TFFT_ERR_UNSUPPORTED;
  return 0;
}

// Elements per thread for a sub-transform of length nsub: the full radix E0
// unless the line is so short that fewer than four threads would share it.
int pick_E(int nsub, int E0) {
  int E = std::min(E0, nsub);
  while (E > 2 && nsub / E < 4) E /= 2;
  return std::max(E, 1);
}

int row_pad(int nsub, int E, int S) {
  const int lanes = std::max(1, nsub / E);
  return lanes < S ? lanes : 0;
}

int col_pad(int C, int S) { return C < S ? S / C : 1; }

int nstages_of(int nsub, int E) {
  if (nsub <= 1) return 1;
  int s = 0;
  int64_t v = 1;
  while (v < nsub) { v *= E; s++; }
  return std::max(s, 1);
}

}  // namespace

namespace tfft {

int geom_pick_E(int nsub, int E0) { return pick_E(nsub, E0); }
int geom_nstages(int nsub, int E) { return nstages_of(nsub, E); }

void two_pass_geometry(int64_t n, int64_t N1, int esize, PassGeom g[2]) {
  const bool c64 = esize == 8;
  const int E0 = c64 ? 16 : 8;
  const int TILE = c64 ? 4096 : 2048;        // elements of one thread block's tile
  const int S = c64 ? 16 : 8;                // elements per 128-byte shared-memory row
  const int64_t M = n / N1;
  // first pass: columns n_rest of length N1, stride M, twiddle wN^{n_rest k1}
  PassGeom& a = g[0];
  a = PassGeom{};
  a.nsub = (int)N1; a.E = pick_E(a.nsub, E0);
  a.LO = M; a.HI = 1;
  a.C = (int)std::min<int64_t>(std::min<int64_t>(TILE / N1, M), 64);
  a.in_es = M; a.in_lo = 1; a.out_es = M; a.out_lo = 1;
  a.in_map = a.mid_map = a.out_map = MAP_COL;
  a.twiddle = 1; a.tw_scale = 1;
  a.pitch = a.nsub + col_pad(a.C, S);
  // second pass: rows of length N2 = M, contiguous, stored transposed
  PassGeom& b = g[1];
  b = PassGeom{};
  const int64_t N2 = M;
  b.nsub = (int)N2; b.E = pick_E(b.nsub, E0);
  b.LO = N1; b.HI = 1;
  b.C = (int)std::min<int64_t>(std::min<int64_t>(TILE / N2, N1), 64);
  b.in_es = 1; b.in_lo = N2; b.out_es = N1; b.out_lo = 1;
  b.in_map = MAP_ROW; b.out_map = MAP_COL; b.mid_map = b.C >= S / 2 ? MAP_COL : MAP_ROW;
  b.pitch = b.nsub + (b.mid_map == MAP_COL ? col_pad(b.C, S) : row_pad(b.nsub, b.E, S));
  for (int i = 0; i < 2; i++) {
    PassGeom& q = g[i];
    q.nthreads = (int)((int64_t)q.C * q.nsub / q.E);
    q.nstages = nstages_of(q.nsub, q.E);
    q.line_blocks = q.LO * q.HI / q.C;
    q.smem = (size_t)q.C * q.pitch * (size_t)esize;
  }
}

}  // namespace tfft

namespace {

void copy_geom(PassPlan& q, const PassGeom& g) {
  q.nsub = g.nsub; q.E = g.E; q.C = g.C; q.pitch = g.pitch;
  q.in_map = g.in_map; q.mid_map = g.mid_map; q.out_map = g.out_map; q.twiddle = g.twiddle;
  q.LO = g.LO; q.HI = g.HI; q.in_es = g.in_es; q.in_lo = g.in_lo; q.in_hi = g.in_hi;
  q.out_es = g.out_es; q.out_lo = g.out_lo; q.out_hi = g.out_hi; q.tw_scale = g.tw_scale;
}

int plan_build(tfft_plan_s* p, const tfft_plan_opts* o) {
  const int64_t n = o->n;
  const bool c64 = o->dtype == TFFT_C64;
  p->esize = c64 ? 8 : 16;
  const int E0 = c64 ? 16 : 8;
  const int TILE = c64 ? 4096 : 2048;        // elements of one thread block's tile
  const int S = c64 ? 16 : 8;                // elements per 128-byte shared-memory row
  const int CMIN = c64 ? 8 : 4;              // lines per tile for 64-byte column runs
  // longest sub-transform of a multi-pass plan; beyond NSUBMAX^3 elements the
  // three passes take sub-transforms up to twice that (32-byte column runs)
  const int NSUBMAX = n > (int64_t)(TILE / CMIN) * (TILE / CMIN) * (TILE / CMIN) ? 2 * TILE / CMIN : TILE / CMIN;

  // complex64 two-pass plans may end in a 1024-point last pass (line-major
  // input rows; 32-byte output column runs), which beats three passes for
  // N = 2^19; a 1024-point first pass (32-byte input column runs) does not
  const int64_t LASTMAX2 = c64 ? 2 * NSUBMAX : NSUBMAX;
  // complex64 two-pass plans run on the 512-thread tiles up to 2048-point
  // factors (32- to 128-byte rows); measured with the checksums on (2^28
  // elements), two passes with a 2048-point first pass beat three up to
  // N = 2^20 (2.26 / 2.48 ms against 2.90 / 2.74 ms at 2^19 / 2^20) and
  // lose from 2^21 (2.58 against 2.56 ms, 2.76 against 2.49 ms at 2^22)
  const int64_t FMAX2 = c64 ? 2048 : NSUBMAX;
  const int64_t TWO_PASS_MAX = c64 ? (int64_t(1) << 20) : (int64_t)NSUBMAX * LASTMAX2;
  // one pass up to 4096 points for both types: complex128 then takes 16
  // values a thread (one 4096-point line a tile of 256 threads)
  const int64_t ONE_PASS_MAX = 4096;
  int passes;
  if (o->force_passes) passes = o->force_passes;
  else if (n <= ONE_PASS_MAX) passes = 1;
  else if (n <= TWO_PASS_MAX) passes = 2;
  else passes = 3;
  const int m = ilog2(n);
  int mf[3] = {m, 0, 0};
  // the largest factor goes to the last pass, whose line-major input rows
  // read with fewer shared-memory bank conflicts the longer they are
  if (passes == 2) { mf[0] = m / 2; mf[1] = m - mf[0]; }
  if (passes == 3) { mf[0] = m / 3; mf[1] = (m - mf[0]) / 2; mf[2] = m - mf[0] - mf[1]; }
  // ... except a 512-point last pass (three radix stages and 64-byte output
  // rows), which runs slower than a 512-point first pass
  if (passes > 1 && mf[passes - 1] == 9 && mf[0] < 9) std::swap(mf[0], mf[passes - 1]);
  // measured at 2^28 elements (every first factor and tile size timed):
  // N = 2^17 with the checksums on runs fastest as 256 x 512 (1.97 ms against
  // 2.01 for 512 x 256, whose 512-point input checksum costs more), without
  // them as 512 x 256 (1.62 against 1.67); N = 2^18 as 1024 x 256 (2.14 ms on,
  // 1.76 off, against 2.19 / 1.83 for 512 x 512)
  if (passes == 2 && c64 && o->abft_mode != TFFT_ABFT_OFF && !o->force_passes && m == 17) {
    mf[0] = 8;
    mf[1] = 9;
  }
  if (passes == 2 && c64 && !o->force_passes && m == 18) {
    mf[0] = 10;
    mf[1] = 8;
  }
  // N = 2^19 and 2^20: a 2048-point first pass (512-thread tiles, 32-byte
  // rows) and a 256- or 512-point last pass
  if (passes == 2 && c64 && !o->force_passes && (m == 19 || m == 20)) {
    mf[0] = 11;
    mf[1] = m - 11;
  }
  // the caller's choice of the first factor (two passes)
  if (o->first_pass_log2) {
    if (passes != 2 || o->first_pass_log2 < 1 || o->first_pass_log2 >= m) return TFFT_ERR_INVALID_ARG;
    mf[0] = o->first_pass_log2;
    mf[1] = m - mf[0];
  }
  if (passes == 1 && n > ONE_PASS_MAX) return TFFT_ERR_INVALID_ARG;
  for (int i = 1; i < passes; i++)
    if (mf[i] < 1) return TFFT_ERR_INVALID_ARG;
  if (passes == 2 && c64) {
    for (int i = 0; i < 2; i++)
      if ((int64_t(1) << mf[i]) > FMAX2) return TFFT_ERR_INVALID_ARG;
  } else if (passes > 1) {
    for (int i = 0; i < passes; i++)
      if ((int64_t(1) << mf[i]) > (passes == 2 && i == 1 ? LASTMAX2 : NSUBMAX)) return TFFT_ERR_INVALID_ARG;
  }
  p->passes = passes;

  int G = o->group > 0 ? o->group : 16;

  if (passes == 1) {
    PassPlan& q = p->pp[0];
    q.nsub = (int)n;
    q.E = pick_E(q.nsub, E0);
    if (n > TILE) {                     // complex128, 4096 points: radix 16
      q.E = v3_radix(1, (int)n);
      q.no_tile = 1;
    }
    q.lines_are_signals = 1;
    int C = std::max(1, TILE / q.nsub);
    while (C > 1 && (G % C != 0 || C > G)) C >>= 1;   // tiles never straddle groups
    while ((int64_t)C * q.nsub / q.E < 32) C <<= 1;  // at least one full warp
    if (C > G) G = C;                                 // tiny n: group grows to the tile
    q.C = C;
    q.in_map = q.mid_map = q.out_map = MAP_ROW;
    q.in_es = q.out_es = 1;
    q.pitch = q.nsub + row_pad(q.nsub, q.E, S);
  } else {
    const int64_t N1 = int64_t(1) << mf[0];
    const int64_t M = n / N1;
    PassGeom g2[2];
    two_pass_geometry(n, N1, (int)p->esize, g2);
    // first pass: columns n_rest of length N1, stride M, twiddle wN^{n_rest k1}
    PassPlan& a = p->pp[0];
    copy_geom(a, g2[0]);
    if (passes == 2) {
      copy_geom(p->pp[1], g2[1]);
    } else {
      const int64_t N2 = int64_t(1) << mf[1], N3 = int64_t(1) << mf[2];
      PassPlan& b = p->pp[1];           // lines (k1, n3) over n2, stride N3
      b.nsub = (int)N2; b.E = pick_E(b.nsub, E0);
      b.LO = N3; b.HI = N1;
      b.C = (int)std::min<int64_t>(std::min<int64_t>(TILE / N2, N3), 64);
      b.in_es = N3; b.in_lo = 1; b.in_hi = M;
      b.out_es = N3; b.out_lo = 1; b.out_hi = M;
      b.in_map = b.mid_map = b.out_map = MAP_COL;
      b.twiddle = 1; b.tw_scale = N1;    // wM^{n3 k2} = wN^{N1 n3 k2}
      b.pitch = b.nsub + col_pad(b.C, S);
      PassPlan& c = p->pp[2];           // lines (k1, k2) over n3, contiguous; store transposed
      c.nsub = (int)N3; c.E = pick_E(c.nsub, E0);
      c.LO = N1; c.HI = N2;
      c.C = (int)std::min<int64_t>(std::min<int64_t>(TILE / N3, N1), 64);
      c.in_es = 1; c.in_lo = M; c.in_hi = N3;
      c.out_es = N1 * N2; c.out_lo = 1; c.out_hi = N1;
      c.in_map = MAP_ROW; c.out_map = MAP_COL; c.mid_map = c.C >= S / 2 ? MAP_COL : MAP_ROW;
      c.pitch = c.nsub + (c.mid_map == MAP_COL ? col_pad(c.C, S) : row_pad(c.nsub, c.E, S));
    }
  }
  p->G = G;
  p->ngroups = (p->batch + G - 1) / G;

  for (int i = 0; i < passes; i++) {
    PassPlan& q = p->pp[i];
    q.nthreads = (int)((int64_t)q.C * q.nsub / q.E);
    if (q.nthreads < 32 || q.nthreads > 512 || q.nthreads % 32 != 0) return TFFT_ERR_UNSUPPORTED;
    q.nstages = nstages_of(q.nsub, q.E);
    q.smem = (size_t)q.C * q.pitch * p->esize;
    q.line_blocks = q.lines_are_signals ? 1 : q.LO * q.HI / q.C;
    int rc = pass_attrs(p, q);
    if (rc) return rc;
  }
  return 0;
}

// Chunks per group (thread blocks sharing a group) and checksum record slots
// per group: one record per chunk, or one per warp and chunk for v3 passes.
void plan_slots(tfft_plan_s* p) {
  for (int i = 0; i < p->passes; i++) {
    PassPlan& q = p->pp[i];
    const int64_t target = (int64_t)2 * p->sms * std::max(1, q.v3 ? q.tbps : q.bps);
    const int64_t lb = q.v3 ? q.vLB : q.line_blocks;
    const int64_t cc = q.v3 ? q.vC : q.C;
    const int64_t base = p->ngroups * lb;
    const int64_t tiles_per_group = q.lines_are_signals ? std::max<int64_t>(1, p->G / cc) : p->G;
    q.parts = 1;
    if (base < target) q.parts = (int)std::min<int64_t>(tiles_per_group, (target + base - 1) / base);
  }
  const PassPlan& f = p->pp[0];
  const PassPlan& l = p->pp[p->passes - 1];
  // v3 writes one record per warp and chunk, the other kernels one per chunk
  p->slots_in = (int64_t)f.parts * (f.v3 ? f.vLB * (f.vnt / 32) : f.line_blocks);
  p->slots_out = (int64_t)l.parts * (l.v3 ? l.vLB * (l.vnt / 32) : l.line_blocks);
  p->vG = p->G;
  p->vgroups = p->ngroups;
  // per-signal records when the passes that encode (the first and the last)
  // run on the tile kernels: the single pass writes one per line, or per warp
  // holding a part of a longer line; the column and last passes one per warp
  // and line block
  p->sigrec = p->abft && f.v3 && l.v3;
  if (p->sigrec) {
    auto per_signal = [&](const PassPlan& q) -> int64_t {
      if (q.role != 0) return q.vLB * (q.vnt / 32);
      const int64_t tpl = q.nsub / v3_radix(p->dtype == TFFT_C64 ? 0 : 1, q.nsub);
      return tpl > 32 ? tpl / 32 : 1;
    };
    p->sslots_in = per_signal(f);
    p->sslots_out = per_signal(l);
    // a multi-pass plan also checks its last pass on its own, against a
    // second left vector (its table takes N entries, built from 48 N bytes of
    // temporary memory at plan time: up to 2^26 elements)
    p->chk2 = p->passes > 1 && p->n <= (int64_t(1) << 26);
  }
  if (p->one_sided) {          // every signal is its own verification group
    p->vG = 1;
    p->vgroups = p->batch;
  }
}

// cuTensorMapEncodeTiled, fetched from the driver through the runtime (no
// link-time dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

bool encode_map(CUtensorMap* m, const MapGeom& g, const void* base) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t gd[3], gs[2];
  cuuint32_t bd[3], es[3] = {1, 1, 1};
  for (int i = 0; i < g.rank; i++) { gd[i] = g.dims[i]; bd[i] = g.box[i]; }
  for (int i = 0; i + 1 < g.rank; i++) gs[i] = g.strides[i];
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)g.rank, const_cast<void*>(base), gd, gs, bd, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, (CUtensorMapSwizzle)g.swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool geom_ok(const MapGeom& g) {
  for (int i = 0; i < g.rank; i++)
    if (g.box[i] < 1 || g.box[i] > 256 || g.dims[i] < g.box[i] || g.dims[i] >= (uint64_t(1) << 32)) return false;
  if ((g.box[0] * 8) % 16) return false;
  for (int i = 0; i + 1 < g.rank; i++)
    if (g.strides[i] % 16 || g.strides[i] >= (uint64_t(1) << 40)) return false;
  return true;
}

// Tile maps of the TMA pipeline for every pass (Section IV-A kernel-level
// tiling expressed as tensor-map boxes).  A pass whose boxes do not fit the
// TMA limits keeps the direct-load kernel.
int plan_tma(tfft_plan_s* p) {
  if (!encode_fn()) return 0;
  const int64_t u = (int64_t)p->esize / 8;     // 8-byte units per element
  const int64_t B = p->batch, es = (int64_t)p->esize;
  for (int i = 0; i < p->passes; i++) {
    PassPlan& q = p->pp[i];
    if (q.no_tile) continue;
    TileMap mi{}, mo{};
    MapGeom gi{}, go{};
    const int64_t nsub = q.nsub, C = q.C;
    if (q.lines_are_signals) {
      if (nsub < 16) continue;
      mi.kind = mo.kind = 1;
      mi.layout = mo.layout = 0;
    } else {
      const bool first = i == 0, last = i == p->passes - 1;
      const int64_t N1 = p->pp[0].nsub, M = p->n / N1;
      const int64_t rows = std::min<int64_t>(nsub, 256);
      auto em_box = [&](TileMap& m) {          // element-major [nsub][C] in boxes of <= 256 rows
        m.kind = 0; m.layout = 1;
        m.nbox = (int)((nsub + rows - 1) / rows);
        m.box_rows = (int)rows;
        m.box_elems = (int)(rows * C);
      };
      if (first) {
        em_box(mi); em_box(mo);
        mi.kind = mo.kind = 2;
        mi.ax = mo.ax = u; mi.by = mo.by = N1;
        gi.rank = 2; gi.dims[0] = M * u; gi.dims[1] = B * N1; gi.strides[0] = M * es;
        gi.box[0] = (uint32_t)(C * u); gi.box[1] = (uint32_t)rows;
        go = gi;
      } else if (!last) {                      // middle pass of three
        const int64_t N2 = nsub, N3 = q.LO;
        em_box(mi); em_box(mo);
        mi.kind = mo.kind = 3;
        mi.ax = mo.ax = u; mi.az = mo.az = 1; mi.bz = mo.bz = N1;
        gi.rank = 3; gi.dims[0] = N3 * u; gi.dims[1] = N2; gi.dims[2] = B * N1;
        gi.strides[0] = N3 * es; gi.strides[1] = M * es;
        gi.box[0] = (uint32_t)(C * u); gi.box[1] = (uint32_t)rows; gi.box[2] = 1;
        go = gi;
      } else if (p->passes == 2) {
        const int64_t N2 = nsub;
        const int64_t S = std::min<int64_t>(N2, 256 / u);   // row split for the box limit
        mi.kind = 3; mi.layout = 0; mi.nbox = 1; mi.bz = N1; mi.cz = 1;
        gi.rank = 3; gi.dims[0] = S * u; gi.dims[1] = N2 / S; gi.dims[2] = B * N1;
        gi.strides[0] = S * es; gi.strides[1] = N2 * es;
        gi.box[0] = (uint32_t)(S * u); gi.box[1] = (uint32_t)(N2 / S); gi.box[2] = (uint32_t)C;
        em_box(mo);
        mo.kind = 2; mo.ax = u; mo.by = N2;
        go.rank = 2; go.dims[0] = N1 * u; go.dims[1] = B * N2; go.strides[0] = N1 * es;
        go.box[0] = (uint32_t)(C * u); go.box[1] = (uint32_t)rows;
      } else {                                 // last pass of three
        const int64_t N3 = nsub, N2 = q.HI;
        mi.kind = 3; mi.layout = 0; mi.nbox = 1; mi.ay = 1; mi.bz = N1; mi.cz = 1;
        gi.rank = 3; gi.dims[0] = N3 * u; gi.dims[1] = N2; gi.dims[2] = B * N1;
        gi.strides[0] = N3 * es; gi.strides[1] = M * es;
        gi.box[0] = (uint32_t)(N3 * u); gi.box[1] = 1; gi.box[2] = (uint32_t)C;
        mo.kind = 3; mo.layout = 1; mo.nbox = 1; mo.box_rows = (int)N3; mo.box_elems = (int)(N3 * C);
        mo.ax = u; mo.ay = 1; mo.bz = N3;
        go.rank = 3; go.dims[0] = N1 * u; go.dims[1] = N2; go.dims[2] = B * N3;
        go.strides[0] = N1 * es; go.strides[1] = N1 * N2 * es;
        go.box[0] = (uint32_t)(C * u); go.box[1] = 1; go.box[2] = (uint32_t)N3;
      }
      if (!geom_ok(gi) || !geom_ok(go)) continue;
    }
    mi.bytes = mo.bytes = (unsigned)(C * nsub * es);
    mi.nbx = mo.nbx = 1;
    if (mi.nbox < 1) mi.nbox = 1;
    if (mo.nbox < 1) mo.nbox = 1;
    q.map_in = mi; q.map_out = mo; q.gin = gi; q.gout = go;
    q.buf_bytes = (unsigned)((C * nsub * es + 1023) / 1024 * 1024);
    const size_t budget = 218 * 1024 - 1024;
    q.nbuf = (int)std::min<size_t>(6, budget / (q.buf_bytes + 8));
    if (q.nbuf < 2) continue;
    q.tsmem = (size_t)q.nbuf * q.buf_bytes + (size_t)q.nbuf * 8 + 1024;
    cudaError_t e = p->dtype == TFFT_C64 ? tile_func_attrs_f32(q.E, q.tsmem, q.nthreads, &q.tbps)
                                         : tile_func_attrs_f64(q.E, q.tsmem, q.nthreads, &q.tbps);
    if (e != cudaSuccess) return cuda_fail(e);
    if (q.tbps < 1) continue;
    q.tma = 1;
  }
  return 0;
}

// The v3 kernel (compile-time geometry, warp-local lines) for every pass it
// has an instantiation for: 256 threads x E values per tile (E = 16 for
// complex64, 8 for complex128), element-major boxes split into column groups
// of at most 128 bytes per row and moved with the matching TMA swizzle.
int plan_v3(tfft_plan_s* p) {
  if (!encode_fn()) return 0;
  const bool c64 = p->dtype == TFFT_C64;
  const int64_t u = (int64_t)p->esize / 8, es = (int64_t)p->esize;
  const int vdt = c64 ? 0 : 1;
  const int vtc = p->prec == TFFT_PREC_TF32X3 ? 3
                : p->prec == TFFT_PREC_BF16X3 ? 2 : (p->prec == TFFT_PREC_TF32 ? 1 : 0);
  const int64_t B = p->batch;
  // one pass on the v3 kernel of `nt` threads (tiles of nt E values); false
  // when that kernel has no instantiation for the pass or its tiles do not fit
  auto try_v3 = [&](int i, int nt) -> bool {
    PassPlan& q = p->pp[i];
    const int64_t nsub = q.nsub;
    const int64_t E = v3_radix(vdt, (int)nsub);
    const int64_t TILE = nt * E;
    const bool wide = nt == 512;
    const int role = q.lines_are_signals ? 0 : (i == p->passes - 1 ? 2 : 1);
    const int64_t C = TILE / nsub;
    if (C < 1 || TILE % nsub) return false;
    if (role == 0 && (C > p->G || p->G % C)) return false;
    if (role != 0 && (C > q.LO || q.LO % C)) return false;
    // chunk indices are 32-bit in the v3 kernels (chunks <= groups x line blocks x G)
    if (p->ngroups * (q.lines_are_signals ? 1 : q.LO * q.HI / C) * (int64_t)p->G >= (int64_t(1) << 31)) return false;
    int bps = 0;
    auto attrs = [&](size_t sm, int* b) {
      if (wide) return v3_attrs_wide(role, (int)nsub, sm, b);
      return vtc ? v3_attrs_tc(vtc, role, (int)nsub, sm, b) : v3_attrs(vdt, role, (int)nsub, sm, b);
    };
    if (attrs(48 * 1024, &bps) != cudaSuccess) { cudaGetLastError(); return false; }
    TileMap mi{}, mo{};
    MapGeom gi = q.gin, go = q.gout;
    const int64_t rows = std::min<int64_t>(nsub, 256);
    const int64_t CS = std::min<int64_t>(C, 128 / es);
    const int rowb = (int)(CS * es);
    const int swz = rowb >= 128 ? (int)CU_TENSOR_MAP_SWIZZLE_128B
                  : rowb >= 64 ? (int)CU_TENSOR_MAP_SWIZZLE_64B
                  : rowb >= 32 ? (int)CU_TENSOR_MAP_SWIZZLE_32B : (int)CU_TENSOR_MAP_SWIZZLE_NONE;
    auto em = [&](TileMap& m, MapGeom& g) {
      m.layout = 1;
      m.nbox = (int)((nsub + rows - 1) / rows); m.box_rows = (int)rows; m.box_elems = (int)(rows * CS);
      m.nbx = (int)(C / CS); m.bx_step = (int)(CS * u); m.bx_elems = (int)(nsub * CS);
      g.box[0] = (uint32_t)(CS * u);
      g.swizzle = swz;
    };
    const int64_t N1 = p->pp[0].nsub, M = p->n / N1;
    if (role == 0) {
      if (nsub * es % 16) return false;
      mi.kind = mo.kind = 1; mi.layout = mo.layout = 0; mi.nbox = mo.nbox = 1; mi.nbx = mo.nbx = 1;
      gi = MapGeom{}; go = MapGeom{};
    } else if (role == 1) {
      const bool first = i == 0;
      mi.kind = mo.kind = first ? 2 : 3;
      mi.ax = mo.ax = u;
      if (first) {
        mi.by = mo.by = N1;
        gi = MapGeom{}; gi.rank = 2; gi.dims[0] = M * u; gi.dims[1] = B * N1; gi.strides[0] = M * es;
        gi.box[1] = (uint32_t)rows;
      } else {
        const int64_t N3 = q.LO;
        mi.az = mo.az = 1; mi.bz = mo.bz = N1;
        gi = MapGeom{}; gi.rank = 3; gi.dims[0] = N3 * u; gi.dims[1] = nsub; gi.dims[2] = B * N1;
        gi.strides[0] = N3 * es; gi.strides[1] = M * es; gi.box[1] = (uint32_t)rows; gi.box[2] = 1;
      }
      em(mi, gi);
      go = gi;
      em(mo, go);
    } else {
      // input: C rows of the line, line-major (rows split in runs of <= 256 units)
      mi = TileMap{};
      mi.kind = 3; mi.layout = 0; mi.nbox = 1; mi.nbx = 1;
      gi = MapGeom{};
      if (p->passes == 2) {
        const int64_t S = std::min<int64_t>(nsub, 256 / u);
        mi.bz = N1; mi.cz = 1;
        gi.rank = 3; gi.dims[0] = S * u; gi.dims[1] = nsub / S; gi.dims[2] = B * N1;
        gi.strides[0] = S * es; gi.strides[1] = nsub * es;
        gi.box[0] = (uint32_t)(S * u); gi.box[1] = (uint32_t)(nsub / S); gi.box[2] = (uint32_t)C;
      } else {
        const int64_t N2 = q.HI;
        if (nsub * u > 256) return false;
        mi.ay = 1; mi.bz = N1; mi.cz = 1;
        gi.rank = 3; gi.dims[0] = nsub * u; gi.dims[1] = N2; gi.dims[2] = B * N1;
        gi.strides[0] = nsub * es; gi.strides[1] = M * es;
        gi.box[0] = (uint32_t)(nsub * u); gi.box[1] = 1; gi.box[2] = (uint32_t)C;
      }
      if (p->passes == 2) {
        mo.kind = 2; mo.ax = u; mo.by = nsub;
        go = MapGeom{}; go.rank = 2; go.dims[0] = N1 * u; go.dims[1] = B * nsub; go.strides[0] = N1 * es;
        go.box[1] = (uint32_t)rows;
      } else {
        const int64_t N3 = nsub, N2 = q.HI;
        mo.kind = 3; mo.ax = u; mo.ay = 1; mo.bz = N3;
        go = MapGeom{}; go.rank = 3; go.dims[0] = N1 * u; go.dims[1] = N2; go.dims[2] = B * N3;
        go.strides[0] = N1 * es; go.strides[1] = N1 * N2 * es; go.box[1] = 1; go.box[2] = (uint32_t)rows;
        // element-major rows along z for the three-pass output: one box of nsub rows
        if (nsub > 256) return false;
      }
      em(mo, go);
    }
    if (role != 0 && (!geom_ok(gi) || !geom_ok(go))) return false;
    mi.bytes = mo.bytes = (unsigned)(C * nsub * es);
    const size_t scr = wide ? (size_t)v3_wide_scratch_bytes((int)nsub) : (size_t)v3_scratch_bytes(vdt, (int)nsub);
    const unsigned buf = (unsigned)((C * nsub * es + 1023) / 1024 * 1024);
    // complex64 (and the tensor-core forms whose operands sit in the line
    // scratch): two blocks per SM, each with at most 110 KB of dynamic
    // shared memory; complex128 and the split-TF32 form (separate operands):
    // one block per SM
    const size_t fixed = scr + (size_t)v3_twiddle_smem_bytes(vdt, (int)nsub) + (size_t)v3_tc_bytes(vtc) + 1024 + 1024;
    size_t budget = (c64 && !wide && (vtc == 0 || v3_tc_two_blocks(vtc)) ? 110 : 220) * 1024;
    if (vtc && fixed + 2 * (size_t)buf > budget) budget = 220 * 1024;   // one block per SM
    if (fixed + 2 * (size_t)buf > budget) return false;
    const int nbuf = (int)std::min<size_t>(4, (budget - fixed) / buf);
    const size_t smem = (size_t)nbuf * buf + fixed;
    if (attrs(smem, &bps) != cudaSuccess || bps < 1) { cudaGetLastError(); return false; }
    // the occupancy query reports one block of the scratch-aliased
    // tensor-core forms per SM; their registers (128) and shared memory
    // (two blocks of at most 110 KB plus 2 KB of static and reserved
    // memory in 228 KB) hold two, which the launch statistics confirm
    if (vtc && v3_tc_two_blocks(vtc) && bps == 1 && budget <= 110 * 1024 && 2 * (smem + 2048) <= 228 * 1024)
      bps = 2;
    q.v3 = 1; q.role = role; q.tma = 1; q.vdt = vdt; q.vtc = vtc;
    q.vC = (int)C;
    q.vLB = q.lines_are_signals ? 1 : q.LO * q.HI / C;
    q.map_in = mi; q.map_out = mo; q.gin = gi; q.gout = go;
    q.nbuf = nbuf; q.buf_bytes = buf; q.tsmem = smem; q.tbps = bps; q.vnt = nt;
    return true;
  };
  for (int i = 0; i < p->passes; i++) {
    const PassPlan& q = p->pp[i];
    const int role = q.lines_are_signals ? 0 : (i == p->passes - 1 ? 2 : 1);
    if (q.no_tile) {                   // the 256-thread v3 tile, else the direct-load kernel
      try_v3(i, 256);
      continue;
    }
    // complex64 column and last passes of 1024 and 2048 points: the
    // 512-thread tiles (twice the lines, twice the row bytes) first; 512-point
    // passes run faster on the 256-thread tiles (two blocks per SM): 0.89
    // against 0.94 ms (column) and 0.94 against 0.96 ms (last) at 2^28
    // elements.  The caller's tile_threads reorders the two.
    const bool wide = c64 && !vtc && role != 0 && q.nsub >= 512 && q.nsub <= 2048;
    const bool wide_first = wide && (p->tile_threads == 512 || (p->tile_threads == 0 && q.nsub >= 1024));
    if (wide_first && try_v3(i, 512)) continue;
    if (try_v3(i, 256)) continue;
    if (wide && !wide_first) try_v3(i, 512);
  }
  return 0;
}

int plan_tables(tfft_plan_s* p) {
  const int64_t n = p->n;
  int rc;
  // stage twiddles: omega_T^m, T = the longest sub-transform
  int T = 1;
  for (int i = 0; i < p->passes; i++) T = std::max(T, p->pp[i].nsub);
  p->tw_sub_n = T;
  {
    std::vector<double> re(T), im(T);
    for (int m = 0; m < T; m++) unit_root(m, T, &re[m], &im[m]);
    if ((rc = upload(p, &p->tw_sub, re, im))) return rc;
  }
  // v3 stage twiddles: for stages st = 1 .. S-1 (radix E, Ns = R0 E^(st-1)),
  // omega_{Ns E}^(q kk) for q = 1 .. E-1, kk < Ns, laid out [q-1][kk]
  for (int i = 0; i < p->passes; i++) {
    PassPlan& q = p->pp[i];
    if (!q.v3) continue;
    const int E = v3_radix(p->dtype == TFFT_C64 ? 0 : 1, q.nsub);
    int S = 0;
    for (int64_t v = 1; v < q.nsub; v *= E) S++;
    S = std::max(S, 1);
    int64_t EP = 1;
    for (int k = 0; k < S - 1; k++) EP *= E;
    const int64_t R0 = q.nsub / EP;
    std::vector<double> re, im;
    int64_t Ns = R0;
    for (int st = 1; st < S; st++, Ns *= E)
      for (int qq = 1; qq < E; qq++)
        for (int64_t kk = 0; kk < Ns; kk++) {
          double a, b;
          unit_root((qq * kk) % (Ns * E), Ns * E, &a, &b);
          re.push_back(a); im.push_back(b);
        }
    if (re.empty()) { re.push_back(1.0); im.push_back(0.0); }
    if ((rc = upload(p, &q.vtw, re, im))) return rc;
  }
  // omega_N^m two-level table (inter-pass twiddles)
  {
    const int lb = (ilog2(n) + 1) / 2;
    p->twN_lbits = lb;
    const int64_t L = int64_t(1) << lb, H = std::max<int64_t>(1, (n + L - 1) / L);
    std::vector<double> re(L), im(L), hre(H), him(H);
    for (int64_t m = 0; m < L; m++) unit_root(m, n, &re[m], &im[m]);
    for (int64_t h = 0; h < H; h++) unit_root(h * L, n, &hre[h], &him[h]);
    if ((rc = upload(p, &p->twN_lo, re, im))) return rc;
    if ((rc = upload(p, &p->twN_hi, hre, him))) return rc;
  }
  // e^{i pi m / (3N)}, 0 <= m <= 3N/2 (checksum weights), two-level
  {
    const int64_t mmax = 3 * n / 2 + 1;
    const int lb = (ilog2(mmax) + 1) / 2;
    p->wt_lbits = lb;
    const int64_t L = int64_t(1) << lb, H = (mmax + L - 1) / L + 1;
    const double pi = 3.14159265358979323846264338327950288;
    std::vector<double> re(L), im(L), hre(H), him(H);
    for (int64_t m = 0; m < L; m++) {
      const double a = pi * (double)m / (3.0 * (double)n);
      re[m] = std::cos(a); im[m] = std::sin(a);
    }
    for (int64_t h = 0; h < H; h++) {
      const double a = pi * (double)(h * L) / (3.0 * (double)n);
      hre[h] = std::cos(a); him[h] = std::sin(a);
    }
    if ((rc = upload(p, &p->wt_lo, re, im))) return rc;
    if ((rc = upload(p, &p->wt_hi, hre, him))) return rc;
  }
  return 0;
}

// w = W r for the signed e_Wang vector, computed on the device by an
// internal complex128 plan of the same length (FP64 accurate), then rounded
// to the plan's element type.
int plan_wtable(tfft_plan_s* p) {
  if (!p->abft || p->rvec != RVEC_SIGNED_WANG) return 0;
  const int64_t n = p->n;
  void* r = nullptr; void* w = nullptr;
  TFFT_CUDA(cudaMalloc(&r, n * 16));
  TFFT_CUDA(cudaMalloc(&w, n * 16));
  cudaError_t e = launch_gen_signs(r, n, p->rseed, nullptr);
  if (e != cudaSuccess) { cudaFree(r); cudaFree(w); return cuda_fail(e); }
  tfft_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  o.n = n; o.batch = 1; o.dtype = TFFT_C128; o.abft_mode = TFFT_ABFT_OFF;
  tfft_plan_t q = nullptr;
  int rc = tfft_plan_ex(&q, &o);
  if (!rc) rc = tfft_exec(q, r, w, nullptr);
  if (!rc) {
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (q) tfft_destroy(q);
  cudaFree(r);
  if (rc) { cudaFree(w); return rc; }
  if (p->dtype == TFFT_C64) {
    void* w32 = nullptr;
    e = cudaMalloc(&w32, n * 8);
    if (e == cudaSuccess) e = launch_c128_to_c64(w, w32, n, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    cudaFree(w);
    if (e != cudaSuccess) { if (w32) cudaFree(w32); return cuda_fail(e); }
    p->wtab = w32;
    p->workspace_bytes += n * 8;
  } else {
    p->wtab = w;
    p->workspace_bytes += n * 16;
  }
  return 0;
}

// u2 for the second check across the last pass: r2_k = r_k w3^floor(E k / N)
// with E the radix of the last stage, 16 (complex64) or 8 (complex128): the
// checksum vector times a phase that steps with the top bits of k.  On the E
// outputs of a last-stage butterfly r2 is r times w3^(q mod 3), so a fault
// confined to them is seen through two sums of the same random signs at
// frequencies a third of a cycle apart (correlated by 1/16 and 1/8); the
// last pass maps its input line with
// output offset L (a class of k modulo M = N / n_last) to the outputs
// L + M k by an n_last-point DFT, so u2[L][n] = sum_k r2[L + M k] w_nl^(n k):
// the classes gathered into rows and transformed by the library's own
// complex128 path, then rounded to the plan's element type.
void make_checks(tfft_plan_s* p, const void* in, void* out, int64_t b0, int64_t nb, VerifyParams& v,
                 FixParams& f);

// Fused verification and correction: single-pass plans with per-signal
// records whose groups one block verifies in a few rounds (at most
// kFuseGroups groups, few records a signal) let the pass kernel's last block
// verify a whole-batch exec and correct the groups it queued (one N-point
// transform in the block's tile ring per group) -- a clean exec is one
// kernel launch.
constexpr int64_t kFuseGroups = 64;
int plan_fused(tfft_plan_s* p) {
  const PassPlan& q = p->pp[0];
  const bool want = p->abft && p->sigrec && p->passes == 1 && q.v3 && q.role == 0 &&
                    p->vgroups <= kFuseGroups && p->sig_split == 0 && p->sig_blk_lanes == 0 &&
                    (int64_t)q.nbuf * q.buf_bytes >= p->n * (int64_t)p->esize && p->n <= 4096 &&
                    p->tw_sub_n == p->n;
  if (!want) return 0;
  VerifyParams v{};
  FixParams f{};
  make_checks(p, nullptr, nullptr, 0, p->batch, v, f);
  v.cond_flag = nullptr;
  TFFT_CUDA(cudaMalloc(&p->fdone, sizeof(unsigned)));
  TFFT_CUDA(cudaMemset(p->fdone, 0, sizeof(unsigned)));
  TFFT_CUDA(cudaMalloc(&p->fverify, sizeof(VerifyParams)));
  TFFT_CUDA(cudaMemcpy(p->fverify, &v, sizeof(VerifyParams), cudaMemcpyHostToDevice));
  p->workspace_bytes += (int64_t)(sizeof(unsigned) + sizeof(VerifyParams));
  p->fuse = 1;
  return 0;
}

int plan_ltab(tfft_plan_s* p) {
  if (!p->chk2) return 0;
  const int64_t n = p->n, nl = p->pp[p->passes - 1].nsub, M = n / nl;
  void* r = nullptr; void* g = nullptr; void* u = nullptr;
  cudaError_t e = cudaMalloc(&r, n * 16);
  if (e == cudaSuccess) e = cudaMalloc(&g, n * 16);
  if (e == cudaSuccess) e = cudaMalloc(&u, n * 16);
  if (e == cudaSuccess)
    e = launch_gen_signs(r, n, p->rseed, nullptr, p->dtype == TFFT_C64 ? 16 : 8, p->rvec == RVEC_SIGNED_WANG ? 1 : 0);
  if (e == cudaSuccess) e = launch_gather_classes(r, g, M, nl, nullptr);
  int rc = e == cudaSuccess ? 0 : cuda_fail(e);
  tfft_plan_t q = nullptr;
  if (!rc) {
    tfft_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.n = nl; o.batch = M; o.dtype = TFFT_C128; o.abft_mode = TFFT_ABFT_OFF;
    rc = tfft_plan_ex(&q, &o);
  }
  if (!rc) rc = tfft_exec(q, g, u, nullptr);
  if (!rc) {
    e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (q) tfft_destroy(q);
  cudaFree(r);
  cudaFree(g);
  if (rc) { if (u) cudaFree(u); return rc; }
  if (p->dtype == TFFT_C64) {
    void* u32 = nullptr;
    e = cudaMalloc(&u32, n * 8);
    if (e == cudaSuccess) e = launch_c128_to_c64(u, u32, n, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    cudaFree(u);
    if (e != cudaSuccess) { if (u32) cudaFree(u32); return cuda_fail(e); }
    p->ltab = u32;
    p->workspace_bytes += n * 8;
  } else {
    p->ltab = u;
    p->workspace_bytes += n * 16;
  }
  return 0;
}

int plan_workspace(tfft_plan_s* p) {
  const size_t sig = (size_t)p->n * p->esize;
  // correction slots: at most 8, within a 1 GiB budget for c1 and the partial sum
  if (p->cap_fix <= 0) {
    int64_t cap = (int64_t(1) << 30) / (int64_t)(2 * sig);
    p->cap_fix = (int)std::max<int64_t>(1, std::min<int64_t>(8, cap));
  }
  p->cap_fix = (int)std::min<int64_t>(p->cap_fix, std::max<int64_t>(1, p->vgroups));
  p->cap_rec = (int)std::min<int64_t>(8, std::max<int64_t>(1, p->vgroups));
  if (p->passes > 1) {
    const int64_t rows = std::max<int64_t>(p->batch, p->abft ? p->cap_fix : 0);
    TFFT_CUDA(cudaMalloc(&p->tmp, rows * sig));
    p->workspace_bytes += rows * (int64_t)sig;
  }
  const size_t nl = (size_t)(3 + p->cap_fix + p->cap_fix + p->cap_rec);
  TFFT_CUDA(cudaMalloc(&p->lists_mem, nl * sizeof(long long)));
  TFFT_CUDA(cudaMemset(p->lists_mem, 0, nl * sizeof(long long)));
  p->lists.fix = p->lists_mem;
  p->lists.fix_signal = p->lists_mem + 1 + p->cap_fix;
  p->lists.rec = p->lists_mem + 1 + 2 * p->cap_fix;
  p->lists.cap_fix = p->cap_fix;
  p->lists.cap_rec = p->cap_rec;
  p->cond_flag = p->lists_mem + nl - 1;
  TFFT_CUDA(cudaMalloc(&p->err_flag, sizeof(int)));
  TFFT_CUDA(cudaMemset(p->err_flag, 0, sizeof(int)));
  TFFT_CUDA(cudaMalloc(&p->counters, sizeof(Counters)));
  TFFT_CUDA(cudaMemset(p->counters, 0, sizeof(Counters)));
  TFFT_CUDA(cudaMalloc(&p->log, sizeof(LogEvent) * kLogRing));
  TFFT_CUDA(cudaMemset(p->log, 0, sizeof(LogEvent) * kLogRing));
  p->workspace_bytes += nl * sizeof(long long) + sizeof(Counters) + sizeof(LogEvent) * kLogRing;
  if (p->abft && p->sigrec) {
    const size_t rin = p->dtype == TFFT_C64 ? sizeof(SigIn<float>) : sizeof(SigIn<double>);
    const size_t rout = p->dtype == TFFT_C64 ? sizeof(SigOut<float>) : sizeof(SigOut<double>);
    TFFT_CUDA(cudaMalloc(&p->sig_in, rin * (size_t)p->batch * (size_t)p->sslots_in));
    TFFT_CUDA(cudaMalloc(&p->sig_out, rout * (size_t)p->batch * (size_t)p->sslots_out));
    p->workspace_bytes += (int64_t)(rin * p->batch * p->sslots_in + rout * p->batch * p->sslots_out);
    if (p->chk2) {
      const size_t rc2 = p->dtype == TFFT_C64 ? sizeof(SigChk<float>) : sizeof(SigChk<double>);
      TFFT_CUDA(cudaMalloc(&p->sig_chk, rc2 * (size_t)p->batch * (size_t)p->sslots_out));
      p->workspace_bytes += (int64_t)(rc2 * p->batch * p->sslots_out);
    }
    p->sig_split = sig_split_of(p->sslots_in + p->sslots_out * (p->chk2 ? 3 : 1), p->batch, p->sms);
    // many signals of a few dozen to a few hundred records: one block per
    // unit of groups, decided in shared memory (no per-signal atomics)
    if (p->sig_split > 0) {
      p->sig_blk_lanes = sig_block_geom(p->sslots_in, p->sslots_out, p->vG, p->vgroups, p->sms, &p->sig_gpb);
      if (p->sig_blk_lanes > 0) p->sig_split = 0;
    }
    if (p->sig_split > 0) {
      const size_t acc = (size_t)p->batch * kSigAcc * sizeof(double);
      TFFT_CUDA(cudaMalloc(&p->sig_acc, acc));
      TFFT_CUDA(cudaMemset(p->sig_acc, 0, acc));
      TFFT_CUDA(cudaMalloc(&p->part_cnt, (size_t)p->vgroups * sizeof(unsigned)));
      TFFT_CUDA(cudaMemset(p->part_cnt, 0, (size_t)p->vgroups * sizeof(unsigned)));
      p->workspace_bytes += (int64_t)(acc + (size_t)p->vgroups * sizeof(unsigned));
    }
    TFFT_CUDA(cudaMalloc(&p->ws_c1, p->cap_fix * sig));
    TFFT_CUDA(cudaMalloc(&p->ws_acc, p->cap_fix * sig));
    p->workspace_bytes += 2 * p->cap_fix * (int64_t)sig;
  } else if (p->abft) {
    TFFT_CUDA(cudaMalloc(&p->rec_in, sizeof(RecIn) * p->vgroups * p->slots_in));
    TFFT_CUDA(cudaMalloc(&p->rec_out, sizeof(RecOut) * p->vgroups * p->slots_out));
    p->vsplit = verify_split(p->slots_in + p->slots_out, p->vgroups, p->sms);
    if (p->vsplit > 1) {
      // accumulators start as zero sums, an empty nonfinite range, zero count
      std::vector<double> init((size_t)p->vgroups * kVerifyAcc, 0.0);
      for (int64_t g = 0; g < p->vgroups; g++) {
        const long long lo = 0x7fffffffffffffffLL, hi = -1;
        std::memcpy(&init[(size_t)g * kVerifyAcc + 9], &lo, sizeof(lo));
        std::memcpy(&init[(size_t)g * kVerifyAcc + 10], &hi, sizeof(hi));
      }
      TFFT_CUDA(cudaMalloc(&p->part_acc, init.size() * sizeof(double)));
      TFFT_CUDA(cudaMemcpy(p->part_acc, init.data(), init.size() * sizeof(double), cudaMemcpyHostToDevice));
      TFFT_CUDA(cudaMalloc(&p->part_cnt, (size_t)p->vgroups * sizeof(unsigned)));
      TFFT_CUDA(cudaMemset(p->part_cnt, 0, (size_t)p->vgroups * sizeof(unsigned)));
      p->workspace_bytes += (int64_t)(init.size() * sizeof(double) + (size_t)p->vgroups * sizeof(unsigned));
    }
    TFFT_CUDA(cudaMalloc(&p->ws_c1, p->cap_fix * sig));
    TFFT_CUDA(cudaMalloc(&p->ws_acc, p->cap_fix * sig));
    p->workspace_bytes += sizeof(RecIn) * p->vgroups * p->slots_in +
                          sizeof(RecOut) * p->vgroups * p->slots_out + 2 * p->cap_fix * (int64_t)sig;
  }
  return 0;
}

// ------------------------------------------------------------------ exec
PassParams base_params(const tfft_plan_s* p, int i) {
  const PassPlan& q = p->pp[i];
  PassParams a;
  std::memset(&a, 0, sizeof(a));
  a.nsub = q.nsub; a.log2nsub = ilog2(q.nsub); a.C = q.C; a.nthreads = q.nthreads;
  a.nstages = q.nstages; a.pitch = q.pitch; a.lines_are_signals = q.lines_are_signals;
  a.in_map = q.in_map; a.mid_map = q.mid_map; a.out_map = q.out_map; a.pass_index = i;
  a.n = p->n; a.batch = p->batch; a.LO = q.LO; a.HI = q.HI;
  a.in_es = q.in_es; a.in_lo = q.in_lo; a.in_hi = q.in_hi;
  a.out_es = q.out_es; a.out_lo = q.out_lo; a.out_hi = q.out_hi;
  a.tw_sub = p->tw_sub; a.tw_sub_stride = p->tw_sub_n / q.nsub;
  a.tw_stage = q.vtw;
  a.twiddle = q.twiddle; a.tw_scale = q.tw_scale;
  a.twN_lo = p->twN_lo; a.twN_hi = p->twN_hi; a.twN_lbits = p->twN_lbits;
  a.group = p->G; a.parts = q.parts; a.ngroups = p->ngroups; a.line_blocks = q.line_blocks;
  a.wt_lo = p->wt_lo; a.wt_hi = p->wt_hi; a.wt_lbits = p->wt_lbits;
  const int nmod3 = (int)(p->n % 3);          // K = 1 - w3^N, w3 = e^{-2 pi i/3}
  a.wk_re = 1.5;
  a.wk_im = nmod3 == 1 ? 0.86602540378443864676 : (nmod3 == 2 ? -0.86602540378443864676 : 0.0);
  if (nmod3 == 0) a.wk_re = 0.0;
  a.rvec = p->rvec; a.rseed = p->rseed; a.wtab = p->wtab;
  a.sigrec = p->sigrec;
  a.conj_in = p->inverse && i == 0;
  a.conj_out = p->inverse && i == p->passes - 1;
  a.out_scale = (p->normalize && i == p->passes - 1) ? 1.0 / (double)p->n : 1.0;
  a.nchunks = p->ngroups * q.parts * q.line_blocks;
  return a;
}

// The tile-copy parameters of pass i (buffers, bounded waits, tensor maps of
// a.in / a.out, encoded once per pointer) for a launch on the TMA kernels.
int prepare_tma(tfft_plan_s* p, PassParams& a, int i) {
  const PassPlan& q = p->pp[i];
  {
    a.nbuf = q.nbuf; a.buf_bytes = q.buf_bytes; a.err_flag = p->err_flag; a.wait_limit = p->wait_limit;
    a.map_in = q.map_in; a.map_out = q.map_out;
    const void* ptrs[2] = {a.in, a.out};
    const MapGeom* geo[2] = {&q.gin, &q.gout};
    const int kinds[2] = {q.map_in.kind, q.map_out.kind};
    for (int d = 0; d < 2; d++) {
      if (kinds[d] < 2) continue;
      if (p->enc_ptr[i][d] != ptrs[d]) {
        if (!encode_map(&p->enc_map[i][d], *geo[d], ptrs[d])) return TFFT_ERR_CUDA;
        p->enc_ptr[i][d] = ptrs[d];
      }
      (d == 0 ? a.tmap_in : a.tmap_out) = p->enc_map[i][d];
    }
  }
  return 0;
}

int launch_pass(tfft_plan_s* p, PassParams& a, int i, int kind, cudaStream_t s) {
  const PassPlan& q = p->pp[i];
  const bool tma = q.tma && a.list == nullptr;
  if (tma) {
    const int rc = prepare_tma(p, a, i);
    if (rc) return rc;
  }
  const int64_t maxgrid = (int64_t)p->sms * (tma ? q.tbps : q.bps);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(a.nchunks, maxgrid));
  const bool v3 = tma && q.v3;
  TimedLaunch tl{};
  if (p->timing) {
    tl.kind = kind;
    TFFT_CUDA(cudaEventCreate(&tl.a)); TFFT_CUDA(cudaEventCreate(&tl.b));
    TFFT_CUDA(cudaEventRecord(tl.a, s));
  }
  cudaError_t e;
  if (v3)
    e = q.vnt == 512 ? launch_v3_wide(q.role, q.nsub, a, grid, q.tsmem, s)
        : q.vtc      ? launch_v3_tc(q.vtc, q.role, q.nsub, a, grid, q.tsmem, s)
                     : launch_v3(q.vdt, q.role, q.nsub, a, grid, q.tsmem, s);
  else if (tma)
    e = p->dtype == TFFT_C64 ? launch_tile_f32(a, q.E, grid, q.tsmem, s) : launch_tile_f64(a, q.E, grid, q.tsmem, s);
  else
    e = p->dtype == TFFT_C64 ? launch_pass_f32(a, q.E, grid, q.smem, s) : launch_pass_f64(a, q.E, grid, q.smem, s);
  if (e != cudaSuccess) return cuda_fail(e);
  p->launches++;
  if (p->timing) {
    TFFT_CUDA(cudaEventRecord(tl.b, s));
    p->timed.push_back(tl);
  }
  return 0;
}

template <typename F>
int timed_launch(tfft_plan_s* p, int kind, cudaStream_t s, F&& f) {
  TimedLaunch tl{};
  if (p->timing) {
    tl.kind = kind;
    TFFT_CUDA(cudaEventCreate(&tl.a)); TFFT_CUDA(cudaEventCreate(&tl.b));
    TFFT_CUDA(cudaEventRecord(tl.a, s));
  }
  cudaError_t e = f();
  if (e != cudaSuccess) return cuda_fail(e);
  p->launches++;
  if (p->timing) {
    TFFT_CUDA(cudaEventRecord(tl.b, s));
    p->timed.push_back(tl);
  }
  return 0;
}

int kind_of(const tfft_plan_s* p, int i) {
  if (p->passes == 1) return 3;
  if (i == 0) return 0;
  return i == p->passes - 1 ? 2 : 1;
}

PassParams main_params(tfft_plan_s* p, int i, const void* in, void* out, int64_t batch, bool user_io,
                       int64_t vgroup0);

// Run the passes from `in` to `out` (through tmp when there are several).
int run_passes(tfft_plan_s* p, const void* in, void* out, cudaStream_t s, bool main_exec,
               const long long* list, int list_identity, int list_cap, int64_t list_block,
               int64_t batch, int kind_override, bool user_io = true, int64_t vgroup0 = 0) {
  // an exec over the signals [b0, b0 + batch) of the plan (b0 = vgroup0 vG,
  // a multiple of G): `in` and `out` already point at signal b0, the records
  // of its verification groups start at group vgroup0
  for (int i = 0; i < p->passes; i++) {
    PassParams a = main_exec ? main_params(p, i, in, out, batch, user_io, vgroup0) : base_params(p, i);
    if (!main_exec) {
      a.batch = batch;
      a.in = (i == 0) ? in : p->tmp;
      a.out = (i == p->passes - 1) ? out : p->tmp;
      if (user_io) {
        a.soff_in = i == 0 ? p->soff : nullptr;
        a.soff_out = i == p->passes - 1 ? p->soff : nullptr;
      }
      a.list = list; a.list_identity = list_identity; a.list_cap = list_cap;
      a.list_block = list_block;
      a.ngroups = list_cap;
      a.parts = 1;
      a.nchunks = (int64_t)list_cap * p->pp[i].line_blocks;
    }
    int rc = launch_pass(p, a, i, kind_override >= 0 ? kind_override : kind_of(p, i), s);
    if (rc) return rc;
  }
  return 0;
}

// The parameters of pass i of an exec over signals [b0, b0 + batch) (b0 =
// vgroup0 vG; in and out already point at signal b0), before the tile-copy
// parameters.
PassParams main_params(tfft_plan_s* p, int i, const void* in, void* out, int64_t batch, bool user_io,
                       int64_t vgroup0) {
  const int64_t ng = (batch + p->G - 1) / p->G;
  PassParams a = base_params(p, i);
  a.batch = batch;
  a.in = (i == 0) ? in : p->tmp;
  a.out = (i == p->passes - 1) ? out : p->tmp;
  if (user_io) {
    a.soff_in = i == 0 ? p->soff : nullptr;
    a.soff_out = i == p->passes - 1 ? p->soff : nullptr;
  }
  a.ngroups = ng;
  a.nchunks = ng * p->pp[i].parts * p->pp[i].line_blocks;
  if (p->pp[i].v3) {
    const PassPlan& q = p->pp[i];
    a.C = q.vC; a.nthreads = q.vnt; a.line_blocks = q.vLB;
    a.nchunks = ng * q.parts * q.vLB;
    a.log2C = ilog2(q.vC); a.log2LO = ilog2(q.LO); a.log2LB = ilog2(q.vLB);
  }
  a.abft_in = p->abft && i == 0;
  a.abft_out = p->abft && i == p->passes - 1;
  a.slots = (i == 0) ? p->slots_in : p->slots_out;
  if (p->passes == 1) a.slots = p->slots_in;
  if (p->abft && p->sigrec) {
    // records of signal b0 = vgroup0 vG onwards
    const int64_t b0 = vgroup0 * p->vG;
    const size_t rin = p->dtype == TFFT_C64 ? sizeof(SigIn<float>) : sizeof(SigIn<double>);
    const size_t rout = p->dtype == TFFT_C64 ? sizeof(SigOut<float>) : sizeof(SigOut<double>);
    a.sig_in = static_cast<unsigned char*>(p->sig_in) + (size_t)b0 * p->sslots_in * rin;
    a.sig_out = static_cast<unsigned char*>(p->sig_out) + (size_t)b0 * p->sslots_out * rout;
    a.sig_slots = (i == 0) ? p->sslots_in : p->sslots_out;
    if (p->chk2 && i == p->passes - 1) {
      const size_t rc2 = p->dtype == TFFT_C64 ? sizeof(SigChk<float>) : sizeof(SigChk<double>);
      a.chk2 = 1;
      a.sig_chk = static_cast<unsigned char*>(p->sig_chk) + (size_t)b0 * p->sslots_out * rc2;
      a.ltab = p->ltab;
    }
  } else if (p->abft) {
    a.rec_in = p->rec_in + vgroup0 * p->slots_in;
    a.rec_out = p->rec_out + vgroup0 * p->slots_out;
  }
  a.fault = p->pending;
  for (int k = 0; k < 3; k++) a.fault_more[k] = p->pending_more[k];
  a.nfault = p->npending;
  if (i == 0 && p->abft) {
    a.zero_on_entry[0] = p->lists.fix;
    a.zero_on_entry[1] = p->lists.rec;
    a.zero_on_entry[2] = p->cond_flag;
  }
  // a whole-batch exec of a fused plan verifies in the pass kernel's last block
  if (p->fuse && vgroup0 == 0 && batch == p->batch) {
    a.fverify = p->fverify;
    a.fdone = p->fdone;
    a.exec_index = p->execs;
    a.pdl = p->pdl_now;
  }
  return a;
}

// The correction sequence (Section III-B) on `s`: gather the queued groups'
// input checksum and partial output sums, transform the checksums, recompute
// the groups that could not be located (other groups: no overlap with the
// gathered ones), then apply the located corrections, which also counts both
// kinds as done.  Every launch returns at once when its list is empty.
int enqueue_correction(tfft_plan_s* p, const FixParams& f, const void* in, void* out, int64_t nb,
                       cudaStream_t s) {
  int rc;
  if ((rc = timed_launch(p, 5, s, [&] { return launch_fix_gather(f, s); }))) return rc;
  // W X e_1 of every queued group, in place in ws_c1
  if ((rc = run_passes(p, p->ws_c1, p->ws_c1, s, false, p->lists.fix, 1, p->cap_fix, 1,
                       p->cap_fix, 5, false)))
    return rc;
  // groups that could not be located: recompute from the input
  if ((rc = run_passes(p, in, out, s, false, p->lists.rec, 0, p->cap_rec, p->vG, nb, 5))) return rc;
  return timed_launch(p, 5, s, [&] { return launch_fix_apply(f, s); });
}

// Builds the graph [verify] -> [if (a group was queued) { correction }] for
// this (in, out): the verification kernel switches the conditional node on
// (cudaGraphSetConditional) when it queues a group, so a clean exec runs one
// graph launch after its passes instead of the five to nine launches of the
// correction sequence.  Returns nonzero (and leaves no graph) on any failure.
int build_correction_graph(tfft_plan_s* p, VerifyParams v, const FixParams& f, const void* in, void* out,
                           bool full) {
  if (p->cgx) { cudaGraphExecDestroy(p->cgx); p->cgx = nullptr; }
  if (p->cg) { cudaGraphDestroy(p->cg); p->cg = nullptr; }
  if (!p->gcap && cudaStreamCreateWithFlags(&p->gcap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle h{};
  cudaGraphNode_t vnode = nullptr;
  cudaGraphNodeParams cp{};
  cudaGraph_t body = nullptr, out_g = nullptr;
  cudaGraphExec_t gx = nullptr;
  bool ok = cudaGraphCreate(&g, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    v.cond_flag = p->cond_flag;
    v.cond = h;
    ok = cudaStreamBeginCaptureToGraph(p->gcap, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      // the passes too (captured, not run: the plan's launch count and
      // timing records stay as they were)
      bool launched = true;
      if (full) {
        const int64_t launches = p->launches;
        const bool timing = p->timing;
        p->timing = false;
        const int fuse = p->fuse;
        p->fuse = 0;                      // the graph holds the separate verification kernel
        launched = run_passes(p, in, out, p->gcap, true, nullptr, 0, 0, 0, p->batch, -1, true, 0) == 0;
        p->fuse = fuse;
        p->timing = timing;
        p->launches = launches;
      }
      launched = launched && launch_verify(v, p->gcap) == cudaSuccess;
      // the node just captured is the verification kernel
      cudaStreamCaptureStatus st{};
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      if (launched && cudaStreamGetCaptureInfo(p->gcap, &st, nullptr, nullptr, &deps, nullptr, &ndeps) == cudaSuccess &&
          ndeps == 1)
        vnode = deps[0];
      ok = cudaStreamEndCapture(p->gcap, &out_g) == cudaSuccess && launched && vnode != nullptr;
    }
  }
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    ok = cudaGraphAddNode(&cn, g, &vnode, nullptr, 1, &cp) == cudaSuccess;
  }
  if (ok) {
    body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(p->gcap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) ==
         cudaSuccess;
    if (ok) {
      // captured, not run: keep the plan's launch count and timing records
      const int64_t launches = p->launches;
      const bool timing = p->timing;
      p->timing = false;
      const int rc = enqueue_correction(p, f, in, out, f.batch, p->gcap);
      p->timing = timing;
      p->launches = launches;
      cudaGraph_t b2 = nullptr;
      ok = cudaStreamEndCapture(p->gcap, &b2) == cudaSuccess && rc == 0;
    }
  }
  cudaKernelNodeParams kp{};
  ok = ok && cudaGraphKernelNodeGetParams(vnode, &kp) == cudaSuccess && kp.kernelParams;
  ok = ok && cudaGraphInstantiate(&gx, g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (gx) cudaGraphExecDestroy(gx);
    if (g) cudaGraphDestroy(g);
    return 1;
  }
  p->cg = g;
  p->cgx = gx;
  p->cg_vnode = vnode;
  p->cg_full = full;
  p->cg_kp = kp;
  p->cg_v = v;
  p->cg_lanes = *static_cast<int*>(kp.kernelParams[1]);
  p->cg_in = in;
  p->cg_out = out;
  return 0;
}

// The verification and correction parameters of an exec over signals
// [b0, b0 + nb) (in and out point at signal b0).
void make_checks(tfft_plan_s* p, const void* in, void* out, int64_t b0, int64_t nb, VerifyParams& v,
                 FixParams& f) {
  const int64_t vg0 = b0 / p->vG;
  v.n = p->n; v.batch = nb; v.group = p->vG; v.ngroups = (nb + p->vG - 1) / p->vG;
  v.group_base = vg0;
  v.slots_in = p->slots_in; v.slots_out = p->slots_out;
  v.rec_in = p->rec_in + vg0 * p->slots_in; v.rec_out = p->rec_out + vg0 * p->slots_out;
  // unit roundoff of the butterfly arithmetic: FP32, FP64, or the tensor-core forms
  const double u = p->dtype != TFFT_C64 ? std::ldexp(1.0, -53)
                 : p->prec == TFFT_PREC_TF32X3 ? std::ldexp(1.0, -20)
                 : p->prec == TFFT_PREC_TF32 ? std::ldexp(1.0, -10)
                 : p->prec == TFFT_PREC_BF16X3 ? std::ldexp(1.0, -17) : std::ldexp(1.0, -24);
  // tau = kappa u (log2 N + 4) sqrt(N) sqrt(E): the log2 N term follows the
  // rounding of the stages, the constant the fixed share of the checksum
  // arithmetic itself (table rounding, FP32 accumulation), which dominates
  // for very short transforms
  const int lg = ilog2(p->n) + 4;
  v.kappa_u_log2n_sqrtn = p->kappa * u * lg * std::sqrt((double)p->n);
  v.detect_only = p->detect_only;
  v.lists = p->lists; v.counters = p->counters; v.log = p->log; v.exec_index = p->execs;
  v.max_blocks = 8 * p->sms;
  v.split = p->vsplit; v.part_acc = p->part_acc; v.part_cnt = p->part_cnt;
  if (p->sigrec) {
    const int64_t b0s = vg0 * p->vG;
    const size_t rin = p->dtype == TFFT_C64 ? sizeof(SigIn<float>) : sizeof(SigIn<double>);
    const size_t rout = p->dtype == TFFT_C64 ? sizeof(SigOut<float>) : sizeof(SigOut<double>);
    v.sigrec = 1;
    v.dtype = p->dtype == TFFT_C64 ? 0 : 1;
    v.sig_in = static_cast<const unsigned char*>(p->sig_in) + (size_t)b0s * p->sslots_in * rin;
    v.sig_out = static_cast<const unsigned char*>(p->sig_out) + (size_t)b0s * p->sslots_out * rout;
    v.sig_slots_in = p->sslots_in; v.sig_slots_out = p->sslots_out;
    v.sig_split = p->sig_split;
    v.sig_blk_lanes = p->sig_blk_lanes; v.sig_gpb = p->sig_gpb;
    v.sig_acc = p->sig_acc ? p->sig_acc + b0s * kSigAcc : nullptr;
    v.part_cnt = p->part_cnt ? p->part_cnt + vg0 : nullptr;
    // a threshold never below that of signals whose every value is the
    // smallest normal number of the element type
    const double tiny = p->dtype == TFFT_C64 ? 1.1754943508222875e-38 : 2.2250738585072014e-308;
    v.tau_floor = v.kappa_u_log2n_sqrtn * std::sqrt((double)p->n) * tiny;
    if (p->chk2) {
      const size_t rc2 = p->dtype == TFFT_C64 ? sizeof(SigChk<float>) : sizeof(SigChk<double>);
      v.chk2 = 1;
      v.sig_chk = static_cast<const unsigned char*>(p->sig_chk) + (size_t)b0s * p->sslots_out * rc2;
      // the last pass alone: its n_last-point transform's rounding
      const int lgl = ilog2(p->pp[p->passes - 1].nsub) + 4;
      v.kappa_u_chk2 = p->kappa * u * lgl * std::sqrt((double)p->n);
    }
  }
  f.n = p->n; f.batch = nb; f.group = p->vG; f.dtype = p->dtype;
  f.in = in; f.out = out; f.soff = p->soff; f.ws_c1 = p->ws_c1; f.ws_acc = p->ws_acc; f.lists = p->lists;
  f.counters = p->counters; f.err_flag = p->err_flag;
}

// Which cached graph a whole-batch exec on a stream that is not being
// captured takes: 2 the whole exec (passes, verification, the conditional
// correction) when no per-kernel timing is on and `allow_full`; 1 the
// verification and correction only (after the passes' stream launches); 0
// none (stream launches).  A graph is built when a pair of buffers comes back
// (an exec that rotates over many buffers keeps the stream launches), and
// again when the kind it needs changes.  An exec with a test fault armed
// builds a whole-exec graph of its own (the fault sits in its pass nodes),
// and the next exec rebuilds the clean one.
int pick_graph(tfft_plan_s* p, const void* in, void* out, cudaStream_t s, int64_t b0, int64_t nb,
               const VerifyParams& v, const FixParams& f, bool allow_full) {
  if (!p->abft || b0 != 0 || nb != p->batch || p->cg_off) return 0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  bool capturing = true;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess) capturing = cs != cudaStreamCaptureStatusNone;
  else cudaGetLastError();        // e.g. the legacy stream during another thread's global capture
  if (capturing) return 0;
  const bool armed = p->npending > 0 || p->pending.mode != 0;
  const bool full = allow_full && !p->timing;
  // a fused plan's exec is its pass kernel alone (it verifies and corrects
  // in its last block): nothing to put in a graph
  if (p->fuse) return 0;
  const bool cached = p->cgx && p->cg_in == in && p->cg_out == out && p->cg_full == full &&
                      !(full && (armed || p->cg_armed));
  const bool again = p->last_in == in && p->last_out == out;
  p->last_in = in;
  p->last_out = out;
  if (cached) return full ? 2 : 1;
  if (!again) return 0;
  if (build_correction_graph(p, v, f, in, out, full)) {
    p->cg_off = true;
    return 0;
  }
  p->cg_armed = full && armed;
  return full ? 2 : 1;
}

// Launches the cached graph with this exec's index in the verification's
// fault-log entries (timed as one launch; the whole-exec graph counts its
// pass launches too).
int launch_graph(tfft_plan_s* p, cudaStream_t s) {
  VerifyParams v2 = p->cg_v;
  v2.exec_index = p->execs;
  int lanes = p->cg_lanes;
  void* args[2] = {&v2, &lanes};
  cudaKernelNodeParams kp = p->cg_kp;
  kp.kernelParams = args;
  TFFT_CUDA(cudaGraphExecKernelNodeSetParams(p->cgx, p->cg_vnode, &kp));
  if (p->cg_full) p->launches += p->passes;
  return timed_launch(p, 4, s, [&] { return cudaGraphLaunch(p->cgx, s); });
}

// The exec over signals [b0, b0 + nb) (b0 a multiple of G, nb > 0): the
// passes, the verification of their groups and the correction path, all on
// `s`, reading in + b0 n and writing out + b0 n.
int exec_range(tfft_plan_s* p, const void* in, void* out, cudaStream_t s, int64_t b0, int64_t nb) {
  const size_t off = (size_t)b0 * (size_t)p->n * p->esize;
  in = static_cast<const unsigned char*>(in) + off;
  out = static_cast<unsigned char*>(out) + off;
  const int64_t vg0 = b0 / p->vG;
  VerifyParams v{};
  FixParams f{};
  if (p->abft) make_checks(p, in, out, b0, nb, v, f);
  const int gk = pick_graph(p, in, out, s, b0, nb, v, f, true);
  if (gk == 2) return launch_graph(p, s);
  // a fused exec (one kernel) on a stream that is not being captured starts
  // its blocks' set-up while the kernel before it finishes
  if (p->fuse && b0 == 0 && nb == p->batch && !p->timing) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cudaGetLastError();
    p->pdl_now = cs == cudaStreamCaptureStatusNone;
  }
  int rc = run_passes(p, in, out, s, true, nullptr, 0, 0, 0, nb, -1, true, vg0);
  p->pdl_now = 0;
  if (rc) return rc;
  if (!p->abft) return 0;
  if (gk == 1) return launch_graph(p, s);
  // the pass kernel of a fused plan verified and corrected the whole batch
  if (p->fuse && b0 == 0 && nb == p->batch) return 0;
  if ((rc = timed_launch(p, 4, s, [&] { return launch_verify(v, s); }))) return rc;
  return enqueue_correction(p, f, in, out, nb, s);
}

// The verification and correction of an exec over signals [b0, b0 + nb)
// whose passes have been enqueued on `s` (in and out point at signal b0).
int exec_checks(tfft_plan_s* p, const void* in, void* out, cudaStream_t s, int64_t b0, int64_t nb) {
  if (!p->abft) return 0;
  VerifyParams v{};
  FixParams f{};
  make_checks(p, in, out, b0, nb, v, f);
  if (pick_graph(p, in, out, s, b0, nb, v, f, false) == 1) return launch_graph(p, s);
  int rc;
  if ((rc = timed_launch(p, 4, s, [&] { return launch_verify(v, s); }))) return rc;
  return enqueue_correction(p, f, in, out, nb, s);
}

int exec_device(tfft_plan_s* p, const void* in, void* out, cudaStream_t s) {
  return exec_range(p, in, out, s, 0, p->batch);
}

bool aligned16(const void* ptr) { return ((uintptr_t)ptr & 15u) == 0; }

}  // namespace

namespace tfft {

int plan_ragged_pass(tfft_plan_t p, int i, RaggedPass* rp) {
  if (!p || !rp || i < 0 || i >= p->passes) return TFFT_ERR_INVALID_ARG;
  const PassPlan& q = p->pp[i];
  *rp = RaggedPass{};
  rp->role = q.role;
  rp->nsub = q.nsub;
  rp->ok = p->dtype == TFFT_C64 && q.tma && q.v3 && q.vnt == 256 && q.vtc == 0 && v3_ragged_has(q.role, q.nsub);
  if (!rp->ok) return TFFT_SUCCESS;
  rp->smem = q.tsmem;
  const int64_t ng = (p->batch + p->G - 1) / p->G;
  rp->nchunks = ng * q.parts * q.vLB;
  const int64_t per_part = (p->G + q.parts - 1) / q.parts;
  rp->tiles_per_chunk = (int)std::max<int64_t>(1, q.role == 0 ? (per_part + q.vC - 1) / q.vC : per_part);
  return TFFT_SUCCESS;
}

int plan_pass_params(tfft_plan_t p, const void* in, void* out, int i, PassParams* a) {
  if (!p || !a || i < 0 || i >= p->passes) return TFFT_ERR_INVALID_ARG;
  *a = main_params(p, i, in, out, p->batch, true, 0);
  return prepare_tma(p, *a, i);
}

int plan_exec_checks(tfft_plan_t p, const void* in, void* out, cudaStream_t s) {
  if (!p) return TFFT_ERR_INVALID_ARG;
  return exec_checks(p, in, out, s, 0, p->batch);
}

void plan_exec_finish(tfft_plan_t p, cudaStream_t s) {
  p->pending = FaultSite{};     // armed faults last one exec
  for (auto& f : p->pending_more) f = FaultSite{};
  p->npending = 0;
  p->execs++;
  p->last_stream = s;
  p->used = true;
}

int plan_set_signal_offsets(tfft_plan_t p, const long long* d_off, const int64_t* h_off, int64_t total) {
  if (!p || !d_off || !h_off || total < p->n) return TFFT_ERR_INVALID_ARG;
  const int64_t es = (int64_t)p->esize, u = es / 8;
  for (int64_t b = 0; b < p->batch; b++)
    if (h_off[b] < 0 || h_off[b] > total - p->n) return TFFT_ERR_INVALID_ARG;
  // every signal on a 16-byte boundary: the bulk copies and the 16-byte
  // stores of the last pass need it
  for (int64_t b = 0; b < p->batch; b++)
    if ((h_off[b] * es) % 16) return TFFT_ERR_UNSUPPORTED;
  PassPlan& f = p->pp[0];
  PassPlan& l = p->pp[p->passes - 1];
  MapGeom g = f.gin;
  if (f.tma && f.map_in.kind >= 2) {
    // the first pass's column boxes: 2-D map over the packed buffer as rows of
    // M columns; an offset that is a multiple of the box width keeps each box
    // inside one row
    if (f.map_in.kind != 2 || g.rank != 2) return TFFT_ERR_UNSUPPORTED;
    const int64_t M = p->n / f.nsub, width = (int64_t)g.box[0] / u;
    if (width < 1 || M % width) return TFFT_ERR_UNSUPPORTED;
    for (int64_t b = 0; b < p->batch; b++)
      if (h_off[b] % width) return TFFT_ERR_UNSUPPORTED;
    g.dims[1] = (uint64_t)((total + M - 1) / M);
    if (!geom_ok(g) || g.dims[1] >= (uint64_t(1) << 31)) return TFFT_ERR_UNSUPPORTED;   // signed coordinates
  }
  // the last pass writes whole signals (bulk stores) or copies its boxes out
  // with plain stores; other store forms keep the contiguous layout
  if (l.tma && !(l.v3 && l.role == 2) && l.map_out.kind != 1) return TFFT_ERR_UNSUPPORTED;
  f.gin = g;
  p->enc_ptr[0][0] = nullptr;
  p->soff = d_off;
  return TFFT_SUCCESS;
}

// Builds a plan from the options as given (no autotuner table); `tuned`
// marks a plan whose pass configuration came from that table.
int plan_create(tfft_plan_t* out, const tfft_plan_opts* o, int tuned) {
  if (!out || !o) return TFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (!is_pow2(o->n) || o->n > (int64_t(1) << 29) || o->batch < 1) return TFFT_ERR_INVALID_ARG;
  if (o->dtype != TFFT_C64 && o->dtype != TFFT_C128) return TFFT_ERR_UNSUPPORTED;
  if (o->abft_mode != TFFT_ABFT_OFF && o->abft_mode != TFFT_ABFT_TWO_SIDED && o->abft_mode != TFFT_ABFT_ONE_SIDED)
    return TFFT_ERR_UNSUPPORTED;
  if (o->group < 0 || o->kappa < 0 || o->max_faults < 0 || o->force_passes < 0 || o->force_passes > 3)
    return TFFT_ERR_INVALID_ARG;
  if (o->checksum_vector != TFFT_R_SIGNED_WANG && o->checksum_vector != TFFT_R_WANG) return TFFT_ERR_INVALID_ARG;
  if ((o->direction != TFFT_FORWARD && o->direction != TFFT_INVERSE) || (o->normalize != 0 && o->normalize != 1))
    return TFFT_ERR_INVALID_ARG;
  if (o->precision < TFFT_PREC_FP32 || o->precision > TFFT_PREC_BF16X3) return TFFT_ERR_INVALID_ARG;
  if (o->wait_polls < -1 || o->first_pass_log2 < 0) return TFFT_ERR_INVALID_ARG;
  if (o->tile_threads != 0 && o->tile_threads != 256 && o->tile_threads != 512) return TFFT_ERR_INVALID_ARG;
  if (o->precision != TFFT_PREC_FP32 && o->dtype != TFFT_C64) return TFFT_ERR_UNSUPPORTED;
  int dev = 0, count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) return TFFT_ERR_NO_DEVICE;
  TFFT_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  TFFT_CUDA(cudaGetDeviceProperties(&prop, dev));
  if (!(prop.major == 10 && prop.minor == 3)) return TFFT_ERR_NO_DEVICE;

  tfft_plan_s* p = new (std::nothrow) tfft_plan_s();
  if (!p) return TFFT_ERR_ALLOC;
  p->n = o->n; p->batch = o->batch; p->dtype = o->dtype; p->abft = o->abft_mode != TFFT_ABFT_OFF;
  p->one_sided = o->abft_mode == TFFT_ABFT_ONE_SIDED;
  p->kappa = o->kappa > 0 ? o->kappa : 2.0;
  p->detect_only = o->detect_only ? 1 : 0;
  p->cap_fix = o->max_faults;
  p->rvec = o->checksum_vector == TFFT_R_WANG ? RVEC_WANG : RVEC_SIGNED_WANG;
  if (o->checksum_seed) p->rseed = (unsigned long long)o->checksum_seed;
  p->inverse = o->direction == TFFT_INVERSE;
  p->prec = o->precision;
  p->normalize = o->normalize;
  p->wait_limit = o->wait_polls == 0 ? (1ll << 20) : (o->wait_polls < 0 ? 0 : (long long)o->wait_polls);
  p->tile_threads = o->tile_threads;
  p->tuned = tuned;
  p->device = dev;
  p->sms = prop.multiProcessorCount;
  int rc = plan_build(p, o);
  if (!rc) rc = plan_tma(p);
  if (!rc) rc = plan_v3(p);
  if (!rc) plan_slots(p);
  if (!rc && (p->one_sided || p->prec != TFFT_PREC_FP32))
    for (int i = 0; i < p->passes; i++)
      if (!p->pp[i].v3) rc = TFFT_ERR_UNSUPPORTED;   // per-signal records and tensor cores live in the tile kernels
  if (!rc) rc = plan_tables(p);
  if (!rc) rc = plan_workspace(p);
  if (!rc) rc = plan_wtable(p);
  if (!rc) rc = plan_ltab(p);
  if (!rc) rc = plan_fused(p);
  if (rc) { free_plan(p); return rc; }
  *out = p;
  return TFFT_SUCCESS;
}

}  // namespace tfft

// =================================================================== C ABI
extern "C" {

int tfft_plan_ex(tfft_plan_t* out, const tfft_plan_opts* o) {
  if (!out || !o) return TFFT_ERR_INVALID_ARG;
  // options that leave the pass configuration to the planner take the
  // autotuner's entry for this transform when there is one; an entry the
  // planner does not admit (a cache file from another build) is passed over
  tfft_plan_opts t;
  if (!o->force_passes && !o->first_pass_log2 && !o->tile_threads && tune_lookup(o, &t) &&
      plan_create(out, &t, 1) == TFFT_SUCCESS)
    return TFFT_SUCCESS;
  return plan_create(out, o, 0);
}

int tfft_plan(tfft_plan_t* out, int64_t n, int64_t batch, int dtype, int abft_mode) {
  tfft_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  o.n = n; o.batch = batch; o.dtype = dtype; o.abft_mode = abft_mode;
  return tfft_plan_ex(out, &o);
}

int tfft_exec(tfft_plan_t p, const void* in, void* out, tfft_stream_t stream) {
  if (!p || !in || !out || !aligned16(in) || !aligned16(out)) return TFFT_ERR_INVALID_ARG;
  const size_t bytes = (size_t)p->batch * p->n * p->esize;
  const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
  if (p->abft && a < b + bytes && b < a + bytes) return TFFT_ERR_INPLACE;
  std::lock_guard<std::mutex> lk(p->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = exec_device(p, in, out, s);
  p->pending = FaultSite{};     // armed faults last one exec
  for (auto& f : p->pending_more) f = FaultSite{};
  p->npending = 0;
  p->execs++;
  p->last_stream = s;
  p->used = true;
  return rc;
}

int tfft_exec_host(tfft_plan_t p, const void* host_in, void* host_out, tfft_stream_t stream) {
  if (!p || !host_in || !host_out) return TFFT_ERR_INVALID_ARG;
  const size_t bytes = (size_t)p->batch * p->n * p->esize;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(p->mu);
  if (!p->stage_in) {
    TFFT_CUDA(cudaMalloc(&p->stage_in, bytes));
    TFFT_CUDA(cudaMalloc(&p->stage_out, bytes));
  }
  // Chunks of whole checksum groups, up to eight: the host-to-device copies
  // run back to back on one copy stream, each chunk's transform starts once
  // its input has landed, and its device-to-host copy overlaps the next
  // chunks' input copies and transforms (the link carries both directions at
  // once).  One chunk when a test fault is armed (its signal index is
  // relative to the whole batch) or the plan addresses signals by offsets.
  const int64_t ng = (p->batch + p->G - 1) / p->G;
  const bool armed = p->npending > 0 || p->pending.mode != 0;
  const int nch = (armed || p->soff) ? 1 : (int)std::min<int64_t>(8, ng);
  const size_t sig = (size_t)p->n * p->esize;
  int rc = 0;
  if (nch == 1) {
    TFFT_CUDA(cudaMemcpyAsync(p->stage_in, host_in, bytes, cudaMemcpyHostToDevice, s));
    rc = exec_range(p, p->stage_in, p->stage_out, s, 0, p->batch);
    if (!rc) TFFT_CUDA(cudaMemcpyAsync(host_out, p->stage_out, bytes, cudaMemcpyDeviceToHost, s));
  } else {
    if (!p->h2d) {
      TFFT_CUDA(cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking));
      TFFT_CUDA(cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking));
      TFFT_CUDA(cudaEventCreateWithFlags(&p->ev_entry, cudaEventDisableTiming));
      TFFT_CUDA(cudaEventCreateWithFlags(&p->ev_end, cudaEventDisableTiming));
      for (int c = 0; c < 8; c++) {
        TFFT_CUDA(cudaEventCreateWithFlags(&p->ev_in[c], cudaEventDisableTiming));
        TFFT_CUDA(cudaEventCreateWithFlags(&p->ev_done[c], cudaEventDisableTiming));
      }
    }
    const int64_t gpc = (ng + nch - 1) / nch;   // groups per chunk
    auto chunk = [&](int c, int64_t* b0, int64_t* nb) {
      *b0 = std::min<int64_t>(p->batch, (int64_t)c * gpc * p->G);
      *nb = std::min<int64_t>(p->batch, (int64_t)(c + 1) * gpc * p->G) - *b0;
    };
    // the copies start after whatever the caller queued on `s` before
    TFFT_CUDA(cudaEventRecord(p->ev_entry, s));
    TFFT_CUDA(cudaStreamWaitEvent(p->h2d, p->ev_entry, 0));
    TFFT_CUDA(cudaStreamWaitEvent(p->d2h, p->ev_entry, 0));
    for (int c = 0; c < nch; c++) {
      int64_t b0, nb;
      chunk(c, &b0, &nb);
      if (nb <= 0) continue;
      TFFT_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(p->stage_in) + b0 * sig,
                                static_cast<const unsigned char*>(host_in) + b0 * sig, (size_t)nb * sig,
                                cudaMemcpyHostToDevice, p->h2d));
      TFFT_CUDA(cudaEventRecord(p->ev_in[c], p->h2d));
    }
    for (int c = 0; c < nch && !rc; c++) {
      int64_t b0, nb;
      chunk(c, &b0, &nb);
      if (nb <= 0) continue;
      TFFT_CUDA(cudaStreamWaitEvent(s, p->ev_in[c], 0));
      rc = exec_range(p, p->stage_in, p->stage_out, s, b0, nb);
      if (rc) break;
      TFFT_CUDA(cudaEventRecord(p->ev_done[c], s));
      TFFT_CUDA(cudaStreamWaitEvent(p->d2h, p->ev_done[c], 0));
      TFFT_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(host_out) + b0 * sig,
                                static_cast<const unsigned char*>(p->stage_out) + b0 * sig, (size_t)nb * sig,
                                cudaMemcpyDeviceToHost, p->d2h));
    }
    // `s` (and so tfft_report) waits for the last copy; the copy streams for
    // each other before the next call reuses the staging buffers
    TFFT_CUDA(cudaEventRecord(p->ev_end, p->d2h));
    TFFT_CUDA(cudaStreamWaitEvent(s, p->ev_end, 0));
    TFFT_CUDA(cudaStreamWaitEvent(p->h2d, p->ev_end, 0));
  }
  p->pending = FaultSite{};
  for (auto& f : p->pending_more) f = FaultSite{};
  p->npending = 0;
  p->execs++;
  p->last_stream = s;
  p->used = true;
  if (rc) return rc;
  TFFT_CUDA(cudaStreamSynchronize(s));
  return TFFT_SUCCESS;
}

int tfft_report_ex(tfft_plan_t p, tfft_stats* st) {
  if (!p || !st) return TFFT_ERR_INVALID_ARG;
  if (p->used) TFFT_CUDA(cudaStreamSynchronize(p->last_stream));
  int err = 0;
  TFFT_CUDA(cudaMemcpy(&err, p->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) return TFFT_ERR_TIMEOUT;
  Counters c;
  TFFT_CUDA(cudaMemcpy(&c, p->counters, sizeof(c), cudaMemcpyDeviceToHost));
  st->detected = (int64_t)c.detected;
  st->corrected = (int64_t)c.corrected;
  st->recomputed = (int64_t)c.recomputed;
  st->uncorrectable = (int64_t)c.uncorrectable;
  st->execs = p->execs;
  st->launches = p->launches;
  double ratio;
  std::memcpy(&ratio, &c.max_clean_ratio_bits, sizeof(ratio));
  st->max_clean_ratio = ratio;
  return TFFT_SUCCESS;
}

int tfft_report(tfft_plan_t p, int64_t* detected, int64_t* corrected) {
  tfft_stats st;
  int rc = tfft_report_ex(p, &st);
  if (rc) return rc;
  if (detected) *detected = st.detected;
  if (corrected) *corrected = st.corrected + st.recomputed;
  return TFFT_SUCCESS;
}

int tfft_reset_counters(tfft_plan_t p) {
  if (!p) return TFFT_ERR_INVALID_ARG;
  if (p->used) TFFT_CUDA(cudaStreamSynchronize(p->last_stream));
  TFFT_CUDA(cudaMemset(p->counters, 0, sizeof(Counters)));
  TFFT_CUDA(cudaMemset(p->err_flag, 0, sizeof(int)));
  p->execs = 0;
  p->launches = 0;
  return TFFT_SUCCESS;
}

int tfft_fault_log(tfft_plan_t p, tfft_fault_event* ev, int capacity, int64_t* total) {
  if (!p || capacity < 0 || (capacity > 0 && !ev)) return TFFT_ERR_INVALID_ARG;
  if (p->used) TFFT_CUDA(cudaStreamSynchronize(p->last_stream));
  Counters c;
  TFFT_CUDA(cudaMemcpy(&c, p->counters, sizeof(c), cudaMemcpyDeviceToHost));
  std::vector<LogEvent> ring(kLogRing);
  TFFT_CUDA(cudaMemcpy(ring.data(), p->log, sizeof(LogEvent) * kLogRing, cudaMemcpyDeviceToHost));
  const int64_t tot = (int64_t)c.log_total;
  if (total) *total = tot;
  const int64_t avail = std::min<int64_t>(tot, kLogRing);
  const int64_t take = std::min<int64_t>(avail, capacity);
  for (int64_t k = 0; k < take; k++) {
    const LogEvent& e = ring[(tot - take + k) % kLogRing];
    ev[k].exec_index = e.exec_index; ev[k].group = e.group; ev[k].signal = e.signal;
    ev[k].action = e.action; ev[k].nonfinite = e.nonfinite;
    ev[k].residual = e.residual; ev[k].tau = e.tau; ev[k].q_re = e.q_re; ev[k].q_im = e.q_im;
  }
  return TFFT_SUCCESS;
}

int tfft_set_fault(tfft_plan_t p, const tfft_fault* f) {
  if (!p || !f) return TFFT_ERR_INVALID_ARG;
  if (f->mode < 0 || f->mode > 4) return TFFT_ERR_INVALID_ARG;
  if (f->mode != 0) {
    if (f->pass < 0 || f->pass >= p->passes) return TFFT_ERR_INVALID_ARG;
    if (f->stage < -1 || f->stage >= p->pp[f->pass].nstages) return TFFT_ERR_INVALID_ARG;
    if (f->signal < 0 || f->signal >= p->batch || (f->mode == 4 && f->signal + 1 >= p->batch))
      return TFFT_ERR_INVALID_ARG;
    if (f->index < 0 || f->index >= p->pp[f->pass].nsub) return TFFT_ERR_INVALID_ARG;
    const int64_t lps = p->pp[f->pass].lines_are_signals ? 1 : p->pp[f->pass].LO * p->pp[f->pass].HI;
    if (f->line < 0 || f->line >= lps) return TFFT_ERR_INVALID_ARG;
    const int w = p->dtype == TFFT_C64 ? 32 : 64;
    if (f->mode == 1 && (f->bit < 0 || f->bit >= 2 * w)) return TFFT_ERR_INVALID_ARG;
  }
  FaultSite s{};
  s.mode = f->mode; s.pass = f->pass; s.stage = f->stage; s.bit = f->bit;
  s.signal = f->signal; s.line = f->line; s.index = f->index; s.factor = f->factor;
  std::lock_guard<std::mutex> lk(p->mu);
  if (s.mode == 0) {
    p->pending = FaultSite{};
    for (auto& f : p->pending_more) f = FaultSite{};
    p->npending = 0;
  } else if (p->npending == 0) {
    p->pending = s;
    p->npending = 1;
  } else if (p->npending < TFFT_MAX_FAULT_SITES) {
    p->pending_more[p->npending - 1] = s;
    p->npending++;
  } else {
    return TFFT_ERR_INVALID_ARG;
  }
  return TFFT_SUCCESS;
}

int tfft_plan_info(tfft_plan_t p, tfft_info* info) {
  if (!p || !info) return TFFT_ERR_INVALID_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n = p->n; info->batch = p->batch; info->dtype = p->dtype;
  info->abft_mode = !p->abft ? TFFT_ABFT_OFF : (p->one_sided ? TFFT_ABFT_ONE_SIDED : TFFT_ABFT_TWO_SIDED);
  info->passes = p->passes;
  for (int i = 0; i < p->passes; i++) {
    info->nsub[i] = p->pp[i].nsub;
    info->stages[i] = p->pp[i].nstages;
    info->lines_per_tile[i] = p->pp[i].C;
    info->lines_per_signal[i] = p->pp[i].lines_are_signals ? 1 : p->pp[i].LO * p->pp[i].HI;
  }
  info->group = p->G;
  info->max_faults = p->cap_fix;
  info->kappa = p->kappa;
  info->workspace_bytes = p->workspace_bytes;
  info->launches_per_exec = p->fuse ? 1 : p->passes + (p->abft ? 3 + 2 * p->passes : 0);
  info->checksum_vector = p->rvec == RVEC_WANG ? TFFT_R_WANG : TFFT_R_SIGNED_WANG;
  info->checksum_seed = p->rseed;
  info->direction = p->inverse ? TFFT_INVERSE : TFFT_FORWARD;
  info->precision = p->prec;
  for (int i = 0; i < 3; i++) info->tile_threads[i] = i < p->passes && p->pp[i].v3 ? p->pp[i].vnt : 0;
  info->tuned = p->tuned;
  info->normalize = p->normalize;
  return TFFT_SUCCESS;
}

int tfft_set_timing(tfft_plan_t p, int enable) {
  if (!p) return TFFT_ERR_INVALID_ARG;
  p->timing = enable ? 1 : 0;
  return TFFT_SUCCESS;
}

int tfft_timing(tfft_plan_t p, double* ms, int64_t* cnt, int nkinds) {
  if (!p || nkinds < 0 || (nkinds > 0 && (!ms || !cnt))) return TFFT_ERR_INVALID_ARG;
  for (int k = 0; k < nkinds; k++) { ms[k] = 0.0; cnt[k] = 0; }
  for (auto& t : p->timed) {
    TFFT_CUDA(cudaEventSynchronize(t.b));
    float el = 0.f;
    TFFT_CUDA(cudaEventElapsedTime(&el, t.a, t.b));
    if (t.kind >= 0 && t.kind < nkinds) { ms[t.kind] += el; cnt[t.kind]++; }
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  p->timed.clear();
  return TFFT_SUCCESS;
}

int tfft_destroy(tfft_plan_t p) {
  if (!p) return TFFT_ERR_INVALID_ARG;
  if (p->used) cudaStreamSynchronize(p->last_stream);
  free_plan(p);
  return TFFT_SUCCESS;
}

const char* tfft_error_string(int status) {
  switch (status) {
    case TFFT_SUCCESS: return "success";
    case TFFT_ERR_INVALID_ARG: return "invalid argument";
    case TFFT_ERR_UNSUPPORTED: return "unsupported dtype, mode or size";
    case TFFT_ERR_CUDA: return "CUDA runtime error";
    case TFFT_ERR_INPLACE: return "in-place transform with ABFT on";
    case TFFT_ERR_ALLOC: return "allocation failed";
    case TFFT_ERR_NO_DEVICE: return "no compute-capability 10.3 CUDA device";
    case TFFT_ERR_TIMEOUT: return "a kernel timed out waiting for a tile copy";
    default: return "unknown status";
  }
}

int tfft_last_cuda_error(void) { return g_last_cuda_error.load(); }

}  // extern "C"
