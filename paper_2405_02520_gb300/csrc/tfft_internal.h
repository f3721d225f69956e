// tfft_internal.h -- device-side parameter blocks shared by the library's
// translation units.  Not part of the public ABI (that is include/tfft.h).
#pragma once

#include <cstdint>
#include <cuda.h>            // CUtensorMap (the tensor-map type only; no driver call is linked)
#include <cuda_runtime.h>

struct tfft_plan_s;   // the plan (plan.cu); tfft_plan_t in include/tfft.h
struct tfft_plan_opts;

namespace tfft {

struct VerifyParams;

// A plan built from the options exactly as given, without the autotuner's
// table (plan.cu); `tuned` marks one whose pass configuration came from it.
int plan_create(tfft_plan_s** out, const tfft_plan_opts* o, int tuned);
// The autotuner's entry for these options (tune.cu): true, with *tuned a
// copy of *o whose pass count, first factor and tile threads are the entry's.
bool tune_lookup(const tfft_plan_opts* o, tfft_plan_opts* tuned);

// How the butterflies of one radix stage are dealt to the threads of a tile.
// ROW: consecutive threads take consecutive butterflies of one line (the
//      line's elements are contiguous in memory).
// COL: consecutive threads take the same butterfly of consecutive lines (the
//      lines are adjacent columns, so their elements are contiguous).
enum MapMode : int { MAP_ROW = 0, MAP_COL = 1 };

constexpr int kMaxThreads = 1024;
constexpr int kLogRing = 1024;     // fault-event log entries

// Fault injection site (Section II-A single-event upset), see tfft_fault.
struct FaultSite {
  int mode;      // 0 none, 1 bit flip, 2 scale, 3 add
  int pass;
  int stage;     // -1 loaded value, 0..nstages-1 stage output
  int bit;
  int64_t signal;
  int64_t line;
  int64_t index;
  double factor;
};

// Partial checksums of one chunk (one thread block's share of one group).
// Input side (first pass): S1 = w^T sum_b x_b, S2 = w^T sum_b (b+1) x_b, and
// the energy sum_b ||x_b||^2.  Output side (last pass): T1 = r^T sum_b y_b,
// T2 = r^T sum_b (b+1) y_b and the range of signals whose partial output sum
// was not finite.
struct RecIn {
  double s1r, s1i, s2r, s2i, energy, pad0, pad1, pad2;
};
struct RecOut {
  double t1r, t1i, t2r, t2i;
  long long nf_min, nf_max;   // signal indices (INT64_MAX / -1 when none)
  double pad0, pad1;
};

// Per-signal checksum records (the tile kernels, when every pass that
// encodes runs on them): the partial sums of one (signal, slot) -- a warp's
// share of one tile of that signal -- in the element type's precision.
//   input side (first pass):  w^T x_b and ||x_b||^2 over the share;
//   output side (last pass):  r^T y_b over the share.
// The verification adds a signal's slots in FP64, tests every signal on its
// own, and forms the group checksums X e_1, X e_3 (Section III) from them.
template <typename real> struct SigIn { real sr, si, en, pad; };
template <typename real> struct SigOut { real tr, ti; };
// Second check of a multi-pass plan, across its last pass only (the last
// pass's own input z and output y, a second left vector
// r2_k = r_k w3^floor(E k / N), E = 16 or 8 the radix of the last stage):
// r2^T y_b and u2^T z_b over the share, u2
// the image of r2 through the last pass (per output class L, the DFT of r2
// restricted to L).
template <typename real> struct SigChk { real tr, ti, sr, si; };

struct Counters {
  unsigned long long detected, corrected, recomputed, uncorrectable;
  unsigned long long log_total, execs;
  unsigned long long max_clean_ratio_bits;   // max |T1-S1|/tau of undetected groups (double bits)
  unsigned long long pad1;
};

// Signal-side encoding vector r of the checksum scheme.
//   RVEC_SIGNED_WANG: r_k = s_k w3^k, s_k = +-1 from bit 63 of output k of
//                     the SplitMix64 stream seeded with rseed; w = W r is
//                     tabulated.  The random signs spread the spectrum of r
//                     (no small w_n, so early-stage faults stay visible); the
//                     w3 phases keep the few outputs that a late-stage fault
//                     touches from cancelling in r^T e.
//   RVEC_WANG       : r_k = w3^k (e_Wang), w in closed form.
enum RVec : int { RVEC_SIGNED_WANG = 0, RVEC_WANG = 1 };

// Output k (0-based) of the SplitMix64 generator of Steele, Lea and Flood
// (OOPSLA 2014) started from state `seed`: mix(seed + (k + 1) * gamma).
__host__ __device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                                   unsigned long long k) {
  unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct LogEvent {   // mirrors tfft_fault_event
  long long exec_index, group, signal;
  int action, nonfinite;
  double residual, tau, q_re, q_im;
};

// Lists filled by the verify kernel, consumed by the correction path.
//   fix list   : groups whose faulty signal was named; entry e -> (group, b*)
//   recompute  : groups recomputed from their input
// list[0] = count, list[1 + e] = group index; fix_signal[e] = b*.
struct Lists {
  long long* fix;         // 1 + cap_fix
  long long* fix_signal;  // cap_fix
  long long* rec;         // 1 + cap_rec
  int cap_fix, cap_rec;
};

// How a tile moves between global and shared memory in the TMA kernel.
//   kind 1: one bulk copy of `rows` contiguous signals (single pass),
//   kind 2 / 3: a 2-D / 3-D tensor-map box; coordinates of the tile whose
//   signal is b, hi-line hi and first lo-line lo0 are
//     x = ax*lo0,  y = ay*hi + by*b + cy*lo0,  z = az*hi + bz*b + cz*lo0
//   (in 8-byte units along x), repeated `nbox` times with y advanced by
//   `box_rows` and the shared-memory destination by `box_elems` elements.
// layout: 0 line-major [C][nsub], 1 element-major [nsub][C] (the dense box).
struct TileMap {
  int kind;
  int layout;
  int nbox;              // boxes along y (rows), y += box_rows, smem += box_elems
  int box_rows;
  int box_elems;
  int nbx;               // boxes along x (column groups), x += bx_step, smem += bx_elems
  int bx_step;
  int bx_elems;
  unsigned bytes;        // bytes of the whole tile (all boxes)
  long long ax, ay, by, cy, az, bz, cz;
};

struct PassParams {
  // ---- geometry of the batched sub-transform of this pass ----
  int nsub, log2nsub;     // line length
  int C;                  // lines per tile (power of two)
  int nthreads;           // C * nsub / E
  int nstages;            // radix stages: E, E, ..., then nsub / E^(nstages-1)
  int pitch;              // shared-memory line pitch in elements (>= nsub)
  int lines_are_signals;  // 1: single pass, a line is a whole signal
  int in_map, mid_map, out_map;
  int pass_index;
  int64_t n;              // signal length N (signal stride in elements)
  int64_t batch;          // signals in the addressed buffers
  int64_t LO, HI;         // lines per signal = LO * HI; C divides LO
  int64_t in_es, in_lo, in_hi;     // element / lo-line / hi-line strides
  int64_t out_es, out_lo, out_hi;
  const void* in;
  void* out;
  // signal b of `in` (`out`) starts at element soff_in[b] (soff_out[b]) instead
  // of b n: a ragged batch read and written in the caller's packing.  Set on
  // the first pass's input and the last pass's output only.
  const long long* soff_in;
  const long long* soff_out;

  // ---- twiddles ----
  const void* tw_sub;     // omega_{tw_sub_n}^m, m < tw_sub_n (stage twiddles)
  const void* tw_stage;   // v3 kernels: per-stage table omega_{Ns R}^(q kk) (see fft_v3.cuh)
  int tw_sub_stride;      // tw_sub_n / nsub
  int twiddle;            // multiply output i of line lo by omega_{tw_n}^{lo*i}
  int64_t tw_scale;       // N / tw_n
  const void* twN_lo;     // omega_N^m = twN_hi[m >> twN_lbits] * twN_lo[m & mask]
  const void* twN_hi;
  int twN_lbits;

  // ---- two-sided ABFT ----
  int abft_in, abft_out;
  int group;              // G
  int parts;              // chunks per (group, line block)
  int64_t ngroups;
  int64_t line_blocks;    // LO * HI / C (1 when lines are signals)
  int64_t slots;          // records per group written by this pass
  RecIn* rec_in;
  RecOut* rec_out;
  const void* wt_lo;      // e^{i pi m / (3N)} = wt_hi[m >> wt_lbits] * wt_lo[m & mask]
  const void* wt_hi;
  int wt_lbits;
  double wk_re, wk_im;    // K = 1 - w3^N
  int rvec;               // RVec
  unsigned long long rseed;
  const void* wtab;       // w = W r, N entries (RVEC_SIGNED_WANG)
  long long* zero_on_entry[3];   // list counts and the correction flag, zeroed by block 0 (first pass of an exec)

  // ---- work list (correction path); list == nullptr for a normal exec ----
  const long long* list;  // list[0] = count, list[1 + e] = block (ignored if list_identity)
  int list_identity;      // block index = entry index
  int list_cap;
  int64_t list_block;     // signals per listed block

  int64_t nchunks;
  FaultSite fault_more[3];   // armed sites after `fault` (tile kernels only)
  int nfault;                // armed sites in total (0..4)
  // inverse / normalised transforms: conj on load (first pass), conj and
  // scale on store (last pass); the checksums see the forward transform
  int conj_in, conj_out;
  // per-signal records (sigrec = 1, tile kernels): this pass's records of
  // signal b at slot k are sig_in / sig_out[b sig_slots + k]
  int sigrec;
  void* sig_in;           // SigIn<real>
  void* sig_out;          // SigOut<real>
  int64_t sig_slots;
  // second check across the last pass (chk2 = 1, last pass only): records
  // sig_chk[b sig_slots + k] (SigChk<real>), u2 = ltab[L nsub + n] for the
  // line whose outputs start at L; r2_k = r_k w3^floor(E k / N), E the radix
  // of the last stage (16 complex64, 8 complex128)
  int chk2;
  void* sig_chk;
  const void* ltab;
  double out_scale;       // 1 unless normalising on the last pass
  int log2C, log2LO, log2LB;   // log2 of C, LO and line_blocks (all powers of two; v3 kernels)
  FaultSite fault;

  // ---- TMA tile pipeline (fft_tile_kernel only) ----
  int nbuf;               // shared-memory tile buffers in the ring
  unsigned buf_bytes;     // bytes per buffer (tile rounded up to 1 KiB)
  int* err_flag;          // set when a bounded wait gives up
  long long wait_limit;   // polls of a tile-arrival wait before it gives up
  // fused verification (single-pass plans of few groups, stream-launched
  // whole-batch execs): every block counts itself in *fdone once its tiles
  // are done, and the last one verifies every group with *fverify (this
  // exec's index in its log entries), then resets the count; nullptr: a
  // separate verification launch
  const VerifyParams* fverify;
  unsigned* fdone;
  long long exec_index;
  // launched as a programmatic dependent of the kernel before it on the
  // stream: the block sets up what reads only plan constants, then waits for
  // that kernel (griddepcontrol.wait) before its first global write or tile
  // load
  int pdl;
  TileMap map_in, map_out;
  CUtensorMap tmap_in;     // 64-byte aligned by its own type
  CUtensorMap tmap_out;
};

// Launchers (one per element type), defined in fft_pass_f32.cu / _f64.cu.
cudaError_t launch_pass_f32(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_pass_f64(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s);
cudaError_t pass_func_attrs_f32(int E, size_t smem, int block, int* blocks_per_sm);
cudaError_t pass_func_attrs_f64(int E, size_t smem, int block, int* blocks_per_sm);
cudaError_t launch_tile_f32(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_tile_f64(const PassParams& p, int E, int grid, size_t smem, cudaStream_t s);
cudaError_t tile_func_attrs_f32(int E, size_t smem, int block, int* blocks_per_sm);
cudaError_t tile_func_attrs_f64(int E, size_t smem, int block, int* blocks_per_sm);
// v3 kernels (fft_v3.cuh): role 0 single pass, 1 column pass, 2 last pass.
// Return cudaErrorInvalidValue for an (nsub, role) without an instantiation.
cudaError_t launch_v3(int dtype, int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs(int dtype, int role, int nsub, size_t smem, int* blocks_per_sm);
int v3_radix(int dtype, int nsub);
int v3_scratch_bytes(int dtype, int nsub);
int v3_twiddle_smem_bytes(int dtype, int nsub);
// 512-thread v3 kernels (v3_f32_wide.cu, complex64): column (role 1) and last
// (role 2) passes of 512, 1024 and 2048 points in tiles of 8192 values.
cudaError_t launch_v3_wide(int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_wide(int role, int nsub, size_t smem, int* blocks_per_sm);
int v3_wide_scratch_bytes(int nsub);
// Tensor-core variants (v3_tc.cu): tc = 3 split TF32, 1 plain TF32.
cudaError_t launch_v3_tc(int tc, int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_tc(int tc, int role, int nsub, size_t smem, int* blocks_per_sm);
int v3_tc_bytes(int tc);
// True for the tensor-core forms that keep their operands in the line scratch
// and so fit two blocks per SM (split BF16, plain TF32).
bool v3_tc_two_blocks(int tc);

// Signal offsets for a plan's exec (ragged batches in the caller's packing):
// signal b of the exec's input and output starts at element off[b] (d_off on
// the device, h_off its host copy, `total` elements in each buffer).  Returns
// TFFT_ERR_UNSUPPORTED when a pass cannot address the signals that way (then
// the caller stages the signals contiguously instead).
int plan_set_signal_offsets(::tfft_plan_s* p, const long long* d_off, const int64_t* h_off, int64_t total);

// Keeps `e` as the value tfft_last_cuda_error() reports; returns TFFT_ERR_CUDA.
int record_cuda_error(cudaError_t e);

// Geometry of one launch of the direct-load pass kernel (fft_pass.cuh): line
// length, values per thread, lines per tile, butterfly maps, strides, the
// shared-memory pitch and size.  two_pass_geometry fills both launches of the
// two-pass factorisation N = N1 x (N / N1) (Section IV-A, "Tiled FFT"): the
// first over columns of stride N / N1 with the inter-pass twiddle, the second
// over contiguous rows, stored transposed into natural order.  The planner and
// the allocation-free entry point take their two-pass geometry from here.
struct PassGeom {
  int nsub = 1, E = 1, C = 1, nthreads = 32, nstages = 1, pitch = 1;
  int in_map = MAP_ROW, mid_map = MAP_ROW, out_map = MAP_ROW, twiddle = 0;
  int64_t LO = 1, HI = 1, in_es = 1, in_lo = 0, in_hi = 0, out_es = 1, out_lo = 0, out_hi = 0;
  int64_t tw_scale = 1, line_blocks = 1;
  size_t smem = 0;
};
void two_pass_geometry(int64_t n, int64_t N1, int esize, PassGeom g[2]);
// Elements per thread, shared-memory row padding and radix-stage count of the
// direct-load pass kernel (see plan.cu).
int geom_pick_E(int nsub, int E0);
int geom_nstages(int nsub, int E);

// Verify / correction kernels (abft_fix.cu).
struct VerifyParams {
  int64_t n, batch;
  int group;
  int64_t ngroups;
  int64_t group_base;           // index of group 0 in the plan (fault log entries)
  int64_t slots_in, slots_out;
  const RecIn* rec_in;
  const RecOut* rec_out;
  double kappa_u_log2n_sqrtn;   // kappa * u * (log2(N) + 4) * sqrt(N)
  int detect_only;
  Lists lists;
  Counters* counters;
  LogEvent* log;
  long long exec_index;
  int max_blocks;               // grid cap (blocks stride over the groups)
  // exec replayed from a CUDA graph: the correction work is the body of a
  // conditional node, switched on (once, by the first thread that queues a
  // group: *cond_flag guards the call) when a group needs it
  long long* cond_flag;         // nullptr outside the graph
  cudaGraphConditionalHandle cond;
  // groups with many records and few groups: `split` blocks per group add
  // their slice's sums into part_acc[g] (9 sums, then the nonfinite range as
  // integers) and count themselves in part_cnt[g]; the last one decides and
  // restores the accumulators (zero sums, empty range, zero count)
  int split;                    // blocks per group (1: one block strides over groups)
  double* part_acc;             // ngroups x kVerifyAcc
  unsigned* part_cnt;           // ngroups
  // per-signal records (sigrec = 1): signal b's records are sig_in[b sig_slots_in + k]
  // and sig_out[b sig_slots_out + k]; dtype 0 float, 1 double
  int sigrec;
  int dtype;
  const void* sig_in;
  const void* sig_out;
  int64_t sig_slots_in, sig_slots_out;
  // signals with many records: `sig_split` warps per signal add their slice
  // into sig_acc[b] (kSigAcc sums) and count themselves in part_cnt[g]; the
  // last warp of a group decides it and restores the sums and the count
  // (0: one lane per signal adds all its records)
  int sig_split;
  double* sig_acc;              // batch x kSigAcc
  // (sig_blk_lanes > 0, in place of the split mode) one block per unit of
  // sig_gpb groups, sig_blk_lanes lanes adding one signal's records
  int sig_blk_lanes, sig_gpb;
  double tau_floor;             // smallest threshold (the element type's tiny values)
  // second check across the last pass: records sig_chk[b sig_slots_out + k],
  // threshold kappa u (log2 n_last + 4) sqrt(N) sqrt(E_b)
  int chk2;
  const void* sig_chk;
  double kappa_u_chk2;
};
constexpr int kVerifyAcc = 12;
constexpr int kSigAcc = 10;
// records a signal may hold for the one-thread-per-signal verification
constexpr int64_t kSigSerialMax = 48;
int sig_split_of(int64_t recs, int64_t batch, int sms);
// lanes per signal of the block verification for signals of rin input-side
// and rout output-side records in `ngroups` groups of `group` (and *gpb, its
// groups per block), or 0 when it would not give every SM a block
int sig_block_geom(int64_t rin, int64_t rout, int64_t group, int64_t ngroups, int sms, int* gpb);
// blocks per group for a group of `recs` records when there are `ngroups`
// groups on `sms` multiprocessors (1 = no split)
int verify_split(int64_t recs, int64_t ngroups, int sms);
cudaError_t launch_verify(const VerifyParams& v, cudaStream_t s);

struct FixParams {
  int64_t n, batch;
  int group;
  int dtype;           // 0 c64, 1 c128
  const void* in;      // user input (read)
  void* out;           // user output (patched)
  const long long* soff;   // signal offsets in `in` and `out` (nullptr: b n)
  void* ws_c1;         // cap_fix x n : gathered sum_b x_b, transformed in place
  void* ws_acc;        // cap_fix x n : sum_{b != b*} y'_b
  Lists lists;
  // fix_apply, the last launch of the correction sequence, counts the
  // corrected and the recomputed groups once their work has run (unless a
  // bounded wait of the exec gave up)
  Counters* counters;
  const int* err_flag;
};
cudaError_t launch_fix_gather(const FixParams& f, cudaStream_t s);
// r_k = s_k w3^k (SplitMix64 signs; s_k = 1 with sign = 0) as complex128 --
// times w3^floor(qdiv k / n) with qdiv > 0 (the second left vector, qdiv the
// radix of the last stage) -- and a complex128 -> complex64 copy.
cudaError_t launch_gen_signs(void* r, int64_t n, unsigned long long seed, cudaStream_t s, int qdiv = 0,
                             int sign = 1);
cudaError_t launch_c128_to_c64(const void* src, void* dst, int64_t n, cudaStream_t s);
// dst[L nl + k] = src[L + M k] for L < M, k < nl (complex128): the classes of
// a vector of length M nl laid out as rows
cudaError_t launch_gather_classes(const void* src, void* dst, int64_t M, int64_t nl, cudaStream_t s);
cudaError_t launch_fix_apply(const FixParams& f, cudaStream_t s);

// Persistent tile kernels for ragged batches (v3_ragged*.cu): one launch
// runs one pass family -- the passes of one role (0 single, 1 column, 2 last;
// complex64, 256 threads) and sub-transform length -- for up to kRaggedMax
// buckets, each with its own pass parameters, all in the launch's parameter
// block (tensor maps included, as in the batched launches).  Its blocks take
// work items -- a range of one bucket's chunks -- in order from `items`
// through the counter *head (zero before the launch); the plan sorts the
// items by work, largest first.
constexpr int kRaggedMax = 24;          // 24 x 1152 bytes of pass parameters: under 32 KB
struct RaggedItem {
  int bucket;             // index into pp
  int pad;
  long long c0, c1;       // chunks [c0, c1) of that bucket's pass
};
struct RaggedParams {
  PassParams pp[kRaggedMax];
  long long nitems;
  const RaggedItem* items;
  unsigned long long* head;
};
// whether a persistent kernel covers the family (role, nsub)
bool v3_ragged_has(int role, int nsub);
cudaError_t v3_ragged_attrs(int role, int nsub, size_t smem, int* bps);
cudaError_t launch_v3_ragged(int role, int nsub, const RaggedParams& r, int grid, size_t smem, cudaStream_t s);

// Plan hooks for the persistent ragged form (plan.cu): what pass i of a
// whole-batch exec would launch, the exec's verification and correction
// after its passes ran elsewhere, and the exec's bookkeeping.
struct RaggedPass {
  int ok;                 // the pass runs on a kernel the persistent form has
  int role, nsub;
  size_t smem;            // dynamic shared memory of a block
  long long nchunks;      // chunks of a whole-batch exec
  int tiles_per_chunk;    // about
};
int plan_ragged_pass(tfft_plan_s* p, int i, RaggedPass* rp);
int plan_pass_params(tfft_plan_s* p, const void* in, void* out, int i, PassParams* a);
int plan_exec_checks(tfft_plan_s* p, const void* in, void* out, cudaStream_t s);
void plan_exec_finish(tfft_plan_s* p, cudaStream_t s);

}  // namespace tfft
