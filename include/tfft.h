/*
 * tfft.h -- C ABI of the GB300 (sm_103a) fault-tolerant batched FFT.
 *
 * The library computes the batched one-dimensional complex-to-complex forward
 * DFT of TurboFFT (Wu et al., arXiv 2405.02520), Section II:
 *
 *     y_j = sum_{n=0}^{N-1} x_n exp(-2 pi i j n / N),   j = 0..N-1,
 *
 * unnormalised, for every signal of a batch, fused with the paper's two-sided
 * algorithm-based fault tolerance (ABFT), Section III (Eqs. two_side_X and
 * two_side_Y, Section III-B "Delayed Batched Correction"): the batch is
 * encoded on the input side with the checksum vector w = W^T r and on the
 * output side with r, where r_j = s_j exp(-2 pi i j / 3) (Wang's e_Wang
 * vector of Section II with seeded random signs s_j = +-1; plain e_Wang is an
 * option), and across each group of G consecutive signals with the all-ones
 * vector and the index weights (1, 2, ..., G).  The left-side checksums are
 * formed per signal (d_b = r^T y_b - w^T x_b) and the group's two-sided
 * residuals from them; a silent data corruption is detected when a signal's
 * own residual or the group's exceeds its threshold, the faulty signal is
 * the one whose own test failed (or, for a detection by the group test
 * alone, the quotient of the weighted and unweighted residuals), and it is
 * corrected by subtracting the batch-checksum divergence
 * (sum_b y'_b - W sum_b x_b) -- no recomputation of that signal.  Multi-pass
 * plans (up to 2^26 points) also check their last pass on its own against a
 * second left vector r2_j = r_j w3^floor(E j / n), E the radix of that
 * pass's last stage (16 complex64, 8 complex128).
 *
 * Data layout (all entry points): `batch` signals of `n` complex values,
 * signal-major [batch][n], each value interleaved (re, im); complex64 is two
 * floats (8 bytes), complex128 two doubles (16 bytes).  Device pointers must be
 * 16-byte aligned.  Output is in natural order.
 *
 * Return codes: 0 (TFFT_SUCCESS) or a negative TFFT_ERR_* value.  Faults that
 * the ABFT detects are NOT errors: tfft_exec is asynchronous and never reports
 * them through its return value; read them with tfft_report / tfft_report_ex.
 *
 * Threading: a plan may be used from one host thread at a time; two execs of
 * one plan must not overlap on the GPU (they share the plan's workspace).
 * Different plans are independent.
 */
#ifndef TFFT_H
#define TFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 (NULL) is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st *tfft_stream_t;

/* Opaque plan, owned by the library: tfft_plan* creates it, tfft_destroy
 * frees it and every device allocation it made. */
typedef struct tfft_plan_s *tfft_plan_t;

enum tfft_dtype { TFFT_C64 = 0, TFFT_C128 = 1 };

enum tfft_abft_mode {
    TFFT_ABFT_OFF = 0,        /* plain FFT                                   */
    TFFT_ABFT_ONE_SIDED = 1,  /* Section III one-sided scheme: the left-side
                                 checksum of every signal alone (w^T x_b vs
                                 r^T y_b); a flagged signal is recomputed from
                                 its input.  Kept as an ablation of the
                                 two-sided scheme; available when every pass
                                 runs on the tile kernels (complex64 n >= 256,
                                 complex128 n >= 128, and all multi-pass n),
                                 otherwise TFFT_ERR_UNSUPPORTED              */
    TFFT_ABFT_TWO_SIDED = 2   /* Section III two-sided checksums             */
};

enum tfft_status {
    TFFT_SUCCESS = 0,
    TFFT_ERR_INVALID_ARG = -1,  /* n not a power of two in [2^0, 2^29], batch
                                   < 1, null or misaligned pointer, bad option */
    TFFT_ERR_UNSUPPORTED = -2,  /* dtype or abft_mode not implemented         */
    TFFT_ERR_CUDA = -3,         /* a CUDA runtime call failed; see
                                   tfft_last_cuda_error()                     */
    TFFT_ERR_INPLACE = -4,      /* in == out with ABFT on: the correction and
                                   the group recompute re-read the input      */
    TFFT_ERR_ALLOC = -5,        /* device or host allocation failed           */
    TFFT_ERR_NO_DEVICE = -6,    /* no CUDA device, or not compute capability
                                   10.3 (the kernels are built for sm_103a)   */
    TFFT_ERR_TIMEOUT = -7       /* a kernel gave up waiting for a tile copy
                                   (bounded wait); the results of the execs
                                   since the last report are not valid        */
};

/*
 * tfft_plan -- plan a batched forward FFT of `batch` signals of length `n`
 * (a power of two, 1 <= n <= 2^29), element type `dtype` (TFFT_C64 or
 * TFFT_C128), fault tolerance `abft_mode` (TFFT_ABFT_OFF or
 * TFFT_ABFT_TWO_SIDED).  Chooses the pass decomposition (one pass when a
 * signal fits one thread block's tile, otherwise the kernel-level tiling of
 * Section IV-A into two or three launches), builds the FP64-accurate twiddle
 * and checksum tables on the host, uploads them, and allocates the workspace
 * (the inter-pass buffer, checksum records, fault lists, counters) on the
 * current CUDA device.  A multi-pass plan with checksums builds its second
 * check's table on the device (a few kernels and a complex128 transform on
 * the legacy default stream, waited for before the call returns); no other
 * plan launches a kernel.  *out receives the plan.
 */
int tfft_plan(tfft_plan_t *out, int64_t n, int64_t batch, int dtype, int abft_mode);

/* Extended options.  Zero-initialise and set what you need; zero means the
 * default for every field except n, batch, dtype, abft_mode. */
typedef struct tfft_plan_opts {
    int64_t n;
    int64_t batch;
    int dtype;
    int abft_mode;
    int group;          /* G: signals per checksum group (default 16)          */
    double kappa;       /* detection threshold constant (default 2); the
                           threshold is kappa*u*(log2(n)+4)*sqrt(n)*sqrt(E),
                           E the input energy ||x_b||^2 of the signal for its
                           own test and sum_b ||x_b||^2 of the group for the
                           group test, u the unit roundoff of dtype (the
                           second check of a multi-pass plan takes log2 of
                           its last pass's length in place of log2(n))      */
    int detect_only;    /* 1: detect and locate but leave outputs uncorrected  */
    int max_faults;     /* groups corrected per exec (default: as many as fit
                           a 1 GiB budget, at most 8); more are counted
                           uncorrectable                                       */
    int force_passes;   /* 0: planner's choice; 1, 2 or 3 forces the count
                           (TFFT_ERR_INVALID_ARG when it cannot tile n)         */
    int checksum_vector;       /* signal-side encoding vector r:
                                  TFFT_R_SIGNED_WANG (default)
                                    r_k = s_k e^{-2 pi i k/3}, s_k = -1 when
                                    bit 63 of output k of the SplitMix64
                                    stream seeded with checksum_seed is set,
                                    else +1 (w = W r tabulated at plan time);
                                  TFFT_R_WANG r_k = e^{-2 pi i k/3} (e_Wang,
                                    Section II; w in closed form)             */
    uint64_t checksum_seed;    /* seed of the signs (0: the default 20240502)  */
    int direction;      /* TFFT_FORWARD (default): y_j = sum_n x_n e^{-2 pi i jn/N};
                           TFFT_INVERSE: y_j = sum_n x_n e^{+2 pi i jn/N}
                           (the inverse DFT of Section II without its 1/N)      */
    int normalize;      /* 1: multiply the output by 1/N (with TFFT_INVERSE the
                           exact inverse of the forward transform); 0: none    */
    int precision;      /* arithmetic of the radix-16 butterflies (complex64):
                           TFFT_PREC_FP32 (default) FP32 CUDA cores;
                           TFFT_PREC_TF32X3 tensor cores, operands split into
                             TF32 high and low parts, three products summed in
                             FP32 (about 21 significant bits);
                           TFFT_PREC_TF32 tensor cores, one TF32 product
                             (about 11 bits);
                           TFFT_PREC_BF16X3 tensor cores, BF16 high and low
                             parts, three products (about 16 bits).
                           The tensor-core forms cover n = 2^8..2^12 and 2^16;
                           other n return TFFT_ERR_UNSUPPORTED.  The detection
                           threshold uses the form's unit roundoff (2^-20,
                           2^-10 and 2^-17 in place of 2^-24).               */
    int wait_polls;     /* polls of a kernel's wait for a tile copy before it
                           gives up (the bounded waits of the TMA pipeline):
                           0 the default 2^20 (about a second), k > 0 that
                           many, -1 none at all -- every such wait gives up at
                           once, the exec's output is not valid and
                           tfft_report returns TFFT_ERR_TIMEOUT; for testing
                           the timeout path                                   */
    int first_pass_log2; /* two-pass plans: log2 of the first pass's
                           sub-transform length N1 (the second takes N/N1);
                           0 the planner's choice; TFFT_ERR_INVALID_ARG when
                           the plan is not two-pass or a factor is out of
                           range                                              */
    int tile_threads;   /* threads of the tile kernels of complex64 column and
                           last passes of 512 to 2048 points (FP32): 256 (tiles
                           of 4096 values, two blocks per SM) or 512 (tiles of
                           8192, one block per SM, twice the lines a tile and
                           twice the bytes a row) where that form has a kernel
                           for the pass, else the other; 0 the planner's
                           choice; other passes ignore it;
                           TFFT_ERR_INVALID_ARG for any other value           */
} tfft_plan_opts;

enum tfft_precision { TFFT_PREC_FP32 = 0, TFFT_PREC_TF32X3 = 1, TFFT_PREC_TF32 = 2, TFFT_PREC_BF16X3 = 3 };

/* The inverse runs the forward machinery on conj(x) and stores conj(.)/N:
 * the checksums of Section III check that forward transform, so detection,
 * location and correction work unchanged in both directions. */
enum tfft_direction { TFFT_FORWARD = 0, TFFT_INVERSE = 1 };

enum tfft_checksum_vector { TFFT_R_SIGNED_WANG = 0, TFFT_R_WANG = 1 };

int tfft_plan_ex(tfft_plan_t *out, const tfft_plan_opts *opts);

/*
 * tfft_exec -- transform `batch` signals from device buffer `in` to device
 * buffer `out` (layout above, each plan->batch*n elements), asynchronously on
 * `stream`.  `in` is never written.  With ABFT on, `in` and `out` must not
 * overlap (TFFT_ERR_INPLACE).  No host synchronisation.  When the same
 * (in, out) pair comes back on a stream that is not being captured, the plan
 * builds (once for that pair) a CUDA graph of the verification and the
 * correction launches, the latter under a conditional node that runs only
 * when a group was flagged; other execs launch them directly.  A
 * single-pass plan of at most 64 checksum groups (tfft_info's
 * launches_per_exec is 1) runs a whole-batch exec as its pass kernel alone:
 * the kernel's last block verifies every group and corrects the flagged
 * ones itself (Section III-B, the one-pass case).  On a stream that is not
 * being captured that kernel is a programmatic dependent launch: its blocks
 * may initialise shared memory while the kernel before it on the stream
 * finishes, and wait for that kernel to complete before they read or write
 * global memory, so stream order holds as for any launch.
 * Returns TFFT_ERR_CUDA if a launch fails.
 */
int tfft_exec(tfft_plan_t p, const void *in, void *out, tfft_stream_t stream);

/*
 * tfft_exec_host -- the same transform on HOST buffers (pinned or pageable;
 * pinned for overlap): copies `host_in` to a plan-owned device buffer, runs
 * the transform, copies the result to `host_out`, and synchronises `stream`
 * before returning.  The batch is cut into up to eight chunks of whole
 * checksum groups: the input copies run back to back on a plan-owned copy
 * stream, each chunk is transformed on `stream` once its input has landed,
 * and its output copy (a second plan-owned stream) overlaps the later
 * chunks' input copies and transforms.  One chunk (copy, transform, copy on
 * `stream`) when the batch is one group or a test fault is armed.  The plan
 * allocates its two device staging buffers, the copy streams and their
 * events on the first call and keeps them until tfft_destroy.
 */
int tfft_exec_host(tfft_plan_t p, const void *host_in, void *host_out, tfft_stream_t stream);

/*
 * tfft_report -- synchronise the stream of the plan's last exec and return
 * the cumulative number of groups in which a fault was detected, and of
 * those that were corrected (by the checksum correction or, when the faulty
 * signal could not be named with confidence, by recomputing the group from
 * its input).  detected - corrected groups were left uncorrected.  Either
 * pointer may be NULL.
 */
int tfft_report(tfft_plan_t p, int64_t *detected, int64_t *corrected);

typedef struct tfft_stats {
    int64_t detected;       /* groups flagged (a signal's test or the group's)    */
    int64_t corrected;      /* fixed by the checksum correction                */
    int64_t recomputed;     /* fixed by recomputing the whole group            */
    int64_t uncorrectable;  /* detected, not fixed (lists full / detect_only)  */
    int64_t execs;          /* tfft_exec calls since plan / reset              */
    int64_t launches;       /* kernels launched since plan / reset             */
    double max_clean_ratio; /* largest residual / threshold of any test (a
                               signal's own, its last-pass check, the group's)
                               in the groups that were NOT flagged
                               (calibration of kappa)                           */
} tfft_stats;

int tfft_report_ex(tfft_plan_t p, tfft_stats *stats);
/* Zeroes the counters and the fault log count, and clears a recorded
 * timeout (TFFT_ERR_TIMEOUT).  Synchronises the plan's last stream. */
int tfft_reset_counters(tfft_plan_t p);

/* One detection, as logged on the device (ring of 1024 entries). */
typedef struct tfft_fault_event {
    int64_t exec_index;     /* 0-based exec count of the plan                   */
    int64_t group;          /* checksum group                                   */
    int64_t signal;         /* located signal (batch index), -1 if not located  */
    int32_t action;         /* 1 corrected, 2 group recomputed, 3 uncorrected   */
    int32_t nonfinite;      /* the residual or a partial sum was not finite     */
    double residual;        /* the failing signal's residual when one signal
                               failed its own test, else |T1 - S1|              */
    double tau;             /* the threshold it was compared with               */
    double q_re, q_im;      /* quotient (T2 - S2) / (T1 - S1)                   */
} tfft_fault_event;

/* Copy up to `capacity` most recent events (oldest first) and the total
 * number logged since plan / reset into *total.  Synchronises. */
int tfft_fault_log(tfft_plan_t p, tfft_fault_event *events, int capacity, int64_t *total);

/*
 * Fault injection (the Section II-A fault model: one soft error in a compute
 * unit).  Arms one fault for the NEXT tfft_exec only.  The kernel that owns
 * the value applies it in registers, after the value is computed and before
 * it is checksummed or stored, so it is a computation error, not a memory
 * error.  Sites: pass p (0-based), stage s (-1 = the value just loaded, 0..
 * stages-1 = the value produced by that radix stage, the last stage's value
 * being the pass output), signal, line (line index within the signal for
 * that pass, see tfft_plan_info) and index (element index within the line in
 * that stage's output order).
 */
enum tfft_fault_mode {
    TFFT_FAULT_NONE = 0,
    TFFT_FAULT_BITFLIP = 1,   /* flip bit `bit` of the value: bits 0..w-1 of
                                 the real part, w..2w-1 of the imaginary part
                                 (w = 32 for C64, 64 for C128)                 */
    TFFT_FAULT_SCALE = 2,     /* multiply the value by (factor + 0 i)          */
    TFFT_FAULT_ADD = 3,       /* add (factor + 0 i) to the value               */
    TFFT_FAULT_ADD_PAIR = 4   /* add (factor + 0 i) to the same value of
                                 signals `signal` and `signal`+1: two faults,
                                 outside the single-event model, to exercise
                                 the recompute fallback                        */
};

typedef struct tfft_fault {
    int mode;
    int pass;
    int stage;
    int bit;
    int64_t signal;
    int64_t line;
    int64_t index;
    double factor;
} tfft_fault;

/* Arms `fault` for the next exec.  Up to TFFT_MAX_FAULT_SITES calls before
 * one exec arm that many sites (sites after the first are honoured by the
 * tile kernels, i.e. complex64 n >= 256, complex128 n >= 128 and every
 * multi-pass n); mode TFFT_FAULT_NONE disarms all.  An exec consumes them. */
int tfft_set_fault(tfft_plan_t p, const tfft_fault *fault);
#define TFFT_MAX_FAULT_SITES 4

typedef struct tfft_info {
    int64_t n, batch;
    int dtype, abft_mode;
    int passes;
    int nsub[3];             /* sub-transform length per pass                 */
    int stages[3];           /* radix stages per pass                          */
    int lines_per_tile[3];
    int64_t lines_per_signal[3];
    int group;
    int max_faults;
    double kappa;
    int64_t workspace_bytes;
    int launches_per_exec;   /* kernels one tfft_exec launches                 */
    int checksum_vector;
    uint64_t checksum_seed;
    int direction;           /* TFFT_FORWARD / TFFT_INVERSE                    */
    int normalize;           /* 1: output scaled by 1/N                        */
    int precision;           /* TFFT_PREC_*                                    */
    int tile_threads[3];     /* threads a block of each pass's tile kernel
                                (256 or 512; 0: a pass on the fallback kernels) */
    int tuned;               /* 1: the pass configuration was taken from the
                                autotuner's table (tfft_autotune)              */
} tfft_info;

int tfft_plan_info(tfft_plan_t p, tfft_info *info);

/*
 * Per-kernel timing for measurement.  When enabled, tfft_exec records a CUDA
 * event pair around every kernel it launches (on the exec stream).
 * tfft_timing synchronises, adds the elapsed times up per kernel kind and
 * clears the record.  kinds: 0 first pass, 1 middle pass, 2 last pass, 3 the
 * single pass, 4 verify, 5 correction path.  Arrays have `nkinds` entries.
 */
int tfft_set_timing(tfft_plan_t p, int enable);
int tfft_timing(tfft_plan_t p, double *ms_per_kind, int64_t *launches_per_kind, int nkinds);

int tfft_destroy(tfft_plan_t p);

/*
 * Autotuner: the run-time form of the paper's kernel-parameter search
 * (Section IV-B "Kernel Parameters", Table I: the decomposition of N and the
 * tile parameters are chosen per N by measurement).  tfft_autotune times,
 * on the caller's device buffers in[batch][n] and out[batch][n] (not
 * overlapping, 16-byte aligned, in holding representative finite data) and
 * stream, every configuration the planner admits for *opts: pass count 1-3,
 * the first factor of two-pass plans, and 256- or 512-thread tiles for the
 * complex64 column and last passes of 512 to 2048 points, plus the
 * planner's own choice.  Each is planned, run twice untimed, then `reps`
 * (1-1000) times between CUDA events; out is overwritten.  opts must leave
 * force_passes, first_pass_log2 and tile_threads at 0 (TFFT_ERR_INVALID_ARG
 * otherwise).  Synchronises the stream.
 *
 * The fastest configuration goes into a process-wide table: a later
 * tfft_plan / tfft_plan_ex whose options leave those three fields at 0 and
 * match an entry's n, dtype, abft_mode and precision is built with the
 * entry's configuration (the entry whose batch is nearest in log2; the
 * plan's tfft_info.tuned is 1).  If the environment variable TFFT_TUNE_CACHE
 * names a file, the table is first read from it (lines
 * "tfft-tune-1 n batch dtype abft_mode precision passes first_pass_log2
 * tile_threads ms"; others are skipped) and every result is appended to it
 * (a file that cannot be written leaves the in-memory entry in place).
 */
typedef struct tfft_tune_result {
    int passes;              /* the fastest configuration: pass count           */
    int first_pass_log2;     /* log2 of its first factor (two passes), else 0   */
    int tile_threads;        /* 256 or 512                                      */
    int candidates;          /* configurations timed                            */
    double ms;               /* its mean time per tfft_exec                     */
    double default_ms;       /* the planner's own choice's time                 */
} tfft_tune_result;

int tfft_autotune(const tfft_plan_opts *opts, const void *in, void *out, tfft_stream_t stream, int reps,
                  tfft_tune_result *result);
/* 1 and *tuned = *opts with the table's configuration when an entry applies
 * to *opts, 0 when none does; no device work. */
int tfft_tune_lookup(const tfft_plan_opts *opts, tfft_plan_opts *tuned);
/* Empties the in-memory table; TFFT_TUNE_CACHE is read again on next use. */
int tfft_tune_clear(void);

/*
 * tfft_exec_noalloc -- the plain forward transform (no ABFT) of `batch`
 * complex64 signals of length `n` from device buffer `in` to device buffer
 * `out` (layout above; in == out is allowed), asynchronously on `stream`,
 * without any allocation.  The paper has no counterpart: this is for callers
 * that may not allocate device memory -- code under a memory manager or
 * sandbox that owns every device allocation, real-time loops that may not
 * block on the allocator -- and therefore cannot create a plan.
 *
 * Limits: n a power of two with 8192 <= n <= 2^18 (the two-pass range) and
 * batch * n <= 2^23 (the 64 MiB scratch); anything else returns
 * TFFT_ERR_INVALID_ARG before any work.  The inter-pass buffer and the
 * twiddle tables are file-scope __device__ arrays (64 MiB + 12 KiB) that a
 * GPU reserves when the library's module holding them is loaded on it, and
 * holds until the process exits; no cudaMalloc, cudaFree or other allocating
 * call is made.  With lazy module loading (the CUDA default) that load
 * happens at the first call on a device, which also looks up the arrays'
 * device addresses (cudaGetSymbolAddress) and the launch occupancies: make
 * that first call early -- before memory is handed to another owner and
 * before any stream capture.  tfft_exec_noalloc(0, 0, NULL, NULL, 0) performs
 * only that set-up on the current device.  If the device has no memory left
 * for the arrays the call returns TFFT_ERR_ALLOC.  All calls share the arrays
 * and leave the last call's contents in them; calls that overlap on the GPU
 * race and give wrong results.
 */
int tfft_exec_noalloc(int64_t n, int64_t batch, const void *in, void *out, tfft_stream_t stream);

/*
 * Ragged batches: `count` signals of different power-of-two lengths
 * `lengths[i]` (2 <= n <= 2^26 for complex64, 1 <= n for complex128), packed
 * back to back in that order -- signal i starts at element
 * sum_{j<i} lengths[j] of `in` and of `out`.  Section II's batched transform
 * is applied to every signal.  No counterpart in the paper, which batches
 * equal lengths only; the two-sided checksums (Section III) run over groups
 * of G consecutive signals of equal length.
 *
 * tfft_ragged_plan: buckets the signals by length and plans one batched
 * transform per bucket.  A bucket's plan reads and writes its signals where
 * they lie in `in` and `out` (per-signal offsets in the first pass's loads
 * and the last pass's stores, no copies) when its passes allow it: each
 * signal on a 16-byte boundary, and for a multi-pass plan each signal's
 * offset a multiple of the first pass's column-box width (16 elements for
 * complex64).  Other buckets are gathered into a staging area before their
 * transform and scattered back after it.  `flags`:
 *   TFFT_RAGGED_AUTOTUNE  time every pass count (one, two or three launches)
 *                         a bucket's length admits and keep the fastest;
 *   TFFT_RAGGED_STAGED    stage every bucket (the copy-based form, kept for
 *                         comparison);
 *   TFFT_RAGGED_PERSISTENT  run the passes of the buckets whose every pass is
 *                         on the 256-thread complex64 tile kernels as pass
 *                         families: the passes of one role and sub-transform
 *                         length, of all such buckets, in one persistent
 *                         launch whose blocks take (bucket, chunk range)
 *                         items, sorted by work, from an atomic counter; each
 *                         family waits for the families of its buckets'
 *                         previous pass, and each bucket then verifies and
 *                         corrects on its own stream.  The other buckets run
 *                         their plans alongside.
 * The caller's `lengths` array is not kept.
 *
 * tfft_ragged_exec: asynchronous on `stream`; gathers the staged buckets,
 * runs the bucket plans (each on its own stream, joined to `stream`,
 * longest length first), scatters the staged results.  The sequence is
 * captured into a CUDA graph on the first exec with given (in, out) and
 * replayed on the next ones.  `in` and `out` must not overlap
 * (TFFT_ERR_INPLACE).
 *
 * tfft_ragged_report: synchronises the device and sums the bucket plans'
 * counters (execs counts tfft_ragged_exec calls).
 * tfft_ragged_set_fault: test hook, arms a fault (tfft_fault, with `signal`
 * ignored) on caller signal `signal` for the next exec, which then runs
 * uncaptured.
 * tfft_ragged_info: number of buckets, and up to `capacity` of their
 * lengths, pass counts and addressing (direct: 1 in place, 0 staged),
 * longest first; any of the arrays may be NULL.
 * tfft_ragged_families: the pass families of the persistent form and the
 * buckets that run in them (0 and 0 without TFFT_RAGGED_PERSISTENT).
 */
typedef struct tfft_ragged_s *tfft_ragged_t;
enum { TFFT_RAGGED_AUTOTUNE = 1, TFFT_RAGGED_STAGED = 2, TFFT_RAGGED_PERSISTENT = 4 };
int tfft_ragged_plan(tfft_ragged_t *out, const int64_t *lengths, int64_t count, int dtype, int abft_mode,
                     int flags);
int tfft_ragged_exec(tfft_ragged_t r, const void *in, void *out, tfft_stream_t stream);
int tfft_ragged_report(tfft_ragged_t r, tfft_stats *stats);
int tfft_ragged_set_fault(tfft_ragged_t r, int64_t signal, const tfft_fault *fault);
int tfft_ragged_info(tfft_ragged_t r, int64_t *buckets, int64_t *lengths, int *passes, int *direct,
                     int64_t capacity);
int tfft_ragged_families(tfft_ragged_t r, int64_t *families, int64_t *persistent_buckets);
int tfft_ragged_destroy(tfft_ragged_t r);

/*
 * tfft_tc_selftest -- one 128 x 32 x 32 product D = A B on the 5th-generation
 * tensor cores through the same code the split-precision DFT uses (no
 * counterpart in the paper, which has no tensor-core path): `a` 128 x 32 and
 * `d` 128 x 32 row-major FP32, `bt` 32 x 32 FP32 holding B transposed (row n
 * = column n of B), all device pointers; `terms` 1 multiplies the TF32-rounded
 * operands, 3 adds the products of the high and low TF32 parts
 * (a_hi b_hi + a_hi b_lo + a_lo b_hi).  Synchronous; returns
 * TFFT_ERR_TIMEOUT if the product did not complete within the wait bound.
 */
int tfft_tc_selftest(const float *a, const float *bt, float *d, int terms);

/*
 * tfft_measure_fma_peak -- measures the fused multiply-add throughput of the
 * current device (no counterpart in the paper; the denominator of the
 * roofline of transforms the arithmetic units bound, complex128 on GB300):
 * 8 x 256 threads per SM each run eight independent chains of `iters`
 * multiply-adds in FP64 (`fp64` = 1) or FP32 (0), timed with CUDA events after
 * one shorter warm-up launch.  *tflops receives 2 flops per multiply-add over
 * the elapsed time.  Synchronous.  Allocates and frees one small buffer.
 */
int tfft_measure_fma_peak(int fp64, int iters, double *tflops);

/* Static string for a status code. */
const char *tfft_error_string(int status);
/* The last cudaError_t value seen by the library in this process. */
int tfft_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TFFT_H */
