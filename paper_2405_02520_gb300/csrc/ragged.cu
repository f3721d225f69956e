// ragged.cu -- batches of signals of different lengths (tfft_ragged_*).
//
// The signals of a ragged batch are packed back to back in the caller's
// order.  The plan sorts them into buckets of equal length; each bucket is an
// ordinary batched plan (with the two-sided checksums over groups of G
// consecutive signals of the bucket).  A bucket is either
//
//   * direct: its plan carries the caller offsets of its signals, so the
//     first pass loads each signal where it lies and the last pass stores it
//     back there (no copies), or
//   * staged: an exec gathers it into a contiguous staging area with one copy
//     kernel over 16-byte chunks and scatters the results back (the fallback
//     for offsets a pass cannot address, and the comparison form).
//
// An exec runs the bucket plans, longest length first, each on its own
// stream so that the short transforms of small buckets overlap the long
// ones.  The whole sequence is captured into a CUDA graph on the first exec
// with a given (in, out) and replayed afterwards (no per-kernel launch cost;
// the small buckets are launch-bound).  An exec with a test fault armed runs
// uncaptured.  At plan time an optional autotuner times the pass counts a
// bucket's length admits (one, two or three launches) and keeps the fastest.
//
// The persistent form (TFFT_RAGGED_PERSISTENT) runs the passes of the
// buckets whose every pass is on the 256-thread complex64 tile kernels as
// pass families instead: all passes of one role and sub-transform length, of
// every such bucket, in one persistent launch whose blocks take (bucket,
// chunk range) items, sorted by work, from an atomic counter.  A family waits
// for the families of the previous pass of its buckets; each bucket then
// verifies and corrects on its own stream.  Other buckets run their plans as
// above, alongside.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tfft_internal.h"

using tfft::record_cuda_error;

namespace {

struct Segment {        // one block's share of a gather or scatter
  long long src, dst;   // byte offsets
  long long bytes;      // a multiple of 16
};

__global__ void ragged_copy_kernel(const Segment* seg, long long nseg, const unsigned char* src,
                                   unsigned char* dst) {
  for (long long s = blockIdx.x; s < nseg; s += gridDim.x) {
    const Segment g = seg[s];
    const uint4* a = reinterpret_cast<const uint4*>(src + g.src);
    uint4* b = reinterpret_cast<uint4*>(dst + g.dst);
    const long long n16 = g.bytes >> 4;
    for (long long i = threadIdx.x; i < n16; i += blockDim.x) b[i] = a[i];
  }
}

struct Bucket {
  int64_t n = 0;
  bool persistent = false;    // its passes run in the pass families
  std::vector<int> fam;       // family of each pass (persistent buckets)
  std::vector<int64_t> sig;   // caller indices of the bucket's signals, in order
  int64_t first = 0;          // index of the bucket's first entry in the offset table
  bool direct = false;        // addressed in place through the offset table
  int64_t base = 0;           // staged: element offset of the bucket in the staging areas
  tfft_plan_t plan = nullptr;
  int passes = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

// One pass family of the persistent form: the pass `pass` (role, nsub) of
// every member bucket.
struct Family {
  int pass = 0, role = 0, nsub = 0;
  std::vector<int> members;                   // bucket indices (at most kRaggedMax)
  std::vector<tfft::RaggedItem> items;        // .bucket: index into members
  tfft::RaggedItem* d_items = nullptr;
  size_t smem = 0;
  int grid = 1;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

}  // namespace

struct tfft_ragged_s {
  int dtype = 0, abft = 0;
  size_t esize = 8;
  int64_t count = 0, total = 0;
  std::vector<int64_t> off;          // caller element offset of every signal
  std::vector<int64_t> local;        // index of every signal inside its bucket
  std::vector<int> bucket_of;        // bucket of every signal
  std::vector<Bucket> buckets;
  long long* d_off = nullptr;        // caller offsets, bucket by bucket
  int64_t staged_total = 0;          // elements of the staged buckets
  void* stage_in = nullptr;
  void* stage_out = nullptr;
  Segment* d_gather = nullptr;
  Segment* d_scatter = nullptr;
  long long nseg = 0;
  int sms = 0;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;        // private stream the graph is captured on
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* g_in = nullptr;
  void* g_out = nullptr;
  bool fault_armed = false;
  int64_t execs = 0;
  // persistent form
  std::vector<Family> fams;
  unsigned long long* d_heads = nullptr;      // one item counter per family
  int64_t fam_launches = 0;
  std::mutex mu;
};

namespace {

void free_ragged(tfft_ragged_s* r) {
  if (r->gexec) cudaGraphExecDestroy(r->gexec);
  if (r->graph) cudaGraphDestroy(r->graph);
  for (auto& f : r->fams) {
    if (f.d_items) cudaFree(f.d_items);
    if (f.stream) cudaStreamDestroy(f.stream);
    if (f.done) cudaEventDestroy(f.done);
  }
  if (r->d_heads) cudaFree(r->d_heads);
  for (auto& b : r->buckets) {
    if (b.plan) tfft_destroy(b.plan);
    if (b.stream) cudaStreamDestroy(b.stream);
    if (b.done) cudaEventDestroy(b.done);
  }
  if (r->fork) cudaEventDestroy(r->fork);
  if (r->cap) cudaStreamDestroy(r->cap);
  for (void* p : {r->stage_in, r->stage_out, (void*)r->d_gather, (void*)r->d_scatter, (void*)r->d_off})
    if (p) cudaFree(p);
  delete r;
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Median-free timing of one plan: the mean of a few execs after a warm-up.
float time_plan(tfft_plan_t p, const void* in, void* out, cudaStream_t s) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  tfft_exec(p, in, out, s);
  cudaEventRecord(a, s);
  for (int i = 0; i < 3; i++) tfft_exec(p, in, out, s);
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

int launch_copy(const tfft_ragged_s* r, const Segment* seg, const void* src, void* dst, cudaStream_t s) {
  if (r->nseg == 0) return TFFT_SUCCESS;
  const long long grid = std::min<long long>(r->nseg, (long long)r->sms * 8);
  ragged_copy_kernel<<<(unsigned)grid, 256, 0, s>>>(seg, r->nseg, static_cast<const unsigned char*>(src),
                                                     static_cast<unsigned char*>(dst));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TFFT_SUCCESS : record_cuda_error(e);
}

const void* bucket_in(const tfft_ragged_s* r, const Bucket& b, const void* in) {
  return b.direct ? in : static_cast<const unsigned char*>(r->stage_in) + (size_t)b.base * r->esize;
}
void* bucket_out(const tfft_ragged_s* r, const Bucket& b, void* out) {
  return b.direct ? out : static_cast<unsigned char*>(r->stage_out) + (size_t)b.base * r->esize;
}

// gather (staged buckets), the pass families and each persistent bucket's
// verification, the other bucket plans on their streams, scatter -- all on or
// joined to `s`
int enqueue(tfft_ragged_s* r, const void* in, void* out, cudaStream_t s) {
  int rc;
  if ((rc = launch_copy(r, r->d_gather, in, r->stage_in, s))) return rc;
  cudaError_t e;
  if (!r->fams.empty() &&
      (e = cudaMemsetAsync(r->d_heads, 0, r->fams.size() * sizeof(unsigned long long), s)) != cudaSuccess)
    return record_cuda_error(e);
  if ((e = cudaEventRecord(r->fork, s)) != cudaSuccess) return record_cuda_error(e);
  // families in pass order: each after the families of its buckets' previous pass
  for (size_t fi = 0; fi < r->fams.size(); fi++) {
    Family& f = r->fams[fi];
    if (f.pass == 0) {
      if ((e = cudaStreamWaitEvent(f.stream, r->fork, 0)) != cudaSuccess) return record_cuda_error(e);
    } else {
      std::vector<int> deps;
      for (int m : f.members) deps.push_back(r->buckets[m].fam[f.pass - 1]);
      std::sort(deps.begin(), deps.end());
      deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
      for (int d : deps)
        if ((e = cudaStreamWaitEvent(f.stream, r->fams[d].done, 0)) != cudaSuccess) return record_cuda_error(e);
    }
    // the members' parameters for this (in, out), with any armed test fault
    tfft::RaggedParams rp{};
    for (size_t k = 0; k < f.members.size(); k++) {
      const Bucket& b = r->buckets[f.members[k]];
      if ((rc = tfft::plan_pass_params(b.plan, bucket_in(r, b, in), bucket_out(r, b, out), f.pass, &rp.pp[k])))
        return rc;
    }
    rp.nitems = (long long)f.items.size();
    rp.items = f.d_items;
    rp.head = r->d_heads + fi;
    if ((e = tfft::launch_v3_ragged(f.role, f.nsub, rp, f.grid, f.smem, f.stream)) != cudaSuccess)
      return record_cuda_error(e);
    r->fam_launches++;
    if ((e = cudaEventRecord(f.done, f.stream)) != cudaSuccess) return record_cuda_error(e);
  }
  for (auto& b : r->buckets) {
    const void* bin = bucket_in(r, b, in);
    void* bout = bucket_out(r, b, out);
    if (b.persistent) {
      if ((e = cudaStreamWaitEvent(b.stream, r->fams[b.fam.back()].done, 0)) != cudaSuccess)
        return record_cuda_error(e);
      if ((rc = tfft::plan_exec_checks(b.plan, bin, bout, b.stream))) return rc;
      tfft::plan_exec_finish(b.plan, b.stream);
    } else {
      if ((e = cudaStreamWaitEvent(b.stream, r->fork, 0)) != cudaSuccess) return record_cuda_error(e);
      if ((rc = tfft_exec(b.plan, bin, bout, (tfft_stream_t)b.stream))) return rc;
    }
    if ((e = cudaEventRecord(b.done, b.stream)) != cudaSuccess) return record_cuda_error(e);
    if ((e = cudaStreamWaitEvent(s, b.done, 0)) != cudaSuccess) return record_cuda_error(e);
  }
  return launch_copy(r, r->d_scatter, r->stage_out, out, s);
}

// The pass families of the buckets whose every pass a persistent kernel
// covers; their work items (ranges of chunks of about equal work, at least
// four tiles each, about four per block of a full grid) sorted largest
// first.  (About one item per block, each at least eight tiles, measured
// slower: 1.90 against 1.87 ms on the 20,000-signal batch; the balance of
// the last items outweighs the restart of the tile pipeline at each item.)
int plan_families(tfft_ragged_s* r) {
  std::map<std::tuple<int, int, int>, int> index;
  for (size_t bi = 0; bi < r->buckets.size(); bi++) {
    Bucket& b = r->buckets[bi];
    std::vector<tfft::RaggedPass> rp(b.passes);
    bool ok = true;
    for (int i = 0; i < b.passes && ok; i++) {
      if (tfft::plan_ragged_pass(b.plan, i, &rp[i]) != TFFT_SUCCESS) return TFFT_ERR_INVALID_ARG;
      ok = rp[i].ok != 0;
    }
    if (!ok) continue;
    b.persistent = true;
    b.fam.resize(b.passes);
    for (int i = 0; i < b.passes; i++) {
      const auto key = std::make_tuple(i, rp[i].role, rp[i].nsub);
      auto it = index.find(key);
      if (it != index.end() && r->fams[it->second].members.size() >= (size_t)tfft::kRaggedMax) {
        index.erase(it);                  // a full family: the next members start another
        it = index.end();
      }
      if (it == index.end()) {
        it = index.emplace(key, (int)r->fams.size()).first;
        r->fams.emplace_back();
        Family& f = r->fams.back();
        f.pass = i; f.role = rp[i].role; f.nsub = rp[i].nsub;
      }
      Family& f = r->fams[it->second];
      f.smem = std::max(f.smem, rp[i].smem);
      b.fam[i] = it->second;
      const int mk = (int)f.members.size();
      f.members.push_back((int)bi);
      // the member's items, appended; sized below once every member is known
      f.items.push_back(tfft::RaggedItem{mk, rp[i].tiles_per_chunk, 0, rp[i].nchunks});
    }
  }
  // families in pass order (stable), so that a family's dependencies come first
  std::vector<int> order(r->fams.size());
  for (size_t k = 0; k < order.size(); k++) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return r->fams[a].pass < r->fams[b].pass; });
  std::vector<int> where(order.size());
  for (size_t k = 0; k < order.size(); k++) where[order[k]] = (int)k;
  std::vector<Family> sorted;
  for (int k : order) sorted.push_back(std::move(r->fams[k]));
  r->fams = std::move(sorted);
  for (auto& b : r->buckets)
    for (int& fi : b.fam) fi = where[fi];
  for (auto& f : r->fams) {
    int bps = 0;
    cudaError_t e = tfft::v3_ragged_attrs(f.role, f.nsub, f.smem, &bps);
    if (e != cudaSuccess || bps < 1) { cudaGetLastError(); return TFFT_ERR_UNSUPPORTED; }
    const int64_t cap = (int64_t)r->sms * bps;
    // one entry per member so far: {member, tiles a chunk, 0, chunks}
    std::vector<tfft::RaggedItem> whole = std::move(f.items);
    f.items.clear();
    int64_t tiles = 0;
    for (const auto& w : whole) tiles += (int64_t)w.pad * w.c1;
    const int64_t item_tiles = std::max<int64_t>(4, (tiles + 4 * cap - 1) / (4 * cap));
    std::vector<std::pair<int64_t, tfft::RaggedItem>> items;
    for (const auto& w : whole) {
      const int64_t per = std::max<int64_t>(1, (item_tiles + w.pad - 1) / w.pad);    // chunks an item
      for (int64_t c = 0; c < w.c1; c += per) {
        const int64_t c1 = std::min<int64_t>(w.c1, c + per);
        items.push_back({(c1 - c) * w.pad, tfft::RaggedItem{w.bucket, 0, c, c1}});
      }
    }
    std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    for (const auto& it : items) f.items.push_back(it.second);
    f.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)f.items.size(), cap));
    if (cudaMalloc(&f.d_items, f.items.size() * sizeof(tfft::RaggedItem)) != cudaSuccess ||
        cudaMemcpy(f.d_items, f.items.data(), f.items.size() * sizeof(tfft::RaggedItem), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&f.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return TFFT_ERR_ALLOC;
    }
  }
  if (!r->fams.empty() && cudaMalloc(&r->d_heads, r->fams.size() * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return TFFT_ERR_ALLOC;
  }
  return TFFT_SUCCESS;
}

// A scratch pair of the packed size for the autotuner's timings of direct
// buckets (zeroed, freed after planning).
struct Scratch {
  void* in = nullptr;
  void* out = nullptr;
  ~Scratch() {
    if (in) cudaFree(in);
    if (out) cudaFree(out);
  }
};

// Plans bucket `b` (force_passes = 0: the planner's choice); a direct bucket
// gets the offset table, and a plan that cannot take it fails with
// TFFT_ERR_UNSUPPORTED.
int plan_bucket(tfft_ragged_s* r, const Bucket& b, const std::vector<long long>& hoff, int force_passes,
                bool direct, tfft_plan_t* out) {
  tfft_plan_opts o;
  std::memset(&o, 0, sizeof(o));
  o.n = b.n; o.batch = (int64_t)b.sig.size(); o.dtype = r->dtype; o.abft_mode = r->abft;
  o.force_passes = force_passes;
  int rc = tfft_plan_ex(out, &o);
  if (rc) return rc;
  if (direct) {
    static_assert(sizeof(long long) == sizeof(int64_t), "offset table entries are 64-bit");
    rc = tfft::plan_set_signal_offsets(*out, r->d_off + b.first,
                                       reinterpret_cast<const int64_t*>(hoff.data()) + b.first, r->total);
    if (rc) { tfft_destroy(*out); *out = nullptr; }
  }
  return rc;
}

}  // namespace

extern "C" int tfft_ragged_plan(tfft_ragged_t* out, const int64_t* lengths, int64_t count, int dtype,
                                int abft_mode, int flags) {
  if (!out || !lengths || count < 1 ||
      (flags & ~(TFFT_RAGGED_AUTOTUNE | TFFT_RAGGED_STAGED | TFFT_RAGGED_PERSISTENT)))
    return TFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype != TFFT_C64 && dtype != TFFT_C128) return TFFT_ERR_UNSUPPORTED;
  const int64_t nmin = dtype == TFFT_C64 ? 2 : 1;   // every signal starts on a 16-byte boundary
  for (int64_t i = 0; i < count; i++)
    if (!pow2(lengths[i]) || lengths[i] < nmin || lengths[i] > (int64_t(1) << 26)) return TFFT_ERR_INVALID_ARG;
  const bool autotune = flags & TFFT_RAGGED_AUTOTUNE, all_staged = flags & TFFT_RAGGED_STAGED;
  tfft_ragged_s* r = new (std::nothrow) tfft_ragged_s();
  if (!r) return TFFT_ERR_ALLOC;
  r->dtype = dtype;
  r->abft = abft_mode;
  r->esize = dtype == TFFT_C64 ? 8 : 16;
  r->count = count;
  r->off.resize(count);
  r->local.resize(count);
  r->bucket_of.resize(count);
  std::map<int64_t, int> index;
  for (int64_t i = 0; i < count; i++) {
    r->off[i] = r->total;
    r->total += lengths[i];
    auto it = index.find(lengths[i]);
    if (it == index.end()) {
      it = index.emplace(lengths[i], (int)r->buckets.size()).first;
      r->buckets.emplace_back();
      r->buckets.back().n = lengths[i];
    }
    Bucket& b = r->buckets[it->second];
    r->bucket_of[i] = it->second;
    r->local[i] = (int64_t)b.sig.size();
    b.sig.push_back(i);
  }
  // longest first: the big transforms start first
  std::sort(r->buckets.begin(), r->buckets.end(), [](const Bucket& a, const Bucket& b) { return a.n > b.n; });
  for (size_t k = 0; k < r->buckets.size(); k++)
    for (int64_t s : r->buckets[k].sig) r->bucket_of[s] = (int)k;
  // offset table: the caller offsets of every bucket's signals, bucket by bucket
  std::vector<long long> hoff;
  hoff.reserve(count);
  for (auto& b : r->buckets) {
    b.first = (int64_t)hoff.size();
    for (int64_t s : b.sig) hoff.push_back((long long)r->off[s]);
  }
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    free_ragged(r);
    return TFFT_ERR_NO_DEVICE;
  }
  r->sms = prop.multiProcessorCount;
  if (cudaMalloc(&r->d_off, hoff.size() * sizeof(long long)) != cudaSuccess ||
      cudaMemcpy(r->d_off, hoff.data(), hoff.size() * sizeof(long long), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&r->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    free_ragged(r);
    return TFFT_ERR_ALLOC;
  }
  // bucket plans: direct where the plan takes the offsets, else staged
  for (auto& b : r->buckets) {
    if (cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_ragged(r);
      return TFFT_ERR_CUDA;
    }
    int rc = TFFT_ERR_UNSUPPORTED;
    if (!all_staged) {
      rc = plan_bucket(r, b, hoff, 0, true, &b.plan);
      b.direct = rc == TFFT_SUCCESS;
    }
    if (rc == TFFT_ERR_UNSUPPORTED) rc = plan_bucket(r, b, hoff, 0, false, &b.plan);
    if (rc) { free_ragged(r); return rc; }
    tfft_info info;
    tfft_plan_info(b.plan, &info);
    b.passes = info.passes;
  }
  // staging areas and copy segments (of at most 64 KiB) for the staged buckets
  for (auto& b : r->buckets)
    if (!b.direct) {
      b.base = r->staged_total;
      r->staged_total += (int64_t)b.sig.size() * b.n;
    }
  std::vector<Segment> gat, sca;
  if (r->staged_total) {
    const size_t bytes = (size_t)r->staged_total * r->esize;
    if (cudaMalloc(&r->stage_in, bytes) != cudaSuccess || cudaMalloc(&r->stage_out, bytes) != cudaSuccess ||
        cudaMemset(r->stage_in, 0, bytes) != cudaSuccess) {
      cudaGetLastError();
      free_ragged(r);
      return TFFT_ERR_ALLOC;
    }
    const long long kSeg = 64 * 1024;
    for (const auto& b : r->buckets) {
      if (b.direct) continue;
      for (size_t j = 0; j < b.sig.size(); j++) {
        const long long src = (long long)r->off[b.sig[j]] * (long long)r->esize;
        const long long dst = (long long)(b.base + (int64_t)j * b.n) * (long long)r->esize;
        const long long len = (long long)b.n * (long long)r->esize;
        for (long long o = 0; o < len; o += kSeg) {
          const long long L = std::min(kSeg, len - o);
          gat.push_back(Segment{src + o, dst + o, L});
          sca.push_back(Segment{dst + o, src + o, L});
        }
      }
    }
    r->nseg = (long long)gat.size();
    if (cudaMalloc(&r->d_gather, gat.size() * sizeof(Segment)) != cudaSuccess ||
        cudaMalloc(&r->d_scatter, sca.size() * sizeof(Segment)) != cudaSuccess ||
        cudaMemcpy(r->d_gather, gat.data(), gat.size() * sizeof(Segment), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r->d_scatter, sca.data(), sca.size() * sizeof(Segment), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      free_ragged(r);
      return TFFT_ERR_ALLOC;
    }
  }
  // the autotuner times every pass count the length admits (a direct bucket
  // keeps only plans that take the offsets) on zeroed buffers of the packed
  // size
  if (autotune) {
    Scratch sc;
    const bool any_direct = std::any_of(r->buckets.begin(), r->buckets.end(), [](const Bucket& b) { return b.direct; });
    if (any_direct) {
      const size_t bytes = (size_t)r->total * r->esize;
      if (cudaMalloc(&sc.in, bytes) != cudaSuccess || cudaMalloc(&sc.out, bytes) != cudaSuccess ||
          cudaMemset(sc.in, 0, bytes) != cudaSuccess) {
        cudaGetLastError();
        free_ragged(r);
        return TFFT_ERR_ALLOC;
      }
    }
    for (auto& b : r->buckets) {
      const size_t boff = (size_t)b.base * r->esize;
      const void* in = b.direct ? sc.in : static_cast<unsigned char*>(r->stage_in) + boff;
      void* o2 = b.direct ? sc.out : static_cast<unsigned char*>(r->stage_out) + boff;
      float best = time_plan(b.plan, in, o2, b.stream);
      for (int passes = 1; passes <= 3; passes++) {
        if (passes == b.passes) continue;
        tfft_plan_t alt = nullptr;
        if (plan_bucket(r, b, hoff, passes, b.direct, &alt) != TFFT_SUCCESS) { cudaGetLastError(); continue; }
        const float ms = time_plan(alt, in, o2, b.stream);
        if (ms < best) {
          tfft_destroy(b.plan);
          b.plan = alt;
          b.passes = passes;
          best = ms;
        } else {
          tfft_destroy(alt);
        }
      }
      tfft_reset_counters(b.plan);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { free_ragged(r); return TFFT_ERR_CUDA; }
  }
  if (flags & TFFT_RAGGED_PERSISTENT) {
    const int rc = plan_families(r);
    if (rc) { free_ragged(r); return rc; }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { free_ragged(r); return TFFT_ERR_CUDA; }
  *out = r;
  return TFFT_SUCCESS;
}

extern "C" int tfft_ragged_exec(tfft_ragged_t r, const void* in, void* out, tfft_stream_t stream) {
  if (!r || !in || !out || (((uintptr_t)in | (uintptr_t)out) & 15u)) return TFFT_ERR_INVALID_ARG;
  const size_t bytes = (size_t)r->total * r->esize;
  const uintptr_t a = (uintptr_t)in, b = (uintptr_t)out;
  if (a < b + bytes && b < a + bytes) return TFFT_ERR_INPLACE;
  std::lock_guard<std::mutex> lk(r->mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  r->execs++;
  if (r->fault_armed) {                  // a test fault: run once, uncaptured
    r->fault_armed = false;
    return enqueue(r, in, out, s);
  }
  if (!r->gexec || r->g_in != in || r->g_out != out) {
    // captured on a private stream (the legacy default stream cannot be
    // captured), launched on the caller's
    if (r->gexec) { cudaGraphExecDestroy(r->gexec); r->gexec = nullptr; }
    if (r->graph) { cudaGraphDestroy(r->graph); r->graph = nullptr; }
    cudaError_t e = cudaStreamBeginCapture(r->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return record_cuda_error(e);
    const int rc = enqueue(r, in, out, r->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(r->cap, &g);
    if (rc || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return rc ? rc : record_cuda_error(e);
    }
    r->graph = g;
    if ((e = cudaGraphInstantiate(&r->gexec, g, 0)) != cudaSuccess) {
      r->gexec = nullptr;
      return record_cuda_error(e);
    }
    r->g_in = in; r->g_out = out;
  }
  const cudaError_t e = cudaGraphLaunch(r->gexec, s);
  return e == cudaSuccess ? TFFT_SUCCESS : record_cuda_error(e);
}

extern "C" int tfft_ragged_report(tfft_ragged_t r, tfft_stats* st) {
  if (!r || !st) return TFFT_ERR_INVALID_ARG;
  std::memset(st, 0, sizeof(*st));
  if (cudaDeviceSynchronize() != cudaSuccess) return TFFT_ERR_CUDA;
  for (auto& b : r->buckets) {
    tfft_stats s;
    const int rc = tfft_report_ex(b.plan, &s);
    if (rc) return rc;
    st->detected += s.detected;
    st->corrected += s.corrected;
    st->recomputed += s.recomputed;
    st->uncorrectable += s.uncorrectable;
    st->launches += s.launches;
    st->max_clean_ratio = std::max(st->max_clean_ratio, s.max_clean_ratio);
  }
  st->launches += r->fam_launches;
  st->execs = r->execs;
  return TFFT_SUCCESS;
}

extern "C" int tfft_ragged_set_fault(tfft_ragged_t r, int64_t signal, const tfft_fault* fault) {
  if (!r || !fault || signal < 0 || signal >= r->count) return TFFT_ERR_INVALID_ARG;
  tfft_fault f = *fault;
  f.signal = r->local[signal];
  const int rc = tfft_set_fault(r->buckets[r->bucket_of[signal]].plan, &f);
  if (rc == TFFT_SUCCESS) r->fault_armed = true;
  return rc;
}

extern "C" int tfft_ragged_info(tfft_ragged_t r, int64_t* buckets, int64_t* lengths, int* passes, int* direct,
                                int64_t capacity) {
  if (!r || !buckets) return TFFT_ERR_INVALID_ARG;
  *buckets = (int64_t)r->buckets.size();
  for (int64_t k = 0; k < std::min<int64_t>(capacity, *buckets); k++) {
    if (lengths) lengths[k] = r->buckets[k].n;
    if (passes) passes[k] = r->buckets[k].passes;
    if (direct) direct[k] = r->buckets[k].direct ? 1 : 0;
  }
  return TFFT_SUCCESS;
}

extern "C" int tfft_ragged_families(tfft_ragged_t r, int64_t* families, int64_t* persistent_buckets) {
  if (!r || !families || !persistent_buckets) return TFFT_ERR_INVALID_ARG;
  *families = (int64_t)r->fams.size();
  *persistent_buckets = 0;
  for (const auto& b : r->buckets) *persistent_buckets += b.persistent ? 1 : 0;
  return TFFT_SUCCESS;
}

extern "C" int tfft_ragged_destroy(tfft_ragged_t r) {
  if (!r) return TFFT_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_ragged(r);
  return TFFT_SUCCESS;
}
