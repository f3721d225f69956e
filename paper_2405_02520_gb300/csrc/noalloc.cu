// noalloc.cu -- tfft_exec_noalloc: the two-pass complex64 transform without
// any allocation, for callers that may not allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is unavailable or not
// allowed -- under a memory manager or sandbox that owns every device
// allocation, or in a real-time loop that may not block on the allocator.
// Such callers cannot create a plan (tfft_plan allocates its workspace), so
// this entry point takes only the caller's input and output buffers and uses,
// for the inter-pass buffer and the twiddle tables, file-scope __device__
// arrays of fixed size.
//
// Those arrays (64 MiB + 12 KiB) are reserved on a GPU when this file's
// module is loaded there and stay until the process exits.  With lazy module
// loading (the CUDA default) that happens at the first call on the device,
// which looks up the arrays' addresses: make that first call -- or the
// set-up-only call tfft_exec_noalloc(0, 0, NULL, NULL, 0) -- early, before
// memory is handed to another owner and before any stream capture.  All calls
// share the arrays and they keep the last call's contents; nothing needs to
// start at zero.  Two calls that overlap on the GPU (different streams, or
// different host threads) race on the shared arrays and produce wrong
// results: serialise them.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tfft_internal.h"

using namespace tfft;

namespace {

constexpr int64_t kScratchElems = int64_t(1) << 23;   // complex64 values (64 MiB)
constexpr int kTab = 512;                               // entries per twiddle table
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_scratch[kScratchElems];
static __device__ __align__(256) float2 g_tw_sub[kTab];
static __device__ __align__(256) float2 g_tw_lo[kTab];
static __device__ __align__(256) float2 g_tw_hi[kTab];

// Set-up state of one device: the arrays' device addresses and, per signal
// length 2^m and pass, the resident blocks per SM of the pass kernel.
constexpr int kMinLog2 = 13, kMaxLog2 = 18;
struct DeviceArrays {
  void* scratch = nullptr;
  void* sub = nullptr;
  void* lo = nullptr;
  void* hi = nullptr;
  int sms = 0;
  int bps[kMaxLog2 + 1][2] = {};
  bool ready = false;
};
DeviceArrays g_arrays[kMaxDevices];
std::mutex g_setup_mu;

// omega_T^m = e^{-2 pi i m / T} in FP64 (sincospi of the exact fraction 2m/T,
// reduced to [0, 1) turn), rounded to complex64.
__device__ float2 root_f64(long long m, long long T) {
  m %= T;
  double s, c;
  sincospi(2.0 * (double)m / (double)T, &s, &c);
  return float2{(float)c, (float)-s};
}

__global__ void noalloc_tables_kernel(float2* sub, int T, float2* lo, int L, float2* hi, int H,
                                      long long n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < T) sub[k] = root_f64(k, T);
  if (k < L) lo[k] = root_f64(k, n);
  if (k < H) hi[k] = root_f64((long long)k * L, n);
}

int ilog2_na(int64_t v) { int k = 0; while ((int64_t(1) << k) < v) k++; return k; }

// Factor of the first pass: N1 = 2^ceil(m/2) (both factors <= 512 for N <= 2^18).
int64_t first_factor(int m) { return int64_t(1) << ((m + 1) / 2); }

int symbol_address(void** ptr, const void* symbol) {
  const cudaError_t e = cudaGetSymbolAddress(ptr, symbol);
  if (e == cudaSuccess) return 0;
  cudaGetLastError();
  // the module is loaded (and its arrays reserved) by the first lookup
  return e == cudaErrorMemoryAllocation ? TFFT_ERR_ALLOC : record_cuda_error(e);
}

// Set-up on the current device, done once by the first call on that device:
// the device addresses of the arrays (their names in host code are host-side
// stand-ins and must never be passed to a kernel) and the occupancy of every
// launch the entry point can make.
int device_arrays(int dev, DeviceArrays** out) {
  if (dev < 0 || dev >= kMaxDevices) return TFFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceArrays& a = g_arrays[dev];
  if (!a.ready) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return TFFT_ERR_NO_DEVICE;
    a.sms = prop.multiProcessorCount;
    int rc;
    if ((rc = symbol_address(&a.scratch, g_scratch))) return rc;
    if ((rc = symbol_address(&a.sub, g_tw_sub))) return rc;
    if ((rc = symbol_address(&a.lo, g_tw_lo))) return rc;
    if ((rc = symbol_address(&a.hi, g_tw_hi))) return rc;
    for (int m = kMinLog2; m <= kMaxLog2; m++) {
      PassGeom g[2];
      two_pass_geometry(int64_t(1) << m, first_factor(m), 8, g);
      for (int pass = 0; pass < 2; pass++) {
        int bps = 0;
        const cudaError_t e = pass_func_attrs_f32(g[pass].E, g[pass].smem, g[pass].nthreads, &bps);
        if (e != cudaSuccess) return record_cuda_error(e);
        if (bps < 1) return TFFT_ERR_UNSUPPORTED;
        a.bps[m][pass] = bps;
      }
    }
    a.ready = true;
  }
  *out = &a;
  return 0;
}

}  // namespace

extern "C" int tfft_exec_noalloc(int64_t n, int64_t batch, const void* in, void* out,
                                 tfft_stream_t stream) {
  const bool setup_only = n == 0 && batch == 0;
  if (!setup_only) {
    if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 15u)) return TFFT_ERR_INVALID_ARG;
    if (n < (int64_t(1) << kMinLog2) || n > (int64_t(1) << kMaxLog2) || (n & (n - 1)) || batch < 1)
      return TFFT_ERR_INVALID_ARG;
    if (batch > kScratchElems / n) return TFFT_ERR_INVALID_ARG;   // batch * n above the scratch
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
  DeviceArrays* arr = nullptr;
  int rc = device_arrays(dev, &arr);
  if (rc || setup_only) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // two passes: N1 x N2 with N1 = 2^ceil(m/2) <= 512, N2 <= 512
  const int m = ilog2_na(n);
  const int64_t N1 = first_factor(m), N2 = n / N1;
  PassGeom g[2];
  two_pass_geometry(n, N1, 8, g);
  const int T = (int)std::max(N1, N2);
  const int lb = (m + 1) / 2;
  const int L = 1 << lb, H = (int)((n + L - 1) / L);
  noalloc_tables_kernel<<<(kTab + 255) / 256, 256, 0, s>>>(
      reinterpret_cast<float2*>(arr->sub), T, reinterpret_cast<float2*>(arr->lo), L,
      reinterpret_cast<float2*>(arr->hi), H, (long long)n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return record_cuda_error(e);

  for (int pass = 0; pass < 2; pass++) {
    const PassGeom& q = g[pass];
    PassParams a;
    std::memset(&a, 0, sizeof(a));
    a.nsub = q.nsub; a.log2nsub = ilog2_na(q.nsub); a.C = q.C; a.nthreads = q.nthreads;
    a.nstages = q.nstages; a.pitch = q.pitch;
    a.in_map = q.in_map; a.mid_map = q.mid_map; a.out_map = q.out_map;
    a.n = n; a.batch = batch; a.LO = q.LO; a.HI = q.HI; a.pass_index = pass;
    a.in_es = q.in_es; a.in_lo = q.in_lo; a.in_hi = q.in_hi;
    a.out_es = q.out_es; a.out_lo = q.out_lo; a.out_hi = q.out_hi;
    a.twiddle = q.twiddle; a.tw_scale = q.tw_scale;
    a.out_scale = 1.0;            // forward, unnormalised
    a.in = pass == 0 ? in : arr->scratch;
    a.out = pass == 0 ? arr->scratch : out;
    a.tw_sub = arr->sub; a.tw_sub_stride = (int)(T / q.nsub);
    a.twN_lo = arr->lo; a.twN_hi = arr->hi; a.twN_lbits = lb;
    a.group = 1; a.parts = 1; a.ngroups = batch;
    a.line_blocks = q.line_blocks;
    a.nchunks = batch * a.line_blocks;
    const int64_t grid = std::min<int64_t>(a.nchunks, (int64_t)arr->sms * arr->bps[m][pass]);
    e = launch_pass_f32(a, q.E, (int)grid, q.smem, s);
    if (e != cudaSuccess) return record_cuda_error(e);
  }
  return TFFT_SUCCESS;
}
