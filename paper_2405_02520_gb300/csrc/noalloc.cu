// noalloc.cu -- tfft_exec_noalloc: the two-pass complex64 transform without
// any allocation, for callers that may not allocate device memory.
//
// Who needs this: code running where cudaMalloc is unavailable or forbidden --
// inside a CUDA-graph capture that must not contain allocation nodes, under a
// memory manager or sandbox that owns every device allocation, or in a
// real-time loop that may not block on the allocator.  Such callers cannot
// create a plan (tfft_plan allocates its workspace), so this entry point takes
// only the caller's input and output buffers and uses, for the inter-pass
// buffer and the twiddle tables, file-scope __device__ arrays of fixed size.
//
// Every GPU that loads the library holds those arrays (64 MiB + 12 KiB) until
// the process exits.  All calls share them and they keep the last call's
// contents; nothing needs to start at zero.  Two calls that overlap on the GPU
// (different streams, or different host threads) race on the shared arrays
// and produce wrong results: serialise them.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tfft_internal.h"

namespace {

constexpr int64_t kScratchElems = int64_t(1) << 23;   // complex64 values (64 MiB)
constexpr int kTab = 512;                               // entries per twiddle table
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_scratch[kScratchElems];
static __device__ __align__(256) float2 g_tw_sub[kTab];
static __device__ __align__(256) float2 g_tw_lo[kTab];
static __device__ __align__(256) float2 g_tw_hi[kTab];

struct DeviceArrays {
  void* scratch = nullptr;
  void* sub = nullptr;
  void* lo = nullptr;
  void* hi = nullptr;
  int sms = 0;
  bool sm103 = false;
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

// Set-up on the current device, done by the first call on that device: the
// device addresses of the arrays (their names in host code are host-side
// stand-ins and must never be passed to a kernel).
int device_arrays(int dev, DeviceArrays** out) {
  if (dev < 0 || dev >= kMaxDevices) return TFFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceArrays& a = g_arrays[dev];
  if (!a.ready) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
    a.sm103 = prop.major == 10 && prop.minor == 3;
    a.sms = prop.multiProcessorCount;
    if (!a.sm103) return TFFT_ERR_NO_DEVICE;
    if (cudaGetSymbolAddress(&a.scratch, g_scratch) != cudaSuccess) return TFFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&a.sub, g_tw_sub) != cudaSuccess) return TFFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&a.lo, g_tw_lo) != cudaSuccess) return TFFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&a.hi, g_tw_hi) != cudaSuccess) return TFFT_ERR_CUDA;
    a.ready = true;
  }
  *out = &a;
  return 0;
}

}  // namespace

using namespace tfft;

extern "C" int tfft_exec_noalloc(int64_t n, int64_t batch, const void* in, void* out,
                                 tfft_stream_t stream) {
  if (!in || !out || (((uintptr_t)in | (uintptr_t)out) & 15u)) return TFFT_ERR_INVALID_ARG;
  if (n < 8192 || n > (int64_t(1) << 18) || (n & (n - 1)) || batch < 1) return TFFT_ERR_INVALID_ARG;
  if (batch > kScratchElems / n) return TFFT_ERR_INVALID_ARG;   // batch * n above the scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TFFT_ERR_NO_DEVICE;
  DeviceArrays* arr = nullptr;
  int rc = device_arrays(dev, &arr);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // two passes: N1 x N2 with N1 = 2^ceil(m/2) <= 512, N2 <= 512
  const int m = ilog2_na(n);
  const int64_t N1 = int64_t(1) << ((m + 1) / 2), N2 = n / N1;
  const int E = 16, TILE = 4096, S = 16;
  const int T = (int)std::max(N1, N2);
  const int lb = (m + 1) / 2;
  const int L = 1 << lb, H = (int)((n + L - 1) / L);
  noalloc_tables_kernel<<<(kTab + 255) / 256, 256, 0, s>>>(
      reinterpret_cast<float2*>(arr->sub), T, reinterpret_cast<float2*>(arr->lo), L,
      reinterpret_cast<float2*>(arr->hi), H, (long long)n);
  if (cudaGetLastError() != cudaSuccess) return TFFT_ERR_CUDA;

  for (int pass = 0; pass < 2; pass++) {
    PassParams a;
    std::memset(&a, 0, sizeof(a));
    const int64_t nsub = pass == 0 ? N1 : N2;
    const int64_t LO = pass == 0 ? N2 : N1;
    const int C = (int)std::min<int64_t>(std::min<int64_t>(TILE / nsub, LO), 64);
    a.nsub = (int)nsub; a.log2nsub = ilog2_na(nsub); a.C = C;
    a.nthreads = (int)(C * nsub / E);
    int st = 0; for (int64_t v = 1; v < nsub; v *= E) st++;
    a.nstages = st;
    a.n = n; a.batch = batch; a.LO = LO; a.HI = 1; a.pass_index = pass;
    a.out_scale = 1.0;            // forward, unnormalised
    if (pass == 0) {
      a.in_es = N2; a.in_lo = 1; a.out_es = N2; a.out_lo = 1;
      a.in_map = a.mid_map = a.out_map = MAP_COL;
      a.pitch = (int)nsub + (C < S ? S / C : 1);
      a.twiddle = 1; a.tw_scale = 1;
      a.in = in; a.out = arr->scratch;
    } else {
      a.in_es = 1; a.in_lo = N2; a.out_es = N1; a.out_lo = 1;
      a.in_map = MAP_ROW; a.out_map = MAP_COL;
      a.mid_map = C >= S / 2 ? MAP_COL : MAP_ROW;
      const int lanes = (int)std::max<int64_t>(1, nsub / E);
      a.pitch = (int)nsub + (a.mid_map == MAP_COL ? (C < S ? S / C : 1) : (lanes < S ? lanes : 0));
      a.in = arr->scratch; a.out = out;
    }
    a.tw_sub = arr->sub; a.tw_sub_stride = (int)(T / nsub);
    a.twN_lo = arr->lo; a.twN_hi = arr->hi; a.twN_lbits = lb;
    a.group = 1; a.parts = 1; a.ngroups = batch;
    a.line_blocks = LO / C;
    a.nchunks = batch * a.line_blocks;
    const size_t smem = (size_t)C * a.pitch * sizeof(float2);
    int bps = 0;
    if (pass_func_attrs_f32(E, smem, a.nthreads, &bps) != cudaSuccess || bps < 1) return TFFT_ERR_CUDA;
    const int64_t grid = std::min<int64_t>(a.nchunks, (int64_t)arr->sms * bps);
    if (launch_pass_f32(a, E, (int)grid, smem, s) != cudaSuccess) return TFFT_ERR_CUDA;
  }
  return TFFT_SUCCESS;
}
