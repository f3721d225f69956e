// tc_selftest.cu -- tfft_tc_selftest: one 128 x 32 x 32 tile through the
// tensor-core path (tc.cuh) in plain or three-term split TF32, for checking
// the descriptors and the tensor-memory handling against a host product.
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/tfft.h"
#include "tc.cuh"

namespace tfft {
namespace {

// One CTA of 128 threads (one warpgroup).  A is 128 x 32 row-major, Bt is
// 32 x 32 with row n holding column n of B, D is 128 x 32 row-major:
// D = A B computed as sum over the split terms of A_x (B_y)^T.
__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(const float* A, const float* Bt, float* D,
                                                             int terms, int* err) {
  __shared__ __align__(1024) unsigned char a_hi[128 * 128];
  __shared__ __align__(1024) unsigned char a_lo[128 * 128];
  __shared__ __align__(1024) unsigned char b_hi[32 * 128];
  __shared__ __align__(1024) unsigned char b_lo[32 * 128];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  const int t = threadIdx.x, warp = t >> 5;

  // operands: rows of 32 values, split into TF32 high and low parts
  for (int c = 0; c < 8; c++) {
    float4 v = reinterpret_cast<const float4*>(A + t * 32)[c];
    float4 h = {tc::to_tf32(v.x), tc::to_tf32(v.y), tc::to_tf32(v.z), tc::to_tf32(v.w)};
    float4 l = {tc::to_tf32(v.x - h.x), tc::to_tf32(v.y - h.y), tc::to_tf32(v.z - h.z), tc::to_tf32(v.w - h.w)};
    *reinterpret_cast<float4*>(a_hi + tc::sw128_off(t, c)) = h;
    *reinterpret_cast<float4*>(a_lo + tc::sw128_off(t, c)) = l;
    if (t < 32) {
      v = reinterpret_cast<const float4*>(Bt + t * 32)[c];
      h = {tc::to_tf32(v.x), tc::to_tf32(v.y), tc::to_tf32(v.z), tc::to_tf32(v.w)};
      l = {tc::to_tf32(v.x - h.x), tc::to_tf32(v.y - h.y), tc::to_tf32(v.z - h.z), tc::to_tf32(v.w - h.w)};
      *reinterpret_cast<float4*>(b_hi + tc::sw128_off(t, c)) = h;
      *reinterpret_cast<float4*>(b_lo + tc::sw128_off(t, c)) = l;
    }
  }
  fence_proxy_async();                 // the generic-proxy writes, before the tensor cores read them
  if (warp == 0) tc::tmem_alloc(&tbase, 32);
  if (t == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t d_tmem = tbase;

  if (t == 0) {
    constexpr uint32_t idesc = tc::instr_desc(2, 128, 32);
    const unsigned char* as[3] = {a_hi, a_hi, a_lo};
    const unsigned char* bs[3] = {b_hi, b_lo, b_hi};
    for (int term = 0; term < terms; term++)
      for (int k = 0; k < 4; k++) {
        const uint64_t ad = tc::smem_desc_sw128(smem_u32(as[term]) + 32u * k);
        const uint64_t bd = tc::smem_desc_sw128(smem_u32(bs[term]) + 32u * k);
        tc::mma_tf32(d_tmem, ad, bd, idesc, (term | k) != 0);
      }
    tc::mma_commit(&bar);
  }
  bool ok = false;
  for (long long it = 0; it < kWaitLimit && !ok; it++) ok = mbar_try_wait(&bar, 0);
  if (!ok) atomicExch(err, 1);
  tc::fence_after_sync();
  float v[32];
  tc::tmem_ld32(d_tmem + ((uint32_t)(32 * (warp & 3)) << 16), v);
  for (int i = 0; i < 32; i++) D[t * 32 + i] = ok ? v[i] : 0.0f;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(d_tmem, 32);
}

}  // namespace
}  // namespace tfft

extern "C" int tfft_tc_selftest(const float* a, const float* bt, float* d, int terms) {
  if (!a || !bt || !d || (terms != 1 && terms != 3)) return TFFT_ERR_INVALID_ARG;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return TFFT_ERR_ALLOC;
  cudaMemset(err, 0, sizeof(int));
  tfft::tc_selftest_kernel<<<1, 128>>>(a, bt, d, terms, err);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return tfft::record_cuda_error(e);
  return h ? TFFT_ERR_TIMEOUT : TFFT_SUCCESS;
}
