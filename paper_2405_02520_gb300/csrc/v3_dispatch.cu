// v3_dispatch.cu -- selects the v3 instantiation for (element type, role, nsub).
#include "fft_v3.cuh"

namespace tfft {

cudaError_t v3_launch_f32_single(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f32_single(int nsub, size_t smem, int* bps);
cudaError_t v3_launch_f32_cols(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f32_cols(int nsub, size_t smem, int* bps);
cudaError_t v3_launch_f32_last(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f32_last(int nsub, size_t smem, int* bps);
cudaError_t v3_launch_f64_single(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f64_single(int nsub, size_t smem, int* bps);
cudaError_t v3_launch_f64_cols(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f64_cols(int nsub, size_t smem, int* bps);
cudaError_t v3_launch_f64_last(int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s);
cudaError_t v3_attrs_f64_last(int nsub, size_t smem, int* bps);

cudaError_t launch_v3(int dtype, int role, int nsub, const PassParams& p, int grid, size_t smem, cudaStream_t s) {
  if (dtype == 0) {
    if (role == 0) return v3_launch_f32_single(nsub, p, grid, smem, s);
    if (role == 1) return v3_launch_f32_cols(nsub, p, grid, smem, s);
    return v3_launch_f32_last(nsub, p, grid, smem, s);
  }
  if (role == 0) return v3_launch_f64_single(nsub, p, grid, smem, s);
  if (role == 1) return v3_launch_f64_cols(nsub, p, grid, smem, s);
  return v3_launch_f64_last(nsub, p, grid, smem, s);
}

cudaError_t v3_attrs(int dtype, int role, int nsub, size_t smem, int* bps) {
  if (dtype == 0) {
    if (role == 0) return v3_attrs_f32_single(nsub, smem, bps);
    if (role == 1) return v3_attrs_f32_cols(nsub, smem, bps);
    return v3_attrs_f32_last(nsub, smem, bps);
  }
  if (role == 0) return v3_attrs_f64_single(nsub, smem, bps);
  if (role == 1) return v3_attrs_f64_cols(nsub, smem, bps);
  return v3_attrs_f64_last(nsub, smem, bps);
}

// Values per thread of the 256-thread v3 kernel: 16 for complex64; 8 for
// complex128, except the 4096-point single pass, which takes 16 (one line a
// tile, three radix-16 stages, up to 255 registers a thread at one block per
// SM) so that one pass covers N = 4096.
int v3_radix(int dtype, int nsub) { return dtype == 0 || nsub == 4096 ? 16 : 8; }

// Bytes of the padded line scratch of a v3 kernel.
int v3_scratch_bytes(int dtype, int nsub) {
  const int es = dtype == 1 ? 16 : 8, e = v3_radix(dtype, nsub);
  const int tile = 256 * e, c = tile / nsub, pg = 128 / es;
  const int pitch = nsub + nsub / pg + (nsub < pg ? 1 : 0);
  return c * pitch * es;
}

// Bytes of shared memory the stage-twiddle table takes in a v3 kernel (0 when
// the kernel reads it from global memory).
int v3_twiddle_smem_bytes(int dtype, int nsub) {
  const int es = dtype == 1 ? 16 : 8, e = v3_radix(dtype, nsub);
  const int b = v3_tw_entries(nsub, e) * es;
  return b <= kV3TwSmemMax ? b : 0;
}

}  // namespace tfft
