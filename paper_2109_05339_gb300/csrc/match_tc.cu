// Tensor-core orientation matching (Sec. II-B) on sm_103a: quantisation of
// images and model images to BF16 / FP8 e4m3, and the fused cross-term +
// top-8 kernel.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <cfloat>

#include "match.h"

namespace spf {

namespace {

// BF16 copy of scale * src rows, zero-padded to Kpad columns.
__global__ void quantize_bf16_kernel(const float* __restrict__ src, int rows, int P2, int Kpad,
                                     float scale, __nv_bfloat16* __restrict__ dst) {
  int64_t total = (int64_t)rows * Kpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(i / Kpad), k = (int)(i - (int64_t)r * Kpad);
    float v = k < P2 ? scale * src[(size_t)r * P2 + k] : 0.f;
    dst[i] = __float2bfloat16_rn(v);
  }
}

// FP8 e4m3 copy with a per-row scale a_r = max_p |scale * src_rp| / 448
// (1 for an all-zero row): dst = e4m3(scale * src / a_r), zero-padded.
__global__ void quantize_fp8_kernel(const float* __restrict__ src, int rows, int P2, int Kpad,
                                    float scale, __nv_fp8_e4m3* __restrict__ dst,
                                    float* __restrict__ row_scale) {
  int r = blockIdx.x;
  if (r >= rows) return;
  const float* row = src + (size_t)r * P2;
  float mx = 0.f;
  for (int k = threadIdx.x; k < P2; k += blockDim.x) mx = fmaxf(mx, fabsf(scale * row[k]));
  __shared__ float sm[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sm[w]);
    sm[0] = m > 0.f ? m / 448.f : 1.f;
    row_scale[r] = sm[0];
  }
  __syncthreads();
  float inv = 1.f / sm[0];
  for (int k = threadIdx.x; k < Kpad; k += blockDim.x) {
    float v = k < P2 ? scale * row[k] * inv : 0.f;
    dst[(size_t)r * Kpad + k] = __nv_fp8_e4m3(v);
  }
}

}  // namespace

int tc_kpad(int P2, int precision) {
  int blk = precision == SPF_BF16 ? 64 : 128;   // one 128-byte swizzle row
  return (int)ceil_div(P2, blk) * blk;
}

int quantize_rows(spf_matcher* m, const float* src, int rows, float scale, void* dst, float* scales,
                  cudaStream_t s) {
  if (rows == 0) return SPF_OK;
  if (m->precision == SPF_BF16) {
    int64_t total = (int64_t)rows * m->Kpad;
    int grid = (int)std::min<int64_t>(ceil_div(total, 256), 152 * 64);
    return launch("quantize_bf16_kernel", s, [&] {
      quantize_bf16_kernel<<<grid, 256, 0, s>>>(src, rows, m->P2, m->Kpad, scale,
                                                static_cast<__nv_bfloat16*>(dst));
    });
  }
  return launch("quantize_fp8_kernel", s, [&] {
    quantize_fp8_kernel<<<rows, 256, 0, s>>>(src, rows, m->P2, m->Kpad, scale,
                                             static_cast<__nv_fp8_e4m3*>(dst), scales);
  });
}

int match_tc_supported(int device) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  return major == 10 && minor == 3;
}

int match_tc_launch(spf_matcher* m, int n_orient, int orient_offset, int nsplit, cudaStream_t s) {
  (void)m; (void)n_orient; (void)orient_offset; (void)nsplit; (void)s;
  set_error("tensor-core matching kernel not built yet");
  return SPF_ERR_UNSUPPORTED;
}

}  // namespace spf
