// Internal layout of an orientation matcher (Sec. II-B).
#pragma once

#include "common.h"

// Image element as FP32: FP32 rows, or 16-bit photon counts (exact in FP32).
static __device__ __forceinline__ float img_elem(const float* x, int p) { return __ldg(x + p); }
static __device__ __forceinline__ float img_elem(const uint16_t* x, int p) { return (float)__ldg(x + p); }
// Four consecutive elements from 4 * p (16-byte FP32 or 8-byte 16-bit load).
static __device__ __forceinline__ float4 img_elem4(const float* x, int p) {
  return __ldg(reinterpret_cast<const float4*>(x) + p);
}
static __device__ __forceinline__ float4 img_elem4(const uint16_t* x, int p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(x) + p);
  return make_float4((float)(u.x & 0xffffu), (float)(u.x >> 16), (float)(u.y & 0xffffu), (float)(u.y >> 16));
}

constexpr int kCand = 8;          // approximate candidates kept per (image, split)
constexpr int kMaxSplits = 64;    // orientation splits of one GEMM launch
constexpr int kMaxChunks = 1024;  // orientation chunks of one deferred re-rank

struct spf_matcher {
  int device = 0;
  int max_images = 0, max_orient = 0, P2 = 0;
  int precision = SPF_FP32, topk = 8;
  int Kpad = 0;                   // padded row length of quantised copies
  int n_img = 0;
  float img_scale = 1.f;
  const float* images = nullptr;
  const uint16_t* images16 = nullptr;   // 16-bit photon counts instead (BF16 / FP8 paths)
  float* x2 = nullptr;            // |img_scale * x_i|^2 (of the quantised rows on the tensor-core paths)
  float* y2 = nullptr;            // |y_j|^2 of the current chunk (likewise)
  void* xq = nullptr;             // quantised images  (max_images x Kpad)
  void* yq = nullptr;             // quantised slices  (max_orient x Kpad)
  float* xs = nullptr;            // FP8 per-image scales
  float* ys = nullptr;            // FP8 per-slice scales
  float* cand_v = nullptr;        // max_images x kMaxSplits x kCand approx scores
  int* cand_i = nullptr;          // ... orientation indices (-1 empty)
  float* st_d = nullptr;          // max_images x topk exact distances (running)
  int* st_i = nullptr;            // max_images x topk indices
  int* err = nullptr;             // device error word (bounded waits, bounds)
  float* wbuf = nullptr;          // P2 square roots of the pixel weights (allocated at create)
  const float* wsq = nullptr;     // == wbuf when a weight mask is set, else nullptr
  // re-rank order (images grouped by their best candidate, so that images
  // sharing candidate model images are re-ranked together and those rows are
  // read from L2); nullptr: natural order
  int* rr_key = nullptr;          // max_images
  int* rr_start = nullptr;        // max_orient + 1 bucket starts / cursors
  int* rr_order = nullptr;        // max_images
  int n_sms = 152;
  int tc_force = 0;               // tensor-core schedule: 0 by the model, 1 contiguous, 2 grid
  // deferred re-rank: the approximate top-kCand per image is carried across
  // orientation chunks and re-ranked once, reading rows from every chunk
  int defer = 0;
  bool pending = false;
  float* ap_v = nullptr;          // max_images x kCand running approximate list
  int* ap_i = nullptr;
  int n_chunks = 0;
  int ch_off_h[kMaxChunks + 1];   // chunk c holds orientations [ch_off[c], ch_off[c + 1])
  const float* ch_ptr_h[kMaxChunks];
  int* ch_off_d = nullptr;
  const float** ch_ptr_d = nullptr;
};

namespace spf {
int match_tc_launch(spf_matcher* m, int n_orient, int orient_offset, int nsplit, cudaStream_t s);
int match_tc_supported(int device);
// out[i] = (float)counts[i], i < n (device buffers).
int counts_to_f32(const uint16_t* counts, int64_t n, float* out, cudaStream_t s);
// Launch schedule of the tensor-core matching kernel (match_tc.cu).
struct TcSched {
  int mode = 0;       // 0: contiguous tile ranges, 1: gi x go grid of image x orientation tile ranges
  int grid = 1;       // CTAs
  int nsplit = 1;     // candidate slots per image the launch writes
  int gi = 0, go = 0;
  double cost = 0.0;  // modelled seconds
};
TcSched tc_schedule(int n_img, int n_orient, int n_sms, int kpad, bool fp8, int force = 0);
}  // namespace spf
