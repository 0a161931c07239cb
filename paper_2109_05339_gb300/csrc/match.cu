// Orientation matching (Sec. II-B): squared Euclidean distance between every
// image and every model image, argmin per image, in three stages.
//
// 1. The cross term x.y of a tile of images against a range of orientations
//    with the norms folded in, keeping a running top-8 list per image so the
//    n_img x n_orient distance matrix never reaches HBM. This file holds the
//    FP32 CUDA-core version (the "plain FP32" path); match_tc.cu holds the
//    BF16 / FP8 tensor-core version writing the same candidate lists.
// 2. Re-rank: per image, merge the candidate lists of all orientation splits
//    by approximate distance (ties to the lower index), take the best topk
//    and recompute their distances exactly in FP32 in the difference form
//    sum_p (x_p - y_p)^2, then merge them into the running list that survives
//    across orientation chunks.
// 3. Results: best index, best and second-best distances.
#include <cfloat>
#include <cmath>

#include "match.h"

namespace spf {

namespace {

// ---------------------------------------------------------------- norms ---
// out[r] = |scale * src_r|^2, one warp per row, FP64 accumulation.
__global__ void row_norms_kernel(const float* __restrict__ src, int rows, int P2, float scale,
                                 float* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const float* row = src + (size_t)warp * P2;
  double acc = 0.0;
  for (int p = lane; p < P2; p += 32) {
    float v = scale * row[p];
    acc += (double)v * (double)v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = (float)acc;
}

__global__ void state_reset_kernel(float* __restrict__ d, int* __restrict__ idx, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    d[i] = FLT_MAX;
    idx[i] = -1;
  }
}

// Insert (s, j) into an ascending list of K entries; equal scores keep the
// earlier entry first, so scanning candidates in increasing j breaks ties to
// the lower index.
template <int K>
__device__ __forceinline__ void list_insert(float* tv, int* ti, float s, int j) {
  if (!(s < tv[K - 1])) return;
  bool placed = false;
#pragma unroll
  for (int q = K - 1; q > 0; --q) {
    bool shift = s < tv[q - 1];
    float nv = shift ? tv[q - 1] : s;
    int ni = shift ? ti[q - 1] : j;
    if (!placed) {
      tv[q] = nv;
      ti[q] = ni;
    }
    placed = placed || !shift;
  }
  if (!placed) {
    tv[0] = s;
    ti[0] = j;
  }
}

// Ordering on (score, index) used when candidate streams are merged out of order.
__device__ __forceinline__ bool before(float a, int ia, float b, int ib) {
  return a < b || (a == b && (unsigned)ia < (unsigned)ib);
}

template <int K>
__device__ __forceinline__ void list_insert_ordered(float* tv, int* ti, float s, int j) {
  if (!before(s, j, tv[K - 1], ti[K - 1])) return;
  bool placed = false;
#pragma unroll
  for (int q = K - 1; q > 0; --q) {
    bool shift = before(s, j, tv[q - 1], ti[q - 1]);
    float nv = shift ? tv[q - 1] : s;
    int ni = shift ? ti[q - 1] : j;
    if (!placed) {
      tv[q] = nv;
      ti[q] = ni;
    }
    placed = placed || !shift;
  }
  if (!placed) {
    tv[0] = s;
    ti[0] = j;
  }
}

// ----------------------------------------------------- FP32 SIMT GEMM ----
// CTA tile: 128 images x 128 orientations, 256 threads with 8x8 outputs,
// k-tiles of 16 staged through shared memory (register prefetch of the next
// tile). Grid: (image tiles, orientation splits); each CTA walks its range
// of orientation tiles and keeps a running top-8 per image row in the
// registers of threads 0..127.
constexpr int BM = 128, BN = 128, BK = 16;

__global__ void __launch_bounds__(256, 2)
simt_match_kernel(const float* __restrict__ X, int n_img, float xscale, const float* __restrict__ Y,
                  int n_orient, int orient_offset, int P2, const float* __restrict__ y2,
                  int tiles_per_split, float* __restrict__ cand_v, int* __restrict__ cand_i) {
  extern __shared__ float smem[];
  float* As = smem;                    // [BK][BM]
  float* Bs = As + BK * BM;            // [BK][BN]
  float* Sc = Bs + BK * BN;            // [BM][BN+1]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * BM;
  const int split = blockIdx.y;
  const int n_ot = (n_orient + BN - 1) / BN;
  const int ot_begin = split * tiles_per_split;
  const int ot_end = min(n_ot, ot_begin + tiles_per_split);

  float tv[kCand];
  int ti[kCand];
#pragma unroll
  for (int q = 0; q < kCand; ++q) {
    tv[q] = FLT_MAX;
    ti[q] = -1;
  }

  // global->register loader mapping: 2048 elements per operand tile
  const int lrow = tid >> 2;           // 0..63 (+64)
  const int lk = (tid & 3) * 4;        // 0,4,8,12

  for (int ot = ot_begin; ot < ot_end; ++ot) {
    const int j0 = ot * BN;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;

    float ra[8], rb[8];
    auto load_tile = [&](int k0) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int row = lrow + 64 * h;
        int gi = i0 + row, gj = j0 + row;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          int k = k0 + lk + e;
          ra[h * 4 + e] = (gi < n_img && k < P2) ? xscale * X[(size_t)gi * P2 + k] : 0.f;
          rb[h * 4 + e] = (gj < n_orient && k < P2) ? Y[(size_t)gj * P2 + k] : 0.f;
        }
      }
    };
    load_tile(0);
    for (int k0 = 0; k0 < P2; k0 += BK) {
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          As[(lk + e) * BM + lrow + 64 * h] = ra[h * 4 + e];
          Bs[(lk + e) * BN + lrow + 64 * h] = rb[h * 4 + e];
        }
      __syncthreads();
      if (k0 + BK < P2) load_tile(k0 + BK);
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        float4 a0 = *reinterpret_cast<const float4*>(As + k * BM + ty * 4);
        float4 a1 = *reinterpret_cast<const float4*>(As + k * BM + 64 + ty * 4);
        float4 b0 = *reinterpret_cast<const float4*>(Bs + k * BN + tx * 4);
        float4 b1 = *reinterpret_cast<const float4*>(Bs + k * BN + 64 + tx * 4);
        float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
    }
    __syncthreads();
    // scores y2 - 2 x.y into the shared tile (rows: ty*4+a or 64+ty*4+a)
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      int r = (a < 4) ? ty * 4 + a : 64 + ty * 4 + (a - 4);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        int c = (b < 4) ? tx * 4 + b : 64 + tx * 4 + (b - 4);
        int gj = j0 + c;
        float yy = gj < n_orient ? y2[gj] : 0.f;
        Sc[r * (BN + 1) + c] = gj < n_orient ? fmaf(-2.f, acc[a][b], yy) : FLT_MAX;
      }
    }
    __syncthreads();
    if (tid < BM) {
      for (int c = 0; c < BN && j0 + c < n_orient; ++c)
        list_insert<kCand>(tv, ti, Sc[tid * (BN + 1) + c], orient_offset + j0 + c);
    }
  }
  if (tid < BM && i0 + tid < n_img) {
    size_t o = ((size_t)(i0 + tid) * kMaxSplits + split) * kCand;
#pragma unroll
    for (int q = 0; q < kCand; ++q) {
      cand_v[o + q] = tv[q];
      cand_i[o + q] = ti[q];
    }
  }
}

// ------------------------------------------------------------ rerank -----
// One CTA per image: merge nsplit candidate lists, take the best topk by
// approximate score, recompute them exactly, merge into the running list.
template <int K>
__global__ void __launch_bounds__(256)
rerank_kernel(const float* __restrict__ X, float xscale, const float* __restrict__ Y, int P2,
              int orient_offset, int n_orient, int nsplit, const float* __restrict__ cand_v,
              const int* __restrict__ cand_i, float* __restrict__ st_d, int* __restrict__ st_i) {
  const int img = blockIdx.x;
  __shared__ float s_v[K];
  __shared__ int s_i[K];
  __shared__ double s_red[8];
  if (threadIdx.x == 0) {
    float tv[K];
    int ti[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      tv[q] = FLT_MAX;
      ti[q] = -1;
    }
    const size_t base = (size_t)img * kMaxSplits * kCand;
    for (int s = 0; s < nsplit; ++s)
      for (int q = 0; q < kCand; ++q) {
        int j = cand_i[base + s * kCand + q];
        if (j >= 0) list_insert_ordered<K>(tv, ti, cand_v[base + s * kCand + q], j);
      }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      s_v[q] = tv[q];
      s_i[q] = ti[q];
    }
  }
  __syncthreads();
  const float* x = X + (size_t)img * P2;
  float exact[K];
  for (int q = 0; q < K; ++q) {
    int j = s_i[q];
    exact[q] = FLT_MAX;
    if (j < 0) continue;                       // uniform across the CTA
    const float* y = Y + (size_t)(j - orient_offset) * P2;
    float acc = 0.f;
    for (int p = threadIdx.x; p < P2; p += blockDim.x) {
      float d = fmaf(xscale, x[p], -y[p]);
      acc = fmaf(d, d, acc);
    }
    double v = (double)acc;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
      s_v[q] = (float)t;                      // reuse as exact distance
    }
    __syncthreads();
    exact[q] = s_v[q];
  }
  if (threadIdx.x == 0) {
    float tv[K];
    int ti[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      tv[q] = st_d[(size_t)img * K + q];
      ti[q] = st_i[(size_t)img * K + q];
    }
#pragma unroll
    for (int q = 0; q < K; ++q)
      if (s_i[q] >= 0) list_insert_ordered<K>(tv, ti, exact[q], s_i[q]);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      st_d[(size_t)img * K + q] = tv[q];
      st_i[(size_t)img * K + q] = ti[q];
    }
  }
}

__global__ void results_kernel(const float* __restrict__ st_d, const int* __restrict__ st_i, int n,
                               int K, int32_t* best_idx, float* best_d, float* second_d,
                               int32_t* topk_idx, float* topk_d) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (best_idx) best_idx[i] = st_i[(size_t)i * K];
  if (best_d) best_d[i] = st_d[(size_t)i * K];
  if (second_d) second_d[i] = K > 1 ? st_d[(size_t)i * K + 1] : FLT_MAX;
  for (int q = 0; q < K; ++q) {
    if (topk_idx) topk_idx[(size_t)i * K + q] = st_i[(size_t)i * K + q];
    if (topk_d) topk_d[(size_t)i * K + q] = st_d[(size_t)i * K + q];
  }
}

}  // namespace

int simt_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                cudaStream_t s) {
  int n_ot = (int)ceil_div(n_orient, BN);
  int tps = (int)ceil_div(n_ot, nsplit);
  dim3 grid((unsigned)ceil_div(m->n_img, BM), (unsigned)nsplit);
  size_t smem = sizeof(float) * (BK * BM + BK * BN + BM * (BN + 1));
  SPF_CUDA(cudaFuncSetAttribute(simt_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  SPF_TRY(launch("simt_match_kernel", s, [&] { simt_match_kernel<<<grid, 256, smem, s>>>(m->images, m->n_img, m->img_scale, slices, n_orient,
                                            orient_offset, m->P2, m->y2, tps, m->cand_v, m->cand_i); }));
  return SPF_OK;
}

int row_norms(const float* src, int rows, int P2, float scale, float* out, cudaStream_t s) {
  if (rows == 0) return SPF_OK;
  SPF_TRY(launch("row_norms_kernel", s, [&] { row_norms_kernel<<<(unsigned)ceil_div(rows, 8), 256, 0, s>>>(src, rows, P2, scale, out); }));
  return SPF_OK;
}

int state_reset(spf_matcher* m, cudaStream_t s) {
  int n = m->n_img * m->topk;
  if (n == 0) return SPF_OK;
  SPF_TRY(launch("state_reset_kernel", s, [&] { state_reset_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(m->st_d, m->st_i, n); }));
  return SPF_OK;
}

int rerank_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                  cudaStream_t s) {
  if (m->n_img == 0) return SPF_OK;
#define SPF_RR(K)                                                                               \
  case K:                                                                                       \
    return launch("rerank_kernel", s, [&] {                                                     \
      rerank_kernel<K><<<m->n_img, 256, 0, s>>>(m->images, m->img_scale, slices, m->P2,         \
                                                orient_offset, n_orient, nsplit, m->cand_v,     \
                                                m->cand_i, m->st_d, m->st_i);                   \
    });
  switch (m->topk) {
    SPF_RR(2) SPF_RR(3) SPF_RR(4) SPF_RR(5) SPF_RR(6) SPF_RR(7) SPF_RR(8)
    default: set_error("topk %d not in 2..8", m->topk); return SPF_ERR_ARG;
  }
#undef SPF_RR
}

int results_launch(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                   int32_t* topk_idx, float* topk_d, cudaStream_t s) {
  if (m->n_img == 0) return SPF_OK;
  SPF_TRY(launch("results_kernel", s, [&] { results_kernel<<<(unsigned)ceil_div(m->n_img, 256), 256, 0, s>>>(
      m->st_d, m->st_i, m->n_img, m->topk, best_idx, best_d, second_d, topk_idx, topk_d); }));
  return SPF_OK;
}

}  // namespace spf
