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
// out[r] = |scale * src_r|^2, one warp per row: four FP32 partial sums per
// lane, combined across the warp in FP64.
__global__ void row_norms_kernel(const float* __restrict__ src, int rows, int P2, float scale,
                                 const float* __restrict__ w, float* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const float* row = src + (size_t)warp * P2;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  const bool vec = !w && (P2 % 4) == 0 && (((uintptr_t)row) & 15) == 0;
  if (vec) {
    const float4* r4 = reinterpret_cast<const float4*>(row);
    for (int p = lane; p < P2 / 4; p += 32) {
      float4 v = __ldg(r4 + p);
      a0 = fmaf(v.x, v.x, a0);
      a1 = fmaf(v.y, v.y, a1);
      a2 = fmaf(v.z, v.z, a2);
      a3 = fmaf(v.w, v.w, a3);
    }
  } else {
    for (int p = lane; p < P2; p += 32) {
      float v = __ldg(row + p);
      if (w) v *= __ldg(w + p);
      a0 = fmaf(v, v, a0);
    }
  }
  double acc = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = (float)(acc * (double)scale * (double)scale);
}

__global__ void state_reset_kernel(float* __restrict__ d, int* __restrict__ idx, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    d[i] = FLT_MAX;
    idx[i] = -1;
  }
}

__global__ void sqrt_weights_kernel(const float* __restrict__ D, int n, float* __restrict__ w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = sqrtf(fmaxf(D[i], 0.f));
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
// CTA tile: 128 images x 128 orientations, 256 threads, each computing an 8x8
// block as four 4x4 quadrants (rows ty*4 and 64+ty*4, columns tx*4 and
// 64+tx*4, conflict-free float4 shared reads). k-tiles of 16 are double-
// buffered in shared memory; the next tile is prefetched through 8 registers
// a thread in two halves: its image rows are loaded at the start of a tile and
// stored half-way through, its model-image rows loaded then and stored at the
// end, so each load has half a tile of FMAs to arrive and one barrier serves
// 16 k. Grid: (image tiles, orientation splits); a CTA walks its range of
// orientation tiles and keeps a running top-8 per image row in shared memory.
constexpr int BM = 128, BN = 128, BK = 16;

// Thread t's share of a 128 x 16 k-tile: row r0 + t / 2, the 8 elements from
// k0 + (t % 2) * 8 (zero beyond rows or P2), scaled and (WGT) weighted.
template <bool VEC, bool WGT>
__device__ __forceinline__ void simt_load(const float* __restrict__ X, int rows, int P2, int r0, int k0,
                                          float scale, const float* __restrict__ w, float (&v)[8]) {
  const int t = threadIdx.x;
  const int row = r0 + (t >> 1), k = k0 + (t & 1) * 8;
  if (VEC) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (row < rows && k + 4 * h < P2) {
        float4 q = __ldg(reinterpret_cast<const float4*>(X + (size_t)row * P2 + k + 4 * h));
        v[4 * h] = scale * q.x; v[4 * h + 1] = scale * q.y; v[4 * h + 2] = scale * q.z; v[4 * h + 3] = scale * q.w;
      } else {
        v[4 * h] = v[4 * h + 1] = v[4 * h + 2] = v[4 * h + 3] = 0.f;
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < 8; ++e)
      v[e] = (row < rows && k + e < P2) ? scale * __ldg(X + (size_t)row * P2 + k + e) : 0.f;
  }
  if (WGT) {
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] *= (k + e < P2) ? __ldg(w + k + e) : 0.f;
  }
}

// v (from simt_load) into the k-major shared tile T[BK][128].
__device__ __forceinline__ void simt_store(float* T, const float (&v)[8]) {
  const int t = threadIdx.x;
  const int row = t >> 1, k = (t & 1) * 8;
#pragma unroll
  for (int e = 0; e < 8; ++e) T[(k + e) * BM + row] = v[e];
}

// 8 k steps of the 8 x 8 register tile from the k-major tiles A and B.
__device__ __forceinline__ void simt_fma8(const float* A, const float* B, int tx, int ty, float (&acc)[8][8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float4 a0 = *reinterpret_cast<const float4*>(A + k * BM + ty * 4);
    float4 a1 = *reinterpret_cast<const float4*>(A + k * BM + 64 + ty * 4);
    float4 b0 = *reinterpret_cast<const float4*>(B + k * BN + tx * 4);
    float4 b1 = *reinterpret_cast<const float4*>(B + k * BN + 64 + tx * 4);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
  }
}

template <bool VEC, bool WGT>
__global__ void __launch_bounds__(256, 2)
simt_match_kernel(const float* __restrict__ X, int n_img, float xscale, const float* __restrict__ Y,
                  int n_orient, int orient_offset, int P2, const float* __restrict__ y2,
                  int tiles_per_split, const float* __restrict__ wsq, float* __restrict__ cand_v,
                  int* __restrict__ cand_i) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* As = smem;                        // [2][BK][BM]
  float* Bs = As + 2 * BK * BM;            // [2][BK][BN]
  float* Sc = Bs + 2 * BK * BN;            // [BM][BN+1]
  float* Lv = Sc + BM * (BN + 1);          // [BM][kCand] running list
  int* Li = reinterpret_cast<int*>(Lv + BM * kCand);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * BM;
  const int split = blockIdx.y;
  const int n_ot = (n_orient + BN - 1) / BN;
  const int ot_begin = split * tiles_per_split;
  const int ot_end = min(n_ot, ot_begin + tiles_per_split);
  if (tid < BM)
    for (int q = 0; q < kCand; ++q) {
      Lv[tid * kCand + q] = FLT_MAX;
      Li[tid * kCand + q] = -1;
    }

  for (int ot = ot_begin; ot < ot_end; ++ot) {
    const int j0 = ot * BN;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    float rv[8];
    __syncthreads();
    simt_load<VEC, WGT>(X, n_img, P2, i0, 0, xscale, wsq, rv);
    simt_store(As, rv);
    simt_load<VEC, WGT>(Y, n_orient, P2, j0, 0, 1.f, wsq, rv);
    simt_store(Bs, rv);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < P2; k0 += BK) {
      const bool more = k0 + BK < P2;
      const float* A = As + buf * BK * BM;
      const float* B = Bs + buf * BK * BN;
      if (more) simt_load<VEC, WGT>(X, n_img, P2, i0, k0 + BK, xscale, wsq, rv);
      simt_fma8(A, B, tx, ty, acc);
      if (more) {
        // the other buffers were last read before the previous barrier
        simt_store(As + (buf ^ 1) * BK * BM, rv);
        simt_load<VEC, WGT>(Y, n_orient, P2, j0, k0 + BK, 1.f, wsq, rv);
      }
      simt_fma8(A + 8 * BM, B + 8 * BN, tx, ty, acc);
      if (more) {
        simt_store(Bs + (buf ^ 1) * BK * BN, rv);
        __syncthreads();
        buf ^= 1;
      }
    }
    // scores |y|^2 - 2 x.y into the shared tile
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int r = (a < 4) ? ty * 4 + a : 64 + ty * 4 + (a - 4);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int c = (b < 4) ? tx * 4 + b : 64 + tx * 4 + (b - 4);
        const int gj = j0 + c;
        Sc[r * (BN + 1) + c] = gj < n_orient ? fmaf(-2.f, acc[a][b], __ldg(y2 + gj)) : FLT_MAX;
      }
    }
    __syncthreads();
    if (tid < BM) {
      float tv[kCand];
      int ti[kCand];
#pragma unroll
      for (int q = 0; q < kCand; ++q) {
        tv[q] = Lv[tid * kCand + q];
        ti[q] = Li[tid * kCand + q];
      }
      for (int c = 0; c < BN && j0 + c < n_orient; ++c)
        list_insert<kCand>(tv, ti, Sc[tid * (BN + 1) + c], orient_offset + j0 + c);
#pragma unroll
      for (int q = 0; q < kCand; ++q) {
        Lv[tid * kCand + q] = tv[q];
        Li[tid * kCand + q] = ti[q];
      }
    }
    __syncthreads();
  }
  if (tid < BM && i0 + tid < n_img) {
    size_t o = ((size_t)(i0 + tid) * kMaxSplits + split) * kCand;
#pragma unroll
    for (int q = 0; q < kCand; ++q) {
      cand_v[o + q] = Lv[tid * kCand + q];
      cand_i[o + q] = Li[tid * kCand + q];
    }
  }
}

// ------------------------------------------------------------ rerank -----
// Re-rank order: images bucketed by the orientation of their best
// approximate candidate (counting sort; bucket n_orient: no candidate).
// Candidates of image i: `ncand` entries from i * stride; key = (best index -
// key_off) / key_div, bucket nkeys when there is none.
__global__ void rr_key_kernel(const float* __restrict__ cand_v, const int* __restrict__ cand_i, int n_img,
                              int stride, int ncand, int key_off, int key_div, int n_orient,
                              int* __restrict__ key, int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_img) return;
  const size_t base = (size_t)i * stride;
  float bv = FLT_MAX;
  int bj = -1;
  for (int q = 0; q < ncand; ++q) {
    const int j = __ldg(cand_i + base + q);
    const float v = __ldg(cand_v + base + q);
    if (j >= 0 && (v < bv || (v == bv && j < bj))) {
      bv = v;
      bj = j;
    }
  }
  int k = bj >= 0 ? (bj - key_off) / key_div : n_orient;
  if (k < 0 || k > n_orient) k = n_orient;
  key[i] = k;
  atomicAdd(count + k, 1);
}

// Exclusive scan of n counts in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) rr_scan_kernel(int* __restrict__ c, int n) {
  __shared__ int warp_sums[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < n; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n ? c[i] : 0;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
      int y = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, y, o);
        if (lane >= o) y += t;
      }
      warp_sums[lane] = y;
    }
    __syncthreads();
    const int excl = carry + (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    if (i < n) c[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void rr_scatter_kernel(const int* __restrict__ key, int n_img, int* __restrict__ start,
                                  int* __restrict__ order) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_img) return;
  order[atomicAdd(start + key[i], 1)] = i;
}

// One CTA per image: merge nsplit candidate lists, take the best topk by
// approximate score, recompute them exactly, merge into the running list.
// Rows of model images: one block Y of rows [orient_offset, ...) or, with
// nch > 0, the blocks ch_ptr[c] holding rows [ch_off[c], ch_off[c + 1]).
struct RowTable {
  const float* Y;
  int orient_offset;
  const int* ch_off;
  const float* const* ch_ptr;
  int nch;
  __device__ __forceinline__ const float* row(int j, int P2) const {
    if (nch == 0) return Y + (size_t)(j - orient_offset) * P2;
    int lo = 0, hi = nch - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(ch_off + mid) <= j) lo = mid;
      else hi = mid - 1;
    }
    return ch_ptr[lo] + (size_t)(j - __ldg(ch_off + lo)) * P2;
  }
};

template <int K, class XT>
__global__ void __launch_bounds__(256)
rerank_kernel(const XT* __restrict__ X, float xscale, RowTable rows, int P2, int stride, int ncand,
              const float* __restrict__ cand_v, const int* __restrict__ cand_i, const float* __restrict__ wsq,
              float* __restrict__ st_d, int* __restrict__ st_i, const int* __restrict__ order) {
  const int img = order ? __ldg(order + blockIdx.x) : blockIdx.x;
  __shared__ float s_v[K];
  __shared__ int s_i[K];
  __shared__ const float* s_row[K];
  if (threadIdx.x == 0) {
    float tv[K];
    int ti[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      tv[q] = FLT_MAX;
      ti[q] = -1;
    }
    const size_t base = (size_t)img * stride;
    for (int q = 0; q < ncand; ++q) {
      int j = cand_i[base + q];
      if (j >= 0) list_insert_ordered<K>(tv, ti, cand_v[base + q], j);
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      s_v[q] = tv[q];
      s_i[q] = ti[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < K) s_row[threadIdx.x] = s_i[threadIdx.x] >= 0 ? rows.row(s_i[threadIdx.x], P2) : nullptr;
  __syncthreads();
  // exact FP32 distances of all candidates in one sweep over the pixels
  const XT* x = X + (size_t)img * P2;
  // empty candidate slots read the first filled slot's row (their sums are
  // never used); an image without candidates skips the sweep
  const float* fb = nullptr;
#pragma unroll
  for (int q = K - 1; q >= 0; --q)
    if (s_row[q]) fb = s_row[q];
  const float* y[K];
#pragma unroll
  for (int q = 0; q < K; ++q) y[q] = s_row[q] ? s_row[q] : fb;
  float acc[K];
#pragma unroll
  for (int q = 0; q < K; ++q) acc[q] = 0.f;
  bool vec = !wsq && (P2 % 4) == 0 && (((uintptr_t)x) & (4 * sizeof(XT) - 1)) == 0;
#pragma unroll
  for (int q = 0; q < K; ++q) vec = vec && (((uintptr_t)y[q]) & 15) == 0;
  if (!fb) {
    // no candidate: nothing to measure
  } else if (vec) {
#pragma unroll 2
    for (int p = threadIdx.x; p < P2 / 4; p += blockDim.x) {
      float4 xv = img_elem4(x, p);
      xv.x *= xscale; xv.y *= xscale; xv.z *= xscale; xv.w *= xscale;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        float4 yv = __ldg(reinterpret_cast<const float4*>(y[q]) + p);
        float d0 = xv.x - yv.x, d1 = xv.y - yv.y, d2 = xv.z - yv.z, d3 = xv.w - yv.w;
        acc[q] = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, acc[q]))));
      }
    }
  } else {
    for (int p = threadIdx.x; p < P2; p += blockDim.x) {
      float xv = xscale * img_elem(x, p);
      const float wp = wsq ? __ldg(wsq + p) : 1.f;
#pragma unroll
      for (int q = 0; q < K; ++q) {
        float d = (xv - __ldg(y[q] + p)) * wp;
        acc[q] = fmaf(d, d, acc[q]);
      }
    }
  }
  __shared__ double s_red[K][8];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double v = (double)acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  float exact[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[q][w];
    exact[q] = (float)t;
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

// Entry c of the deferred re-rank's chunk table, written in stream order.
__global__ void chunk_table_kernel(int* __restrict__ off, const float** __restrict__ ptr, int c, int lo, int hi,
                                   const float* rows) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    off[c] = lo;
    off[c + 1] = hi;
    ptr[c] = rows;
  }
}

// Running approximate top-kCand per image across orientation chunks (deferred
// re-rank): the nsplit * kCand candidates of this launch merged into ap.
__global__ void cand_merge_kernel(const float* __restrict__ cand_v, const int* __restrict__ cand_i, int n_img,
                                  int nsplit, float* __restrict__ ap_v, int* __restrict__ ap_i) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_img) return;
  float tv[kCand];
  int ti[kCand];
#pragma unroll
  for (int q = 0; q < kCand; ++q) {
    tv[q] = ap_v[(size_t)i * kCand + q];
    ti[q] = ap_i[(size_t)i * kCand + q];
  }
  const size_t base = (size_t)i * kMaxSplits * kCand;
  for (int q = 0; q < nsplit * kCand; ++q) {
    const int j = __ldg(cand_i + base + q);
    if (j >= 0) list_insert_ordered<kCand>(tv, ti, __ldg(cand_v + base + q), j);
  }
#pragma unroll
  for (int q = 0; q < kCand; ++q) {
    ap_v[(size_t)i * kCand + q] = tv[q];
    ap_i[(size_t)i * kCand + q] = ti[q];
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

// Orientation splits of a CUDA-core launch: the split count whose makespan,
// (waves of CTAs over two per SM) x (orientation tiles per split), is
// smallest; counts that would leave a split empty are skipped. The merged top
// list does not depend on the count (candidates merge in (score, index)
// order).
int simt_splits(int n_img, int n_orient, int n_sms) {
  const int64_t img_tiles = ceil_div(n_img, BM), or_tiles = ceil_div(n_orient, BN);
  const int64_t slots = 2 * (int64_t)std::max(n_sms, 1);
  int best = 1;
  int64_t best_span = INT64_MAX;
  for (int sp = 1; sp <= std::min<int64_t>(or_tiles, kMaxSplits); ++sp) {
    const int64_t tps = ceil_div(or_tiles, sp);
    if (ceil_div(or_tiles, tps) != sp) continue;
    const int64_t span = ceil_div(img_tiles * sp, slots) * tps;
    if (span < best_span) {
      best_span = span;
      best = sp;
    }
  }
  return best;
}

int simt_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                cudaStream_t s) {
  int n_ot = (int)ceil_div(n_orient, BN);
  int tps = (int)ceil_div(n_ot, nsplit);
  dim3 grid((unsigned)ceil_div(m->n_img, BM), (unsigned)nsplit);
  size_t smem = sizeof(float) * (2 * BK * BM + 2 * BK * BN + BM * (BN + 1) + 2 * BM * kCand);
  const bool vec = (m->P2 % 4) == 0 && ((uintptr_t)m->images % 16) == 0 && ((uintptr_t)slices % 16) == 0;
  auto go = [&](auto kernel) -> int {
    SPF_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return launch("simt_match_kernel", s, [&] {
      kernel<<<grid, 256, smem, s>>>(m->images, m->n_img, m->img_scale, slices, n_orient, orient_offset, m->P2,
                                     m->y2, tps, m->wsq, m->cand_v, m->cand_i);
    });
  };
  if (m->wsq) return vec ? go(simt_match_kernel<true, true>) : go(simt_match_kernel<false, true>);
  return vec ? go(simt_match_kernel<true, false>) : go(simt_match_kernel<false, false>);
}

int row_norms_w(const float* src, int rows, int P2, float scale, const float* w, float* out,
                cudaStream_t s) {
  if (rows == 0) return SPF_OK;
  SPF_TRY(launch("row_norms_kernel", s, [&] {
    row_norms_kernel<<<(unsigned)ceil_div(rows, 8), 256, 0, s>>>(src, rows, P2, scale, w, out);
  }));
  return SPF_OK;
}

int row_norms(const float* src, int rows, int P2, float scale, float* out, cudaStream_t s) {
  if (rows == 0) return SPF_OK;
  SPF_TRY(row_norms_w(src, rows, P2, scale, nullptr, out, s));
  return SPF_OK;
}

int state_reset(spf_matcher* m, cudaStream_t s) {
  m->n_chunks = 0;
  m->pending = false;
  int n = m->n_img * m->topk;
  if (n == 0) return SPF_OK;
  SPF_TRY(launch("state_reset_kernel", s, [&] { state_reset_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(m->st_d, m->st_i, n); }));
  if (m->defer) {
    const int na = m->n_img * kCand;
    SPF_TRY(launch("state_reset_kernel", s, [&] {
      state_reset_kernel<<<(unsigned)ceil_div(na, 256), 256, 0, s>>>(m->ap_v, m->ap_i, na);
    }));
  }
  return SPF_OK;
}

// Exact FP32 re-rank of candidate lists (stride and count per image) with
// model-image rows from `rows`; images visited grouped by their best
// candidate (bucket = (index - key_off) / key_div, at most max_orient + 1).
static int rerank_core(spf_matcher* m, const RowTable& rows, const float* cv, const int* ci, int stride,
                       int ncand, int key_off, int key_div, int nkeys, cudaStream_t s) {
  if (m->n_img == 0) return SPF_OK;
  const int* order = nullptr;
  if (m->rr_order && nkeys <= m->max_orient) {
    const unsigned g = (unsigned)ceil_div(m->n_img, 256);
    SPF_CUDA(cudaMemsetAsync(m->rr_start, 0, sizeof(int) * ((size_t)nkeys + 1), s));
    SPF_TRY(launch("rr_key_kernel", s, [&] {
      rr_key_kernel<<<g, 256, 0, s>>>(cv, ci, m->n_img, stride, ncand, key_off, key_div, nkeys, m->rr_key,
                                      m->rr_start);
    }));
    SPF_TRY(launch("rr_scan_kernel", s, [&] { rr_scan_kernel<<<1, 1024, 0, s>>>(m->rr_start, nkeys + 1); }));
    SPF_TRY(launch("rr_scatter_kernel", s, [&] {
      rr_scatter_kernel<<<g, 256, 0, s>>>(m->rr_key, m->n_img, m->rr_start, m->rr_order);
    }));
    order = m->rr_order;
  }
#define SPF_RR(K)                                                                                   \
  case K:                                                                                           \
    return launch("rerank_kernel", s, [&] {                                                         \
      if (m->images16)                                                                              \
        rerank_kernel<K, uint16_t><<<m->n_img, 256, 0, s>>>(m->images16, m->img_scale, rows, m->P2, \
                                                            stride, ncand, cv, ci, m->wsq, m->st_d,  \
                                                            m->st_i, order);                        \
      else                                                                                          \
        rerank_kernel<K, float><<<m->n_img, 256, 0, s>>>(m->images, m->img_scale, rows, m->P2,      \
                                                         stride, ncand, cv, ci, m->wsq, m->st_d,     \
                                                         m->st_i, order);                           \
    });
  switch (m->topk) {
    SPF_RR(2) SPF_RR(3) SPF_RR(4) SPF_RR(5) SPF_RR(6) SPF_RR(7) SPF_RR(8)
    default: set_error("topk %d not in 2..8", m->topk); return SPF_ERR_ARG;
  }
#undef SPF_RR
}

int rerank_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                  cudaStream_t s) {
  if (m->defer) {
    // keep this launch's best candidates and the rows they point into; the
    // exact re-rank runs once, when the results are read
    SPF_CHECK_ARG(m->n_chunks < kMaxChunks, "deferred re-rank: more than %d chunks", kMaxChunks);
    SPF_CHECK_ARG(m->n_chunks == 0 || orient_offset >= m->ch_off_h[m->n_chunks],
                  "deferred re-rank: chunks must come in increasing, non-overlapping orientation ranges");
    const int c = m->n_chunks;
    m->ch_off_h[c] = orient_offset;
    m->ch_ptr_h[c] = slices;
    m->ch_off_h[c + 1] = orient_offset + n_orient;
    ++m->n_chunks;
    m->pending = true;
    SPF_TRY(launch("chunk_table_kernel", s, [&] {
      chunk_table_kernel<<<1, 32, 0, s>>>(m->ch_off_d, m->ch_ptr_d, c, orient_offset, orient_offset + n_orient,
                                          slices);
    }));
    return launch("cand_merge_kernel", s, [&] {
      cand_merge_kernel<<<(unsigned)ceil_div(m->n_img, 256), 256, 0, s>>>(m->cand_v, m->cand_i, m->n_img, nsplit,
                                                                        m->ap_v, m->ap_i);
    });
  }
  RowTable rows{slices, orient_offset, nullptr, nullptr, 0};
  return rerank_core(m, rows, m->cand_v, m->cand_i, kMaxSplits * kCand, nsplit * kCand, orient_offset, 1,
                     n_orient, s);
}

int rerank_flush(spf_matcher* m, cudaStream_t s) {
  if (!m->defer || !m->pending) return SPF_OK;
  m->pending = false;
  const int n = m->n_chunks;
  const int lo = m->ch_off_h[0], total = m->ch_off_h[n] - lo;
  const int div = (int)std::max<int64_t>(1, ceil_div(total, std::max(1, m->max_orient)));
  RowTable rows{nullptr, 0, m->ch_off_d, m->ch_ptr_d, n};
  return rerank_core(m, rows, m->ap_v, m->ap_i, kCand, kCand, lo, div, (int)ceil_div(total, div), s);
}

int results_launch(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                   int32_t* topk_idx, float* topk_d, cudaStream_t s) {
  if (m->n_img == 0) return SPF_OK;
  SPF_TRY(rerank_flush(m, s));
  SPF_TRY(launch("results_kernel", s, [&] { results_kernel<<<(unsigned)ceil_div(m->n_img, 256), 256, 0, s>>>(
      m->st_d, m->st_i, m->n_img, m->topk, best_idx, best_d, second_d, topk_idx, topk_d); }));
  return SPF_OK;
}

}  // namespace spf

namespace spf {
int set_mask_weights(spf_matcher* m, const float* D, cudaStream_t s) {
  if (!D) {
    m->wsq = nullptr;
    return SPF_OK;
  }
  SPF_TRY(launch("sqrt_weights_kernel", s, [&] {
    sqrt_weights_kernel<<<(unsigned)ceil_div(m->P2, 256), 256, 0, s>>>(D, m->P2, m->wbuf);
  }));
  m->wsq = m->wbuf;
  return SPF_OK;
}
}  // namespace spf

namespace spf {
namespace {

// out[i] = counts[i] (16-bit photon counts to FP32), 8 per thread: one 16-byte
// load and two 16-byte stores (both buffers 16-byte aligned), then the tail.
__global__ void counts_to_f32_vec_kernel(const uint16_t* __restrict__ c, int64_t n, float* __restrict__ out) {
  const int64_t n8 = n / 8;
  const uint4* c8 = reinterpret_cast<const uint4*>(c);
  float4* o4 = reinterpret_cast<float4*>(out);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n8; i += stride) {
    const uint4 v = __ldg(c8 + i);
    o4[2 * i] = make_float4((float)(v.x & 0xffffu), (float)(v.x >> 16), (float)(v.y & 0xffffu), (float)(v.y >> 16));
    o4[2 * i + 1] =
        make_float4((float)(v.z & 0xffffu), (float)(v.z >> 16), (float)(v.w & 0xffffu), (float)(v.w >> 16));
  }
  for (int64_t i = n8 * 8 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (float)__ldg(c + i);
}

__global__ void counts_to_f32_kernel(const uint16_t* __restrict__ c, int64_t n, float* __restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)__ldg(c + i);
}

}  // namespace

int counts_to_f32(const uint16_t* counts, int64_t n, float* out, cudaStream_t s) {
  if (n == 0) return SPF_OK;
  const bool vec = (((uintptr_t)counts | (uintptr_t)out) & 15) == 0;
  const int64_t work = vec ? ceil_div(n, 8) : n;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(work, 256), (int64_t)device_sms() * 16);
  if (vec)
    return launch("counts_to_f32_kernel", s, [&] { counts_to_f32_vec_kernel<<<grid, 256, 0, s>>>(counts, n, out); }, 6.0 * n);
  return launch("counts_to_f32_kernel", s, [&] { counts_to_f32_kernel<<<grid, 256, 0, s>>>(counts, n, out); }, 6.0 * n);
}
}  // namespace spf
