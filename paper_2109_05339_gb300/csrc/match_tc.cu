// Tensor-core orientation matching (Sec. II-B) on sm_103a: quantisation of
// images and model images to BF16 / FP8 e4m3, and the fused cross-term +
// top-8 kernel.
//
// The cross term X Y^T (images x model images, K = pixels) is the dense
// contraction of the matching step, so it runs on the 5th-generation tensor
// cores: tcgen05.mma with both operands K-major in shared memory (128-byte
// swizzle, staged by TMA through a 3-deep mbarrier ring) and FP32
// accumulators in tensor memory. A CTA owns a 256-image x 256-orientation
// tile as two 128 x 256 accumulators, i.e. all 512 TMEM columns. Warp roles:
// warp 0 issues TMA loads, warp 1 issues MMAs (one elected lane each), warp 2
// owns the TMEM allocation, warps 4..11 are the epilogue: each thread reads
// one image row of an accumulator with tcgen05.ld, forms |y|^2 - 2 x.y (times
// the FP8 row scales) and keeps a running top-8 in registers while the CTA
// walks its contiguous range of tiles, so no distance ever reaches HBM.
// Every mbarrier wait is bounded by wall-clock time; on expiry the CTA sets
// an error bit, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cfloat>
#include <vector>

#include "match.h"
#include "tc.h"

namespace spf {

namespace {

__device__ __forceinline__ float block_sum_f64(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return (float)t;
}

// BF16 copy of scale * src rows (padding columns stay zero from creation)
// and the squared norms of the quantised rows, one CTA per row. With the
// norms of the quantised rows the approximate distance is the exact distance
// between the quantised image and model image (up to the FP32 accumulation of
// the cross term): an image equal to a model image scores 0 against it, and
// the rounding of the two rows enters only through their difference.
template <class XT>
__global__ void __launch_bounds__(256) quantize_bf16_kernel(const XT* __restrict__ src, int P2,
                                                            int Kpad, float scale,
                                                            const float* __restrict__ w,
                                                            __nv_bfloat16* __restrict__ dst,
                                                            float* __restrict__ norms) {
  const int r = blockIdx.x;
  const XT* row = src + (size_t)r * P2;
  __nv_bfloat16* out = dst + (size_t)r * Kpad;
  float a0 = 0.f, a1 = 0.f;
  if (!w && (P2 % 4) == 0 && (((uintptr_t)row) & (4 * sizeof(XT) - 1)) == 0) {
    for (int p = threadIdx.x; p < P2 / 4; p += blockDim.x) {
      float4 v = img_elem4(row, p);
      v.x *= scale; v.y *= scale; v.z *= scale; v.w *= scale;
      __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
      const float2 ql = __bfloat1622float2(lo), qh = __bfloat1622float2(hi);
      a0 = fmaf(ql.x, ql.x, fmaf(ql.y, ql.y, a0));
      a1 = fmaf(qh.x, qh.x, fmaf(qh.y, qh.y, a1));
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo);
      pk.y = *reinterpret_cast<uint32_t*>(&hi);
      reinterpret_cast<uint2*>(out)[p] = pk;
    }
  } else {
    for (int p = threadIdx.x; p < P2; p += blockDim.x) {
      float v = scale * img_elem(row, p);
      if (w) v *= __ldg(w + p);
      const __nv_bfloat16 q = __float2bfloat16_rn(v);
      const float qf = __bfloat162float(q);
      a0 = fmaf(qf, qf, a0);
      out[p] = q;
    }
  }
  __shared__ double sh[8];
  float n = block_sum_f64((double)a0 + (double)a1, sh);
  if (threadIdx.x == 0) norms[r] = n;
}

// One e4m3 code (round to nearest, saturating), its square added to sq
// (exact: 8 significant bits).
__device__ __forceinline__ uint32_t fp8_code(float v, float& sq) {
  __nv_fp8_e4m3 q;
  q.__x = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
  const float f = static_cast<float>(q);
  sq = fmaf(f, f, sq);
  return q.__x;
}

// FP8 e4m3 copy with a per-row scale a_r = max_p |scale * src_rp| / 448
// (1 for an all-zero row): dst = e4m3(scale * src / a_r); also the squared
// norms of the quantised rows, a_r^2 sum_p dst_p^2 (the distance between
// quantised rows, as for BF16). One CTA per row, two passes over it: the
// maximum, then the codes. Long rows take 512 threads, two CTAs per SM, so
// that about 300 rows (45 MB of FP32 rows of 36,864 pixels) are in flight and
// the second pass reads the row from L2; where the row allows, four elements
// a step (16-byte FP32 or 8-byte 16-bit loads, one 4-byte store of codes),
// four steps unrolled so that each thread has four loads in flight.
template <class XT>
__global__ void __launch_bounds__(512, 2) quantize_fp8_kernel(const XT* __restrict__ src, int P2,
                                                            int Kpad, float scale,
                                                            const float* __restrict__ w,
                                                            __nv_fp8_e4m3* __restrict__ dst,
                                                            float* __restrict__ row_scale,
                                                            float* __restrict__ norms) {
  const int r = blockIdx.x;
  const XT* row = src + (size_t)r * P2;
  __nv_fp8_e4m3* out = dst + (size_t)r * Kpad;
  const bool vec = (P2 % 4) == 0 && (((uintptr_t)row) & (4 * sizeof(XT) - 1)) == 0;
  const int n4 = vec ? P2 / 4 : 0;
  const float4 one = make_float4(1.f, 1.f, 1.f, 1.f);
  float mx = 0.f;
#pragma unroll 4
  for (int p = threadIdx.x; p < n4; p += blockDim.x) {
    const float4 v = img_elem4(row, p);
    const float4 c = w ? __ldg(reinterpret_cast<const float4*>(w) + p) : one;
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(scale * v.x * c.x), fabsf(scale * v.y * c.y)),
                         fmaxf(fabsf(scale * v.z * c.z), fabsf(scale * v.w * c.w))));
  }
  for (int k = 4 * n4 + threadIdx.x; k < P2; k += blockDim.x)
    mx = fmaxf(mx, fabsf(scale * img_elem(row, k) * (w ? __ldg(w + k) : 1.f)));
  __shared__ float sm[32];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, sm[i]);
    sm[0] = m > 0.f ? m / 448.f : 1.f;
    row_scale[r] = sm[0];
  }
  __syncthreads();
  const float a = sm[0], inv = 1.f / a;
  float a0 = 0.f;
#pragma unroll 4
  for (int p = threadIdx.x; p < n4; p += blockDim.x) {
    const float4 v = img_elem4(row, p);
    const float4 c = w ? __ldg(reinterpret_cast<const float4*>(w) + p) : one;
    const uint32_t b0 = fp8_code(scale * v.x * c.x * inv, a0), b1 = fp8_code(scale * v.y * c.y * inv, a0);
    const uint32_t b2 = fp8_code(scale * v.z * c.z * inv, a0), b3 = fp8_code(scale * v.w * c.w * inv, a0);
    reinterpret_cast<uint32_t*>(out)[p] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
  }
  for (int k = 4 * n4 + threadIdx.x; k < P2; k += blockDim.x) {
    __nv_fp8_e4m3 q;
    q.__x = (__nv_fp8_storage_t)fp8_code(scale * img_elem(row, k) * (w ? __ldg(w + k) : 1.f) * inv, a0);
    out[k] = q;
  }
  const float n = block_sum_f64((double)a0, sh);
  if (threadIdx.x == 0) norms[r] = n * a * a;
}

}  // namespace

int tc_kpad(int P2, int precision) {
  int blk = precision == SPF_BF16 ? 64 : 128;   // one 128-byte swizzle row
  return (int)ceil_div(P2, blk) * blk;
}

template <class XT>
int quantize_rows_t(spf_matcher* m, const XT* src, int rows, float scale, void* dst, float* scales,
                    float* norms, cudaStream_t s) {
  if (rows == 0) return SPF_OK;
  if (m->precision == SPF_BF16) {
    return launch("quantize_bf16_kernel", s, [&] {
      quantize_bf16_kernel<XT><<<rows, 256, 0, s>>>(src, m->P2, m->Kpad, scale, m->wsq,
                                                    static_cast<__nv_bfloat16*>(dst), norms);
    }, (double)rows * m->P2 * (sizeof(XT) + 2.0));
  }
  const int threads = m->P2 >= 8192 ? 512 : 256;
  return launch("quantize_fp8_kernel", s, [&] {
    quantize_fp8_kernel<XT><<<rows, threads, 0, s>>>(src, m->P2, m->Kpad, scale, m->wsq,
                                                     static_cast<__nv_fp8_e4m3*>(dst), scales, norms);
  }, (double)rows * m->P2 * (sizeof(XT) + 1.0));
}

int quantize_rows(spf_matcher* m, const float* src, int rows, float scale, void* dst, float* scales,
                  float* norms, cudaStream_t s) {
  return quantize_rows_t(m, src, rows, scale, dst, scales, norms, s);
}

int quantize_rows_u16(spf_matcher* m, const uint16_t* src, int rows, float scale, void* dst, float* scales,
                      float* norms, cudaStream_t s) {
  return quantize_rows_t(m, src, rows, scale, dst, scales, norms, s);
}

int match_tc_supported(int device) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  return major == 10 && minor == 3;
}

namespace {

constexpr int kTcTile = 256;                 // images and orientations per tile
constexpr int kTcStages = 3;
constexpr uint32_t kTcHalf = 32 * 1024;      // one operand tile per stage (256 rows x 128 B)
constexpr uint32_t kTcStage = 2 * kTcHalf;
constexpr int kTcThreads = 384;

// Which tiles each CTA computes. mode 0: contiguous ranges of the row-major
// (image tile, orientation tile) order -- consecutive CTAs share image
// tiles when there are few of them. mode 1: a gi x go grid of CTAs; CTA
// (a, b) takes the image tiles of range a and the orientation tiles of range
// b, image tile by image tile. The go CTAs of a row then work on the same
// image tile and the gi CTAs of a column on the same orientation tile at the
// same time, so each operand tile is read from HBM about once per row or
// column instead of once per tile when the image tiles outnumber the CTAs.
struct TcParams {
  int n_img, n_orient, orient_offset, nkb;
  int n_it, n_ot, total, grid;
  int mode, gi, go;
  const float* y2;
  const float* xs;   // FP8 image scales (nullptr for BF16)
  const float* ys;   // FP8 slice scales
  float* cand_v;
  int* cand_i;
  int* err;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Instruction descriptor: FP32 accumulate, A/B format code, K-major A and B,
// N = 256, M = 128.
__host__ __device__ constexpr uint32_t idesc(uint32_t ab_format) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
}

template <bool FP8>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  if constexpr (FP8) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc(0)), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc(1)), "r"(acc));
  }
}

template <int K>
__device__ __forceinline__ void tc_insert(float* tv, int* ti, float s, int j) {
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

__host__ __device__ inline int work_start(int c, int total, int grid) {
  return (int)((long long)c * total / grid);
}

// The tiles of one CTA, in the order it computes them (image tile major).
struct TcWork {
  int mode, n_ot;
  int q0, q1;          // mode 0: [q0, q1) of the row-major tile order
  int i0, o0, ni, no;  // mode 1: image tiles [i0, i0 + ni) x orientation tiles [o0, o0 + no)
  __device__ __forceinline__ int count() const { return mode == 0 ? q1 - q0 : ni * no; }
  __device__ __forceinline__ void tile(int t, int& it, int& ot) const {
    if (mode == 0) {
      const int q = q0 + t;
      it = q / n_ot;
      ot = q - it * n_ot;
    } else {
      const int a = t / no;
      it = i0 + a;
      ot = o0 + (t - a * no);
    }
  }
};

__device__ __forceinline__ TcWork tc_work(const TcParams& p, int c) {
  TcWork w;
  w.mode = p.mode;
  w.n_ot = p.n_ot;
  if (p.mode == 0) {
    w.q0 = work_start(c, p.total, p.grid);
    w.q1 = work_start(c + 1, p.total, p.grid);
    w.i0 = w.o0 = w.ni = w.no = 0;
  } else {
    const int a = c / p.go, b = c - a * p.go;
    w.i0 = work_start(a, p.n_it, p.gi);
    w.ni = work_start(a + 1, p.n_it, p.gi) - w.i0;
    w.o0 = work_start(b, p.n_ot, p.go);
    w.no = work_start(b + 1, p.n_ot, p.go) - w.o0;
    w.q0 = w.q1 = 0;
  }
  return w;
}

// First CTA whose contiguous work range contains item q.
__host__ __device__ inline int owner_cta(int q, int total, int grid) {
  int c = (int)(((long long)q * grid) / total);
  while (c + 1 < grid && work_start(c + 1, total, grid) <= q) ++c;
  while (c > 0 && work_start(c, total, grid) > q) --c;
  return c;
}

template <bool FP8>
__global__ void __launch_bounds__(kTcThreads, 1)
tc_match_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kTcStages * kTcStage);
  uint64_t* empty = full + kTcStages;
  uint64_t* tfull = empty + kTcStages;
  uint64_t* tempty = tfull + 1;
  uint64_t* done = tempty + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x;
  const TcWork work = tc_work(p, c);
  const int n_tiles = work.count();

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 8);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tslot)), "r"(512) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ---------------------------------------------------------- producer --
    if (lane == 0) {
      uint32_t last_phase[kTcStages];
      bool used[kTcStages];
      for (int s = 0; s < kTcStages; ++s) used[s] = false;
      uint32_t it = 0;
      bool ok = true;
      for (int q = 0; q < n_tiles && ok; ++q) {
        int ti_, to_;
        work.tile(q, ti_, to_);
        for (int kb = 0; kb < p.nkb; ++kb, ++it) {
          const int s = it % kTcStages;
          const uint32_t ph = (it / kTcStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, p.err)) { ok = false; break; }
          uint8_t* a = smem + s * kTcStage;
          mbar_arrive_expect_tx(&full[s], kTcStage);
          const int kx = kb * (FP8 ? 128 : 64);
          tma_load_2d(a, &tmA, kx, ti_ * kTcTile, &full[s]);
          tma_load_2d(a + kTcHalf, &tmB, kx, to_ * kTcTile, &full[s]);
          last_phase[s] = ph;
          used[s] = true;
        }
      }
      // never leave with copies in flight
      for (int s = 0; s < kTcStages; ++s)
        if (used[s]) mbar_wait(&full[s], last_phase[s], abort_flag, p.err, false);
    }
  } else if (warp == 1) {
    // --------------------------------------------------------- MMA issue --
    if (lane == 0) {
      uint32_t it = 0, t = 0;
      bool ok = true;
      for (int q = 0; q < n_tiles && ok; ++q, ++t) {
        if (!mbar_wait(tempty, (t & 1u) ^ 1u, abort_flag, p.err)) break;
        tc_fence_after();
        for (int kb = 0; kb < p.nkb; ++kb, ++it) {
          const int s = it % kTcStages;
          const uint32_t ph = (it / kTcStages) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag, p.err)) { ok = false; break; }
          tc_fence_after();
          const uint32_t a = smem_u32(smem + s * kTcStage);
          const uint32_t b = a + kTcHalf;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t bd = sdesc(b + kk * 32);
#pragma unroll
            for (int g = 0; g < 2; ++g)
              mma<FP8>(tmem + g * 256, sdesc(a + g * (kTcHalf / 2) + kk * 32), bd,
                       (kb | kk) != 0 ? 1u : 0u);
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(tfull);
      }
      // all issued MMAs complete before the CTA frees TMEM
      mma_commit(done);
      mbar_wait(done, 0, abort_flag, p.err, false);
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------- epilogue --
    const int g = (warp - 4) >> 2;          // accumulator: image rows 0..127 or 128..255
    const int quarter = warp & 3;           // TMEM lanes 32*quarter .. +31
    const int row = g * 128 + quarter * 32 + lane;
    float tv[kCand];
    int tix[kCand];
    int cur_it = -1;
    uint32_t t = 0;
    auto flush = [&](int it_) {
      const int i = it_ * kTcTile + row;
      if (i < p.n_img) {
        const int slot = p.mode == 0 ? c - owner_cta(it_ * p.n_ot, p.total, p.grid) : c % p.go;
        const size_t o = ((size_t)i * kMaxSplits + slot) * kCand;
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
          p.cand_v[o + k] = tv[k];
          p.cand_i[o + k] = tix[k];
        }
      }
    };
    for (int q = 0; q < n_tiles; ++q, ++t) {
      int it_, to_;
      work.tile(q, it_, to_);
      if (it_ != cur_it) {
        if (cur_it >= 0) flush(cur_it);
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
          tv[k] = FLT_MAX;
          tix[k] = -1;
        }
        cur_it = it_;
      }
      if (!mbar_wait(tfull, t & 1u, abort_flag, p.err)) break;
      tc_fence_after();
      const int i = it_ * kTcTile + row;
      const float xs = FP8 ? (i < p.n_img ? -2.f * p.xs[i] : 0.f) : -2.f;
      const int j0 = to_ * kTcTile;
#pragma unroll 1
      for (int ch = 0; ch < 8; ++ch) {
        float acc[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * 256 + ch * 32), acc);
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
          const int j = j0 + ch * 32 + cc;
          if (j < p.n_orient) {
            const float f = FP8 ? xs * __ldg(p.ys + j) : xs;
            tc_insert<kCand>(tv, tix, fmaf(f, acc[cc], __ldg(p.y2 + j)), p.orient_offset + j);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
    }
    if (cur_it >= 0 && !*abort_flag) flush(cur_it);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

int make_map(CUtensorMap* map, void* base, int rows, int Kpad, bool fp8) {
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return SPF_ERR_UNSUPPORTED;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kpad * (fp8 ? 1 : 2)};
  const cuuint32_t box[2] = {fp8 ? 128u : 64u, (cuuint32_t)kTcTile};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base,
                   dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d) for %d x %d", (int)r, rows, Kpad);
    return SPF_ERR_CUDA;
  }
  return SPF_OK;
}

}  // namespace

// Schedule of one launch: the contiguous order (mode 0) or the gi x go grid
// (mode 1), whichever a simple model predicts faster. Per CTA tile the model
// charges the tensor-core time of 2 x 256 x 256 x K multiply-adds and, for the
// whole launch, the HBM time of the operand tiles that concurrent CTAs do
// not share (an operand that fits half the L2 is read once).
TcSched tc_schedule(int n_img, int n_orient, int n_sms, int kpad, bool fp8, int force) {
  const int n_it = (int)ceil_div(n_img, kTcTile), n_ot = (int)ceil_div(n_orient, kTcTile);
  const int64_t total = (int64_t)n_it * n_ot;
  const double tile_bytes = (double)kTcTile * kpad * (fp8 ? 1.0 : 2.0);
  const double t_tile = 2.0 * kTcTile * kTcTile * kpad / (fp8 ? 22.6e12 : 11.3e12);   // s per tile per SM
  const double bw = 6.0e12, l2_half = 64.0e6;
  auto traffic = [&](double share_a, double share_b) {
    const double a_all = n_it * tile_bytes, b_all = n_ot * tile_bytes;
    const double a = a_all <= l2_half ? a_all : total * tile_bytes / std::max(1.0, share_a);
    const double b = b_all <= l2_half ? b_all : total * tile_bytes / std::max(1.0, share_b);
    return (a + b) / bw;
  };
  TcSched best;
  {
    int G = (int)std::min<int64_t>({(int64_t)n_sms, total, (int64_t)n_it * (kMaxSplits - 1)});
    G = std::max(G, 1);
    int ns = 1;
    for (int it = 0; it < n_it; ++it) {
      int a = owner_cta(it * n_ot, (int)total, G), b = owner_cta(it * n_ot + n_ot - 1, (int)total, G);
      ns = std::max(ns, b - a + 1);
    }
    best.mode = 0;
    best.grid = G;
    best.nsplit = ns;
    best.gi = best.go = 0;
    best.cost = std::max(ceil_div(total, G) * t_tile, traffic((double)G / n_it, (double)G / n_ot));
  }
  if (force == 1) return best;
  if (force == 2) best.cost = 1e30;   // the best grid, whatever the contiguous order costs
  for (int go = 1; go <= std::min(n_ot, kMaxSplits); ++go) {
    const int gi = std::min(n_it, n_sms / go);
    if (gi < 1) break;
    const double cost = std::max((double)ceil_div(n_it, gi) * ceil_div(n_ot, go) * t_tile, traffic(go, gi));
    if (cost < 0.97 * best.cost) {
      best.mode = 1;
      best.grid = gi * go;
      best.nsplit = go;
      best.gi = gi;
      best.go = go;
      best.cost = cost;
    }
  }
  return best;
}

int match_tc_launch(spf_matcher* m, int n_orient, int orient_offset, int nsplit, cudaStream_t s) {
  const bool fp8 = m->precision == SPF_FP8;
  CUtensorMap ta, tb;
  SPF_TRY(make_map(&ta, m->xq, m->n_img, m->Kpad, fp8));
  SPF_TRY(make_map(&tb, m->yq, n_orient, m->Kpad, fp8));
  const TcSched sch = tc_schedule(m->n_img, n_orient, m->n_sms, m->Kpad, fp8, m->tc_force);
  const int G = sch.grid;
  if (sch.nsplit != nsplit) {
    set_error("internal: split count %d != %d", sch.nsplit, nsplit);
    return SPF_ERR_ARG;
  }
  TcParams p;
  p.n_img = m->n_img;
  p.n_orient = n_orient;
  p.orient_offset = orient_offset;
  p.nkb = m->Kpad / (fp8 ? 128 : 64);
  p.n_it = (int)ceil_div(m->n_img, kTcTile);
  p.n_ot = (int)ceil_div(n_orient, kTcTile);
  p.total = p.n_it * p.n_ot;
  p.grid = G;
  p.mode = sch.mode;
  p.gi = sch.gi;
  p.go = sch.go;
  p.y2 = m->y2;
  p.xs = fp8 ? m->xs : nullptr;
  p.ys = fp8 ? m->ys : nullptr;
  p.cand_v = m->cand_v;
  p.cand_i = m->cand_i;
  p.err = m->err;
  // slots a CTA range does not reach stay empty (index -1)
  SPF_CUDA(cudaMemsetAsync(m->cand_i, 0xff, sizeof(int) * (size_t)m->n_img * kMaxSplits * kCand, s));
  const size_t smem = kTcStages * kTcStage + 1024 + 256;
  if (fp8) {
    SPF_CUDA(cudaFuncSetAttribute(tc_match_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    return launch("tc_match_fp8", s, [&] { tc_match_kernel<true><<<G, kTcThreads, smem, s>>>(ta, tb, p); });
  }
  SPF_CUDA(cudaFuncSetAttribute(tc_match_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  return launch("tc_match_bf16", s, [&] { tc_match_kernel<false><<<G, kTcThreads, smem, s>>>(ta, tb, p); });
}

}  // namespace spf
