// Type-2 (slicing) and type-1 (merging) NUFFT kernels (sm_103a).
//
// Slicing (Sec. II-A) evaluates Re sum_n A_n exp(-i n.t) at the rotated
// detector points; merging (Sec. II-C) needs the adjoint sums. Both follow the
// exponential-of-semicircle NUFFT that the paper runs through cuFINUFFT
// (Sec. III-A), with these GB300-side choices:
//   * points are never stored: each kernel recomputes t = R(quat) q_lab on
//     the fly from the orientation and pixel index (rotation fused into the
//     interpolation and spreading kernels);
//   * kernel weights come from per-tap polynomials in mirror form (see
//     es_poly) instead of sqrt / exp per tap;
//   * points are counting-sorted by the fine-grid cell of their tap origin
//     (bin-major; within a 4^3-cell bin by 2^3 cell block), once per fixed
//     orientation set (point sets);
//   * type 2 deconvolves into the zero-padded cube (mode entries only), runs
//     the pruned hand-written FFT and keeps the real part. On point sets the
//     window of each bin is contracted with the points' x weights on the
//     tensor cores (tcgen05 kind::tf32 with hi/lo split operands) and each
//     point finishes its y and z sums in registers; the per-call path
//     gathers w^3 taps per point from x-shifted halo copies of the grid;
//   * type 1 gives each warp a private shared-memory subgrid of one bin:
//     contributing points are queued, staged 32 at a time, and a lane owns a
//     fixed column of two window rows over 8 planes, accumulating a whole 2^3
//     cell block of points in registers (packed FP32 FMAs) before a plain
//     read-modify-write of the subgrid (no two lanes touch one cell);
//     subgrids go back to the fine grid as vector reductions once per
//     subproblem. No shared-memory atomics are used.
#include <cmath>
#include <type_traits>
#include <vector>

#include "plan.h"
#include "tc.h"

namespace spf {

namespace {

// ------------------------------------------------------------ points ------
// Division of point ids (< 2^31) by the pixel count, by multiplication with
// a precomputed reciprocal (Granlund and Montgomery, "Division by invariant
// integers using multiplication", PLDI 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (umulhi(n, m) + n) >> l; n + umulhi
// stays below 2^32 because n < 2^31.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t d_) : d(d_) {
    l = 0;
    while ((1ull << l) < d) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> l; }
};

// Fine-grid coordinate u = t * n_f / (2 pi) of a point, folded into
// [-n_f/2, n_f/2] (a no-op for unit quaternions, |t| < pi; it keeps every
// index in range for any input). Explicit rounding intrinsics keep the value
// bit-identical in every kernel that recomputes it (sorting, spreading).
struct QuatPts {
  const float4* quats;   // (w, x, y, z) per orientation
  const float* qlab;     // P2 x 3
  FastDiv P2;
  float scale;           // fine-grid cells per unit q
  const int* oidx;       // optional orientation index per row (merge)
  int nq;                // rows of quats when oidx is given
  int* err;
  float nf, inv_nf;
  __device__ __forceinline__ float fold(float u) const {
    return __fsub_rn(u, __fmul_rn(nf, rintf(__fmul_rn(u, inv_nf))));
  }
  // The loads of a point (orientation and pixel), apart from the arithmetic,
  // so that kernels can issue them ahead of use.
  struct Raw {
    float4 q;
    float qx, qy, qz;
  };
  __device__ __forceinline__ Raw load(uint32_t id) const {
    uint32_t j = P2.div(id), p = id - j * P2.d;
    if (oidx) {
      int o = __ldg(oidx + j);
      if (o < 0 || o >= nq) {
        atomicOr(err, 4);
        o = min(max(o, 0), nq - 1);
      }
      j = (uint32_t)o;
    }
    Raw r;
    r.q = __ldg(quats + j);
    r.qx = __ldg(qlab + 3 * p);
    r.qy = __ldg(qlab + 3 * p + 1);
    r.qz = __ldg(qlab + 3 * p + 2);
    return r;
  }
  __device__ __forceinline__ float3 operator()(uint32_t id) const { return rotate(load(id)); }
  __device__ __forceinline__ float3 rotate(const Raw& rw) const {
    const float w = rw.q.x, x = rw.q.y, y = rw.q.z, z = rw.q.w;
    const float qx = rw.qx, qy = rw.qy, qz = rw.qz;
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float r00 = 1.f - 2.f * __fadd_rn(yy, zz), r01 = 2.f * __fsub_rn(xy, wz), r02 = 2.f * __fadd_rn(xz, wy);
    float r10 = 2.f * __fadd_rn(xy, wz), r11 = 1.f - 2.f * __fadd_rn(xx, zz), r12 = 2.f * __fsub_rn(yz, wx);
    float r20 = 2.f * __fsub_rn(xz, wy), r21 = 2.f * __fadd_rn(yz, wx), r22 = 1.f - 2.f * __fadd_rn(xx, yy);
    float ux = __fmaf_rn(r00, qx, __fmaf_rn(r01, qy, __fmul_rn(r02, qz)));
    float uy = __fmaf_rn(r10, qx, __fmaf_rn(r11, qy, __fmul_rn(r12, qz)));
    float uz = __fmaf_rn(r20, qx, __fmaf_rn(r21, qy, __fmul_rn(r22, qz)));
    return make_float3(fold(__fmul_rn(ux, scale)), fold(__fmul_rn(uy, scale)), fold(__fmul_rn(uz, scale)));
  }
};

struct ExplicitPts {
  const float* pts;      // npts x 3 radians
  float scale;           // n_f / (2 pi)
  __device__ __forceinline__ static float wrap_pi(float t) {
    const float two_pi = 6.28318530717958647692f;
    return __fsub_rn(t, __fmul_rn(two_pi, rintf(__fmul_rn(t, 0.15915494309189533577f))));
  }
  __device__ __forceinline__ float3 operator()(uint32_t id) const {
    float tx = wrap_pi(__ldg(pts + 3 * (size_t)id));
    float ty = wrap_pi(__ldg(pts + 3 * (size_t)id + 1));
    float tz = wrap_pi(__ldg(pts + 3 * (size_t)id + 2));
    return make_float3(__fmul_rn(tx, scale), __fmul_rn(ty, scale), __fmul_rn(tz, scale));
  }
};

// ---------------------------------------------------------- strengths -----
// Strength of the point with id `id` at position `pos` of the sorted order.
struct StrPtr {        // v[id]
  static constexpr bool kByPos = false;
  static constexpr bool kConsume = false;
  const float* v;
  __device__ __forceinline__ float operator()(uint32_t id, uint32_t) const { return __ldg(v + id); }
};
// v[pos]: strengths stored in the sorted order (coalesced), consumed: each
// entry is read by one warp, which sets a nonzero one back to zero, so the
// array is all zeros after the spread (class sums need no clearing pass).
struct StrSorted {
  static constexpr bool kByPos = true;
  static constexpr bool kConsume = true;
  float* v;
};
struct StrImage {      // D[p] * scale * image[id]
  static constexpr bool kByPos = false;
  static constexpr bool kConsume = false;
  const float* img;
  const float* D;
  FastDiv P2;
  float scale;
  __device__ __forceinline__ float operator()(uint32_t id, uint32_t) const {
    float v = scale * __ldg(img + id);
    return D ? v * __ldg(D + (id - P2.div(id) * P2.d)) : v;
  }
};
struct StrWeights {    // D[p] (ones if D is NULL)
  static constexpr bool kByPos = false;
  static constexpr bool kConsume = false;
  const float* D;
  FastDiv P2;
  __device__ __forceinline__ float operator()(uint32_t id, uint32_t) const {
    return D ? __ldg(D + (id - P2.div(id) * P2.d)) : 1.f;
  }
};

struct StrCount {     // D[p] * count[j] for point id = j * P2 + p
  static constexpr bool kByPos = false;
  static constexpr bool kConsume = false;
  const float* cnt;
  const float* D;
  FastDiv P2;
  __device__ __forceinline__ float operator()(uint32_t id, uint32_t) const {
    const uint32_t j = P2.div(id);
    const float c = __ldg(cnt + j);
    return D ? c * __ldg(D + (id - j * P2.d)) : c;
  }
};

__device__ __forceinline__ int wrap_index(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Wrap for arguments known to lie in [-n, 2n): one correction, no division.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ES weights of the W cells l0 .. l0+W-1 nearest to u (l0 = ceil(u - W/2)),
// from the kernel's per-tap polynomials in t = 2 (l0 - u + W/2) - 1 (Horner).
template <int W>
__device__ __forceinline__ int es_weights(float u, const EsPoly& ep, float* wt) {
  const int l0 = (int)ceilf(u - 0.5f * W);
  const float t = 2.f * ((float)l0 - u + 0.5f * W) - 1.f;
  constexpr int P = es_degree(W);
#pragma unroll
  for (int d = 0; d < W; ++d) {
    float v = ep.c[d][P];
#pragma unroll
    for (int i = P - 1; i >= 0; --i) v = fmaf(v, t, ep.c[d][i]);
    wt[d] = v;
  }
  return l0;
}

// The same for the three coordinates of a point: x and y share packed FP32
// FMAs (one Horner chain on (t_x, t_y)), z runs alongside.
template <int W>
__device__ __forceinline__ int3 es_weights3(float3 u, const EsPoly& ep, float* wx, float* wy, float* wz) {
  const int lx = (int)ceilf(u.x - 0.5f * W), ly = (int)ceilf(u.y - 0.5f * W), lz = (int)ceilf(u.z - 0.5f * W);
  const float2 txy = make_float2(2.f * ((float)lx - u.x + 0.5f * W) - 1.f, 2.f * ((float)ly - u.y + 0.5f * W) - 1.f);
  const float tz = 2.f * ((float)lz - u.z + 0.5f * W) - 1.f;
  // mirror form: taps d and W-1-d from the even and odd halves in s = t^2
  constexpr int P = es_degree(W);
  constexpr int NE = P / 2 + 1, NO = (P + 1) / 2;   // even / odd coefficient counts
  const float2 sxy = __fmul2_rn(txy, txy);
  const float sz = tz * tz;
#pragma unroll
  for (int d = 0; d < (W + 1) / 2; ++d) {
    float2 e = ep.e2[d][NE - 1];
    float ez = ep.e2[d][NE - 1].x;
#pragma unroll
    for (int k = NE - 2; k >= 0; --k) {
      e = __ffma2_rn(e, sxy, ep.e2[d][k]);
      ez = fmaf(ez, sz, ep.e2[d][k].x);
    }
    if (2 * d + 1 == W) {   // middle tap: even
      wx[d] = e.x;
      wy[d] = e.y;
      wz[d] = ez;
    } else {
      float2 o = ep.o2[d][NO - 1];
      float oz = ep.o2[d][NO - 1].x;
#pragma unroll
      for (int k = NO - 2; k >= 0; --k) {
        o = __ffma2_rn(o, sxy, ep.o2[d][k]);
        oz = fmaf(oz, sz, ep.o2[d][k].x);
      }
      const float2 to = __fmul2_rn(txy, o);
      wx[d] = e.x + to.x;
      wy[d] = e.y + to.y;
      wz[d] = fmaf(tz, oz, ez);
      wx[W - 1 - d] = e.x - to.x;
      wy[W - 1 - d] = e.y - to.y;
      wz[W - 1 - d] = fmaf(-tz, oz, ez);
    }
  }
  return make_int3(lx, ly, lz);
}

// ------------------------------------------------------------ type 2 ------
// cube[k mod nf] = A[k] p_kx p_ky p_kz for |k| <= Mh, zero elsewhere.
// Only the N^3 mode entries are written: the pruned forward FFT reads
// nothing else of the cube.
__global__ void deconv_pad_kernel(const float* __restrict__ A, int N, const float* __restrict__ p,
                                  int nf, float2* __restrict__ cube) {
  int64_t total = (int64_t)N * N * N;
  int Mh = (N - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(i % N), b = (int)((i / N) % N), c = (int)(i / ((int64_t)N * N));
    const float v = A[i] * p[a] * p[b] * p[c];
    int gx = a - Mh, gy = b - Mh, gz = c - Mh;
    gx += gx < 0 ? nf : 0;
    gy += gy < 0 ? nf : 0;
    gz += gz < 0 ? nf : 0;
    cube[((size_t)gz * nf + gy) * nf + gx] = make_float2(v, 0.f);
  }
}

// Fine cell of a point's tap origin: c = ceil(u - W/2) + floor(W/2), wrapped,
// and its sort key (bin-major). Returned l0 is the unwrapped first tap.
struct SortGeom {
  int nf;
  int nb0, nb1, nb2;
};

// Sort key of a point: its tap-origin cell, bin-major, the cells of a bin
// ordered by their 2^3 cell block. With BlockOnly the cells of one 2^3 block
// share a key, so a block's points keep the order in which the sort meets
// them (runs of neighbouring pixels of one orientation stay together)
// instead of being ordered by cell.
template <int W, bool BlockOnly = false>
__device__ __forceinline__ int point_key(float3 u, const SortGeom& g) {
  constexpr int H = W / 2;
  int cx = wrap1((int)ceilf(u.x - 0.5f * W) + H, g.nf);
  int cy = wrap1((int)ceilf(u.y - 0.5f * W) + H, g.nf);
  int cz = wrap1((int)ceilf(u.z - 0.5f * W) + H, g.nf);
  constexpr int B = kBinLog;
  int bin = ((cz >> B) * g.nb1 + (cy >> B)) * g.nb0 + (cx >> B);
  // cell inside the 4^3 bin, ordered by its 2^3 cell pair block first: the
  // points of one block are contiguous (the spreading accumulates a block's
  // points in registers)
  const int pair = (((cz >> 1) & 1) << 2) | (((cy >> 1) & 1) << 1) | ((cx >> 1) & 1);
  if (BlockOnly) return (bin << (3 * B)) | (pair << 3);
  const int sub = ((cz & 1) << 2) | ((cy & 1) << 1) | (cx & 1);
  return (bin << (3 * B)) | (pair << 3) | sub;
}

// Runs of equal keys in adjacent lanes (consecutive ids: neighbouring pixels
// of one orientation, mostly one cell) share one atomic. For lane l: its
// run's first lane, its rank in the run and the run's length (valid in the
// first lane).
struct KeyRun {
  int leader, rank, len;
};
__device__ __forceinline__ KeyRun key_run(int key) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || key != prev);
  const unsigned upto = lane == 31 ? heads : heads & ((2u << lane) - 1u);   // heads at or below lane
  const int leader = 31 - __clz(upto);
  const unsigned above = lane == 31 ? 0u : heads & ~((2u << lane) - 1u);   // heads above lane
  const int next = above ? __ffs(above) - 1 : 32;
  return {leader, lane - leader, next - lane};
}

template <int W, class Pts, bool BlockOnly>
__global__ void key_count_kernel(Pts pts, int64_t npts, SortGeom g, int* __restrict__ count) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int key = -1;
  if (id < npts) key = point_key<W, BlockOnly>(pts((uint32_t)id), g);
  const KeyRun run = key_run(key);
  if (key >= 0 && run.rank == 0) atomicAdd(count + key, run.len);
}

template <int W, class Pts, bool BlockOnly>
__global__ void key_scatter_kernel(Pts pts, int64_t npts, SortGeom g, const int* __restrict__ start,
                                   int* __restrict__ fill, uint32_t* __restrict__ sorted, int* err) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int key = -1;
  if (id < npts) key = point_key<W, BlockOnly>(pts((uint32_t)id), g);
  const KeyRun run = key_run(key);
  int base = 0;
  if (key >= 0 && run.rank == 0) base = atomicAdd(fill + key, run.len);
  base = __shfl_sync(0xffffffffu, base, run.leader);
  if (key >= 0) {
    int pos = start[key] + base + run.rank;
    if (pos < start[key + 1]) sorted[pos] = (uint32_t)id;
    else atomicOr(err, 1);   // counting and scattering disagreed: skip, never overrun
  }
}

// ---- exclusive scan of n ints in three passes (block sums, their scan, apply)
__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan across a 256-thread block; *total receives the block sum.
__device__ __forceinline__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[8];
  __shared__ int tot_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int inc = warp_incl_scan(v);
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int w = lane < 8 ? ws[lane] : 0;
    const int wi = warp_incl_scan(w);
    if (lane < 8) ws[lane] = wi - w;
    if (lane == 7) tot_s = wi;
  }
  __syncthreads();
  const int res = ws[wid] + inc - v;
  *total = tot_s;
  __syncthreads();
  return res;
}

__global__ void __launch_bounds__(256) scan_sums_kernel(const int* __restrict__ in, int64_t n,
                                                        int* __restrict__ bsum) {
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  int acc = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += in[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __shared__ int ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    bsum[blockIdx.x] = t;
  }
}

// exclusive scan of nb <= 1024 block sums in place; out_total = their sum
__global__ void __launch_bounds__(1024) scan_block_sums_kernel(int* __restrict__ bsum, int nb,
                                                               int* __restrict__ out_total) {
  __shared__ int sh[1024];
  int t = threadIdx.x;
  int v = t < nb ? bsum[t] : 0;
  sh[t] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int a = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += a;
    __syncthreads();
  }
  if (t < nb) bsum[t] = sh[t] - v;
  if (t == 1023) *out_total = sh[1023];
}

__global__ void __launch_bounds__(256) scan_apply_kernel(const int* __restrict__ in, int64_t n,
                                                         const int* __restrict__ bsum,
                                                         int* __restrict__ out) {
  int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
  int running = bsum[blockIdx.x];
  constexpr int ITEMS = 8;
  for (int64_t base = b0; base < b1; base += 256 * ITEMS) {
    int64_t i0 = base + (int64_t)threadIdx.x * ITEMS;
    int v[ITEMS];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      v[k] = (i0 + k < b1) ? in[i0 + k] : 0;
      sum += v[k];
    }
    int tot;
    int pre = block_excl_scan(sum, &tot) + running;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      if (i0 + k < b1) out[i0 + k] = pre;
      pre += v[k];
    }
    running += tot;
  }
}

// Cut each bin's sorted range into subproblems of at most kSubPts points.
__global__ void build_subs_kernel(const int* __restrict__ start, int nbins, int4* __restrict__ subs,
                                  int64_t max_subs, int* __restrict__ nsubs, int* err) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  int s0 = start[(int64_t)b * kBinCells], s1 = start[(int64_t)(b + 1) * kBinCells];
  int c = s1 - s0;
  if (c <= 0) return;
  int k = (c + kSubPts - 1) / kSubPts;
  int o = atomicAdd(nsubs, k);
  if (o + k > max_subs) {
    atomicOr(err, 1);
    return;
  }
  for (int q = 0; q < k; ++q) subs[o + q] = make_int4(b, s0 + q * kSubPts, min(kSubPts, c - q * kSubPts), 0);
}

// Cut each 2^3 cell block's sorted range (keys bin 512 + block 8 .. + 7) into
// subproblems of at most kSubPts points; the block is numbered on the grid
// of blocks (2 nb per axis).
__global__ void build_block_subs_kernel(const int* __restrict__ start, int nbins, int nb0, int nb1,
                                        int4* __restrict__ subs, int64_t max_subs, int* __restrict__ nsubs,
                                        int* err) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nbins * 8) return;
  const int b = q >> 3, pr = q & 7;
  const int s0 = start[(int64_t)b * kBinCells + pr * 8], s1 = start[(int64_t)b * kBinCells + pr * 8 + 8];
  const int c = s1 - s0;
  if (c <= 0) return;
  const int bx = b % nb0, by = (b / nb0) % nb1, bz = b / (nb0 * nb1);
  const int kx = 2 * bx + (pr & 1), ky = 2 * by + ((pr >> 1) & 1), kz = 2 * bz + (pr >> 2);
  const int blk = (kz * (2 * nb1) + ky) * (2 * nb0) + kx;
  const int k = (c + kSubPts - 1) / kSubPts;
  const int o = atomicAdd(nsubs, k);
  if (o + k > max_subs) {
    atomicOr(err, 1);
    return;
  }
  for (int u = 0; u < k; ++u) subs[o + u] = make_int4(blk, s0 + u * kSubPts, min(kSubPts, c - u * kSubPts), 0);
}

// Class sums: cls[inv[j P2 + p]] += b_scale D[p] img[i][p] and cnt[j] += 1
// for every image i whose orientation index oidx[i] - off = j is in [0, M),
// i.e. the class sums in the sorted order of the points (inv maps a point id
// to its sorted position), so that spreading reads them coalesced. Only
// nonzero pixels are added (photon-count images are sparse). One block per
// (image, 1024-pixel chunk).
__global__ void class_sum_kernel(const float* __restrict__ img, const int* __restrict__ oidx, int n_img,
                                 int off, int M, int P2, const float* __restrict__ D, float b_scale,
                                 const uint32_t* __restrict__ inv, float* __restrict__ cls,
                                 float* __restrict__ cnt) {
  const int chunks = (P2 + 1023) / 1024;
  const int i = blockIdx.x / chunks, c = blockIdx.x - i * chunks;
  if (i >= n_img) return;
  const int j = __ldg(oidx + i) - off;
  if (j < 0 || j >= M) return;
  const float* row = img + (size_t)i * P2;
  const uint32_t* pos = inv + (size_t)j * P2;
  // 4 pixels per thread (blockDim 256): loads first, then the scatter
  const int p_end = min(P2, (c + 1) * 1024);
  float v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int p = c * 1024 + threadIdx.x + 256 * k;
    v[k] = p < p_end ? b_scale * __ldg(row + p) * (D ? __ldg(D + p) : 1.f) : 0.f;
  }
  uint32_t at[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) at[k] = v[k] != 0.f ? __ldg(pos + c * 1024 + threadIdx.x + 256 * k) : 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (v[k] != 0.f) atomicAdd(cls + at[k], v[k]);
  if (c == 0 && threadIdx.x == 0) atomicAdd(cnt + j, 1.f);
}

// The same for every image at once over a list of point sets holding
// consecutive orientation chunks of `chunk` orientations (the last may be
// shorter): image i's orientation o = oidx[i] lies in set c = o / chunk at
// local index o - c chunk, so one pass over the images fills every set's
// class sums and counts. An index outside [0, n_total) sets the error word.
// A persistent grid walks the (image, 1024-pixel chunk) tasks, two per
// iteration with their loads issued together; rows whose pixel count is a
// multiple of 4 are read as 16-byte vectors.
constexpr int kClassTask = 1024;
__device__ __forceinline__ float4 load4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 load4(const uint16_t* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  return make_float4((float)(u.x & 0xffffu), (float)(u.x >> 16), (float)(u.y & 0xffffu), (float)(u.y >> 16));
}
__device__ __forceinline__ float load1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float load1(const uint16_t* p) { return (float)__ldg(p); }

template <class XT>
__global__ void __launch_bounds__(256) class_sum_sets_kernel(
    const XT* __restrict__ img, const int* __restrict__ oidx, int n_img, int chunk, int n_total, int P2,
    const float* __restrict__ D, float b_scale, const uint32_t* const* __restrict__ inv_tab,
    float* const* __restrict__ cls_tab, float* const* __restrict__ cnt_tab, int* err, int base_aligned) {
  const int chunks = (P2 + kClassTask - 1) / kClassTask;
  const int64_t ntask = (int64_t)n_img * chunks;
  const bool vec = base_aligned && (P2 & 3) == 0;
  for (int64_t t0 = blockIdx.x; t0 < ntask; t0 += 2 * (int64_t)gridDim.x) {
    float v[2][4];
    int o[2], p0[2];
    int64_t row[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t task = t0 + h * (int64_t)gridDim.x;
      o[h] = -1;
      p0[h] = 0;
      row[h] = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) v[h][k] = 0.f;
      if (task >= ntask) continue;
      const int i = (int)(task / chunks), c = (int)(task - (int64_t)i * chunks);
      o[h] = __ldg(oidx + i);
      p0[h] = c * kClassTask + 4 * threadIdx.x;
      row[h] = (int64_t)i * P2;
      if (o[h] < 0 || o[h] >= n_total) {
        if (threadIdx.x == 0 && c == 0) atomicOr(err, 4);
        o[h] = -1;
        continue;
      }
      if (vec && p0[h] + 3 < P2) {
        const float4 x = load4(img + row[h] + p0[h]);
        v[h][0] = x.x;
        v[h][1] = x.y;
        v[h][2] = x.z;
        v[h][3] = x.w;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (p0[h] + k < P2) v[h][k] = load1(img + row[h] + p0[h] + k);
      }
      if (c == 0 && threadIdx.x == 0) {
        const int set = o[h] / chunk;
        atomicAdd(cnt_tab[set] + (o[h] - set * chunk), 1.f);
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (o[h] < 0) continue;
      const int set = o[h] / chunk, j = o[h] - set * chunk;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (v[h][k] == 0.f) continue;
        const int p = p0[h] + k;
        const float val = b_scale * v[h][k] * (D ? __ldg(D + p) : 1.f);
        atomicAdd(cls_tab[set] + __ldg(inv_tab[set] + (size_t)j * P2 + p), val);
      }
    }
  }
}

// inv[ids[i]] = i: sorted position of every point id.
__global__ void inverse_order_kernel(const uint32_t* __restrict__ ids, int64_t n, uint32_t* __restrict__ inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    inv[__ldg(ids + i)] = (uint32_t)i;
}

// ------------------------------------------------------------ type 2 ------
// Halo copies: four x-shifted periodic copies of G on np x np x npx cells,
// Gq[k][z][y][x] = G[(z - H) mod nf][(y - H) mod nf][(x + k - H) mod nf],
// np = nf + W, npx = np + 8 rounded up to 4. A tap row starting at halo x
// lx is Gq[lx & 3][z][y][(lx & ~3) .. + 7]: two aligned float4 loads.
__global__ void halo_kernel(const float* __restrict__ G, int nf, int np, int npx, int H,
                            float* __restrict__ Gq) {
  const int64_t per = (int64_t)np * np * npx;
  const int64_t total = 4 * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / per);
    const int64_t r = i - k * per;
    const int x = (int)(r % npx), y = (int)((r / npx) % np), z = (int)(r / ((int64_t)npx * np));
    const int gx = wrap1(x + k - H, nf), gy = wrap1(y - H, nf), gz = wrap1(z - H, nf);
    Gq[i] = G[((size_t)gz * nf + gy) * nf + gx];
  }
}

__host__ __device__ inline int halo_npx(int nf, int W) { return ((nf + W + 8) + 3) & ~3; }

__device__ __forceinline__ float wrap_cells(float u, float nf) {
  u -= nf * floorf(u / nf);
  return u >= nf ? u - nf : u;
}

// c_j = sum over W^3 taps of G[l] phi phi phi, one thread per point, points
// visited in sorted order when `sorted` is given. The point is wrapped into
// [0, nf) and each of its W^2 tap rows is read from the halo copies as two
// aligned float4 loads.
template <int W, class Pts>
__global__ void __launch_bounds__(256) interp_kernel(const float* __restrict__ Gq, int nf, Pts pts,
                                                     int64_t npts, const uint32_t* __restrict__ sorted,
                                                     EsPoly ep, float* __restrict__ out) {
  static_assert(W <= 8, "two float4 per tap row");
  constexpr int H = W / 2;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npts) return;
  const uint32_t id = sorted ? __ldg(sorted + i) : (uint32_t)i;
  const float fn = (float)nf;
  float3 u = pts(id);
  u.x = wrap_cells(u.x, fn);
  u.y = wrap_cells(u.y, fn);
  u.z = wrap_cells(u.z, fn);
  float wx[8], wy[W], wz[W];
  const int lx = es_weights<W>(u.x, ep, wx) + H;     // in [0, nf], halo frame
  const int ly = es_weights<W>(u.y, ep, wy) + H;
  const int lz = es_weights<W>(u.z, ep, wz) + H;
#pragma unroll
  for (int d = W; d < 8; ++d) wx[d] = 0.f;
  const int np = nf + W, npx = halo_npx(nf, W);
  const int k = lx & 3;
  const float* base = Gq + (size_t)k * np * np * npx + ((size_t)lz * np + ly) * npx + (lx - k);
  float acc = 0.f;
#pragma unroll
  for (int dz = 0; dz < W; ++dz) {
    const float* plane = base + (size_t)dz * np * npx;
    float accy = 0.f;
#pragma unroll
    for (int dy = 0; dy < W; ++dy) {
      const float4* row = reinterpret_cast<const float4*>(plane + dy * npx);
      const float4 a = __ldg(row), b = __ldg(row + 1);
      float accx = a.x * wx[0];
      accx = fmaf(a.y, wx[1], accx);
      accx = fmaf(a.z, wx[2], accx);
      accx = fmaf(a.w, wx[3], accx);
      accx = fmaf(b.x, wx[4], accx);
      accx = fmaf(b.y, wx[5], accx);
      accx = fmaf(b.z, wx[6], accx);
      accx = fmaf(b.w, wx[7], accx);
      accy = fmaf(accx, wy[dy], accy);
    }
    acc = fmaf(accy, wz[dz], acc);
  }
  out[id] = acc;
}

// ---- type 2 on the tensor cores -------------------------------------------
// For the points of one block of B^3 cells (B = 2: a 2^3 cell block of the
// sorted set) all W^3 taps lie in the S^3 window of G (S = W + B - 1) whose
// corner is the block's first cell minus H. With the
// window as the matrix B[n][x] = G[z][y][x], n = z S + y, and each point's x
// weights placed at their window columns, A[p][x] = phi_x,p(x) (zero outside
// its W columns), the product T = A B^T holds T[p][n] = sum_x G[z][y][x]
// phi_x,p(x), and c_p = sum_(z,y) T[p][z S + y] phi_z,p(z) phi_y,p(y). T is
// formed by tcgen05.mma (kind::tf32; M = 128 points, N = S^2 rounded up to
// 16, K = 8 window columns per step) into tensor memory; one thread per
// point reads its row back and contracts it with its z and y weights. At
// w = 7 the window is 8^3: N = 64, one K step.
//
// FP32 accuracy from TF32 inputs: every operand value v is split into
// hi = tf32(v) and lo = v - hi, and T = A_hi B_hi + A_hi B_lo + A_lo B_hi;
// the dropped A_lo B_lo term and the tensor core's truncation of lo are
// O(2^-21) relative. Both parts share a 128-byte swizzled row of the operand
// tile: hi at K 0..15, lo at K 16..31.
// Interpolation works per block of 2^BLOG cells per axis: 2^3 cell blocks
// where the points are dense, the 4^3 bins where they are sparse (a block's
// MMA groups of 128 points would then run mostly empty).
constexpr int kIBlockDense = 256;   // points per 2^3 block from which blocks pay off

template <int W, int BLOG>
struct InterpTcCfg {
  static constexpr int H = W / 2;
  static constexpr int BS = 1 << BLOG;              // block cells per axis
  static constexpr int S = BS + W - 1;              // window cells per axis
  static constexpr int NN = ((S * S + 15) / 16) * 16;   // MMA N
  static constexpr int KSTEPS = S <= 8 ? 1 : 2;     // 8 window columns per MMA
  static constexpr int PTS = 128;                   // points per MMA (M)
  static constexpr uint32_t TILE = 128 * 128;       // one operand tile (bytes)
  static constexpr int TCOLS = 128;                 // tensor-memory columns
  // CTAs per SM: 4 x 128 threads leave 128 registers a thread and take all
  // 4 x 128 of the 512 TMEM columns; the operand tiles and barriers take
  // 33 KB, and 48 KB are requested so that residency stays below five CTAs
  // (their TMEM columns always fit)
  static constexpr int CTAS = 4;
  static constexpr size_t SMEM = 48 * 1024;
  static_assert(1024 + 2 * TILE + 64 <= SMEM, "shared memory layout");
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NN >> 3) << 17) |
                                    ((128u >> 4) << 24);
  static_assert(NN <= TCOLS && NN <= 128, "window rows exceed one tile");
  static_assert(S <= 16, "window columns exceed K = 16");
};

// Nearest TF32 value (10 explicit mantissa bits; ties away from zero) by
// integer rounding of the FP32 pattern.
__device__ __forceinline__ float tf32_round(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// v = hi + lo with hi = tf32(v) and lo = v - hi (exact; |lo| <= 2^-11 |v|).
// The tensor core reads lo at TF32 precision (truncation), an error of at
// most 2^-21 |v|.
__device__ __forceinline__ void split_tf32(float v, float& hi, float& lo) {
  hi = tf32_round(v);
  lo = v - hi;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// e[i] = w[i - o] for 0 <= i - o < W, else 0; o in [0, MAXO]; i in [0, L).
template <int W, int L, int MAXO = 3>
__device__ __forceinline__ void shift_weights(const float* w, int o, float* e) {
  float t[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    const float a = i < W ? w[i] : 0.f;
    const float b = i >= 1 && i - 1 < W ? w[i - 1] : 0.f;
    t[i] = (o & 1) ? b : a;
  }
#pragma unroll
  for (int i = 0; i < L; ++i) e[i] = MAXO >= 2 && (o & 2) ? (i >= 2 ? t[i - 2] : 0.f) : t[i];
}

template <int W, int BLOG, class Pts>
__global__ void __launch_bounds__(128, InterpTcCfg<W, BLOG>::CTAS)
interp_tc_kernel(const float* __restrict__ G, Pts pts, SortGeom g, EsPoly ep,
                 const uint32_t* __restrict__ sorted, const int4* __restrict__ subs, int* __restrict__ nsubs,
                 float* __restrict__ out, int* err) {
  using C = InterpTcCfg<W, BLOG>;
  constexpr int S = C::S;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* As = smem;
  uint8_t* Bs = smem + C::TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * C::TILE);
  uint64_t* done = bar + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
  int* next = reinterpret_cast<int*>(tslot + 2);
  const int t = threadIdx.x, warp = t >> 5;
  const int nf = g.nf;

  if (t == 0) {
    mbar_init(bar, 1);
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tslot)), "r"(C::TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // window rows n >= S^2 are read by the MMA: keep them zero
  for (int i = t; i < (int)(C::TILE / 16); i += 128)
    reinterpret_cast<float4*>(Bs)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t a_addr = smem_u32(As), b_addr = smem_u32(Bs);
  const int nsub = nsubs[0];
  uint32_t phase = 0;
  bool issued = false;

  for (;;) {
    if (t == 0) *next = atomicAdd(nsubs + 1, 1);
    __syncthreads();
    const int sidx = *next;
    const bool stop = sidx >= nsub || *abort_flag;
    __syncthreads();
    if (stop) break;
    const int4 sub = subs[sidx];
    // block coordinates on the grid of C::BS^3-cell blocks
    const int nbx = g.nb0 << (kBinLog - BLOG), nby = g.nb1 << (kBinLog - BLOG);
    const int bx = sub.x % nbx, by = (sub.x / nbx) % nby, bz = sub.x / (nbx * nby);
    const int ox0 = bx * C::BS - C::H, oy0 = by * C::BS - C::H, oz0 = bz * C::BS - C::H;
    // window -> B (hi | lo), 4 columns per task (the window's S columns and
    // the zeros up to the K steps' columns); every load of the thread is
    // issued before the first is used
    {
      constexpr int CH = C::KSTEPS * 2;   // 4-column chunks the MMA reads
      constexpr int TASKS = S * S * CH, ITER = (TASKS + 127) / 128;
      float v[ITER][4];
#pragma unroll
      for (int k = 0; k < ITER; ++k) {
        const int task = t + 128 * k;
        const int n = task / CH, c = task - n * CH;
        const int z = n / S, y = n - z * S;
        const float* row = G + ((size_t)wrap1(oz0 + z, nf) * nf + wrap1(oy0 + y, nf)) * nf;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int x = 4 * c + e;
          v[k][e] = task < TASKS && x < S ? __ldg(row + wrap1(ox0 + x, nf)) : 0.f;
        }
      }
#pragma unroll
      for (int k = 0; k < ITER; ++k) {
        const int task = t + 128 * k;
        if (task < TASKS) {
          const int n = task / CH, c = task - n * CH;
          float4 hi, lo;
          split_tf32(v[k][0], hi.x, lo.x);
          split_tf32(v[k][1], hi.y, lo.y);
          split_tf32(v[k][2], hi.z, lo.z);
          split_tf32(v[k][3], hi.w, lo.w);
          *reinterpret_cast<float4*>(Bs + swz128(n, c)) = hi;
          *reinterpret_cast<float4*>(Bs + swz128(n, c + 4)) = lo;
        }
      }
    }
    bool aborted = false;
    // loads run one block ahead: the next block's id is fetched while this
    // block is staged, its orientation and pixel while this block's MMA runs
    uint32_t id = t < sub.z ? __ldg(sorted + sub.y + t) : 0u;
    typename Pts::Raw raw = pts.load(id);
    for (int base = 0; base < sub.z; base += C::PTS) {
      const int i = base + t;
      const bool valid = i < sub.z;
      const uint32_t id_next = i + C::PTS < sub.z ? __ldg(sorted + sub.y + i + C::PTS) : 0u;
      bool ok = false;
      int ox = 0, oy = 0, oz = 0;
      float3 u = make_float3(0.f, 0.f, 0.f);
      if (valid) {
        u = pts.rotate(raw);
        const int cx = wrap1((int)ceilf(u.x - 0.5f * W) + C::H, nf);
        const int cy = wrap1((int)ceilf(u.y - 0.5f * W) + C::H, nf);
        const int cz = wrap1((int)ceilf(u.z - 0.5f * W) + C::H, nf);
        ok = (cx >> BLOG) == bx && (cy >> BLOG) == by && (cz >> BLOG) == bz;
        if (!ok) atomicOr(err, 1);   // cannot happen when sorting and interpolation agree
        ox = cx & (C::BS - 1);
        oy = cy & (C::BS - 1);
        oz = cz & (C::BS - 1);
      }
      float wx[W], wy[W], wz[W];
      es_weights3<W>(u, ep, wx, wy, wz);
      {
        // A row t: the x weights at their window columns, hi | lo (the
        // columns the K steps read)
        constexpr int L = 8 * C::KSTEPS;
        float ax[L];
        shift_weights<W, L, C::BS - 1>(wx, ox, ax);
#pragma unroll
        for (int c = 0; c < L / 4; ++c) {
          float4 hi, lo;
          split_tf32(ok ? ax[4 * c] : 0.f, hi.x, lo.x);
          split_tf32(ok ? ax[4 * c + 1] : 0.f, hi.y, lo.y);
          split_tf32(ok ? ax[4 * c + 2] : 0.f, hi.z, lo.z);
          split_tf32(ok ? ax[4 * c + 3] : 0.f, hi.w, lo.w);
          *reinterpret_cast<float4*>(As + swz128(t, c)) = hi;
          *reinterpret_cast<float4*>(As + swz128(t, c + 4)) = lo;
        }
      }
      // y and z weights at their window rows, kept in registers over the MMA
      float ey_r[S], ez_r[S];
      shift_weights<W, S, C::BS - 1>(wy, oy, ey_r);
      shift_weights<W, S, C::BS - 1>(wz, oz, ez_r);
      fence_proxy_async_smem();
      tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < C::KSTEPS; ++kk) {
          const uint64_t ahi = sdesc(a_addr + 32 * kk), alo = sdesc(a_addr + 64 + 32 * kk);
          const uint64_t bhi = sdesc(b_addr + 32 * kk), blo = sdesc(b_addr + 64 + 32 * kk);
          mma_tf32(tmem, alo, bhi, C::IDESC, kk > 0 ? 1u : 0u);
          mma_tf32(tmem, ahi, blo, C::IDESC, 1u);
          mma_tf32(tmem, ahi, bhi, C::IDESC, 1u);
        }
        mma_commit(bar);
        issued = true;
      }
      raw = pts.load(id_next);
      mbar_wait(bar, phase, abort_flag, err);
      phase ^= 1u;
      tc_fence_after();
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      // T row -> c_p: az[z] = sum_y T[z S + y] ey[y], c_p = sum_z az[z] ez[z];
      // for even S the y sums take adjacent columns in packed FP32 pairs
      float acc = 0.f;
      if constexpr (S % 2 == 0) {
        float2 az[S], ey[S / 2];
#pragma unroll
        for (int k = 0; k < S / 2; ++k) ey[k] = make_float2(ey_r[2 * k], ey_r[2 * k + 1]);
#pragma unroll
        for (int z = 0; z < S; ++z) az[z] = make_float2(0.f, 0.f);
#pragma unroll
        for (int ch = 0; ch < C::NN / 16; ++ch) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 16), v);
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            const int n = ch * 16 + e;
            if (n < S * S) az[n / S] = __ffma2_rn(make_float2(v[e], v[e + 1]), ey[(n % S) / 2], az[n / S]);
          }
        }
#pragma unroll
        for (int z = 0; z < S; ++z) acc = fmaf(az[z].x + az[z].y, ez_r[z], acc);
      } else {
        float az[S];
        const float* ey = ey_r;
#pragma unroll
        for (int z = 0; z < S; ++z) az[z] = 0.f;
#pragma unroll
        for (int ch = 0; ch < C::NN / 16; ++ch) {
          float v[16];
          tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 16), v);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int n = ch * 16 + e;
            if (n < S * S) az[n / S] = fmaf(v[e], ey[n % S], az[n / S]);
          }
        }
#pragma unroll
        for (int z = 0; z < S; ++z) acc = fmaf(az[z], ez_r[z], acc);
      }
      if (ok) out[id] = acc;
      id = id_next;
      // no barrier here: a thread rewrites its A row only after the MMA that
      // read it has completed (the wait above), and the next MMA overwrites
      // tensor memory only after the next block's barrier, which every
      // thread reaches after its tensor-memory loads of this block
    }
    if (aborted) break;
  }
  // no MMA may still be running when the columns are freed
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
    if (issued) {
      mma_commit(done);
      mbar_wait(done, 0, abort_flag, err, false);
    }
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ type 1 ------
// Per-warp shared-memory subgrid of one 4^3-cell bin: S planes of ROWS rows of
// 16 floats, S = 4 + W - 1 cells per axis. A lane (r = lane / 8, dx =
// lane % 8) owns window rows dy = r and r + 4 and column dx. Column c of row R
// is stored at c ^ (8 * ((R >> 1) & 1)): among any 4 consecutive rows the two
// of equal parity then sit on disjoint halves of their 16-bank group, so one
// instruction's 32 accesses are conflict-free.
//
// For W < 8 the 8 lane columns and rows have room for a window one cell
// wider than the kernel, so a warp accumulates the points of a whole 2^3
// block of cells (PAIR): the window starts at the block's even corner and a
// point whose cell is odd along an axis takes its weights shifted by one.
// Register runs then cover 8 cells instead of one, at W + 1 instead of W
// planes of FMAs.
template <int W>
struct SpreadCfg {
  static constexpr int H = W / 2;
  static constexpr bool PAIR = W < 8;
  static constexpr int WZ = PAIR ? W + 1 : W;   // accumulated planes
  static constexpr int WZ2 = (WZ + 1) / 2;      // plane pairs (packed FP32 FMAs)
  static constexpr int S = kBin + W - 1;   // cells per axis touched by a bin's points
  // x is stored from the 4-aligned cell (bin corner - 4), so that the
  // subgrid's rows go back to the fine grid as aligned 2- or 4-float vectors
  static constexpr int PADX = kBin - H;
  static constexpr int ROWS = kBin + 7;    // rows reached by the (r, r + 4) lane rows
  static constexpr int RS = 16;
  static constexpr int PLANE = ROWS * RS;
  static constexpr int GRID = S * PLANE;
  // staged point: key, -, -, -, wz[8], v wx[8], wy in lane-row order
  // (wy[0], wy[4], wy[1], wy[5], ...: a lane's rows r and r + 4 side by side)
  static constexpr int REC = 28;
  static constexpr int STAGE = 32 * REC;
  static constexpr int QUEUE = 2 * 64;     // up to 63 queued (id, strength) pairs
  static constexpr int PER_WARP = GRID + STAGE + QUEUE;
  static constexpr int WARPS = W < 8 ? 20 : 19;
  static constexpr size_t SMEM = (size_t)WARPS * PER_WARP * sizeof(float);
  static_assert(SMEM <= 227 * 1024, "shared memory per block");
};

__device__ __forceinline__ int swz(int R, int c) { return R * 16 + (c ^ (((R >> 1) & 1) << 3)); }

template <int W>
__device__ __forceinline__ void flush_columns(float* grid, int lx, int ly, int lz, int r, int dx,
                                              float2 (&acc)[SpreadCfg<W>::WZ2][2]) {
  using C = SpreadCfg<W>;
  const int a0 = swz(ly + r, C::PADX + lx + dx), a1 = swz(ly + r + 4, C::PADX + lx + dx);
  float* p = grid + lz * C::PLANE;
#pragma unroll
  for (int dz = 0; dz < C::WZ; ++dz) {
    const int q = dz >> 1;
    p[dz * C::PLANE + a0] += (dz & 1) ? acc[q][0].y : acc[q][0].x;
    p[dz * C::PLANE + a1] += (dz & 1) ? acc[q][1].y : acc[q][1].x;
  }
#pragma unroll
  for (int q = 0; q < C::WZ2; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
}

// Stage points q[0 .. n) of the queue (lane k: point k) and add them to the
// register accumulators in order, writing the accumulators back to the
// subgrid whenever the window corner changes.
template <int W, class Pts>
__device__ __forceinline__ void spread_batch(const Pts& pts, const EsPoly& ep, int nf, int bx, int by, int bz,
                                             const uint2* queue, int n, float* stage, float* grid, int lane,
                                             int r, int dx, int& cur, float2 (&acc)[SpreadCfg<W>::WZ2][2],
                                             int* err) {
  using C = SpreadCfg<W>;
  bool keep = lane < n;
  int key = 0, sx = 0, sy = 0, sz = 0;
  float v = 0.f;
  float wx[W], wy[W], wz[W];
  if (keep) {
    const uint2 e = queue[lane];
    v = __uint_as_float(e.y);
    const float3 u = pts(e.x);
    const int3 l0 = es_weights3<W>(u, ep, wx, wy, wz);
    const int lx = l0.x, ly = l0.y, lz = l0.z;
    // tap-origin cell, wrapped; its position inside the bin is the local origin
    const int cx = wrap1(lx + C::H, nf), cy = wrap1(ly + C::H, nf), cz = wrap1(lz + C::H, nf);
    const int ox = cx & (kBin - 1), oy = cy & (kBin - 1), oz = cz & (kBin - 1);
    if ((cx >> kBinLog) != bx || (cy >> kBinLog) != by || (cz >> kBinLog) != bz) {
      atomicOr(err, 1);   // cannot happen when sorting and spreading agree
      keep = false;
    }
    // window corner (the pair block's even corner under PAIR) and the
    // point's shift inside the window
    sx = C::PAIR ? (ox & 1) : 0;
    sy = C::PAIR ? (oy & 1) : 0;
    sz = C::PAIR ? (oz & 1) : 0;
    key = (ox - sx) | ((oy - sy) << 4) | ((oz - sz) << 8);
  }
  const unsigned kept = __ballot_sync(0xffffffffu, keep);
  const int nrec = __popc(kept);
  if (keep) {
    float* rec = stage + __popc(kept & ((1u << lane) - 1u)) * C::REC;
    rec[0] = __int_as_float(key);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const float z0 = d < W ? wz[d] : 0.f, x0 = d < W ? wx[d] : 0.f, y0 = d < W ? wy[d] : 0.f;
      const float z1 = d >= 1 && d - 1 < W ? wz[d - 1] : 0.f;
      const float x1 = d >= 1 && d - 1 < W ? wx[d - 1] : 0.f;
      const float y1 = d >= 1 && d - 1 < W ? wy[d - 1] : 0.f;
      rec[4 + d] = sz ? z1 : z0;
      rec[12 + d] = v * (sx ? x1 : x0);      // strength folded into the x weights
      rec[20 + 2 * (d & 3) + (d >> 2)] = sy ? y1 : y0;
    }
  }
  __syncwarp();
  // add record `rec` to the accumulators (its window is the current one)
  auto add = [&](const float* rec) {
    const float a = rec[12 + dx];
    const float2 wy = *reinterpret_cast<const float2*>(rec + 20 + 2 * r);
    const float c0 = a * wy.x, c1 = a * wy.y;
    const float2 c00 = make_float2(c0, c0), c11 = make_float2(c1, c1);
    const float4 z0 = *reinterpret_cast<const float4*>(rec + 4);
    const float4 z1 = *reinterpret_cast<const float4*>(rec + 8);
    const float2 zp[4] = {make_float2(z0.x, z0.y), make_float2(z0.z, z0.w), make_float2(z1.x, z1.y),
                          make_float2(z1.z, z1.w)};
#pragma unroll
    for (int q = 0; q < C::WZ2; ++q) {
      acc[q][0] = __ffma2_rn(zp[q], c00, acc[q][0]);
      acc[q][1] = __ffma2_rn(zp[q], c11, acc[q][1]);
    }
  };
  int k = 0;
  // a batch whose records all share one window (the usual case: points are
  // sorted by cell block) is added with no per-record window check
  if (nrec > 0) {
    const int key0 = __float_as_int(stage[0]);
    const bool same = lane >= nrec || __float_as_int(stage[lane * C::REC]) == key0;
    if (__all_sync(0xffffffffu, same)) {
      if (key0 != cur) {
        if (cur >= 0) flush_columns<W>(grid, cur & 15, (cur >> 4) & 15, cur >> 8, r, dx, acc);
        cur = key0;
      }
#pragma unroll 8
      for (; k < nrec; ++k) add(stage + k * C::REC);
    }
  }
  while (k < nrec) {
    const float* rec = stage + k * C::REC;
    const int key_k = __float_as_int(rec[0]);   // uniform: every lane reads record k
    // two records in the current window: no write-back check between them
    if (key_k == cur && k + 1 < nrec && __float_as_int(rec[C::REC]) == cur) {
      add(rec);
      add(rec + C::REC);
      k += 2;
      continue;
    }
    if (key_k != cur) {
      if (cur >= 0) flush_columns<W>(grid, cur & 15, (cur >> 4) & 15, cur >> 8, r, dx, acc);
      cur = key_k;
    }
    add(rec);
    ++k;
  }
  __syncwarp();
}

template <int W, class Pts, class Str>
__global__ void __launch_bounds__(32 * SpreadCfg<W>::WARPS, 1)
spread_kernel(Pts pts, Str str, SortGeom g, EsPoly ep, const uint32_t* __restrict__ sorted,
              const int4* __restrict__ subs, int* __restrict__ nsubs, float* __restrict__ out, int* err) {
  using C = SpreadCfg<W>;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* grid = smem + warp * C::PER_WARP;
  float* stage = grid + C::GRID;
  uint2* queue = reinterpret_cast<uint2*>(stage + C::STAGE);
  const int r = lane >> 3, dx = lane & 7;
  const int nf = g.nf;
  for (int c = lane; c < C::GRID; c += 32) grid[c] = 0.f;
  __syncwarp();
  const int nsub = nsubs[0];
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(nsubs + 1, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= nsub) break;
    const int4 sub = subs[s];
    const int bx = sub.x % g.nb0, by = (sub.x / g.nb0) % g.nb1, bz = sub.x / (g.nb0 * g.nb1);
    int cur = -1;   // window corner (x | y << 4 | z << 8) of the points in acc
    float2 acc[C::WZ2][2];   // [plane pair][row r, r + 4]
#pragma unroll
    for (int q = 0; q < C::WZ2; ++q) acc[q][0] = acc[q][1] = make_float2(0.f, 0.f);
    // Points with nonzero strength are queued (in order) and staged 32 at a
    // time, so the weights are computed for contributing points only. The
    // points are read 128 at a time (lane + 32 e, e < 4: coalesced), the
    // next 128's ids (and sorted-order strengths) while these are queued.
    const uint32_t* ids = sorted + sub.y;
    const uint32_t pos0 = (uint32_t)sub.y;
    const int n = sub.z;
    uint32_t idn[4];
    float vn[4];
    auto fetch = [&](int b) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = b + lane + 32 * e;
        idn[e] = i < n ? __ldg(ids + i) : 0u;
        if constexpr (Str::kConsume) vn[e] = i < n ? str.v[pos0 + i] : 0.f;
      }
      // the consumed sums are zeroed after all four loads are issued
      if constexpr (Str::kConsume) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (vn[e] != 0.f) str.v[pos0 + b + lane + 32 * e] = 0.f;
      }
    };
    fetch(0);
    int q = 0;   // queued points
    for (int base = 0; base < n; base += 128) {
      uint32_t idc[4];
      float vc[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        idc[e] = idn[e];
        if constexpr (Str::kByPos) vc[e] = vn[e];
      }
      if (base + 128 < n) fetch(base + 128);
      if constexpr (!Str::kByPos) {
#pragma unroll
        for (int e = 0; e < 4; ++e) vc[e] = base + lane + 32 * e < n ? str(idc[e], 0u) : 0.f;
      }
      // one copy of the batch code (not unrolled: it is large)
#pragma unroll 1
      for (int e = 0; e < 4; ++e) {
        const uint32_t id_e = e == 0 ? idc[0] : e == 1 ? idc[1] : e == 2 ? idc[2] : idc[3];
        const float v_e = e == 0 ? vc[0] : e == 1 ? vc[1] : e == 2 ? vc[2] : vc[3];
        const bool nz = base + lane + 32 * e < n && v_e != 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) queue[q + __popc(m & ((1u << lane) - 1u))] = make_uint2(id_e, __float_as_uint(v_e));
        q += __popc(m);
        __syncwarp();
        if (q >= 32) {
          spread_batch<W, Pts>(pts, ep, nf, bx, by, bz, queue, 32, stage, grid, lane, r, dx, cur, acc,
                                                   err);
          uint2 tail = make_uint2(0u, 0u);
          if (lane < q - 32) tail = queue[32 + lane];
          __syncwarp();
          if (lane < q - 32) queue[lane] = tail;
          q -= 32;
          __syncwarp();
        }
      }
    }
    if (q > 0)
      spread_batch<W, Pts>(pts, ep, nf, bx, by, bz, queue, q, stage, grid, lane, r, dx, cur, acc,
                                            err);
    if (cur >= 0) flush_columns<W>(grid, cur & 15, (cur >> 4) & 15, cur >> 8, r, dx, acc);
    __syncwarp();
    // add the subgrid to the fine grid and clear it: rows of 12 stored x
    // cells from the 4-aligned cell bin corner - 4, as 3 float4 (n_f = 0 mod
    // 4) or 6 float2 (n_f = 2 mod 4) vector reductions, skipping zero vectors
    const int ox = bx * kBin - kBin, oy = by * kBin - C::H, oz = bz * kBin - C::H;
    if ((nf & 3) == 0) {
      for (int task = lane; task < C::S * C::S * 3; task += 32) {
        const int row = task / 3, m = task - 3 * row;
        const int y = row % C::S, z = row / C::S;
        float4* p = reinterpret_cast<float4*>(grid + z * C::PLANE + swz(y, 4 * m));
        const float4 val = *p;
        if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f) {
          *p = make_float4(0.f, 0.f, 0.f, 0.f);
          const int gx = wrap1(ox + 4 * m, nf), gy = wrap1(oy + y, nf), gz = wrap1(oz + z, nf);
          atomicAdd(reinterpret_cast<float4*>(out + ((size_t)gz * nf + gy) * nf + gx), val);
        }
      }
    } else {
      for (int task = lane; task < C::S * C::S * 6; task += 32) {
        const int row = task / 6, m = task - 6 * row;
        const int y = row % C::S, z = row / C::S;
        float2* p = reinterpret_cast<float2*>(grid + z * C::PLANE + swz(y, 2 * m));
        const float2 val = *p;
        if (val.x != 0.f || val.y != 0.f) {
          *p = make_float2(0.f, 0.f);
          const int gx = wrap1(ox + 2 * m, nf), gy = wrap1(oy + y, nf), gz = wrap1(oz + z, nf);
          atomicAdd(reinterpret_cast<float2*>(out + ((size_t)gz * nf + gy) * nf + gx), val);
        }
      }
    }
    __syncwarp();
  }
}

// out[k] (+)= Re(cube[k mod nf]) p_kx p_ky p_kz for the n_modes^3 modes.
// Re F at the signed mode (kx, ky, kz): from the full cube (hx = 0) or from
// the half spectrum of a real input (columns kx = 0 .. hx-1; F(-k) =
// conj F(k) supplies kx < 0).
__device__ __forceinline__ float mode_re(const float2* __restrict__ F, int nf, int hx, int kx, int ky, int kz) {
  if (hx == 0) return F[((size_t)wrap_index(kz, nf) * nf + wrap_index(ky, nf)) * nf + wrap_index(kx, nf)].x;
  if (kx < 0) {
    kx = -kx;
    ky = -ky;
    kz = -kz;
  }
  return F[((size_t)wrap_index(kz, nf) * nf + wrap_index(ky, nf)) * hx + kx].x;
}

__global__ void crop_deconv_kernel(const float2* __restrict__ cube, int nf, int hx, int n_modes,
                                   const float* __restrict__ p, float* __restrict__ out,
                                   int accumulate) {
  int64_t total = (int64_t)n_modes * n_modes * n_modes;
  int Mh = (n_modes - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % n_modes), y = (int)((i / n_modes) % n_modes), z = (int)(i / ((int64_t)n_modes * n_modes));
    float v = mode_re(cube, nf, hx, x - Mh, y - Mh, z - Mh) * p[x] * p[y] * p[z];
    out[i] = accumulate ? out[i] + v : v;
  }
}

// Toeplitz kernel: K(d) = Re(cube[d mod nfT]) p_dx p_dy p_dz embedded at
// d mod PT of a zeroed complex PT^3 cube.
__global__ void crop_embed_kernel(const float2* __restrict__ cube, int nf, int hx, int n_modes,
                                  const float* __restrict__ p, int PT, float2* __restrict__ emb) {
  int64_t total = (int64_t)n_modes * n_modes * n_modes;
  int Mh = (n_modes - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % n_modes), y = (int)((i / n_modes) % n_modes), z = (int)(i / ((int64_t)n_modes * n_modes));
    float v = mode_re(cube, nf, hx, x - Mh, y - Mh, z - Mh) * p[x] * p[y] * p[z];
    int ex = wrap_index(x - Mh, PT), ey = wrap_index(y - Mh, PT), ez = wrap_index(z - Mh, PT);
    emb[((size_t)ez * PT + ey) * PT + ex] = make_float2(v, 0.f);
  }
}

__global__ void accumulate_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t n,
                                  int accumulate) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = accumulate ? dst[i] + src[i] : src[i];
}

int grid_for(int64_t n, int threads = 256) {
  int64_t b = ceil_div(n, threads);
  return (int)std::min<int64_t>(b, (int64_t)device_sms() * 32);
}

// Counting sort of npts points by tap-origin cell into `sorted`.
template <int W, class Pts>
int sort_points(Grid& g, uint32_t* sorted, Pts pts, int64_t npts, int* err, cudaStream_t s,
                bool block_only = false) {
  BinSort& b = g.bins;
  SortGeom geom{g.nf, b.nb[0], b.nb[1], b.nb[2]};
  SPF_CUDA(cudaMemsetAsync(b.count, 0, sizeof(int) * b.nkeys, s));
  SPF_CUDA(cudaMemsetAsync(b.fill, 0, sizeof(int) * b.nkeys, s));
  const unsigned nb = (unsigned)ceil_div(npts, 256);
  SPF_TRY(launch("key_count_kernel", s, [&] {
    if (block_only) key_count_kernel<W, Pts, true><<<nb, 256, 0, s>>>(pts, npts, geom, b.count);
    else key_count_kernel<W, Pts, false><<<nb, 256, 0, s>>>(pts, npts, geom, b.count);
  }));
  SPF_TRY(launch("scan_sums_kernel", s,
                 [&] { scan_sums_kernel<<<kScanBlocks, 256, 0, s>>>(b.count, b.nkeys, b.block_sums); }));
  SPF_TRY(launch("scan_block_sums_kernel", s, [&] {
    scan_block_sums_kernel<<<1, 1024, 0, s>>>(b.block_sums, kScanBlocks, b.start + b.nkeys);
  }));
  SPF_TRY(launch("scan_apply_kernel", s, [&] {
    scan_apply_kernel<<<kScanBlocks, 256, 0, s>>>(b.count, b.nkeys, b.block_sums, b.start);
  }));
  return launch("key_scatter_kernel", s, [&] {
    if (block_only) key_scatter_kernel<W, Pts, true><<<nb, 256, 0, s>>>(pts, npts, geom, b.start, b.fill, sorted, err);
    else key_scatter_kernel<W, Pts, false><<<nb, 256, 0, s>>>(pts, npts, geom, b.start, b.fill, sorted, err);
  });
}

// Tensor-core interpolation of an already sorted set (its subproblems give
// the bins) from g.real.
template <int W, class Pts>
int interp_tc(spf_plan* P, Pts pts, const SortedSet& set, int64_t npts, float* out, cudaStream_t s) {
  Grid& g = P->g;
  SortGeom geom{g.nf, g.bins.nb[0], g.bins.nb[1], g.bins.nb[2]};
  const EsPoly& ep = P->poly;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  // 2^3 blocks when a block holds a few MMA groups on average over the
  // occupied part of the grid (about half the cells), else 4^3 bins
  const bool blocks = set.bsubs && npts >= (int64_t)kIBlockDense * 8 * g.bins.nbins / 2;
  auto run = [&](auto blog, const int4* subs, int* nsubs) -> int {
    constexpr int BLOG = decltype(blog)::value;
    using C = InterpTcCfg<W, BLOG>;
    SPF_CUDA(cudaMemsetAsync(nsubs + 1, 0, sizeof(int), s));   // work cursor
    SPF_CUDA(cudaFuncSetAttribute(interp_tc_kernel<W, BLOG, Pts>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)C::SMEM));
    return launch("interp_tc_kernel", s, [&] {
      interp_tc_kernel<W, BLOG, Pts><<<C::CTAS * sms, 128, C::SMEM, s>>>(g.real, pts, geom, ep, set.ids, subs,
                                                                       nsubs, out, P->err);
    });
  };
  if (blocks) return run(std::integral_constant<int, 1>{}, set.bsubs, set.nbsubs);
  return run(std::integral_constant<int, kBinLog>{}, set.subs, set.nsubs);
}

template <int W, class Pts>
int interp_w(spf_plan* P, Pts pts, int64_t npts, bool use_sort, float* out, cudaStream_t s) {
  if (npts == 0) return SPF_OK;
  Grid& g = P->g;
  const uint32_t* order = nullptr;
  if (use_sort) {
    SPF_TRY((sort_points<W, Pts>(g, P->sorted, pts, npts, P->err, s)));
    order = P->sorted;
  }
  const EsPoly& ep = P->poly;
  return launch("interp_kernel", s, [&] {
    interp_kernel<W, Pts><<<(unsigned)ceil_div(npts, 256), 256, 0, s>>>(g.halo, g.nf, pts, npts, order,
                                                                       ep, out);
  });
}

// Sort the points of grid g into `set` and cut its bins into subproblems.
template <int W, class Pts>
int sort_and_cut(spf_plan* P, Grid& g, Pts pts, int64_t npts, SortedSet& set, int* err, cudaStream_t s,
                 bool block_only = false) {
  BinSort& b = g.bins;
  SPF_TRY((sort_points<W, Pts>(g, set.ids, pts, npts, err, s, block_only)));
  SPF_CUDA(cudaMemsetAsync(set.nsubs, 0, 2 * sizeof(int), s));
  SPF_TRY(launch("build_subs_kernel", s, [&] {
    build_subs_kernel<<<(unsigned)ceil_div(b.nbins, 256), 256, 0, s>>>(b.start, b.nbins, set.subs,
                                                                      set.max_subs, set.nsubs, err);
  }));
  if (!set.bsubs) return SPF_OK;
  SPF_CUDA(cudaMemsetAsync(set.nbsubs, 0, 2 * sizeof(int), s));
  return launch("build_subs_kernel", s, [&] {
    build_block_subs_kernel<<<(unsigned)ceil_div((int64_t)b.nbins * 8, 256), 256, 0, s>>>(
        b.start, b.nbins, b.nb[0], b.nb[1], set.bsubs, set.max_bsubs, set.nbsubs, err);
  });
}

// Spread onto g.real the points of an already sorted set (the grid cleared
// first unless `clear` is false: then the spread adds to what it holds).
template <int W, class Pts, class Str>
int spread_sorted(spf_plan* P, Grid& g, Pts pts, Str str, int64_t npts, const SortedSet& set, int* err,
                  cudaStream_t s, bool clear = true) {
  BinSort& b = g.bins;
  if (clear) SPF_CUDA(cudaMemsetAsync(g.real, 0, sizeof(float) * (size_t)g.nf * g.nf * g.nf, s));
  if (npts == 0) return SPF_OK;
  SPF_CUDA(cudaMemsetAsync(set.nsubs + 1, 0, sizeof(int), s));   // work cursor
  using C = SpreadCfg<W>;
  SPF_CUDA(cudaFuncSetAttribute(spread_kernel<W, Pts, Str>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)C::SMEM));
  SortGeom geom{g.nf, b.nb[0], b.nb[1], b.nb[2]};
  const EsPoly& ep = P->poly;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device);
  return launch(&g == &P->gT ? "spread_toeplitz_kernel" : "spread_kernel", s, [&] {
    spread_kernel<W, Pts, Str><<<sms, 32 * C::WARPS, C::SMEM, s>>>(pts, str, geom, ep, set.ids,
                                                                   set.subs, set.nsubs, g.real, err);
  });
}

template <int W, class Pts, class Str>
int spread_w(spf_plan* P, Grid& g, Pts pts, Str str, int64_t npts, int* err, cudaStream_t s,
             bool clear = true) {
  SortedSet set{P->sorted, g.bins.subs, g.bins.nsubs, g.bins.max_subs};
  if (npts > 0) SPF_TRY((sort_and_cut<W, Pts>(P, g, pts, npts, set, err, s)));
  return spread_sorted<W, Pts, Str>(P, g, pts, str, npts, set, err, s, clear);
}

}  // namespace

// ------------------------------------------------------------ drivers -----
#define SPF_W_SWITCH(w, stmt)                                                     \
  switch (w) {                                                                    \
    case 5: { constexpr int W = 5; stmt; } break;                                 \
    case 6: { constexpr int W = 6; stmt; } break;                                 \
    case 7: { constexpr int W = 7; stmt; } break;                                 \
    case 8: { constexpr int W = 8; stmt; } break;                                 \
    default: set_error("kernel width %d not built", w); return SPF_ERR_UNSUPPORTED; \
  }

// Fine-grid real part G of the deconvolved, padded model (type-2 set-up).
int type2_setup(spf_plan* P, const float* A, cudaStream_t s, bool halo) {
  Grid& g = P->g;
  const int64_t nm3 = (int64_t)P->N * P->N * P->N;
  SPF_TRY(launch("deconv_pad_kernel", s,
                 [&] { deconv_pad_kernel<<<grid_for(nm3), 256, 0, s>>>(A, P->N, g.deconv, g.nf, g.cube); },
                 12.0 * nm3));
  SPF_TRY(fft3_exec_ex(&g.fft, g.cube, nullptr, g.real, nullptr, -1, P->Mh + 1, 0, s));
  if (!halo) return SPF_OK;
  const int np = g.nf + P->w, npx = halo_npx(g.nf, P->w);
  const int64_t tot = 4 * (int64_t)np * np * npx;
  return launch("halo_kernel", s, [&] {
    halo_kernel<<<grid_for(tot), 256, 0, s>>>(g.real, g.nf, np, npx, P->w / 2, g.halo);
  }, 4.0 * tot + 4.0 * g.nf * (double)g.nf * g.nf);
}

// Slices of M orientations; sorted in chunks of whole orientations that fit
// the plan's sort buffer, unsorted when not even one orientation fits.
int type2_quat(spf_plan* P, const float* quats, int M, const float* qlab, int P2, float* out,
               cudaStream_t s) {
  const int64_t per = P->max_points / P2;
  if (per <= 0) {
    QuatPts pts{reinterpret_cast<const float4*>(quats), qlab, FastDiv((uint32_t)P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
    SPF_W_SWITCH(P->w, SPF_TRY((interp_w<W, QuatPts>(P, pts, (int64_t)M * P2, false, out, s))));
    return SPF_OK;
  }
  for (int64_t j0 = 0; j0 < M; j0 += per) {
    const int m = (int)std::min<int64_t>(per, M - j0);
    QuatPts pts{reinterpret_cast<const float4*>(quats) + j0, qlab, FastDiv((uint32_t)P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
    float* o = out + j0 * P2;
    SPF_W_SWITCH(P->w, SPF_TRY((interp_w<W, QuatPts>(P, pts, (int64_t)m * P2, true, o, s))));
  }
  return SPF_OK;
}

int type2_explicit(spf_plan* P, const float* t, int64_t npts, float* out, cudaStream_t s) {
  const bool sort = npts <= P->max_points;
  ExplicitPts pts{t, (float)(P->g.nf / (2.0 * M_PI))};
  SPF_W_SWITCH(P->w, SPF_TRY((interp_w<W, ExplicitPts>(P, pts, npts, sort, out, s))));
  return SPF_OK;
}

// Type-1 of `str` at the points onto grid g, then FFT and crop/deconvolve
// into out (n_modes^3) when out is given.
static int type1_finish(spf_plan* P, Grid& g, float* out, int accumulate, cudaStream_t s);

template <class Pts, class Str>
static int type1_run(spf_plan* P, Grid& g, Pts pts, Str str, int64_t npts, float* out,
                     int accumulate, int* err, cudaStream_t s) {
  SPF_W_SWITCH(P->w, SPF_TRY((spread_w<W, Pts, Str>(P, g, pts, str, npts, err, s))));
  return type1_finish(P, g, out, accumulate, s);
}

int type1_quat(spf_plan* P, const float* g_vals, const float* quats, int M, const float* qlab,
               int P2, float* out, int accumulate, int* err, cudaStream_t s) {
  QuatPts pts{reinterpret_cast<const float4*>(quats), qlab, FastDiv((uint32_t)P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
  return type1_run(P, P->g, pts, StrPtr{g_vals}, (int64_t)M * P2, out, accumulate, err, s);
}

int type1_explicit(spf_plan* P, const float* v, const float* t, int64_t npts, float* out,
                   int accumulate, int* err, cudaStream_t s) {
  ExplicitPts pts{t, (float)(P->g.nf / (2.0 * M_PI))};
  return type1_run(P, P->g, pts, StrPtr{v}, npts, out, accumulate, err, s);
}

// FFT of the spread grid g.real, then real part and deconvolution into out.
// Transform of the real spread grid, modes |k| < h only: real-input (half
// spectrum, hx = h columns) on the precompiled sides, else complex.
static int type1_modes(Grid& g, int h, int* hx, cudaStream_t s) {
  if (fft3_real_supported(&g.fft)) {
    *hx = h;
    return fft3_r2c_modes(&g.fft, g.real, h, +1, g.cube, s);
  }
  *hx = 0;
  return fft3_exec_ex(&g.fft, g.cube, g.real, nullptr, nullptr, +1, 0, h, s);
}

static int type1_finish(spf_plan* P, Grid& g, float* out, int accumulate, cudaStream_t s) {
  int h = (g.n_modes + 1) / 2, hx = 0;
  SPF_TRY(type1_modes(g, h, &hx, s));
  int64_t m3 = (int64_t)g.n_modes * g.n_modes * g.n_modes;
  return launch("crop_deconv_kernel", s, [&] {
    crop_deconv_kernel<<<grid_for(m3), 256, 0, s>>>(g.cube, g.nf, hx, g.n_modes, g.deconv, out, accumulate);
  }, (accumulate ? 16.0 : 12.0) * m3);
}

// Toeplitz kernel from the spread T-grid: FFT, K(d) = Re, circulant
// embedding, FFT, real part (+)-> kernel_hat.
static int kernel_finish(spf_plan* P, float* kernel_hat, int accumulate, cudaStream_t s) {
  Grid& g = P->gT;
  int h = (g.n_modes + 1) / 2, hx = 0;
  SPF_TRY(type1_modes(g, h, &hx, s));
  int64_t PT3 = (int64_t)P->PT * P->PT * P->PT;
  // the embedding fills the (2N-1)^3 wrapped range the pruned FFT reads
  int64_t m3 = (int64_t)g.n_modes * g.n_modes * g.n_modes;
  SPF_TRY(launch("crop_embed_kernel", s, [&] {
    crop_embed_kernel<<<grid_for(m3), 256, 0, s>>>(g.cube, g.nf, hx, g.n_modes, g.deconv, P->PT, P->cubeP);
  }, 16.0 * m3));
  SPF_TRY(fft3_exec_ex(&P->fftP, P->cubeP, nullptr, P->realP, nullptr, -1, P->N, 0, s));
  return launch("accumulate_kernel", s, [&] {
    accumulate_kernel<<<grid_for(PT3), 256, 0, s>>>(P->realP, kernel_hat, PT3, accumulate);
  }, (accumulate ? 12.0 : 8.0) * PT3);
}

// Merge: RHS onto the N-mode grid, Toeplitz kernel onto the (2N-1)-mode grid.
// mode: kMergeClear clears a grid before spreading onto it, kMergeFinish
// transforms it into the output afterwards; a deferred merge spreads several
// chunks with neither and finishes once (merge_finish).
int merge_run(spf_plan* P, const float* images, const float* quats, int n_quats, const int* oidx,
              int n_img, const float* qlab, int P2, const float* D, float b_scale, float* rhs,
              float* kernel_hat, int accumulate, int* err, cudaStream_t s, int mode, bool want_rhs,
              bool want_kernel) {
  const float4* q4 = reinterpret_cast<const float4*>(quats);
  int64_t npts = (int64_t)n_img * P2;
  const bool clear = (mode & kMergeClear) != 0, finish = (mode & kMergeFinish) != 0;
  if (want_rhs) {
    QuatPts pts{q4, qlab, FastDiv((uint32_t)P2), P->g.cells_per_q, oidx, n_quats, err, (float)P->g.nf, 1.f / (float)P->g.nf};
    StrImage str{images, D, FastDiv((uint32_t)P2), b_scale};
    SPF_W_SWITCH(P->w, SPF_TRY((spread_w<W, QuatPts, StrImage>(P, P->g, pts, str, npts, err, s, clear))));
    if (finish) SPF_TRY(type1_finish(P, P->g, rhs, accumulate, s));
  }
  if (want_kernel) {
    QuatPts pts{q4, qlab, FastDiv((uint32_t)P2), P->gT.cells_per_q, oidx, n_quats, err, (float)P->gT.nf, 1.f / (float)P->gT.nf};
    StrWeights str{D, FastDiv((uint32_t)P2)};
    SPF_W_SWITCH(P->w, SPF_TRY((spread_w<W, QuatPts, StrWeights>(P, P->gT, pts, str, npts, err, s, clear))));
    if (finish) SPF_TRY(kernel_finish(P, kernel_hat, accumulate, s));
  }
  return SPF_OK;
}

// Class sums of all images into consecutive point sets in one pass (the sets'
// sums and counts cleared first); merge_points then runs with
// kMergeSumsDone. Tables: device arrays of the sets' inverse orders, class
// sums and counts.
int class_sums_sets(spf_points* const* sets, int nsets, const uint32_t* const* inv_tab, float* const* cls_tab,
                    float* const* cnt_tab, const float* images, const uint16_t* images16, const int* oidx, int n_img,
                    int chunk, int n_total, const float* D, float b_scale, int* err, cudaStream_t s) {
  for (int c = 0; c < nsets; ++c) {
    spf_points* S = sets[c];
    // the right-hand-side spread leaves the sums zeroed: no clearing pass then
    if (!S->cls_zero) SPF_CUDA(cudaMemsetAsync(S->cls, 0, sizeof(float) * (size_t)S->M * S->P2, s));
    S->cls_zero = false;
    SPF_CUDA(cudaMemsetAsync(S->cnt, 0, sizeof(float) * (size_t)S->M, s));
  }
  if (n_img == 0 || nsets == 0) return SPF_OK;
  const int P2 = sets[0]->P2;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tasks = (int64_t)n_img * ceil_div(P2, kClassTask);
  const unsigned blocks = (unsigned)std::min<int64_t>(tasks, (int64_t)sms * 8);
  // rows of 16-bit counts are read as 8-byte vectors when 8-byte aligned
  if (images16)
    return launch("class_sum_kernel", s, [&] {
      class_sum_sets_kernel<uint16_t><<<blocks, 256, 0, s>>>(images16, oidx, n_img, chunk, n_total, P2, D, b_scale,
                                                             inv_tab, cls_tab, cnt_tab, err,
                                                             ((uintptr_t)images16 & 7) == 0);
    }, 2.0 * n_img * (double)P2);
  return launch("class_sum_kernel", s, [&] {
    class_sum_sets_kernel<float><<<blocks, 256, 0, s>>>(images, oidx, n_img, chunk, n_total, P2, D, b_scale,
                                                        inv_tab, cls_tab, cnt_tab, err, ((uintptr_t)images & 15) == 0);
  }, 4.0 * n_img * (double)P2);
}

// Deferred merge: clear both fine grids / transform what they hold.
int merge_begin(spf_plan* P, cudaStream_t s) {
  SPF_CUDA(cudaMemsetAsync(P->g.real, 0, sizeof(float) * (size_t)P->g.nf * P->g.nf * P->g.nf, s));
  SPF_CUDA(cudaMemsetAsync(P->gT.real, 0, sizeof(float) * (size_t)P->gT.nf * P->gT.nf * P->gT.nf, s));
  return SPF_OK;
}

int merge_finish(spf_plan* P, float* rhs, float* kernel_hat, int accumulate, cudaStream_t s) {
  if (rhs) SPF_TRY(type1_finish(P, P->g, rhs, accumulate, s));
  if (kernel_hat) SPF_TRY(kernel_finish(P, kernel_hat, accumulate, s));
  return SPF_OK;
}

// ------------------------------------------------------- point sets -------
int points_build(spf_plan* P, spf_points* S, cudaStream_t s) {
  const int64_t npts = (int64_t)S->M * S->P2;
  if (npts == 0) return SPF_OK;
  const float4* q4 = reinterpret_cast<const float4*>(S->quats);
  QuatPts pn{q4, S->qlab, FastDiv((uint32_t)S->P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
  // slicing works per 2^3 cell block and the right-hand-side spread per
  // block window, so the cells of a block share a key: the block's points
  // stay in the sort's meeting order (runs of one orientation's neighbouring
  // pixels), and the interpolation's stores touch fewer sectors
  SPF_W_SWITCH(P->w, SPF_TRY((sort_and_cut<W, QuatPts>(P, P->g, pn, npts, S->setN, P->err, s, true))));
  if (S->flags & SPF_POINTS_SLICE_ONLY) return SPF_OK;
  SPF_TRY(launch("inverse_order_kernel", s, [&] {
    inverse_order_kernel<<<grid_for(npts), 256, 0, s>>>(S->setN.ids, npts, S->invN);
  }));
  QuatPts pt{q4, S->qlab, FastDiv((uint32_t)S->P2), P->gT.cells_per_q, nullptr, 0, P->err, (float)P->gT.nf, 1.f / (float)P->gT.nf};
  SPF_W_SWITCH(P->w, SPF_TRY((sort_and_cut<W, QuatPts>(P, P->gT, pt, npts, S->setT, P->err, s))));
  return SPF_OK;
}

int slice_points(spf_plan* P, spf_points* S, const float* A, float* out, cudaStream_t s) {
  const int64_t npts = (int64_t)S->M * S->P2;
  if (npts == 0) return SPF_OK;
  SPF_TRY(type2_setup(P, A, s, false));
  QuatPts pts{reinterpret_cast<const float4*>(S->quats), S->qlab, FastDiv((uint32_t)S->P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
  SPF_W_SWITCH(P->w, SPF_TRY((interp_tc<W, QuatPts>(P, pts, S->setN, npts, out, s))));
  return SPF_OK;
}

int merge_points(spf_plan* P, spf_points* S, const float* images, const int* oidx, int n_img, int off,
                 const float* D, float b_scale, float* rhs, float* kernel_hat, int accumulate,
                 cudaStream_t s, int mode, bool want_rhs, bool want_kernel) {
  const int64_t npts = (int64_t)S->M * S->P2;
  if (!(mode & kMergeSumsDone)) {
    if (!S->cls_zero) SPF_CUDA(cudaMemsetAsync(S->cls, 0, sizeof(float) * (size_t)npts, s));
    SPF_CUDA(cudaMemsetAsync(S->cnt, 0, sizeof(float) * (size_t)S->M, s));
    S->cls_zero = false;
  }
  if (n_img > 0 && !(mode & kMergeSumsDone)) {
    const int chunks = (int)ceil_div(S->P2, 1024);
    const int64_t blocks = (int64_t)n_img * chunks;
    SPF_TRY(launch("class_sum_kernel", s, [&] {
      class_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(images, oidx, n_img, off, S->M, S->P2, D, b_scale,
                                                        S->invN, S->cls, S->cnt);
    }));
  }
  const float4* q4 = reinterpret_cast<const float4*>(S->quats);
  const bool clear = (mode & kMergeClear) != 0, finish = (mode & kMergeFinish) != 0;
  if (want_rhs) {
    QuatPts pts{q4, S->qlab, FastDiv((uint32_t)S->P2), P->g.cells_per_q, nullptr, 0, P->err, (float)P->g.nf, 1.f / (float)P->g.nf};
    // the spread reads the sums in sorted order and zeroes the nonzero ones,
    // so the set's sums are all zero afterwards
    StrSorted str{S->cls};
    SPF_W_SWITCH(P->w, SPF_TRY((spread_sorted<W, QuatPts, StrSorted>(P, P->g, pts, str, npts, S->setN,
                                                                    P->err, s, clear))));
    S->cls_zero = true;
    if (finish) SPF_TRY(type1_finish(P, P->g, rhs, accumulate, s));
  }
  if (want_kernel) {
    QuatPts pts{q4, S->qlab, FastDiv((uint32_t)S->P2), P->gT.cells_per_q, nullptr, 0, P->err, (float)P->gT.nf, 1.f / (float)P->gT.nf};
    StrCount str{S->cnt, D, FastDiv((uint32_t)S->P2)};
    SPF_W_SWITCH(P->w, SPF_TRY((spread_sorted<W, QuatPts, StrCount>(P, P->gT, pts, str, npts, S->setT,
                                                                   P->err, s, clear))));
    if (finish) SPF_TRY(kernel_finish(P, kernel_hat, accumulate, s));
  }
  return SPF_OK;
}

// Allocation of one grid's buffers and bin-sort scratch.
int grid_init(Grid* g, int n_modes, int nf, double cells_per_q, int w, double beta,
              int64_t max_points, bool interp_source) {
  g->n_modes = n_modes;
  g->nf = nf;
  g->cells_per_q = (float)cells_per_q;
  std::vector<double> p(n_modes);
  deconv_factors(n_modes, nf, w, beta, p.data());
  std::vector<float> pf(p.begin(), p.end());
  SPF_TRY(dev_alloc((void**)&g->deconv, sizeof(float) * n_modes, "deconvolution factors"));
  SPF_CUDA(cudaMemcpy(g->deconv, pf.data(), sizeof(float) * n_modes, cudaMemcpyHostToDevice));
  size_t n3 = (size_t)nf * nf * nf;
  SPF_TRY(dev_alloc((void**)&g->real, sizeof(float) * n3, "fine grid"));
  if (interp_source) {
    const size_t np = (size_t)nf + w, npx = (size_t)halo_npx(nf, w);
    SPF_TRY(dev_alloc((void**)&g->halo, sizeof(float) * 4 * np * np * npx, "shifted halo copies"));
  }
  SPF_TRY(dev_alloc((void**)&g->cube, sizeof(float2) * n3, "fine cube"));
  SPF_TRY(fft3_create(&g->fft, nf, nf, nf));
  BinSort& b = g->bins;
  for (int a = 0; a < 3; ++a) b.nb[a] = (int)ceil_div(nf, kBin);
  b.nbins = b.nb[0] * b.nb[1] * b.nb[2];
  b.nkeys = (int64_t)b.nbins * kBinCells;
  b.max_subs = b.nbins + max_points / kSubPts + 1;
  SPF_TRY(dev_alloc((void**)&b.count, sizeof(int) * b.nkeys, "sort counts"));
  SPF_TRY(dev_alloc((void**)&b.fill, sizeof(int) * b.nkeys, "sort cursors"));
  SPF_TRY(dev_alloc((void**)&b.start, sizeof(int) * (b.nkeys + 1), "sort starts"));
  SPF_TRY(dev_alloc((void**)&b.block_sums, sizeof(int) * kScanBlocks, "scan partials"));
  SPF_TRY(dev_alloc((void**)&b.subs, sizeof(int4) * b.max_subs, "subproblems"));
  SPF_TRY(dev_alloc((void**)&b.nsubs, 2 * sizeof(int), "subproblem count"));
  return SPF_OK;
}

void grid_free(Grid* g) {
  cudaFree(g->deconv);
  cudaFree(g->real);
  cudaFree(g->halo);
  cudaFree(g->cube);
  fft3_destroy(&g->fft);
  cudaFree(g->bins.count);
  cudaFree(g->bins.fill);
  cudaFree(g->bins.start);
  cudaFree(g->bins.block_sums);
  cudaFree(g->bins.subs);
  cudaFree(g->bins.nsubs);
  *g = Grid();
}

}  // namespace spf
