// Type-2 (slicing) and type-1 (merging) NUFFT kernels, FP32 (sm_103a).
//
// Slicing (Sec. II-A) evaluates Re sum_n A_n exp(-i n.t) at the rotated
// detector points; merging (Sec. II-C) needs the adjoint sums. Both follow the
// exponential-of-semicircle NUFFT that the paper runs through cuFINUFFT
// (Sec. III-A), with these GB300-side choices:
//   * points are never stored: each kernel recomputes t = R(quat) q_lab on
//     the fly from the orientation and pixel index (a1 fused into a4/a9);
//   * type 2 deconvolves into a zero-padded complex cube, runs the pruned
//     hand-written FFT, keeps only the real part (the model is real, so the
//     slice is the real part) and gathers w^3 taps per point from that real
//     fine grid, which stays resident in L2;
//   * type 1 bin-sorts the points into 8^3-cell boxes (counting sort with
//     warp-aggregated atomics), spreads each box's points into a shared-
//     memory subgrid with shared atomics, then adds the subgrid into the fine
//     grid; dense boxes near q = 0 are split into fixed-size subproblems so
//     one box never serialises the grid; then FFT, real part, deconvolve.
#include <cmath>
#include <vector>

#include "plan.h"

namespace spf {

namespace {

// ------------------------------------------------------------ points ------
// Fine-grid coordinate u = t * n_f / (2 pi) of a point, unwrapped, |u| < n_f/2
// for rotated detector points. Explicit rounding intrinsics keep the value
// bit-identical in every kernel that recomputes it (binning, spreading).
struct QuatPts {
  const float4* quats;   // (w, x, y, z) per orientation
  const float* qlab;     // P2 x 3
  uint32_t P2;
  float scale;           // fine-grid cells per unit q
  const int* oidx;       // optional orientation index per row (merge)
  int nq;                // rows of quats when oidx is given
  int* err;
  __device__ __forceinline__ float3 operator()(uint32_t id) const {
    uint32_t j = id / P2, p = id - j * P2;
    if (oidx) {
      int o = __ldg(oidx + j);
      if (o < 0 || o >= nq) {
        atomicOr(err, 4);
        o = min(max(o, 0), nq - 1);
      }
      j = (uint32_t)o;
    }
    float4 q = __ldg(quats + j);
    float w = q.x, x = q.y, y = q.z, z = q.w;
    float qx = __ldg(qlab + 3 * p), qy = __ldg(qlab + 3 * p + 1), qz = __ldg(qlab + 3 * p + 2);
    float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float r00 = 1.f - 2.f * __fadd_rn(yy, zz), r01 = 2.f * __fsub_rn(xy, wz), r02 = 2.f * __fadd_rn(xz, wy);
    float r10 = 2.f * __fadd_rn(xy, wz), r11 = 1.f - 2.f * __fadd_rn(xx, zz), r12 = 2.f * __fsub_rn(yz, wx);
    float r20 = 2.f * __fsub_rn(xz, wy), r21 = 2.f * __fadd_rn(yz, wx), r22 = 1.f - 2.f * __fadd_rn(xx, yy);
    float ux = __fmaf_rn(r00, qx, __fmaf_rn(r01, qy, __fmul_rn(r02, qz)));
    float uy = __fmaf_rn(r10, qx, __fmaf_rn(r11, qy, __fmul_rn(r12, qz)));
    float uz = __fmaf_rn(r20, qx, __fmaf_rn(r21, qy, __fmul_rn(r22, qz)));
    return make_float3(__fmul_rn(ux, scale), __fmul_rn(uy, scale), __fmul_rn(uz, scale));
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
struct StrPtr {
  const float* v;
  __device__ __forceinline__ float operator()(uint32_t id) const { return __ldg(v + id); }
};
struct StrImage {      // D[p] * scale * image[id]
  const float* img;
  const float* D;
  uint32_t P2;
  float scale;
  __device__ __forceinline__ float operator()(uint32_t id) const {
    float v = scale * __ldg(img + id);
    return D ? v * __ldg(D + (id % P2)) : v;
  }
};
struct StrWeights {    // D[p] (ones if D is NULL)
  const float* D;
  uint32_t P2;
  __device__ __forceinline__ float operator()(uint32_t id) const {
    return D ? __ldg(D + (id % P2)) : 1.f;
  }
};

__device__ __forceinline__ int wrap_index(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// ES weights of the W cells l0 .. l0+W-1 nearest to u (l0 = ceil(u - W/2)).
template <int W>
__device__ __forceinline__ int es_weights(float u, float beta, float* wt) {
  int l0 = (int)ceilf(u - 0.5f * W);
  const float s = 2.f / W;
#pragma unroll
  for (int d = 0; d < W; ++d) {
    float z = ((float)(l0 + d) - u) * s;
    float r = fmaxf(0.f, 1.f - z * z);
    wt[d] = expf(beta * (sqrtf(r) - 1.f));
  }
  return l0;
}

// ------------------------------------------------------------ type 2 ------
// cube[k mod nf] = A[k] p_kx p_ky p_kz for |k| <= Mh, zero elsewhere.
__global__ void deconv_pad_kernel(const float* __restrict__ A, int N, const float* __restrict__ p,
                                  int nf, float2* __restrict__ cube) {
  int64_t total = (int64_t)nf * nf * nf;
  int Mh = (N - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % nf), y = (int)((i / nf) % nf), z = (int)(i / ((int64_t)nf * nf));
    int kx = x <= Mh ? x : x - nf, ky = y <= Mh ? y : y - nf, kz = z <= Mh ? z : z - nf;
    float v = 0.f;
    if (kx >= -Mh && kx <= Mh && ky >= -Mh && ky <= Mh && kz >= -Mh && kz <= Mh) {
      int a = ((kz + Mh) * N + (ky + Mh)) * N + (kx + Mh);
      v = A[a] * p[kx + Mh] * p[ky + Mh] * p[kz + Mh];
    }
    cube[i] = make_float2(v, 0.f);
  }
}

// c_j = sum over W^3 taps of G[l] phi phi phi (periodic wrap), one thread per point.
template <int W, class Pts>
__global__ void __launch_bounds__(256) interp_kernel(const float* __restrict__ G, int nf, Pts pts,
                                                     int64_t npts, float beta, float* __restrict__ out) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (id >= npts) return;
  float3 u = pts((uint32_t)id);
  float wx[W], wy[W], wz[W];
  int lx = es_weights<W>(u.x, beta, wx);
  int ly = es_weights<W>(u.y, beta, wy);
  int lz = es_weights<W>(u.z, beta, wz);
  int ix[W];
#pragma unroll
  for (int d = 0; d < W; ++d) ix[d] = wrap_index(lx + d, nf);
  float acc = 0.f;
#pragma unroll
  for (int dz = 0; dz < W; ++dz) {
    const float* plane = G + (size_t)wrap_index(lz + dz, nf) * nf * nf;
    float accy = 0.f;
#pragma unroll
    for (int dy = 0; dy < W; ++dy) {
      const float* row = plane + (size_t)wrap_index(ly + dy, nf) * nf;
      float accx = 0.f;
#pragma unroll
      for (int dx = 0; dx < W; ++dx) accx = fmaf(__ldg(row + ix[dx]), wx[dx], accx);
      accy = fmaf(accx, wy[dy], accy);
    }
    acc = fmaf(accy, wz[dz], acc);
  }
  out[id] = acc;
}

// ------------------------------------------------------------ type 1 ------
struct BinGeom {
  int nf;
  int nb0, nb1, nb2;
};

__device__ __forceinline__ int point_bin(float3 u, const BinGeom& g) {
  int cx = wrap_index((int)floorf(u.x), g.nf);
  int cy = wrap_index((int)floorf(u.y), g.nf);
  int cz = wrap_index((int)floorf(u.z), g.nf);
  return ((cz / kBin) * g.nb1 + (cy / kBin)) * g.nb0 + (cx / kBin);
}

template <class Pts>
__global__ void bin_count_kernel(Pts pts, int64_t npts, BinGeom g, int* __restrict__ count) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int bin = -1;
  if (id < npts) bin = point_bin(pts((uint32_t)id), g);
  unsigned grp = __match_any_sync(0xffffffffu, bin);
  int lane = threadIdx.x & 31;
  if (bin >= 0 && lane == __ffs(grp) - 1) atomicAdd(count + bin, __popc(grp));
}

template <class Pts>
__global__ void bin_scatter_kernel(Pts pts, int64_t npts, BinGeom g, const int* __restrict__ start,
                                   int* __restrict__ fill, uint32_t* __restrict__ sorted,
                                   int* err) {
  int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int bin = -1;
  if (id < npts) bin = point_bin(pts((uint32_t)id), g);
  unsigned grp = __match_any_sync(0xffffffffu, bin);
  int lane = threadIdx.x & 31;
  int leader = __ffs(grp) - 1;
  int rank = __popc(grp & ((1u << lane) - 1u));
  int base = 0;
  if (bin >= 0 && lane == leader) base = atomicAdd(fill + bin, __popc(grp));
  base = __shfl_sync(grp, base, leader);
  if (bin >= 0) {
    int pos = start[bin] + base + rank;
    if (pos < start[bin + 1]) sorted[pos] = (uint32_t)id;
    else atomicOr(err, 1);   // counting and scattering disagreed: skip, never overrun
  }
}

// Exclusive scans of the bin counts and of their subproblem counts, one CTA.
__global__ void __launch_bounds__(1024) bin_scan_kernel(const int* __restrict__ count, int nbins,
                                                        int* __restrict__ start,
                                                        int* __restrict__ sub_start,
                                                        int* __restrict__ nsubs) {
  __shared__ long long s_pts[1024];
  __shared__ int s_sub[1024];
  int t = threadIdx.x;
  int chunk = (nbins + 1023) / 1024;
  int b0 = t * chunk, b1 = min(nbins, b0 + chunk);
  long long sp = 0;
  int ss = 0;
  for (int b = b0; b < b1; ++b) {
    int c = count[b];
    sp += c;
    ss += (c + kSubPts - 1) / kSubPts;
  }
  s_pts[t] = sp;
  s_sub[t] = ss;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    long long vp = t >= off ? s_pts[t - off] : 0;
    int vs = t >= off ? s_sub[t - off] : 0;
    __syncthreads();
    s_pts[t] += vp;
    s_sub[t] += vs;
    __syncthreads();
  }
  long long run_p = t ? s_pts[t - 1] : 0;
  int run_s = t ? s_sub[t - 1] : 0;
  for (int b = b0; b < b1; ++b) {
    int c = count[b];
    start[b] = (int)run_p;
    sub_start[b] = run_s;
    run_p += c;
    run_s += (c + kSubPts - 1) / kSubPts;
  }
  if (t == 1023) {
    start[nbins] = (int)s_pts[1023];
    sub_start[nbins] = s_sub[1023];
    *nsubs = s_sub[1023];
  }
}

__global__ void build_subs_kernel(const int* __restrict__ count, const int* __restrict__ start,
                                  const int* __restrict__ sub_start, int nbins,
                                  int4* __restrict__ subs) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  int c = count[b];
  int s0 = sub_start[b];
  for (int k = 0; k * kSubPts < c; ++k)
    subs[s0 + k] = make_int4(b, start[b] + k * kSubPts, min(kSubPts, c - k * kSubPts), 0);
}

// One CTA per subproblem (grid-stride over the device-side count): spread its
// points into a (kBin+W)^3 shared subgrid, then add the subgrid to the grid.
template <int W, class Pts, class Str>
__global__ void __launch_bounds__(256) spread_kernel(Pts pts, Str str, BinGeom g, float beta,
                                                     const uint32_t* __restrict__ sorted,
                                                     const int4* __restrict__ subs,
                                                     const int* __restrict__ nsubs,
                                                     float* __restrict__ grid, int* err) {
  constexpr int S = kBin + W;
  constexpr int H = W / 2;
  __shared__ float sg[S * S * S];
  const int nf = g.nf;
  const int nsub = *nsubs;
  for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
    int4 sub = subs[s];
    int bx = sub.x % g.nb0, by = (sub.x / g.nb0) % g.nb1, bz = sub.x / (g.nb0 * g.nb1);
    int ox = bx * kBin - H, oy = by * kBin - H, oz = bz * kBin - H;
    for (int c = threadIdx.x; c < S * S * S; c += blockDim.x) sg[c] = 0.f;
    __syncthreads();
    for (int i = threadIdx.x; i < sub.z; i += blockDim.x) {
      uint32_t id = sorted[sub.y + i];
      float3 u = pts(id);
      float v = str(id);
      float wx[W], wy[W], wz[W];
      int lx = es_weights<W>(u.x, beta, wx);
      int ly = es_weights<W>(u.y, beta, wy);
      int lz = es_weights<W>(u.z, beta, wz);
      // shift the taps into the wrapped frame of the point's bin
      int fx = (int)floorf(u.x), fy = (int)floorf(u.y), fz = (int)floorf(u.z);
      lx += wrap_index(fx, nf) - fx - ox;
      ly += wrap_index(fy, nf) - fy - oy;
      lz += wrap_index(fz, nf) - fz - oz;
      if (lx < 0 || ly < 0 || lz < 0 || lx > S - W || ly > S - W || lz > S - W) {
        atomicOr(err, 1);  // cannot happen when binning and spreading agree
        continue;
      }
#pragma unroll
      for (int dz = 0; dz < W; ++dz) {
        float vz = v * wz[dz];
#pragma unroll
        for (int dy = 0; dy < W; ++dy) {
          float vzy = vz * wy[dy];
          float* row = sg + ((lz + dz) * S + (ly + dy)) * S + lx;
#pragma unroll
          for (int dx = 0; dx < W; ++dx) atomicAdd(row + dx, vzy * wx[dx]);
        }
      }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < S * S * S; c += blockDim.x) {
      float val = sg[c];
      if (val != 0.f) {
        int cx = c % S, cy = (c / S) % S, cz = c / (S * S);
        int gx = wrap_index(ox + cx, nf), gy = wrap_index(oy + cy, nf), gz = wrap_index(oz + cz, nf);
        atomicAdd(grid + ((size_t)gz * nf + gy) * nf + gx, val);
      }
    }
    __syncthreads();
  }
}

// out[k] (+)= Re(cube[k mod nf]) p_kx p_ky p_kz for the n_modes^3 modes.
__global__ void crop_deconv_kernel(const float2* __restrict__ cube, int nf, int n_modes,
                                   const float* __restrict__ p, float* __restrict__ out,
                                   int accumulate) {
  int64_t total = (int64_t)n_modes * n_modes * n_modes;
  int Mh = (n_modes - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % n_modes), y = (int)((i / n_modes) % n_modes), z = (int)(i / ((int64_t)n_modes * n_modes));
    int gx = wrap_index(x - Mh, nf), gy = wrap_index(y - Mh, nf), gz = wrap_index(z - Mh, nf);
    float v = cube[((size_t)gz * nf + gy) * nf + gx].x * p[x] * p[y] * p[z];
    out[i] = accumulate ? out[i] + v : v;
  }
}

// Toeplitz kernel: K(d) = Re(cube[d mod nfT]) p_dx p_dy p_dz embedded at
// d mod PT of a zeroed complex PT^3 cube.
__global__ void crop_embed_kernel(const float2* __restrict__ cube, int nf, int n_modes,
                                  const float* __restrict__ p, int PT, float2* __restrict__ emb) {
  int64_t total = (int64_t)n_modes * n_modes * n_modes;
  int Mh = (n_modes - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x = (int)(i % n_modes), y = (int)((i / n_modes) % n_modes), z = (int)(i / ((int64_t)n_modes * n_modes));
    int gx = wrap_index(x - Mh, nf), gy = wrap_index(y - Mh, nf), gz = wrap_index(z - Mh, nf);
    float v = cube[((size_t)gz * nf + gy) * nf + gx].x * p[x] * p[y] * p[z];
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
  return (int)std::min<int64_t>(b, 152 * 32);
}

template <int W, class Pts>
int interp_w(const Grid& g, Pts pts, int64_t npts, float beta, float* out, cudaStream_t s) {
  if (npts == 0) return SPF_OK;
  SPF_TRY(launch("interp_kernel", s, [&] { interp_kernel<W, Pts><<<(unsigned)ceil_div(npts, 256), 256, 0, s>>>(g.real, g.nf, pts, npts, beta, out); }));
  return SPF_OK;
}

template <int W, class Pts, class Str>
int spread_w(Grid& g, uint32_t* sorted, Pts pts, Str str, int64_t npts, float beta, int* err,
             cudaStream_t s) {
  BinSort& b = g.bins;
  BinGeom geom{g.nf, b.nb[0], b.nb[1], b.nb[2]};
  SPF_CUDA(cudaMemsetAsync(b.count, 0, sizeof(int) * b.nbins, s));
  SPF_CUDA(cudaMemsetAsync(b.fill, 0, sizeof(int) * b.nbins, s));
  SPF_CUDA(cudaMemsetAsync(g.real, 0, sizeof(float) * (size_t)g.nf * g.nf * g.nf, s));
  if (npts > 0) {
    unsigned nb = (unsigned)ceil_div(npts, 256);
    SPF_TRY(launch("bin_count_kernel", s, [&] { bin_count_kernel<Pts><<<nb, 256, 0, s>>>(pts, npts, geom, b.count); }));
    SPF_TRY(launch("bin_scan_kernel", s, [&] { bin_scan_kernel<<<1, 1024, 0, s>>>(b.count, b.nbins, b.start, b.sub_start, b.nsubs); }));
    SPF_TRY(launch("bin_scatter_kernel", s, [&] { bin_scatter_kernel<Pts><<<nb, 256, 0, s>>>(pts, npts, geom, b.start, b.fill, sorted, err); }));
    SPF_TRY(launch("build_subs_kernel", s, [&] { build_subs_kernel<<<(unsigned)ceil_div(b.nbins, 256), 256, 0, s>>>(b.count, b.start, b.sub_start,
                                                                      b.nbins, b.subs); }));
    SPF_TRY(launch("spread_kernel", s, [&] { spread_kernel<W, Pts, Str><<<152 * 8, 256, 0, s>>>(pts, str, geom, beta, sorted, b.subs,
                                                       b.nsubs, g.real, err); }));
  }
  return SPF_OK;
}

}  // namespace

// ------------------------------------------------------------ drivers -----
#define SPF_W_DISPATCH(w, call) \
  switch (w) {                  \
    case 5: { constexpr int W = 5; return call; } \
    case 6: { constexpr int W = 6; return call; } \
    case 7: { constexpr int W = 7; return call; } \
    case 8: { constexpr int W = 8; return call; } \
    default: set_error("kernel width %d not built", w); return SPF_ERR_UNSUPPORTED; \
  }

// Fine-grid real part G of the deconvolved, padded model (type-2 set-up).
int type2_setup(spf_plan* P, const float* A, cudaStream_t s) {
  Grid& g = P->g;
  int64_t n3 = (int64_t)g.nf * g.nf * g.nf;
  SPF_TRY(launch("deconv_pad_kernel", s, [&] { deconv_pad_kernel<<<grid_for(n3), 256, 0, s>>>(A, P->N, g.deconv, g.nf, g.cube); }));
  return fft3_exec_ex(&g.fft, g.cube, nullptr, g.real, nullptr, -1, P->Mh + 1, 0, s);
}

int type2_quat(spf_plan* P, const float* quats, int M, const float* qlab, int P2, float* out,
               cudaStream_t s) {
  QuatPts pts{reinterpret_cast<const float4*>(quats), qlab, (uint32_t)P2, P->g.cells_per_q, nullptr, 0, P->err};
  SPF_W_DISPATCH(P->w, (interp_w<W, QuatPts>(P->g, pts, (int64_t)M * P2, (float)P->beta, out, s)));
}

int type2_explicit(spf_plan* P, const float* t, int64_t npts, float* out, cudaStream_t s) {
  ExplicitPts pts{t, (float)(P->g.nf / (2.0 * M_PI))};
  SPF_W_DISPATCH(P->w, (interp_w<W, ExplicitPts>(P->g, pts, npts, (float)P->beta, out, s)));
}

// Type-1 of `str` at the points onto grid g, then FFT and crop/deconvolve
// into out (n_modes^3), or into the Toeplitz embedding when emb != NULL.
template <class Pts, class Str>
static int type1_run(spf_plan* P, Grid& g, Pts pts, Str str, int64_t npts, float* out,
                     int accumulate, int* err, cudaStream_t s) {
  int rc;
  switch (P->w) {
    case 5: rc = spread_w<5, Pts, Str>(g, P->sorted, pts, str, npts, (float)P->beta, err, s); break;
    case 6: rc = spread_w<6, Pts, Str>(g, P->sorted, pts, str, npts, (float)P->beta, err, s); break;
    case 7: rc = spread_w<7, Pts, Str>(g, P->sorted, pts, str, npts, (float)P->beta, err, s); break;
    case 8: rc = spread_w<8, Pts, Str>(g, P->sorted, pts, str, npts, (float)P->beta, err, s); break;
    default: set_error("kernel width %d not built", P->w); return SPF_ERR_UNSUPPORTED;
  }
  if (rc != SPF_OK) return rc;
  int h = (g.n_modes + 1) / 2;
  SPF_TRY(fft3_exec_ex(&g.fft, g.cube, g.real, nullptr, nullptr, +1, 0, h, s));
  if (out) {
    int64_t m3 = (int64_t)g.n_modes * g.n_modes * g.n_modes;
    SPF_TRY(launch("crop_deconv_kernel", s, [&] { crop_deconv_kernel<<<grid_for(m3), 256, 0, s>>>(g.cube, g.nf, g.n_modes, g.deconv, out, accumulate); }));
  }
  return SPF_OK;
}

int type1_quat(spf_plan* P, const float* g_vals, const float* quats, int M, const float* qlab,
               int P2, float* out, int accumulate, int* err, cudaStream_t s) {
  QuatPts pts{reinterpret_cast<const float4*>(quats), qlab, (uint32_t)P2, P->g.cells_per_q, nullptr, 0, P->err};
  return type1_run(P, P->g, pts, StrPtr{g_vals}, (int64_t)M * P2, out, accumulate, err, s);
}

int type1_explicit(spf_plan* P, const float* v, const float* t, int64_t npts, float* out,
                   int accumulate, int* err, cudaStream_t s) {
  ExplicitPts pts{t, (float)(P->g.nf / (2.0 * M_PI))};
  return type1_run(P, P->g, pts, StrPtr{v}, npts, out, accumulate, err, s);
}

// Merge: RHS onto the N-mode grid, Toeplitz kernel onto the (2N-1)-mode grid.
int merge_run(spf_plan* P, const float* images, const float* quats, int n_quats,
              const int* oidx, int n_img, const float* qlab, int P2, const float* D, float b_scale,
              float* rhs, float* kernel_hat, int accumulate, int* err, cudaStream_t s) {
  const float4* q4 = reinterpret_cast<const float4*>(quats);
  int64_t npts = (int64_t)n_img * P2;
  if (rhs) {
    QuatPts pts{q4, qlab, (uint32_t)P2, P->g.cells_per_q, oidx, n_quats, err};
    SPF_TRY(type1_run(P, P->g, pts, StrImage{images, D, (uint32_t)P2, b_scale}, npts, rhs,
                      accumulate, err, s));
  }
  if (kernel_hat) {
    QuatPts pts{q4, qlab, (uint32_t)P2, P->gT.cells_per_q, oidx, n_quats, err};
    SPF_TRY(type1_run(P, P->gT, pts, StrWeights{D, (uint32_t)P2}, npts, nullptr, 0, err, s));
    // K(d) -> circulant embedding -> FFT -> real part (+)-> kernel_hat
    int64_t PT3 = (int64_t)P->PT * P->PT * P->PT;
    SPF_CUDA(cudaMemsetAsync(P->cubeP, 0, sizeof(float2) * PT3, s));
    int64_t m3 = (int64_t)P->gT.n_modes * P->gT.n_modes * P->gT.n_modes;
    SPF_TRY(launch("crop_embed_kernel", s, [&] { crop_embed_kernel<<<grid_for(m3), 256, 0, s>>>(P->gT.cube, P->gT.nf, P->gT.n_modes,
                                                   P->gT.deconv, P->PT, P->cubeP); }));
    SPF_TRY(fft3_exec_ex(&P->fftP, P->cubeP, nullptr, P->realP, nullptr, -1, P->N, 0, s));
    SPF_TRY(launch("accumulate_kernel", s, [&] { accumulate_kernel<<<grid_for(PT3), 256, 0, s>>>(P->realP, kernel_hat, PT3, accumulate); }));
  }
  return SPF_OK;
}

// Allocation of one grid's buffers and bin-sort scratch.
int grid_init(Grid* g, int n_modes, int nf, double cells_per_q, int w, double beta,
              int64_t max_points) {
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
  SPF_TRY(dev_alloc((void**)&g->cube, sizeof(float2) * n3, "fine cube"));
  SPF_TRY(fft3_create(&g->fft, nf, nf, nf));
  BinSort& b = g->bins;
  for (int a = 0; a < 3; ++a) b.nb[a] = (int)ceil_div(nf, kBin);
  b.nbins = b.nb[0] * b.nb[1] * b.nb[2];
  b.max_subs = b.nbins + max_points / kSubPts + 1;
  SPF_TRY(dev_alloc((void**)&b.count, sizeof(int) * b.nbins, "bin counts"));
  SPF_TRY(dev_alloc((void**)&b.fill, sizeof(int) * b.nbins, "bin fill"));
  SPF_TRY(dev_alloc((void**)&b.start, sizeof(int) * (b.nbins + 1), "bin starts"));
  SPF_TRY(dev_alloc((void**)&b.sub_start, sizeof(int) * (b.nbins + 1), "subproblem starts"));
  SPF_TRY(dev_alloc((void**)&b.subs, sizeof(int4) * b.max_subs, "subproblems"));
  SPF_TRY(dev_alloc((void**)&b.nsubs, sizeof(int), "subproblem count"));
  return SPF_OK;
}

void grid_free(Grid* g) {
  cudaFree(g->deconv);
  cudaFree(g->real);
  cudaFree(g->cube);
  fft3_destroy(&g->fft);
  cudaFree(g->bins.count);
  cudaFree(g->bins.fill);
  cudaFree(g->bins.start);
  cudaFree(g->bins.sub_start);
  cudaFree(g->bins.subs);
  cudaFree(g->bins.nsubs);
  *g = Grid();
}

}  // namespace spf
