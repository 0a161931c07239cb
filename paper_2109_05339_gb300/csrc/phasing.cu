// Phasing (Sec. II-D): error reduction, hybrid input-output and shrinkwrap on
// the model's N^3 grid, with the transforms as exact DFTs.
//
// The paper recovers the density from the merged diffraction volume by
// applying real-space constraints on rho and reciprocal-space constraints on
// its transform back and forth (ER, HIO, shrinkwrap). Here the grid is the
// model's own (N odd; index n in {-M..M}^3 stored with offset M), the data
// are the magnitudes amp_m = sqrt(max(I_m, 0)) of the merged autocorrelation's
// transform (amp < 0: a mode left free), and
//   forward   rho^_m = sum_n rho_n exp(-2 pi i m.n / N)
//   inverse   rho_n  = N^-3 sum_m rho^_m exp(+2 pi i m.n / N).
// The configured N are prime (17, 101, 151), so a transform is three passes
// of direct DFTs along one axis each: a CTA stages 32 lines in shared memory
// (loads and stores coalesced along x), every output is a sum over the line
// with twiddles from an N-entry table (exponent m n mod N advanced by
// addition). An iteration is five passes: forward x (reading the real
// iterate) and y; one z pass doing forward z, the modulus projection with its
// FP64 error, and inverse z; inverse y; inverse x with the ER / HIO update of
// the iterate in its store. The cube stays L2-resident at N = 151 (28 MB).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.h"
#include "reduce.h"

struct spf_phaser {
  int device = 0;
  int N = 0, M = 0;
  int64_t n3 = 0;
  float2* cube = nullptr;      // N^3 complex work
  float* rho = nullptr;        // iterate
  float* amp = nullptr;        // magnitudes (< 0: free)
  uint8_t* support = nullptr;
  float* blur = nullptr;       // shrinkwrap blur of |rho|
  float* g1 = nullptr;         // 1D transfer function of the shrinkwrap Gaussian
  float2* tw = nullptr;        // exp(+2 pi i j / N), j < N
  double* part = nullptr;      // per-block FP64 partials
  unsigned* count = nullptr;
  double* sc = nullptr;        // [sum (|F| - amp)^2, sum amp^2]
  unsigned* maxbits = nullptr; // max of the blur (bit pattern of a non-negative float)
};

namespace spf {
namespace {

constexpr int kTL = 32;      // lines per tile
constexpr int kThreads = 256;
constexpr int kMaxN = 401;   // two N x 33 complex tiles + two twiddle tables in shared memory

enum ZMode { kZForward = 0, kZModulus = 1, kZBlur = 2, kZAmplitude = 3 };
enum XMode { kXComplex = 0, kXUpdate = 1, kXReal = 2 };

struct PassArgs {
  int N, M;
  float2* cube;
  const float2* tw;
  // x-axis forward pass reading a real array (|v| when in_abs)
  const float* in_real;
  int in_abs;
  // z-pass epilogue
  const float* amp;
  float* amp_out;
  const float* g1;
  double* part;
  unsigned* count;
  double* sc;
  // x-axis inverse pass epilogue
  float* rho;
  const uint8_t* support;
  float beta, scale;
  int hio, positivity;
  float* real_out;
  unsigned* maxbits;
};

// out[b][t] = sum_a in[a][t] exp(sign 2 pi i m_b n_a / N) over the staged
// tile (row stride kTL + 1), m_b = b - M, n_a = a - M; tw holds
// exp(sign 2 pi i k / N), k < N. Thread (line group q = tid % 8, row group
// r = tid / 8) computes lines t = 4q .. 4q + 3 of rows b = r + 32 k, k <
// kRows, per round of 32 kRows rows: each twiddle, with its index advanced by
// addition mod N, serves four lines (20 complex multiply-adds per five
// twiddles and four inputs). Lines past nlines are zero in the tile.
constexpr int kRows = 5;
__device__ __forceinline__ void dft_tile(const float2* __restrict__ in, float2* __restrict__ out,
                                         const float2* __restrict__ tw, int N, int M, int nlines) {
  const int q = threadIdx.x & 7, r = threadIdx.x >> 3;
  const int t0 = 4 * q;
  const int nM = N - M;   // -M mod N
  for (int b0 = 0; b0 < N; b0 += 32 * kRows) {
    int e[kRows], st[kRows];
    float2 acc[kRows][4];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int m = b0 + r + 32 * k - M;
      const int sm = ((m % N) + N) % N;
      st[k] = sm;
      e[k] = (sm * nM) % N;
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[k][j] = make_float2(0.f, 0.f);
    }
    if (t0 < nlines) {
      for (int a = 0; a < N; ++a) {
        const float2* row = in + a * (kTL + 1) + t0;
        const float2 v[4] = {row[0], row[1], row[2], row[3]};
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
          const float2 w = tw[e[k]];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[k][j].x = fmaf(v[j].x, w.x, fmaf(-v[j].y, w.y, acc[k][j].x));
            acc[k][j].y = fmaf(v[j].x, w.y, fmaf(v[j].y, w.x, acc[k][j].y));
          }
          e[k] += st[k];
          e[k] -= e[k] >= N ? N : 0;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
      const int b = b0 + r + 32 * k;
      if (b < N)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[b * (kTL + 1) + t0 + j] = acc[k][j];
    }
  }
}

// Tile geometry of one pass: 32 lines that are consecutive in the coalesced
// direction, and the global index of element a of tile line t.
template <int AXIS>
struct Tile {
  int N;
  int64_t base;   // first line's offset
  int nlines;     // valid lines in the tile
  __device__ __forceinline__ Tile(int N_, int tile) : N(N_) {
    if (AXIS == 0) {          // lines are rows (z, y); tile = 32 consecutive rows
      base = (int64_t)tile * kTL;
      nlines = (int)min((int64_t)kTL, (int64_t)N * N - base);
    } else {                  // lines along y (outer z) or z (outer y); tile = 32 consecutive x
      const int tiles_x = (N + kTL - 1) / kTL;
      const int outer = tile / tiles_x, x0 = (tile - outer * tiles_x) * kTL;
      base = (AXIS == 1 ? (int64_t)outer * N * N : (int64_t)outer * N) + x0;
      nlines = min(kTL, N - x0);
    }
  }
  // element a of line t
  __device__ __forceinline__ int64_t at(int a, int t) const {
    if (AXIS == 0) return (base + t) * N + a;
    if (AXIS == 1) return base + (int64_t)a * N + t;
    return base + (int64_t)a * N * N + t;
  }
};

// Index e of the staging loop over the N x 32 tile -> (a, t) with consecutive
// threads on consecutive global addresses.
template <int AXIS>
__device__ __forceinline__ void tile_coord(int e, int N, int& a, int& t) {
  if (AXIS == 0) {
    t = e / N;
    a = e - t * N;
  } else {
    a = e / kTL;
    t = e - a * kTL;
  }
}

template <int AXIS>
__device__ __forceinline__ int tiles_of(int N) {
  return AXIS == 0 ? (N * N + kTL - 1) / kTL : ((N + kTL - 1) / kTL) * N;
}

// One pass along AXIS with sign `sign`. AXIS 0 forward may read a real
// array; AXIS 0 inverse may end in an epilogue (XMode); AXIS 2 may be the
// forward / pointwise / inverse sandwich (ZMode).
template <int AXIS, int ZM, int XM>
__global__ void __launch_bounds__(kThreads) dft_pass_kernel(PassArgs p, float sign) {
  extern __shared__ float2 sm[];
  const int N = p.N, M = p.M;
  float2* T = sm;                         // input tile  [N][33]
  float2* O = sm + N * (kTL + 1);         // output tile [N][33]
  float2* W = O + N * (kTL + 1);          // twiddles with the pass's sign, then with the other
  float2* Wc = W + N;
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const float2 w = p.tw[i];
    W[i] = make_float2(w.x, sign * w.y);
    Wc[i] = make_float2(w.x, -sign * w.y);
  }
  double acc_num = 0.0, acc_den = 0.0;
  float vmax = 0.f;
  const int ntiles = tiles_of<AXIS>(N);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const Tile<AXIS> tl(N, tile);
    __syncthreads();
    for (int e = threadIdx.x; e < N * kTL; e += kThreads) {
      int a, tt;
      tile_coord<AXIS>(e, N, a, tt);
      float2 v = make_float2(0.f, 0.f);
      if (tt < tl.nlines) {
        const int64_t gi = tl.at(a, tt);
        if (AXIS == 0 && p.in_real) {
          const float r = p.in_real[gi];
          v = make_float2(p.in_abs ? fabsf(r) : r, 0.f);
        } else {
          v = p.cube[gi];
        }
      }
      T[a * (kTL + 1) + tt] = v;
    }
    __syncthreads();
    dft_tile(T, O, W, N, M, tl.nlines);
    __syncthreads();
    if constexpr (AXIS == 2 && ZM != kZForward) {
      // pointwise step on the forward transform of the 32 lines, then the
      // inverse transform back into T (not for amplitudes)
      for (int e = threadIdx.x; e < N * kTL; e += kThreads) {
        int a, tt;
        tile_coord<AXIS>(e, N, a, tt);
        if (tt >= tl.nlines) continue;
        float2& c = O[a * (kTL + 1) + tt];
        const int64_t gi = tl.at(a, tt);
        if (ZM == kZModulus) {
          const float am = p.amp[gi];
          if (am >= 0.f) {
            const float mag = sqrtf(c.x * c.x + c.y * c.y);
            const double d = (double)mag - (double)am;
            acc_num += d * d;
            acc_den += (double)am * (double)am;
            if (mag > 0.f) {
              const float f = am / mag;
              c = make_float2(c.x * f, c.y * f);
            } else {
              c = make_float2(am, 0.f);
            }
          }
        } else if (ZM == kZBlur) {
          // separable transfer function of the normalised Gaussian; the
          // line index along z is a, the y and x indices come from gi
          const int64_t r = gi % ((int64_t)N * N);
          const float f = p.g1[a] * p.g1[(int)(r / N)] * p.g1[(int)(r % N)];
          c = make_float2(c.x * f, c.y * f);
        } else if (ZM == kZAmplitude) {
          p.amp_out[gi] = sqrtf(fmaxf(c.x, 0.f));
        }
      }
      if constexpr (ZM != kZAmplitude) {
        __syncthreads();
        dft_tile(O, T, Wc, N, M, tl.nlines);
        __syncthreads();
        for (int e = threadIdx.x; e < N * kTL; e += kThreads) {
          int a, tt;
          tile_coord<AXIS>(e, N, a, tt);
          if (tt < tl.nlines) p.cube[tl.at(a, tt)] = T[a * (kTL + 1) + tt];
        }
      }
    } else {
    // store O
    for (int e = threadIdx.x; e < N * kTL; e += kThreads) {
      int a, tt;
      tile_coord<AXIS>(e, N, a, tt);
      if (tt >= tl.nlines) continue;
      const int64_t gi = tl.at(a, tt);
      const float2 c = O[a * (kTL + 1) + tt];
      if (AXIS == 0 && XM == kXUpdate) {
        // rho' = P_M rho where (support and, with positivity, P_M rho > 0);
        // elsewhere 0 (ER) or rho - beta P_M rho (HIO)
        const float pm = c.x * p.scale;
        const bool keep = p.support[gi] && (!p.positivity || pm > 0.f);
        const float old = p.rho[gi];
        p.rho[gi] = keep ? pm : (p.hio ? old - p.beta * pm : 0.f);
      } else if (AXIS == 0 && XM == kXReal) {
        const float v = c.x * p.scale;
        p.real_out[gi] = v;
        vmax = fmaxf(vmax, v);
      } else {
        p.cube[gi] = c;
      }
    }
    }
  }
  if (AXIS == 2 && ZM == kZModulus) {
    // the last block adds the per-block partials in block order
    __shared__ bool last;
    const double s0 = block_sum(acc_num), s1 = block_sum(acc_den);
    if (threadIdx.x == 0) {
      p.part[2 * blockIdx.x] = s0;
      p.part[2 * blockIdx.x + 1] = s1;
      __threadfence();
      last = atomicAdd(p.count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      double a = 0.0, b = 0.0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        a += __ldcg(p.part + 2 * i);
        b += __ldcg(p.part + 2 * i + 1);
      }
      a = block_sum(a);
      b = block_sum(b);
      if (threadIdx.x == 0) {
        p.sc[0] = a;
        p.sc[1] = b;
        *p.count = 0u;
      }
    }
  }
  if (AXIS == 0 && XM == kXReal) {
    // blur values are non-negative: their bit patterns order like the values
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0) atomicMax(p.maxbits, __float_as_uint(vmax));
  }
}

// errors[k] = sqrt(sc[0] / sc[1]) (0 when there is no data).
__global__ void fourier_error_kernel(const double* __restrict__ sc, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = sc[1] > 0.0 ? sqrt(sc[0] / sc[1]) : 0.0;
}

// g1[b] = sum_{d=-M..M} exp(-d^2 / (2 sigma^2)) cos(2 pi m_b d / N) / sum_d exp(...),
// m_b = b - M: the transfer function of the normalised 1D Gaussian (real,
// the kernel being even); the 3D transfer function is g1(mx) g1(my) g1(mz).
__global__ void gauss_transfer_kernel(int N, double sigma, float* __restrict__ g1) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= N) return;
  const int M = (N - 1) / 2, m = b - M;
  double num = 0.0, den = 0.0;
  for (int d = -M; d <= M; ++d) {
    const double w = exp(-(double)d * d / (2.0 * sigma * sigma));
    const int e = ((m * d) % N + N) % N;
    num += w * cospi(2.0 * e / N);
    den += w;
  }
  g1[b] = (float)(num / den);
}

// support = blur > threshold * max(blur).
__global__ void threshold_kernel(const float* __restrict__ blur, int64_t n, const unsigned* __restrict__ maxbits,
                                 float threshold, uint8_t* __restrict__ support) {
  const float cut = threshold * __uint_as_float(*maxbits);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    support[i] = blur[i] > cut ? 1 : 0;
}

size_t pass_smem(int N) { return (size_t)(2 * N * (kTL + 1) + 2 * N) * sizeof(float2); }

template <int AXIS, int ZM, int XM>
int pass(const spf_phaser* ph, const PassArgs& a, float sign, cudaStream_t s, const char* name) {
  const size_t smem = pass_smem(ph->N);
  SPF_CUDA(cudaFuncSetAttribute(dft_pass_kernel<AXIS, ZM, XM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  const int sms = device_sms();
  const int nt = AXIS == 0 ? (int)ceil_div((int64_t)ph->N * ph->N, kTL) : (int)ceil_div(ph->N, kTL) * ph->N;
  const int grid = std::min(nt, 2 * sms);
  // bytes: each line read once and written once (complex), plus the side arrays
  const double bytes = 16.0 * ph->n3 + ((AXIS == 2 && ZM == kZModulus) ? 4.0 * ph->n3 : 0.0);
  return launch(name, s, [&] { dft_pass_kernel<AXIS, ZM, XM><<<grid, kThreads, smem, s>>>(a, sign); }, bytes);
}

PassArgs base_args(const spf_phaser* ph) {
  PassArgs a{};
  a.N = ph->N;
  a.M = ph->M;
  a.cube = ph->cube;
  a.tw = ph->tw;
  a.amp = ph->amp;
  a.part = ph->part;
  a.count = ph->count;
  a.sc = ph->sc;
  a.rho = ph->rho;
  a.support = ph->support;
  a.maxbits = ph->maxbits;
  a.scale = 1.f;
  return a;
}

}  // namespace

int phase_iterate(spf_phaser* ph, int hio, int iters, float beta, int positivity, double* errors, cudaStream_t s) {
  PassArgs a = base_args(ph);
  a.beta = beta;
  a.hio = hio;
  a.positivity = positivity;
  a.scale = (float)(1.0 / (double)ph->n3);
  for (int k = 0; k < iters; ++k) {
    a.in_real = ph->rho;
    a.in_abs = 0;
    SPF_TRY((pass<0, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_x")));
    a.in_real = nullptr;
    SPF_TRY((pass<1, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_y")));
    SPF_TRY((pass<2, kZModulus, kXComplex>(ph, a, -1.f, s, "phase_modulus_z")));
    if (errors)
      SPF_TRY(launch("phase_error_kernel", s, [&] { fourier_error_kernel<<<1, 32, 0, s>>>(ph->sc, errors + k); }));
    SPF_TRY((pass<1, kZForward, kXComplex>(ph, a, +1.f, s, "phase_dft_y")));
    SPF_TRY((pass<0, kZForward, kXUpdate>(ph, a, +1.f, s, "phase_update_x")));
  }
  return SPF_OK;
}

int phase_shrinkwrap(spf_phaser* ph, float sigma, float threshold, cudaStream_t s) {
  SPF_TRY(launch("phase_gauss_kernel", s, [&] {
    gauss_transfer_kernel<<<(unsigned)ceil_div(ph->N, 128), 128, 0, s>>>(ph->N, (double)sigma, ph->g1);
  }));
  SPF_CUDA(cudaMemsetAsync(ph->maxbits, 0, sizeof(unsigned), s));
  PassArgs a = base_args(ph);
  a.g1 = ph->g1;
  a.in_real = ph->rho;
  a.in_abs = 1;
  SPF_TRY((pass<0, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_x")));
  a.in_real = nullptr;
  SPF_TRY((pass<1, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_y")));
  SPF_TRY((pass<2, kZBlur, kXComplex>(ph, a, -1.f, s, "phase_blur_z")));
  SPF_TRY((pass<1, kZForward, kXComplex>(ph, a, +1.f, s, "phase_dft_y")));
  a.real_out = ph->blur;
  a.scale = (float)(1.0 / (double)ph->n3);
  SPF_TRY((pass<0, kZForward, kXReal>(ph, a, +1.f, s, "phase_blur_x")));
  return launch("phase_threshold_kernel", s, [&] {
    threshold_kernel<<<(unsigned)std::min<int64_t>(ceil_div(ph->n3, 256), 4096), 256, 0, s>>>(
        ph->blur, ph->n3, ph->maxbits, threshold, ph->support);
  }, 5.0 * ph->n3);
}

int phase_amplitudes(spf_phaser* ph, const float* x, cudaStream_t s) {
  PassArgs a = base_args(ph);
  a.in_real = x;
  a.in_abs = 0;
  a.amp_out = ph->amp;
  SPF_TRY((pass<0, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_x")));
  a.in_real = nullptr;
  SPF_TRY((pass<1, kZForward, kXComplex>(ph, a, -1.f, s, "phase_dft_y")));
  return pass<2, kZAmplitude, kXComplex>(ph, a, -1.f, s, "phase_amplitude_z");
}

}  // namespace spf

using namespace spf;

namespace {
struct DevGuard {
  int prev = -1, rc = SPF_OK;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      set_error("cudaSetDevice(%d) failed", dev);
      rc = SPF_ERR_CUDA;
    }
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void phaser_free(spf_phaser* ph) {
  if (!ph) return;
  cudaFree(ph->cube);
  cudaFree(ph->rho);
  cudaFree(ph->amp);
  cudaFree(ph->support);
  cudaFree(ph->blur);
  cudaFree(ph->g1);
  cudaFree(ph->tw);
  cudaFree(ph->part);
  cudaFree(ph->count);
  cudaFree(ph->sc);
  cudaFree(ph->maxbits);
  delete ph;
}
}  // namespace

extern "C" {

int spf_phaser_create(spf_phaser** out, int N, int device) {
  clear_error();
  SPF_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  SPF_CHECK_ARG(N >= 3 && N <= kMaxN && N % 2 == 1, "N must be odd in 3..%d (got %d)", kMaxN, N);
  DevGuard dev(device);
  if (dev.rc != SPF_OK) return dev.rc;
  spf_phaser* ph = new spf_phaser();
  ph->device = device;
  ph->N = N;
  ph->M = (N - 1) / 2;
  ph->n3 = (int64_t)N * N * N;
  int rc = SPF_OK;
  auto A = [&](void** p, size_t b, const char* w) {
    if (rc == SPF_OK) rc = dev_alloc(p, b, w);
  };
  A((void**)&ph->cube, sizeof(float2) * ph->n3, "phasing cube");
  A((void**)&ph->rho, sizeof(float) * ph->n3, "phasing iterate");
  A((void**)&ph->amp, sizeof(float) * ph->n3, "phasing magnitudes");
  A((void**)&ph->support, ph->n3, "phasing support");
  A((void**)&ph->blur, sizeof(float) * ph->n3, "shrinkwrap blur");
  A((void**)&ph->g1, sizeof(float) * N, "shrinkwrap transfer");
  A((void**)&ph->tw, sizeof(float2) * N, "phasing twiddles");
  // per-block partial sums of the passes (at most 2 blocks per SM) and of
  // the reductions, with room to spare
  A((void**)&ph->part, sizeof(double) * 2 * 2 * (size_t)std::max(device_sms(), 152) * 8, "phasing partials");
  A((void**)&ph->count, sizeof(unsigned), "phasing counter");
  A((void**)&ph->sc, sizeof(double) * 2, "phasing scalars");
  A((void**)&ph->maxbits, sizeof(unsigned), "blur maximum");
  if (rc == SPF_OK) {
    std::vector<float2> tw(N);
    for (int j = 0; j < N; ++j) {
      const double ang = 2.0 * M_PI * (double)j / (double)N;
      tw[j] = make_float2((float)cos(ang), (float)sin(ang));
    }
    cudaError_t e = cudaMemcpy(ph->tw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ph->count, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(ph->amp, 0, sizeof(float) * ph->n3);
    if (e == cudaSuccess) e = cudaMemset(ph->support, 1, ph->n3);
    if (e == cudaSuccess) e = cudaMemset(ph->rho, 0, sizeof(float) * ph->n3);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("phaser set-up: %s", cudaGetErrorString(e));
      rc = SPF_ERR_CUDA;
    }
  }
  if (rc != SPF_OK) {
    phaser_free(ph);
    return rc;
  }
  *out = ph;
  return SPF_OK;
}

int spf_phaser_destroy(spf_phaser* ph) {
  clear_error();
  if (!ph) return SPF_OK;
  DevGuard dev(ph->device);
  cudaDeviceSynchronize();
  phaser_free(ph);
  return SPF_OK;
}

int spf_phaser_set_amplitudes(spf_phaser* ph, const float* amp, void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph && amp, "NULL pointer");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  SPF_CUDA(cudaMemcpyAsync(ph->amp, amp, sizeof(float) * ph->n3, cudaMemcpyDeviceToDevice, as_stream(stream)));
  return SPF_OK;
}

int spf_phaser_amplitudes_from_model(spf_phaser* ph, const float* x, void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph && x, "NULL pointer");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return phase_amplitudes(ph, x, as_stream(stream));
}

int spf_phaser_set_state(spf_phaser* ph, const float* rho, const uint8_t* support, void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph && (rho || support), "NULL pointer");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  if (rho) SPF_CUDA(cudaMemcpyAsync(ph->rho, rho, sizeof(float) * ph->n3, cudaMemcpyDeviceToDevice, s));
  if (support) SPF_CUDA(cudaMemcpyAsync(ph->support, support, ph->n3, cudaMemcpyDeviceToDevice, s));
  return SPF_OK;
}

int spf_phaser_iterate(spf_phaser* ph, int method, int iters, float beta, int positivity, double* errors,
                       void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph != nullptr, "phaser is NULL");
  SPF_CHECK_ARG(method == SPF_PHASE_ER || method == SPF_PHASE_HIO, "unknown phasing method %d", method);
  SPF_CHECK_ARG(iters >= 0, "iters must be >= 0");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return phase_iterate(ph, method == SPF_PHASE_HIO, iters, beta, positivity, errors, as_stream(stream));
}

int spf_phaser_shrinkwrap(spf_phaser* ph, float sigma, float threshold, void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph != nullptr, "phaser is NULL");
  SPF_CHECK_ARG(sigma > 0.f && threshold >= 0.f && threshold < 1.f, "sigma > 0 and 0 <= threshold < 1 required");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return phase_shrinkwrap(ph, sigma, threshold, as_stream(stream));
}

int spf_phaser_get(spf_phaser* ph, float* rho, uint8_t* support, float* amp, void* stream) {
  clear_error();
  SPF_CHECK_ARG(ph != nullptr, "phaser is NULL");
  DevGuard dev(ph->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  if (rho) SPF_CUDA(cudaMemcpyAsync(rho, ph->rho, sizeof(float) * ph->n3, cudaMemcpyDeviceToDevice, s));
  if (support) SPF_CUDA(cudaMemcpyAsync(support, ph->support, ph->n3, cudaMemcpyDeviceToDevice, s));
  if (amp) SPF_CUDA(cudaMemcpyAsync(amp, ph->amp, sizeof(float) * ph->n3, cudaMemcpyDeviceToDevice, s));
  return SPF_OK;
}

}  // extern "C"
