// Internal helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstdio>
#include <string>

#include "../../include/spf.h"

namespace spf {

// Thread-local message of the last failing C-ABI call.
void set_error(const char* fmt, ...);
void clear_error();

struct Status {
  int code = SPF_OK;
};

#define SPF_CHECK_ARG(cond, ...)          \
  do {                                    \
    if (!(cond)) {                        \
      ::spf::set_error(__VA_ARGS__);      \
      return SPF_ERR_ARG;                 \
    }                                     \
  } while (0)

#define SPF_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      ::spf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      return SPF_ERR_CUDA;                                                              \
    }                                                                                   \
  } while (0)

#define SPF_LAUNCH_CHECK()                                                               \
  do {                                                                                   \
    cudaError_t e_ = cudaGetLastError();                                                 \
    if (e_ != cudaSuccess) {                                                             \
      ::spf::set_error("%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_));  \
      return SPF_ERR_CUDA;                                                               \
    }                                                                                    \
  } while (0)

#define SPF_TRY(expr)          \
  do {                         \
    int s_ = (expr);           \
    if (s_ != SPF_OK) return s_; \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Streaming multiprocessors of the current device (queried once per device;
// 152 if the query fails), for sizing grid-stride launches.
inline int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int n = 0;
    cache[dev] = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0 ? n : 152;
  }
  return cache[dev];
}

// Launch tracing (profile.cu): every kernel launch goes through launch(),
// which counts it and, while profiling is on, brackets it with CUDA events
// on its stream and adds `bytes` -- the algorithmic global-memory bytes the
// launch must move (each input element read once, each output written once;
// 0 where not stated) -- to the kernel's total.
extern std::atomic<long long> g_launches;
bool prof_on();
int prof_begin(const char* name, cudaStream_t s, double bytes);
void prof_end(int slot, cudaStream_t s);

template <class F>
inline int launch(const char* name, cudaStream_t s, F&& f, double bytes = 0.0) {
  int slot = prof_on() ? prof_begin(name, s, bytes) : -1;
  f();
  cudaError_t e = cudaGetLastError();
  if (slot >= 0) prof_end(slot, s);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (e != cudaSuccess) {
    set_error("launch of %s: %s", name, cudaGetErrorString(e));
    return SPF_ERR_CUDA;
  }
  return SPF_OK;
}

// Device allocation with OOM reporting.
int dev_alloc(void** p, size_t bytes, const char* what);

// ------------------------------------------------------------------ FFT ----
// Batched complex 3D FFT on an n2 x n1 x n0 cube (x = n0 fastest), written
// for 2/3/5-smooth sides. sign = -1: sum x exp(-2 pi i k l / n) (forward);
// sign = +1: exp(+...) without normalisation.
struct FFTAxisPlan {
  int n = 0;
  int nrad = 0;
  int radix[16];
  float2* twiddle = nullptr;  // n entries exp(-2 pi i k / n), device
};

struct FFT3 {
  int n0 = 0, n1 = 0, n2 = 0;
  FFTAxisPlan ax[3];
};

int fft3_create(FFT3* p, int n0, int n1, int n2);
void fft3_destroy(FFT3* p);
// In-place complex 3D transform of `data` (n2*n1*n0 float2).
// zero_halfwidth_in h > 0: the input is zero outside the wrapped index range
// {0..h-1} U {n-h+1..n-1} on every axis (a zero-padded mode cube); lines that
// are known to stay zero are skipped (axis order z, y, x).
// needed_halfwidth_out h > 0: only outputs inside that wrapped range on every
// axis are needed (a cropped mode cube); lines that cannot reach them are
// skipped (axis order x, y, z). Outside, the cube holds partial results.
int fft3_exec(const FFT3* p, float2* data, int sign, int zero_halfwidth_in,
              int needed_halfwidth_out, cudaStream_t s);
// As fft3_exec, plus: in_real (optional) -- the first pass reads this real
// cube instead of `data` (not with zero_halfwidth_in > 0); out_real
// (optional) -- the last pass writes only the real part there; post_mul
// (optional) -- the last pass multiplies every output by this real cube.
// With zero_halfwidth_in > 0 the input outside its range is never read.
int fft3_exec_ex(const FFT3* p, float2* data, const float* in_real, float* out_real,
                 const float* post_mul, int sign, int zero_halfwidth_in,
                 int needed_halfwidth_out, cudaStream_t s);
// IFFT(kernel * FFT(data)) in place (no 1/n^3 factor; forward sign -1), the
// input zero outside the half width zero_halfwidth_in range (never read) and
// outputs needed inside needed_halfwidth_out.
int fft3_convolve(const FFT3* p, float2* data, const float* kernel, int zero_halfwidth_in,
                  int needed_halfwidth_out, cudaStream_t s);
// Real-input circular convolution: the real vector x (Nm^3, Nm odd,
// 2 Nm - 1 <= side) embedded at wrapped positions of the cube (model index a
// -> (a - (Nm - 1) / 2) mod side), IFFT(kernel * FFT(embed x)) read back at
// the same positions (forward sign -1, no 1/n^3 factor) and passed through
// the epilogue ep into y. kernel is a real cube in the full layout and must
// be real and even. With `add` given the transformed vector is
// add + (*beta) x, also stored to x_new. work holds side^2 (side / 2 + 1)
// complex values. Only for the cube sides that fft3_real_supported accepts.
bool fft3_real_supported(const FFT3* p);
// Last step of fft3_convolve_real: y = scale * conv + lambda * xin at the
// model indices; with `part`, FP64 per-block partial sums of xin . y (xin
// required; part holds fft3_real_conv_blocks entries), and with `count` too
// the last block adds them in block order and updates the CG scalars sc
// (p.Ap and alpha).
struct RealConvEpilogue {
  float scale = 1.f, lambda = 0.f;
  const float* xin = nullptr;
  double* part = nullptr;
  double* sc = nullptr;
  unsigned* count = nullptr;
};
int fft3_real_conv_blocks(const FFT3* p, int Nm);
// Modes |k| < h (every axis) of the transform (sign `sign`) of the real cube
// `in` (side^3): out[side][side][h] holds the columns kx = 0 .. h-1 at
// wrapped ky, kz (only ky in the wrapped range of half width h are final);
// kx < 0 follows from F(-k) = conj F(k). Sides as fft3_real_supported.
int fft3_r2c_modes(const FFT3* p, const float* in, int h, int sign, float2* out, cudaStream_t s);
int fft3_convolve_real(const FFT3* p, int Nm, const float* x, const float* add, const double* beta,
                       float* x_new, const float* kernel, float2* work, float* y, const RealConvEpilogue& ep,
                       cudaStream_t s);

}  // namespace spf
