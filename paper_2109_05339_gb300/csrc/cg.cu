// Toeplitz normal operator and conjugate gradient (Sec. II-C, Eq. 2).
//
// H x = crop(IFFT(K^ * FFT(pad x))) / P_T^3 + lambda x, with K^ the FFT of
// the circulant embedding of the "type-1 with ones" kernel (real and even).
// On the precompiled cube sides the convolution is real-input: the rows of
// x are transformed in pairs along x to half spectra, the y and z passes run
// on the half spectrum with the product by K^ inside the z pass (forward,
// multiply, inverse in one launch), and paired rows come back real. Other
// sides transform the padded cube as complex data with the product fused
// into the x pass. Either way lines that stay zero are skipped on the way in
// and lines that cannot reach the cropped N^3 output on the way out. Inner
// products and residual norms are
// accumulated in FP64 (per-block partials reduced in a fixed order, so the
// result is deterministic); alpha and beta are computed on the device and
// never read by the host.
#include <algorithm>
#include <cmath>

#include "plan.h"
#include "reduce.h"

namespace spf {

namespace {

constexpr int kRedBlocks = 296;   // fixed grid for deterministic reductions
constexpr int kRedThreads = 256;

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// cube (PT^3 complex) = x at n mod PT (|n| <= Mh), zero elsewhere.
// x (N^3) into the circulant-embedding cube at n mod PT. Only those N^3
// entries are written: the pruned forward FFT reads nothing else.
__global__ void pad_kernel(const float* __restrict__ x, int N, int PT, float2* __restrict__ cube) {
  int64_t total = (int64_t)N * N * N;
  int Mh = (N - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(i % N), b = (int)((i / N) % N), c = (int)(i / ((int64_t)N * N));
    int gx = wrapi(a - Mh, PT), gy = wrapi(b - Mh, PT), gz = wrapi(c - Mh, PT);
    cube[((size_t)gz * PT + gy) * PT + gx] = make_float2(x[i], 0.f);
  }
}

// out = Re(cube[n mod PT]) / PT^3 + lambda x; partial sums of x . out
// (finalised in the kernel, mode 1, when `count` is given).
__global__ void crop_apply_kernel(const float2* __restrict__ cube, int N, int PT, float inv_n,
                                  float lambda, const float* __restrict__ x, float* __restrict__ out,
                                  double* __restrict__ part, double* __restrict__ sc, unsigned* count) {
  int64_t n3 = (int64_t)N * N * N;
  int Mh = (N - 1) / 2;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(i % N), b = (int)((i / N) % N), c = (int)(i / ((int64_t)N * N));
    int gx = wrapi(a - Mh, PT), gy = wrapi(b - Mh, PT), gz = wrapi(c - Mh, PT);
    float v = cube[((size_t)gz * PT + gy) * PT + gx].x * inv_n + lambda * x[i];
    out[i] = v;
    acc += (double)x[i] * (double)v;
  }
  double s = block_sum(acc);
  if (count) partial_and_finalize(s, part, sc, 1, nullptr, count);
  else if (threadIdx.x == 0 && part) part[blockIdx.x] = s;
}

// x = x0; r = rhs + lambda x0 - Hx0; p = r; partial |r|^2.
__global__ void cg_init_kernel(const float* __restrict__ rhs, const float* __restrict__ x0,
                               const float* __restrict__ Hx0, float lambda, int64_t n,
                               float* __restrict__ x, float* __restrict__ r, float* __restrict__ p,
                               double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float xv = x0[i];
    float rv = rhs[i] + lambda * xv - Hx0[i];
    x[i] = xv;
    r[i] = rv;
    p[i] = rv;
    acc += (double)rv * (double)rv;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// sc = [rr, pAp, alpha, beta, rr_new, res]
// mode 0: rr = sum; mode 1: pAp = sum, alpha = rr / pAp;
// mode 2: rr_new = sum, beta = rr_new / rr, rr = rr_new. res = sqrt(rr).
__global__ void finalize_kernel(const double* __restrict__ part, int nparts, double* __restrict__ sc,
                                int mode, double* __restrict__ res_out) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += part[i];
  double s = block_sum(v);
  if (threadIdx.x == 0) cg_scalars(s, sc, mode, res_out);
}


// x += alpha p; r -= alpha Ap; partial |r|^2.
__global__ void cg_update_kernel(float* __restrict__ x, float* __restrict__ r,
                                 const float* __restrict__ p, const float* __restrict__ Ap,
                                 double* __restrict__ sc, int64_t n, double* __restrict__ part,
                                 double* __restrict__ res_out, unsigned* count) {
  const float alpha = (float)sc[2];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fmaf(alpha, p[i], x[i]);
    float rv = fmaf(-alpha, Ap[i], r[i]);
    r[i] = rv;
    acc += (double)rv * (double)rv;
  }
  partial_and_finalize(block_sum(acc), part, sc, 2, res_out, count);
}

// p = r + beta p (beta from the last step; 0 after cg_begin), and p into the
// circulant-embedding cube at n mod PT (as pad_kernel).
__global__ void pad_dir_kernel(const float* __restrict__ r, float* __restrict__ p,
                               const double* __restrict__ sc, int N, int PT, float2* __restrict__ cube) {
  const float beta = (float)sc[3];
  const int64_t total = (int64_t)N * N * N;
  const int Mh = (N - 1) / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float pv = fmaf(beta, p[i], r[i]);
    p[i] = pv;
    const int a = (int)(i % N), b = (int)((i / N) % N), c = (int)(i / ((int64_t)N * N));
    const int gx = wrapi(a - Mh, PT), gy = wrapi(b - Mh, PT), gz = wrapi(c - Mh, PT);
    cube[((size_t)gz * PT + gy) * PT + gx] = make_float2(pv, 0.f);
  }
}


// Per-block partials of x.Tx, x.rhs and |x - x0|^2 (FP64).
__global__ void objective_kernel(const float* __restrict__ x, const float* __restrict__ Tx,
                                 const float* __restrict__ rhs, const float* __restrict__ x0, int64_t n,
                                 double* __restrict__ part) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double xv = x[i];
    a += xv * (double)Tx[i];
    b += xv * (double)rhs[i];
    const double d = xv - (double)x0[i];
    c += d * d;
  }
  a = block_sum(a);
  b = block_sum(b);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
  }
}

// out[0] = xTx - 2 x.rhs + b2[0], out[1] = |x - x0|^2.
__global__ void objective_finalize_kernel(const double* __restrict__ part, int nparts,
                                          const double* __restrict__ b2, double* __restrict__ out) {
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    a += part[3 * i];
    b += part[3 * i + 1];
    c += part[3 * i + 2];
  }
  a = block_sum(a);
  b = block_sum(b);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    out[0] = a - 2.0 * b + (b2 ? b2[0] : 0.0);
    out[1] = c;
  }
}

// out (+)= sum_{i,p} D[p] (scale img[i,p])^2, FP64, per-block partials then one block.
__global__ void wsumsq_kernel(const float* __restrict__ img, int64_t n, int P2, const float* __restrict__ D,
                              float scale, double* __restrict__ part) {
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)scale * (double)img[i];
    a += (D ? (double)D[i % P2] : 1.0) * v * v;
  }
  a = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void wsumsq_finalize_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out,
                                       int accumulate) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += part[i];
  a = block_sum(a);
  if (threadIdx.x == 0) out[0] = accumulate ? out[0] + a : a;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(ceil_div(n, 256), (int64_t)device_sms() * 32); }

}  // namespace

// out = H x, and (optionally) per-block partials of x . out.
int toeplitz_apply(spf_plan* P, const float* khat, double lambda, const float* x, float* out,
                   double* part, cudaStream_t s) {
  const int N = P->N, PT = P->PT;
  int64_t PT3 = (int64_t)PT * PT * PT;
  if (fft3_real_supported(&P->fftP)) {
    RealConvEpilogue ep;
    ep.scale = (float)(1.0 / (double)PT3);
    ep.lambda = (float)lambda;
    ep.xin = x;
    ep.part = part;
    return fft3_convolve_real(&P->fftP, N, x, nullptr, nullptr, nullptr, khat, P->cubeP, out, ep, s);
  }
  const double n3 = (double)N * N * N;
  SPF_TRY(launch("pad_kernel", s, [&] { pad_kernel<<<grid_for((int64_t)N * N * N), 256, 0, s>>>(x, N, PT, P->cubeP); },
                 12.0 * n3));
  SPF_TRY(fft3_convolve(&P->fftP, P->cubeP, khat, P->Mh + 1, P->Mh + 1, s));
  SPF_TRY(launch("crop_apply_kernel", s, [&] { crop_apply_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(P->cubeP, N, PT, (float)(1.0 / (double)PT3),
                                                       (float)lambda, x, out, part, nullptr, nullptr); },
                 16.0 * n3));
  return SPF_OK;
}

int cg_begin(spf_plan* P, const float* khat, double lambda, const float* rhs, const float* x0,
             float* x, double* res, cudaStream_t s) {
  int64_t n3 = (int64_t)P->N * P->N * P->N;
  SPF_TRY(toeplitz_apply(P, khat, lambda, x0, P->cg_Ap, nullptr, s));
  SPF_TRY(launch("cg_init_kernel", s, [&] { cg_init_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(rhs, x0, P->cg_Ap, (float)lambda, n3, x,
                                                    P->cg_r, P->cg_p, P->cg_part); }, 24.0 * n3));
  SPF_TRY(launch("finalize_kernel", s, [&] { finalize_kernel<<<1, kRedThreads, 0, s>>>(P->cg_part, kRedBlocks, P->cg_sc, 0, res); }));
  return SPF_OK;
}

int cg_step(spf_plan* P, const float* khat, double lambda, float* x, double* res, cudaStream_t s) {
  // p = r + beta p is applied while padding p (beta of the previous step, 0
  // after cg_begin); both inner products are finalised inside their kernels
  const int N = P->N, PT = P->PT;
  const int64_t n3 = (int64_t)N * N * N, PT3 = (int64_t)PT * PT * PT;
  if (fft3_real_supported(&P->fftP)) {
    // real-input transforms: the direction update rides on the first pass,
    // Ap = Hp + lambda p and p.Ap (finalised: alpha) on the last
    RealConvEpilogue ep;
    ep.scale = (float)(1.0 / (double)PT3);
    ep.lambda = (float)lambda;
    ep.xin = P->cg_p;
    ep.part = P->cg_part;
    ep.sc = P->cg_sc;
    ep.count = P->cg_count;
    SPF_TRY(fft3_convolve_real(&P->fftP, N, P->cg_p, P->cg_r, P->cg_sc + 3, P->cg_p, khat, P->cubeP, P->cg_Ap, ep,
                               s));
  } else {
    SPF_TRY(launch("pad_kernel", s, [&] { pad_dir_kernel<<<grid_for(n3), 256, 0, s>>>(P->cg_r, P->cg_p, P->cg_sc, N, PT, P->cubeP); },
                   20.0 * n3));
    SPF_TRY(fft3_convolve(&P->fftP, P->cubeP, khat, P->Mh + 1, P->Mh + 1, s));
    SPF_TRY(launch("crop_apply_kernel", s, [&] {
      crop_apply_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(P->cubeP, N, PT, (float)(1.0 / (double)PT3), (float)lambda,
                                                           P->cg_p, P->cg_Ap, P->cg_part, P->cg_sc, P->cg_count);
    }, 16.0 * n3));
  }
  return launch("cg_update_kernel", s, [&] {
    cg_update_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(x, P->cg_r, P->cg_p, P->cg_Ap, P->cg_sc, n3, P->cg_part,
                                                        res, P->cg_count);
  }, 24.0 * n3);
}

int cg_alloc(spf_plan* P) {
  size_t n3 = (size_t)P->N * P->N * P->N;
  SPF_TRY(dev_alloc((void**)&P->cg_r, sizeof(float) * n3, "cg r"));
  SPF_TRY(dev_alloc((void**)&P->cg_p, sizeof(float) * n3, "cg p"));
  SPF_TRY(dev_alloc((void**)&P->cg_Ap, sizeof(float) * n3, "cg Ap"));
  SPF_TRY(dev_alloc((void**)&P->cg_sc, sizeof(double) * 8, "cg scalars"));
  // partials of the reduction kernels and of the convolution's last launch
  const int nparts = std::max(kRedBlocks, fft3_real_conv_blocks(&P->fftP, P->N));
  SPF_TRY(dev_alloc((void**)&P->cg_part, sizeof(double) * nparts, "cg partials"));
  SPF_TRY(dev_alloc((void**)&P->cg_count, sizeof(unsigned), "cg reduction counter"));
  SPF_CUDA(cudaMemset(P->cg_sc, 0, sizeof(double) * 8));
  SPF_CUDA(cudaMemset(P->cg_count, 0, sizeof(unsigned)));
  return SPF_OK;
}

}  // namespace spf

namespace spf {
int cg_objective(spf_plan* P, const float* khat, const float* rhs, const float* x, const float* x0,
                 const double* b2, double* out, cudaStream_t s) {
  const int64_t n3 = (int64_t)P->N * P->N * P->N;
  SPF_TRY(toeplitz_apply(P, khat, 0.0, x, P->cg_Ap, nullptr, s));
  SPF_TRY(launch("objective_kernel", s, [&] {
    objective_kernel<<<kRedBlocks / 3, kRedThreads, 0, s>>>(x, P->cg_Ap, rhs, x0, n3, P->cg_part);
  }));
  return launch("objective_finalize_kernel", s, [&] {
    objective_finalize_kernel<<<1, kRedThreads, 0, s>>>(P->cg_part, kRedBlocks / 3, b2, out);
  });
}

int weighted_sumsq(spf_plan* P, const float* img, int64_t n, int P2, const float* D, float scale,
                   double* out, int accumulate, cudaStream_t s) {
  SPF_TRY(launch("wsumsq_kernel", s, [&] {
    wsumsq_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(img, n, P2, D, scale, P->cg_part);
  }));
  return launch("wsumsq_finalize_kernel", s, [&] {
    wsumsq_finalize_kernel<<<1, kRedThreads, 0, s>>>(P->cg_part, kRedBlocks, out, accumulate);
  });
}
}  // namespace spf

// ------------------------------------------------------------ L-curve ----
// Corner of the L-curve (Sec. II-C: the regularisation parameter is chosen on
// the L-curve): with s = log lambda, rho = log |A x - b|_D and eta =
// log |x - x0| (half the logs of the squared norms), the curvature of
// (rho(s), eta(s)) is kappa = (rho' eta'' - rho'' eta') / (rho'^2 + eta'^2)^(3/2),
// derivatives by three-point finite differences on the uneven grid s, at the
// interior points. Host arithmetic on the n scalars of a sweep.
extern "C" int spf_lcurve_corner(const double* lams, const double* res2, const double* reg2, int n, int* index,
                                 double* kappa) {
  using namespace spf;
  clear_error();
  SPF_CHECK_ARG(n >= 3 && lams && res2 && reg2 && index, "need n >= 3 points and non-NULL arrays");
  for (int i = 0; i < n; ++i) {
    SPF_CHECK_ARG(lams[i] > 0.0 && res2[i] > 0.0 && reg2[i] > 0.0, "lambda and both norms must be positive");
    SPF_CHECK_ARG(i == 0 || lams[i] > lams[i - 1], "lambdas must increase");
  }
  int best = -1;
  double kbest = 0.0;
  for (int i = 1; i + 1 < n; ++i) {
    const double s0 = std::log(lams[i - 1]), s1 = std::log(lams[i]), s2 = std::log(lams[i + 1]);
    const double h0 = s1 - s0, h1 = s2 - s1;
    auto d1 = [&](double y0, double y1, double y2) {
      return -h1 / (h0 * (h0 + h1)) * y0 + (h1 - h0) / (h0 * h1) * y1 + h0 / (h1 * (h0 + h1)) * y2;
    };
    auto d2 = [&](double y0, double y1, double y2) {
      return 2.0 * (y0 / (h0 * (h0 + h1)) - y1 / (h0 * h1) + y2 / (h1 * (h0 + h1)));
    };
    const double r0 = 0.5 * std::log(res2[i - 1]), r1 = 0.5 * std::log(res2[i]), r2 = 0.5 * std::log(res2[i + 1]);
    const double e0 = 0.5 * std::log(reg2[i - 1]), e1 = 0.5 * std::log(reg2[i]), e2 = 0.5 * std::log(reg2[i + 1]);
    const double rp = d1(r0, r1, r2), rpp = d2(r0, r1, r2), ep = d1(e0, e1, e2), epp = d2(e0, e1, e2);
    const double k = (rp * epp - rpp * ep) / std::pow(rp * rp + ep * ep, 1.5);
    if (kappa) kappa[i - 1] = k;
    if (best < 0 || k > kbest) {
      best = i;
      kbest = k;
    }
  }
  *index = best;
  return SPF_OK;
}

