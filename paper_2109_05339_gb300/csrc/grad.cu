// Gradient-based merge (the differentiation pattern): the weighted slice
// loss, its gradient and a steepest-descent step with exact line search, with
// slices recomputed chunk by chunk instead of stored.
//
//   L(x) = 1/2 sum_{i,p} D_p (S_i x - b_scale img_ip)^2 + lambda/2 |x - x0|^2
//   grad = S^T D (S x - b) + lambda (x - x0)
//
// S_i x is the slice of model x at image i's orientation (type 2, Sec. II-A)
// and S^T the type-1 adjoint (Sec. II-C). For models even in n (real,
// Friedel-symmetric intensities) S^T D S = Re(A^H D A), so L is the Tikhonov
// objective of Eq. 2 that CG solves with the Toeplitz operator. L is
// quadratic: along -g the exact minimiser is x - (g.g / g.Hg) g with
// H = S^T D S + lambda I. Loss, inner products and step length are FP64 and
// stay on the device.
#include <algorithm>

#include "plan.h"
#include "reduce.h"

namespace spf {
int type2_setup(spf_plan* P, const float* A, cudaStream_t s, bool halo);
int type2_quat(spf_plan* P, const float* quats, int M, const float* qlab, int P2, float* out,
               cudaStream_t s);
int type1_quat(spf_plan* P, const float* g_vals, const float* quats, int M, const float* qlab,
               int P2, float* out, int accumulate, int* err, cudaStream_t s);

namespace {

constexpr int kBlocks = 296;   // fixed grid: deterministic FP64 reductions
constexpr int kThreads = 256;

// The last block of a launch adds the per-block partials (in block order)
// of `nv` sums: target[k] (+)= scale[k] * sum_b part[b * nv + k].
template <int NV>
__device__ void finish_sums(const double (&s_block)[NV], double* __restrict__ part, unsigned* __restrict__ count,
                            double* __restrict__ target, const double (&scale)[NV], bool accumulate) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) part[blockIdx.x * NV + k] = s_block[k];
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(part + i * NV + k);
    const double s = block_sum(v);
    if (threadIdx.x == 0) target[k] = (accumulate ? target[k] : 0.0) + scale[k] * s;
  }
  if (threadIdx.x == 0) *count = 0u;
}

// r = s - b_scale img (in place in s), loss (+)= 1/2 sum D r^2, then s = D r.
__global__ void __launch_bounds__(kThreads) residual_kernel(float* __restrict__ s, const float* __restrict__ img,
                                                            int64_t n, int P2, float b_scale,
                                                            const float* __restrict__ D, double* __restrict__ part,
                                                            unsigned* count, double* __restrict__ loss) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float r = s[i] - b_scale * __ldg(img + i);
    const float w = D ? __ldg(D + i % P2) : 1.f;
    acc += 0.5 * (double)w * (double)r * (double)r;
    s[i] = w * r;
  }
  const double sb[1] = {block_sum(acc)};
  const double one[1] = {1.0};
  finish_sums<1>(sb, part, count, loss, one, true);
}

// s = D s (the weights of the normal operator).
__global__ void weight_kernel(float* __restrict__ s, int64_t n, int P2, const float* __restrict__ D) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s[i] *= __ldg(D + i % P2);
}

// out += lambda (v - v0); with `loss`, loss += lambda/2 |v - v0|^2 (v0 NULL: 0).
__global__ void __launch_bounds__(kThreads) ridge_kernel(float* __restrict__ out, const float* __restrict__ v,
                                                         const float* __restrict__ v0, int64_t n, float lambda,
                                                         double* __restrict__ part, unsigned* count,
                                                         double* __restrict__ loss) {
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float d = v[i] - (v0 ? v0[i] : 0.f);
    out[i] += lambda * d;
    acc += (double)d * (double)d;
  }
  if (!loss) return;
  const double sb[1] = {block_sum(acc)};
  const double half_lam[1] = {0.5 * (double)lambda};
  finish_sums<1>(sb, part, count, loss, half_lam, true);
}

// sc[0] = g.g, sc[1] = g.Hg.
__global__ void __launch_bounds__(kThreads) dots_kernel(const float* __restrict__ g, const float* __restrict__ Hg,
                                                        int64_t n, double* __restrict__ part, unsigned* count,
                                                        double* __restrict__ sc) {
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double gv = g[i];
    a += gv * gv;
    b += gv * (double)Hg[i];
  }
  const double sb[2] = {block_sum(a), block_sum(b)};
  const double one[2] = {1.0, 1.0};
  finish_sums<2>(sb, part, count, sc, one, false);
}

// x -= (g.g / g.Hg) g; no step when g.Hg <= 0 or g = 0.
__global__ void step_kernel(float* __restrict__ x, const float* __restrict__ g, int64_t n,
                            const double* __restrict__ sc) {
  const double gg = sc[0], gHg = sc[1];
  const float t = (gHg > 0.0 && gg > 0.0) ? (float)(gg / gHg) : 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fmaf(-t, g[i], x[i]);
}

unsigned grid_of(int64_t n) { return (unsigned)std::min<int64_t>(ceil_div(n, kThreads), (int64_t)device_sms() * 16); }

// S^T D (S v - b) [loss and b when img is given] or S^T D S v, summed over
// image chunks into out (overwritten).
int normal_pass(spf_plan* P, const float* v, const float* quats, int n_img, const float* qlab, int P2,
                const float* img, float b_scale, const float* D, int chunk, float* work, double* loss,
                float* out, cudaStream_t s) {
  SPF_TRY(type2_setup(P, v, s, true));
  for (int c0 = 0; c0 < n_img; c0 += chunk) {
    const int m = std::min(chunk, n_img - c0);
    const int64_t n = (int64_t)m * P2;
    const float* q = quats + 4 * (size_t)c0;
    SPF_TRY(type2_quat(P, q, m, qlab, P2, work, s));
    if (img) {
      const float* b = img + (size_t)c0 * P2;
      SPF_TRY(launch("residual_kernel", s, [&] {
        residual_kernel<<<kBlocks, kThreads, 0, s>>>(work, b, n, P2, b_scale, D, P->grad_part, P->grad_count, loss);
      }, 16.0 * n));
    } else if (D) {
      SPF_TRY(launch("weight_kernel", s, [&] { weight_kernel<<<grid_of(n), kThreads, 0, s>>>(work, n, P2, D); },
                     8.0 * n));
    }
    SPF_TRY(type1_quat(P, work, q, m, qlab, P2, out, c0 > 0 ? 1 : 0, P->err, s));
  }
  if (n_img == 0) SPF_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)P->N * P->N * P->N, s));
  return SPF_OK;
}

}  // namespace

int grad_alloc(spf_plan* P) {
  SPF_TRY(dev_alloc((void**)&P->grad_part, sizeof(double) * 2 * kBlocks, "gradient partials"));
  SPF_TRY(dev_alloc((void**)&P->grad_count, sizeof(unsigned), "gradient reduction counter"));
  SPF_TRY(dev_alloc((void**)&P->grad_sc, sizeof(double) * 4, "gradient scalars"));
  SPF_CUDA(cudaMemset(P->grad_count, 0, sizeof(unsigned)));
  SPF_CUDA(cudaMemset(P->grad_sc, 0, sizeof(double) * 4));
  return SPF_OK;
}

int slice_loss_grad(spf_plan* P, const float* x, const float* x0, const float* quats, int n_img, const float* qlab,
                    int P2, const float* img, float b_scale, const float* D, double lambda, int chunk, float* work,
                    double* loss, float* grad, cudaStream_t s) {
  const int64_t n3 = (int64_t)P->N * P->N * P->N;
  SPF_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
  SPF_TRY(normal_pass(P, x, quats, n_img, qlab, P2, img, b_scale, D, chunk, work, loss, grad, s));
  if (lambda != 0.0) {
    SPF_TRY(launch("ridge_kernel", s, [&] {
      ridge_kernel<<<kBlocks, kThreads, 0, s>>>(grad, x, x0, n3, (float)lambda, P->grad_part, P->grad_count, loss);
    }, 16.0 * n3));
  }
  return SPF_OK;
}

int slice_normal_apply(spf_plan* P, const float* v, const float* quats, int n_img, const float* qlab, int P2,
                       const float* D, double lambda, int chunk, float* work, float* out, cudaStream_t s) {
  const int64_t n3 = (int64_t)P->N * P->N * P->N;
  SPF_TRY(normal_pass(P, v, quats, n_img, qlab, P2, nullptr, 1.f, D, chunk, work, nullptr, out, s));
  if (lambda != 0.0) {
    SPF_TRY(launch("ridge_kernel", s, [&] {
      ridge_kernel<<<kBlocks, kThreads, 0, s>>>(out, v, nullptr, n3, (float)lambda, nullptr, nullptr, nullptr);
    }, 12.0 * n3));
  }
  return SPF_OK;
}

int gradient_step(spf_plan* P, float* x, const float* x0, const float* quats, int n_img, const float* qlab, int P2,
                  const float* img, float b_scale, const float* D, double lambda, int chunk, float* work,
                  float* grad, float* Hg, double* loss, cudaStream_t s) {
  const int64_t n3 = (int64_t)P->N * P->N * P->N;
  SPF_TRY(slice_loss_grad(P, x, x0, quats, n_img, qlab, P2, img, b_scale, D, lambda, chunk, work, loss, grad, s));
  SPF_TRY(slice_normal_apply(P, grad, quats, n_img, qlab, P2, D, lambda, chunk, work, Hg, s));
  SPF_TRY(launch("dots_kernel", s, [&] {
    dots_kernel<<<kBlocks, kThreads, 0, s>>>(grad, Hg, n3, P->grad_part, P->grad_count, P->grad_sc);
  }, 8.0 * n3));
  return launch("step_kernel", s, [&] { step_kernel<<<grid_of(n3), kThreads, 0, s>>>(x, grad, n3, P->grad_sc); },
                12.0 * n3);
}

}  // namespace spf
