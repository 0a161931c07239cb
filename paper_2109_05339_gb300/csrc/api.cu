// C ABI of the library: argument checks, plan and matcher lifetimes, and the
// orchestration of the kernels of nufft.cu, cg.cu, match.cu and match_tc.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "match.h"
#include "plan.h"

namespace spf {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

void clear_error() { g_err.clear(); }

int dev_alloc(void** p, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
    return SPF_ERR_OOM;
  }
  return SPF_OK;
}

// Makes `dev` current for the scope and restores the caller's device after.
struct DeviceScope {
  int prev = -1;
  int rc = SPF_OK;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) {
      cudaError_t e = cudaSetDevice(dev);
      if (e != cudaSuccess) {
        set_error("cudaSetDevice(%d): %s", dev, cudaGetErrorString(e));
        rc = SPF_ERR_CUDA;
      }
    }
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// nufft.cu
int type2_setup(spf_plan* P, const float* A, cudaStream_t s, bool halo = true);
int type2_quat(spf_plan* P, const float* quats, int M, const float* qlab, int P2, float* out,
               cudaStream_t s);
int type2_explicit(spf_plan* P, const float* t, int64_t npts, float* out, cudaStream_t s);
int type1_quat(spf_plan* P, const float* g, const float* quats, int M, const float* qlab, int P2,
               float* out, int accumulate, int* err, cudaStream_t s);
int type1_explicit(spf_plan* P, const float* v, const float* t, int64_t npts, float* out,
                   int accumulate, int* err, cudaStream_t s);
int merge_run(spf_plan* P, const float* images, const float* quats, int n_quats,
              const int* oidx, int n_img, const float* qlab, int P2, const float* D, float b_scale,
              float* rhs, float* kernel_hat, int accumulate, int* err, cudaStream_t s, int mode,
              bool want_rhs, bool want_kernel);
int merge_begin(spf_plan* P, cudaStream_t s);
int merge_finish(spf_plan* P, float* rhs, float* kernel_hat, int accumulate, cudaStream_t s);
int grid_init(Grid* g, int n_modes, int nf, double cells_per_q, int w, double beta,
              int64_t max_points, bool interp_source);
int points_build(spf_plan* P, spf_points* S, cudaStream_t s);
int slice_points(spf_plan* P, spf_points* S, const float* A, float* out, cudaStream_t s);
int merge_points(spf_plan* P, spf_points* S, const float* images, const int* oidx, int n_img, int off,
                 const float* D, float b_scale, float* rhs, float* kernel_hat, int accumulate,
                 cudaStream_t s, int mode, bool want_rhs, bool want_kernel);
void grid_free(Grid* g);
// cg.cu
int toeplitz_apply(spf_plan* P, const float* khat, double lambda, const float* x, float* out,
                   double* part, cudaStream_t s);
int cg_begin(spf_plan* P, const float* khat, double lambda, const float* rhs, const float* x0,
             float* x, double* res, cudaStream_t s);
int cg_step(spf_plan* P, const float* khat, double lambda, float* x, double* res, cudaStream_t s);
int cg_alloc(spf_plan* P);
// grad.cu
int grad_alloc(spf_plan* P);
int slice_loss_grad(spf_plan* P, const float* x, const float* x0, const float* quats, int n_img, const float* qlab,
                    int P2, const float* img, float b_scale, const float* D, double lambda, int chunk, float* work,
                    double* loss, float* grad, cudaStream_t s);
int slice_normal_apply(spf_plan* P, const float* v, const float* quats, int n_img, const float* qlab, int P2,
                       const float* D, double lambda, int chunk, float* work, float* out, cudaStream_t s);
int gradient_step(spf_plan* P, float* x, const float* x0, const float* quats, int n_img, const float* qlab, int P2,
                  const float* img, float b_scale, const float* D, double lambda, int chunk, float* work,
                  float* grad, float* Hg, double* loss, cudaStream_t s);
int cg_objective(spf_plan* P, const float* khat, const float* rhs, const float* x, const float* x0,
                 const double* b2, double* out, cudaStream_t s);
int weighted_sumsq(spf_plan* P, const float* img, int64_t n, int P2, const float* D, float scale,
                   double* out, int accumulate, cudaStream_t s);
// match.cu / match_tc.cu
int simt_splits(int n_img, int n_orient, int n_sms);
int simt_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                cudaStream_t s);
int row_norms(const float* src, int rows, int P2, float scale, float* out, cudaStream_t s);
int row_norms_w(const float* src, int rows, int P2, float scale, const float* w, float* out,
                cudaStream_t s);
int set_mask_weights(spf_matcher* m, const float* D, cudaStream_t s);
int state_reset(spf_matcher* m, cudaStream_t s);
int rerank_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                  cudaStream_t s);
int results_launch(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                   int32_t* topk_idx, float* topk_d, cudaStream_t s);
int quantize_rows(spf_matcher* m, const float* src, int rows, float scale, void* dst, float* scales,
                  float* norms, cudaStream_t s);
int quantize_rows_u16(spf_matcher* m, const uint16_t* src, int rows, float scale, void* dst, float* scales,
                      float* norms, cudaStream_t s);
int tc_kpad(int P2, int precision);

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static void plan_free(spf_plan* P) {
  if (!P) return;
  grid_free(&P->g);
  grid_free(&P->gT);
  cudaFree(P->cubeP);
  cudaFree(P->realP);
  fft3_destroy(&P->fftP);
  cudaFree(P->sorted);
  cudaFree(P->cg_r);
  cudaFree(P->cg_p);
  cudaFree(P->cg_Ap);
  cudaFree(P->cg_sc);
  cudaFree(P->cg_part);
  cudaFree(P->cg_count);
  cudaFree(P->grad_part);
  cudaFree(P->grad_count);
  cudaFree(P->grad_sc);
  cudaFree(P->err);
  delete P;
}

static int plan_init(spf_plan* P) {
  const int N = P->N;
  es_params(P->eps, &P->w, &P->beta);
  es_poly(P->w, P->beta, &P->poly);
  P->Mh = (N - 1) / 2;
  double dq = P->qmax / P->Mh;
  double dr = 1.0 / (N * dq);
  P->radians_per_q = 2.0 * M_PI * dr;
  int nf = fine_size(N, P->w);
  int nfT = fine_size(2 * N - 1, P->w);
  SPF_TRY(grid_init(&P->g, N, nf, nf * dr, P->w, P->beta, P->max_points, true));
  SPF_TRY(grid_init(&P->gT, 2 * N - 1, nfT, nfT * dr, P->w, P->beta, P->max_points, false));
  P->PT = smooth_even_at_least(2 * N - 1);
  size_t PT3 = (size_t)P->PT * P->PT * P->PT;
  SPF_TRY(dev_alloc((void**)&P->cubeP, sizeof(float2) * PT3, "Toeplitz cube"));
  SPF_TRY(dev_alloc((void**)&P->realP, sizeof(float) * PT3, "Toeplitz real scratch"));
  SPF_TRY(fft3_create(&P->fftP, P->PT, P->PT, P->PT));
  SPF_TRY(dev_alloc((void**)&P->sorted, sizeof(uint32_t) * (size_t)std::max<int64_t>(1, P->max_points),
                    "sorted point ids"));
  SPF_TRY(cg_alloc(P));
  SPF_TRY(grad_alloc(P));
  SPF_TRY(dev_alloc((void**)&P->err, sizeof(int), "error word"));
  SPF_CUDA(cudaMemset(P->err, 0, sizeof(int)));
  SPF_CUDA(cudaDeviceSynchronize());
  return SPF_OK;
}

static int check_plan(const spf_plan* P) {
  SPF_CHECK_ARG(P != nullptr, "plan is NULL");
  return SPF_OK;
}

// Calls that write the plan's fine grids are refused while a deferred merge
// keeps its partial sums there.
static int check_grids_free(const spf_plan* P) {
  SPF_CHECK_ARG(!P->merge_open,
                "a deferred merge is open on this plan (spf_merge_begin without spf_merge_finish): "
                "its partial sums occupy the fine grids this call would overwrite");
  return SPF_OK;
}

}  // namespace spf

using namespace spf;

extern "C" {

const char* spf_last_error_string(void) { return g_err.c_str(); }

int spf_version(void) { return 1; }

int spf_plan_create(spf_plan** out, int N, double qmax, double eps, int64_t max_points, int device) {
  clear_error();
  SPF_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  SPF_CHECK_ARG(N >= 3 && N <= 1023 && (N % 2) == 1, "N must be odd in 3..1023 (got %d)", N);
  SPF_CHECK_ARG(qmax > 0.0, "qmax must be positive");
  SPF_CHECK_ARG(eps >= 1e-7 && eps <= 1e-4, "eps must be in [1e-7, 1e-4] (got %g)", eps);
  SPF_CHECK_ARG(max_points >= 0 && max_points <= 0x7fffffffLL, "max_points must be in [0, 2^31)");
  DeviceScope dev(device);
  if (dev.rc != SPF_OK) return dev.rc;
  spf_plan* P = new spf_plan();
  P->device = device;
  P->N = N;
  P->qmax = qmax;
  P->eps = eps;
  P->max_points = max_points;
  int rc = plan_init(P);
  if (rc != SPF_OK) {
    plan_free(P);
    return rc;
  }
  *out = P;
  return SPF_OK;
}

int spf_plan_destroy(spf_plan* plan) {
  clear_error();
  if (!plan) return SPF_OK;
  DeviceScope dev(plan->device);
  cudaDeviceSynchronize();
  plan_free(plan);
  return SPF_OK;
}

int spf_plan_status(spf_plan* plan) {
  clear_error();
  SPF_TRY(check_plan(plan));
  DeviceScope dev(plan->device);
  SPF_CUDA(cudaDeviceSynchronize());
  int e = 0;
  SPF_CUDA(cudaMemcpy(&e, plan->err, sizeof(int), cudaMemcpyDeviceToHost));
  SPF_CUDA(cudaMemset(plan->err, 0, sizeof(int)));
  if (e) {
    set_error("device error word 0x%x (1: a point fell outside its bin, 4: an orientation "
              "index was out of range)", e);
    return SPF_ERR_ARG;
  }
  return SPF_OK;
}

int spf_plan_sizes(const spf_plan* plan, int* nf, int* nfT, int* PT, int* w) {
  clear_error();
  SPF_TRY(check_plan(plan));
  if (nf) *nf = plan->g.nf;
  if (nfT) *nfT = plan->gT.nf;
  if (PT) *PT = plan->PT;
  if (w) *w = plan->w;
  return SPF_OK;
}

int spf_slice_model(spf_plan* plan, const float* A, const float* quats, int M, const float* q_lab,
                    int P2, float* slices, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(M >= 0 && P2 > 0, "M >= 0 and P2 > 0 required");
  SPF_CHECK_ARG((int64_t)M * P2 <= 0xffffffffLL, "M*P2 must be < 2^32");
  SPF_CHECK_ARG(A && q_lab && (M == 0 || (quats && slices)), "NULL pointer");
  SPF_CHECK_ARG(M == 0 || aligned16(quats), "quats must be 16-byte aligned");
  if (M == 0) return SPF_OK;
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  SPF_TRY(type2_setup(plan, A, s));
  return type2_quat(plan, quats, M, q_lab, P2, slices, s);
}

int spf_slice_adjoint(spf_plan* plan, const float* g, const float* quats, int M, const float* q_lab,
                      int P2, float* gradA, int accumulate, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(M >= 0 && P2 > 0, "M >= 0 and P2 > 0 required");
  SPF_CHECK_ARG((int64_t)M * P2 <= plan->max_points, "M*P2 = %lld exceeds max_points %lld",
                (long long)M * P2, (long long)plan->max_points);
  SPF_CHECK_ARG(gradA && q_lab && (M == 0 || (quats && g)), "NULL pointer");
  SPF_CHECK_ARG(M == 0 || aligned16(quats), "quats must be 16-byte aligned");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return type1_quat(plan, g, quats, M, q_lab, P2, gradA, accumulate, plan->err, as_stream(stream));
}

int spf_nufft_type2(spf_plan* plan, const float* A, const float* pts, int64_t npts, float* out,
                    void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(npts >= 0 && npts <= 0xffffffffLL, "npts must be in [0, 2^32)");
  SPF_CHECK_ARG(A && (npts == 0 || (pts && out)), "NULL pointer");
  if (npts == 0) return SPF_OK;
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  SPF_TRY(type2_setup(plan, A, s));
  return type2_explicit(plan, pts, npts, out, s);
}

int spf_nufft_type1(spf_plan* plan, const float* v, const float* pts, int64_t npts, float* out,
                    int accumulate, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(npts >= 0 && npts <= plan->max_points, "npts %lld exceeds max_points %lld",
                (long long)npts, (long long)plan->max_points);
  SPF_CHECK_ARG(out && (npts == 0 || (pts && v)), "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return type1_explicit(plan, v, pts, npts, out, accumulate, plan->err, as_stream(stream));
}

int spf_merge_images(spf_plan* plan, const float* images, const float* quats, int n_quats,
                     const int32_t* orient_idx, int n_img, const float* q_lab, int P2,
                     const float* D, float b_scale, float* rhs, float* kernel_hat, int accumulate,
                     void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(n_img >= 0 && P2 > 0, "n_img >= 0 and P2 > 0 required");
  SPF_CHECK_ARG((int64_t)n_img * P2 <= plan->max_points, "n_img*P2 = %lld exceeds max_points %lld",
                (long long)n_img * P2, (long long)plan->max_points);
  SPF_CHECK_ARG(q_lab && (rhs || kernel_hat), "NULL pointer");
  SPF_CHECK_ARG(n_img == 0 || (quats && aligned16(quats)), "quats must be 16-byte aligned");
  SPF_CHECK_ARG(n_img == 0 || !rhs || images, "images is NULL");
  SPF_CHECK_ARG(orient_idx ? n_quats > 0 : n_quats >= n_img,
                "quats must hold n_img rows, or n_quats > 0 rows with orient_idx");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return merge_run(plan, images, quats, n_quats, orient_idx, n_img, q_lab, P2, D, b_scale, rhs,
                   kernel_hat, accumulate, plan->err, as_stream(stream), kMergeClear | kMergeFinish,
                   rhs != nullptr, kernel_hat != nullptr);
}

int spf_cg_begin(spf_plan* plan, const float* kernel_hat, double lambda, const float* rhs,
                 const float* x0, float* x, double* res_norm, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(kernel_hat && rhs && x0 && x, "NULL pointer");
  SPF_CHECK_ARG(lambda >= 0.0, "lambda must be >= 0");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return cg_begin(plan, kernel_hat, lambda, rhs, x0, x, res_norm, as_stream(stream));
}

int spf_cg_merge_step(spf_plan* plan, const float* kernel_hat, double lambda, float* x,
                      double* res_norm, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(kernel_hat && x, "NULL pointer");
  SPF_CHECK_ARG(lambda >= 0.0, "lambda must be >= 0");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return cg_step(plan, kernel_hat, lambda, x, res_norm, as_stream(stream));
}

int spf_cg_objective(spf_plan* plan, const float* kernel_hat, const float* rhs, const float* x,
                     const float* x0, const double* b_norm2, double* out, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(kernel_hat && rhs && x && x0 && out, "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return cg_objective(plan, kernel_hat, rhs, x, x0, b_norm2, out, as_stream(stream));
}

int spf_weighted_sumsq(spf_plan* plan, const float* images, int n_img, int P2, const float* D,
                       float scale, double* out, int accumulate, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(n_img >= 0 && P2 > 0 && out && (n_img == 0 || images), "bad arguments");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return weighted_sumsq(plan, images, (int64_t)n_img * P2, P2, D, scale, out, accumulate,
                        as_stream(stream));
}

static int check_grad_args(const spf_plan* P, const float* quats, int n_img, const float* q_lab, int P2,
                           double lambda, int chunk, const float* work) {
  SPF_CHECK_ARG(n_img >= 0 && P2 > 0 && chunk >= 1, "n_img >= 0, P2 > 0 and chunk >= 1 required");
  SPF_CHECK_ARG((int64_t)chunk * P2 <= P->max_points, "chunk*P2 = %lld exceeds max_points %lld",
                (long long)chunk * P2, (long long)P->max_points);
  SPF_CHECK_ARG(lambda >= 0.0, "lambda must be >= 0");
  SPF_CHECK_ARG(q_lab && work && (n_img == 0 || quats), "NULL pointer");
  SPF_CHECK_ARG(n_img == 0 || aligned16(quats), "quats must be 16-byte aligned");
  return SPF_OK;
}

int spf_slice_loss_grad(spf_plan* plan, const float* x, const float* x0, const float* quats, int n_img,
                        const float* q_lab, int P2, const float* images, float b_scale, const float* D,
                        double lambda, int chunk, float* work, double* loss, float* grad, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_TRY(check_grad_args(plan, quats, n_img, q_lab, P2, lambda, chunk, work));
  SPF_CHECK_ARG(x && loss && grad && (n_img == 0 || images) && (lambda == 0.0 || x0), "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return slice_loss_grad(plan, x, x0, quats, n_img, q_lab, P2, images, b_scale, D, lambda, chunk, work, loss, grad,
                         as_stream(stream));
}

int spf_slice_normal_apply(spf_plan* plan, const float* v, const float* quats, int n_img, const float* q_lab,
                           int P2, const float* D, double lambda, int chunk, float* work, float* out,
                           void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_TRY(check_grad_args(plan, quats, n_img, q_lab, P2, lambda, chunk, work));
  SPF_CHECK_ARG(v && out, "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return slice_normal_apply(plan, v, quats, n_img, q_lab, P2, D, lambda, chunk, work, out, as_stream(stream));
}

int spf_gradient_step(spf_plan* plan, float* x, const float* x0, const float* quats, int n_img,
                      const float* q_lab, int P2, const float* images, float b_scale, const float* D,
                      double lambda, int chunk, float* work, float* grad, float* Hg, double* loss,
                      void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_TRY(check_grad_args(plan, quats, n_img, q_lab, P2, lambda, chunk, work));
  SPF_CHECK_ARG(x && grad && Hg && loss && (n_img == 0 || images) && (lambda == 0.0 || x0), "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return gradient_step(plan, x, x0, quats, n_img, q_lab, P2, images, b_scale, D, lambda, chunk, work, grad, Hg,
                       loss, as_stream(stream));
}

int spf_toeplitz_apply(spf_plan* plan, const float* kernel_hat, double lambda, const float* x,
                       float* out, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(kernel_hat && x && out, "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return toeplitz_apply(plan, kernel_hat, lambda, x, out, nullptr, as_stream(stream));
}

// ------------------------------------------------------------- matcher ---
static void matcher_free(spf_matcher* m) {
  if (!m) return;
  cudaFree(m->x2);
  cudaFree(m->y2);
  cudaFree(m->xq);
  cudaFree(m->yq);
  cudaFree(m->xs);
  cudaFree(m->ys);
  cudaFree(m->cand_v);
  cudaFree(m->cand_i);
  cudaFree(m->st_d);
  cudaFree(m->st_i);
  cudaFree(m->err);
  cudaFree(m->wbuf);
  cudaFree(m->rr_key);
  cudaFree(m->rr_start);
  cudaFree(m->rr_order);
  cudaFree(m->ap_v);
  cudaFree(m->ap_i);
  cudaFree(m->ch_off_d);
  cudaFree(m->ch_ptr_d);
  delete m;
}

int spf_matcher_create(spf_matcher** out, int max_images, int max_orient_chunk, int P2,
                       int precision, int topk, int device) {
  clear_error();
  SPF_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  SPF_CHECK_ARG(max_images >= 0 && max_orient_chunk >= 0 && P2 > 0, "bad sizes");
  SPF_CHECK_ARG(precision == SPF_FP32 || precision == SPF_BF16 || precision == SPF_FP8,
                "unknown precision %d", precision);
  SPF_CHECK_ARG(topk >= 2 && topk <= SPF_MAX_TOPK, "topk must be in 2..%d", SPF_MAX_TOPK);
  DeviceScope dev(device);
  if (dev.rc != SPF_OK) return dev.rc;
  spf_matcher* m = new spf_matcher();
  m->device = device;
  m->max_images = max_images;
  m->max_orient = max_orient_chunk;
  m->P2 = P2;
  m->precision = precision;
  m->topk = topk;
  int rc = SPF_OK;
  cudaDeviceGetAttribute(&m->n_sms, cudaDevAttrMultiProcessorCount, device);
  auto A = [&](void** p, size_t b, const char* w) {
    if (rc == SPF_OK) rc = dev_alloc(p, b, w);
  };
  A((void**)&m->x2, sizeof(float) * max_images, "image norms");
  A((void**)&m->y2, sizeof(float) * max_orient_chunk, "slice norms");
  A((void**)&m->cand_v, sizeof(float) * (size_t)max_images * kMaxSplits * kCand, "candidates");
  A((void**)&m->cand_i, sizeof(int) * (size_t)max_images * kMaxSplits * kCand, "candidates");
  A((void**)&m->st_d, sizeof(float) * (size_t)max_images * topk, "running list");
  A((void**)&m->st_i, sizeof(int) * (size_t)max_images * topk, "running list");
  A((void**)&m->err, sizeof(int), "error word");
  A((void**)&m->wbuf, sizeof(float) * P2, "pixel weights");
  A((void**)&m->rr_key, sizeof(int) * std::max(max_images, 1), "re-rank keys");
  A((void**)&m->rr_start, sizeof(int) * ((size_t)max_orient_chunk + 1), "re-rank buckets");
  A((void**)&m->rr_order, sizeof(int) * std::max(max_images, 1), "re-rank order");
  A((void**)&m->ap_v, sizeof(float) * (size_t)std::max(max_images, 1) * kCand, "approximate candidates");
  A((void**)&m->ap_i, sizeof(int) * (size_t)std::max(max_images, 1) * kCand, "approximate candidates");
  A((void**)&m->ch_off_d, sizeof(int) * (kMaxChunks + 1), "re-rank chunk offsets");
  A((void**)&m->ch_ptr_d, sizeof(float*) * kMaxChunks, "re-rank chunk rows");
  if (rc == SPF_OK && precision != SPF_FP32) {
    if (!match_tc_supported(device)) {
      set_error("tensor-core matching needs an sm_103 device");
      rc = SPF_ERR_UNSUPPORTED;
    }
    m->Kpad = tc_kpad(P2, precision);
    size_t eb = precision == SPF_BF16 ? 2 : 1;
    A(&m->xq, eb * (size_t)max_images * m->Kpad, "quantised images");
    A(&m->yq, eb * (size_t)max_orient_chunk * m->Kpad, "quantised slices");
    A((void**)&m->xs, sizeof(float) * max_images, "image scales");
    A((void**)&m->ys, sizeof(float) * max_orient_chunk, "slice scales");
    if (rc == SPF_OK) {
      // zero once so padding columns stay zero for every later call
      cudaMemset(m->xq, 0, eb * (size_t)max_images * m->Kpad);
      cudaMemset(m->yq, 0, eb * (size_t)max_orient_chunk * m->Kpad);
    }
  }
  if (rc == SPF_OK) {
    cudaError_t e = cudaMemset(m->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("matcher set-up: %s", cudaGetErrorString(e));
      rc = SPF_ERR_CUDA;
    }
  }
  if (rc != SPF_OK) {
    matcher_free(m);
    return rc;
  }
  *out = m;
  return SPF_OK;
}

int spf_matcher_destroy(spf_matcher* m) {
  clear_error();
  if (!m) return SPF_OK;
  DeviceScope dev(m->device);
  cudaDeviceSynchronize();
  matcher_free(m);
  return SPF_OK;
}

int spf_matcher_status(spf_matcher* m) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  DeviceScope dev(m->device);
  SPF_CUDA(cudaDeviceSynchronize());
  int e = 0;
  SPF_CUDA(cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost));
  SPF_CUDA(cudaMemset(m->err, 0, sizeof(int)));
  if (e & 2) {
    set_error("a tensor-core pipeline wait timed out (error word 0x%x)", e);
    return SPF_ERR_TIMEOUT;
  }
  if (e) {
    set_error("device error word 0x%x", e);
    return SPF_ERR_CUDA;
  }
  return SPF_OK;
}

int spf_matcher_set_mask(spf_matcher* m, const float* D, void* stream) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  DeviceScope dev(m->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return set_mask_weights(m, D, as_stream(stream));
}

int spf_matcher_set_rerank(spf_matcher* m, int deferred) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  SPF_CHECK_ARG(deferred == 0 || deferred == 1, "deferred must be 0 or 1");
  SPF_CHECK_ARG(!m->pending, "a deferred re-rank is pending: read the results first");
  m->defer = deferred;
  return SPF_OK;
}

int spf_matcher_set_schedule(spf_matcher* m, int schedule) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  SPF_CHECK_ARG(schedule >= 0 && schedule <= 2, "schedule must be 0 (model), 1 (contiguous) or 2 (grid)");
  m->tc_force = schedule;
  return SPF_OK;
}

int spf_matcher_set_images(spf_matcher* m, const float* images, int n_img, float img_scale,
                           void* stream) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  SPF_CHECK_ARG(n_img >= 0 && n_img <= m->max_images, "n_img %d exceeds max_images %d", n_img,
                m->max_images);
  SPF_CHECK_ARG(n_img == 0 || images, "images is NULL");
  DeviceScope dev(m->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  m->images = images;
  m->images16 = nullptr;
  m->n_img = n_img;
  m->img_scale = img_scale;
  if (m->precision == SPF_FP32)
    SPF_TRY(row_norms_w(images, n_img, m->P2, img_scale, m->wsq, m->x2, s));
  else
    SPF_TRY(quantize_rows(m, images, n_img, img_scale, m->xq, m->xs, m->x2, s));
  return state_reset(m, s);
}

int spf_matcher_set_images_u16(spf_matcher* m, const uint16_t* images, int n_img, float img_scale,
                               void* stream) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  if (m->precision == SPF_FP32) {
    set_error("16-bit images need a BF16 or FP8 matcher");
    return SPF_ERR_UNSUPPORTED;
  }
  SPF_CHECK_ARG(n_img >= 0 && n_img <= m->max_images, "n_img %d exceeds max_images %d", n_img,
                m->max_images);
  SPF_CHECK_ARG(n_img == 0 || images, "images is NULL");
  SPF_CHECK_ARG(((uintptr_t)images & 1) == 0, "images must be 2-byte aligned");
  DeviceScope dev(m->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  m->images = nullptr;
  m->images16 = images;
  m->n_img = n_img;
  m->img_scale = img_scale;
  SPF_TRY(quantize_rows_u16(m, images, n_img, img_scale, m->xq, m->xs, m->x2, s));
  return state_reset(m, s);
}

int spf_matcher_add_slices(spf_matcher* m, const float* slices, int n_orient, int orient_offset,
                           void* stream) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  SPF_CHECK_ARG(n_orient >= 0 && n_orient <= m->max_orient, "n_orient %d exceeds max %d",
                n_orient, m->max_orient);
  SPF_CHECK_ARG(orient_offset >= 0 && (int64_t)orient_offset + n_orient <= 0x7fffffffLL,
                "bad orient_offset");
  SPF_CHECK_ARG(n_orient == 0 || slices, "slices is NULL");
  if (n_orient == 0 || m->n_img == 0) return SPF_OK;
  DeviceScope dev(m->device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  int nsplit;
  if (m->precision == SPF_FP32) {
    SPF_TRY(row_norms_w(slices, n_orient, m->P2, 1.f, m->wsq, m->y2, s));
    nsplit = simt_splits(m->n_img, n_orient, m->n_sms);
    SPF_TRY(simt_launch(m, slices, n_orient, orient_offset, nsplit, s));
  } else {
    SPF_TRY(quantize_rows(m, slices, n_orient, 1.f, m->yq, m->ys, m->y2, s));
    nsplit = tc_schedule(m->n_img, n_orient, m->n_sms, m->Kpad, m->precision == SPF_FP8, m->tc_force).nsplit;
    SPF_TRY(match_tc_launch(m, n_orient, orient_offset, nsplit, s));
  }
  return rerank_launch(m, slices, n_orient, orient_offset, nsplit, s);
}

int spf_matcher_results(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                        int32_t* topk_idx, float* topk_d, void* stream) {
  clear_error();
  SPF_CHECK_ARG(m != nullptr, "matcher is NULL");
  DeviceScope dev(m->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return results_launch(m, best_idx, best_d, second_d, topk_idx, topk_d, as_stream(stream));
}

int spf_match_orientations(spf_matcher* m, const float* images, int n_img, float img_scale,
                           const float* slices, int n_orient, int32_t* best_idx, float* best_d,
                           float* second_d, void* stream) {
  SPF_TRY(spf_matcher_set_images(m, images, n_img, img_scale, stream));
  SPF_TRY(spf_matcher_add_slices(m, slices, n_orient, 0, stream));
  return spf_matcher_results(m, best_idx, best_d, second_d, nullptr, nullptr, stream);
}

int spf_counts_to_f32(const uint16_t* counts, int64_t n, float* out, void* stream) {
  clear_error();
  SPF_CHECK_ARG(n >= 0, "n must be >= 0 (got %lld)", (long long)n);
  SPF_CHECK_ARG(n == 0 || (counts && out), "counts and out must be non-NULL");
  SPF_CHECK_ARG(((uintptr_t)counts & 1) == 0, "counts must be 2-byte aligned");
  return counts_to_f32(counts, n, out, as_stream(stream));
}

// ------------------------------------------------------------ point sets --
static void points_free(spf_points* S) {
  if (!S) return;
  cudaFree(S->quats);
  cudaFree(S->qlab);
  cudaFree(S->setN.ids);
  cudaFree(S->setN.subs);
  cudaFree(S->setN.nsubs);
  cudaFree(S->setN.bsubs);
  cudaFree(S->setN.nbsubs);
  cudaFree(S->setT.ids);
  cudaFree(S->setT.subs);
  cudaFree(S->setT.nsubs);
  cudaFree(S->invN);
  cudaFree(S->cls);
  cudaFree(S->cnt);
  delete S;
}

int spf_points_create(spf_points** out, spf_plan* plan, const float* quats, int M, const float* q_lab,
                      int P2, int flags, void* stream) {
  clear_error();
  SPF_CHECK_ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  SPF_TRY(check_plan(plan));
  SPF_CHECK_ARG(M >= 0 && P2 > 0, "M >= 0 and P2 > 0 required");
  SPF_CHECK_ARG((int64_t)M * P2 <= 0x7fffffffLL, "M*P2 must be < 2^31");
  SPF_CHECK_ARG(q_lab && (M == 0 || quats), "NULL pointer");
  SPF_CHECK_ARG(flags == 0 || flags == SPF_POINTS_SLICE_ONLY, "unknown flags %d", flags);
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  spf_points* S = new spf_points();
  S->plan = plan;
  S->device = plan->device;
  S->M = M;
  S->P2 = P2;
  S->flags = flags;
  const bool full = flags == 0;
  const int64_t npts = (int64_t)M * P2;
  int rc = SPF_OK;
  auto A = [&](void** p, size_t b, const char* w) {
    if (rc == SPF_OK) rc = dev_alloc(p, b, w);
  };
  A((void**)&S->quats, sizeof(float) * 4 * std::max(M, 1), "point-set orientations");
  A((void**)&S->qlab, sizeof(float) * 3 * P2, "point-set q-points");
  S->setN.max_subs = plan->g.bins.nbins + npts / kSubPts + 1;
  S->setT.max_subs = plan->gT.bins.nbins + npts / kSubPts + 1;
  A((void**)&S->setN.ids, sizeof(uint32_t) * std::max<int64_t>(npts, 1), "sorted ids");
  A((void**)&S->setN.subs, sizeof(int4) * S->setN.max_subs, "subproblems");
  A((void**)&S->setN.nsubs, 2 * sizeof(int), "subproblem count");
  S->setN.max_bsubs = 8 * (int64_t)plan->g.bins.nbins + npts / kSubPts + 1;
  A((void**)&S->setN.bsubs, sizeof(int4) * S->setN.max_bsubs, "block subproblems");
  A((void**)&S->setN.nbsubs, 2 * sizeof(int), "block subproblem count");
  if (full) {
    A((void**)&S->setT.ids, sizeof(uint32_t) * std::max<int64_t>(npts, 1), "sorted ids");
    A((void**)&S->setT.subs, sizeof(int4) * S->setT.max_subs, "subproblems");
    A((void**)&S->setT.nsubs, 2 * sizeof(int), "subproblem count");
    A((void**)&S->invN, sizeof(uint32_t) * std::max<int64_t>(npts, 1), "inverse order");
    A((void**)&S->cls, sizeof(float) * std::max<int64_t>(npts, 1), "class sums");
    A((void**)&S->cnt, sizeof(float) * std::max(M, 1), "class counts");
  }
  if (rc != SPF_OK) {
    points_free(S);
    return rc;
  }
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaSuccess;
  if (M > 0) e = cudaMemcpyAsync(S->quats, quats, sizeof(float) * 4 * M, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S->qlab, q_lab, sizeof(float) * 3 * P2, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    set_error("copy of the point set: %s", cudaGetErrorString(e));
    points_free(S);
    return SPF_ERR_CUDA;
  }
  rc = points_build(plan, S, s);
  if (rc != SPF_OK) {
    points_free(S);
    return rc;
  }
  *out = S;
  return SPF_OK;
}

int spf_points_destroy(spf_points* pts) {
  clear_error();
  if (!pts) return SPF_OK;
  DeviceScope dev(pts->device);
  cudaDeviceSynchronize();
  points_free(pts);
  return SPF_OK;
}

int spf_slice_points(spf_plan* plan, spf_points* pts, const float* A, float* slices, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(pts && pts->plan == plan, "point set is NULL or belongs to another plan");
  SPF_CHECK_ARG(A && (pts->M == 0 || slices), "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return slice_points(plan, pts, A, slices, as_stream(stream));
}

int spf_merge_points(spf_plan* plan, spf_points* pts, const float* images, const int32_t* orient_idx,
                     int n_img, int orient_offset, const float* D, float b_scale, float* rhs,
                     float* kernel_hat, int accumulate, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_grids_free(plan));
  SPF_CHECK_ARG(pts && pts->plan == plan, "point set is NULL or belongs to another plan");
  SPF_CHECK_ARG(pts->flags == 0, "the point set was created for slicing only");
  SPF_CHECK_ARG(n_img >= 0 && (n_img == 0 || (images && orient_idx)), "NULL pointer");
  SPF_CHECK_ARG(rhs || kernel_hat, "rhs and kernel_hat are both NULL");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return merge_points(plan, pts, images, orient_idx, n_img, orient_offset, D, b_scale, rhs, kernel_hat,
                      accumulate, as_stream(stream), kMergeClear | kMergeFinish, rhs != nullptr,
                      kernel_hat != nullptr);
}

int spf_merge_begin(spf_plan* plan, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  SPF_TRY(merge_begin(plan, as_stream(stream)));
  plan->merge_open = true;
  return SPF_OK;
}

static int check_merge_open(const spf_plan* P) {
  SPF_CHECK_ARG(P->merge_open, "no deferred merge is open on this plan (call spf_merge_begin first)");
  return SPF_OK;
}

int spf_merge_points_add(spf_plan* plan, spf_points* pts, const float* images, const int32_t* orient_idx,
                         int n_img, int orient_offset, const float* D, float b_scale, int want_rhs,
                         int want_kernel, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_merge_open(plan));
  SPF_CHECK_ARG(pts && pts->plan == plan, "point set is NULL or belongs to another plan");
  SPF_CHECK_ARG(pts->flags == 0, "the point set was created for slicing only");
  SPF_CHECK_ARG(n_img >= 0 && (n_img == 0 || (images && orient_idx)), "NULL pointer");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return merge_points(plan, pts, images, orient_idx, n_img, orient_offset, D, b_scale, nullptr, nullptr, 0,
                      as_stream(stream), 0, want_rhs != 0, want_kernel != 0);
}

int spf_merge_images_add(spf_plan* plan, const float* images, const float* quats, int n_quats,
                         const int32_t* orient_idx, int n_img, const float* q_lab, int P2, const float* D,
                         float b_scale, int want_rhs, int want_kernel, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_merge_open(plan));
  SPF_CHECK_ARG(n_img >= 0 && P2 > 0, "n_img >= 0 and P2 > 0 required");
  SPF_CHECK_ARG((int64_t)n_img * P2 <= plan->max_points, "n_img*P2 = %lld exceeds max_points %lld",
                (long long)n_img * P2, (long long)plan->max_points);
  SPF_CHECK_ARG(q_lab != nullptr, "NULL pointer");
  SPF_CHECK_ARG(n_img == 0 || (quats && aligned16(quats)), "quats must be 16-byte aligned");
  SPF_CHECK_ARG(n_img == 0 || !want_rhs || images, "images is NULL");
  SPF_CHECK_ARG(orient_idx ? n_quats > 0 : n_quats >= n_img,
                "quats must hold n_img rows, or n_quats > 0 rows with orient_idx");
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  return merge_run(plan, images, quats, n_quats, orient_idx, n_img, q_lab, P2, D, b_scale, nullptr, nullptr,
                   0, plan->err, as_stream(stream), 0, want_rhs != 0, want_kernel != 0);
}

int spf_merge_finish(spf_plan* plan, float* rhs, float* kernel_hat, int accumulate, void* stream) {
  clear_error();
  SPF_TRY(check_plan(plan));
  SPF_TRY(check_merge_open(plan));
  DeviceScope dev(plan->device);
  if (dev.rc != SPF_OK) return dev.rc;
  plan->merge_open = false;
  return merge_finish(plan, rhs, kernel_hat, accumulate, as_stream(stream));
}

}  // extern "C"
