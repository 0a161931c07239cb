// One M-TIP slice -> match -> merge -> CG iteration (Fig. 3 without phasing)
// as native host orchestration of the library's kernels.
//
// The reference orientations are fixed across iterations (Sec. II-A: a
// predetermined set), so the driver takes them once (spf_mtip_set_orientations):
// it renumbers them along a Morton curve of the quaternions (orientations
// close in index are close on SO(3), so images re-ranked together share
// candidate model images in L2), and either sorts the rotated points of every
// orientation chunk once and keeps them (16 bytes per orientation x pixel);
// or, when that exceeds the memory budget, keeps only each chunk's sort for
// slicing (4 bytes per orientation x pixel) and merges image chunks at their
// matched orientations; or, when that too exceeds it, re-sorts each chunk's
// points for slicing on every iteration. An iteration:
//   1. slicing (Sec. II-A) and matching (Sec. II-B), streamed in orientation
//      chunks through one slice buffer; the matcher's running top-k survives
//      across chunks;
//   2. merging (Sec. II-C): every chunk is spread onto the plan's fine grids
//      (class sums and counts at the kept points, or images at their matched
//      orientations), which are transformed once into the right-hand side and
//      the Toeplitz kernel -- the type-1 sums are linear;
//   3. CG on Eq. 2 from x0 = the current model with lambda = lam_rel * sum D
//      over all merged pixels.
// Indices returned to the caller are in the caller's numbering.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "match.h"
#include "plan.h"

namespace spf {
int points_build(spf_plan* P, spf_points* S, cudaStream_t s);
int slice_points(spf_plan* P, spf_points* S, const float* A, float* out, cudaStream_t s);
int merge_points(spf_plan* P, spf_points* S, const float* images, const int* oidx, int n_img, int off,
                 const float* D, float b_scale, float* rhs, float* kernel_hat, int accumulate,
                 cudaStream_t s, int mode, bool want_rhs, bool want_kernel);
int merge_run(spf_plan* P, const float* images, const float* quats, int n_quats, const int* oidx,
              int n_img, const float* qlab, int P2, const float* D, float b_scale, float* rhs,
              float* kernel_hat, int accumulate, int* err, cudaStream_t s, int mode, bool want_rhs,
              bool want_kernel);
int merge_begin(spf_plan* P, cudaStream_t s);
int class_sums_sets(spf_points* const* sets, int nsets, const uint32_t* const* inv_tab, float* const* cls_tab,
                    float* const* cnt_tab, const float* images, const uint16_t* images16, const int* oidx, int n_img,
                    int chunk, int n_total, const float* D, float b_scale, int* err, cudaStream_t s);
int merge_finish(spf_plan* P, float* rhs, float* kernel_hat, int accumulate, cudaStream_t s);
int cg_begin(spf_plan* P, const float* khat, double lambda, const float* rhs, const float* x0,
             float* x, double* res, cudaStream_t s);
int cg_step(spf_plan* P, const float* khat, double lambda, float* x, double* res, cudaStream_t s);

namespace {

// out[i] = map[in[i]] (in[i] < 0 stays -1): orientation indices between the
// driver's numbering and the caller's.
__global__ void remap_index_kernel(const int* __restrict__ in, int64_t n, const int* __restrict__ map, int nmap,
                                   int* __restrict__ out, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int v = in[i];
    if (v < 0) {
      out[i] = -1;
    } else if (v >= nmap) {
      atomicOr(err, 4);   // an orientation index outside the set
      out[i] = 0;
    } else {
      out[i] = __ldg(map + v);
    }
  }
}

int remap(const int* in, int64_t n, const int* map, int nmap, int* out, int* err, cudaStream_t s) {
  if (n == 0) return SPF_OK;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 4096);
  return launch("remap_index_kernel", s,
                [&] { remap_index_kernel<<<grid, 256, 0, s>>>(in, n, map, nmap, out, err); }, 12.0 * n);
}

// Morton code of (x, y, z) of a unit quaternion (w, x, y, z), each quantised
// to 10 bits; the permutation that sorts the codes (stable).
std::vector<int> morton_order(const std::vector<float>& q, int M) {
  std::vector<uint64_t> key(M);
  for (int j = 0; j < M; ++j) {
    uint64_t c[3];
    for (int a = 0; a < 3; ++a) {
      const double v = std::nearbyint(((double)q[4 * j + 1 + a] + 1.0) * 0.5 * 1023.0);
      c[a] = (uint64_t)std::min(1023.0, std::max(0.0, v));
    }
    uint64_t k = 0;
    for (int bit = 0; bit < 10; ++bit)
      for (int a = 0; a < 3; ++a) k |= ((c[a] >> bit) & 1ull) << (3 * bit + a);
    key[j] = k;
  }
  std::vector<int> order(M);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
  return order;
}

constexpr int64_t kPointSetBytes = 16;   // per kept (orientation, pixel): two sort orders, inverse, class sum
constexpr int64_t kSliceSetBytes = 4;    // per kept (orientation, pixel) of a slice-only set: its sort order

}  // namespace
}  // namespace spf

struct spf_mtip {
  spf_mtip_config cfg{};
  spf_plan* plan = nullptr;
  spf_matcher* matcher = nullptr;
  bool cache_points = false;
  bool slice_sets = false;         // slice-only point sets kept per chunk; the merge streams
  bool keep_slices = false;        // slices of all chunks kept: one deferred re-rank
  int orient_chunk = 0, img_chunk = 0;
  // orientation set in the driver's numbering
  bool have_set = false;
  float* quats_sorted = nullptr;   // n_orient x 4
  float* qlab = nullptr;           // P2 x 3
  int* order = nullptr;            // driver index -> caller index
  int* inv = nullptr;              // caller index -> driver index
  std::vector<spf_points*> sets;   // kept point sets (full, or slice-only), one per orientation chunk
  uint32_t** inv_tab = nullptr;    // device tables of the sets' inverse orders, class sums, counts
  float** cls_tab = nullptr;
  float** cnt_tab = nullptr;
  spf_points stream_set;           // streaming: one slice-only set, re-sorted per chunk per call
  float* slices = nullptr;         // orient_chunk x P2, or n_orient x P2 when kept
  float* img32 = nullptr;          // max_images x P2: 16-bit counts converted to FP32 (FP32
                                   // matching or streamed merges only)
  int* best_sorted = nullptr;      // max_images
  int* best = nullptr;             // max_images (caller numbering)
  int* topk_tmp = nullptr;         // max_images x topk
  float* rhs = nullptr;            // N^3
  float* khat = nullptr;           // P_T^3
  float* x = nullptr;              // N^3
  const float* D = nullptr;        // pixel weights (caller-owned) or NULL
  double d_sum = 0.0;              // sum of D over one image (P2 without weights)
  int* err = nullptr;              // device error word of the driver's own kernels
  // host-buffer iteration: two input slots, a copy stream
  bool host_path = false;
  cudaStream_t copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  float* slotA[2] = {nullptr, nullptr};
  void* slotImg[2] = {nullptr, nullptr};
  cudaEvent_t up0[2] = {nullptr, nullptr}, up1[2] = {nullptr, nullptr};   // timing of each slot's image upload
  int upload_mode = SPF_UPLOAD_SM;
  int held_slot = -1;              // slot handed out by spf_mtip_upload_host, not yet released
  long long host_calls = 0;
};

namespace spf {
namespace {

struct DevScope {
  int prev = -1;
  int rc = SPF_OK;
  explicit DevScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) {
      set_error("cudaSetDevice(%d) failed", dev);
      rc = SPF_ERR_CUDA;
    }
  }
  ~DevScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void free_sets(spf_mtip* h) {
  for (auto* p : h->sets) spf_points_destroy(p);
  h->sets.clear();
  cudaFree(h->inv_tab);
  cudaFree(h->cls_tab);
  cudaFree(h->cnt_tab);
  h->inv_tab = nullptr;
  h->cls_tab = nullptr;
  h->cnt_tab = nullptr;
}

void mtip_free(spf_mtip* h) {
  if (!h) return;
  free_sets(h);
  cudaFree(h->stream_set.setN.ids);
  cudaFree(h->stream_set.setN.subs);
  cudaFree(h->stream_set.setN.nsubs);
  cudaFree(h->stream_set.setN.bsubs);
  cudaFree(h->stream_set.setN.nbsubs);
  cudaFree(h->quats_sorted);
  cudaFree(h->qlab);
  cudaFree(h->order);
  cudaFree(h->inv);
  cudaFree(h->slices);
  cudaFree(h->img32);
  cudaFree(h->best_sorted);
  cudaFree(h->best);
  cudaFree(h->topk_tmp);
  cudaFree(h->rhs);
  cudaFree(h->khat);
  cudaFree(h->x);
  cudaFree(h->err);
  for (int b = 0; b < 2; ++b) {
    cudaFree(h->slotA[b]);
    cudaFree(h->slotImg[b]);
    if (h->copied[b]) cudaEventDestroy(h->copied[b]);
    if (h->freed[b]) cudaEventDestroy(h->freed[b]);
    if (h->up0[b]) cudaEventDestroy(h->up0[b]);
    if (h->up1[b]) cudaEventDestroy(h->up1[b]);
  }
  if (h->copy) cudaStreamDestroy(h->copy);
  if (h->matcher) spf_matcher_destroy(h->matcher);
  if (h->plan) spf_plan_destroy(h->plan);
  delete h;
}

size_t image_elem(int type) { return type == SPF_IMAGES_U16 ? 2 : 4; }

// Copy of n16 16-byte vectors from page-locked host memory mapped into the
// device's address space: the SMs read over the CPU-GPU link, kUploadVec
// vectors in flight per thread, so that a few CTAs (few SMs taken from the
// call computing alongside) keep the link busy.
constexpr int kUploadVec = 8;
constexpr int kUploadCtas = 32;
__global__ void __launch_bounds__(512) upload_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                     size_t n16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += kUploadVec * stride) {
    uint4 v[kUploadVec];
#pragma unroll
    for (int k = 0; k < kUploadVec; ++k)
      if (i + k * stride < n16) v[k] = src[i + k * stride];
#pragma unroll
    for (int k = 0; k < kUploadVec; ++k)
      if (i + k * stride < n16) dst[i + k * stride] = v[k];
  }
}

// Device address of host bytes [p, p + n) when both ends are page-locked and
// mapped with the same offset (one registered range), else NULL.
const void* mapped_range(const void* p, size_t n) {
  if (n == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess || cudaPointerGetAttributes(
          &a1, static_cast<const char*>(p) + (n - 1)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if (static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) != (ptrdiff_t)(n - 1))
    return nullptr;
  return a0.devicePointer;
}

// Host-to-device upload of the images on the copy stream, by the mode set.
int upload_images(spf_mtip* h, void* dst, const void* src, size_t bytes, cudaStream_t s) {
  if (h->upload_mode == SPF_UPLOAD_SM) {
    const void* dsrc = mapped_range(src, bytes);
    if (dsrc && ((uintptr_t)dsrc & 15) == 0 && ((uintptr_t)dst & 15) == 0) {
      const size_t n16 = bytes / 16, tail = bytes - 16 * n16;
      if (n16 > 0)
        SPF_TRY(launch("upload_kernel", s, [&] {
          upload_kernel<<<kUploadCtas, 512, 0, s>>>(static_cast<const uint4*>(dsrc), static_cast<uint4*>(dst), n16);
        }, 2.0 * (double)(16 * n16)));
      if (tail > 0)
        SPF_CUDA(cudaMemcpyAsync(static_cast<char*>(dst) + 16 * n16, static_cast<const char*>(src) + 16 * n16,
                                 tail, cudaMemcpyHostToDevice, s));
      return SPF_OK;
    }
  }
  SPF_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  return SPF_OK;
}

int check_images(const spf_mtip* h, const void* images, int type, int n_img);

int check_upload(const spf_mtip* h, int image_type, const void* images_host, int n_img) {
  SPF_CHECK_ARG(h->host_path, "the driver was created without host-buffer slots (host_image_type = -1)");
  SPF_CHECK_ARG(image_type == h->cfg.host_image_type, "image type %d differs from the slots' type %d", image_type,
                h->cfg.host_image_type);
  return check_images(h, images_host, image_type, n_img);
}

// The model and the images of a host-buffer call into slot b = the call
// count's parity, on the copy stream once the call two back has released
// that slot; `s` waits for the copies.
int upload_slot(spf_mtip* h, const float* A_host, const void* images_host, int image_type, int n_img,
                cudaStream_t s, int* slot) {
  const int b = (int)(h->host_calls & 1);
  const size_t n3 = (size_t)h->cfg.N * h->cfg.N * h->cfg.N;
  SPF_CUDA(cudaStreamWaitEvent(h->copy, h->freed[b], 0));
  SPF_CUDA(cudaMemcpyAsync(h->slotA[b], A_host, sizeof(float) * n3, cudaMemcpyHostToDevice, h->copy));
  SPF_CUDA(cudaEventRecord(h->up0[b], h->copy));
  SPF_TRY(upload_images(h, h->slotImg[b], images_host, image_elem(image_type) * (size_t)n_img * h->cfg.P2, h->copy));
  SPF_CUDA(cudaEventRecord(h->up1[b], h->copy));
  SPF_CUDA(cudaEventRecord(h->copied[b], h->copy));
  SPF_CUDA(cudaStreamWaitEvent(s, h->copied[b], 0));
  ++h->host_calls;
  *slot = b;
  return SPF_OK;
}

// The images of a call: FP32 rows, or 16-bit photon counts, which the BF16 /
// FP8 matcher and the class sums of kept point sets read themselves; an
// FP32 copy is made only for the consumers that need one (the FP32 matcher,
// the streamed merge).
struct ImgIn {
  const float* f = nullptr;
  const uint16_t* u = nullptr;
};

int images_in(spf_mtip* h, const void* images, int type, int n_img, bool match, bool merge, ImgIn* in,
              cudaStream_t s) {
  if (type == SPF_IMAGES_F32) {
    in->f = static_cast<const float*>(images);
    return SPF_OK;
  }
  in->u = static_cast<const uint16_t*>(images);
  const bool need_f32 = (match && h->matcher->precision == SPF_FP32) || (merge && !h->cache_points);
  if (need_f32) {
    SPF_TRY(counts_to_f32(in->u, (int64_t)n_img * h->cfg.P2, h->img32, s));
    in->f = h->img32;
  }
  return SPF_OK;
}

// Slicing and matching over every orientation chunk; results in the driver's
// numbering into best_sorted (and the matcher's candidate lists).
int match_core(spf_mtip* h, const float* A, const ImgIn& img, int n_img, float img_scale, cudaStream_t s) {
  spf_plan* P = h->plan;
  const int P2 = h->cfg.P2, M = h->cfg.n_orient;
  if (img.u && h->matcher->precision != SPF_FP32)
    SPF_TRY(spf_matcher_set_images_u16(h->matcher, img.u, n_img, img_scale, s));
  else
    SPF_TRY(spf_matcher_set_images(h->matcher, img.f, n_img, img_scale, s));
  for (int c = 0, c0 = 0; c0 < M; ++c, c0 += h->orient_chunk) {
    const int m = std::min(h->orient_chunk, M - c0);
    float* out = h->keep_slices ? h->slices + (size_t)c0 * P2 : h->slices;
    if (h->cache_points || h->slice_sets) {
      SPF_TRY(slice_points(P, h->sets[c], A, out, s));
    } else {
      spf_points& S = h->stream_set;
      S.M = m;
      S.quats = h->quats_sorted + 4 * (size_t)c0;
      SPF_TRY(points_build(P, &S, s));
      SPF_TRY(slice_points(P, &S, A, out, s));
    }
    SPF_TRY(spf_matcher_add_slices(h->matcher, out, m, c0, s));
  }
  return SPF_OK;
}

// Deferred merge at driver-numbered orientations into rhs and khat.
int merge_core(spf_mtip* h, const ImgIn& img, int n_img, float img_scale, const int* best_sorted, float* rhs,
               float* khat, cudaStream_t s) {
  spf_plan* P = h->plan;
  const int P2 = h->cfg.P2, M = h->cfg.n_orient;
  SPF_TRY(merge_begin(P, s));
  if (h->cache_points) {
    // one pass over the images forms every set's class sums, then each set
    // spreads its sums (leaving them zeroed for the next call) and its counts
    SPF_TRY(class_sums_sets(h->sets.data(), (int)h->sets.size(), h->inv_tab, h->cls_tab, h->cnt_tab,
                            img.u ? nullptr : img.f, img.u, best_sorted, n_img, h->orient_chunk, M, h->D,
                            img_scale, h->err, s));
    for (size_t c = 0; c < h->sets.size(); ++c)
      SPF_TRY(merge_points(P, h->sets[c], nullptr, best_sorted, n_img, (int)c * h->orient_chunk, h->D, img_scale,
                           nullptr, nullptr, 0, s, kMergeSumsDone, true, true));
  } else {
    for (int i0 = 0; i0 < n_img; i0 += h->img_chunk) {
      const int ni = std::min(h->img_chunk, n_img - i0);
      SPF_TRY(merge_run(P, img.f + (size_t)i0 * P2, h->quats_sorted, M, best_sorted + i0, ni, h->qlab, P2, h->D,
                        img_scale, nullptr, nullptr, 0, P->err, s, 0, true, true));
    }
  }
  return merge_finish(P, rhs, khat, 0, s);
}

int solve_core(spf_mtip* h, const float* rhs, const float* khat, const float* x0, double lam_rel, int64_t n_total,
               int cg_iters, float* x, double* lambda_out, double* res_hist, cudaStream_t s) {
  const double per_img = h->D ? h->d_sum : (double)h->cfg.P2;
  const double lam = lam_rel * per_img * (double)n_total;
  if (lambda_out) *lambda_out = lam;
  SPF_TRY(cg_begin(h->plan, khat, lam, rhs, x0, x, res_hist, s));
  for (int k = 0; k < cg_iters; ++k) SPF_TRY(cg_step(h->plan, khat, lam, x, res_hist ? res_hist + k + 1 : nullptr, s));
  return SPF_OK;
}

int check_handle(const spf_mtip* h, bool need_set) {
  SPF_CHECK_ARG(h != nullptr, "driver is NULL");
  SPF_CHECK_ARG(!need_set || h->have_set, "no orientation set: call spf_mtip_set_orientations first");
  return SPF_OK;
}

int check_images(const spf_mtip* h, const void* images, int type, int n_img) {
  SPF_CHECK_ARG(type == SPF_IMAGES_F32 || type == SPF_IMAGES_U16, "unknown image type %d", type);
  SPF_CHECK_ARG(n_img >= 1 && n_img <= h->cfg.max_images, "n_img %d outside 1..%d", n_img, h->cfg.max_images);
  SPF_CHECK_ARG(images != nullptr, "images is NULL");
  SPF_CHECK_ARG(((uintptr_t)images & (image_elem(type) - 1)) == 0, "images misaligned for their type");
  return SPF_OK;
}

}  // namespace
}  // namespace spf

using namespace spf;

extern "C" {

int spf_mtip_create(spf_mtip** out, const spf_mtip_config* cfg) {
  clear_error();
  SPF_CHECK_ARG(out != nullptr && cfg != nullptr, "NULL pointer");
  *out = nullptr;
  const spf_mtip_config& c = *cfg;
  SPF_CHECK_ARG(c.P2 > 0 && c.max_images >= 1 && c.n_orient >= 1, "P2, max_images and n_orient must be positive");
  SPF_CHECK_ARG(c.orient_chunk >= 0 && c.img_chunk >= 0, "chunk sizes must be >= 0 (0: all at once)");
  SPF_CHECK_ARG(c.cache_points >= -1 && c.cache_points <= 2, "cache_points must be -1, 0, 1 or 2");
  SPF_CHECK_ARG(c.host_image_type >= -1 && c.host_image_type <= SPF_IMAGES_U16, "unknown host image type");
  SPF_CHECK_ARG(c.keep_slices >= -1 && c.keep_slices <= 1, "keep_slices must be -1, 0 or 1");
  const int chunk = std::min(c.n_orient, c.orient_chunk > 0 ? c.orient_chunk : c.n_orient);
  SPF_CHECK_ARG((int64_t)chunk * c.P2 < 0x7fffffffLL, "orient_chunk x P2 must be < 2^31");
  DevScope dev(c.device);
  if (dev.rc != SPF_OK) return dev.rc;
  spf_mtip* h = new spf_mtip();
  h->cfg = c;
  const int P2 = c.P2;
  h->orient_chunk = chunk;
  if (c.cache_points >= 0) {
    h->cache_points = c.cache_points == 1;
    h->slice_sets = c.cache_points == 2;
  } else {
    int64_t budget = c.point_budget_bytes;
    if (budget <= 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
      budget = (int64_t)(fr / 2);
    }
    h->cache_points = kPointSetBytes * (int64_t)c.n_orient * P2 <= budget;
    h->slice_sets = !h->cache_points && kSliceSetBytes * (int64_t)c.n_orient * P2 <= budget;
  }
  if (c.keep_slices >= 0) {
    h->keep_slices = c.keep_slices == 1;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = 0;
    h->keep_slices = (double)c.n_orient * P2 * sizeof(float) <= 0.25 * (double)fr;
  }
  const int64_t cap = (0x7fffffffLL) / P2;
  h->img_chunk = (int)std::min<int64_t>({(int64_t)c.max_images, c.img_chunk > 0 ? c.img_chunk : c.max_images, cap});
  int64_t max_pts = (int64_t)h->orient_chunk * P2;
  if (!h->cache_points) max_pts = std::max<int64_t>(max_pts, (int64_t)h->img_chunk * P2);
  int rc = spf_plan_create(&h->plan, c.N, c.qmax, c.eps, max_pts, c.device);
  if (rc == SPF_OK) rc = spf_matcher_create(&h->matcher, c.max_images, h->orient_chunk, P2, c.precision, c.topk,
                                            c.device);
  auto A = [&](void** p, size_t b, const char* w) {
    if (rc == SPF_OK) rc = dev_alloc(p, b, w);
  };
  const size_t n3 = (size_t)c.N * c.N * c.N;
  const size_t PT3 = h->plan ? (size_t)h->plan->PT * h->plan->PT * h->plan->PT : 0;
  A((void**)&h->quats_sorted, sizeof(float) * 4 * (size_t)c.n_orient, "driver orientations");
  A((void**)&h->qlab, sizeof(float) * 3 * (size_t)P2, "driver detector");
  A((void**)&h->order, sizeof(int) * (size_t)c.n_orient, "orientation order");
  A((void**)&h->inv, sizeof(int) * (size_t)c.n_orient, "inverse orientation order");
  A((void**)&h->slices, sizeof(float) * (size_t)(h->keep_slices ? c.n_orient : h->orient_chunk) * P2,
    h->keep_slices ? "slices of all chunks" : "slice chunk");
  if (rc == SPF_OK) rc = spf_matcher_set_rerank(h->matcher, h->keep_slices ? 1 : 0);
  // an FP32 copy of 16-bit images only for the consumers that need one
  if (c.precision == SPF_FP32 || !h->cache_points)
    A((void**)&h->img32, sizeof(float) * (size_t)c.max_images * P2, "FP32 images");
  A((void**)&h->best_sorted, sizeof(int) * (size_t)c.max_images, "matches (driver numbering)");
  A((void**)&h->best, sizeof(int) * (size_t)c.max_images, "matches");
  A((void**)&h->topk_tmp, sizeof(int) * (size_t)c.max_images * std::max(c.topk, 1), "top-k lists");
  A((void**)&h->rhs, sizeof(float) * n3, "right-hand side");
  A((void**)&h->khat, sizeof(float) * std::max<size_t>(PT3, 1), "Toeplitz kernel");
  A((void**)&h->x, sizeof(float) * n3, "merged model");
  A((void**)&h->err, sizeof(int), "driver error word");
  if (rc == SPF_OK && !h->cache_points && !h->slice_sets) {
    spf_points& S = h->stream_set;
    S.plan = h->plan;
    S.device = c.device;
    S.P2 = P2;
    S.flags = SPF_POINTS_SLICE_ONLY;
    const int64_t np = (int64_t)h->orient_chunk * P2;
    S.setN.max_subs = h->plan->g.bins.nbins + np / kSubPts + 1;
    A((void**)&S.setN.ids, sizeof(uint32_t) * (size_t)np, "streamed sorted ids");
    A((void**)&S.setN.subs, sizeof(int4) * (size_t)S.setN.max_subs, "streamed subproblems");
    A((void**)&S.setN.nsubs, 2 * sizeof(int), "streamed subproblem count");
    S.setN.max_bsubs = 8 * (int64_t)h->plan->g.bins.nbins + np / kSubPts + 1;
    A((void**)&S.setN.bsubs, sizeof(int4) * (size_t)S.setN.max_bsubs, "streamed block subproblems");
    A((void**)&S.setN.nbsubs, 2 * sizeof(int), "streamed block subproblem count");
  }
  if (rc == SPF_OK && c.host_image_type >= 0) {
    h->host_path = true;
    for (int b = 0; b < 2; ++b) {
      A((void**)&h->slotA[b], sizeof(float) * n3, "host-path model slot");
      A(&h->slotImg[b], image_elem(c.host_image_type) * (size_t)c.max_images * P2, "host-path image slot");
    }
    cudaError_t e = cudaSuccess;
    if (rc == SPF_OK) e = cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&h->copied[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->freed[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(h->freed[b], h->copy);
      if (e == cudaSuccess) e = cudaEventCreate(&h->up0[b]);
      if (e == cudaSuccess) e = cudaEventCreate(&h->up1[b]);
    }
    if (rc == SPF_OK && e != cudaSuccess) {
      set_error("driver streams and events: %s", cudaGetErrorString(e));
      rc = SPF_ERR_CUDA;
    }
  }
  if (rc == SPF_OK) {
    cudaError_t e = cudaMemset(h->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("driver set-up: %s", cudaGetErrorString(e));
      rc = SPF_ERR_CUDA;
    }
  }
  if (rc != SPF_OK) {
    mtip_free(h);
    return rc;
  }
  *out = h;
  return SPF_OK;
}

int spf_mtip_destroy(spf_mtip* h) {
  clear_error();
  if (!h) return SPF_OK;
  DevScope dev(h->cfg.device);
  cudaDeviceSynchronize();
  mtip_free(h);
  return SPF_OK;
}

int spf_mtip_info(const spf_mtip* h, int* cache_points, int* orient_chunk, int* img_chunk, int* keep_slices) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  if (keep_slices) *keep_slices = h->keep_slices ? 1 : 0;
  if (cache_points) *cache_points = h->cache_points ? 1 : h->slice_sets ? 2 : 0;
  if (orient_chunk) *orient_chunk = h->orient_chunk;
  if (img_chunk) *img_chunk = h->img_chunk;
  return SPF_OK;
}

int spf_morton_order(const float* quats_host, int M, int32_t* order_host) {
  clear_error();
  SPF_CHECK_ARG(M >= 0 && (M == 0 || (quats_host && order_host)), "bad arguments");
  std::vector<float> q(quats_host, quats_host + 4 * (size_t)M);
  const std::vector<int> order = morton_order(q, M);
  std::copy(order.begin(), order.end(), order_host);
  return SPF_OK;
}

spf_plan* spf_mtip_plan(spf_mtip* h) { return h ? h->plan : nullptr; }
spf_matcher* spf_mtip_matcher(spf_mtip* h) { return h ? h->matcher : nullptr; }

int spf_mtip_status(spf_mtip* h) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_TRY(spf_plan_status(h->plan));
  SPF_TRY(spf_matcher_status(h->matcher));
  DevScope dev(h->cfg.device);
  int e = 0;
  SPF_CUDA(cudaMemcpy(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost));
  SPF_CUDA(cudaMemset(h->err, 0, sizeof(int)));
  if (e) {
    set_error("driver error word 0x%x (4: an orientation index outside the set)", e);
    return SPF_ERR_ARG;
  }
  return SPF_OK;
}

int spf_mtip_set_orientations(spf_mtip* h, const float* quats, const float* q_lab, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_CHECK_ARG(quats && q_lab, "NULL pointer");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  const int M = h->cfg.n_orient, P2 = h->cfg.P2;
  std::vector<float> q(4 * (size_t)M);
  SPF_CUDA(cudaMemcpyAsync(q.data(), quats, sizeof(float) * q.size(), cudaMemcpyDeviceToHost, s));
  SPF_CUDA(cudaStreamSynchronize(s));
  const std::vector<int> order = morton_order(q, M);
  std::vector<int> inv(M);
  std::vector<float> qs(4 * (size_t)M);
  for (int i = 0; i < M; ++i) {
    inv[order[i]] = i;
    for (int a = 0; a < 4; ++a) qs[4 * (size_t)i + a] = q[4 * (size_t)order[i] + a];
  }
  h->have_set = false;
  free_sets(h);
  SPF_CUDA(cudaMemcpyAsync(h->order, order.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s));
  SPF_CUDA(cudaMemcpyAsync(h->inv, inv.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s));
  SPF_CUDA(cudaMemcpyAsync(h->quats_sorted, qs.data(), sizeof(float) * qs.size(), cudaMemcpyHostToDevice, s));
  SPF_CUDA(cudaMemcpyAsync(h->qlab, q_lab, sizeof(float) * 3 * (size_t)P2, cudaMemcpyDeviceToDevice, s));
  if (h->cache_points) {
    for (int c0 = 0; c0 < M; c0 += h->orient_chunk) {
      const int m = std::min(h->orient_chunk, M - c0);
      spf_points* p = nullptr;
      SPF_TRY(spf_points_create(&p, h->plan, h->quats_sorted + 4 * (size_t)c0, m, h->qlab, P2, 0, stream));
      h->sets.push_back(p);
    }
    const size_t n = h->sets.size();
    std::vector<uint32_t*> it(n);
    std::vector<float*> ct(n), nt(n);
    for (size_t c = 0; c < n; ++c) {
      it[c] = h->sets[c]->invN;
      ct[c] = h->sets[c]->cls;
      nt[c] = h->sets[c]->cnt;
    }
    SPF_TRY(dev_alloc((void**)&h->inv_tab, sizeof(uint32_t*) * n, "point-set table"));
    SPF_TRY(dev_alloc((void**)&h->cls_tab, sizeof(float*) * n, "point-set table"));
    SPF_TRY(dev_alloc((void**)&h->cnt_tab, sizeof(float*) * n, "point-set table"));
    SPF_CUDA(cudaMemcpyAsync(h->inv_tab, it.data(), sizeof(uint32_t*) * n, cudaMemcpyHostToDevice, s));
    SPF_CUDA(cudaMemcpyAsync(h->cls_tab, ct.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, s));
    SPF_CUDA(cudaMemcpyAsync(h->cnt_tab, nt.data(), sizeof(float*) * n, cudaMemcpyHostToDevice, s));
    SPF_CUDA(cudaStreamSynchronize(s));
  } else if (h->slice_sets) {
    for (int c0 = 0; c0 < M; c0 += h->orient_chunk) {
      const int m = std::min(h->orient_chunk, M - c0);
      spf_points* p = nullptr;
      SPF_TRY(spf_points_create(&p, h->plan, h->quats_sorted + 4 * (size_t)c0, m, h->qlab, P2,
                                SPF_POINTS_SLICE_ONLY, stream));
      h->sets.push_back(p);
    }
  } else {
    h->stream_set.qlab = h->qlab;
  }
  SPF_CUDA(cudaStreamSynchronize(s));   // the host copies above are freed on return
  h->have_set = true;
  return SPF_OK;
}

int spf_mtip_set_mask(spf_mtip* h, const float* D, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  SPF_TRY(spf_matcher_set_mask(h->matcher, D, stream));
  h->D = D;
  h->d_sum = (double)h->cfg.P2;
  if (D) {
    std::vector<float> w(h->cfg.P2);
    SPF_CUDA(cudaMemcpyAsync(w.data(), D, sizeof(float) * w.size(), cudaMemcpyDeviceToHost, s));
    SPF_CUDA(cudaStreamSynchronize(s));
    double t = 0.0;
    for (float v : w) {
      SPF_CHECK_ARG(v >= 0.f, "pixel weights must be >= 0");
      t += v;
    }
    h->d_sum = t;
  }
  return SPF_OK;
}

int spf_mtip_match(spf_mtip* h, const float* A, const void* images, int image_type, int n_img, float img_scale,
                   int32_t* best, float* best_d, float* second_d, int32_t* topk_idx, float* topk_d, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, true));
  SPF_TRY(check_images(h, images, image_type, n_img));
  SPF_CHECK_ARG(A && best, "NULL pointer");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  ImgIn img;
  SPF_TRY(images_in(h, images, image_type, n_img, true, false, &img, s));
  SPF_TRY(match_core(h, A, img, n_img, img_scale, s));
  SPF_TRY(spf_matcher_results(h->matcher, h->best_sorted, best_d, second_d, topk_idx ? h->topk_tmp : nullptr,
                              topk_d, stream));
  SPF_TRY(remap(h->best_sorted, n_img, h->order, h->cfg.n_orient, best, h->err, s));
  if (topk_idx)
    SPF_TRY(remap(h->topk_tmp, (int64_t)n_img * h->cfg.topk, h->order, h->cfg.n_orient, topk_idx, h->err, s));
  return SPF_OK;
}

int spf_mtip_merge(spf_mtip* h, const void* images, int image_type, int n_img, float img_scale, const int32_t* best,
                   float* rhs, float* kernel_hat, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, true));
  SPF_TRY(check_images(h, images, image_type, n_img));
  SPF_CHECK_ARG(best && rhs && kernel_hat, "NULL pointer");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  ImgIn img;
  SPF_TRY(images_in(h, images, image_type, n_img, false, true, &img, s));
  SPF_TRY(remap(best, n_img, h->inv, h->cfg.n_orient, h->best_sorted, h->err, s));
  return merge_core(h, img, n_img, img_scale, h->best_sorted, rhs, kernel_hat, s);
}

int spf_mtip_solve(spf_mtip* h, const float* rhs, const float* kernel_hat, const float* x0, double lam_rel,
                   int64_t n_img_total, int cg_iters, float* x, double* lambda_out, double* res_hist, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_CHECK_ARG(rhs && kernel_hat && x0 && x, "NULL pointer");
  SPF_CHECK_ARG(lam_rel > 0.0 && n_img_total >= 1 && cg_iters >= 0, "lam_rel > 0, n_img_total >= 1, cg_iters >= 0");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  return solve_core(h, rhs, kernel_hat, x0, lam_rel, n_img_total, cg_iters, x, lambda_out, res_hist,
                    as_stream(stream));
}

int spf_mtip_iteration(spf_mtip* h, const float* A, const void* images, int image_type, int n_img, float img_scale,
                       int cg_iters, double lam_rel, int32_t* best, float* x, double* lambda_out, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, true));
  SPF_TRY(check_images(h, images, image_type, n_img));
  SPF_CHECK_ARG(A && x, "NULL pointer");
  SPF_CHECK_ARG(lam_rel > 0.0 && cg_iters >= 0, "lam_rel > 0 and cg_iters >= 0 required");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  ImgIn img;
  SPF_TRY(images_in(h, images, image_type, n_img, true, true, &img, s));
  SPF_TRY(match_core(h, A, img, n_img, img_scale, s));
  SPF_TRY(spf_matcher_results(h->matcher, h->best_sorted, nullptr, nullptr, nullptr, nullptr, stream));
  SPF_TRY(remap(h->best_sorted, n_img, h->order, h->cfg.n_orient, best ? best : h->best, h->err, s));
  SPF_TRY(merge_core(h, img, n_img, img_scale, h->best_sorted, h->rhs, h->khat, s));
  return solve_core(h, h->rhs, h->khat, A, lam_rel, n_img, cg_iters, x, lambda_out, nullptr, s);
}

int spf_mtip_iteration_host(spf_mtip* h, const float* A_host, const void* images_host, int image_type, int n_img,
                            float img_scale, int cg_iters, double lam_rel, int32_t* best_host, float* x_host,
                            double* lambda_out, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, true));
  SPF_TRY(check_upload(h, image_type, images_host, n_img));
  SPF_CHECK_ARG(A_host && best_host && x_host, "NULL pointer");
  SPF_CHECK_ARG(lam_rel > 0.0 && cg_iters >= 0, "lam_rel > 0 and cg_iters >= 0 required");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  cudaStream_t s = as_stream(stream);
  const size_t n3 = (size_t)h->cfg.N * h->cfg.N * h->cfg.N;
  int b = 0;
  SPF_TRY(upload_slot(h, A_host, images_host, image_type, n_img, s, &b));
  SPF_TRY(spf_mtip_iteration(h, h->slotA[b], h->slotImg[b], image_type, n_img, img_scale, cg_iters, lam_rel,
                             h->best, h->x, lambda_out, stream));
  SPF_CUDA(cudaMemcpyAsync(best_host, h->best, sizeof(int) * (size_t)n_img, cudaMemcpyDeviceToHost, s));
  SPF_CUDA(cudaMemcpyAsync(x_host, h->x, sizeof(float) * n3, cudaMemcpyDeviceToHost, s));
  SPF_CUDA(cudaEventRecord(h->freed[b], s));
  return SPF_OK;
}

int spf_mtip_upload_host(spf_mtip* h, const float* A_host, const void* images_host, int image_type, int n_img,
                         float** A_dev, const void** images_dev, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_TRY(check_upload(h, image_type, images_host, n_img));
  SPF_CHECK_ARG(A_host && A_dev && images_dev, "NULL pointer");
  SPF_CHECK_ARG(h->held_slot < 0, "the previous upload was not released (spf_mtip_release_upload)");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  int b = 0;
  SPF_TRY(upload_slot(h, A_host, images_host, image_type, n_img, as_stream(stream), &b));
  h->held_slot = b;
  *A_dev = h->slotA[b];
  *images_dev = h->slotImg[b];
  return SPF_OK;
}

int spf_mtip_release_upload(spf_mtip* h, void* stream) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_CHECK_ARG(h->held_slot >= 0, "no upload is held");
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  SPF_CUDA(cudaEventRecord(h->freed[h->held_slot], as_stream(stream)));
  h->held_slot = -1;
  return SPF_OK;
}

int spf_mtip_set_upload(spf_mtip* h, int mode) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_CHECK_ARG(mode == SPF_UPLOAD_COPY || mode == SPF_UPLOAD_SM, "unknown upload mode %d", mode);
  h->upload_mode = mode;
  return SPF_OK;
}

int spf_mtip_last_upload_ms(spf_mtip* h, float* ms) {
  clear_error();
  SPF_TRY(check_handle(h, false));
  SPF_CHECK_ARG(ms != nullptr, "NULL pointer");
  *ms = -1.f;
  if (!h->host_path || h->host_calls == 0) return SPF_OK;
  DevScope dev(h->cfg.device);
  if (dev.rc != SPF_OK) return dev.rc;
  const int b = (int)((h->host_calls - 1) & 1);
  SPF_CUDA(cudaEventSynchronize(h->up1[b]));
  SPF_CUDA(cudaEventElapsedTime(ms, h->up0[b], h->up1[b]));
  return SPF_OK;
}

}  // extern "C"
