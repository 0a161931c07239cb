// Orientation matching without any device allocation.
//
// Some callers cannot allocate device memory at the point where they match:
// code embedded in a host framework that owns the device memory pool and
// forbids cudaMalloc next to it (the framework's allocator must see every
// byte), or real-time acquisition loops that must not touch the allocator,
// whose calls can block and synchronise the device. This entry point runs the
// same FP32 matching kernels as spf_matcher_* (fused distance + running
// top-8, exact FP32 re-rank of the 8 candidates), but its scratch -- row
// norms, candidate lists and running lists -- lives in one statically sized
// device array that every GPU loading this library holds until exit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "match.h"

namespace spf {
int simt_splits(int n_img, int n_orient, int n_sms);
int simt_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                cudaStream_t s);
int row_norms(const float* src, int rows, int P2, float scale, float* out, cudaStream_t s);
int state_reset(spf_matcher* m, cudaStream_t s);
int rerank_launch(spf_matcher* m, const float* slices, int n_orient, int orient_offset, int nsplit,
                  cudaStream_t s);
int results_launch(spf_matcher* m, int32_t* best_idx, float* best_d, float* second_d,
                   int32_t* topk_idx, float* topk_d, cudaStream_t s);
}  // namespace spf

namespace {

constexpr int kStaticMaxImages = SPF_STATIC_MATCH_MAX_IMAGES;
constexpr int kStaticMaxOrient = SPF_STATIC_MATCH_MAX_ORIENT;
constexpr int kStaticTopk = 8;

// byte offsets of the pieces inside the scratch array (each 256-aligned)
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffX2 = 0;
constexpr size_t kOffY2 = kOffX2 + align256(sizeof(float) * kStaticMaxImages);
constexpr size_t kOffCandV = kOffY2 + align256(sizeof(float) * kStaticMaxOrient);
constexpr size_t kOffCandI =
    kOffCandV + align256(sizeof(float) * (size_t)kStaticMaxImages * kMaxSplits * kCand);
constexpr size_t kOffStD =
    kOffCandI + align256(sizeof(int) * (size_t)kStaticMaxImages * kMaxSplits * kCand);
constexpr size_t kOffStI = kOffStD + align256(sizeof(float) * (size_t)kStaticMaxImages * kStaticTopk);
constexpr size_t kScratchBytes = kOffStI + align256(sizeof(int) * (size_t)kStaticMaxImages * kStaticTopk);

static_assert(kScratchBytes == 4526080, "scratch size stated in include/spf.h");
static __device__ __align__(256) unsigned char g_match_scratch[kScratchBytes];

// Device address of g_match_scratch per device ordinal, with the CUDA
// context it was looked up in. In host code the symbol's name is only a
// host-side stand-in, so its address is looked up with the device current:
// once per device, and again whenever the current context is another one
// (after cudaDeviceReset, or a context the caller made current through the
// driver API), where the module -- and the array -- live elsewhere.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct ScratchAddr {
  CUcontext ctx = nullptr;
  void* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f);
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  SPF_CUDA(cudaGetDevice(&dev));
  SPF_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> g(g_mu);
  ScratchAddr& a = g_scratch[dev];
  CUcontext ctx = current_context();
  if (!a.ptr || !ctx || ctx != a.ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_match_scratch);
    if (e != cudaSuccess || !p) {
      spf::set_error("cudaGetSymbolAddress of the static matching scratch failed on device %d: %s",
                     dev, cudaGetErrorString(e));
      return SPF_ERR_CUDA;
    }
    a.ptr = p;
    a.ctx = current_context();   // the look-up made the runtime's context current
  }
  *out = static_cast<unsigned char*>(a.ptr);
  return SPF_OK;
}

}  // namespace

using namespace spf;

extern "C" int spf_match_orientations_static(const float* images, int n_img, float img_scale,
                                             const float* slices, int n_orient, int P2,
                                             int32_t* best_idx, float* best_d, float* second_d,
                                             void* stream) {
  clear_error();
  SPF_CHECK_ARG(n_img >= 0 && n_img <= kStaticMaxImages,
                "n_img %d exceeds the static-scratch limit of %d images", n_img, kStaticMaxImages);
  SPF_CHECK_ARG(n_orient >= 0 && n_orient <= kStaticMaxOrient,
                "n_orient %d exceeds the static-scratch limit of %d model images", n_orient,
                kStaticMaxOrient);
  SPF_CHECK_ARG(P2 > 0, "P2 must be positive");
  SPF_CHECK_ARG(n_img == 0 || (images && best_idx && best_d && second_d), "NULL pointer");
  SPF_CHECK_ARG(n_img == 0 || n_orient == 0 || slices, "slices is NULL");
  if (n_img == 0) return SPF_OK;
  unsigned char* base = nullptr;
  SPF_TRY(scratch_for_current_device(&base));
  cudaStream_t s = as_stream(stream);

  // A matcher view whose buffers all point into the static array.
  spf_matcher m;
  int dev = 0;
  SPF_CUDA(cudaGetDevice(&dev));
  m.device = dev;
  cudaDeviceGetAttribute(&m.n_sms, cudaDevAttrMultiProcessorCount, dev);
  m.max_images = kStaticMaxImages;
  m.max_orient = kStaticMaxOrient;
  m.P2 = P2;
  m.precision = SPF_FP32;
  m.topk = kStaticTopk;
  m.n_img = n_img;
  m.img_scale = img_scale;
  m.images = images;
  m.x2 = reinterpret_cast<float*>(base + kOffX2);
  m.y2 = reinterpret_cast<float*>(base + kOffY2);
  m.cand_v = reinterpret_cast<float*>(base + kOffCandV);
  m.cand_i = reinterpret_cast<int*>(base + kOffCandI);
  m.st_d = reinterpret_cast<float*>(base + kOffStD);
  m.st_i = reinterpret_cast<int*>(base + kOffStI);

  // The running lists keep the previous call's contents: reset them.
  SPF_TRY(row_norms(images, n_img, P2, img_scale, m.x2, s));
  SPF_TRY(state_reset(&m, s));
  if (n_orient > 0) {
    SPF_TRY(row_norms(slices, n_orient, P2, 1.f, m.y2, s));
    const int nsplit = simt_splits(n_img, n_orient, m.n_sms);
    SPF_TRY(simt_launch(&m, slices, n_orient, 0, nsplit, s));
    SPF_TRY(rerank_launch(&m, slices, n_orient, 0, nsplit, s));
  }
  return results_launch(&m, best_idx, best_d, second_d, nullptr, nullptr, s);
}
