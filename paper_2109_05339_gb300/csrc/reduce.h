// FP64 block reductions and the conjugate-gradient scalar update, shared by
// the kernels that end a CG inner product (the Toeplitz convolution's last
// pass and the CG vector kernels). Each translation unit gets its own copy.
#pragma once

#include <cuda_runtime.h>

namespace spf {
namespace {

__device__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// CG scalars from the reduced sum s: mode 0 r.r (and beta = 0), mode 1 p.Ap
// and alpha, mode 2 the new r.r and beta.
__device__ __forceinline__ void cg_scalars(double s, double* __restrict__ sc, int mode,
                                           double* __restrict__ res_out) {
  if (mode == 0) {
    sc[0] = s;
    sc[3] = 0.0;
  } else if (mode == 1) {
    sc[1] = s;
    sc[2] = s > 0.0 ? sc[0] / s : 0.0;
  } else {
    sc[4] = s;
    sc[3] = sc[0] > 0.0 ? s / sc[0] : 0.0;
    sc[0] = s;
  }
  sc[5] = sqrt(sc[0]);
  if (res_out) *res_out = sc[5];
}

// Store this block's partial; the last block to finish sums all partials (in
// the fixed order of finalize_kernel: the same result) and updates the CG
// scalars, so no separate reduction launch is needed.
__device__ void partial_and_finalize(double s_block, double* __restrict__ part, double* __restrict__ sc,
                                     int mode, double* __restrict__ res_out, unsigned* __restrict__ count) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s_block;
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(part + i);
  const double s = block_sum(v);
  if (threadIdx.x == 0) {
    cg_scalars(s, sc, mode, res_out);
    *count = 0u;
  }
}

}  // namespace
}  // namespace spf
