// Internal layout of a NUFFT / merge plan.
#pragma once

#include "common.h"

namespace spf {

// Counting sort of nonuniform points by the fine-grid cell of their tap
// origin, in bin-major order: key = bin * 64 + (cell within the 4^3 bin).
// Points with equal keys share their whole w^3 tap window. Each bin's points
// are then cut into subproblems of at most kSubPts points.
constexpr int kBinLog = 2;
constexpr int kBin = 1 << kBinLog;
constexpr int kBinCells = kBin * kBin * kBin;
constexpr int kSubPts = 4096;
constexpr int kScanBlocks = 1024;

struct BinSort {
  int nb[3] = {0, 0, 0};     // bins per axis
  int nbins = 0;
  int64_t nkeys = 0;         // nbins * 512
  int64_t max_subs = 0;
  int* count = nullptr;      // nkeys points per key
  int* fill = nullptr;       // nkeys scatter cursors
  int* start = nullptr;      // nkeys + 1 exclusive scan
  int* block_sums = nullptr; // kScanBlocks scan partials
  int4* subs = nullptr;      // max_subs: (bin, first, npts, 0)
  int* nsubs = nullptr;      // [0] subproblem count, [1] work cursor
};

// ES kernel weights as polynomials: tap d (0 <= d < w) of a point at
// fractional offset x in [0, 1) has weight sum_i c[d][i] t^i, t = 2x - 1,
// of degree es_degree(w) (see es_poly).
struct EsPoly {
  float c[8][10];
  float2 c2[8][10];   // each coefficient twice: two points or axes per packed FMA
  // Mirror form: tap w-1-d is tap d at -t, so for d < (w+1)/2 the taps are
  // E_d(t^2) +- t O_d(t^2) with the even and odd coefficient halves
  // e2[d][k] = c[d][2k], o2[d][k] = c[d][2k+1] (each twice, packed FMAs).
  float2 e2[4][5];
  float2 o2[4][5];
};
__host__ __device__ constexpr int es_degree(int w) { return w < 7 ? w + 1 : w; }

struct Grid {
  int nf = 0;                // fine grid side
  int n_modes = 0;           // modes per axis (odd)
  float cells_per_q = 0.f;   // fine-grid cells per unit physical q
  float* deconv = nullptr;   // n_modes deconvolution factors p_k (device)
  float* real = nullptr;     // nf^3 real grid (spread target / type-2 FFT output)
  float* halo = nullptr;     // 4 x-shifted periodic copies of `real` with a w/2 halo (interp source)
  float2* cube = nullptr;    // nf^3 complex work cube
  FFT3 fft;
  BinSort bins;
};

// A sorted point set of one grid: ids in sorted order, its subproblems, and
// [count, work cursor] of the subproblem list.
struct SortedSet {
  uint32_t* ids = nullptr;
  int4* subs = nullptr;
  int* nsubs = nullptr;
  int64_t max_subs = 0;
  // optional: the same points cut per 2^3 cell block (interpolation's
  // subproblems), (block, first, npts, 0)
  int4* bsubs = nullptr;
  int* nbsubs = nullptr;
  int64_t max_bsubs = 0;
};

}  // namespace spf

struct spf_plan {
  int device = 0;
  int N = 0, Mh = 0;
  double qmax = 0, eps = 0;
  int w = 0;
  double beta = 0;
  spf::EsPoly poly;           // polynomial form of the kernel for the device
  double radians_per_q = 0;   // 2 pi dr
  int64_t max_points = 0;
  spf::Grid g;                // N modes (slicing, RHS)
  spf::Grid gT;               // 2N-1 modes (Toeplitz kernel)
  int PT = 0;                 // circulant embedding side
  float2* cubeP = nullptr;    // PT^3 complex work
  float* realP = nullptr;     // PT^3 real scratch
  spf::FFT3 fftP;
  uint32_t* sorted = nullptr; // max_points sorted point ids
  // CG state
  float* cg_r = nullptr;
  float* cg_p = nullptr;
  float* cg_Ap = nullptr;
  double* cg_sc = nullptr;    // [rr, pAp, alpha, beta, rr_new, res]
  double* cg_part = nullptr;  // per-block partial sums
  unsigned* cg_count = nullptr;  // blocks done with a fused reduction (last one finalises)
  int* err = nullptr;         // device error word (bit 1: point outside its bin)
  double* grad_part = nullptr;   // gradient merge: per-block partials (2 per block)
  unsigned* grad_count = nullptr;
  double* grad_sc = nullptr;     // [g.g, g.Hg]
  bool merge_open = false;    // a deferred merge holds partial sums in the fine grids
};

// Orientations x pixels of a fixed orientation set, sorted once for both grids.
struct spf_points {
  spf_plan* plan = nullptr;
  int device = 0;
  int M = 0, P2 = 0;
  int flags = 0;              // SPF_POINTS_SLICE_ONLY: setN only
  float* quats = nullptr;     // M x 4 copy
  float* qlab = nullptr;      // P2 x 3 copy
  spf::SortedSet setN;        // N-mode grid (slicing, right-hand side)
  spf::SortedSet setT;        // (2N-1)-mode grid (Toeplitz kernel)
  uint32_t* invN = nullptr;   // position of point id in setN's sorted order
  float* cls = nullptr;       // class sums of weighted images, in setN's sorted order
  float* cnt = nullptr;       // M class counts
  bool cls_zero = false;      // cls holds zeros only (the right-hand-side spread consumed it)
};

namespace spf {
// Merge modes (nufft.cu): clear the fine grid before spreading, transform it
// into the output after.
constexpr int kMergeClear = 1;
constexpr int kMergeFinish = 2;
constexpr int kMergeSumsDone = 4;   // point sets: class sums already formed (class_sums_sets)
// Host side of the ES kernel set-up (es.cu).
void es_params(double eps, int* w, double* beta);
void es_poly(int w, double beta, EsPoly* out);
int fine_size(int n_modes, int w);
int smooth_even_at_least(int n);
void deconv_factors(int n_modes, int nf, int w, double beta, double* out);
}  // namespace spf
