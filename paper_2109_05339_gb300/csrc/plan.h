// Internal layout of a NUFFT / merge plan.
#pragma once

#include "common.h"

namespace spf {

// Bin sort of nonuniform points into fine-grid boxes of kBin^3 cells, split
// into subproblems of at most kSubPts points (one CTA each).
constexpr int kBin = 8;
constexpr int kSubPts = 2048;

struct BinSort {
  int nb[3] = {0, 0, 0};     // bins per axis
  int nbins = 0;
  int64_t max_subs = 0;
  int* count = nullptr;      // nbins
  int* fill = nullptr;       // nbins
  int* start = nullptr;      // nbins + 1
  int* sub_start = nullptr;  // nbins + 1
  int4* subs = nullptr;      // max_subs: (bin, first, npts, 0)
  int* nsubs = nullptr;      // 1
};

struct Grid {
  int nf = 0;                // fine grid side
  int n_modes = 0;           // modes per axis (odd)
  float cells_per_q = 0.f;   // fine-grid cells per unit physical q
  float* deconv = nullptr;   // n_modes deconvolution factors p_k (device)
  float* real = nullptr;     // nf^3 real grid (spread target / interp source)
  float2* cube = nullptr;    // nf^3 complex work cube
  FFT3 fft;
  BinSort bins;
};

}  // namespace spf

struct spf_plan {
  int device = 0;
  int N = 0, Mh = 0;
  double qmax = 0, eps = 0;
  int w = 0;
  double beta = 0;
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
  int* err = nullptr;         // device error word (bit 1: point outside its bin)
};

namespace spf {
// Host side of the ES kernel set-up (es.cu).
void es_params(double eps, int* w, double* beta);
int fine_size(int n_modes, int w);
int smooth_even_at_least(int n);
void deconv_factors(int n_modes, int nf, int w, double beta, double* out);
}  // namespace spf
