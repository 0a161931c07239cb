// Host-side set-up of the exponential-of-semicircle (ES) NUFFT kernel.
//
// The paper slices and merges with the FINUFFT / cuFINUFFT libraries
// (Sec. III-A), whose published method spreads with
//   phi(z) = exp(beta (sqrt(1 - z^2) - 1)),  |z| <= 1,
// over w fine-grid cells, w = ceil(log10(1/eps)) + 1, beta = 2.30 w, on a
// grid upsampled by 2. Deconvolution divides mode k by the kernel's Fourier
// transform; per axis the factor is
//   p_k = 2 / (w int_{-1}^{1} phi(z) cos(k a z) dz),  a = w pi / n_f,
// evaluated here in FP64 by Gauss-Legendre quadrature (nodes from Newton's
// method on the Legendre recurrence) and cast to float for the kernels.
#include <cmath>
#include <vector>

#include "plan.h"

namespace spf {

void es_params(double eps, int* w, double* beta) {
  *w = (int)std::ceil(std::log10(1.0 / eps)) + 1;
  *beta = 2.30 * (*w);
}

int smooth_even_at_least(int n) {
  if (n < 2) n = 2;
  if (n % 2) ++n;
  for (;; n += 2) {
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    while (m % 5 == 0) m /= 5;
    if (m == 1) return n;
  }
}

int fine_size(int n_modes, int w) { return smooth_even_at_least(std::max(2 * n_modes, 2 * w)); }

// Gauss-Legendre nodes and weights on [-1, 1].
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
  x.assign(n, 0.0);
  wt.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      // P_n(z) and P_n'(z) by the three-term recurrence
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1.0 : p1;
      double pm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    double wi = 2.0 / ((1.0 - z * z) * dp * dp);
    wt[i] = wi;
    wt[n - 1 - i] = wi;
  }
}

// Polynomial form of the kernel for the device. A point u has its first tap
// at l0 = ceil(u - w/2); with x = l0 - (u - w/2) in [0, 1) tap d sits at
// z_d = (2x + 2d - w) / w. Each phi(z_d(x)) is replaced by its Chebyshev
// interpolant of degree es_degree(w) in t = 2x - 1 (nodes t_k = cos(pi (k +
// 1/2) / (degree + 1))), rewritten in powers of t for Horner's rule. This is
// the piecewise-polynomial kernel evaluation of the FINUFFT library's
// published method (Barnett, Magland and af Klinteberg, SIAM J. Sci. Comput.
// 41 (2019), Sec. 3.1.1), with coefficients computed here in FP64. The
// largest absolute error (kernel peak 1) is 5e-6, 6e-7, 1.5e-7, 7e-9 for
// w = 5, 6, 7, 8, i.e. below eps / 6 for eps = 10^(1 - w).
void es_poly(int w, double beta, EsPoly* out) {
  *out = EsPoly();
  const int P = es_degree(w), n = P + 1;
  if (w < 1 || w > 8) return;
  // taps d < (w+1)/2 are interpolated; tap w-1-d is tap d at -t (the
  // kernel is even and the taps are placed symmetrically), so its
  // coefficients are c[d][i] (-1)^i exactly
  const int half = (w + 1) / 2;
  for (int d = 0; d < half; ++d) {
    std::vector<double> f(n), a(n, 0.0);
    for (int k = 0; k < n; ++k) {
      const double t = std::cos(M_PI * (k + 0.5) / n), x = 0.5 * (t + 1.0);
      const double z = (2.0 * x + 2.0 * d - w) / w;
      const double s = 1.0 - z * z;
      f[k] = std::fabs(z) <= 1.0 ? std::exp(beta * (std::sqrt(s > 0 ? s : 0) - 1.0)) : 0.0;
    }
    for (int j = 0; j < n; ++j) {
      double acc = 0.0;
      for (int k = 0; k < n; ++k) acc += f[k] * std::cos(j * M_PI * (k + 0.5) / n);
      a[j] = (j == 0 ? 1.0 : 2.0) * acc / n;
    }
    // sum_j a_j T_j(t) in powers of t: T_0 = 1, T_1 = t, T_j+1 = 2t T_j - T_j-1
    std::vector<double> m(n, 0.0), t0(n, 0.0), t1(n, 0.0), t2(n, 0.0);
    t0[0] = 1.0;
    if (n > 1) t1[1] = 1.0;
    for (int i = 0; i < n; ++i) m[i] += a[0] * t0[i];
    if (n > 1)
      for (int i = 0; i < n; ++i) m[i] += a[1] * t1[i];
    for (int j = 2; j < n; ++j) {
      for (int i = 0; i < n; ++i) t2[i] = (i > 0 ? 2.0 * t1[i - 1] : 0.0) - t0[i];
      for (int i = 0; i < n; ++i) m[i] += a[j] * t2[i];
      t0 = t1;
      t1 = t2;
    }
    if (2 * d + 1 == w) {   // the middle tap is even in t
      for (int i = 1; i < n; i += 2) m[i] = 0.0;
    }
    for (int i = 0; i < n; ++i) {
      const float c = (float)m[i], cm = (i & 1) ? -c : c;
      out->c[d][i] = c;
      out->c2[d][i] = make_float2(c, c);
      out->c[w - 1 - d][i] = cm;
      out->c2[w - 1 - d][i] = make_float2(cm, cm);
      if (i / 2 < 5) {
        if (i & 1) out->o2[d][i / 2] = make_float2(c, c);
        else out->e2[d][i / 2] = make_float2(c, c);
      }
    }
  }
}

void deconv_factors(int n_modes, int nf, int w, double beta, double* out) {
  const int nq = 256;
  std::vector<double> z, wq;
  gauss_legendre(nq, z, wq);
  std::vector<double> f(nq);
  for (int q = 0; q < nq; ++q) {
    double s = 1.0 - z[q] * z[q];
    f[q] = wq[q] * std::exp(beta * (std::sqrt(s > 0 ? s : 0) - 1.0));
  }
  const int Mh = (n_modes - 1) / 2;
  const double a = w * M_PI / nf;
  for (int k = -Mh; k <= Mh; ++k) {
    double J = 0.0;
    for (int q = 0; q < nq; ++q) J += f[q] * std::cos(k * a * z[q]);
    out[k + Mh] = 2.0 / (w * J);
  }
}

}  // namespace spf
