// Hand-written batched 3D FFT for 2/3/5-smooth cube sides (sm_103a).
//
// The uniform FFT inside the NUFFT (the cuFINUFFT calls of Sec. III-A) and
// the circulant convolution of the Toeplitz method (Sec. II-C) both need
// complex 3D transforms of sides 36..640. One kernel transforms a batch of
// 1D lines along one axis: the lines are staged through shared memory with
// coalesced global accesses (whole rows for the contiguous axis; tiles of 8
// or 16 neighbouring lines for the strided axes), transformed there by
// self-sorting (Stockham) radix-2/3/4/5/9 passes with twiddles from an FP64-
// built table, and written back in natural order. Three launches make a 3D
// transform. Lines known to be all zero (zero-padded input) or whose output
// is not needed (cropped output) are skipped.
//
// Real data (the spread grids of type 1, the Toeplitz convolution of the
// real CG vectors) start with a real-input pass along x on the precompiled
// sides: two real rows form one complex line, the two half spectra are
// separated after the line FFT, and the y and z passes then run on the
// half spectrum only (the Toeplitz product with its real, even kernel
// inside the z pass). The convolution ends with the matching inverse row
// pass, which applies the CG operator's epilogue.
#include <cmath>
#include <vector>

#include "common.h"
#include "reduce.h"

namespace spf {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxElems = 4096;                       // elements per CTA tile
constexpr int kEPT = kMaxElems / kThreads;            // 16 per thread

struct LineSet {
  // Lines of one pass are indexed by (a, b); b is the fast line coordinate.
  // Each coordinate runs over at most two half-open ranges.
  int a_lo[2], a_hi[2];
  int b_lo[2], b_hi[2];
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by sign * i
__device__ __forceinline__ float2 mul_si(float2 a, float sign) { return make_float2(-sign * a.y, sign * a.x); }

template <int R>
__device__ __forceinline__ void dft(float2* v, float sign);

template <>
__device__ __forceinline__ void dft<2>(float2* v, float) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<3>(float2* v, float sign) {
  const float h = 0.86602540378443864676f;  // sqrt(3)/2
  float2 s = cadd(v[1], v[2]);
  float2 d = csub(v[1], v[2]);
  float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
  float2 t = mul_si(make_float2(h * d.x, h * d.y), sign);
  v[0] = cadd(v[0], s);
  v[1] = cadd(m, t);
  v[2] = csub(m, t);
}

template <>
__device__ __forceinline__ void dft<4>(float2* v, float sign) {
  float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
  float2 c = cadd(v[1], v[3]), d = mul_si(csub(v[1], v[3]), sign);
  v[0] = cadd(a, c);
  v[2] = csub(a, c);
  v[1] = cadd(b, d);
  v[3] = csub(b, d);
}

template <>
__device__ __forceinline__ void dft<5>(float2* v, float sign) {
  const float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
  const float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
  const float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
  const float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
  float2 a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  float2 a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  float2 x0 = v[0];
  float2 r1 = make_float2(x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y);
  float2 r2 = make_float2(x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y);
  float2 i1 = mul_si(make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y), sign);
  float2 i2 = mul_si(make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y), sign);
  v[0] = make_float2(x0.x + a1.x + a2.x, x0.y + a1.y + a2.y);
  v[1] = cadd(r1, i1);
  v[4] = csub(r1, i1);
  v[2] = cadd(r2, i2);
  v[3] = csub(r2, i2);
}

// 9-point DFT as 3 x 3: with n = 3 n1 + n2 and k = k1 + 3 k2,
// X[k1 + 3 k2] = sum_n2 w3^(n2 k2) [w9^(n2 k1) sum_n1 x[3 n1 + n2] w3^(n1 k1)],
// w_m = exp(sign 2 pi i / m).
template <>
__device__ __forceinline__ void dft<9>(float2* v, float sign) {
  const float c1 = 0.76604444311897803520f, s1 = 0.64278760968653932632f;   // 2 pi / 9
  const float c2 = 0.17364817766693034885f, s2 = 0.98480775301220805936f;   // 4 pi / 9
  const float c4 = -0.93969262078590838405f, s4 = 0.34202014332566873304f;  // 8 pi / 9
  float2 a[3] = {v[0], v[3], v[6]}, b[3] = {v[1], v[4], v[7]}, c[3] = {v[2], v[5], v[8]};
  dft<3>(a, sign);
  dft<3>(b, sign);
  dft<3>(c, sign);
  b[1] = cmul(b[1], make_float2(c1, sign * s1));
  b[2] = cmul(b[2], make_float2(c2, sign * s2));
  c[1] = cmul(c[1], make_float2(c2, sign * s2));
  c[2] = cmul(c[2], make_float2(c4, sign * s4));
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    float2 t[3] = {a[k1], b[k1], c[k1]};
    dft<3>(t, sign);
    v[k1] = t[0];
    v[k1 + 3] = t[1];
    v[k1 + 6] = t[2];
  }
}

// One self-sorting pass of radix R over `lines` lines of length n in `buf`.
// Butterfly j of a line reads elements j + r n/R, multiplies by
// w^{k r} (k = j mod Ns, w = exp(sign 2 pi i / (Ns R))), transforms, and
// writes to (j / Ns) Ns R + k + r Ns.
template <int R>
__device__ void stockham_pass(float2* buf, int n, int lines, int Ns, const float2* __restrict__ tw,
                              float sign) {
  constexpr int Q = (kEPT + R - 1) / R;
  const int nb_line = n / R;
  const int nb = lines * nb_line;
  const int tstep = n / (Ns * R);
  float2 v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int b = threadIdx.x + q * kThreads;
    if (b < nb) {
      int line = b / nb_line, j = b - line * nb_line;
      const float2* src = buf + line * n + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[r * nb_line];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    int b = threadIdx.x + q * kThreads;
    if (b < nb) {
      int line = b / nb_line, j = b - line * nb_line;
      int k = j % Ns;
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(&tw[(k * r * tstep) % n]);
          w.y *= -sign;  // table holds exp(-2 pi i m / n); sign=+1 conjugates
          v[q][r] = cmul(v[q][r], make_float2(w.x, w.y));
        }
      }
      dft<R>(v[q], sign);
      float2* dst = buf + line * n + (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

struct PassArgs {
  float2* data;          // complex cube (in place) unless in_real / out_real
  const float* in_real;  // optional real input (imaginary part zero)
  float* out_real;       // optional real-part output
  const float* post_mul; // optional real factor applied to outputs (same layout)
  int n;                 // line length
  int64_t es;            // element stride along the line
  int64_t sa, sb;        // strides of the line coordinates a and b
  LineSet ls;
  int in_lo[2], in_hi[2];  // positions along the line that are read; the rest count as zero
  int out_lo[2], out_hi[2];  // positions along the line that are written (the rest are not needed)
  int convolve;          // transform, multiply by post_mul, transform back (-sign)
  int64_t pm_es, pm_sa, pm_sb;  // strided convolution: post_mul strides (along the line, a, b)
  int lines_per_cta;     // contiguous: lines per CTA; strided: b-lines per CTA
  int nrad;
  int radix[16];
  const float2* tw;
  float sign;
};

__device__ __forceinline__ int range_count(int lo, int hi) { return hi > lo ? hi - lo : 0; }

// Position i of a line is read (else it counts as zero: pruned input).
__device__ __forceinline__ bool in_read_range(const PassArgs& A, int i) {
  return (i >= A.in_lo[0] && i < A.in_hi[0]) || (i >= A.in_lo[1] && i < A.in_hi[1]);
}

// Position i of a line is stored (else the next pass does not read it).
__device__ __forceinline__ bool in_write_range(const PassArgs& A, int i) {
  return (i >= A.out_lo[0] && i < A.out_hi[0]) || (i >= A.out_lo[1] && i < A.out_hi[1]);
}

// Map the i-th selected coordinate to its value, over two ranges.
__device__ __forceinline__ int pick(int i, const int* lo, const int* hi) {
  int c0 = range_count(lo[0], hi[0]);
  return i < c0 ? lo[0] + i : lo[1] + (i - c0);
}

__device__ void run_passes(const PassArgs& A, float2* buf, int lines) {
  int Ns = 1;
  for (int p = 0; p < A.nrad; ++p) {
    int R = A.radix[p];
    if (R == 4) stockham_pass<4>(buf, A.n, lines, Ns, A.tw, A.sign);
    else if (R == 2) stockham_pass<2>(buf, A.n, lines, Ns, A.tw, A.sign);
    else if (R == 3) stockham_pass<3>(buf, A.n, lines, Ns, A.tw, A.sign);
    else stockham_pass<5>(buf, A.n, lines, Ns, A.tw, A.sign);
    Ns *= R;
  }
}

// Lines along a stride-es axis, tile of `lines_per_cta` consecutive b values
// (b stride 1 = x) for one a; global accesses coalesced across b.
__global__ void __launch_bounds__(kThreads) fft_strided_kernel(PassArgs A) {
  extern __shared__ float2 sbuf[];
  const int n = A.n, T = A.lines_per_cta;
  int nb_sel = range_count(A.ls.b_lo[0], A.ls.b_hi[0]) + range_count(A.ls.b_lo[1], A.ls.b_hi[1]);
  int tiles_b = (nb_sel + T - 1) / T;
  int tile = blockIdx.x % tiles_b;
  int ai = blockIdx.x / tiles_b;
  int a = pick(ai, A.ls.a_lo, A.ls.a_hi);
  int first = tile * T;
  int nlines = min(T, nb_sel - first);
  const int64_t base_a = (int64_t)a * A.sa;
  // load: element (line l, position i) -> sbuf[l * n + i]
  for (int e = threadIdx.x; e < nlines * n; e += kThreads) {
    int l = e % nlines, i = e / nlines;
    int b = pick(first + l, A.ls.b_lo, A.ls.b_hi);
    int64_t g = base_a + (int64_t)b * A.sb + (int64_t)i * A.es;
    sbuf[l * n + i] = !in_read_range(A, i) ? make_float2(0.f, 0.f)
                      : A.in_real ? make_float2(A.in_real[g], 0.f) : A.data[g];
  }
  __syncthreads();
  run_passes(A, sbuf, nlines);
  for (int e = threadIdx.x; e < nlines * n; e += kThreads) {
    int l = e % nlines, i = e / nlines;
    if (!in_write_range(A, i)) continue;
    int b = pick(first + l, A.ls.b_lo, A.ls.b_hi);
    int64_t g = base_a + (int64_t)b * A.sb + (int64_t)i * A.es;
    float2 v = sbuf[l * n + i];
    if (A.post_mul) {
      float f = A.post_mul[g];
      v.x *= f;
      v.y *= f;
    }
    if (A.out_real) A.out_real[g] = v.x;
    else A.data[g] = v;
  }
}

// Lines along the contiguous axis; lines indexed by (a, b) with both strided.
__global__ void __launch_bounds__(kThreads) fft_contig_kernel(PassArgs A) {
  extern __shared__ float2 sbuf[];
  const int n = A.n, L = A.lines_per_cta;
  int na = range_count(A.ls.a_lo[0], A.ls.a_hi[0]) + range_count(A.ls.a_lo[1], A.ls.a_hi[1]);
  int nbs = range_count(A.ls.b_lo[0], A.ls.b_hi[0]) + range_count(A.ls.b_lo[1], A.ls.b_hi[1]);
  int total = na * nbs;
  int first = blockIdx.x * L;
  int nlines = min(L, total - first);
  for (int e = threadIdx.x; e < nlines * n; e += kThreads) {
    int l = e / n, i = e - l * n;
    int li = first + l;
    int a = pick(li / nbs, A.ls.a_lo, A.ls.a_hi);
    int b = pick(li % nbs, A.ls.b_lo, A.ls.b_hi);
    int64_t g = (int64_t)a * A.sa + (int64_t)b * A.sb + i;
    sbuf[e] = !in_read_range(A, i) ? make_float2(0.f, 0.f)
              : A.in_real ? make_float2(A.in_real[g], 0.f) : A.data[g];
  }
  __syncthreads();
  run_passes(A, sbuf, nlines);
  for (int e = threadIdx.x; e < nlines * n; e += kThreads) {
    int l = e / n, i = e - l * n;
    if (!in_write_range(A, i)) continue;
    int li = first + l;
    int a = pick(li / nbs, A.ls.a_lo, A.ls.a_hi);
    int b = pick(li % nbs, A.ls.b_lo, A.ls.b_hi);
    int64_t g = (int64_t)a * A.sa + (int64_t)b * A.sb + i;
    float2 v = sbuf[e];
    if (A.post_mul) {
      float f = A.post_mul[g];
      v.x *= f;
      v.y *= f;
    }
    if (A.out_real) A.out_real[g] = v.x;
    else A.data[g] = v;
  }
}

// ---------------------------------------------------------------------------
// Compile-time variants for the sides the workloads use. The radix plan, the
// lines per CTA and every index divisor are constants, so butterfly and
// element index arithmetic is multiply-shift instead of integer division;
// per-line global offsets are computed once per CTA.
template <int... Rs>
struct Rad {};

template <int N>
struct RadixPlan;
template <> struct RadixPlan<36> { using type = Rad<4, 9>; };
template <> struct RadixPlan<72> { using type = Rad<4, 2, 9>; };
template <> struct RadixPlan<162> { using type = Rad<2, 9, 9>; };
template <> struct RadixPlan<216> { using type = Rad<4, 2, 3, 9>; };
template <> struct RadixPlan<320> { using type = Rad<4, 4, 4, 5>; };
template <> struct RadixPlan<324> { using type = Rad<4, 9, 9>; };
template <> struct RadixPlan<432> { using type = Rad<4, 4, 3, 9>; };
template <> struct RadixPlan<640> { using type = Rad<4, 4, 4, 2, 5>; };

template <int N, int LINES, int R, int Ns>
__device__ __forceinline__ void pass_ct(float2* buf, int nlines, const float2* __restrict__ tw,
                                        float sign) {
  constexpr int NB = N / R;
  constexpr int Q = (LINES * NB + kThreads - 1) / kThreads;
  constexpr int TSTEP = N / (Ns * R);
  const int nb = nlines * NB;
  float2 v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < nb) {
      const int line = b / NB, j = b - line * NB;
      const float2* src = buf + line * N + j;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[r * NB];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = threadIdx.x + q * kThreads;
    if (b < nb) {
      const int line = b / NB, j = b - line * NB;
      const int k = j % Ns;
      if (Ns > 1 && k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[k * r * TSTEP];   // shared-memory table
          w.y *= -sign;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft<R>(v[q], sign);
      float2* dst = buf + line * N + (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

template <int N, int LINES, int Ns, int R, int... Rest>
__device__ __forceinline__ void passes_ct(float2* buf, int nlines, const float2* __restrict__ tw,
                                          float sign, Rad<R, Rest...>) {
  pass_ct<N, LINES, R, Ns>(buf, nlines, tw, sign);
  if constexpr (sizeof...(Rest) > 0) passes_ct<N, LINES, Ns * R>(buf, nlines, tw, sign, Rad<Rest...>{});
}

template <int N>
__host__ __device__ constexpr int ct_lines() { return kMaxElems / N; }

// Element (position i, global offset g) of a line into shared memory: complex
// input by an asynchronous copy (no register round trip, every copy of the
// thread in flight at once), real input through registers, zero outside the
// read range. cp_async_wait() before the CTA synchronises.
__device__ __forceinline__ void stage_elem(const PassArgs& A, float2* dst, int i, int64_t g) {
  if (!in_read_range(A, i)) {
    *dst = make_float2(0.f, 0.f);
  } else if (A.in_real) {
    *dst = make_float2(__ldg(A.in_real + g), 0.f);
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(A.data + g)
                 : "memory");
  }
}

__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Twiddle table of one axis into shared memory (n entries).
__device__ __forceinline__ void stage_twiddles(float2* stw, const float2* __restrict__ tw, int n) {
  for (int k = threadIdx.x; k < n; k += kThreads) stw[k] = __ldg(tw + k);
}

__device__ __forceinline__ void store_elem(const PassArgs& A, int64_t g, float2 v) {
  if (A.post_mul) {
    const float f = __ldg(A.post_mul + g);
    v.x *= f;
    v.y *= f;
  }
  if (A.out_real) A.out_real[g] = v.x;
  else A.data[g] = v;
}

template <int N>
__global__ void __launch_bounds__(kThreads) fft_contig_ct(PassArgs A) {
  constexpr int L = ct_lines<N>();
  extern __shared__ float2 sbuf[];
  __shared__ int64_t lbase[L];
  const int na = range_count(A.ls.a_lo[0], A.ls.a_hi[0]) + range_count(A.ls.a_lo[1], A.ls.a_hi[1]);
  const int nbs = range_count(A.ls.b_lo[0], A.ls.b_hi[0]) + range_count(A.ls.b_lo[1], A.ls.b_hi[1]);
  const int first = blockIdx.x * L;
  const int nlines = min(L, na * nbs - first);
  if (threadIdx.x < nlines) {
    const int li = first + threadIdx.x;
    const int a = pick(li / nbs, A.ls.a_lo, A.ls.a_hi);
    const int b = pick(li % nbs, A.ls.b_lo, A.ls.b_hi);
    lbase[threadIdx.x] = (int64_t)a * A.sa + (int64_t)b * A.sb;
  }
  __syncthreads();
  float2* stw = sbuf + L * N;
  stage_twiddles(stw, A.tw, N);
  for (int e = threadIdx.x; e < nlines * N; e += kThreads) {
    const int l = e / N, i = e - l * N;
    stage_elem(A, sbuf + e, i, lbase[l] + i);
  }
  cp_async_wait();
  __syncthreads();
  passes_ct<N, L, 1>(sbuf, nlines, stw, A.sign, typename RadixPlan<N>::type{});
  if (A.convolve) {
    // the last forward pass and the first inverse pass of a convolution act
    // on the same lines: multiply in shared memory and transform back
    for (int e = threadIdx.x; e < nlines * N; e += kThreads) {
      const int l = e / N, i = e - l * N;
      const float f = __ldg(A.post_mul + lbase[l] + i);
      sbuf[e] = make_float2(sbuf[e].x * f, sbuf[e].y * f);
    }
    __syncthreads();
    passes_ct<N, L, 1>(sbuf, nlines, stw, -A.sign, typename RadixPlan<N>::type{});
    for (int e = threadIdx.x; e < nlines * N; e += kThreads) {
      const int l = e / N, i = e - l * N;
      if (in_write_range(A, i)) A.data[lbase[l] + i] = sbuf[e];
    }
    return;
  }
  for (int e = threadIdx.x; e < nlines * N; e += kThreads) {
    const int l = e / N, i = e - l * N;
    if (in_write_range(A, i)) store_elem(A, lbase[l] + i, sbuf[e]);
  }
}

// Strided axes: a CTA takes kStrideTile neighbouring lines (consecutive b,
// stride 1 in memory) and keeps them column-major in shared memory, element
// (position i, line l) at i * kStrideTile + l. Sixteen lines make every
// global row segment 128 contiguous bytes, and a half warp's butterfly
// operands (one j, sixteen lines) fill one 128-byte shared-memory row, so
// neither the staging copies nor the passes conflict on banks.
constexpr int kStrideTile = 16;

template <int N, int R, int Ns>
__device__ __forceinline__ void pass_col(float2* buf, int nlines, const float2* __restrict__ tw, float sign) {
  constexpr int T = kStrideTile;
  constexpr int NB = N / R;
  constexpr int Q = (T * NB + kThreads - 1) / kThreads;
  constexpr int TSTEP = N / (Ns * R);
  float2 v[Q][R];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = threadIdx.x + q * kThreads;
    const int l = b % T, j = b / T;
    if (b < T * NB && l < nlines) {
      const float2* src = buf + j * T + l;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[r * NB * T];
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = threadIdx.x + q * kThreads;
    const int l = b % T, j = b / T;
    if (b < T * NB && l < nlines) {
      const int k = j % Ns;
      if (Ns > 1 && k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[k * r * TSTEP];   // shared-memory table
          w.y *= -sign;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft<R>(v[q], sign);
      float2* dst = buf + ((j / Ns) * Ns * R + k) * T + l;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns * T] = v[q][r];
    }
  }
  __syncthreads();
}

template <int N, int Ns, int R, int... Rest>
__device__ __forceinline__ void passes_col(float2* buf, int nlines, const float2* __restrict__ tw, float sign,
                                           Rad<R, Rest...>) {
  pass_col<N, R, Ns>(buf, nlines, tw, sign);
  if constexpr (sizeof...(Rest) > 0) passes_col<N, Ns * R>(buf, nlines, tw, sign, Rad<Rest...>{});
}

template <int N>
__global__ void __launch_bounds__(kThreads) fft_strided_ct(PassArgs A) {
  constexpr int T = kStrideTile;
  extern __shared__ float2 sbuf[];
  __shared__ int64_t lbase[T], pbase[T];
  const int nb_sel = range_count(A.ls.b_lo[0], A.ls.b_hi[0]) + range_count(A.ls.b_lo[1], A.ls.b_hi[1]);
  const int tiles_b = (nb_sel + T - 1) / T;
  const int tile = blockIdx.x % tiles_b;
  const int a = pick(blockIdx.x / tiles_b, A.ls.a_lo, A.ls.a_hi);
  const int first = tile * T;
  const int nlines = min(T, nb_sel - first);
  if (threadIdx.x < nlines) {
    const int b = pick(first + threadIdx.x, A.ls.b_lo, A.ls.b_hi);
    lbase[threadIdx.x] = (int64_t)a * A.sa + (int64_t)b * A.sb;
    pbase[threadIdx.x] = (int64_t)a * A.pm_sa + (int64_t)b * A.pm_sb;
  }
  __syncthreads();
  float2* stw = sbuf + T * N;
  float* skern = reinterpret_cast<float*>(sbuf + T * N + N);   // convolution: the kernel's lines
  stage_twiddles(stw, A.tw, N);
  for (int e = threadIdx.x; e < T * N; e += kThreads) {
    const int l = e % T, i = e / T;
    if (l < nlines) stage_elem(A, sbuf + e, i, lbase[l] + (int64_t)i * A.es);
  }
  if (A.convolve) {
    // the kernel's values are copied alongside the data, ahead of the passes
    for (int e = threadIdx.x; e < T * N; e += kThreads) {
      const int l = e % T, i = e / T;
      if (l < nlines)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(
                         skern + e)),
                     "l"(A.post_mul + pbase[l] + (int64_t)i * A.pm_es)
                     : "memory");
    }
  }
  cp_async_wait();
  __syncthreads();
  passes_col<N, 1>(sbuf, nlines, stw, A.sign, typename RadixPlan<N>::type{});
  if (A.convolve) {
    // forward transform, product with the kernel (its own strides), inverse
    for (int e = threadIdx.x; e < T * N; e += kThreads) {
      const float f = skern[e];
      const float2 v = sbuf[e];
      sbuf[e] = make_float2(v.x * f, v.y * f);
    }
    __syncthreads();
    passes_col<N, 1>(sbuf, nlines, stw, -A.sign, typename RadixPlan<N>::type{});
    for (int e = threadIdx.x; e < T * N; e += kThreads) {
      const int l = e % T, i = e / T;
      if (l < nlines && in_write_range(A, i)) A.data[lbase[l] + (int64_t)i * A.es] = sbuf[e];
    }
    return;
  }
  for (int e = threadIdx.x; e < T * N; e += kThreads) {
    const int l = e % T, i = e / T;
    if (l < nlines && in_write_range(A, i)) store_elem(A, lbase[l] + (int64_t)i * A.es, sbuf[e]);
  }
}

// ------------------------------------------------------ real-input rows -----
// Transforms along x for the circulant convolution of a real vector x
// (Nm^3, [z][y][x]) embedded at wrapped positions of an N-point cube (model
// index a -> (a - Mh) mod N, Mh = (Nm - 1) / 2). Two rows u, w of x share one
// complex line c = u + i w; with C = FFT(c) the rows' own transforms are
// U[k] = (C[k] + conj C[-k]) / 2 and W[k] = (C[k] - conj C[-k]) / (2i). Only
// k = 0 .. N/2 is kept (the rest is the conjugate mirror of a real row), in
// the half-spectrum cube [N][N][N/2 + 1]. The inverse rebuilds C from the
// two half spectra and takes u = Re c, w = Im c.
template <int N>
__host__ __device__ constexpr int rc_lines() { return (kMaxElems / N) < 8 ? (kMaxElems / N) : 8; }
constexpr int RC_GROUP = 4;   // elements per thread whose loads are issued together

// Model index held at line position i of the wrapped embedding, or -1.
__device__ __forceinline__ int model_index(int i, int N, int Nm, int Mh) {
  const int a = i <= Mh ? i + Mh : i - N + Mh;
  return (i <= Mh || i >= N - Mh) && a >= 0 && a < Nm ? a : -1;
}

// Line position of model index b.
__device__ __forceinline__ int wrap_pos(int b, int N, int Mh) { return b >= Mh ? b - Mh : b - Mh + N; }

// Forward transform of row pairs (2m, 2m + 1) of plane c (line li = c HP + m,
// HP = (Nm + 1) / 2; a missing last row reads as zero). The row value is
// x, or add + beta x when `add` is given (then also stored to x_new).
template <int N>
__global__ void __launch_bounds__(kThreads) r2c_rows_ct(const float* x, const float* __restrict__ add,
                                                         const double* __restrict__ beta, float* x_new,
                                                         const float2* __restrict__ tw, int Nm,
                                                         float2* __restrict__ out) {
  constexpr int L = rc_lines<N>(), H = N / 2 + 1;
  extern __shared__ float2 sbuf[];
  const int Mh = (Nm - 1) / 2, HP = (Nm + 1) / 2;
  const int first = blockIdx.x * L;
  const int nlines = min(L, Nm * HP - first);
  float2* stw = sbuf + L * N;
  stage_twiddles(stw, tw, N);
  const float bt = add ? (float)__ldg(beta) : 0.f;
  // groups of RC_GROUP elements per thread: every load of a group is issued
  // before the first is used (x_new may alias x: each element is loaded and
  // stored by one thread, loads first)
  constexpr int IT = (L * N + kThreads - 1) / kThreads;
#pragma unroll
  for (int k0 = 0; k0 < IT; k0 += RC_GROUP) {
    float u[RC_GROUP], w[RC_GROUP], au[RC_GROUP], aw[RC_GROUP];
    int64_t r0[RC_GROUP];
    bool has[RC_GROUP], second[RC_GROUP];
#pragma unroll
    for (int k = 0; k < RC_GROUP; ++k) {
      const int e = threadIdx.x + (k0 + k) * kThreads;
      const int l = e / N, i = e - l * N;
      const int a = model_index(i, N, Nm, Mh);
      u[k] = w[k] = au[k] = aw[k] = 0.f;
      r0[k] = 0;
      has[k] = k0 + k < IT && e < L * N && l < nlines && a >= 0;
      second[k] = false;
      if (has[k]) {
        const int li = first + l, c = li / HP, m = li - c * HP;
        r0[k] = ((int64_t)c * Nm + 2 * m) * Nm + a;
        second[k] = 2 * m + 1 < Nm;
        u[k] = x[r0[k]];
        if (second[k]) w[k] = x[r0[k] + Nm];
        if (add) {
          au[k] = __ldg(add + r0[k]);
          if (second[k]) aw[k] = __ldg(add + r0[k] + Nm);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < RC_GROUP; ++k) {
      const int e = threadIdx.x + (k0 + k) * kThreads;
      if (k0 + k >= IT || e >= L * N) continue;
      float uu = u[k], ww = w[k];
      if (has[k] && add) {
        uu = fmaf(bt, uu, au[k]);
        x_new[r0[k]] = uu;
        if (second[k]) {
          ww = fmaf(bt, ww, aw[k]);
          x_new[r0[k] + Nm] = ww;
        }
      }
      sbuf[e] = make_float2(uu, ww);
    }
  }
  __syncthreads();
  passes_ct<N, L, 1>(sbuf, nlines, stw, -1.f, typename RadixPlan<N>::type{});
  for (int e = threadIdx.x; e < L * H; e += kThreads) {
    const int l = e / H, k = e - l * H;
    if (l >= nlines) continue;
    const int li = first + l, c = li / HP, m = li - c * HP;
    const float2 ck = sbuf[l * N + k], cm = sbuf[l * N + (k == 0 ? 0 : N - k)];
    const int64_t plane = (int64_t)wrap_pos(c, N, Mh) * N;
    out[(plane + wrap_pos(2 * m, N, Mh)) * H + k] = make_float2(0.5f * (ck.x + cm.x), 0.5f * (ck.y - cm.y));
    if (2 * m + 1 < Nm)
      out[(plane + wrap_pos(2 * m + 1, N, Mh)) * H + k] =
          make_float2(0.5f * (ck.y + cm.y), -0.5f * (ck.x - cm.x));
  }
}

// Inverse of the above: row pairs of the half-spectrum cube back to the
// real rows, y = ep.scale * row + ep.lambda * ep.xin at the model indices
// (Nm^3), with the epilogue's FP64 partial sums of xin . y.
template <int N>
__global__ void __launch_bounds__(kThreads) c2r_rows_ct(const float2* __restrict__ in,
                                                         const float2* __restrict__ tw, int Nm, float* y,
                                                         RealConvEpilogue ep) {
  constexpr int L = rc_lines<N>(), H = N / 2 + 1;
  extern __shared__ float2 sbuf[];
  const int Mh = (Nm - 1) / 2, HP = (Nm + 1) / 2;
  const int first = blockIdx.x * L;
  const int nlines = min(L, Nm * HP - first);
  float2* stw = sbuf + L * N;
  stage_twiddles(stw, tw, N);
  // the half-spectrum loads of a group of elements go out together
  constexpr int IT = (L * N + kThreads - 1) / kThreads;
#pragma unroll
  for (int k0 = 0; k0 < IT; k0 += RC_GROUP) {
    float2 u[RC_GROUP], w[RC_GROUP];
#pragma unroll
    for (int q = 0; q < RC_GROUP; ++q) {
      const int e = threadIdx.x + (k0 + q) * kThreads;
      const int l = e / N, k = e - l * N;
      u[q] = w[q] = make_float2(0.f, 0.f);
      if (k0 + q < IT && e < L * N && l < nlines) {
        const int li = first + l, c = li / HP, m = li - c * HP;
        const int64_t plane = (int64_t)wrap_pos(c, N, Mh) * N;
        const int kk = k < H ? k : N - k;
        u[q] = __ldg(in + (plane + wrap_pos(2 * m, N, Mh)) * H + kk);
        if (2 * m + 1 < Nm) w[q] = __ldg(in + (plane + wrap_pos(2 * m + 1, N, Mh)) * H + kk);
      }
    }
#pragma unroll
    for (int q = 0; q < RC_GROUP; ++q) {
      const int e = threadIdx.x + (k0 + q) * kThreads;
      if (k0 + q >= IT || e >= L * N) continue;
      const int k = e % N;
      // C[k] = U[k] + i W[k]; past N/2, U[k] = conj U[N - k] (and W alike)
      sbuf[e] = k < H ? make_float2(u[q].x - w[q].y, u[q].y + w[q].x)
                      : make_float2(u[q].x + w[q].y, w[q].x - u[q].y);
    }
  }
  __syncthreads();
  passes_ct<N, L, 1>(sbuf, nlines, stw, 1.f, typename RadixPlan<N>::type{});
  double acc = 0.0;
  // epilogue over the Nm <= N/2 + 1 model positions of each line; y may
  // alias xin (one thread loads, then stores, each element)
  constexpr int OT = (L * (N / 2 + 1) + kThreads - 1) / kThreads;
#pragma unroll
  for (int k0 = 0; k0 < OT; k0 += RC_GROUP) {
    float v[RC_GROUP][2], xv[RC_GROUP][2];
    int64_t r0[RC_GROUP];
    bool has[RC_GROUP], second[RC_GROUP];
#pragma unroll
    for (int q = 0; q < RC_GROUP; ++q) {
      const int e = threadIdx.x + (k0 + q) * kThreads;
      const int l = e / Nm, a = e - l * Nm;
      has[q] = k0 + q < OT && e < L * Nm && l < nlines;
      second[q] = false;
      r0[q] = 0;
      v[q][0] = v[q][1] = xv[q][0] = xv[q][1] = 0.f;
      if (has[q]) {
        const int li = first + l, c = li / HP, m = li - c * HP;
        const float2 t = sbuf[l * N + wrap_pos(a, N, Mh)];
        v[q][0] = t.x;
        v[q][1] = t.y;
        r0[q] = ((int64_t)c * Nm + 2 * m) * Nm + a;
        second[q] = 2 * m + 1 < Nm;
        if (ep.xin) {
          xv[q][0] = ep.xin[r0[q]];
          if (second[q]) xv[q][1] = ep.xin[r0[q] + Nm];
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RC_GROUP; ++q) {
      if (!has[q]) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !second[q]) continue;
        float o = v[q][h] * ep.scale;
        if (ep.xin) {
          o = fmaf(ep.lambda, xv[q][h], o);
          acc += (double)xv[q][h] * (double)o;
        }
        y[r0[q] + h * Nm] = o;
      }
    }
  }
  if (ep.part) {
    const double sblk = block_sum(acc);
    if (ep.count) partial_and_finalize(sblk, ep.part, ep.sc, 1, nullptr, ep.count);
    else if (threadIdx.x == 0) ep.part[blockIdx.x] = sblk;
  }
}

// Forward transform (sign `sign`) of the rows of a real N^3 cube in pairs
// (2m, 2m + 1) of plane c (line li = c N/2 + m), keeping the half-spectrum
// columns k < h (row stride h) in out[N][N][h].
template <int N>
__global__ void __launch_bounds__(kThreads) r2c_cube_ct(const float* __restrict__ in,
                                                         const float2* __restrict__ tw, float sign, int h,
                                                         float2* __restrict__ out) {
  constexpr int L = rc_lines<N>(), HP = N / 2;
  extern __shared__ float2 sbuf[];
  const int first = blockIdx.x * L;
  const int nlines = min(L, N * HP - first);
  float2* stw = sbuf + L * N;
  stage_twiddles(stw, tw, N);
  for (int e = threadIdx.x; e < L * N; e += kThreads) {
    const int l = e / N, i = e - l * N;
    float2 v = make_float2(0.f, 0.f);
    if (l < nlines) {
      const int li = first + l, c = li / HP, m = li - c * HP;
      const int64_t r0 = ((int64_t)c * N + 2 * m) * N + i;
      v = make_float2(__ldg(in + r0), __ldg(in + r0 + N));
    }
    sbuf[e] = v;
  }
  __syncthreads();
  passes_ct<N, L, 1>(sbuf, nlines, stw, sign, typename RadixPlan<N>::type{});
  for (int e = threadIdx.x; e < L * h; e += kThreads) {
    const int l = e / h, k = e - l * h;
    if (l >= nlines) continue;
    const int li = first + l, c = li / HP, m = li - c * HP;
    const float2 ck = sbuf[l * N + k], cm = sbuf[l * N + (k == 0 ? 0 : N - k)];
    const int64_t r0 = ((int64_t)c * N + 2 * m) * h + k;
    out[r0] = make_float2(0.5f * (ck.x + cm.x), 0.5f * (ck.y - cm.y));
    out[r0 + h] = make_float2(0.5f * (ck.y + cm.y), -0.5f * (ck.x - cm.x));
  }
}

template <int N>
int launch_r2c_cube_ct(const FFT3* p, const float* in, int sign, int h, float2* out, cudaStream_t s) {
  constexpr int L = rc_lines<N>();
  const unsigned grid = (unsigned)ceil_div((int64_t)N * (N / 2), L);
  const size_t smem = (size_t)(L + 1) * N * sizeof(float2);
  const float2* tw = p->ax[0].twiddle;
  const double bytes = (double)N * N * N * 4.0 + (double)N * N * h * 8.0;
  return launch("fft_r2c_cube_kernel", s,
                [&] { r2c_cube_ct<N><<<grid, kThreads, smem, s>>>(in, tw, (float)sign, h, out); }, bytes);
}

template <int N>
unsigned rows_grid(int Nm) {
  return (unsigned)ceil_div((int64_t)Nm * ((Nm + 1) / 2), rc_lines<N>());
}

template <int N>
int launch_rows_ct(bool forward, const FFT3* p, int Nm, const float* x, const float* add,
                   const double* beta, float* x_new, float2* work, float* y, const RealConvEpilogue& ep,
                   cudaStream_t s) {
  constexpr int L = rc_lines<N>();
  const unsigned grid = rows_grid<N>(Nm);
  const size_t smem = (size_t)(L + 1) * N * sizeof(float2);   // lines and the twiddle table
  const float2* tw = p->ax[0].twiddle;
  // rows of the Nm^3 vector (and of `add`, with x_new written) against the
  // Nm x Nm half-spectrum rows of H = N/2 + 1 columns that hold data
  const double vec = (double)Nm * Nm * Nm * 4.0, half = (double)Nm * Nm * (N / 2 + 1) * 8.0;
  if (forward)
    return launch("fft_r2c_rows_kernel", s,
                  [&] { r2c_rows_ct<N><<<grid, kThreads, smem, s>>>(x, add, beta, x_new, tw, Nm, work); },
                  vec * (add ? 3.0 : 1.0) + half);
  return launch("fft_c2r_rows_kernel", s,
                [&] { c2r_rows_ct<N><<<grid, kThreads, smem, s>>>(work, tw, Nm, y, ep); },
                half + vec * (ep.xin ? 2.0 : 1.0));
}

template <int N>
int launch_ct(PassArgs& A, bool contiguous, int na, int nb, double bytes, cudaStream_t s) {
  if (contiguous) {
    constexpr int L = ct_lines<N>();
    const int grid = (int)ceil_div((int64_t)na * nb, L);
    const size_t smem = (size_t)(L + 1) * N * sizeof(float2);   // lines and the twiddle table
    return launch("fft_contig_kernel", s, [&] { fft_contig_ct<N><<<grid, kThreads, smem, s>>>(A); }, bytes);
  }
  constexpr int T = kStrideTile;
  const int64_t grid = ceil_div(nb, T) * (int64_t)na;
  // lines and the twiddle table, and for a convolution the kernel's lines
  const size_t smem = (size_t)(T + 1) * N * sizeof(float2) + (A.convolve ? (size_t)T * N * sizeof(float) : 0);
  if (smem > 48 * 1024)
    SPF_CUDA(cudaFuncSetAttribute(fft_strided_ct<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return launch("fft_strided_kernel", s,
                [&] { fft_strided_ct<N><<<(unsigned)grid, kThreads, smem, s>>>(A); }, bytes);
}

int factorize(int n, int* radix) {
  int k = 0;
  while (n % 4 == 0) { radix[k++] = 4; n /= 4; }
  while (n % 2 == 0) { radix[k++] = 2; n /= 2; }
  while (n % 3 == 0) { radix[k++] = 3; n /= 3; }
  while (n % 5 == 0) { radix[k++] = 5; n /= 5; }
  return n == 1 ? k : -1;
}

void full_range(int n, int* lo, int* hi) {
  lo[0] = 0; hi[0] = n; lo[1] = 0; hi[1] = 0;
}

// Wrapped range {0..h-1} U {n-h+1..n-1} (h = half width incl. zero).
void wrapped_range(int n, int h, int* lo, int* hi) {
  if (h <= 0 || 2 * h - 1 >= n) { full_range(n, lo, hi); return; }
  lo[0] = 0; hi[0] = h; lo[1] = n - h + 1; hi[1] = n;
}

int count(const int* lo, const int* hi) {
  return std::max(0, hi[0] - lo[0]) + std::max(0, hi[1] - lo[1]);
}

// Algorithmic bytes of one pass: every line reads its positions inside the
// read range (4 bytes real, 8 complex), writes its positions inside the
// write range (4 or 8 bytes) and reads n real factors when it multiplies by
// post_mul.
double pass_bytes(const PassArgs& A, int na, int nb) {
  const double lines = (double)na * nb;
  const double rd = count(A.in_lo, A.in_hi), wr = count(A.out_lo, A.out_hi);
  const double ein = A.in_real ? 4.0 : 8.0, eout = A.out_real ? 4.0 : 8.0;
  const double pm = A.post_mul ? 4.0 * A.n : 0.0;
  return lines * (rd * ein + wr * eout + pm);
}

int launch_pass(PassArgs A, bool contiguous, cudaStream_t s) {
  int na = count(A.ls.a_lo, A.ls.a_hi), nb = count(A.ls.b_lo, A.ls.b_hi);
  if (na == 0 || nb == 0) return SPF_OK;
  const double bytes = pass_bytes(A, na, nb);
  switch (A.n) {
    case 36: return launch_ct<36>(A, contiguous, na, nb, bytes, s);
    case 72: return launch_ct<72>(A, contiguous, na, nb, bytes, s);
    case 162: return launch_ct<162>(A, contiguous, na, nb, bytes, s);
    case 216: return launch_ct<216>(A, contiguous, na, nb, bytes, s);
    case 320: return launch_ct<320>(A, contiguous, na, nb, bytes, s);
    case 324: return launch_ct<324>(A, contiguous, na, nb, bytes, s);
    case 432: return launch_ct<432>(A, contiguous, na, nb, bytes, s);
    case 640: return launch_ct<640>(A, contiguous, na, nb, bytes, s);
    default: break;
  }
  if (contiguous) {
    A.lines_per_cta = std::max(1, kMaxElems / A.n);
    int64_t total = (int64_t)na * nb;
    int grid = (int)ceil_div(total, A.lines_per_cta);
    size_t smem = (size_t)A.lines_per_cta * A.n * sizeof(float2);
    return launch("fft_contig_kernel", s,
                  [&] { fft_contig_kernel<<<grid, kThreads, smem, s>>>(A); }, bytes);
  } else {
    A.lines_per_cta = std::max(1, std::min(16, kMaxElems / A.n));
    int tiles_b = (int)ceil_div(nb, A.lines_per_cta);
    int64_t grid = (int64_t)tiles_b * na;
    size_t smem = (size_t)A.lines_per_cta * A.n * sizeof(float2);
    return launch("fft_strided_kernel", s,
                  [&] { fft_strided_kernel<<<(unsigned)grid, kThreads, smem, s>>>(A); }, bytes);
  }
}

}  // namespace

int fft3_create(FFT3* p, int n0, int n1, int n2) {
  p->n0 = n0; p->n1 = n1; p->n2 = n2;
  int ns[3] = {n0, n1, n2};
  for (int a = 0; a < 3; ++a) {
    FFTAxisPlan& ax = p->ax[a];
    ax.n = ns[a];
    ax.nrad = factorize(ns[a], ax.radix);
    SPF_CHECK_ARG(ax.nrad >= 0, "fft: side %d is not 2/3/5-smooth", ns[a]);
    SPF_CHECK_ARG(ns[a] <= kMaxElems, "fft: side %d too large", ns[a]);
    std::vector<float2> tw(ns[a]);
    for (int m = 0; m < ns[a]; ++m) {
      double ang = -2.0 * M_PI * (double)m / (double)ns[a];
      tw[m] = make_float2((float)cos(ang), (float)sin(ang));
    }
    SPF_TRY(dev_alloc((void**)&ax.twiddle, ns[a] * sizeof(float2), "fft twiddles"));
    SPF_CUDA(cudaMemcpy(ax.twiddle, tw.data(), ns[a] * sizeof(float2), cudaMemcpyHostToDevice));
  }
  // the largest tile needs 32 KB of dynamic shared memory
  SPF_CUDA(cudaFuncSetAttribute(fft_strided_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxElems * (int)sizeof(float2)));
  SPF_CUDA(cudaFuncSetAttribute(fft_contig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxElems * (int)sizeof(float2)));
  return SPF_OK;
}

void fft3_destroy(FFT3* p) {
  for (int a = 0; a < 3; ++a) {
    if (p->ax[a].twiddle) cudaFree(p->ax[a].twiddle);
    p->ax[a].twiddle = nullptr;
  }
}

// Generic pass launcher over axis `axis` (0 = x, 1 = y, 2 = z).
// One axis pass over the lines (a, b) in the given ranges; positions along
// the line outside [in_lo, in_hi) (two ranges; nullptr: all) read as zero.
static int axis_pass(const FFT3* p, int axis, float2* data, const float* in_real, float* out_real,
                     const float* post_mul, int sign, const int* a_lo, const int* a_hi,
                     const int* b_lo, const int* b_hi, cudaStream_t s, const int* in_lo = nullptr,
                     const int* in_hi = nullptr, bool convolve = false, int row = 0,
                     const int* out_lo = nullptr, const int* out_hi = nullptr) {
  PassArgs A;
  A.data = data;
  A.in_real = in_real;
  A.out_real = out_real;
  A.post_mul = post_mul;
  A.convolve = convolve ? 1 : 0;
  const FFTAxisPlan& ax = p->ax[axis];
  A.n = ax.n;
  A.nrad = ax.nrad;
  for (int i = 0; i < ax.nrad; ++i) A.radix[i] = ax.radix[i];
  A.tw = ax.twiddle;
  A.sign = (float)sign;
  // row > 0: the data is the half-spectrum cube of a real-input transform,
  // rows of `row` entries; post_mul keeps the full cube's strides
  const int64_t n0 = row > 0 ? row : p->n0, n1 = p->n1;
  const int64_t f0 = p->n0, f1 = p->n1;
  for (int i = 0; i < 2; ++i) {
    A.ls.a_lo[i] = a_lo[i]; A.ls.a_hi[i] = a_hi[i];
    A.ls.b_lo[i] = b_lo[i]; A.ls.b_hi[i] = b_hi[i];
    A.in_lo[i] = in_lo ? in_lo[i] : 0;
    A.in_hi[i] = in_hi ? in_hi[i] : (i == 0 ? ax.n : 0);
    A.out_lo[i] = out_lo ? out_lo[i] : 0;
    A.out_hi[i] = out_hi ? out_hi[i] : (i == 0 ? ax.n : 0);
  }
  if (axis == 0) {          // lines (z, y): a = z, b = y
    A.es = 1; A.sa = n1 * n0; A.sb = n0;
    A.pm_es = 1; A.pm_sa = f1 * f0; A.pm_sb = f0;
    return launch_pass(A, true, s);
  } else if (axis == 1) {   // lines (z, x): a = z, b = x
    A.es = n0; A.sa = n1 * n0; A.sb = 1;
    A.pm_es = f0; A.pm_sa = f1 * f0; A.pm_sb = 1;
    return launch_pass(A, false, s);
  } else {                  // lines (y, x): a = y, b = x
    A.es = n1 * n0; A.sa = n0; A.sb = 1;
    A.pm_es = f1 * f0; A.pm_sa = f0; A.pm_sb = 1;
    return launch_pass(A, false, s);
  }
}

// Exposed pass with real input / output and a real post-multiplier, used by
// the NUFFT and Toeplitz code to fuse the first read and last write.
int fft3_exec_ex(const FFT3* p, float2* data, const float* in_real, float* out_real,
                 const float* post_mul, int sign, int zero_hw_in, int need_hw_out,
                 cudaStream_t s) {
  // A real input is read by the first pass only; with zero-line pruning the
  // skipped lines would never be written, so the two do not combine.
  SPF_CHECK_ARG(!(in_real && zero_hw_in > 0), "fft: real input with pruned input lines");
  int fx_lo[2], fx_hi[2], fy_lo[2], fy_hi[2], fz_lo[2], fz_hi[2];
  full_range(p->n0, fx_lo, fx_hi);
  full_range(p->n1, fy_lo, fy_hi);
  full_range(p->n2, fz_lo, fz_hi);
  int rx_lo[2], rx_hi[2], ry_lo[2], ry_hi[2];
  if (zero_hw_in > 0) {
    // Only the wrapped index range of half width zero_hw_in along each axis
    // holds data: each pass reads its line only there (so the caller need
    // not zero the rest of the cube) and only the lines whose other
    // coordinates lie in the ranges already transformed.
    int rz_lo[2], rz_hi[2];
    wrapped_range(p->n0, zero_hw_in, rx_lo, rx_hi);
    wrapped_range(p->n1, zero_hw_in, ry_lo, ry_hi);
    wrapped_range(p->n2, zero_hw_in, rz_lo, rz_hi);
    SPF_TRY(axis_pass(p, 2, data, nullptr, nullptr, nullptr, sign, ry_lo, ry_hi, rx_lo, rx_hi, s, rz_lo, rz_hi));
    SPF_TRY(axis_pass(p, 1, data, nullptr, nullptr, nullptr, sign, fz_lo, fz_hi, rx_lo, rx_hi, s, ry_lo, ry_hi));
    SPF_TRY(axis_pass(p, 0, data, nullptr, out_real, post_mul, sign, fz_lo, fz_hi, fy_lo, fy_hi, s, rx_lo,
                      rx_hi));
    return SPF_OK;
  }
  // each pass stores only what the next one reads, the last only the
  // output range needed
  int rz_lo[2], rz_hi[2];
  wrapped_range(p->n0, need_hw_out, rx_lo, rx_hi);
  wrapped_range(p->n1, need_hw_out, ry_lo, ry_hi);
  wrapped_range(p->n2, need_hw_out, rz_lo, rz_hi);
  SPF_TRY(axis_pass(p, 0, data, in_real, nullptr, nullptr, sign, fz_lo, fz_hi, fy_lo, fy_hi, s, nullptr, nullptr,
                    false, 0, rx_lo, rx_hi));
  SPF_TRY(axis_pass(p, 1, data, nullptr, nullptr, nullptr, sign, fz_lo, fz_hi, rx_lo, rx_hi, s, nullptr, nullptr,
                    false, 0, ry_lo, ry_hi));
  SPF_TRY(axis_pass(p, 2, data, nullptr, out_real, post_mul, sign, ry_lo, ry_hi, rx_lo, rx_hi, s, nullptr, nullptr,
                    false, 0, rz_lo, rz_hi));
  return SPF_OK;
}

// Circular convolution in place: IFFT(kernel * FFT(data)) without the 1/n^3,
// forward sign -1. Input data only in the wrapped range of half width
// zero_hw_in along each axis (the rest is never read), output needed only in
// the range of half width need_hw_out. The forward x pass, the product and
// the inverse x pass run as one pass over the same lines.
int fft3_convolve(const FFT3* p, float2* data, const float* kernel, int zero_hw_in, int need_hw_out,
                  cudaStream_t s) {
  const int n0 = p->n0;
  const bool fused = n0 == 36 || n0 == 72 || n0 == 162 || n0 == 216 || n0 == 320 || n0 == 324 ||
                     n0 == 432 || n0 == 640;
  if (!fused || zero_hw_in <= 0) {
    SPF_TRY(fft3_exec_ex(p, data, nullptr, nullptr, kernel, -1, zero_hw_in, 0, s));
    return fft3_exec_ex(p, data, nullptr, nullptr, nullptr, +1, 0, need_hw_out, s);
  }
  int fy_lo[2], fy_hi[2], fz_lo[2], fz_hi[2];
  full_range(p->n1, fy_lo, fy_hi);
  full_range(p->n2, fz_lo, fz_hi);
  int rx_lo[2], rx_hi[2], ry_lo[2], ry_hi[2], rz_lo[2], rz_hi[2];
  wrapped_range(p->n0, zero_hw_in, rx_lo, rx_hi);
  wrapped_range(p->n1, zero_hw_in, ry_lo, ry_hi);
  wrapped_range(p->n2, zero_hw_in, rz_lo, rz_hi);
  SPF_TRY(axis_pass(p, 2, data, nullptr, nullptr, nullptr, -1, ry_lo, ry_hi, rx_lo, rx_hi, s, rz_lo, rz_hi));
  SPF_TRY(axis_pass(p, 1, data, nullptr, nullptr, nullptr, -1, fz_lo, fz_hi, rx_lo, rx_hi, s, ry_lo, ry_hi));
  int ox_lo[2], ox_hi[2], oy_lo[2], oy_hi[2], oz_lo[2], oz_hi[2];
  wrapped_range(p->n0, need_hw_out, ox_lo, ox_hi);
  wrapped_range(p->n1, need_hw_out, oy_lo, oy_hi);
  wrapped_range(p->n2, need_hw_out, oz_lo, oz_hi);
  SPF_TRY(axis_pass(p, 0, data, nullptr, nullptr, kernel, -1, fz_lo, fz_hi, fy_lo, fy_hi, s, rx_lo, rx_hi,
                    /*convolve=*/true, 0, ox_lo, ox_hi));
  SPF_TRY(axis_pass(p, 1, data, nullptr, nullptr, nullptr, +1, fz_lo, fz_hi, ox_lo, ox_hi, s, nullptr, nullptr,
                    false, 0, oy_lo, oy_hi));
  return axis_pass(p, 2, data, nullptr, nullptr, nullptr, +1, oy_lo, oy_hi, ox_lo, ox_hi, s, nullptr, nullptr, false,
                   0, oz_lo, oz_hi);
}

#define SPF_SIDE_SWITCH(n, expr)       \
  switch (n) {                         \
    case 36: { constexpr int S = 36; expr; }   \
    case 72: { constexpr int S = 72; expr; }   \
    case 162: { constexpr int S = 162; expr; } \
    case 216: { constexpr int S = 216; expr; } \
    case 320: { constexpr int S = 320; expr; } \
    case 324: { constexpr int S = 324; expr; } \
    case 432: { constexpr int S = 432; expr; } \
    case 640: { constexpr int S = 640; expr; } \
    default: break;                    \
  }

static int launch_rows(bool forward, const FFT3* p, int Nm, const float* x, const float* add,
                       const double* beta, float* x_new, float2* work, float* y, const RealConvEpilogue& ep,
                       cudaStream_t s) {
  SPF_SIDE_SWITCH(p->n0, return launch_rows_ct<S>(forward, p, Nm, x, add, beta, x_new, work, y, ep, s));
  set_error("fft: no real-input row transform for side %d", p->n0);
  return SPF_ERR_UNSUPPORTED;
}

int fft3_real_conv_blocks(const FFT3* p, int Nm) {
  SPF_SIDE_SWITCH(p->n0, return (int)rows_grid<S>(Nm));
  return 0;
}

// Modes |k| < h of the transform of a real cube: real-input row transforms
// along x keeping columns kx < h, then y and z passes on those columns (z
// only on the lines whose y frequency is in the wrapped range of half
// width h). out[nf][nf][h]; kx < 0 follows from F(-k) = conj F(k).
int fft3_r2c_modes(const FFT3* p, const float* in, int h, int sign, float2* out, cudaStream_t s) {
  SPF_CHECK_ARG(fft3_real_supported(p), "fft: side %d has no real-input transform", p->n0);
  const int n = p->n0;
  SPF_CHECK_ARG(h >= 1 && 2 * h - 1 <= n, "fft: %d modes do not fit side %d", 2 * h - 1, n);
  int f_lo[2], f_hi[2], k_lo[2], k_hi[2], r_lo[2], r_hi[2];
  full_range(n, f_lo, f_hi);
  full_range(h, k_lo, k_hi);
  wrapped_range(n, h, r_lo, r_hi);
  int rc;
  switch (n) {
    case 36: rc = launch_r2c_cube_ct<36>(p, in, sign, h, out, s); break;
    case 72: rc = launch_r2c_cube_ct<72>(p, in, sign, h, out, s); break;
    case 162: rc = launch_r2c_cube_ct<162>(p, in, sign, h, out, s); break;
    case 216: rc = launch_r2c_cube_ct<216>(p, in, sign, h, out, s); break;
    case 320: rc = launch_r2c_cube_ct<320>(p, in, sign, h, out, s); break;
    case 324: rc = launch_r2c_cube_ct<324>(p, in, sign, h, out, s); break;
    case 432: rc = launch_r2c_cube_ct<432>(p, in, sign, h, out, s); break;
    case 640: rc = launch_r2c_cube_ct<640>(p, in, sign, h, out, s); break;
    default: rc = SPF_ERR_UNSUPPORTED; break;
  }
  SPF_TRY(rc);
  // the y pass stores the rows the z pass reads, the z pass the planes kept
  SPF_TRY(axis_pass(p, 1, out, nullptr, nullptr, nullptr, sign, f_lo, f_hi, k_lo, k_hi, s, nullptr, nullptr, false,
                    h, r_lo, r_hi));
  return axis_pass(p, 2, out, nullptr, nullptr, nullptr, sign, r_lo, r_hi, k_lo, k_hi, s, nullptr, nullptr, false,
                   h, r_lo, r_hi);
}

bool fft3_real_supported(const FFT3* p) {
  const int n = p->n0;
  return p->n1 == n && p->n2 == n &&
         (n == 36 || n == 72 || n == 162 || n == 216 || n == 320 || n == 324 || n == 432 || n == 640);
}

// y = IFFT(kernel * FFT(embed x)) at the model indices, for real x: real-
// input row transforms along x, then y and z passes on the half spectrum
// (the z pass forward, times the kernel, and back in one launch).
int fft3_convolve_real(const FFT3* p, int Nm, const float* x, const float* add, const double* beta,
                       float* x_new, const float* kernel, float2* work, float* y, const RealConvEpilogue& ep,
                       cudaStream_t s) {
  SPF_CHECK_ARG(fft3_real_supported(p), "fft: side %d has no real-input convolution", p->n0);
  const int n = p->n0, H = n / 2 + 1, Mh = (Nm - 1) / 2;
  SPF_CHECK_ARG(Nm >= 1 && Nm % 2 == 1 && 2 * Nm - 1 <= n, "fft: vector side %d does not embed in %d", Nm, n);
  int r_lo[2], r_hi[2], f_lo[2], f_hi[2], k_lo[2], k_hi[2];
  wrapped_range(n, Mh + 1, r_lo, r_hi);   // rows and planes holding data, and those needed
  full_range(n, f_lo, f_hi);
  full_range(H, k_lo, k_hi);
  SPF_CHECK_ARG(!ep.part || ep.xin, "fft: epilogue partial sums need xin");
  SPF_TRY(launch_rows(true, p, Nm, x, add, beta, x_new, work, nullptr, ep, s));
  SPF_TRY(axis_pass(p, 1, work, nullptr, nullptr, nullptr, -1, r_lo, r_hi, k_lo, k_hi, s, r_lo, r_hi, false, H));
  // the inverse y pass reads the planes z in the data range only, and the
  // inverse rows read the rows y in it
  SPF_TRY(axis_pass(p, 2, work, nullptr, nullptr, kernel, -1, f_lo, f_hi, k_lo, k_hi, s, r_lo, r_hi, true, H,
                    r_lo, r_hi));
  SPF_TRY(axis_pass(p, 1, work, nullptr, nullptr, nullptr, +1, r_lo, r_hi, k_lo, k_hi, s, nullptr, nullptr, false,
                    H, r_lo, r_hi));
  return launch_rows(false, p, Nm, nullptr, nullptr, nullptr, nullptr, work, y, ep, s);
}

}  // namespace spf

namespace spf {
int fft3_exec(const FFT3* p, float2* data, int sign, int zero_hw_in, int need_hw_out,
              cudaStream_t s) {
  return fft3_exec_ex(p, data, nullptr, nullptr, nullptr, sign, zero_hw_in, need_hw_out, s);
}
}  // namespace spf
