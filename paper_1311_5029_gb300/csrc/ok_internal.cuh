// Internal definitions shared by the CUDA sources of the OK-action W-form library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <math.h>
#include <cuda_fp16.h>

#include "../../include/ok.h"

namespace okgb {

// ---------------------------------------------------------------------------- double-float
// A real number held as the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2
// (about 48 significand bits).  Arithmetic uses the error-free transformations TwoSum (Knuth) and
// TwoProd (with FMA), as in Joldes, Muller and Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44 (2017): the products are the "DWTimesDW"
// form and the sums add the low parts without a second TwoSum, so an operation's absolute error is
// a few 2^-48 times the magnitude of its operands.  On GB300 the FP32 pipes are 58 times faster
// than the FP64 pipe, which makes this the faster way to FP64-level accuracy for the stencil.
// nvcc does not reassociate floating-point expressions, and none of the sums below contains a
// product that FMA contraction could merge.
struct dd {
  float hi, lo;
  dd() = default;
  __host__ __device__ __forceinline__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ dd(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ __forceinline__ dd(int i) : dd((double)i) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__host__ __device__ __forceinline__ dd dd_renorm(float s, float e) {
  const float h = s + e;
  return dd(h, e - (h - s));
}
__host__ __device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  float e = (a.hi - (s - bb)) + (b.hi - bb);
  e += a.lo + b.lo;
  return dd_renorm(s, e);
}
__host__ __device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__host__ __device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd_renorm(p, e);
}
// fma overloads in this namespace so that templates calling fma(x, y, z) work for float, double
// and dd alike.
__host__ __device__ __forceinline__ float fma(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
__host__ __device__ __forceinline__ dd fma(dd a, dd b, dd c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = p + c.hi;
  const float bb = s - p;
  float t = (p - (s - bb)) + (c.hi - bb);
  t += e + c.lo;
  return dd_renorm(s, t);
}

// ---------------------------------------------------------------------------- complex numbers
template <typename R> struct cx { R re, im; };

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> z; z.re = a; z.im = b; return z; }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator-(cx<R> a) { return mk(-a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return mk(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ cx<R> cj(cx<R> a) { return mk(a.re, -a.im); }
// i * a and -i * a
template <typename R> __host__ __device__ __forceinline__ cx<R> ti(cx<R> a) { return mk(-a.im, a.re); }
template <typename R> __host__ __device__ __forceinline__ cx<R> tmi(cx<R> a) { return mk(a.im, -a.re); }
// acc + a * b and acc + conj(a) * b
template <typename R> __host__ __device__ __forceinline__ cx<R> fma_c(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
template <typename R> __host__ __device__ __forceinline__ cx<R> fma_cj(cx<R> a, cx<R> b, cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}

// 3x3 complex colour matrix, row-major.
template <typename R> struct M3 { cx<R> e[9]; };

template <typename R> __host__ __device__ __forceinline__ M3<R> m_zero() { M3<R> m; for (int k = 0; k < 9; ++k) m.e[k] = mk<R>(0, 0); return m; }
template <typename R> __host__ __device__ __forceinline__ M3<R> m_eye() { M3<R> m = m_zero<R>(); m.e[0] = m.e[4] = m.e[8] = mk<R>(1, 0); return m; }
template <typename R> __host__ __device__ __forceinline__ M3<R> m_mul(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      cx<R> s = mk<R>(0, 0);
      for (int k = 0; k < 3; ++k) s = fma_c(a.e[3 * i + k], b.e[3 * k + j], s);
      c.e[3 * i + j] = s;
    }
  return c;
}
template <typename R> __host__ __device__ __forceinline__ M3<R> m_dag(const M3<R>& a) {
  M3<R> c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.e[3 * i + j] = cj(a.e[3 * j + i]);
  return c;
}
template <typename R> __host__ __device__ __forceinline__ M3<R> m_add(const M3<R>& a, const M3<R>& b) { M3<R> c; for (int k = 0; k < 9; ++k) c.e[k] = a.e[k] + b.e[k]; return c; }
template <typename R> __host__ __device__ __forceinline__ M3<R> m_sub(const M3<R>& a, const M3<R>& b) { M3<R> c; for (int k = 0; k < 9; ++k) c.e[k] = a.e[k] - b.e[k]; return c; }
template <typename R> __host__ __device__ __forceinline__ M3<R> m_scale(cx<R> s, const M3<R>& a) { M3<R> c; for (int k = 0; k < 9; ++k) c.e[k] = s * a.e[k]; return c; }
template <typename R> __host__ __device__ __forceinline__ M3<R> m_rscale(R s, const M3<R>& a) { M3<R> c; for (int k = 0; k < 9; ++k) c.e[k] = s * a.e[k]; return c; }

// ---------------------------------------------------------------------------- W layout
// Per site the stored forward set is NMAT colour matrices (see ok_precompute.cu for the list).
// Sites are grouped in blocks of 32 consecutive sites; within a block, element e (0..8) of
// matrix m of the site in lane l lives at ((blk * NMAT + m) * 9 + e) * 32 + l, so a warp
// handling 32 consecutive sites reads each element as one contiguous 32-wide row.
constexpr int NMAT = 43;
constexpr int LANES = 32;
constexpr int SITE_ELEMS = NMAT * 9;   // complex numbers stored per site

// Matrix indices inside a site record.
constexpr int M_Y0P = 0;    // 1/4 (D0 + c0 + i S0): blocks (00 minus c0/4 part) y3, (01), (10)
constexpr int M_Y0M = 3;    // 1/4 (D0 + c0 - i S0)
constexpr int M_UT = 6;     // U_t / 2
constexpr int M_ST = 7;     // S^+_4 / 2: blocks (00) = -(11), (01), (10)
constexpr int M_WP = 10;    // direction i: 10 + 8 i + {0..3} = P+ / 2 blocks 00,01,10,11; +4.. P- / 2
constexpr int M_VII = 34;   // 34 + i: U_i(x) U_i(x+i)
constexpr int M_VIJ = 37;   // 37 + pair: (c2 / 4 u0) (U_i U_j(x+i) + U_j U_i(x+j)), pairs xy, xz, yz
constexpr int M_XIJ = 40;   // 40 + pair: (c2 / 4 u0) (U_i U_j^dag(x-j+i) + U_j^dag(x-j) U_i(x-j))

// Scalars of the stored representation.
struct WScalars {
  double u0, plaq, inv2kappa;
  double c0q;    // u0 / (2 kappa) / 4, on the diagonal blocks of Y0+-
  double a_ii;   // c4 / (2 u0)
  double b_ii;   // (c1 + 2 c2) / (4 u0)
};

// Lattice geometry passed by value to kernels.
struct Geom {
  int L[4];      // X, Y, Z, T
  int bcneg;     // bit mu set: antiperiodic in direction mu
  int V;         // number of sites
  int nblk;      // ceil(V / 32)
  int sms;       // set by persistent launches: multiprocessors of the device (0 = unknown)
  int S[4];      // site-index strides: 1, X, X Y, X Y Z
};

// ---------------------------------------------------------------------------- launch helpers
void count_launch();
// Kernels executed by replays of a CUDA graph (n > 0) or launched only into a graph capture (n < 0).
void adjust_launches(long long n);
unsigned long long launches();
void set_cuda_error(cudaError_t e);

// Brackets one kernel launch with CUDA events when tracing is enabled (ok_trace_enable).
struct TraceScope {
  const char* name;
  cudaStream_t st;
  cudaEvent_t a, b;  // start and end events; null when this launch is not traced
  TraceScope(const char* n, cudaStream_t s);
  ~TraceScope();
};

inline int grid_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

}  // namespace okgb

namespace okgb {
// Launch shapes chosen by the autotuner (ok_autotune); zero means the built-in default.
struct Tune {
  int staged[2];  // single right-hand side, [FP32 W, FP16 W]: 1 = stream the forward W by TMA
  int mr_nr[2];   // multi right-hand side: right-hand sides per thread (1..4)
  int mr_bx[2];   // multi right-hand side: blocks per grid row (0 = as many as fit)
};
}  // namespace okgb

// The opaque handle.
struct ok_W {
  okgb::Geom g;
  ok_lattice lat;
  int precs;
  okgb::WScalars sc;
  ok_coeffs coeffs;  // as given to ok_precompute_W (the on-the-fly apply evaluates the W formulas)
  void* W64;     // cx<double>[nblk * SITE_ELEMS * 32]
  void* W32;     // cx<float>[...]
  void* Wdf;     // cx<dd>[...]: FP64-accurate double-float copy
  void* W16;     // cx<__half>[...]: half-precision copy
  void* L32;     // cx<float>[nblk][4][9][32]: FP32 links, site-blocked (OK_W_LINKS), for the preconditioner network
  void* Wtc;     // [V][804] FP16 complex words: blocks of the tensor-core apply (OK_W_F16_TC, ok_tc.cu)
  void* EB32;    // cx<float>[nblk][6][9][32]: FP32 clover fields E_k, B_k, site-blocked (OK_W_OTF)
  size_t bytes;
  int device;
  mutable okgb::Tune tune;
};

#define OK_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) {                               \
      okgb::set_cuda_error(_e);                            \
      return OK_ECUDA;                                     \
    }                                                      \
  } while (0)

#define OK_LAUNCH_CHECK()                                  \
  do {                                                     \
    okgb::count_launch();                                  \
    cudaError_t _e = cudaGetLastError();                   \
    if (_e != cudaSuccess) {                               \
      okgb::set_cuda_error(_e);                            \
      return OK_ECUDA;                                     \
    }                                                      \
  } while (0)
