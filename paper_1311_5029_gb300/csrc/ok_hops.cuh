// Spinor loads and stores, the gather of a neighbour's spin projections, and the small spin and
// colour operations of the hops (Eq. minFlopForm in the h+- = u +- l basis of ok_apply.cu), shared
// by the stored-W apply (ok_apply.cu) and the on-the-fly apply (ok_apply_otf.cu).
#pragma once
#include "ok_pair.cuh"

namespace okgb {

constexpr int APPLY_THREADS = 128;

template <typename R> struct Half { cx<R> v[2][3]; };

// ---------------------------------------------------------------------------- loads
template <typename R>
__device__ __forceinline__ void load_spinor(const cx<R>* __restrict__ psi, int site, cx<R> (&v)[12]);

template <>
__device__ __forceinline__ void load_spinor<double>(const cx<double>* __restrict__ psi, int site, cx<double> (&v)[12]) {
  const double2* p = reinterpret_cast<const double2*>(psi) + (size_t)site * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 d = __ldg(p + k);
    v[k] = mk(d.x, d.y);
  }
}

template <>
__device__ __forceinline__ void load_spinor<float>(const cx<float>* __restrict__ psi, int site, cx<float> (&v)[12]) {
  const float4* p = reinterpret_cast<const float4*>(psi) + (size_t)site * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float4 d = __ldg(p + k);
    v[2 * k] = mk(d.x, d.y);
    v[2 * k + 1] = mk(d.z, d.w);
  }
}

template <typename R>
__device__ __forceinline__ void store_spinor(cx<R>* __restrict__ out, int site, const cx<R> (&v)[12]);

template <>
__device__ __forceinline__ void store_spinor<double>(cx<double>* __restrict__ out, int site, const cx<double> (&v)[12]) {
  double2* p = reinterpret_cast<double2*>(out) + (size_t)site * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = make_double2(v[k].re, v[k].im);
}

template <>
__device__ __forceinline__ void store_spinor<float>(cx<float>* __restrict__ out, int site, const cx<float> (&v)[12]) {
  float4* p = reinterpret_cast<float4*>(out) + (size_t)site * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
}

// Gather the neighbour at offset d and form h+ = u + l, h- = u - l (with the boundary sign).
template <typename R, int D0, int D1, int D2, int D3>
__device__ __forceinline__ int gather_h(const cx<R>* __restrict__ psi, const int (&c)[4], const Geom& g,
                                        Half<R>& hp, Half<R>& hm, Half<R>* up = nullptr, Half<R>* lo = nullptr) {
  bool neg;
  int n = nbr_site<D0, D1, D2, D3>(c, g, neg);
  cx<R> v[12];
  load_spinor<R>(psi, n, v);
  if (neg) {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = -v[k];
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      hp.v[s][a] = v[3 * s + a] + v[3 * (s + 2) + a];
      hm.v[s][a] = v[3 * s + a] - v[3 * (s + 2) + a];
      if (up) up->v[s][a] = v[3 * s + a];
      if (lo) lo->v[s][a] = v[3 * (s + 2) + a];
    }
  return n;
}

// sigma_k on a 2-spinor: out = sigma_k y  (k = 0, 1, 2 for x, y, z), added with factor f (+1 or -1)
template <typename R>
__device__ __forceinline__ void add_sigma(Half<R>& acc, int k, const Half<R>& y, R f) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (k == 0) {
      acc.v[0][a] = acc.v[0][a] + f * y.v[1][a];
      acc.v[1][a] = acc.v[1][a] + f * y.v[0][a];
    } else if (k == 1) {
      acc.v[0][a] = acc.v[0][a] + f * tmi(y.v[1][a]);
      acc.v[1][a] = acc.v[1][a] + f * ti(y.v[0][a]);
    } else {
      acc.v[0][a] = acc.v[0][a] + f * y.v[0][a];
      acc.v[1][a] = acc.v[1][a] - f * y.v[1][a];
    }
  }
}

template <typename R>
__device__ __forceinline__ void add_scaled(Half<R>& acc, R f, const Half<R>& y) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc.v[s][a].re = fma(f, y.v[s][a].re, acc.v[s][a].re);
      acc.v[s][a].im = fma(f, y.v[s][a].im, acc.v[s][a].im);
    }
}

// y_s = V h_s or V^dag h_s for both spins
template <typename R, bool DAG>
__device__ __forceinline__ void colour2(Half<R>& y, const M3<R>& V, const Half<R>& h) {
  if (DAG) { mdv(y.v[0], V, h.v[0]); mdv(y.v[1], V, h.v[1]); }
  else { mv(y.v[0], V, h.v[0]); mv(y.v[1], V, h.v[1]); }
}

}  // namespace okgb
