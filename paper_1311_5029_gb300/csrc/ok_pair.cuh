// Device helpers shared by the apply kernels: W element loads, colour algebra, lattice
// geometry and the thread-pair hop functions (two threads per site, one per spin projection).
#pragma once

#include "ok_launch.cuh"

#include <type_traits>

namespace okgb {

// Read-only load of one FP32 W element.  Variant 0: plain __ldg; 1: not allocated in L1 (a W
// element is used by exactly one thread, so L1 is left to the neighbour spinors); 2: with a 256-byte
// L2 prefetch hint (a matrix element row of 32 sites is 256 bytes, read by two warps); 3: both.
#ifndef OK_W_LOAD
#define OK_W_LOAD 0
#endif
__device__ __forceinline__ float2 ldg_w(const float2* p) {
  float2 d;
#if OK_W_LOAD == 1
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(d.x), "=f"(d.y) : "l"(p));
#elif OK_W_LOAD == 2
  asm volatile("ld.global.nc.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(d.x), "=f"(d.y) : "l"(p));
#elif OK_W_LOAD == 3
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(d.x), "=f"(d.y) : "l"(p));
#else
  d = __ldg(p);
#endif
  return d;
}

// Matrix m of the site record of `site`.
template <typename R>
__device__ __forceinline__ M3<R> wmat(const cx<R>* __restrict__ W, int site, int m) {
  const size_t base = ((size_t)(site >> 5) * NMAT + m) * (9 * LANES) + (site & 31);
  M3<R> a;
  if constexpr (std::is_same<R, double>::value) {
    const double2* p = reinterpret_cast<const double2*>(W) + base;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      double2 d = __ldg(p + e * LANES);
      a.e[e] = mk<R>(d.x, d.y);
    }
  } else {
    const float2* p = reinterpret_cast<const float2*>(W) + base;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      float2 d = ldg_w(p + e * LANES);
      a.e[e] = mk<R>(d.x, d.y);
    }
  }
  return a;
}

// Matrix m of the site record of `site` from the half-precision copy, widened to FP32.
__device__ __forceinline__ M3<float> wmat(const cx<__half>* __restrict__ W, int site, int m) {
  const size_t base = ((size_t)(site >> 5) * NMAT + m) * (9 * LANES) + (site & 31);
  const unsigned* p = reinterpret_cast<const unsigned*>(W) + base;
  M3<float> a;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const unsigned u = __ldg(p + e * LANES);
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
    a.e[e] = mk<float>(f.x, f.y);
  }
  return a;
}

// Arithmetic type of a stored W element type (FP16 elements are widened to FP32).
template <typename WT> struct WReal { using type = WT; };
template <> struct WReal<__half> { using type = float; };

// W source reading any site's record from global memory.
template <typename WT> struct GlobalW {
  const cx<WT>* __restrict__ p;
  __device__ __forceinline__ M3<typename WReal<WT>::type> operator()(int site, int m) const { return wmat(p, site, m); }
};

// ---------------------------------------------------------------------------- colour algebra
// y += A v, y -= A v, y += A^dag v, y -= A^dag v
template <typename R> __device__ __forceinline__ void mv_add(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) y[r] = fma_c(A.e[3 * r + c], v[c], y[r]);
}
template <typename R> __device__ __forceinline__ void mv_sub(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) y[r] = fma_c(-A.e[3 * r + c], v[c], y[r]);
}
template <typename R> __device__ __forceinline__ void mdv_add(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) y[r] = fma_cj(A.e[3 * c + r], v[c], y[r]);
}
template <typename R> __device__ __forceinline__ void mdv_sub(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) y[r] = fma_cj(-A.e[3 * c + r], v[c], y[r]);
}
template <typename R> __device__ __forceinline__ void mv(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    y[r] = A.e[3 * r] * v[0];
    y[r] = fma_c(A.e[3 * r + 1], v[1], y[r]);
    y[r] = fma_c(A.e[3 * r + 2], v[2], y[r]);
  }
}
template <typename R> __device__ __forceinline__ void mdv(cx<R> (&y)[3], const M3<R>& A, const cx<R> (&v)[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    y[r] = cj(A.e[r]) * v[0];
    y[r] = fma_cj(A.e[3 + r], v[1], y[r]);
    y[r] = fma_cj(A.e[6 + r], v[2], y[r]);
  }
}

// ---------------------------------------------------------------------------- geometry
// Neighbour x + d with fermion boundary sign; |d_mu| <= 2.  The coordinate is wrapped by at most
// two conditional subtractions (two are needed only when L_mu < |d_mu|, on lattices of extent 1
// or 2); the sign flips once per wrap across an antiperiodic boundary.
template <int D0, int D1, int D2, int D3>
__device__ __forceinline__ int nbr_site(const int (&c)[4], const Geom& g, bool& neg) {
  const int d[4] = {D0, D1, D2, D3};
  int idx = 0;
  neg = false;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    int x = c[mu];
    if (d[mu] != 0) {
      const int L = g.L[mu];
      x += d[mu];
      int wraps = 0;
      if (d[mu] > 0) {
        if (x >= L) { x -= L; wraps = 1; if (x >= L) { x -= L; wraps = 2; } }
      } else {
        if (x < 0) { x += L; wraps = 1; if (x < 0) { x += L; wraps = 2; } }
      }
      if (((g.bcneg >> mu) & 1) && (wraps & 1)) neg = !neg;
    }
    idx += x * g.S[mu];
  }
  return idx;
}


// ============================================================================ two threads per site
// The pair (lanes 2k, 2k+1) shares one site.  Thread p = 0 accumulates acc+ and loads the upper
// spin half u of every spinor it needs, thread p = 1 accumulates acc- and loads the lower half l;
// the other half arrives through one shuffle.  Spatial hops then split without duplicated work:
// p = 0 uses (D + S)/2 forward and (D - S)/2 backward, p = 1 the other two.  W^0, the temporal hop
// and the colour matrices of the two-hop terms are read by both threads (the same addresses, one
// transaction per warp).  Half the registers per thread and twice the warps per SM keep more
// global loads in flight than one thread per site can.

template <typename R> struct H6 { cx<R> v[2][3]; };

template <typename R>
__device__ __forceinline__ void load_half(const cx<R>* __restrict__ psi, int site, int p, H6<R>& h) {
  if constexpr (sizeof(R) == 8) {
    const double2* q = reinterpret_cast<const double2*>(psi) + (size_t)site * 12 + 6 * p;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      double2 d = __ldg(q + k);
      h.v[k / 3][k % 3] = mk<R>(d.x, d.y);
    }
  } else {
    const float4* q = reinterpret_cast<const float4*>(psi) + (size_t)site * 6 + 3 * p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 d = __ldg(q + k);
      h.v[(2 * k) / 3][(2 * k) % 3] = mk<R>(d.x, d.y);
      h.v[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk<R>(d.z, d.w);
    }
  }
}

template <typename R>
__device__ __forceinline__ void store_half(cx<R>* __restrict__ out, int site, int p, const H6<R>& h) {
  if constexpr (sizeof(R) == 8) {
    double2* q = reinterpret_cast<double2*>(out) + (size_t)site * 12 + 6 * p;
#pragma unroll
    for (int k = 0; k < 6; ++k) q[k] = make_double2(h.v[k / 3][k % 3].re, h.v[k / 3][k % 3].im);
  } else {
    float4* q = reinterpret_cast<float4*>(out) + (size_t)site * 6 + 3 * p;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const cx<R>& a = h.v[(2 * k) / 3][(2 * k) % 3];
      const cx<R>& b = h.v[(2 * k + 1) / 3][(2 * k + 1) % 3];
      q[k] = make_float4(a.re, a.im, b.re, b.im);
    }
  }
}

template <typename R>
__device__ __forceinline__ H6<R> partner(const H6<R>& h, unsigned mask) {
  H6<R> o;
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      o.v[s][a].re = __shfl_xor_sync(mask, h.v[s][a].re, 1);
      o.v[s][a].im = __shfl_xor_sync(mask, h.v[s][a].im, 1);
    }
  return o;
}

struct Pair {
  int p;          // 0: acc+ thread, 1: acc- thread
  unsigned mask;  // the two lanes of the pair
};

// Gather the neighbour at offset D: mine = own half, oth = partner's half, h = h+ (p = 0) or h- (p = 1).
template <typename R, int D0, int D1, int D2, int D3>
__device__ __forceinline__ int gather_pair(const cx<R>* __restrict__ psi, const int (&c)[4], const Geom& g, const Pair& pr,
                                           H6<R>& h, H6<R>* u = nullptr, H6<R>* l = nullptr) {
  bool neg;
  int n = nbr_site<D0, D1, D2, D3>(c, g, neg);
  H6<R> mine;
  load_half<R>(psi, n, pr.p, mine);
  if (neg) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) mine.v[s][a] = -mine.v[s][a];
  }
  H6<R> oth = partner(mine, pr.mask);
  // p = 0: h+ = mine + oth (u = mine);  p = 1: h- = oth - mine (u = oth)
  const R sg = pr.p ? R(-1) : R(1);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cx<R> m = mine.v[s][a], o = oth.v[s][a];
      h.v[s][a] = mk<R>(sg * m.re + o.re, sg * m.im + o.im);
      if (u) u->v[s][a] = pr.p ? o : m;
      if (l) l->v[s][a] = pr.p ? m : o;
    }
  return n;
}

template <typename R, bool DAG, typename WS>
__device__ __forceinline__ void block2h(const WS& W, int site, int m, const H6<R>& h, H6<R>& acc) {
  M3<R> b;
  b = W(site, m + 0);
  if (DAG) mdv_add(acc.v[0], b, h.v[0]); else mv_add(acc.v[0], b, h.v[0]);
  b = W(site, m + 1);
  if (DAG) mdv_add(acc.v[1], b, h.v[0]); else mv_add(acc.v[0], b, h.v[1]);
  b = W(site, m + 2);
  if (DAG) mdv_add(acc.v[0], b, h.v[1]); else mv_add(acc.v[1], b, h.v[0]);
  b = W(site, m + 3);
  if (DAG) mdv_add(acc.v[1], b, h.v[1]); else mv_add(acc.v[1], b, h.v[1]);
}

template <typename R>
__device__ __forceinline__ void add_sigma_h(H6<R>& acc, int k, const H6<R>& y, R f) {
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

template <typename R, bool DAG>
__device__ __forceinline__ void colour2h(H6<R>& y, const M3<R>& V, const H6<R>& h) {
  if (DAG) { mdv(y.v[0], V, h.v[0]); mdv(y.v[1], V, h.v[1]); }
  else { mv(y.v[0], V, h.v[0]); mv(y.v[1], V, h.v[1]); }
}

// Each hop function takes FWD / BWD flags so that the forward and the backward halves of the
// stencil can run in different warps (the split kernel below).
template <typename R, int I, bool FWD = true, bool BWD = true, typename WS>
__device__ __forceinline__ void pair_spatial(const WS& W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                             const Geom& g, int s, const Pair& pr, H6<R>& acc) {
  const int base = M_WP + 8 * I;
  H6<R> h;
  if constexpr (FWD) {
    gather_pair<R, I == 0, I == 1, I == 2, 0>(psi, c, g, pr, h);
    block2h<R, false>(W, s, base + 4 * pr.p, h, acc);
  }
  if constexpr (BWD) {
    int n = gather_pair<R, -(I == 0), -(I == 1), -(I == 2), 0>(psi, c, g, pr, h);
    block2h<R, true>(W, n, base + 4 * (1 - pr.p), h, acc);
  }
}

// acc+ += S h+ - U l (p = 0);  acc- += -S h- + U l (p = 1)   [forward, matrices at x]
// acc+ += -U^dag u - S^dag h+;  acc- += -U^dag u + S^dag h-   [backward, matrices at x - t]
template <typename R, bool FWD = true, bool BWD = true, typename WS>
__device__ __forceinline__ void pair_time(const WS& W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                          const Geom& g, int s, const Pair& pr, H6<R>& acc) {
  const R sg = pr.p ? R(-1) : R(1);
  H6<R> h, u, l;
  if constexpr (FWD) {
    gather_pair<R, 0, 0, 0, 1>(psi, c, g, pr, h, nullptr, &l);
    // acc += sg (S h - U l),  S = [[s3, n1], [n2, -s3]]
    H6<R> sh;
    M3<R> s3 = W(s, M_ST + 0);
    mv(sh.v[0], s3, h.v[0]);
    mv(sh.v[1], s3, h.v[1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) sh.v[1][a] = -sh.v[1][a];
    M3<R> n1 = W(s, M_ST + 1);
    mv_add(sh.v[0], n1, h.v[1]);
    M3<R> n2 = W(s, M_ST + 2);
    mv_add(sh.v[1], n2, h.v[0]);
    M3<R> U = W(s, M_UT);
    mv_sub(sh.v[0], U, l.v[0]);
    mv_sub(sh.v[1], U, l.v[1]);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc.v[q][a].re = fma(sg, sh.v[q][a].re, acc.v[q][a].re);
        acc.v[q][a].im = fma(sg, sh.v[q][a].im, acc.v[q][a].im);
      }
  }
  if constexpr (BWD) {
    int n = gather_pair<R, 0, 0, 0, -1>(psi, c, g, pr, h, &u, nullptr);
    // S^dag h = [[s3^dag, n2^dag], [n1^dag, -s3^dag]] h ; acc += -U^dag u - sg S^dag h
    H6<R> sh;
    M3<R> s3 = W(n, M_ST + 0);
    mdv(sh.v[0], s3, h.v[0]);
    mdv(sh.v[1], s3, h.v[1]);
#pragma unroll
    for (int a = 0; a < 3; ++a) sh.v[1][a] = -sh.v[1][a];
    M3<R> n2 = W(n, M_ST + 2);
    mdv_add(sh.v[0], n2, h.v[1]);
    M3<R> n1 = W(n, M_ST + 1);
    mdv_add(sh.v[1], n1, h.v[0]);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc.v[q][a].re = fma(-sg, sh.v[q][a].re, acc.v[q][a].re);
        acc.v[q][a].im = fma(-sg, sh.v[q][a].im, acc.v[q][a].im);
      }
    M3<R> U = W(n, M_UT);
    mdv_sub(acc.v[0], U, u.v[0]);
    mdv_sub(acc.v[1], U, u.v[1]);
  }
}

template <typename R>
__device__ __forceinline__ void add_scaled_h(H6<R>& acc, R a, const H6<R>& y) {
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      acc.v[q][k].re = fma(a, y.v[q][k].re, acc.v[q][k].re);
      acc.v[q][k].im = fma(a, y.v[q][k].im, acc.v[q][k].im);
    }
}

// W^{++}_ii: acc+- += (a +- b sigma_i) V h+-  forward,  (a -+ b sigma_i) V^dag h+-  backward.
template <typename R, int I, bool FWD = true, bool BWD = true, typename WS>
__device__ __forceinline__ void pair_two(const WS& W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                         const Geom& g, int s, const Pair& pr, R a, R b, H6<R>& acc) {
  const R sb = pr.p ? -b : b;
  H6<R> h, y;
  if constexpr (FWD) {
    gather_pair<R, 2 * (I == 0), 2 * (I == 1), 2 * (I == 2), 0>(psi, c, g, pr, h);
    M3<R> V = W(s, M_VII + I);
    colour2h<R, false>(y, V, h);
    add_scaled_h(acc, a, y);
    add_sigma_h(acc, I, y, sb);
  }
  if constexpr (BWD) {
    int n = gather_pair<R, -2 * (I == 0), -2 * (I == 1), -2 * (I == 2), 0>(psi, c, g, pr, h);
    M3<R> V = W(n, M_VII + I);
    colour2h<R, true>(y, V, h);
    add_scaled_h(acc, a, y);
    add_sigma_h(acc, I, y, -sb);
  }
}

// Diagonal pair (I, J): acc+- += +-(s_I + s_J) V h, -+(s_I + s_J) V^dag h (x-I-J),
//                       +-(s_I - s_J) X h (x+I-J), -+(s_I - s_J) X^dag h (x-I+J).
template <typename R, int I, int J, int P, bool FWD = true, bool BWD = true, typename WS>
__device__ __forceinline__ void pair_diag(const WS& W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                          const Geom& g, int s, const Pair& pr, H6<R>& acc) {
  constexpr int A0 = (I == 0) + (J == 0), A1 = (I == 1) + (J == 1), A2 = (I == 2) + (J == 2);
  constexpr int B0 = (I == 0) - (J == 0), B1 = (I == 1) - (J == 1), B2 = (I == 2) - (J == 2);
  const R sg = pr.p ? R(-1) : R(1);
  H6<R> h, y;
  M3<R> V;
  if constexpr (FWD) {
    gather_pair<R, A0, A1, A2, 0>(psi, c, g, pr, h);
    V = W(s, M_VIJ + P);
    colour2h<R, false>(y, V, h); add_sigma_h(acc, I, y, sg); add_sigma_h(acc, J, y, sg);
    gather_pair<R, B0, B1, B2, 0>(psi, c, g, pr, h);
    V = W(s, M_XIJ + P);
    colour2h<R, false>(y, V, h); add_sigma_h(acc, I, y, sg); add_sigma_h(acc, J, y, -sg);
  }
  if constexpr (BWD) {
    int n = gather_pair<R, -A0, -A1, -A2, 0>(psi, c, g, pr, h);
    V = W(n, M_VIJ + P);
    colour2h<R, true>(y, V, h); add_sigma_h(acc, I, y, -sg); add_sigma_h(acc, J, y, -sg);
    n = gather_pair<R, -B0, -B1, -B2, 0>(psi, c, g, pr, h);
    V = W(n, M_XIJ + P);
    colour2h<R, true>(y, V, h); add_sigma_h(acc, I, y, -sg); add_sigma_h(acc, J, y, sg);
  }
}

// On-site term W^0 psi_x (both halves of the pair): p = 0 forms A = Y+ (u - i l), p = 1 forms
// B = Y- (u + i l); acc = (A + B) + i (A - B) for p = 0 and (A + B) - i (A - B) for p = 1.
template <typename R, typename WS>
__device__ __forceinline__ void pair_onsite(const WS& W, const cx<R>* __restrict__ psi, int s, const Pair& pr, R c0q,
                                            H6<R>& acc) {
  H6<R> mine, oth, v, Rm;
  load_half<R>(psi, s, pr.p, mine);
  oth = partner(mine, pr.mask);
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cx<R> u = pr.p ? oth.v[q][k] : mine.v[q][k];
      cx<R> l = pr.p ? mine.v[q][k] : oth.v[q][k];
      v.v[q][k] = pr.p ? u + ti(l) : u - ti(l);
      Rm.v[q][k] = c0q * v.v[q][k];
    }
  const int m0 = pr.p ? M_Y0M : M_Y0P;
  M3<R> y = W(s, m0 + 0);
  mv_add(Rm.v[0], y, v.v[0]); mv_sub(Rm.v[1], y, v.v[1]);
  y = W(s, m0 + 1);
  mv_add(Rm.v[0], y, v.v[1]);
  y = W(s, m0 + 2);
  mv_add(Rm.v[1], y, v.v[0]);
  H6<R> Rp = partner(Rm, pr.mask);
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.v[q][k] = (Rm.v[q][k] + Rp.v[q][k]) + ti(Rm.v[q][k] - Rp.v[q][k]);
}

}  // namespace okgb
