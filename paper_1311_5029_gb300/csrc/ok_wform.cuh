// The forward W matrices of one site (Sec. 2.2, Eqs. shifted_W_first .. shifted_W_last) in the
// stored representation of ok_precompute.cu, computed in precision R from the links and the
// clover fields E_k, B_k.  Two users: the precompute (R = double, or the double-float dd on the FP32
// pipes; every matrix is stored) and the on-the-fly apply (R = float; each group of matrices is
// built where a hop needs it and used at once).  The accessor A provides the inputs:
//   M3<R> A::U(int site, int mu)   the link U_mu(site)
//   M3<R> A::F(int site, int k)    E_k(site) for k = 0, 1, 2 and B_{k-3}(site) for k = 3, 4, 5
// Gauge fields are periodic, so neighbour sites wrap without a sign.
#pragma once
#include "ok_internal.cuh"

namespace okgb {

// ---------------------------------------------------------------------------- indexing
__device__ __forceinline__ int wrapi(int x, int L) {
  int r = x % L;
  return r < 0 ? r + L : r;
}

struct Site {
  int c[4];
};

__device__ __forceinline__ Site site_coords(int s, const Geom& g) {
  Site p;
  p.c[0] = s % g.L[0]; s /= g.L[0];
  p.c[1] = s % g.L[1]; s /= g.L[1];
  p.c[2] = s % g.L[2]; s /= g.L[2];
  p.c[3] = s;
  return p;
}

// Site index of x + (d0, d1, d2, d3) with periodic wrapping.
__device__ __forceinline__ int nbr(const Site& p, const Geom& g, int d0, int d1, int d2, int d3) {
  int x = wrapi(p.c[0] + d0, g.L[0]);
  int y = wrapi(p.c[1] + d1, g.L[1]);
  int z = wrapi(p.c[2] + d2, g.L[2]);
  int t = wrapi(p.c[3] + d3, g.L[3]);
  return x + g.L[0] * (y + g.L[1] * (z + g.L[2] * t));
}

__device__ __forceinline__ int nbr_dir(const Site& p, const Geom& g, int mu, int n, int nu = 0, int m = 0) {
  int d[4] = {0, 0, 0, 0};
  d[mu] += n;
  d[nu] += m;
  return nbr(p, g, d[0], d[1], d[2], d[3]);
}

__device__ __forceinline__ int levi(int i, int j, int k) {
  if (i == j || j == k || i == k) return 0;
  return ((j - i + 3) % 3 == 1) ? 1 : -1;
}

namespace wform {

// W^0: D0 = -(c_B zeta + 16 c5)/(2 u0^3) i sum sigma_k B_k, S0 = -(c_E zeta)/(2 u0^3) sum sigma_k E_k;
// yp[j], ym[j] are the stored blocks Y0P + j, Y0M + j of Y+- = (D0 +- i S0) / 4 =
// [[y_z, y_x - i y_y], [y_x + i y_y, -y_z]].
template <typename R, class A>
__device__ __forceinline__ void onsite(const A& a, int s, const ok_coeffs& c, double u0, M3<R> (&yp)[3], M3<R> (&ym)[3]) {
  const double u03 = u0 * u0 * u0;
  const R cd = (R)(-(c.c_B * c.zeta + 16.0 * c.c5) / (2.0 * u03));
  const R cs = (R)(-(c.c_E * c.zeta) / (2.0 * u03));
  const cx<R> I = mk<R>(0, 1);
  M3<R> p[3], m[3];
  for (int k = 0; k < 3; ++k) {
    M3<R> d = m_scale(mk<R>(0, cd), a.F(s, 3 + k));   // i cd B_k
    M3<R> ie = m_scale(I, m_rscale(cs, a.F(s, k)));   // i cs E_k
    p[k] = m_rscale((R)0.25, m_add(d, ie));
    m[k] = m_rscale((R)0.25, m_sub(d, ie));
  }
  yp[0] = p[2];
  yp[1] = m_sub(p[0], m_scale(I, p[1]));
  yp[2] = m_add(p[0], m_scale(I, p[1]));
  ym[0] = m[2];
  ym[1] = m_sub(m[0], m_scale(I, m[1]));
  ym[2] = m_add(m[0], m_scale(I, m[1]));
}

// W^+_4 = [[0, S4], [S4, -U4]] with S4 = c_EE/(2 u0^4) (U_t E(x+t) - E(x) U_t), summed over sigma_k:
// uh = U_t / 2 (stored M_UT) and t[j] the stored blocks M_ST + j of S4 / 2.
template <typename R, class A>
__device__ __forceinline__ void temporal(const A& a, const Site& p, const Geom& g, int s, const ok_coeffs& c, double u0,
                                         M3<R>& uh, M3<R> (&t)[3]) {
  const double u04 = u0 * u0 * u0 * u0;
  const cx<R> I = mk<R>(0, 1);
  const M3<R> Ut = a.U(s, 3);
  const int st = nbr_dir(p, g, 3, 1);
  const R ct = (R)(0.5 * c.c_EE / (2.0 * u04));
  M3<R> tk[3];
  for (int k = 0; k < 3; ++k) tk[k] = m_rscale(ct, m_sub(m_mul(Ut, a.F(st, k)), m_mul(a.F(s, k), Ut)));
  uh = m_rscale((R)0.5, Ut);
  t[0] = tk[2];
  t[1] = m_sub(tk[0], m_scale(I, tk[1]));
  t[2] = m_add(tk[0], m_scale(I, tk[1]));
}

// W^+_i = [[D, S], [S, D]] for spatial direction i: put(sg * 4 + j, block) receives the stored
// blocks M_WP + 8 i + 4 sg + j, the 2x2 spin blocks (00, 01, 10, 11) of (D +- S) / 2, as they are
// formed (a caller that stores them keeps no array of them).
//   S = 1 (x) b0 + sum_l sigma_l (x) b_l,  D = 1 (x) a0 + sum_l sigma_l (x) a_l.
template <typename R, class A, class Put>
__device__ __forceinline__ void spatial_to(const A& a, const Site& p, const Geom& g, int s, int i, const ok_coeffs& c,
                                           double u0, Put&& put) {
  const double u04 = u0 * u0 * u0 * u0;
  const cx<R> I = mk<R>(0, 1);
  const M3<R> Ui = a.U(s, i);
  const int si = nbr_dir(p, g, i, 1);
  const R c3f = (R)(c.c3 / (2.0 * u04));
  M3<R> b[4], av[4];
  // b0 = i c3f (U_i B_i(x+i) + B_i(x) U_i)
  b[0] = m_scale(mk<R>(0, c3f), m_add(m_mul(Ui, a.F(si, 3 + i)), m_mul(a.F(s, 3 + i), Ui)));
  for (int l = 0; l < 3; ++l) {
    M3<R> acc = (l == i) ? m_rscale((R)(0.5 * (c.zeta - 2.0 * c.c1 - 12.0 * c.c2)), Ui) : m_zero<R>();
    for (int k = 0; k < 3; ++k) {
      const int e = levi(i, k, l);
      if (e == 0) continue;
      acc = m_sub(acc, m_rscale(c3f * (R)e, m_sub(m_mul(Ui, a.F(si, 3 + k)), m_mul(a.F(s, 3 + k), Ui))));
    }
    b[1 + l] = acc;
  }
  av[0] = m_rscale((R)(-0.5 * (c.r_s * c.zeta + 8.0 * c.c4)), Ui);
  const R cst = (R)(0.25 * c.c5 * (1.0 / (u0 * u0) - 1.0 / u04));
  const R c5f = (R)(c.c5 / u04);
  M3<R> staple[3];
  for (int k = 0; k < 3; ++k) {
    if (k == i) { staple[k] = m_zero<R>(); continue; }
    // U_k(x) U_i(x+k) U_k(x+i)^dag - U_k(x-k)^dag U_i(x-k) U_k(x-k+i)
    const M3<R> up = m_mul(m_mul(a.U(s, k), a.U(nbr_dir(p, g, k, 1), i)), m_dag(a.U(si, k)));
    const int smk = nbr_dir(p, g, k, -1);
    const M3<R> dn = m_mul(m_mul(m_dag(a.U(smk, k)), a.U(smk, i)), a.U(nbr_dir(p, g, k, -1, i, 1), k));
    staple[k] = m_sub(up, dn);
  }
  for (int l = 0; l < 3; ++l) {
    M3<R> acc = m_zero<R>();
    for (int k = 0; k < 3; ++k) {
      const int e = levi(i, l, k);
      if (e == 0) continue;
      acc = m_add(acc, m_scale(mk<R>(0, cst * (R)e), staple[k]));
    }
    if (l != i) acc = m_add(acc, m_scale(mk<R>(0, c5f), m_add(m_mul(Ui, a.F(si, 3 + l)), m_mul(a.F(s, 3 + l), Ui))));
    av[1 + l] = acc;
  }
  // blocks of (D +- S)/2: 00 = q0 + q3, 01 = q1 - i q2, 10 = q1 + i q2, 11 = q0 - q3
  for (int sg = 0; sg < 2; ++sg) {
    M3<R> w[4];
    for (int k = 0; k < 4; ++k) w[k] = m_rscale((R)0.5, sg == 0 ? m_add(av[k], b[k]) : m_sub(av[k], b[k]));
    put(4 * sg + 0, m_add(w[0], w[3]));
    put(4 * sg + 1, m_sub(w[1], m_scale(I, w[2])));
    put(4 * sg + 2, m_add(w[1], m_scale(I, w[2])));
    put(4 * sg + 3, m_sub(w[0], w[3]));
  }
}
// The same into an array q[8].
template <typename R, class A>
__device__ __forceinline__ void spatial(const A& a, const Site& p, const Geom& g, int s, int i, const ok_coeffs& c,
                                        double u0, M3<R> (&q)[8]) {
  spatial_to<R>(a, p, g, s, i, c, u0, [&](int k, const M3<R>& m) { q[k] = m; });
}

// W^{++}_ii: the colour matrix V = U_i(x) U_i(x+i) (stored M_VII + i).
template <typename R, class A>
__device__ __forceinline__ M3<R> twohop(const A& a, const Site& p, const Geom& g, int s, int i) {
  return m_mul(a.U(s, i), a.U(nbr_dir(p, g, i, 1), i));
}

// W^{++}_ij and W^{+-}_ij of the pair i < j: v = c2/(4 u0) (U_i(x) U_j(x+i) + U_j(x) U_i(x+j)) and
// x = c2/(4 u0) (U_i(x) U_j(x-j+i)^dag + U_j(x-j)^dag U_i(x-j)) (stored M_VIJ + pair, M_XIJ + pair).
template <typename R, class A>
__device__ __forceinline__ void diag_v(const A& a, const Site& p, const Geom& g, int s, int i, int j, const ok_coeffs& c,
                                       double u0, M3<R>& v) {
  const R cij = (R)(c.c2 / (4.0 * u0));
  v = m_rscale(cij, m_add(m_mul(a.U(s, i), a.U(nbr_dir(p, g, i, 1), j)), m_mul(a.U(s, j), a.U(nbr_dir(p, g, j, 1), i))));
}
template <typename R, class A>
__device__ __forceinline__ void diag_x(const A& a, const Site& p, const Geom& g, int s, int i, int j, const ok_coeffs& c,
                                       double u0, M3<R>& x) {
  const R cij = (R)(c.c2 / (4.0 * u0));
  const int smj = nbr_dir(p, g, j, -1);
  x = m_rscale(cij, m_add(m_mul(a.U(s, i), m_dag(a.U(nbr_dir(p, g, j, -1, i, 1), j))),
                          m_mul(m_dag(a.U(smj, j)), a.U(smj, i))));
}

}  // namespace wform
}  // namespace okgb
