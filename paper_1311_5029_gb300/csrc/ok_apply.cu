// M psi in the W form (Eq. minFlopForm): one thread per site gathers the on-site spinor and the
// 26 neighbour spinors (x +- mu, x +- 2i, x +- i +- j) and multiplies them by the stored forward
// matrices at x, or by the backward ones obtained on the fly from the forward matrices stored at
// the neighbour (Eqs. conjugate and opp_diag_pre_mat: W^-_{mu,x} = gamma5 W^{+ dagger}_{mu,x-mu}
// gamma5 and so on).
//
// Spin handling.  With psi = (u, l) its upper and lower 2-spin halves, every hop except W^0 is
// block diagonal in h+- = u +- l, so the kernel accumulates
//   acc+ = (out_u + out_l) / 2,   acc- = (out_u - out_l) / 2
// (the 1/2 is folded into the stored matrices) and writes out_u = acc+ + acc-,
// out_l = acc+ - acc- at the end.  W^0 is block diagonal in u -+ i l instead.  In this basis the
// 148 colour matrix-vector products per site are the only dense work.
//
// Precision R = double or float: loads, arithmetic and stores in R.  Fused epilogues feed the
// BiCGStab reductions (ok_reduce.cuh) without a second pass over the output.
#include "ok_hops.cuh"

#include <type_traits>

namespace okgb {

// ---------------------------------------------------------------------------- hop kernels
// acc0 += B00 h0 + B01 h1, acc1 += B10 h0 + B11 h1 (blocks at matrices m .. m+3 of `site`);
// DAG: acc0 += B00^dag h0 + B10^dag h1, acc1 += B01^dag h0 + B11^dag h1.
template <typename R, bool DAG>
__device__ __forceinline__ void block2(const cx<R>* __restrict__ W, int site, int m, const Half<R>& h, Half<R>& acc) {
  M3<R> b;
  b = wmat(W, site, m + 0);
  if (DAG) mdv_add(acc.v[0], b, h.v[0]); else mv_add(acc.v[0], b, h.v[0]);
  b = wmat(W, site, m + 1);
  if (DAG) mdv_add(acc.v[1], b, h.v[0]); else mv_add(acc.v[0], b, h.v[1]);
  b = wmat(W, site, m + 2);
  if (DAG) mdv_add(acc.v[0], b, h.v[1]); else mv_add(acc.v[1], b, h.v[0]);
  b = wmat(W, site, m + 3);
  if (DAG) mdv_add(acc.v[1], b, h.v[1]); else mv_add(acc.v[1], b, h.v[1]);
}

// Spatial nearest neighbours in direction I.
template <typename R, int I>
__device__ __forceinline__ void hop_spatial(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                            const Geom& g, int s, Half<R>& ap, Half<R>& am) {
  constexpr int mp = M_WP + 8 * I, mm = mp + 4;
  Half<R> hp, hm;
  // forward: acc+ += (P+ / 2) h+, acc- += (P- / 2) h-, P at x
  gather_h<R, I == 0, I == 1, I == 2, 0>(psi, c, g, hp, hm);
  block2<R, false>(W, s, mp, hp, ap);
  block2<R, false>(W, s, mm, hm, am);
  // backward: acc+ += (P- / 2)^dag h+, acc- += (P+ / 2)^dag h-, P at x - I
  int n = gather_h<R, -(I == 0), -(I == 1), -(I == 2), 0>(psi, c, g, hp, hm);
  block2<R, true>(W, n, mm, hp, ap);
  block2<R, true>(W, n, mp, hm, am);
}

// Temporal nearest neighbours: W^+_4 = [[0, S], [S, -U]], W^-_4 = [[-U^dag, -S^dag], [-S^dag, 0]].
template <typename R>
__device__ __forceinline__ void hop_time(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                         const Geom& g, int s, Half<R>& ap, Half<R>& am) {
  Half<R> hp, hm, lo, up, w;
  // forward at x: acc+ += S h+ - U l, acc- += U l - S h- (stored halves)
  gather_h<R, 0, 0, 0, 1>(psi, c, g, hp, hm, nullptr, &lo);
  {
    M3<R> U = wmat(W, s, M_UT);
    colour2<R, false>(w, U, lo);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) { ap.v[q][a] = ap.v[q][a] - w.v[q][a]; am.v[q][a] = am.v[q][a] + w.v[q][a]; }
    M3<R> s3 = wmat(W, s, M_ST + 0);
    mv_add(ap.v[0], s3, hp.v[0]); mv_sub(ap.v[1], s3, hp.v[1]);
    mv_sub(am.v[0], s3, hm.v[0]); mv_add(am.v[1], s3, hm.v[1]);
    M3<R> n1 = wmat(W, s, M_ST + 1);
    mv_add(ap.v[0], n1, hp.v[1]); mv_sub(am.v[0], n1, hm.v[1]);
    M3<R> n2 = wmat(W, s, M_ST + 2);
    mv_add(ap.v[1], n2, hp.v[0]); mv_sub(am.v[1], n2, hm.v[0]);
  }
  // backward from x - t: acc+ += -U^dag u - S^dag h+, acc- += -U^dag u + S^dag h-
  int n = gather_h<R, 0, 0, 0, -1>(psi, c, g, hp, hm, &up, nullptr);
  {
    M3<R> U = wmat(W, n, M_UT);
    colour2<R, true>(w, U, up);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int a = 0; a < 3; ++a) { ap.v[q][a] = ap.v[q][a] - w.v[q][a]; am.v[q][a] = am.v[q][a] - w.v[q][a]; }
    // S^dag = [[s3^dag, n2^dag], [n1^dag, -s3^dag]]
    M3<R> s3 = wmat(W, n, M_ST + 0);
    mdv_sub(ap.v[0], s3, hp.v[0]); mdv_add(ap.v[1], s3, hp.v[1]);
    mdv_add(am.v[0], s3, hm.v[0]); mdv_sub(am.v[1], s3, hm.v[1]);
    M3<R> n1 = wmat(W, n, M_ST + 1);
    mdv_sub(ap.v[1], n1, hp.v[0]); mdv_add(am.v[1], n1, hm.v[0]);
    M3<R> n2 = wmat(W, n, M_ST + 2);
    mdv_sub(ap.v[0], n2, hp.v[1]); mdv_add(am.v[0], n2, hm.v[1]);
  }
}

// Straight two-hop neighbours x +- 2I: W^{++}_ii = (a + b sigma_i) V on h+, (a - b sigma_i) V on h-.
template <typename R, int I>
__device__ __forceinline__ void hop_two(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                        const Geom& g, int s, R a, R b, Half<R>& ap, Half<R>& am) {
  Half<R> hp, hm, y;
  gather_h<R, 2 * (I == 0), 2 * (I == 1), 2 * (I == 2), 0>(psi, c, g, hp, hm);
  M3<R> V = wmat(W, s, M_VII + I);
  colour2<R, false>(y, V, hp);
  add_scaled(ap, a, y); add_sigma(ap, I, y, b);
  colour2<R, false>(y, V, hm);
  add_scaled(am, a, y); add_sigma(am, I, y, -b);
  int n = gather_h<R, -2 * (I == 0), -2 * (I == 1), -2 * (I == 2), 0>(psi, c, g, hp, hm);
  V = wmat(W, n, M_VII + I);
  colour2<R, true>(y, V, hp);
  add_scaled(ap, a, y); add_sigma(ap, I, y, -b);
  colour2<R, true>(y, V, hm);
  add_scaled(am, a, y); add_sigma(am, I, y, b);
}

// Diagonal neighbours of the pair (I, J), I < J, P = pair index:
//   x+I+J: acc+ += (s_I + s_J) V h+, acc- -= (s_I + s_J) V h-             (V at x)
//   x-I-J: acc+ -= (s_I + s_J) V^dag h+, acc- += (s_I + s_J) V^dag h-     (V at x-I-J)
//   x+I-J: acc+ += (s_I - s_J) X h+, acc- -= (s_I - s_J) X h-             (X at x)
//   x-I+J: acc+ -= (s_I - s_J) X^dag h+, acc- += (s_I - s_J) X^dag h-     (X at x-I+J)
template <typename R, int I, int J, int P>
__device__ __forceinline__ void hop_diag(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi, const int (&c)[4],
                                         const Geom& g, int s, Half<R>& ap, Half<R>& am) {
  constexpr int A0 = (I == 0) + (J == 0), A1 = (I == 1) + (J == 1), A2 = (I == 2) + (J == 2);
  constexpr int B0 = (I == 0) - (J == 0), B1 = (I == 1) - (J == 1), B2 = (I == 2) - (J == 2);
  Half<R> hp, hm, y;
  M3<R> V;
  gather_h<R, A0, A1, A2, 0>(psi, c, g, hp, hm);
  V = wmat(W, s, M_VIJ + P);
  colour2<R, false>(y, V, hp); add_sigma(ap, I, y, R(1)); add_sigma(ap, J, y, R(1));
  colour2<R, false>(y, V, hm); add_sigma(am, I, y, R(-1)); add_sigma(am, J, y, R(-1));
  int n = gather_h<R, -A0, -A1, -A2, 0>(psi, c, g, hp, hm);
  V = wmat(W, n, M_VIJ + P);
  colour2<R, true>(y, V, hp); add_sigma(ap, I, y, R(-1)); add_sigma(ap, J, y, R(-1));
  colour2<R, true>(y, V, hm); add_sigma(am, I, y, R(1)); add_sigma(am, J, y, R(1));
  gather_h<R, B0, B1, B2, 0>(psi, c, g, hp, hm);
  V = wmat(W, s, M_XIJ + P);
  colour2<R, false>(y, V, hp); add_sigma(ap, I, y, R(1)); add_sigma(ap, J, y, R(-1));
  colour2<R, false>(y, V, hm); add_sigma(am, I, y, R(-1)); add_sigma(am, J, y, R(1));
  n = gather_h<R, -B0, -B1, -B2, 0>(psi, c, g, hp, hm);
  V = wmat(W, n, M_XIJ + P);
  colour2<R, true>(y, V, hp); add_sigma(ap, I, y, R(-1)); add_sigma(ap, J, y, R(1));
  colour2<R, true>(y, V, hm); add_sigma(am, I, y, R(1)); add_sigma(am, J, y, R(-1));
}

// ---------------------------------------------------------------------------- the kernel
template <typename R, int EPI>
__global__ void __launch_bounds__(APPLY_THREADS) apply_kernel(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi,
                                                              cx<R>* __restrict__ out, Geom g, R c0q, R a_ii, R b_ii,
                                                              EpiArgs<R> ep) {
  if (ep.halt && *ep.halt) return;
  const int s = blockIdx.x * APPLY_THREADS + threadIdx.x;
  double red[3] = {0.0, 0.0, 0.0};
  if (s < g.V) {
    int c[4];
    {
      int r = s;
      c[0] = r % g.L[0]; r /= g.L[0];
      c[1] = r % g.L[1]; r /= g.L[1];
      c[2] = r % g.L[2]; c[3] = r / g.L[2];
    }
    Half<R> ap, am;
    cx<R> x0[12];
    // on-site: a = u - i l, b = u + i l; A = Y+ a, B = Y- b; acc+- = (A + B) +- i (A - B)
    load_spinor<R>(psi, s, x0);
    {
      Half<R> a, b, A, B;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          a.v[q][k] = x0[3 * q + k] - ti(x0[3 * (q + 2) + k]);
          b.v[q][k] = x0[3 * q + k] + ti(x0[3 * (q + 2) + k]);
          A.v[q][k] = c0q * a.v[q][k];
          B.v[q][k] = c0q * b.v[q][k];
        }
      M3<R> y = wmat(W, s, M_Y0P + 0);
      mv_add(A.v[0], y, a.v[0]); mv_sub(A.v[1], y, a.v[1]);
      y = wmat(W, s, M_Y0P + 1);
      mv_add(A.v[0], y, a.v[1]);
      y = wmat(W, s, M_Y0P + 2);
      mv_add(A.v[1], y, a.v[0]);
      y = wmat(W, s, M_Y0M + 0);
      mv_add(B.v[0], y, b.v[0]); mv_sub(B.v[1], y, b.v[1]);
      y = wmat(W, s, M_Y0M + 1);
      mv_add(B.v[0], y, b.v[1]);
      y = wmat(W, s, M_Y0M + 2);
      mv_add(B.v[1], y, b.v[0]);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          cx<R> P = A.v[q][k] + B.v[q][k], Q = A.v[q][k] - B.v[q][k];
          ap.v[q][k] = P + ti(Q);
          am.v[q][k] = P - ti(Q);
        }
    }
    hop_spatial<R, 0>(W, psi, c, g, s, ap, am);
    hop_spatial<R, 1>(W, psi, c, g, s, ap, am);
    hop_spatial<R, 2>(W, psi, c, g, s, ap, am);
    hop_time<R>(W, psi, c, g, s, ap, am);
    hop_two<R, 0>(W, psi, c, g, s, a_ii, b_ii, ap, am);
    hop_two<R, 1>(W, psi, c, g, s, a_ii, b_ii, ap, am);
    hop_two<R, 2>(W, psi, c, g, s, a_ii, b_ii, ap, am);
    hop_diag<R, 0, 1, 0>(W, psi, c, g, s, ap, am);
    hop_diag<R, 0, 2, 1>(W, psi, c, g, s, ap, am);
    hop_diag<R, 1, 2, 2>(W, psi, c, g, s, ap, am);

    cx<R> o[12];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        o[3 * q + k] = ap.v[q][k] + am.v[q][k];
        o[3 * (q + 2) + k] = ap.v[q][k] - am.v[q][k];
      }
    if (EPI == EPI_RESID) {
      cx<R> bv[12];
      load_spinor<R>(ep.b, s, bv);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        o[k] = bv[k] - o[k];
        const double ore = (double)o[k].re, oim = (double)o[k].im;
        const double bre = (double)bv[k].re, bim = (double)bv[k].im;
        red[0] += ore * ore + oim * oim;
        red[1] += bre * bre + bim * bim;
      }
    }
    store_spinor<R>(out, s, o);
    if constexpr (EPI == EPI_DOT) {
      cx<R> rh[12];
      load_spinor<R>(ep.rhat, s, rh);
      cx<R> d = mk<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 12; ++k) d = fma_cj(rh[k], o[k], d);
      red[0] = d.re;
      red[1] = d.im;
    } else if constexpr (EPI == EPI_TS) {
      cx<R> d = mk<R>(0, 0);
      R n2 = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        d = fma_cj(o[k], x0[k], d);
        n2 += o[k].re * o[k].re + o[k].im * o[k].im;
      }
      red[0] = d.re;
      red[1] = d.im;
      red[2] = n2;
    }
  }
  if (EPI == EPI_DOT || EPI == EPI_RESID) {
    double v2[2] = {red[0], red[1]};
    grid_reduce<2, APPLY_THREADS>(v2, ep.ra, ep.ticket);
  } else if (EPI == EPI_TS) {
    grid_reduce<3, APPLY_THREADS>(red, ep.ra, ep.ticket);
  }
}

#ifndef OK_APPLY_MINB
#define OK_APPLY_MINB 1
#endif

template <typename R, int EPI>
__global__ void __launch_bounds__(APPLY_THREADS, OK_APPLY_MINB) apply_pair_kernel(const cx<R>* __restrict__ W, const cx<R>* __restrict__ psi,
                                                                   cx<R>* __restrict__ out, Geom g, R c0q, R a_ii, R b_ii,
                                                                   EpiArgs<R> ep) {
  if (ep.halt && *ep.halt) return;
  const int tid = blockIdx.x * APPLY_THREADS + threadIdx.x;
  const int s = tid >> 1;
  Pair pr;
  pr.p = threadIdx.x & 1;
  pr.mask = 3u << (threadIdx.x & 30);
  double red[3] = {0.0, 0.0, 0.0};
  if (s < g.V) {
    int c[4];
    {
      int r = s;
      c[0] = r % g.L[0]; r /= g.L[0];
      c[1] = r % g.L[1]; r /= g.L[1];
      c[2] = r % g.L[2]; c[3] = r / g.L[2];
    }
    H6<R> acc;
    {
      // on-site: p = 0 forms A = Y+ (u - i l), p = 1 forms B = Y- (u + i l); acc = (A + B) + i (A - B)
      // for p = 0 and (A + B) - i (A - B) for p = 1, i.e. acc = (R + Rp) + i (R - Rp) for both.
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
      M3<R> y = wmat(W, s, m0 + 0);
      mv_add(Rm.v[0], y, v.v[0]); mv_sub(Rm.v[1], y, v.v[1]);
      y = wmat(W, s, m0 + 1);
      mv_add(Rm.v[0], y, v.v[1]);
      y = wmat(W, s, m0 + 2);
      mv_add(Rm.v[1], y, v.v[0]);
      H6<R> Rp = partner(Rm, pr.mask);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc.v[q][k] = (Rm.v[q][k] + Rp.v[q][k]) + ti(Rm.v[q][k] - Rp.v[q][k]);
    }
    const GlobalW<R> Wg{W};
    pair_spatial<R, 0>(Wg, psi, c, g, s, pr, acc);
    pair_spatial<R, 1>(Wg, psi, c, g, s, pr, acc);
    pair_spatial<R, 2>(Wg, psi, c, g, s, pr, acc);
    pair_time<R>(Wg, psi, c, g, s, pr, acc);
    pair_two<R, 0>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
    pair_two<R, 1>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
    pair_two<R, 2>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
    pair_diag<R, 0, 1, 0>(Wg, psi, c, g, s, pr, acc);
    pair_diag<R, 0, 2, 1>(Wg, psi, c, g, s, pr, acc);
    pair_diag<R, 1, 2, 2>(Wg, psi, c, g, s, pr, acc);

    // out_u = acc+ + acc- (p = 0 writes it), out_l = acc+ - acc- (p = 1)
    H6<R> ap = partner(acc, pr.mask), o;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) o.v[q][k] = pr.p ? ap.v[q][k] - acc.v[q][k] : acc.v[q][k] + ap.v[q][k];
    if (EPI == EPI_RESID) {
      H6<R> bv;
      load_half<R>(ep.b, s, pr.p, bv);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          o.v[q][k] = bv.v[q][k] - o.v[q][k];
          red[0] += (double)o.v[q][k].re * o.v[q][k].re + (double)o.v[q][k].im * o.v[q][k].im;
          red[1] += (double)bv.v[q][k].re * bv.v[q][k].re + (double)bv.v[q][k].im * bv.v[q][k].im;
        }
    }
    store_half<R>(out, s, pr.p, o);
    if (EPI == EPI_DOT) {
      H6<R> rh;
      load_half<R>(ep.rhat, s, pr.p, rh);
      cx<R> d = mk<R>(0, 0);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) d = fma_cj(rh.v[q][k], o.v[q][k], d);
      red[0] = d.re;
      red[1] = d.im;
    } else if (EPI == EPI_TS) {
      H6<R> x0;
      load_half<R>(psi, s, pr.p, x0);
      cx<R> d = mk<R>(0, 0);
      R n2 = 0;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          d = fma_cj(o.v[q][k], x0.v[q][k], d);
          n2 += o.v[q][k].re * o.v[q][k].re + o.v[q][k].im * o.v[q][k].im;
        }
      red[0] = d.re;
      red[1] = d.im;
      red[2] = n2;
    }
  }
  if (EPI == EPI_DOT || EPI == EPI_RESID) {
    double v2[2] = {red[0], red[1]};
    grid_reduce<2, APPLY_THREADS>(v2, ep.ra, ep.ticket);
  } else if (EPI == EPI_TS) {
    grid_reduce<3, APPLY_THREADS>(red, ep.ra, ep.ticket);
  }
}

// ============================================================================ split kernel
// A block of 128 threads covers 32 sites.  Warps 0-1 (thread pairs as above) do the on-site term
// and the 13 forward hops, warps 2-3 the 13 backward hops of the same sites; the backward half
// hands its partial sums over through shared memory.  Each thread's chain of dependent
// load-then-multiply rounds is half as long as in the pair kernel, so twice as many global loads
// are in flight per resident site.
//
// Staged form (STAGED = true): the forward half reads its own tile's W record from shared memory.
// The record of a 32-site tile is contiguous in the site-blocked layout, so the Tensor Memory
// Accelerator streams it (cp.async.bulk: one thread issues, an mbarrier counts the bytes) in
// NCHUNK chunks, one per group of hops, through OK_STAGES shared-memory slots.  The copy of chunk
// q + OK_STAGES is issued as soon as both forward warps are done with chunk q, across the block's
// tiles, so the DRAM stream of W is kept in flight by the copy engine instead of by registers.
// The backward half gathers the neighbours' matrices with ordinary loads: the block that owns
// that tile streamed them shortly before, so they are L2 hits.
constexpr int SPLIT_THREADS = 128;
constexpr int SPLIT_SITES = 32;
static_assert(SPLIT_SITES == LANES, "a tile is one site block of the W layout");

// 4 resident blocks per SM (128 registers per thread): measured best on 16^3 x 32 for the
// unstaged form (102 us against 119 us with 2 blocks and 117 us with 5).
#ifndef OK_SPLIT_MINB
#define OK_SPLIT_MINB 4
#endif
// Resident blocks for the variants with a fused reduction (they hold a few more live values).
#ifndef OK_SPLIT_MINB_EPI
#define OK_SPLIT_MINB_EPI 4
#endif

#ifndef OK_STAGES
#define OK_STAGES 2
#endif
constexpr int NCHUNK = 7;     // W0 | W+t | W+x | W+y | W+z | W++ii | W++ij, W+-ij
constexpr int CHUNK_MAX = 8;  // matrices in the largest chunk
__device__ __forceinline__ int chunk_first(int c) {
  return c == 0 ? M_Y0P : c == 1 ? M_UT : c == 5 ? M_VII : c == 6 ? M_VIJ : M_WP + 8 * (c - 2);
}
__device__ __forceinline__ int chunk_count(int c) { return c == 0 ? 6 : c == 1 ? 4 : c == 5 ? 3 : c == 6 ? 6 : 8; }
// A staged matrix occupies its own 9 x 32 elements plus 16 bytes: the two threads of a pair read
// matrices 4 apart, which this shift puts in different shared-memory banks.
template <typename WT> constexpr int smat_elems() { return 9 * LANES + 16 / (int)sizeof(cx<WT>); }
template <typename WT> constexpr int slot_elems() { return CHUNK_MAX * smat_elems<WT>(); }
template <typename WT> constexpr size_t staged_smem() { return (size_t)OK_STAGES * slot_elems<WT>() * sizeof(cx<WT>); }

// Bounded waits: a wait that has not completed after about 2^30 SM cycles (half a second) gives
// up, counts itself here and lets the kernel run to its end (the result is then invalid).
__device__ unsigned g_wait_timeouts;
// Failure injection for the bounded waits: extra bytes that block 0 declares for its first chunk
// (which its copies never deliver, so that wait runs out).  0 outside the failure-detection test.
__device__ unsigned g_stage_test_bytes;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits until phase `parity` of `bar` completes or `limit` SM cycles pass; a wait that runs out
// is counted in g_wait_timeouts when `count` is set.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit = 1LL << 30,
                                          bool count = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      if (count) atomicAdd(&g_wait_timeouts, 1u);
      return false;
    }
  }
  return true;
}
// Global -> shared bulk copy completing on `bar` (both addresses 16-byte aligned, bytes % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Named barrier 1 over the 64 forward threads (non-aligned form: lanes may arrive diverged).
__device__ __forceinline__ void fwd_bar_sync() { asm volatile("barrier.sync 1, 64;" ::: "memory"); }

// W source reading the tile's own matrices [m0, m0 + count) from a staged chunk.
template <typename WT> struct StagedW {
  const cx<WT>* slot;
  int m0;
  __device__ __forceinline__ M3<typename WReal<WT>::type> operator()(int site, int m) const {
    const cx<WT>* q = slot + (m - m0) * smat_elems<WT>() + (site & (LANES - 1));
    M3<typename WReal<WT>::type> a;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      if constexpr (std::is_same<WT, __half>::value) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(q + e * LANES));
        a.e[e] = mk<float>(f.x, f.y);
      } else if constexpr (std::is_same<WT, float>::value) {
        const float2 f = *reinterpret_cast<const float2*>(q + e * LANES);
        a.e[e] = mk<float>(f.x, f.y);
      } else {
        const double2 f = *reinterpret_cast<const double2*>(q + e * LANES);
        a.e[e] = mk<double>(f.x, f.y);
      }
    }
    return a;
  }
};

#ifndef OK_TILE_SWIZZLE
#define OK_TILE_SWIZZLE 1
#endif
// First tile of this block; the block then walks every gridDim.x-th tile.  With OK_TILE_SWIZZLE,
// on a grid of G = k S blocks (S multiprocessors) the blocks b, b + S, b + 2S, ..., which a full
// persistent grid places on one SM, take consecutive tiles, so that their neighbour gathers (the
// rows above and below a tile) can share L1.
__device__ __forceinline__ int tile_rank(int sms) {
  const int b = blockIdx.x, G = gridDim.x;
  if (OK_TILE_SWIZZLE && sms > 0 && G % sms == 0) return (b % sms) * (G / sms) + b / sms;
  return b;
}

// Issue the copies of chunk q of this block (tile tile_rank + (q / NCHUNK) gridDim.x) into slot
// q % OK_STAGES.  Called by one thread.
template <typename WT>
__device__ __forceinline__ void issue_chunk(const cx<WT>* __restrict__ W, cx<WT>* stage, unsigned long long* full, int q,
                                            int rank) {
  const int tile = rank + (q / NCHUNK) * gridDim.x;
  const int c = q % NCHUNK, slot = q % OK_STAGES;
  const int m0 = chunk_first(c), n = chunk_count(c);
  constexpr unsigned mbytes = 9 * LANES * sizeof(cx<WT>);
  // The slot was last read through the generic proxy; order those reads before the async writes.
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const unsigned extra = (q == 0 && blockIdx.x == 0) ? g_stage_test_bytes : 0u;
  mbar_expect_tx(&full[slot], n * mbytes + extra);
  for (int j = 0; j < n; ++j)
    bulk_g2s(stage + (size_t)slot * slot_elems<WT>() + (size_t)j * smat_elems<WT>(),
             W + ((size_t)tile * NMAT + m0 + j) * (9 * LANES), mbytes, &full[slot]);
}

template <typename R, int EPI, typename WT, bool STAGED>
__global__ void __launch_bounds__(SPLIT_THREADS, EPI == EPI_NONE ? OK_SPLIT_MINB : OK_SPLIT_MINB_EPI) apply_split_kernel(const cx<WT>* __restrict__ W, const cx<R>* __restrict__ psi,
                                                                                   cx<R>* __restrict__ out, Geom g, R c0q, R a_ii, R b_ii,
                                                                                   EpiArgs<R> ep) {
  if (ep.halt && *ep.halt) return;
  // Persistent: each block walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...  The hand-off buffer
  // is double-buffered by tile parity, so one barrier per tile suffices: the backward half writes
  // buffer k & 1 for tile k only after the barrier of tile k - 1, which the forward half passes
  // only after it has read buffer (k - 2) & 1 = k & 1.
  __shared__ cx<R> xch[2][64][6];
  __shared__ __align__(16) cx<R> xev[EPI == EPI_NONE ? 1 : 2][64][6];
  __shared__ __align__(8) unsigned long long full[STAGED ? OK_STAGES : 1];
  extern __shared__ __align__(128) unsigned char stage_raw[];
  cx<WT>* stage = reinterpret_cast<cx<WT>*>(stage_raw);
  const int half = threadIdx.x >> 6;  // warp-uniform: 0 forward, 1 backward
  const int t = threadIdx.x & 63;
  Pair pr;
  pr.p = t & 1;
  pr.mask = 3u << (threadIdx.x & 30);
  const GlobalW<WT> Wg{W};
  // Per-thread partial sums over this thread's few sites stay in the field's precision (fewer
  // registers); the block and grid reductions that follow are FP64.
  R red[3] = {0, 0, 0};
  const int ntiles = (g.V + SPLIT_SITES - 1) / SPLIT_SITES;
  const int rank = tile_rank(g.sms);
  const int nq = (STAGED && rank < ntiles) ? ((ntiles - 1 - rank) / (int)gridDim.x + 1) * NCHUNK : 0;
  int qc = 0;  // next chunk (forward warps)
  bool staged_ok = true;
  // Failure path: a wait that runs out sets stage_abort; no further chunk is issued, the block
  // finishes without waiting (its results are invalid and the timeout is counted), and thread 0
  // waits once more, briefly, for every chunk it issued but did not see arrive, so that no bulk
  // copy is in flight when the block exits.
  __shared__ int stage_abort;
  int issued = 0, unwaited_from = -1;
  if constexpr (STAGED) {
    if (threadIdx.x == 0) {
      for (int k = 0; k < OK_STAGES; ++k) mbar_init(&full[k], 1);
      mbar_fence_init();
      stage_abort = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (; issued < OK_STAGES && issued < nq; ++issued) issue_chunk<WT>(W, stage, full, issued, rank);
  }
  // Wait for chunk qc; the forward warps then read it through a StagedW.
  auto chunk = [&](int m0) {
    const int slot = qc % OK_STAGES;
    if (staged_ok) {
      staged_ok = mbar_wait(&full[slot], (qc / OK_STAGES) & 1);
      if (!staged_ok) {
        stage_abort = 1;
        unwaited_from = qc;
      }
    }
    return StagedW<WT>{stage + (size_t)slot * slot_elems<WT>(), m0};
  };
  // Both forward warps are done with chunk qc: its slot takes chunk qc + OK_STAGES.
  auto release = [&]() {
    fwd_bar_sync();
    if (threadIdx.x == 0 && qc + OK_STAGES < nq && !stage_abort) {
      issue_chunk<WT>(W, stage, full, qc + OK_STAGES, rank);
      ++issued;
    }
    ++qc;
  };
  int kb = 0;
  for (int tile = rank; tile < ntiles; tile += gridDim.x, kb ^= 1) {
  const int s = tile * SPLIT_SITES + (t >> 1);
  const bool active = s < g.V;
  H6<R> acc;
#pragma unroll
  for (int qq = 0; qq < 2; ++qq)
#pragma unroll
    for (int k = 0; k < 3; ++k) acc.v[qq][k] = mk<R>(0, 0);
  int c[4] = {0, 0, 0, 0};
  if (active) {
    int r = s;
    c[0] = r % g.L[0]; r /= g.L[0];
    c[1] = r % g.L[1]; r /= g.L[1];
    c[2] = r % g.L[2]; c[3] = r / g.L[2];
  }
  if (half == 0) {
    if constexpr (STAGED) {
      // Every forward thread takes part in the waits and barriers, active or not.
      { auto w = chunk(M_Y0P); if (active) pair_onsite<R>(w, psi, s, pr, c0q, acc); release(); }
      { auto w = chunk(M_UT); if (active) pair_time<R, true, false>(w, psi, c, g, s, pr, acc); release(); }
      { auto w = chunk(M_WP + 0); if (active) pair_spatial<R, 0, true, false>(w, psi, c, g, s, pr, acc); release(); }
      { auto w = chunk(M_WP + 8); if (active) pair_spatial<R, 1, true, false>(w, psi, c, g, s, pr, acc); release(); }
      { auto w = chunk(M_WP + 16); if (active) pair_spatial<R, 2, true, false>(w, psi, c, g, s, pr, acc); release(); }
      {
        auto w = chunk(M_VII);
        if (active) {
          pair_two<R, 0, true, false>(w, psi, c, g, s, pr, a_ii, b_ii, acc);
          pair_two<R, 1, true, false>(w, psi, c, g, s, pr, a_ii, b_ii, acc);
          pair_two<R, 2, true, false>(w, psi, c, g, s, pr, a_ii, b_ii, acc);
        }
        release();
      }
      {
        auto w = chunk(M_VIJ);
        if (active) {
          pair_diag<R, 0, 1, 0, true, false>(w, psi, c, g, s, pr, acc);
          pair_diag<R, 0, 2, 1, true, false>(w, psi, c, g, s, pr, acc);
          pair_diag<R, 1, 2, 2, true, false>(w, psi, c, g, s, pr, acc);
        }
        release();
      }
    } else if (active) {
      pair_onsite<R>(Wg, psi, s, pr, c0q, acc);
      pair_spatial<R, 0, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_spatial<R, 1, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_spatial<R, 2, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_time<R, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_two<R, 0, true, false>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_two<R, 1, true, false>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_two<R, 2, true, false>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_diag<R, 0, 1, 0, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_diag<R, 0, 2, 1, true, false>(Wg, psi, c, g, s, pr, acc);
      pair_diag<R, 1, 2, 2, true, false>(Wg, psi, c, g, s, pr, acc);
    }
  } else if (active) {
      // The epilogue's own half-spinor (rhat, b, or the y of <out, y>) is copied into shared memory
      // asynchronously (cp.async, no registers held) while this half works through its hops.
      if constexpr (EPI != EPI_NONE) {
        const cx<R>* src = EPI == EPI_DOT ? ep.rhat : EPI == EPI_RESID ? ep.b : (ep.rhat ? ep.rhat : psi);
        const char* gsrc = reinterpret_cast<const char*>(src + (size_t)s * 12 + 6 * pr.p);
        char* dst = reinterpret_cast<char*>(&xev[kb][t][0]);
#pragma unroll
        for (int k = 0; k < (int)(6 * sizeof(cx<R>)) / 16; ++k)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst + 16 * k)), "l"(gsrc + 16 * k)
                       : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      pair_spatial<R, 0, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_spatial<R, 1, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_spatial<R, 2, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_time<R, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_two<R, 0, false, true>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_two<R, 1, false, true>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_two<R, 2, false, true>(Wg, psi, c, g, s, pr, a_ii, b_ii, acc);
      pair_diag<R, 0, 1, 0, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_diag<R, 0, 2, 1, false, true>(Wg, psi, c, g, s, pr, acc);
      pair_diag<R, 1, 2, 2, false, true>(Wg, psi, c, g, s, pr, acc);
#pragma unroll
      for (int qq = 0; qq < 2; ++qq)
#pragma unroll
        for (int k = 0; k < 3; ++k) xch[kb][t][3 * qq + k] = acc.v[qq][k];
      if constexpr (EPI != EPI_NONE) asm volatile("cp.async.wait_all;" ::: "memory");
  }
  __syncthreads();
  if (half == 0 && active) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc.v[q][k] = acc.v[q][k] + xch[kb][t][3 * q + k];
    // out_u = acc+ + acc- (p = 0 writes it), out_l = acc+ - acc- (p = 1)
    H6<R> ap = partner(acc, pr.mask), o, ev;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        o.v[q][k] = pr.p ? ap.v[q][k] - acc.v[q][k] : acc.v[q][k] + ap.v[q][k];
        if (EPI != EPI_NONE) ev.v[q][k] = xev[kb][t][3 * q + k];
      }
    if (EPI == EPI_RESID) {
      const H6<R>& bv = ev;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          o.v[q][k] = bv.v[q][k] - o.v[q][k];
          red[0] += (double)o.v[q][k].re * o.v[q][k].re + (double)o.v[q][k].im * o.v[q][k].im;
          red[1] += (double)bv.v[q][k].re * bv.v[q][k].re + (double)bv.v[q][k].im * bv.v[q][k].im;
        }
    }
    store_half<R>(out, s, pr.p, o);
    if (EPI == EPI_DOT) {
      const H6<R>& rh = ev;
      cx<R> d = mk<R>(0, 0);
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) d = fma_cj(rh.v[q][k], o.v[q][k], d);
      red[0] += d.re;
      red[1] += d.im;
    } else if (EPI == EPI_TS) {
      const H6<R>& x0 = ev;
      cx<R> d = mk<R>(0, 0);
      R n2 = 0;
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          d = fma_cj(o.v[q][k], x0.v[q][k], d);
          n2 += o.v[q][k].re * o.v[q][k].re + o.v[q][k].im * o.v[q][k].im;
        }
      red[0] += d.re;
      red[1] += d.im;
      red[2] += n2;
    }
  }
  }  // tiles
  if constexpr (STAGED) {
    if (threadIdx.x == 0 && unwaited_from >= 0)
      for (int q = unwaited_from; q < issued; ++q) mbar_wait(&full[q % OK_STAGES], (q / OK_STAGES) & 1, 1LL << 24, false);
  }
  if (EPI == EPI_DOT || EPI == EPI_RESID) {
    double v2[2] = {(double)red[0], (double)red[1]};
    grid_reduce<2, SPLIT_THREADS>(v2, ep.ra, ep.ticket);
  } else if (EPI == EPI_TS) {
    double v3[3] = {(double)red[0], (double)red[1], (double)red[2]};
    grid_reduce<3, SPLIT_THREADS>(v3, ep.ra, ep.ticket);
  }
}

// ---------------------------------------------------------------------------- launchers
// Kernel variant per precision: 0 = one thread per site, 1 = thread pair per site, 2 = split
// (forward and backward halves in different warps).  FP64 is bound by the FP64 pipe, where one
// thread per site does the least arithmetic; FP32 is bound by memory latency, where the split
// kernel keeps the most loads in flight.
#ifndef OK_APPLY64_VARIANT
#define OK_APPLY64_VARIANT 0
#endif
#ifndef OK_APPLY32_VARIANT
#define OK_APPLY32_VARIANT 2
#endif
template <typename R> constexpr int apply_variant() { return sizeof(R) == 8 ? OK_APPLY64_VARIANT : OK_APPLY32_VARIANT; }

// Persistent grid of the split kernel: as many blocks as fit on the device at once (from the
// occupancy calculator for this instantiation and its dynamic shared memory), at most one per tile.
template <typename R, int EPI, typename WT, bool STAGED>
static void launch_split(const cx<WT>* W, const cx<R>* psi, cx<R>* out, const Geom& g, R c0q, R a, R b,
                         const EpiArgs<R>& ep, cudaStream_t st) {
  static int resident = 0;
  const size_t dyn = STAGED ? staged_smem<WT>() : 0;
  auto kern = apply_split_kernel<R, EPI, WT, STAGED>;
  if (resident == 0) {
    // Static plus dynamic shared memory above 48 KB needs the opt-in (the FP32 reducing variants).
    if (dyn > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, SPLIT_THREADS, dyn) != cudaSuccess || nb < 1) nb = 1;
    resident = nb * sm_count();
  }
  const int tiles = grid_for(g.V, SPLIT_SITES);
  Geom gs = g;
  gs.sms = sm_count();
  kern<<<tiles < resident ? tiles : resident, SPLIT_THREADS, dyn, st>>>(W, psi, out, gs, c0q, a, b, ep);
}

// The split kernel streams the forward W through shared memory by TMA when the handle's tuning
// record says so (ok_autotune); the default reads it with ordinary loads, which measured faster
// on 16^3 x 32 (the staging slots take L1 capacity that the neighbour spinors use).
template <typename R, int EPI>
static void launch_variant(const cx<R>* W, const cx<R>* psi, cx<R>* out, const Geom& g, R c0q, R a, R b,
                           const EpiArgs<R>& ep, bool staged, cudaStream_t st) {
  constexpr int v = apply_variant<R>();
  if constexpr (v == 2) {
    if (staged) launch_split<R, EPI, R, true>(W, psi, out, g, c0q, a, b, ep, st);
    else launch_split<R, EPI, R, false>(W, psi, out, g, c0q, a, b, ep, st);
  }
  else if constexpr (v == 1)
    apply_pair_kernel<R, EPI><<<grid_for(2LL * g.V, APPLY_THREADS), APPLY_THREADS, 0, st>>>(W, psi, out, g, c0q, a, b, ep);
  else
    apply_kernel<R, EPI><<<grid_for(g.V, APPLY_THREADS), APPLY_THREADS, 0, st>>>(W, psi, out, g, c0q, a, b, ep);
}

template <typename R>
int launch_apply(const ok_W* Wh, const cx<R>* psi, cx<R>* out, int epi, const EpiArgs<R>& ep, cudaStream_t st) {
  const cx<R>* W = (const cx<R>*)(sizeof(R) == 8 ? Wh->W64 : Wh->W32);
  if (!W) return OK_EINVAL;
  if (epi < EPI_NONE || epi > EPI_RESID) return OK_EINVAL;
  const Geom& g = Wh->g;
  R c0q = (R)Wh->sc.c0q, a = (R)Wh->sc.a_ii, b = (R)Wh->sc.b_ii;
  const bool stg = sizeof(R) == 4 && Wh->tune.staged[0] == 1;
  static const char* n64[4] = {"apply_f64", "apply_f64_dot", "apply_f64_ts", "apply_f64_resid"};
  static const char* n32[4] = {"apply_f32", "apply_f32_dot", "apply_f32_ts", "apply_f32_resid"};
  {
    TraceScope ts(sizeof(R) == 8 ? n64[epi] : n32[epi], st);
    switch (epi) {
      case EPI_NONE: launch_variant<R, EPI_NONE>(W, psi, out, g, c0q, a, b, ep, stg, st); break;
      case EPI_DOT: launch_variant<R, EPI_DOT>(W, psi, out, g, c0q, a, b, ep, stg, st); break;
      case EPI_TS: launch_variant<R, EPI_TS>(W, psi, out, g, c0q, a, b, ep, stg, st); break;
      default: launch_variant<R, EPI_RESID>(W, psi, out, g, c0q, a, b, ep, stg, st); break;
    }
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

// Upper bound of the grid size of any apply variant (sizes the reduction partials).
int apply_blocks_needed(const ok_W* Wh) { return grid_for(Wh->g.V, SPLIT_SITES); }

// FP32 fields and arithmetic with the half-precision copy of W (split kernel, all epilogues).
int launch_apply_w16(const ok_W* Wh, const cx<float>* psi, cx<float>* out, int epi, const EpiArgs<float>& ep, cudaStream_t st) {
  const cx<__half>* W = (const cx<__half>*)Wh->W16;
  if (!W) return OK_EINVAL;
  if (epi < EPI_NONE || epi > EPI_RESID) return OK_EINVAL;
  const Geom& g = Wh->g;
  const float c0q = (float)Wh->sc.c0q, a = (float)Wh->sc.a_ii, b = (float)Wh->sc.b_ii;
  static const char* names[4] = {"apply_w16", "apply_w16_dot", "apply_w16_ts", "apply_w16_resid"};
  {
    TraceScope ts(names[epi], st);
    if (Wh->tune.staged[1] == 1) {
      switch (epi) {
        case EPI_NONE: launch_split<float, EPI_NONE, __half, true>(W, psi, out, g, c0q, a, b, ep, st); break;
        case EPI_DOT: launch_split<float, EPI_DOT, __half, true>(W, psi, out, g, c0q, a, b, ep, st); break;
        case EPI_TS: launch_split<float, EPI_TS, __half, true>(W, psi, out, g, c0q, a, b, ep, st); break;
        default: launch_split<float, EPI_RESID, __half, true>(W, psi, out, g, c0q, a, b, ep, st); break;
      }
    } else {
      switch (epi) {
        case EPI_NONE: launch_split<float, EPI_NONE, __half, false>(W, psi, out, g, c0q, a, b, ep, st); break;
        case EPI_DOT: launch_split<float, EPI_DOT, __half, false>(W, psi, out, g, c0q, a, b, ep, st); break;
        case EPI_TS: launch_split<float, EPI_TS, __half, false>(W, psi, out, g, c0q, a, b, ep, st); break;
        default: launch_split<float, EPI_RESID, __half, false>(W, psi, out, g, c0q, a, b, ep, st); break;
      }
    }
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

// Failure injection for the bounded waits (see g_stage_test_bytes).
int set_stage_test_bytes(unsigned bytes) {
  if (bytes % 16 != 0 || bytes > (1u << 16)) return OK_EINVAL;
  if (cudaMemcpyToSymbol(g_stage_test_bytes, &bytes, sizeof(unsigned)) != cudaSuccess) return OK_ECUDA;
  return OK_SUCCESS;
}

// Bounded waits that gave up since the last reset (see g_wait_timeouts).
int read_wait_timeouts(unsigned* n, bool reset) {
  if (cudaMemcpyFromSymbol(n, g_wait_timeouts, sizeof(unsigned)) != cudaSuccess) return OK_ECUDA;
  if (reset) {
    const unsigned zero = 0;
    if (cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(unsigned)) != cudaSuccess) return OK_ECUDA;
  }
  return OK_SUCCESS;
}

template int launch_apply<double>(const ok_W*, const cx<double>*, cx<double>*, int, const EpiArgs<double>&, cudaStream_t);
template int launch_apply<float>(const ok_W*, const cx<float>*, cx<float>*, int, const EpiArgs<float>&, cudaStream_t);

}  // namespace okgb
