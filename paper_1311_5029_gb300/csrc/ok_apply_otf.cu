// On-the-fly W (the precalculation of Sec. 2.2 undone): M psi in FP32 from the links and clover
// fields, with every W group rebuilt where a hop needs it.
#include "ok_hops.cuh"
#include "ok_wform.cuh"

namespace okgb {
namespace {

// M psi in FP32 without a stored W.  Each group of forward matrices that a hop needs (the on-site
// Y+-, U_t / 2 with the blocks of S4 / 2, the eight (D +- S) / 2 blocks of one spatial direction,
// V_ii, V_ij, X_ij) is rebuilt from the FP32 links and clover fields by the formulas of
// ok_wform.cuh, at x for a forward hop and at the neighbour for a backward one, and then used
// exactly as apply_kernel uses the stored set.  Per site it reads 720 bytes of inputs (links 288,
// clover fields 432; the neighbours' come from L1 and L2) instead of 3096 bytes of FP32 W, and it
// rebuilds every group twice (about 2 x 75 colour matrix products).
struct BlockedInputs {
  const cx<float>* __restrict__ L;    // links [nblk][4][9][32]
  const cx<float>* __restrict__ EB;   // clover fields [nblk][6][9][32]
  __device__ __forceinline__ static M3<float> get(const cx<float>* __restrict__ p, int site, int n, int m) {
    const float2* q = reinterpret_cast<const float2*>(p) + ((size_t)(site >> 5) * n + m) * 9 * LANES + (site & (LANES - 1));
    M3<float> a;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float2 v = __ldg(q + e * LANES);
      a.e[e] = mk(v.x, v.y);
    }
    return a;
  }
  __device__ __forceinline__ M3<float> U(int site, int mu) const { return get(L, site, 4, mu); }
  __device__ __forceinline__ M3<float> F(int site, int k) const { return get(EB, site, 6, k); }
};

// block2 on four given blocks b[0..3] (00, 01, 10, 11).
template <typename R, bool DAG>
__device__ __forceinline__ void block2m(const M3<R>* b, const Half<R>& h, Half<R>& acc) {
  if (DAG) {
    mdv_add(acc.v[0], b[0], h.v[0]);
    mdv_add(acc.v[1], b[1], h.v[0]);
    mdv_add(acc.v[0], b[2], h.v[1]);
    mdv_add(acc.v[1], b[3], h.v[1]);
  } else {
    mv_add(acc.v[0], b[0], h.v[0]);
    mv_add(acc.v[0], b[1], h.v[1]);
    mv_add(acc.v[1], b[2], h.v[0]);
    mv_add(acc.v[1], b[3], h.v[1]);
  }
}

struct OtfArgs {
  BlockedInputs in;
  ok_coeffs cf;
  double u0;
};

// The W groups (inlined at their 14 uses: as non-inlined functions the kernel spilled the groups'
// matrices to local memory and ran 17 % slower, 782 us against 667 us at 16^3 x 32).
__device__ __forceinline__ void build_onsite(const OtfArgs& A, int s, M3<float> (&yp)[3], M3<float> (&ym)[3]) {
  wform::onsite<float>(A.in, s, A.cf, A.u0, yp, ym);
}
__device__ __forceinline__ void build_temporal(const OtfArgs& A, const Geom& g, int s, M3<float>& uh, M3<float> (&t)[3]) {
  wform::temporal<float>(A.in, site_coords(s, g), g, s, A.cf, A.u0, uh, t);
}
__device__ __forceinline__ void build_spatial(const OtfArgs& A, const Geom& g, int s, int i, M3<float> (&q)[8]) {
  wform::spatial<float>(A.in, site_coords(s, g), g, s, i, A.cf, A.u0, q);
}
__device__ __forceinline__ void build_twohop(const OtfArgs& A, const Geom& g, int s, int i, M3<float>& v) {
  v = wform::twohop<float>(A.in, site_coords(s, g), g, s, i);
}
__device__ __forceinline__ void build_diag(const OtfArgs& A, const Geom& g, int s, int i, int j, bool x, M3<float>& v) {
  if (x) wform::diag_x<float>(A.in, site_coords(s, g), g, s, i, j, A.cf, A.u0, v);
  else wform::diag_v<float>(A.in, site_coords(s, g), g, s, i, j, A.cf, A.u0, v);
}

// The hops of hop_spatial, hop_time, hop_two and hop_diag with rebuilt matrices.
template <int I>
__device__ __forceinline__ void otf_spatial(const OtfArgs& A, const cx<float>* __restrict__ psi, const int (&c)[4],
                                            const Geom& g, int s, Half<float>& ap, Half<float>& am) {
  Half<float> hp, hm;
  M3<float> q[8];
  gather_h<float, I == 0, I == 1, I == 2, 0>(psi, c, g, hp, hm);
  build_spatial(A, g, s, I, q);
  block2m<float, false>(q, hp, ap);
  block2m<float, false>(q + 4, hm, am);
  const int n = gather_h<float, -(I == 0), -(I == 1), -(I == 2), 0>(psi, c, g, hp, hm);
  build_spatial(A, g, n, I, q);
  block2m<float, true>(q + 4, hp, ap);
  block2m<float, true>(q, hm, am);
}

__device__ __forceinline__ void otf_time(const OtfArgs& A, const cx<float>* __restrict__ psi, const int (&c)[4],
                                         const Geom& g, int s, Half<float>& ap, Half<float>& am) {
  Half<float> hp, hm, lo, up, w;
  M3<float> U, t[3];
  gather_h<float, 0, 0, 0, 1>(psi, c, g, hp, hm, nullptr, &lo);
  build_temporal(A, g, s, U, t);
  colour2<float, false>(w, U, lo);
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a) { ap.v[q][a] = ap.v[q][a] - w.v[q][a]; am.v[q][a] = am.v[q][a] + w.v[q][a]; }
  mv_add(ap.v[0], t[0], hp.v[0]); mv_sub(ap.v[1], t[0], hp.v[1]);
  mv_sub(am.v[0], t[0], hm.v[0]); mv_add(am.v[1], t[0], hm.v[1]);
  mv_add(ap.v[0], t[1], hp.v[1]); mv_sub(am.v[0], t[1], hm.v[1]);
  mv_add(ap.v[1], t[2], hp.v[0]); mv_sub(am.v[1], t[2], hm.v[0]);
  const int n = gather_h<float, 0, 0, 0, -1>(psi, c, g, hp, hm, &up, nullptr);
  build_temporal(A, g, n, U, t);
  colour2<float, true>(w, U, up);
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a) { ap.v[q][a] = ap.v[q][a] - w.v[q][a]; am.v[q][a] = am.v[q][a] - w.v[q][a]; }
  mdv_sub(ap.v[0], t[0], hp.v[0]); mdv_add(ap.v[1], t[0], hp.v[1]);
  mdv_add(am.v[0], t[0], hm.v[0]); mdv_sub(am.v[1], t[0], hm.v[1]);
  mdv_sub(ap.v[1], t[1], hp.v[0]); mdv_add(am.v[1], t[1], hm.v[0]);
  mdv_sub(ap.v[0], t[2], hp.v[1]); mdv_add(am.v[0], t[2], hm.v[1]);
}

template <int I>
__device__ __forceinline__ void otf_two(const OtfArgs& A, const cx<float>* __restrict__ psi, const int (&c)[4],
                                        const Geom& g, int s, float a, float b, Half<float>& ap,
                                        Half<float>& am) {
  Half<float> hp, hm, y;
  gather_h<float, 2 * (I == 0), 2 * (I == 1), 2 * (I == 2), 0>(psi, c, g, hp, hm);
  M3<float> V;
  build_twohop(A, g, s, I, V);
  colour2<float, false>(y, V, hp);
  add_scaled(ap, a, y); add_sigma(ap, I, y, b);
  colour2<float, false>(y, V, hm);
  add_scaled(am, a, y); add_sigma(am, I, y, -b);
  const int n = gather_h<float, -2 * (I == 0), -2 * (I == 1), -2 * (I == 2), 0>(psi, c, g, hp, hm);
  build_twohop(A, g, n, I, V);
  colour2<float, true>(y, V, hp);
  add_scaled(ap, a, y); add_sigma(ap, I, y, -b);
  colour2<float, true>(y, V, hm);
  add_scaled(am, a, y); add_sigma(am, I, y, b);
}

template <int I, int J>
__device__ __forceinline__ void otf_diag(const OtfArgs& A, const cx<float>* __restrict__ psi, const int (&c)[4],
                                         const Geom& g, int s, Half<float>& ap, Half<float>& am) {
  constexpr int A0 = (I == 0) + (J == 0), A1 = (I == 1) + (J == 1), A2 = (I == 2) + (J == 2);
  constexpr int B0 = (I == 0) - (J == 0), B1 = (I == 1) - (J == 1), B2 = (I == 2) - (J == 2);
  Half<float> hp, hm, y;
  M3<float> V;
  gather_h<float, A0, A1, A2, 0>(psi, c, g, hp, hm);
  build_diag(A, g, s, I, J, false, V);
  colour2<float, false>(y, V, hp); add_sigma(ap, I, y, 1.f); add_sigma(ap, J, y, 1.f);
  colour2<float, false>(y, V, hm); add_sigma(am, I, y, -1.f); add_sigma(am, J, y, -1.f);
  int n = gather_h<float, -A0, -A1, -A2, 0>(psi, c, g, hp, hm);
  build_diag(A, g, n, I, J, false, V);
  colour2<float, true>(y, V, hp); add_sigma(ap, I, y, -1.f); add_sigma(ap, J, y, -1.f);
  colour2<float, true>(y, V, hm); add_sigma(am, I, y, 1.f); add_sigma(am, J, y, 1.f);
  gather_h<float, B0, B1, B2, 0>(psi, c, g, hp, hm);
  build_diag(A, g, s, I, J, true, V);
  colour2<float, false>(y, V, hp); add_sigma(ap, I, y, 1.f); add_sigma(ap, J, y, -1.f);
  colour2<float, false>(y, V, hm); add_sigma(am, I, y, -1.f); add_sigma(am, J, y, 1.f);
  n = gather_h<float, -B0, -B1, -B2, 0>(psi, c, g, hp, hm);
  build_diag(A, g, n, I, J, true, V);
  colour2<float, true>(y, V, hp); add_sigma(ap, I, y, -1.f); add_sigma(ap, J, y, 1.f);
  colour2<float, true>(y, V, hm); add_sigma(am, I, y, 1.f); add_sigma(am, J, y, -1.f);
}

__global__ void __launch_bounds__(APPLY_THREADS) apply_otf_kernel(OtfArgs A, const cx<float>* __restrict__ psi,
                                                                  cx<float>* __restrict__ out, Geom g, float c0q, float a_ii,
                                                                  float b_ii) {
  const int s = blockIdx.x * APPLY_THREADS + threadIdx.x;
  if (s >= g.V) return;
  const Site p = site_coords(s, g);
  int c[4];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) c[mu] = p.c[mu];
  Half<float> ap, am;
  cx<float> x0[12];
  // on-site, as in apply_kernel: a = u - i l, b = u + i l; A = Y+ a, B = Y- b; acc+- = (A + B) +- i (A - B)
  load_spinor<float>(psi, s, x0);
  {
    M3<float> yp[3], ym[3];
    build_onsite(A, s, yp, ym);
    Half<float> a, b, PA, PB;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        a.v[q][k] = x0[3 * q + k] - ti(x0[3 * (q + 2) + k]);
        b.v[q][k] = x0[3 * q + k] + ti(x0[3 * (q + 2) + k]);
        PA.v[q][k] = c0q * a.v[q][k];
        PB.v[q][k] = c0q * b.v[q][k];
      }
    mv_add(PA.v[0], yp[0], a.v[0]); mv_sub(PA.v[1], yp[0], a.v[1]);
    mv_add(PA.v[0], yp[1], a.v[1]);
    mv_add(PA.v[1], yp[2], a.v[0]);
    mv_add(PB.v[0], ym[0], b.v[0]); mv_sub(PB.v[1], ym[0], b.v[1]);
    mv_add(PB.v[0], ym[1], b.v[1]);
    mv_add(PB.v[1], ym[2], b.v[0]);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<float> P = PA.v[q][k] + PB.v[q][k], Q = PA.v[q][k] - PB.v[q][k];
        ap.v[q][k] = P + ti(Q);
        am.v[q][k] = P - ti(Q);
      }
  }
  otf_spatial<0>(A, psi, c, g, s, ap, am);
  otf_spatial<1>(A, psi, c, g, s, ap, am);
  otf_spatial<2>(A, psi, c, g, s, ap, am);
  otf_time(A, psi, c, g, s, ap, am);
  otf_two<0>(A, psi, c, g, s, a_ii, b_ii, ap, am);
  otf_two<1>(A, psi, c, g, s, a_ii, b_ii, ap, am);
  otf_two<2>(A, psi, c, g, s, a_ii, b_ii, ap, am);
  otf_diag<0, 1>(A, psi, c, g, s, ap, am);
  otf_diag<0, 2>(A, psi, c, g, s, ap, am);
  otf_diag<1, 2>(A, psi, c, g, s, ap, am);
  cx<float> o[12];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      o[3 * q + k] = ap.v[q][k] + am.v[q][k];
      o[3 * (q + 2) + k] = ap.v[q][k] - am.v[q][k];
    }
  store_spinor<float>(out, s, o);
}

}  // namespace

int launch_apply_otf(const ok_W* Wh, const cx<float>* psi, cx<float>* out, cudaStream_t st) {
  if (!Wh->L32 || !Wh->EB32) return OK_EINVAL;
  const Geom& g = Wh->g;
  OtfArgs A{BlockedInputs{(const cx<float>*)Wh->L32, (const cx<float>*)Wh->EB32}, Wh->coeffs, Wh->sc.u0};
  {
    TraceScope ts("apply_otf", st);
    apply_otf_kernel<<<grid_for(g.V, APPLY_THREADS), APPLY_THREADS, 0, st>>>(A, psi, out, g, (float)Wh->sc.c0q,
                                                                             (float)Wh->sc.a_ii, (float)Wh->sc.b_ii);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

}  // namespace okgb
