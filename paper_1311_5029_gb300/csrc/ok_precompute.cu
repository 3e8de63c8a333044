// Precalculation of the W matrices (Sec. 2.2 "Precalculation"; Eqs. shifted_W_first ..
// shifted_W_last): mean plaquette and tadpole factor u0, clover fields E_i and B_i, and the
// forward set of W matrices per site in the site-blocked layout of ok_internal.cuh.
//
// Stored representation (NMAT = 43 colour matrices per site, all arithmetic FP64):
//   The apply works in the basis h+- = psi_upper +- psi_lower of the two 2-spin halves, in which
//   every hop except W^0 and W^+-_4 is block diagonal (W^+_i = [[D, S], [S, D]] acts as D + S on
//   h+ and D - S on h-).  So the stored matrices are:
//   * W^0 = u0/(2 kappa) + [[D0, S0], [-S0, D0]]: the 2x2 spin blocks of Y+- = (D0 +- i S0) / 4,
//     which act on u -+ i l; the constant u0/(2 kappa)/4 is added to the diagonal blocks on the
//     fly.  D0 = sum_k sigma_k d_k, S0 = sum_k sigma_k s_k, so each Y is [[y3, y1 - i y2],
//     [y1 + i y2, -y3]]: 3 matrices per sign.                                    (6 matrices)
//   * W^+_4 = [[0, S4], [S4, -U4]]: U4 / 2 and the blocks of S4 / 2.                 (4)
//   * W^+_i: the four 2x2 spin blocks of (D^+_i + S^+_i) / 2 and of (D^+_i - S^+_i) / 2. (24)
//   * W^{++}_ii = [[a V, b sigma_i V], [b sigma_i V, a V]]: V = U_i(x) U_i(x+i).       (3)
//   * W^{++}_ij, W^{+-}_ij = [[0, S], [S, 0]] with S = c2/(2 u0) (sigma_i +- sigma_j) X:
//     the colour part X times c2 / (4 u0).                                             (6)
//   The backward matrices come from these at the neighbouring site by Eqs. conjugate and
//   opp_diag_pre_mat inside the apply.
#include "ok_launch.cuh"
#include "ok_split.cuh"
#include "ok_wform.cuh"
#include <new>

namespace okgb {

template <typename LT>
__device__ __forceinline__ M3<double> load_link(const cx<LT>* __restrict__ U, int site, int mu) {
  M3<double> m;
  const cx<LT>* p = U + ((size_t)site * 4 + mu) * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    cx<LT> v = p[k];
    m.e[k] = mk<double>((double)v.re, (double)v.im);
  }
  return m;
}

__device__ __forceinline__ M3<double> load_eb(const cx<double>* __restrict__ EB, int site, int k) {
  M3<double> m;
  const cx<double>* p = EB + ((size_t)site * 6 + k) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) m.e[e] = p[e];
  return m;
}

// ---------------------------------------------------------------------------- block reduction
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < THREADS / 32; ++i) r += sh[i];
  }
  __syncthreads();
  return r;
}

// The inputs of the W formulas in the precompute: canonical links (FP64 or FP32) and the FP64 clover
// fields of clover_kernel.
template <typename LT>
struct CanonInputs {
  const cx<LT>* __restrict__ links;
  const cx<double>* __restrict__ EB;
  __device__ __forceinline__ M3<double> U(int site, int mu) const { return load_link(links, site, mu); }
  __device__ __forceinline__ M3<double> F(int site, int k) const { return load_eb(EB, site, k); }
};

// The inputs as double-float pairs (converted once per precompute): the W formulas then run on the
// FP32 pipes, which GB300 executes 58 times faster than its FP64 pipe, with errors of about 1e-13
// relative instead of FP64 rounding.
struct DDInputs {
  const cx<dd>* __restrict__ links;  // [V][4][9]
  const cx<dd>* __restrict__ EB;     // [V][6][9]
  __device__ __forceinline__ static M3<dd> get(const cx<dd>* __restrict__ p) {
    M3<dd> m;
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p) + e);
      m.e[e] = mk(dd(v.x, v.y), dd(v.z, v.w));
    }
    return m;
  }
  __device__ __forceinline__ M3<dd> U(int site, int mu) const { return get(links + ((size_t)site * 4 + mu) * 9); }
  __device__ __forceinline__ M3<dd> F(int site, int k) const { return get(EB + ((size_t)site * 6 + k) * 9); }
};

// Complex FP64 or FP32 values -> double-float pairs (hi = RN(d), lo = RN(d - hi)).
template <typename T>
__global__ void to_dd_kernel(const cx<T>* __restrict__ in, cx<dd>* __restrict__ out, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const cx<T> v = in[i];
  out[i] = mk(dd((double)v.re), dd((double)v.im));
}


// ---------------------------------------------------------------------------- K1: clover + plaquette
// F_{mu nu} = (Q - Q^dagger) / 8 with Q the four plaquette leaves around x traversed mu-then-nu;
// E_i = F_{t i}, B_i = eps_ijk F_jk / 2.  The plaquette leaf U_mu(x) U_nu(x+mu) U_mu^dag(x+nu)
// U_nu^dag(x) also feeds the mean plaquette.
constexpr int K1_THREADS = 128;

// One thread per (site, plane): blockIdx.y is the plane (mu, nu), mu < nu, in the order (0,1),
// (0,2), (0,3), (1,2), (1,3), (2,3).  In precision R from the input accessor `in` (U(site, mu)); the
// field is stored in FP64 in its E or B slot, and the plaquette leaf summed in FP64 into the
// partial of block (blockIdx.y, blockIdx.x).
template <typename R, class In>
__device__ __forceinline__ void clover_body(const In& in, const Geom& g, cx<double>* __restrict__ EB,
                                            double* __restrict__ plaq_part) {
  __shared__ double sh[K1_THREADS / 32];
  const int s = blockIdx.x * K1_THREADS + threadIdx.x;
  const int pl = blockIdx.y;
  const int mu = pl < 3 ? 0 : pl < 5 ? 1 : 2;
  const int nu = pl < 3 ? pl + 1 : pl < 5 ? pl - 1 : 3;
  double retr = 0.0;
  if (s < g.V) {
    const Site p = site_coords(s, g);
    const M3<R> Umx = in.U(s, mu), Unx = in.U(s, nu);
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    const M3<R> l1 = m_mul(m_mul(Umx, in.U(nbr_dir(p, g, mu, 1), nu)),
                           m_mul(m_dag(in.U(nbr_dir(p, g, nu, 1), mu)), m_dag(Unx)));
    retr = (double)l1.e[0].re + (double)l1.e[4].re + (double)l1.e[8].re;
    M3<R> Q = l1;
    // leaf 2: U_nu(x) U_mu(x+nu-mu)^dag U_nu(x-mu)^dag U_mu(x-mu)
    Q = m_add(Q, m_mul(m_mul(Unx, m_dag(in.U(nbr_dir(p, g, nu, 1, mu, -1), mu))),
                       m_mul(m_dag(in.U(nbr_dir(p, g, mu, -1), nu)), in.U(nbr_dir(p, g, mu, -1), mu))));
    // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
    Q = m_add(Q, m_mul(m_mul(m_dag(in.U(nbr_dir(p, g, mu, -1), mu)), m_dag(in.U(nbr_dir(p, g, mu, -1, nu, -1), nu))),
                       m_mul(in.U(nbr_dir(p, g, mu, -1, nu, -1), mu), in.U(nbr_dir(p, g, nu, -1), nu))));
    // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag
    Q = m_add(Q, m_mul(m_mul(m_dag(in.U(nbr_dir(p, g, nu, -1), nu)), in.U(nbr_dir(p, g, nu, -1), mu)),
                       m_mul(in.U(nbr_dir(p, g, nu, -1, mu, 1), nu), m_dag(Umx))));
    const M3<R> f = m_rscale((R)0.125, m_sub(Q, m_dag(Q)));
    // F_{mu nu} is E_i = F_{t i} = -F_{i t} (nu = t) or B_k = F_{(k+1)(k+2)} (indices mod 3)
    int slot;
    double sg;
    if (nu == 3) { slot = mu; sg = -1.0; }
    else { const int k = 3 - mu - nu; slot = 3 + k; sg = (nu == (mu + 1) % 3) ? 1.0 : -1.0; }
    cx<double>* out = EB + ((size_t)s * 6 + slot) * 9;
    for (int e = 0; e < 9; ++e) out[e] = mk(sg * (double)f.e[e].re, sg * (double)f.e[e].im);
  }
  double tot = block_sum<K1_THREADS>(retr, sh);
  if (threadIdx.x == 0) plaq_part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}
// FP64, and double-float at 4 blocks per SM (128 registers: 1.38 ms against 1.54 ms at the
// compiler's 168 registers, 16^3 x 32).
template <class In>
__global__ void __launch_bounds__(K1_THREADS) clover_kernel(In in, Geom g, cx<double>* __restrict__ EB,
                                                            double* __restrict__ plaq_part) {
  clover_body<double>(in, g, EB, plaq_part);
}
__global__ void __launch_bounds__(K1_THREADS, 4) clover_kernel_dd(DDInputs in, Geom g, cx<double>* __restrict__ EB,
                                                                  double* __restrict__ plaq_part) {
  clover_body<dd>(in, g, EB, plaq_part);
}

// Sum the per-block plaquette partials in a fixed order; derive u0 and the stored scalars.
__global__ void scalars_kernel(const double* __restrict__ plaq_part, int nparts, Geom g, ok_coeffs c,
                               WScalars* __restrict__ out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += plaq_part[i];
  // fixed-shape tree over the 32 lanes of each warp, then warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += sh[w];
    WScalars s;
    s.plaq = tot / (18.0 * (double)g.V);
    s.u0 = c.u0 > 0.0 ? c.u0 : pow(s.plaq, 0.25);
    s.inv2kappa = c.kappa > 0.0 ? 1.0 / (2.0 * c.kappa) : c.am0 + 1.0 + 3.0 * c.r_s * c.zeta + 18.0 * c.c4;
    s.c0q = 0.25 * s.u0 * s.inv2kappa;
    s.a_ii = c.c4 / (2.0 * s.u0);
    s.b_ii = (c.c1 + 2.0 * c.c2) / (4.0 * s.u0);
    *out = s;
  }
}

// ---------------------------------------------------------------------------- K2: W matrices
struct WOut {
  cx<double>* W64;
  cx<float>* W32;
  cx<dd>* Wdf;
  cx<__half>* W16;
};

__device__ __forceinline__ void store_mat(const WOut& o, int site, int m, const M3<double>& a) {
  size_t blk = (size_t)(site >> 5);
  int lane = site & 31;
  size_t base = (blk * NMAT + m) * 9 * LANES + lane;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    if (o.W64) o.W64[base + (size_t)e * LANES] = a.e[e];
    if (o.W32) o.W32[base + (size_t)e * LANES] = mk<float>((float)a.e[e].re, (float)a.e[e].im);
    if (o.Wdf) o.Wdf[base + (size_t)e * LANES] = mk<dd>(split_df(a.e[e].re), split_df(a.e[e].im));
    if (o.W16) o.W16[base + (size_t)e * LANES] = mk<__half>(__float2half_rn((float)a.e[e].re), __float2half_rn((float)a.e[e].im));
  }
}

// The same stores from a double-float result (the FP32-pipe precompute, used when no native FP64
// copy is kept): the double-float copy takes the pairs as they are, the FP32 and FP16 copies the
// rounded high parts.
__device__ __forceinline__ void store_mat(const WOut& o, int site, int m, const M3<dd>& a) {
  size_t blk = (size_t)(site >> 5);
  int lane = site & 31;
  size_t base = (blk * NMAT + m) * 9 * LANES + lane;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    if (o.Wdf) o.Wdf[base + (size_t)e * LANES] = a.e[e];
    const float re = a.e[e].re.hi + a.e[e].re.lo, im = a.e[e].im.hi + a.e[e].im.lo;
    if (o.W32) o.W32[base + (size_t)e * LANES] = mk<float>(re, im);
    if (o.W16) o.W16[base + (size_t)e * LANES] = mk<__half>(__float2half_rn(re), __float2half_rn(im));
  }
}

constexpr int K2_THREADS = 64;


// part 0: W^0 and W^+_4; parts 1..3: W^+_i for i = part - 1; part 4: W^{++}_ii, W^{++}_ij, W^{+-}_ij
// (the formulas of ok_wform.cuh, in precision R: FP64 from CanonInputs, double-float from DDInputs).
template <typename R, class In>
__device__ __forceinline__ void w_body(const In& in, const Geom& g, const ok_coeffs& c, const WScalars* __restrict__ scp,
                                       const WOut& o, int part) {
  int s = blockIdx.x * K2_THREADS + threadIdx.x;
  if (s >= g.V) return;
  const double u0 = scp->u0;
  const Site p = site_coords(s, g);
  if (part == 0) {
    M3<R> yp[3], ym[3], t[3], uh;
    wform::onsite<R>(in, s, c, u0, yp, ym);
    for (int j = 0; j < 3; ++j) {
      store_mat(o, s, M_Y0P + j, yp[j]);
      store_mat(o, s, M_Y0M + j, ym[j]);
    }
    wform::temporal<R>(in, p, g, s, c, u0, uh, t);
    store_mat(o, s, M_UT, uh);
    for (int j = 0; j < 3; ++j) store_mat(o, s, M_ST + j, t[j]);
    return;
  }
  if (part >= 1 && part <= 3) {
    const int i = part - 1;
    wform::spatial_to<R>(in, p, g, s, i, c, u0, [&](int k, const M3<R>& m) { store_mat(o, s, M_WP + 8 * i + k, m); });
    return;
  }
  // part 4: two-hop colour matrices
  for (int i = 0; i < 3; ++i) store_mat(o, s, M_VII + i, wform::twohop<R>(in, p, g, s, i));
  int pr = 0;
  for (int i = 0; i < 3; ++i) {
    for (int j = i + 1; j < 3; ++j, ++pr) {
      M3<R> v, x;
      wform::diag_v<R>(in, p, g, s, i, j, c, u0, v);
      wform::diag_x<R>(in, p, g, s, i, j, c, u0, x);
      store_mat(o, s, M_VIJ + pr, v);
      store_mat(o, s, M_XIJ + pr, x);
    }
  }
}
// FP64, and double-float at 8 blocks per SM (128 registers: 2.14 ms against 2.46 ms per step at
// the compiler's 168 registers, 16^3 x 32).
template <class In>
__global__ void __launch_bounds__(K2_THREADS) w_kernel(In in, Geom g, ok_coeffs c, const WScalars* __restrict__ scp,
                                                       WOut o, int part) {
  w_body<double>(in, g, c, scp, o, part);
}
__global__ void __launch_bounds__(K2_THREADS, 8) w_kernel_dd(DDInputs in, Geom g, ok_coeffs c,
                                                             const WScalars* __restrict__ scp, WOut o, int part) {
  w_body<dd>(in, g, c, scp, o, part);
}

// ---------------------------------------------------------------------------- expand (inspection)
template <typename R>
__device__ __forceinline__ M3<double> fetch(const cx<R>* __restrict__ W, int site, int m) {
  size_t blk = (size_t)(site >> 5);
  int lane = site & 31;
  size_t base = (blk * NMAT + m) * 9 * LANES + lane;
  M3<double> a;
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    cx<R> v = W[base + (size_t)e * LANES];
    a.e[e] = mk<double>((double)v.re, (double)v.im);
  }
  return a;
}

// out[(3 * (2 * tr + sr) + cr) * 12 + 3 * (2 * tc + sc) + cc] for spin block (tr, tc) and
// inner 2x2 spin entry (sr, sc).
__device__ __forceinline__ void put(cx<double>* o, int tr, int tc, int sr, int sc, const M3<double>& a, cx<double> f) {
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      cx<double>& d = o[(3 * (2 * tr + sr) + r) * 12 + 3 * (2 * tc + sc) + q];
      d = d + f * a.e[3 * r + q];
    }
}

// Add the 6x6 matrix sum_{sr,sc} blk[sr][sc] (x) colour into spin block (tr, tc) times f.
__device__ __forceinline__ void put6(cx<double>* o, int tr, int tc, const M3<double> b[4], cx<double> f) {
  put(o, tr, tc, 0, 0, b[0], f);
  put(o, tr, tc, 0, 1, b[1], f);
  put(o, tr, tc, 1, 0, b[2], f);
  put(o, tr, tc, 1, 1, b[3], f);
}

// 2x2 Pauli matrix entries sigma_k[r][c] as complex.
__device__ __forceinline__ cx<double> pauli(int k, int r, int c) {
  if (k == 0) return mk<double>(r != c ? 1.0 : 0.0, 0.0);
  if (k == 1) return r == c ? mk<double>(0.0, 0.0) : mk<double>(0.0, r == 0 ? -1.0 : 1.0);
  return r != c ? mk<double>(0.0, 0.0) : mk<double>(r == 0 ? 1.0 : -1.0, 0.0);
}

template <typename R>
__global__ void expand_kernel(const cx<R>* __restrict__ W, Geom g, const WScalars* __restrict__ scp, int kind,
                              cx<double>* __restrict__ out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const WScalars sc = *scp;
  cx<double>* o = out + (size_t)s * 144;
  for (int k = 0; k < 144; ++k) o[k] = mk<double>(0.0, 0.0);
  const cx<double> one = mk<double>(1.0, 0.0);
  const cx<double> I = mk<double>(0.0, 1.0);
  if (kind == 0) {
    M3<double> yp[4], ym[4];
    M3<double> c0 = m_rscale(sc.c0q, m_eye<double>());
    M3<double> a0 = fetch(W, s, M_Y0P), a1 = fetch(W, s, M_Y0P + 1), a2 = fetch(W, s, M_Y0P + 2);
    yp[0] = m_add(a0, c0); yp[1] = a1; yp[2] = a2; yp[3] = m_sub(c0, a0);
    M3<double> b0 = fetch(W, s, M_Y0M), b1 = fetch(W, s, M_Y0M + 1), b2 = fetch(W, s, M_Y0M + 2);
    ym[0] = m_add(b0, c0); ym[1] = b1; ym[2] = b2; ym[3] = m_sub(c0, b0);
    // W0 = [[D', S], [-S, D']] with D' = 2 (Y+ + Y-), S = -2 i (Y+ - Y-)
    const cx<double> two = mk<double>(2.0, 0.0), m2i = mk<double>(0.0, -2.0), p2i = mk<double>(0.0, 2.0);
    for (int tt = 0; tt < 2; ++tt) {
      put6(o, tt, tt, yp, two);
      put6(o, tt, tt, ym, two);
    }
    put6(o, 0, 1, yp, m2i); put6(o, 0, 1, ym, p2i);
    put6(o, 1, 0, yp, p2i); put6(o, 1, 0, ym, m2i);
    return;
  }
  if (kind >= 1 && kind <= 3) {
    int i = kind - 1;
    M3<double> pp[4], pm[4];
    for (int k = 0; k < 4; ++k) { pp[k] = fetch(W, s, M_WP + 8 * i + k); pm[k] = fetch(W, s, M_WP + 8 * i + 4 + k); }
    // D = P+ + P-, S = P+ - P- (stored halves)
    const cx<double> mone = mk<double>(-1.0, 0.0);
    for (int tr = 0; tr < 2; ++tr)
      for (int tc = 0; tc < 2; ++tc) {
        put6(o, tr, tc, pp, one);
        put6(o, tr, tc, pm, tr == tc ? one : mone);
      }
    return;
  }
  if (kind == 4) {
    M3<double> Uh = fetch(W, s, M_UT);
    M3<double> t0 = fetch(W, s, M_ST), t1 = fetch(W, s, M_ST + 1), t2 = fetch(W, s, M_ST + 2);
    M3<double> S[4] = {t0, t1, t2, m_rscale(-1.0, t0)};
    const cx<double> two = mk<double>(2.0, 0.0);
    put6(o, 0, 1, S, two);
    put6(o, 1, 0, S, two);
    put(o, 1, 1, 0, 0, Uh, mk<double>(-2.0, 0.0));
    put(o, 1, 1, 1, 1, Uh, mk<double>(-2.0, 0.0));
    return;
  }
  if (kind >= 5 && kind <= 7) {
    int i = kind - 5;
    M3<double> V = fetch(W, s, M_VII + i);
    for (int tr = 0; tr < 2; ++tr)
      for (int tc = 0; tc < 2; ++tc)
        for (int sr = 0; sr < 2; ++sr)
          for (int scc = 0; scc < 2; ++scc) {
            // [[D, S], [S, D]], D = 2 a (1 (x) V), S = 2 b (sigma_i (x) V)
            cx<double> f = mk<double>(0.0, 0.0);
            if (tr == tc && sr == scc) f = mk<double>(2.0 * sc.a_ii, 0.0);
            if (tr != tc) f = (2.0 * sc.b_ii) * pauli(i, sr, scc);
            if (f.re != 0.0 || f.im != 0.0) put(o, tr, tc, sr, scc, V, f);
          }
    return;
  }
  if (kind >= 8 && kind <= 13) {
    int pr = (kind - 8) % 3;
    int i = pr == 2 ? 1 : 0;
    int j = pr == 0 ? 1 : 2;
    bool plus = kind <= 10;
    M3<double> X = fetch(W, s, (plus ? M_VIJ : M_XIJ) + pr);
    for (int sr = 0; sr < 2; ++sr)
      for (int scc = 0; scc < 2; ++scc) {
        cx<double> f = pauli(i, sr, scc) + (plus ? one : mk<double>(-1.0, 0.0)) * pauli(j, sr, scc);
        f = 2.0 * f;
        if (f.re != 0.0 || f.im != 0.0) {
          put(o, 0, 1, sr, scc, X, f);
          put(o, 1, 0, sr, scc, X, f);
        }
      }
    return;
  }
  (void)I;
}

// ---------------------------------------------------------------------------- host side
static int check_lattice(const ok_lattice* lat, Geom* g) {
  if (!lat) return OK_EINVAL;
  long long V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (lat->dims[mu] < 1 || lat->dims[mu] > OK_MAX_SITES) return OK_EINVAL;
    if (lat->bc[mu] != 1 && lat->bc[mu] != -1) return OK_EINVAL;
    V *= lat->dims[mu];
    if (V > OK_MAX_SITES) return OK_EINVAL;
  }
  g->bcneg = 0;
  for (int mu = 0; mu < 4; ++mu) {
    g->L[mu] = lat->dims[mu];
    if (lat->bc[mu] == -1) g->bcneg |= 1 << mu;
  }
  g->V = (int)V;
  g->nblk = (int)((V + LANES - 1) / LANES);
  g->sms = 0;
  g->S[0] = 1;
  for (int mu = 1; mu < 4; ++mu) g->S[mu] = g->S[mu - 1] * g->L[mu - 1];
  return OK_SUCCESS;
}

int geom_from_lattice(const ok_lattice* lat, Geom* g) { return check_lattice(lat, g); }

template <typename LT>
static int run_precompute(ok_W* W, const void* links, const ok_coeffs* c, cudaStream_t st,
                          cx<double>* EB, double* part, WScalars* dsc, cx<double>* W64tmp) {
  const Geom& g = W->g;
  const cx<LT>* U = (const cx<LT>*)links;
  int nb1 = grid_for(g.V, K1_THREADS);
  int nb2 = grid_for(g.V, K2_THREADS);
  WOut o{W->W64 ? (cx<double>*)W->W64 : W64tmp, (cx<float>*)W->W32, (cx<dd>*)W->Wdf, (cx<__half>*)W->W16};
  const bool any_w = o.W64 || o.W32 || o.Wdf || o.W16;  // (a handle for the on-the-fly apply stores none)
  // A native FP64 copy (kept, or read by the tensor-core build) is computed in FP64; otherwise the
  // clover fields and W are computed in double-float on the FP32 pipes, from double-float copies of
  // the links and fields.
  const bool fp64 = o.W64 != nullptr;
  cx<dd>* ldd = nullptr;
  cx<dd>* ebdd = nullptr;
  auto release = [&]() {
    if (ldd) cudaFreeAsync(ldd, st);
    if (ebdd) cudaFreeAsync(ebdd, st);
  };
  if (!fp64 && any_w) {
    cudaError_t e = cudaMallocAsync((void**)&ldd, (size_t)g.V * 36 * sizeof(cx<dd>), st);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&ebdd, (size_t)g.V * 54 * sizeof(cx<dd>), st);
    if (e != cudaSuccess) {
      release();
      set_cuda_error(e);
      return OK_ENOMEM;
    }
  }
  {
    TraceScope ts("clover", st);
    // with the W formulas in double-float, the clover fields too (1.48 ms against 2.06 ms in FP64 at
    // 16^3 x 32); the plaquette of either is summed in FP64
    if (ldd) {
      to_dd_kernel<LT><<<grid_for(36LL * g.V, 256), 256, 0, st>>>(U, ldd, 36LL * g.V);
      count_launch();
      clover_kernel_dd<<<dim3(nb1, 6), K1_THREADS, 0, st>>>(DDInputs{ldd, nullptr}, g, EB, part);
    } else {
      clover_kernel<<<dim3(nb1, 6), K1_THREADS, 0, st>>>(CanonInputs<LT>{U, EB}, g, EB, part);
    }
  }
  count_launch();
  {
    TraceScope ts("plaquette_u0", st);
    scalars_kernel<<<1, 256, 0, st>>>(part, 6 * nb1, g, *c, dsc);
  }
  count_launch();
  if (any_w) {
    TraceScope ts("w_build", st);
    if (fp64) {
      const CanonInputs<LT> in{U, EB};
      for (int part_id = 0; part_id < 5; ++part_id) {
        w_kernel<<<nb2, K2_THREADS, 0, st>>>(in, g, *c, dsc, o, part_id);
        count_launch();
      }
    } else {
      to_dd_kernel<double><<<grid_for(54LL * g.V, 256), 256, 0, st>>>(EB, ebdd, 54LL * g.V);
      count_launch();
      const DDInputs in{ldd, ebdd};
      for (int part_id = 0; part_id < 5; ++part_id) {
        w_kernel_dd<<<nb2, K2_THREADS, 0, st>>>(in, g, *c, dsc, o, part_id);
        count_launch();
      }
    }
  }
  const cudaError_t e = cudaGetLastError();
  release();
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return OK_ECUDA;
  }
  return OK_SUCCESS;
}

// Clover fields (FP64, [V][6][9]) -> the FP32 copy of an OK_W_OTF handle, site-blocked like W:
// element e of field k (E_0..2, B_0..2) of the site in lane l of block blk at ((blk * 6 + k) * 9 + e) * 32 + l.
__global__ void eb_blocked_kernel(const cx<double>* __restrict__ in, cx<float>* __restrict__ out, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // (site, k, e) in input order
  if (i >= 54LL * V) return;
  const int site = (int)(i / 54), r = (int)(i % 54);
  const int k = r / 9, e = r % 9;
  const cx<double> u = in[i];
  out[(((size_t)(site >> 5) * 6 + k) * 9 + e) * LANES + (site & 31)] = mk<float>((float)u.re, (float)u.im);
}

// Links -> the FP32 copy kept in the handle (OK_W_LINKS), in the site-blocked layout of W:
// element e of U_mu at the site in lane l of block blk is at ((blk * 4 + mu) * 9 + e) * 32 + l,
// so a warp over 32 consecutive sites reads each element as one 256-byte row.
template <typename T>
__global__ void links_blocked_kernel(const cx<T>* __restrict__ in, cx<float>* __restrict__ out, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // (site, mu, e) in input order
  if (i >= 36LL * V) return;
  const int site = (int)(i / 36), r = (int)(i % 36);
  const int mu = r / 9, e = r % 9;
  const cx<T> u = in[i];
  out[(((size_t)(site >> 5) * 4 + mu) * 9 + e) * LANES + (site & 31)] = mk<float>((float)u.re, (float)u.im);
}

// The handle's arrays come from the device's default stream-ordered memory pool.  Let the pool
// keep up to 8 GiB of freed memory (instead of returning it at every synchronisation), so that a
// caller that builds and frees a handle per gauge field does not pay for mapping it each time.
// Raised once per device, and only if the pool is at its default of 0.
static void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static bool done[64] = {};
  if (dev < 0 || dev >= 64 || done[dev]) return;
  done[dev] = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  unsigned long long thr = 0;
  if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess || thr != 0) return;
  thr = 8ULL << 30;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
}

int precompute(const ok_lattice* lat, const void* links, ok_prec links_prec, const ok_coeffs* c,
               int precs, cudaStream_t st, ok_W** W_out) {
  if (!lat || !links || !c || !W_out) return OK_EINVAL;
  if (links_prec != OK_F64 && links_prec != OK_F32) return OK_EINVAL;
  if ((precs & (OK_W_F64 | OK_W_F32 | OK_W_DF64 | OK_W_F16 | OK_W_F16_TC | OK_W_OTF)) == 0 ||
      (precs & ~(OK_W_F64 | OK_W_F32 | OK_W_DF64 | OK_W_F16 | OK_W_LINKS | OK_W_F16_TC | OK_W_OTF)))
    return OK_EINVAL;
  if (!(c->u0 > 0.0) && c->u0 > 0.0) return OK_EINVAL;
  *W_out = nullptr;
  Geom g;
  if (check_lattice(lat, &g) != OK_SUCCESS) return OK_EINVAL;
  ok_W* W = new (std::nothrow) ok_W();
  if (!W) return OK_ENOMEM;
  W->g = g;
  W->lat = *lat;
  W->precs = precs;
  W->coeffs = *c;
  OK_CUDA_TRY(cudaGetDevice(&W->device));
  size_t elems = (size_t)g.nblk * SITE_ELEMS * LANES;
  // Stream-ordered allocations (cheap when the pool already holds the memory, e.g. one handle per
  // step); only the last site block, whose lanes past V are never written, is cleared.
  const size_t tail = (size_t)(g.nblk - 1) * SITE_ELEMS * LANES;
  keep_pool_memory();
  int rc = OK_SUCCESS;
  cx<double>* EB = nullptr;
  double* part = nullptr;
  WScalars* dsc = nullptr;
  void* W64tmp = nullptr;  // FP64 matrices for the tensor-core copy when OK_W_F64 is not kept
  auto fail = [&](int code) {
    for (void* q : {(void*)EB, (void*)part, (void*)dsc, W64tmp, W->W64, W->W32, W->Wdf, W->W16, W->L32, W->Wtc, W->EB32})
      if (q) cudaFreeAsync(q, st);
    delete W;
    return code;
  };
  cudaError_t e;
  if (precs & OK_W_F64) {
    e = cudaMallocAsync(&W->W64, elems * sizeof(cx<double>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(static_cast<cx<double>*>(W->W64) + tail, 0, (elems - tail) * sizeof(cx<double>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (precs & OK_W_F32) {
    e = cudaMallocAsync(&W->W32, elems * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(static_cast<cx<float>*>(W->W32) + tail, 0, (elems - tail) * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (precs & OK_W_DF64) {
    e = cudaMallocAsync(&W->Wdf, elems * sizeof(cx<dd>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(static_cast<cx<dd>*>(W->Wdf) + tail, 0, (elems - tail) * sizeof(cx<dd>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (precs & OK_W_F16) {
    e = cudaMallocAsync(&W->W16, elems * sizeof(cx<__half>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(static_cast<cx<__half>*>(W->W16) + tail, 0, (elems - tail) * sizeof(cx<__half>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (precs & OK_W_F16_TC) {
    e = cudaMallocAsync(&W->Wtc, (size_t)g.V * tc_record_bytes(), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    if (!(precs & OK_W_F64)) {
      e = cudaMallocAsync(&W64tmp, elems * sizeof(cx<double>), st);
      if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    }
  }
  const size_t nlink = (size_t)g.nblk * LANES * 4 * 9;  // blocked: whole 32-site blocks
  const size_t neb = (size_t)g.nblk * LANES * 6 * 9;  // clover fields, blocked
  if (precs & OK_W_OTF) {
    e = cudaMallocAsync(&W->EB32, neb * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(W->EB32, 0, neb * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (precs & (OK_W_LINKS | OK_W_OTF)) {
    e = cudaMallocAsync(&W->L32, nlink * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
    e = cudaMemsetAsync(W->L32, 0, nlink * sizeof(cx<float>), st);
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
    const int nbl = grid_for(36LL * g.V, 256);
    if (links_prec == OK_F32)
      links_blocked_kernel<float><<<nbl, 256, 0, st>>>((const cx<float>*)links, (cx<float>*)W->L32, g.V);
    else
      links_blocked_kernel<double><<<nbl, 256, 0, st>>>((const cx<double>*)links, (cx<float>*)W->L32, g.V);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  W->bytes = (W->W64 ? elems * sizeof(cx<double>) : 0) + (W->W32 ? elems * sizeof(cx<float>) : 0) +
             (W->Wdf ? elems * sizeof(cx<dd>) : 0) + (W->W16 ? elems * sizeof(cx<__half>) : 0) +
             (W->L32 ? nlink * sizeof(cx<float>) : 0) + (W->Wtc ? (size_t)g.V * tc_record_bytes() : 0) +
             (W->EB32 ? neb * sizeof(cx<float>) : 0);
  int nb1 = grid_for(g.V, K1_THREADS);
  e = cudaMallocAsync((void**)&EB, (size_t)g.V * 6 * 9 * sizeof(cx<double>), st);
  if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
  e = cudaMallocAsync((void**)&part, (size_t)6 * nb1 * sizeof(double), st);
  if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
  e = cudaMallocAsync((void**)&dsc, sizeof(WScalars), st);
  if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ENOMEM); }
  rc = links_prec == OK_F64 ? run_precompute<double>(W, links, c, st, EB, part, dsc, (cx<double>*)W64tmp)
                            : run_precompute<float>(W, links, c, st, EB, part, dsc, (cx<double>*)W64tmp);
  if (rc != OK_SUCCESS) return fail(rc);
  if (W->EB32) {
    eb_blocked_kernel<<<grid_for(54LL * g.V, 256), 256, 0, st>>>(EB, (cx<float>*)W->EB32, g.V);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  }
  if (W->Wtc) {
    rc = launch_tc_build(W, W->W64 ? (const cx<double>*)W->W64 : (const cx<double>*)W64tmp, dsc, st);
    if (rc != OK_SUCCESS) return fail(rc);
  }
  e = cudaMemcpyAsync(&W->sc, dsc, sizeof(WScalars), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { set_cuda_error(e); return fail(OK_ECUDA); }
  cudaFreeAsync(EB, st);
  cudaFreeAsync(part, st);
  cudaFreeAsync(dsc, st);
  if (W64tmp) cudaFreeAsync(W64tmp, st);
  EB = nullptr; part = nullptr; dsc = nullptr; W64tmp = nullptr;
  *W_out = W;
  return OK_SUCCESS;
}

int expand(const ok_W* W, ok_prec prec, int kind, void* out, cudaStream_t st) {
  if (!W || !out || kind < 0 || kind > 13) return OK_EINVAL;
  if (prec == OK_F16_TC) return launch_tc_expand(W, kind, (cx<double>*)out, st);
  const void* src = prec == OK_F64 ? (W->W64 ? W->W64 : W->Wdf) : prec == OK_F32 ? W->W32 : prec == OK_F32_W16 ? W->W16 : nullptr;
  if (!src) return OK_EINVAL;
  WScalars* dsc = nullptr;
  OK_CUDA_TRY(cudaMallocAsync((void**)&dsc, sizeof(WScalars), st));
  cudaError_t e = cudaMemcpyAsync(dsc, &W->sc, sizeof(WScalars), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { cudaFreeAsync(dsc, st); set_cuda_error(e); return OK_ECUDA; }
  int nb = grid_for(W->g.V, 64);
  TraceScope ts("expand", st);
  if (prec == OK_F64 && !W->W64)
    expand_kernel<dd><<<nb, 64, 0, st>>>((const cx<dd>*)src, W->g, dsc, kind, (cx<double>*)out);
  else if (prec == OK_F64)
    expand_kernel<double><<<nb, 64, 0, st>>>((const cx<double>*)src, W->g, dsc, kind, (cx<double>*)out);
  else if (prec == OK_F32_W16)
    expand_kernel<__half><<<nb, 64, 0, st>>>((const cx<__half>*)src, W->g, dsc, kind, (cx<double>*)out);
  else
    expand_kernel<float><<<nb, 64, 0, st>>>((const cx<float>*)src, W->g, dsc, kind, (cx<double>*)out);
  count_launch();
  e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(dsc, st);
  if (e != cudaSuccess || e2 != cudaSuccess) { set_cuda_error(e != cudaSuccess ? e : e2); return OK_ECUDA; }
  return OK_SUCCESS;
}

}  // namespace okgb
