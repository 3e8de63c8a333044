// FP64-accurate M psi on the FP32 pipes: double-float W (OK_W_DF64) and fields, one thread per
// site, the stencil walked as a table.
//
// The operator is the one of the other apply kernels (Eq. minFlopForm in the spin basis where
// every hop except W^0 is block diagonal in h+- = u +- l; see ok_apply.cu): per site 27 offsets
// and 148 colour matrix-vector products y = V h or V^dag h, each added to one or two of the four
// accumulators acc+-(spin 0, 1) with a factor 1, a_ii or b_ii times a unit (+-1, +-i, +-1 +- i).
// Written out with every product inlined, that is about 100 K FP32 instructions of straight-line
// code per thread in double-float arithmetic, far beyond the instruction caches.  Here the
// products are entries of a table in the kernel's parameter space and one compact loop body
// executes them: the offset's neighbour spinor is gathered once into shared memory (three
// half-spinor slots per thread), then every entry loads its matrix, multiplies and accumulates.
// All threads of a block walk the same entries, so the table reads and the branches on an
// entry's fields are uniform.
//
// Double-float: a row of a product sums six real products with TwoProd and TwoSum, deferring the
// renormalisation to the end of the row (Joldes, Muller, Popescu, ACM TOMS 44 (2017), the
// building blocks of ok_internal.cuh); accumulators are renormalised at every addition.
#include "ok_dd.cuh"
#include "ok_dd_table.cuh"

namespace okgb {

namespace {

constexpr int DD_THREADS = 128;
#ifndef OK_DD_MINB
#define OK_DD_MINB 4
#endif

using namespace ddtab;

// ---------------------------------------------------------------------------- double-float pieces
__device__ __forceinline__ cx<dd> ld4(const float4* p) {
  const float4 v = __ldg(p);
  return mk(dd(v.x, v.y), dd(v.z, v.w));
}
// (s, t) = a * b as an unnormalised pair: s the rounded product of the high parts, t the rest.
__device__ __forceinline__ void prod_first(float& s, float& t, dd a, dd b) {
  s = a.hi * b.hi;
  t = fmaf(a.hi, b.hi, -s);
  t = fmaf(a.hi, b.lo, t);
  t = fmaf(a.lo, b.hi, t);
}
// (s, t) += a * b: TwoSum of the high parts, every low-order term into t.
__device__ __forceinline__ void prod_acc(float& s, float& t, dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s2 = s + p;
  const float bb = s2 - s;
  t += (s - (s2 - bb)) + (p - bb);
  t += e;
  s = s2;
}
__device__ __forceinline__ dd dneg(dd a) { return dd(-a.hi, -a.lo); }

__device__ __forceinline__ dd dflip(dd a, unsigned m) {
  return dd(__uint_as_float(__float_as_uint(a.hi) ^ m), __uint_as_float(__float_as_uint(a.lo) ^ m));
}

// y = V v, or V^dag v when adj, for the matrix at wp (element e at wp + e * LANES).  One body for
// both forms: the adjoint reads element (c, r) for (r, c) and flips the sign of its imaginary
// part; a row's three elements are loaded as the row starts.
__device__ __forceinline__ void matvec(const float4* __restrict__ wp, bool adj, const cx<dd> (&v)[3], cx<dd> (&y)[3]) {
  const int sr = adj ? 1 : 3, sc = adj ? 3 : 1;
  const unsigned cj = adj ? 0x80000000u : 0u;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    cx<dd> e[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      e[c] = ld4(wp + (r * sr + c * sc) * LANES);
      e[c].im = dflip(e[c].im, cj);
    }
    float sr_, tr, si, ti_;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // (a.re v.re - a.im v.im) + i (a.re v.im + a.im v.re)
      if (c == 0) {
        prod_first(sr_, tr, e[c].re, v[c].re);
        prod_first(si, ti_, e[c].re, v[c].im);
      } else {
        prod_acc(sr_, tr, e[c].re, v[c].re);
        prod_acc(si, ti_, e[c].re, v[c].im);
      }
      prod_acc(sr_, tr, dneg(e[c].im), v[c].im);
      prod_acc(si, ti_, e[c].im, v[c].re);
    }
    y[r] = mk(dd_renorm(sr_, tr), dd_renorm(si, ti_));
  }
}

// w = unit x y for the units 1, i, -1, -i (codes 0..3: a quarter turn per step, exact) and
// 1 + i, 1 - i, -1 - i, -1 + i (codes 4..7: g (1 + s i), s = -1 for odd codes, g = -1 from 6 on).
__device__ __forceinline__ void times_unit(const cx<dd> (&y)[3], int u, cx<dd> (&w)[3]) {
  if (u < 4) {
    const bool sw = u & 1;
    const unsigned mr = (((u + 1) >> 1) & 1) ? 0x80000000u : 0u, mi = ((u >> 1) & 1) ? 0x80000000u : 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) w[k] = mk(dflip(sw ? y[k].im : y[k].re, mr), dflip(sw ? y[k].re : y[k].im, mi));
  } else {
    const unsigned ms = (u & 1) ? 0x80000000u : 0u, mg = (u & 2) ? 0x80000000u : 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      w[k] = mk(dflip(y[k].re - dflip(y[k].im, ms), mg), dflip(y[k].im + dflip(y[k].re, ms), mg));
  }
}

// Neighbour x + d of the site with coordinates c, with the fermion sign of every wrap across an
// antiperiodic boundary (|d_mu| <= 2, so at most two wraps per direction).
__device__ __forceinline__ int nbr_of(const int (&c)[4], const Geom& g, const DDHop& hop, bool& neg) {
  int n = 0;
  neg = false;
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    int x = c[mu] + hop.d[mu];
    int wraps = 0;
    if (x >= L) { x -= L; wraps = 1; if (x >= L) { x -= L; wraps = 2; } }
    if (x < 0) { x += L; wraps = 1; if (x < 0) { x += L; wraps = 2; } }
    if (((g.bcneg >> mu) & 1) && (wraps & 1)) neg = !neg;
    n += x * g.S[mu];
  }
  return n;
}

// Prefetch into L1 (no registers held): the next entry's matrix, the next offset's spinor.
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }
__device__ __forceinline__ const float4* wmat_dd(const float4* W, int site, int m) {
  return W + ((size_t)(site >> 5) * NMAT + m) * (9 * LANES) + (site & 31);
}
__device__ __forceinline__ void prefetch_mat(const float4* wp) {
#pragma unroll
  for (int e = 0; e < 9; ++e) prefetch_l1(wp + e * LANES);
}

__device__ __forceinline__ void add_to(cx<dd> (&acc)[3], const cx<dd> (&w)[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) acc[k] = mk(acc[k].re + w[k].re, acc[k].im + w[k].im);
}

// ---------------------------------------------------------------------------- the kernel
template <int EPI>
__global__ void __launch_bounds__(DD_THREADS, OK_DD_MINB)
    apply_dd_kernel(const float4* __restrict__ W, const float4* __restrict__ psi, double2* __restrict__ out, Geom g,
                    dd c0q2, dd a_ii, dd b_ii, const double2* __restrict__ rhs, RedArgs ra, unsigned* ticket,
                    const int* halt, const __grid_constant__ DDTable tab) {
  if (EPI != EPI_NONE && halt && *halt) return;
  // Three half-spinor slots per thread, [slot * 6 + spin * 3 + colour][thread]: a thread's
  // accesses to one entry hit consecutive 16-byte words across the warp.
  __shared__ float4 slot[18][DD_THREADS];
  const int tid = threadIdx.x;
  const int s = blockIdx.x * DD_THREADS + tid;
  double red[2] = {0.0, 0.0};
  if (s < g.V) {
    int c[4];
    {
      int r = s;
      c[0] = r % g.L[0]; r /= g.L[0];
      c[1] = r % g.L[1]; r /= g.L[1];
      c[2] = r % g.L[2]; c[3] = r / g.L[2];
    }
    cx<dd> acc0[3], acc1[3], acc2[3], acc3[3];
    bool neg_next;
    int n_next = nbr_of(c, g, tab.hop[0], neg_next);
#pragma unroll 1
    for (int hh = 0; hh < DD_HOPS; ++hh) {
      const DDHop hop = tab.hop[hh];
      const int n = n_next;
      const bool neg = neg_next;
      // the next offset's neighbour: its spinor is prefetched now, its first matrix with this
      // offset's last entry
      if (hh + 1 < DD_HOPS) {
        n_next = nbr_of(c, g, tab.hop[hh + 1], neg_next);
        const float4* pn = psi + (size_t)n_next * 12;
        prefetch_l1(pn);
        prefetch_l1(pn + 8);
        prefetch_l1(pn + 11);
      }
      {
        const float4* pp = psi + (size_t)n * 12;
        cx<dd> v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          v[k] = ld4(pp + k);
          if (neg) v[k] = mk(dneg(v[k].re), dneg(v[k].im));
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const cx<dd> u = v[3 * q + k], l = v[3 * (q + 2) + k];
            cx<dd> h0, h1;
            if (hop.kind == DD_ONSITE) {
              h0 = mk(u.re + l.im, u.im - l.re);  // u - i l
              h1 = mk(u.re - l.im, u.im + l.re);  // u + i l
            } else {
              h0 = mk(u.re + l.re, u.im + l.im);
              h1 = mk(u.re - l.re, u.im - l.im);
            }
            slot[0 * 6 + 3 * q + k][tid] = make_float4(h0.re.hi, h0.re.lo, h0.im.hi, h0.im.lo);
            slot[1 * 6 + 3 * q + k][tid] = make_float4(h1.re.hi, h1.re.lo, h1.im.hi, h1.im.lo);
            if (hop.kind == DD_THIRD_L || hop.kind == DD_THIRD_U) {
              const cx<dd> t3 = hop.kind == DD_THIRD_L ? l : u;
              slot[2 * 6 + 3 * q + k][tid] = make_float4(t3.re.hi, t3.re.lo, t3.im.hi, t3.im.lo);
            }
          }
        if (hop.kind == DD_ONSITE) {
          // the c0q part of W^0: acc+ = 2 c0q (u + l), acc- = 2 c0q (u - l)
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const cx<dd> u0 = v[k], u1 = v[3 + k], l0 = v[6 + k], l1 = v[9 + k];
            acc0[k] = mk(c0q2 * (u0.re + l0.re), c0q2 * (u0.im + l0.im));
            acc1[k] = mk(c0q2 * (u1.re + l1.re), c0q2 * (u1.im + l1.im));
            acc2[k] = mk(c0q2 * (u0.re - l0.re), c0q2 * (u0.im - l0.im));
            acc3[k] = mk(c0q2 * (u1.re - l1.re), c0q2 * (u1.im - l1.im));
          }
        }
      }
      const int a_end = hop.first + hop.count;
#pragma unroll 1
      for (int ai = hop.first; ai < a_end; ++ai) {
        const DDAct A = tab.act[ai];
        const int ws = (A.flags & 1) ? n : s;
        const int src = A.flags >> 2;
        const float4* wp = wmat_dd(W, ws, A.m);
        if (ai + 1 < a_end) {
          const DDAct B = tab.act[ai + 1];
          prefetch_mat(wmat_dd(W, (B.flags & 1) ? n : s, B.m));
        } else if (hh + 1 < DD_HOPS) {
          const DDAct B = tab.act[tab.hop[hh + 1].first];
          prefetch_mat(wmat_dd(W, (B.flags & 1) ? n_next : s, B.m));
        }
        cx<dd> v[3], y[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float4 f = slot[src * 3 + k][tid];
          v[k] = mk(dd(f.x, f.y), dd(f.z, f.w));
        }
        matvec(wp, A.flags & 2, v, y);
        // the one or two accumulators, each with its scalar and unit (a rolled loop: one copy of
        // the code)
#pragma unroll 1
        for (int j = 0; j < 2; ++j) {
          const int d = j ? A.dst[1] : A.dst[0];
          if (d < 0) break;
          const int mul = j ? A.mul[1] : A.mul[0];
          const int sc = mul & 3, un = mul >> 2;
          cx<dd> w[3];
          times_unit(y, un, w);
          if (sc != S1) {
            const dd f = sc == SA ? a_ii : b_ii;
#pragma unroll
            for (int k = 0; k < 3; ++k) w[k] = mk(f * w[k].re, f * w[k].im);
          }
          switch (d) {
            case 0: add_to(acc0, w); break;
            case 1: add_to(acc1, w); break;
            case 2: add_to(acc2, w); break;
            default: add_to(acc3, w); break;
          }
        }
      }
    }
    // out_u = acc+ + acc-, out_l = acc+ - acc-, rounded to FP64
    double2* op = out + (size_t)s * 12;
    const double2* bp = EPI == EPI_RESID ? rhs + (size_t)s * 12 : nullptr;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const cx<dd> p = q == 0 ? acc0[k] : acc1[k];
        const cx<dd> m = q == 0 ? acc2[k] : acc3[k];
        const cx<dd> up = mk(p.re + m.re, p.im + m.im), lo = mk(p.re - m.re, p.im - m.im);
        double2 ou = make_double2((double)up.re, (double)up.im);
        double2 ol = make_double2((double)lo.re, (double)lo.im);
        if (EPI == EPI_RESID) {
          const double2 bu = bp[3 * q + k], bl = bp[3 * (q + 2) + k];
          ou = make_double2(bu.x - ou.x, bu.y - ou.y);
          ol = make_double2(bl.x - ol.x, bl.y - ol.y);
          red[0] += ou.x * ou.x + ou.y * ou.y + ol.x * ol.x + ol.y * ol.y;
          red[1] += bu.x * bu.x + bu.y * bu.y + bl.x * bl.x + bl.y * bl.y;
        }
        op[3 * q + k] = ou;
        op[3 * (q + 2) + k] = ol;
      }
  }
  if (EPI == EPI_RESID) grid_reduce<2, DD_THREADS>(red, ra, ticket);
}

// The table, built once on the host.
const DDTable& dd_table() {
  static const DDTable t = build_table();
  return t;
}

}  // namespace

int launch_apply_dd(const ok_W* Wh, const cx<dd>* psi_df, cx<double>* out, int epi, const EpiArgs<dd>& ep, cudaStream_t st) {
  if (!Wh->Wdf || (epi != EPI_NONE && epi != EPI_RESID)) return OK_EINVAL;
  if (epi == EPI_RESID && !ep.b) return OK_EINVAL;
  const DDTable& tab = dd_table();
  if (tab.hop[0].count == 0) return OK_EINTERNAL;
  const Geom& g = Wh->g;
  const int nb = grid_for(g.V, DD_THREADS);
  const dd c0q2(2.0 * Wh->sc.c0q), a(Wh->sc.a_ii), b(Wh->sc.b_ii);
  const float4* W = reinterpret_cast<const float4*>(Wh->Wdf);
  const float4* psi = reinterpret_cast<const float4*>(psi_df);
  double2* o = reinterpret_cast<double2*>(out);
  const double2* rhs = reinterpret_cast<const double2*>(ep.b);
  {
    TraceScope ts(epi == EPI_RESID ? "apply_df64_resid" : "apply_df64", st);
    if (epi == EPI_RESID)
      apply_dd_kernel<EPI_RESID><<<nb, DD_THREADS, 0, st>>>(W, psi, o, g, c0q2, a, b, rhs, ep.ra, ep.ticket, ep.halt, tab);
    else
      apply_dd_kernel<EPI_NONE><<<nb, DD_THREADS, 0, st>>>(W, psi, o, g, c0q2, a, b, rhs, ep.ra, ep.ticket, ep.halt, tab);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

}  // namespace okgb
