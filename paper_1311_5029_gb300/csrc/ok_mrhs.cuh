// Multi-right-hand-side application (kernel templates): out_r = M psi_r for nrhs spinor fields in one launch
// (the 12 spin-colour sources of a propagator).  The split-kernel organisation of the single
// right-hand side apply is kept (a block covers a 32-site tile, warps 0-1 do the on-site term and
// the forward hops, warps 2-3 the backward hops, two threads per site split by spin projection),
// and every thread carries NR right-hand sides: each W colour matrix it loads is applied to NR
// half-spinors, so the W stream is read once per NR fields and the FP32 pipe does the rest.  The
// blocks of grid row y handle right-hand sides y NR .. y NR + NR - 1; the rows sweep the lattice
// together, so the W record of a tile is fetched from DRAM once per application and served from
// L2 to the other rows.
//
// Fused epilogues (EPI_DOT, EPI_TS) reduce per right-hand side into that right-hand side's solver
// state; right-hand sides whose state has halted are skipped, so converged systems cost no
// reductions and keep their state.
#pragma once

#include "ok_pair.cuh"

namespace okgb {

namespace mrhs {

constexpr int MR_THREADS = 128;
constexpr int MR_SITES = 32;

template <int NR> constexpr int mr_minb() { return NR <= 2 ? 4 : 2; }

// h' = sg h (sg = +1 for p = 0, -1 for p = 1), l' = sg l and u of the neighbour at offset D.
template <typename R, int D0, int D1, int D2, int D3>
__device__ __forceinline__ int gather_signed(const cx<R>* __restrict__ psi, const int (&c)[4], const Geom& g, const Pair& pr,
                                             H6<R>& h, H6<R>* u, H6<R>* l) {
  bool neg;
  const int n = nbr_site<D0, D1, D2, D3>(c, g, neg);
  H6<R> mine;
  load_half<R>(psi, n, pr.p, mine);
  if (neg) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) mine.v[s][a] = -mine.v[s][a];
  }
  const H6<R> oth = partner(mine, pr.mask);
  const R sg = pr.p ? R(-1) : R(1);
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cx<R> m = mine.v[s][a], o = oth.v[s][a];
      h.v[s][a] = mk<R>(m.re + sg * o.re, m.im + sg * o.im);  // p = 0: u + l;  p = 1: l - u = -(u - l)
      if (u) u->v[s][a] = pr.p ? o : m;
      if (l) l->v[s][a] = pr.p ? -m : o;
    }
  return n;
}

// acc_r += 2x2 spin blocks of matrices m .. m + 3 (or their adjoints) times h_r, r < NR.
template <typename R, int NR, bool DAG, typename WS>
__device__ __forceinline__ void mr_block2h(const WS& W, int site, int m, const H6<R> (&h)[NR], H6<R> (&acc)[NR]) {
  M3<R> b = W(site, m + 0);
#pragma unroll
  for (int r = 0; r < NR; ++r) { if (DAG) mdv_add(acc[r].v[0], b, h[r].v[0]); else mv_add(acc[r].v[0], b, h[r].v[0]); }
  b = W(site, m + 1);
#pragma unroll
  for (int r = 0; r < NR; ++r) { if (DAG) mdv_add(acc[r].v[1], b, h[r].v[0]); else mv_add(acc[r].v[0], b, h[r].v[1]); }
  b = W(site, m + 2);
#pragma unroll
  for (int r = 0; r < NR; ++r) { if (DAG) mdv_add(acc[r].v[0], b, h[r].v[1]); else mv_add(acc[r].v[1], b, h[r].v[0]); }
  b = W(site, m + 3);
#pragma unroll
  for (int r = 0; r < NR; ++r) { if (DAG) mdv_add(acc[r].v[1], b, h[r].v[1]); else mv_add(acc[r].v[1], b, h[r].v[1]); }
}

template <typename R, int NR, int I, bool FWD, typename WS>
__device__ __forceinline__ void mr_spatial(const WS& W, const cx<R>* __restrict__ psi, long long rs, const int (&c)[4],
                                           const Geom& g, int s, const Pair& pr, H6<R> (&acc)[NR]) {
  const int base = M_WP + 8 * I;
  H6<R> h[NR];
  if constexpr (FWD) {
#pragma unroll
    for (int r = 0; r < NR; ++r) gather_pair<R, I == 0, I == 1, I == 2, 0>(psi + r * rs, c, g, pr, h[r]);
    mr_block2h<R, NR, false>(W, s, base + 4 * pr.p, h, acc);
  } else {
    int n = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) n = gather_pair<R, -(I == 0), -(I == 1), -(I == 2), 0>(psi + r * rs, c, g, pr, h[r]);
    mr_block2h<R, NR, true>(W, n, base + 4 * (1 - pr.p), h, acc);
  }
}

// Temporal hop with the thread's sign folded into the gathered spinors (see pair_time):
//   forward   acc0 += s3 h'0 + n1 h'1 - U l'0,   acc1 += -s3 h'1 + n2 h'0 - U l'1
//   backward  acc0 -= s3^ h'0 + n2^ h'1 + U^ u0, acc1 += s3^ h'1 - n1^ h'0 - U^ u1   (^ = adjoint)
template <typename R, int NR, bool FWD, typename WS>
__device__ __forceinline__ void mr_time(const WS& W, const cx<R>* __restrict__ psi, long long rs, const int (&c)[4],
                                        const Geom& g, int s, const Pair& pr, H6<R> (&acc)[NR]) {
  H6<R> h[NR], x[NR];
  if constexpr (FWD) {
#pragma unroll
    for (int r = 0; r < NR; ++r) gather_signed<R, 0, 0, 0, 1>(psi + r * rs, c, g, pr, h[r], nullptr, &x[r]);
    M3<R> A = W(s, M_ST + 0);
#pragma unroll
    for (int r = 0; r < NR; ++r) { mv_add(acc[r].v[0], A, h[r].v[0]); mv_sub(acc[r].v[1], A, h[r].v[1]); }
    A = W(s, M_ST + 1);
#pragma unroll
    for (int r = 0; r < NR; ++r) mv_add(acc[r].v[0], A, h[r].v[1]);
    A = W(s, M_ST + 2);
#pragma unroll
    for (int r = 0; r < NR; ++r) mv_add(acc[r].v[1], A, h[r].v[0]);
    A = W(s, M_UT);
#pragma unroll
    for (int r = 0; r < NR; ++r) { mv_sub(acc[r].v[0], A, x[r].v[0]); mv_sub(acc[r].v[1], A, x[r].v[1]); }
  } else {
    int n = 0;
#pragma unroll
    for (int r = 0; r < NR; ++r) n = gather_signed<R, 0, 0, 0, -1>(psi + r * rs, c, g, pr, h[r], &x[r], nullptr);
    M3<R> A = W(n, M_ST + 0);
#pragma unroll
    for (int r = 0; r < NR; ++r) { mdv_sub(acc[r].v[0], A, h[r].v[0]); mdv_add(acc[r].v[1], A, h[r].v[1]); }
    A = W(n, M_ST + 2);
#pragma unroll
    for (int r = 0; r < NR; ++r) mdv_sub(acc[r].v[0], A, h[r].v[1]);
    A = W(n, M_ST + 1);
#pragma unroll
    for (int r = 0; r < NR; ++r) mdv_sub(acc[r].v[1], A, h[r].v[0]);
    A = W(n, M_UT);
#pragma unroll
    for (int r = 0; r < NR; ++r) { mdv_sub(acc[r].v[0], A, x[r].v[0]); mdv_sub(acc[r].v[1], A, x[r].v[1]); }
  }
}

// W^{++}_ii: acc+- += (a +- b sigma_i) V h+-  forward,  (a -+ b sigma_i) V^dag h+-  backward.
template <typename R, int NR, int I, bool FWD, typename WS>
__device__ __forceinline__ void mr_two(const WS& W, const cx<R>* __restrict__ psi, long long rs, const int (&c)[4],
                                       const Geom& g, int s, const Pair& pr, R a, R b, H6<R> (&acc)[NR]) {
  const R sb = pr.p ? -b : b;
  H6<R> h[NR];
  int n = s;
  if constexpr (FWD) {
#pragma unroll
    for (int r = 0; r < NR; ++r) gather_pair<R, 2 * (I == 0), 2 * (I == 1), 2 * (I == 2), 0>(psi + r * rs, c, g, pr, h[r]);
  } else {
#pragma unroll
    for (int r = 0; r < NR; ++r) n = gather_pair<R, -2 * (I == 0), -2 * (I == 1), -2 * (I == 2), 0>(psi + r * rs, c, g, pr, h[r]);
  }
  const M3<R> V = W(n, M_VII + I);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    H6<R> y;
    colour2h<R, !FWD>(y, V, h[r]);
    add_scaled_h(acc[r], a, y);
    add_sigma_h(acc[r], I, y, FWD ? sb : -sb);
  }
}

// Diagonal pair (I, J): +-(s_I + s_J) V h (x+I+J) and +-(s_I - s_J) X h (x+I-J) forward, the
// adjoints with opposite signs from x-I-J and x-I+J backward.
template <typename R, int NR, int I, int J, int P, bool FWD, typename WS>
__device__ __forceinline__ void mr_diag(const WS& W, const cx<R>* __restrict__ psi, long long rs, const int (&c)[4],
                                        const Geom& g, int s, const Pair& pr, H6<R> (&acc)[NR]) {
  constexpr int A0 = (I == 0) + (J == 0), A1 = (I == 1) + (J == 1), A2 = (I == 2) + (J == 2);
  constexpr int B0 = (I == 0) - (J == 0), B1 = (I == 1) - (J == 1), B2 = (I == 2) - (J == 2);
  const R sg = pr.p ? R(-1) : R(1);
  const R f = FWD ? sg : -sg;
  H6<R> h[NR];
  int n = s;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if constexpr (FWD) gather_pair<R, A0, A1, A2, 0>(psi + r * rs, c, g, pr, h[r]);
    else n = gather_pair<R, -A0, -A1, -A2, 0>(psi + r * rs, c, g, pr, h[r]);
  }
  M3<R> V = W(n, M_VIJ + P);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    H6<R> y;
    colour2h<R, !FWD>(y, V, h[r]);
    add_sigma_h(acc[r], I, y, f);
    add_sigma_h(acc[r], J, y, f);
  }
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if constexpr (FWD) gather_pair<R, B0, B1, B2, 0>(psi + r * rs, c, g, pr, h[r]);
    else n = gather_pair<R, -B0, -B1, -B2, 0>(psi + r * rs, c, g, pr, h[r]);
  }
  V = W(n, M_XIJ + P);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    H6<R> y;
    colour2h<R, !FWD>(y, V, h[r]);
    add_sigma_h(acc[r], I, y, f);
    add_sigma_h(acc[r], J, y, -f);
  }
}

template <int NR, int EPI, typename WT>
__global__ void __launch_bounds__(MR_THREADS, mr_minb<NR>())
    apply_mrhs_kernel(const cx<WT>* __restrict__ W, const cx<float>* __restrict__ psi, cx<float>* __restrict__ out, long long rs,
                      Geom g, float c0q, float a_ii, float b_ii, MultiEpi ep) {
  using R = float;
  const int r0 = blockIdx.y * NR;  // first right-hand side of this grid row
  bool live[NR];
  bool any = EPI == EPI_NONE;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    live[r] = EPI == EPI_NONE || ep.st[r0 + r].halt == HALT_NONE;
    any = any || live[r];
  }
  if (!any) return;
  const cx<R>* P = psi + r0 * rs;
  cx<R>* O = out + r0 * rs;
  __shared__ cx<R> xch[2][64][NR][6];
  __shared__ cx<R> xev[EPI == EPI_NONE ? 1 : 2][64][EPI == EPI_NONE ? 1 : NR][6];
  const int half = threadIdx.x >> 6;
  const int t = threadIdx.x & 63;
  Pair pr;
  pr.p = t & 1;
  pr.mask = 3u << (threadIdx.x & 30);
  const GlobalW<WT> Wg{W};
  R red[NR][3];
#pragma unroll
  for (int r = 0; r < NR; ++r) red[r][0] = red[r][1] = red[r][2] = 0;
  const int ntiles = (g.V + MR_SITES - 1) / MR_SITES;
  int kb = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, kb ^= 1) {
    const int s = tile * MR_SITES + (t >> 1);
    const bool active = s < g.V;
    H6<R> acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[r].v[q][k] = mk<R>(0, 0);
    if (active) {
      int c[4];
      int rr = s;
      c[0] = rr % g.L[0]; rr /= g.L[0];
      c[1] = rr % g.L[1]; rr /= g.L[1];
      c[2] = rr % g.L[2]; c[3] = rr / g.L[2];
      if (half == 0) {
#pragma unroll
        for (int r = 0; r < NR; ++r) pair_onsite<R>(Wg, P + r * rs, s, pr, c0q, acc[r]);
        mr_time<R, NR, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_spatial<R, NR, 0, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_spatial<R, NR, 1, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_spatial<R, NR, 2, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_two<R, NR, 0, true>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_two<R, NR, 1, true>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_two<R, NR, 2, true>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_diag<R, NR, 0, 1, 0, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_diag<R, NR, 0, 2, 1, true>(Wg, P, rs, c, g, s, pr, acc);
        mr_diag<R, NR, 1, 2, 2, true>(Wg, P, rs, c, g, s, pr, acc);
      } else {
        mr_spatial<R, NR, 0, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_spatial<R, NR, 1, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_spatial<R, NR, 2, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_time<R, NR, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_two<R, NR, 0, false>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_two<R, NR, 1, false>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_two<R, NR, 2, false>(Wg, P, rs, c, g, s, pr, a_ii, b_ii, acc);
        mr_diag<R, NR, 0, 1, 0, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_diag<R, NR, 0, 2, 1, false>(Wg, P, rs, c, g, s, pr, acc);
        mr_diag<R, NR, 1, 2, 2, false>(Wg, P, rs, c, g, s, pr, acc);
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) xch[kb][t][r][3 * q + k] = acc[r].v[q][k];
        if (EPI != EPI_NONE) {
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            H6<R> ev;
            load_half<R>((EPI == EPI_DOT || ep.rhat) ? ep.rhat + (r0 + r) * rs : P + r * rs, s, pr.p, ev);
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
              for (int k = 0; k < 3; ++k) xev[kb][t][EPI == EPI_NONE ? 0 : r][3 * q + k] = ev.v[q][k];
          }
        }
      }
    }
    __syncthreads();
    if (half == 0 && active) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int k = 0; k < 3; ++k) acc[r].v[q][k] = acc[r].v[q][k] + xch[kb][t][r][3 * q + k];
        // out_u = acc+ + acc- (p = 0 writes it), out_l = acc+ - acc- (p = 1)
        const H6<R> ap = partner(acc[r], pr.mask);
        H6<R> o;
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int k = 0; k < 3; ++k) o.v[q][k] = pr.p ? ap.v[q][k] - acc[r].v[q][k] : acc[r].v[q][k] + ap.v[q][k];
        store_half<R>(O + r * rs, s, pr.p, o);
        if (EPI == EPI_DOT) {
          cx<R> d = mk<R>(0, 0);
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) d = fma_cj(xev[kb][t][EPI == EPI_NONE ? 0 : r][3 * q + k], o.v[q][k], d);
          red[r][0] += d.re;
          red[r][1] += d.im;
        } else if (EPI == EPI_TS) {
          cx<R> d = mk<R>(0, 0);
          R n2 = 0;
#pragma unroll
          for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              d = fma_cj(o.v[q][k], xev[kb][t][EPI == EPI_NONE ? 0 : r][3 * q + k], d);
              n2 += o.v[q][k].re * o.v[q][k].re + o.v[q][k].im * o.v[q][k].im;
            }
          red[r][0] += d.re;
          red[r][1] += d.im;
          red[r][2] += n2;
        }
      }
    }
  }
  if constexpr (EPI != EPI_NONE) {
    // One deterministic grid reduction per live right-hand side (the same for every block of the
    // row, so each reduction sees all gridDim.x blocks), into that right-hand side's state.
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (!live[r]) continue;
      SolverState* st = ep.st + r0 + r;
      const RedArgs ra{st, ep.part + (size_t)(r0 + r) * ep.pstride, nullptr, ep.fin};
      if (EPI == EPI_DOT) {
        double v2[2] = {(double)red[r][0], (double)red[r][1]};
        grid_reduce<2, MR_THREADS>(v2, ra, &st->ticket[ep.slot]);
      } else {
        double v3[3] = {(double)red[r][0], (double)red[r][1], (double)red[r][2]};
        grid_reduce<3, MR_THREADS>(v3, ra, &st->ticket[ep.slot]);
      }
    }
  }
}

template <int NR, int EPI, typename WT>
int launch_nr(const ok_W* Wh, const cx<WT>* W, const cx<float>* psi, cx<float>* out, int nrhs, const MultiEpi& ep,
              int blocks_x, cudaStream_t st) {
  const Geom& g = Wh->g;
  static int resident = 0;
  auto kern = apply_mrhs_kernel<NR, EPI, WT>;
  if (resident == 0) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, MR_THREADS, 0) != cudaSuccess || nb < 1) nb = 1;
    resident = nb * sm_count();
  }
  const int rows = nrhs / NR;
  const int tiles = grid_for(g.V, MR_SITES);
  int bx = blocks_x > 0 ? blocks_x : resident / rows;
  if (bx < 1) bx = 1;
  if (bx > tiles) bx = tiles;
  kern<<<dim3(bx, rows), MR_THREADS, 0, st>>>(W, psi, out, 12LL * g.V, g, (float)Wh->sc.c0q, (float)Wh->sc.a_ii,
                                              (float)Wh->sc.b_ii, ep);
  return OK_SUCCESS;
}

template <int EPI, typename WT>
int launch_epi(const ok_W* Wh, const cx<WT>* W, const cx<float>* psi, cx<float>* out, int nrhs, int nr, const MultiEpi& ep,
               int blocks_x, cudaStream_t st) {
  switch (nr) {
    case 1: return launch_nr<1, EPI, WT>(Wh, W, psi, out, nrhs, ep, blocks_x, st);
    case 2: return launch_nr<2, EPI, WT>(Wh, W, psi, out, nrhs, ep, blocks_x, st);
    case 4: return launch_nr<4, EPI, WT>(Wh, W, psi, out, nrhs, ep, blocks_x, st);
    default: return OK_EINVAL;
  }
}

// All epilogues for one W storage type (explicitly instantiated in ok_mrhs.cu and ok_mrhs16.cu,
// which compile in parallel).
template <typename WT>
int launch_wt(const ok_W* Wh, const cx<WT>* W, const cx<float>* psi, cx<float>* out, int nrhs, int epi, const MultiEpi& ep,
              const MultiShape& shape, cudaStream_t st) {
  if (epi == EPI_NONE) return launch_epi<EPI_NONE, WT>(Wh, W, psi, out, nrhs, shape.nr, ep, shape.blocks_x, st);
  if (epi == EPI_DOT) return launch_epi<EPI_DOT, WT>(Wh, W, psi, out, nrhs, shape.nr, ep, shape.blocks_x, st);
  return launch_epi<EPI_TS, WT>(Wh, W, psi, out, nrhs, shape.nr, ep, shape.blocks_x, st);
}

}  // namespace mrhs

}  // namespace okgb
