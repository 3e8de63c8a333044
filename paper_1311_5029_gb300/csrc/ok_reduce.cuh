// Deterministic grid reductions and the device-resident BiCGStab state.
//
// A reducing kernel gives every thread NP double-precision contributions.  Each block sums them
// with a fixed warp-shuffle tree and writes one partial per quantity; the last block to finish
// (atomic ticket) sums the partials in block order with a fixed tree, so results are bitwise
// reproducible for a given launch shape, and then runs a finalisation hook on thread 0.
#pragma once

#include "ok_internal.cuh"

namespace okgb {

// Complex as two doubles in device scalars.
struct dcx { double re, im; };

__host__ __device__ __forceinline__ dcx dmk(double a, double b) { dcx z; z.re = a; z.im = b; return z; }
__host__ __device__ __forceinline__ dcx dmul(dcx a, dcx b) { return dmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__host__ __device__ __forceinline__ dcx ddiv(dcx a, dcx b) {
  double d = b.re * b.re + b.im * b.im;
  return dmk((a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d);
}
__host__ __device__ __forceinline__ double dabs2(dcx a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ bool dfinite(dcx a) { return isfinite(a.re) && isfinite(a.im); }

// BiCGStab state in device memory (one per solve).
struct SolverState {
  dcx rho;       // <rhat, r>
  dcx alpha;
  dcx omega;
  dcx beta;
  dcx rv;        // <rhat, v>
  double rr;     // |r|^2 of the iterated residual
  double bb;     // |b|^2
  double rhat2;  // |rhat|^2
  double rmax2;  // max |r|^2 since the last reliable update (mixed mode)
  double tol2;   // tol^2
  double delta2; // delta^2 (mixed mode; 0 = never)
  double tt;     // <t, t>
  double aux[4]; // extra sums returned by reductions
  int iter;      // completed iterations
  int maxiter;
  int halt;      // nonzero: skip further iteration kernels (see HALT_*)
  int pad;
  unsigned ticket[8];
};

enum : int {
  HALT_NONE = 0,
  HALT_CONVERGED = 1,   // iterated residual below tol
  HALT_UPDATE = 2,      // mixed mode: reliable update due
  HALT_BREAKDOWN = 3,   // rho, <rhat, v> or omega vanished
  HALT_NONFINITE = 4,   // NaN or Inf in a scalar
  HALT_MAXITER = 5,
};

// Which finalisation runs after a reduction.
enum : int {
  FIN_NONE = 0,        // only store the sums in state->aux
  FIN_ALPHA = 1,       // sums = (Re, Im) <rhat, v>: alpha = rho / <rhat, v>
  FIN_OMEGA = 2,       // sums = (Re, Im) <t, s>, <t, t>: omega
  FIN_XR = 3,          // sums = (Re, Im) <rhat, r>, <r, r>: beta, convergence, reliable trigger
  FIN_RESTART = 4,     // sums = <r, r>: rho = rhat2 = rr = rmax2 = <r, r> (rhat = p = r)
  FIN_CONTINUE = 5,    // sums = (Re, Im) <rhat, r>, <r, r>: rho_new, beta (after a reliable update)
  FIN_RESID = 6,       // sums = <b - M x, b - M x>, <b, b>: store |b|^2 (the residual stays in aux)
};

struct RedArgs {
  SolverState* st;   // may be null for FIN_NONE with `out`
  double* part;      // [gridDim.x * NP]
  double* out;       // optional: final sums copied here (NP doubles)
  int fin;
};

__device__ __forceinline__ void finalise(SolverState* st, int fin, const double* v) {
  if (!st) return;
  switch (fin) {
    case FIN_ALPHA: {
      dcx rv = dmk(v[0], v[1]);
      st->rv = rv;
      if (!dfinite(rv)) { st->halt = HALT_NONFINITE; break; }
      // breakdown if |<rhat, v>| is tiny against |rhat| |v| (|v| is not summed: use |rhat| |r|)
      if (dabs2(rv) <= 1e-60 * st->rhat2 * st->rr || dabs2(rv) == 0.0) { st->halt = HALT_BREAKDOWN; break; }
      st->alpha = ddiv(st->rho, rv);
      break;
    }
    case FIN_OMEGA: {
      dcx ts = dmk(v[0], v[1]);
      double tt = v[2];
      st->tt = tt;
      if (!dfinite(ts) || !isfinite(tt)) { st->halt = HALT_NONFINITE; break; }
      if (tt == 0.0) { st->omega = dmk(0.0, 0.0); break; }  // s = 0 exactly: x update is complete
      st->omega = dmk(ts.re / tt, ts.im / tt);
      break;
    }
    case FIN_XR: {
      dcx rho_new = dmk(v[0], v[1]);
      double rr = v[2];
      st->rr = rr;
      st->iter += 1;
      if (!dfinite(rho_new) || !isfinite(rr)) { st->halt = HALT_NONFINITE; break; }
      if (rr > st->rmax2) st->rmax2 = rr;
      if (rr < st->tol2 * st->bb) { st->halt = st->delta2 > 0.0 ? HALT_UPDATE : HALT_CONVERGED; break; }
      if (st->delta2 > 0.0 && rr < st->delta2 * st->rmax2) { st->halt = HALT_UPDATE; break; }
      if (dabs2(st->omega) == 0.0 || dabs2(rho_new) <= 1e-60 * st->rhat2 * rr) { st->halt = HALT_BREAKDOWN; break; }
      st->beta = dmul(ddiv(rho_new, st->rho), ddiv(st->alpha, st->omega));
      st->rho = rho_new;
      if (st->iter >= st->maxiter) st->halt = HALT_MAXITER;
      break;
    }
    case FIN_RESTART: {
      st->rr = v[0];
      st->rho = dmk(v[0], 0.0);
      st->rhat2 = v[0];
      st->rmax2 = v[0];
      st->halt = HALT_NONE;
      if (!isfinite(v[0])) st->halt = HALT_NONFINITE;
      break;
    }
    case FIN_RESID:
      st->bb = v[1];
      break;
    case FIN_CONTINUE: {
      dcx rho_new = dmk(v[0], v[1]);
      double rr = v[2];
      st->rr = rr;
      st->rmax2 = rr;
      st->halt = HALT_NONE;
      if (!dfinite(rho_new) || !isfinite(rr)) { st->halt = HALT_NONFINITE; break; }
      if (dabs2(st->omega) == 0.0 || dabs2(rho_new) <= 1e-60 * st->rhat2 * rr) { st->halt = HALT_BREAKDOWN; break; }
      st->beta = dmul(ddiv(rho_new, st->rho), ddiv(st->alpha, st->omega));
      st->rho = rho_new;
      break;
    }
    default:
      break;
  }
  for (int k = 0; k < 3; ++k) st->aux[k] = v[k];
}

// Sum NP values over the block (fixed tree); thread 0 receives the totals.
template <int NP, int THREADS>
__device__ __forceinline__ void block_sums(double v[NP], double (*sh)[THREADS / 32]) {
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      double x = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) x += sh[k][w];
      v[k] = x;
    }
  }
  __syncthreads();
}

// Block partials, then the last block reduces all partials and finalises.
template <int NP, int THREADS>
__device__ __forceinline__ void grid_reduce(double v[NP], const RedArgs& ra, unsigned* ticket) {
  __shared__ double sh[NP][THREADS / 32];
  __shared__ int last;
  block_sums<NP, THREADS>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) ra.part[(size_t)blockIdx.x * NP + k] = v[k];
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Thread t sums partials t, t + THREADS, ... in that order; RED_UNROLL loads are issued before
  // they are added, so the tail is not a chain of dependent L2 round trips.
  constexpr int RED_UNROLL = 8;
  double w[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) w[k] = 0.0;
  const unsigned G = gridDim.x;
  for (unsigned b0 = threadIdx.x; b0 < G; b0 += THREADS * RED_UNROLL) {
    double tmp[RED_UNROLL][NP];
#pragma unroll
    for (int u = 0; u < RED_UNROLL; ++u) {
      const unsigned b = b0 + u * THREADS;
#pragma unroll
      for (int k = 0; k < NP; ++k) tmp[u][k] = b < G ? __ldcg(ra.part + (size_t)b * NP + k) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < RED_UNROLL; ++u)
#pragma unroll
      for (int k = 0; k < NP; ++k) w[k] += tmp[u][k];
  }
  block_sums<NP, THREADS>(w, sh);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NP && k < 4; ++k) tot[k] = w[k];
    if (ra.out) {
#pragma unroll
      for (int k = 0; k < NP; ++k) ra.out[k] = w[k];
    }
    finalise(ra.st, ra.fin, tot);
  }
}

}  // namespace okgb
