// BiCGStab vector updates with fused inner products (the "vector addition" work the paper times
// in Table 1c).  Vectors are complex arrays of n = 12 V entries, processed in 16-byte units
// (one complex double or two complex floats).  Every kernel first reads the solver's halt flag
// so that iterations enqueued after convergence are no-ops; scalars (alpha, omega, beta) are read
// from the device-resident state, so no host round trip is needed between kernels.
//
// The three iteration kernels (update_s, update_xr, update_p) also run batched over several
// right-hand sides: grid row blockIdx.y works on vectors offset by blockIdx.y * n with state
// st[blockIdx.y] and its own reduction partials (one launch for all systems of a multi-RHS solve).
#include "ok_launch.cuh"

#include <mutex>
#include <utility>
#include <vector>

namespace okgb {

constexpr int BLAS_THREADS = 256;

template <typename R> struct Unit;
template <> struct Unit<double> {
  using T = double2;
  static constexpr int NC = 1;
  __device__ static __forceinline__ void get(const T& u, cx<double> (&c)[1]) { c[0] = mk(u.x, u.y); }
  __device__ static __forceinline__ T put(const cx<double> (&c)[1]) { return make_double2(c[0].re, c[0].im); }
};
template <> struct Unit<float> {
  using T = float4;
  static constexpr int NC = 2;
  __device__ static __forceinline__ void get(const T& u, cx<float> (&c)[2]) { c[0] = mk(u.x, u.y); c[1] = mk(u.z, u.w); }
  __device__ static __forceinline__ T put(const cx<float> (&c)[2]) { return make_float4(c[0].re, c[0].im, c[1].re, c[1].im); }
};

template <typename R> __device__ __forceinline__ cx<R> scal(dcx z) { return mk<R>((R)z.re, (R)z.im); }

// ---------------------------------------------------------------------------- FP32-pipe grid sums
// The reductions of the FP32 kernels keep every partial sum as a double-float pair (hi + lo, two
// floats, about 44 significand bits; ok_internal.cuh): each thread adds its chunk sums into pairs,
// each block sums its threads' pairs with a fixed shuffle tree, and the last block sums the block
// partials the same way before the FP64 finalisation.  All of it runs on the FP32 pipes.  FP64
// arithmetic runs at 1/58 of the FP32 rate on this part; done in FP64, the block trees cost more
// than streaming the vectors, and the last block's tree kept one SM busy for about 6 us after the
// others had finished.  The order of every sum is fixed by the launch shape.
template <typename R> struct RedT { using T = double; };
template <> struct RedT<float> { using T = dd; };
__device__ __forceinline__ void red_add(double& a, double c) { a += c; }
__device__ __forceinline__ void red_add(dd& a, float c) { a = a + dd(c, 0.f); }
__device__ __forceinline__ dd shfl_xor_dd(dd a, int o) {
  return dd(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
}

template <int NP, int THREADS>
__device__ __forceinline__ void block_sums_dd(dd (&v)[NP], dd (*sh)[THREADS / 32]) {
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    dd x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = x + shfl_xor_dd(x, o);
    if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      dd x = sh[k][0];
      for (int w = 1; w < THREADS / 32; ++w) x = x + sh[k][w];
      v[k] = x;
    }
  }
  __syncthreads();
}

// grid_reduce (ok_reduce.cuh) in double-float: block partials stored as doubles (hi + lo, exact),
// the last block sums them and finalises.
template <int NP, int THREADS>
__device__ __forceinline__ void grid_reduce_dd(dd (&v)[NP], const RedArgs& ra, unsigned* ticket) {
  __shared__ dd sh[NP][THREADS / 32];
  __shared__ int last;
  block_sums_dd<NP, THREADS>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NP; ++k) ra.part[(size_t)blockIdx.x * NP + k] = (double)v[k];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  dd w[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) w[k] = dd(0.f, 0.f);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += THREADS)
#pragma unroll
    for (int k = 0; k < NP; ++k) w[k] = w[k] + dd(__ldcg(ra.part + (size_t)b * NP + k));
  block_sums_dd<NP, THREADS>(w, sh);
  if (threadIdx.x == 0) {
    *ticket = 0u;
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < NP && k < 4; ++k) tot[k] = (double)w[k];
    if (ra.out) {
#pragma unroll
      for (int k = 0; k < NP; ++k) ra.out[k] = tot[k];
    }
    finalise(ra.st, ra.fin, tot);
  }
}

// The grid reduction of the precision R's kernels.
template <typename R, int NP>
__device__ __forceinline__ void grid_reduce_r(typename RedT<R>::T (&v)[NP], const RedArgs& ra, unsigned* ticket) {
  if constexpr (sizeof(R) == 4) grid_reduce_dd<NP, BLAS_THREADS>(v, ra, ticket);
  else grid_reduce<NP, BLAS_THREADS>(v, ra, ticket);
}

#define OK_GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)BLAS_THREADS + threadIdx.x; i < (n); i += (long long)gridDim.x * BLAS_THREADS)

// The reducing kernels sum RED_CHUNK units per thread in the vectors' own precision and add each
// chunk's sums into the thread's FP64 totals: FP64 arithmetic runs at a small fraction of the FP32
// rate on this part, so an FP64 conversion and add per unit would bound the kernel.  A chunk's
// units (stride: the grid) are loaded together.  The order of every sum is fixed by the launch
// shape, so results are reproducible.
constexpr int RED_CHUNK = 8;
#define OK_CHUNK_STRIDE(i0, n) \
  for (long long i0 = blockIdx.x * (long long)BLAS_THREADS + threadIdx.x; i0 < (n); i0 += (long long)gridDim.x * BLAS_THREADS * RED_CHUNK)
#define OK_CHUNK_UNITS(i, i0, n)                   \
  _Pragma("unroll") for (int u_ = 0; u_ < RED_CHUNK; ++u_) \
    if (const long long i = (i0) + (long long)u_ * gridDim.x * BLAS_THREADS; i < (n))

// s = r - alpha v
template <typename R>
__global__ void __launch_bounds__(BLAS_THREADS) update_s_kernel(const typename Unit<R>::T* __restrict__ r,
                                                                const typename Unit<R>::T* __restrict__ v,
                                                                typename Unit<R>::T* __restrict__ s, long long nu,
                                                                const SolverState* __restrict__ st) {
  const long long off = (long long)blockIdx.y * nu;
  r += off; v += off; s += off; st += blockIdx.y;
  if (st->halt) return;
  using U = Unit<R>;
  const cx<R> al = scal<R>(st->alpha);
  OK_GRID_STRIDE(i, nu) {
    cx<R> a[U::NC], b[U::NC];
    U::get(r[i], a);
    U::get(v[i], b);
#pragma unroll
    for (int k = 0; k < U::NC; ++k) a[k] = a[k] - al * b[k];
    s[i] = U::put(a);
  }
}

// x += alpha p + omega s;  r = s - omega t;  sums <rhat, r>, <r, r>  ->  FIN_XR.  With sx set (right
// preconditioning: p and sx are the preconditioned directions P p and P s) x += alpha p + omega sx.
template <typename R>
__global__ void __launch_bounds__(BLAS_THREADS) update_xr_kernel(typename Unit<R>::T* __restrict__ x,
                                                                 const typename Unit<R>::T* __restrict__ p,
                                                                 const typename Unit<R>::T* __restrict__ s,
                                                                 const typename Unit<R>::T* __restrict__ t,
                                                                 typename Unit<R>::T* __restrict__ r,
                                                                 const typename Unit<R>::T* __restrict__ rhat,
                                                                 long long nu, SolverState* __restrict__ st,
                                                                 RedArgs ra, long long pstride,
                                                                 const typename Unit<R>::T* __restrict__ sx) {
  const long long off = (long long)blockIdx.y * nu;
  x += off; p += off; s += off; t += off; r += off; rhat += off; st += blockIdx.y;
  if (sx) sx += off;
  ra.st = st;
  ra.part += (long long)blockIdx.y * pstride;
  if (st->halt) return;
  using U = Unit<R>;
  const cx<R> al = scal<R>(st->alpha), om = scal<R>(st->omega);
  typename RedT<R>::T red[3] = {0, 0, 0};
  OK_CHUNK_STRIDE(i0, nu) {
    cx<R> d = mk<R>(0, 0);
    R n2 = 0;
    OK_CHUNK_UNITS(i, i0, nu) {
      cx<R> xv[U::NC], pv[U::NC], sv[U::NC], tv[U::NC], hv[U::NC], zv[U::NC];
      U::get(x[i], xv);
      U::get(p[i], pv);
      U::get(s[i], sv);
      U::get(t[i], tv);
      U::get(rhat[i], hv);
      if (sx) U::get(sx[i], zv);
#pragma unroll
      for (int k = 0; k < U::NC; ++k) {
        xv[k] = xv[k] + al * pv[k] + om * (sx ? zv[k] : sv[k]);
        sv[k] = sv[k] - om * tv[k];
        d = fma_cj(hv[k], sv[k], d);
        n2 += sv[k].re * sv[k].re + sv[k].im * sv[k].im;
      }
      x[i] = U::put(xv);
      r[i] = U::put(sv);
    }
    red_add(red[0], d.re);
    red_add(red[1], d.im);
    red_add(red[2], n2);
  }
  grid_reduce_r<R, 3>(red, ra, &st->ticket[2]);
}

// p = r + beta (p - omega v)
template <typename R>
__global__ void __launch_bounds__(BLAS_THREADS) update_p_kernel(typename Unit<R>::T* __restrict__ p,
                                                                const typename Unit<R>::T* __restrict__ r,
                                                                const typename Unit<R>::T* __restrict__ v,
                                                                long long nu, const SolverState* __restrict__ st) {
  const long long off = (long long)blockIdx.y * nu;
  p += off; r += off; v += off; st += blockIdx.y;
  if (st->halt) return;
  using U = Unit<R>;
  const cx<R> be = scal<R>(st->beta), om = scal<R>(st->omega);
  OK_GRID_STRIDE(i, nu) {
    cx<R> pv[U::NC], rv[U::NC], vv[U::NC];
    U::get(p[i], pv);
    U::get(r[i], rv);
    U::get(v[i], vv);
#pragma unroll
    for (int k = 0; k < U::NC; ++k) pv[k] = rv[k] + be * (pv[k] - om * vv[k]);
    p[i] = U::put(pv);
  }
}

// The inner products a BiCGStab half-iteration takes from its application of M, in a pass of their
// own (the FP32 applications run without a fused epilogue; the separate pass over two vectors
// costs less than the epilogue did): ALPHA: <a, b> (a = rhat, b = v) -> FIN_ALPHA;
// OMEGA: <a, b>, <a, a> (a = t, b = s) -> FIN_OMEGA.
template <typename R, bool OMEGA>
__global__ void __launch_bounds__(BLAS_THREADS) dots_kernel(const typename Unit<R>::T* __restrict__ a,
                                                            const typename Unit<R>::T* __restrict__ b, long long nu,
                                                            SolverState* __restrict__ st, RedArgs ra, unsigned* ticket) {
  if (st->halt) return;
  using U = Unit<R>;
  typename RedT<R>::T red[3] = {0, 0, 0};
  OK_CHUNK_STRIDE(i0, nu) {
    cx<R> d = mk<R>(0, 0);
    R n2 = 0;
    OK_CHUNK_UNITS(i, i0, nu) {
      cx<R> av[U::NC], bv[U::NC];
      U::get(a[i], av);
      U::get(b[i], bv);
#pragma unroll
      for (int k = 0; k < U::NC; ++k) {
        d = fma_cj(av[k], bv[k], d);
        if (OMEGA) n2 += av[k].re * av[k].re + av[k].im * av[k].im;
      }
    }
    red_add(red[0], d.re);
    red_add(red[1], d.im);
    red_add(red[2], n2);
  }
  if (OMEGA) {
    grid_reduce_r<R, 3>(red, ra, ticket);
  } else {
    typename RedT<R>::T v2[2] = {red[0], red[1]};
    grid_reduce_r<R, 2>(v2, ra, ticket);
  }
}

// Restart: rhat = p = r (same precision), sum <r, r> -> FIN_RESTART.
template <typename R>
__global__ void __launch_bounds__(BLAS_THREADS) restart_kernel(const typename Unit<R>::T* __restrict__ r,
                                                               typename Unit<R>::T* __restrict__ rhat,
                                                               typename Unit<R>::T* __restrict__ p, long long nu,
                                                               SolverState* __restrict__ st, RedArgs ra) {
  using U = Unit<R>;
  typename RedT<R>::T red[1] = {0};
  OK_CHUNK_STRIDE(i0, nu) {
    R n2 = 0;
    OK_CHUNK_UNITS(i, i0, nu) {
      typename U::T u = r[i];
      rhat[i] = u;
      p[i] = u;
      cx<R> a[U::NC];
      U::get(u, a);
#pragma unroll
      for (int k = 0; k < U::NC; ++k) n2 += a[k].re * a[k].re + a[k].im * a[k].im;
    }
    red_add(red[0], n2);
  }
  grid_reduce_r<R, 1>(red, ra, &st->ticket[3]);
}

// Mixed precision: r32 = (float) r64; RESTART: rhat = p = r32 and FIN_RESTART on <r, r>;
// otherwise FIN_CONTINUE on <rhat, r32>, <r32, r32>.  Units are complex doubles here.
template <bool RESTART>
__global__ void __launch_bounds__(BLAS_THREADS) demote_kernel(const double2* __restrict__ r64, float2* __restrict__ r32,
                                                              float2* __restrict__ rhat, float2* __restrict__ p,
                                                              long long n, SolverState* __restrict__ st, RedArgs ra) {
  double red[3] = {0.0, 0.0, 0.0};
  OK_CHUNK_STRIDE(i0, n) {
    float c[3] = {0.f, 0.f, 0.f};
    OK_CHUNK_UNITS(i, i0, n) {
      double2 d = r64[i];
      float2 f = make_float2((float)d.x, (float)d.y);
      r32[i] = f;
      if (RESTART) {
        rhat[i] = f;
        p[i] = f;
        c[0] += f.x * f.x + f.y * f.y;
      } else {
        float2 h = rhat[i];
        c[0] += h.x * f.x + h.y * f.y;
        c[1] += h.x * f.y - h.y * f.x;
        c[2] += f.x * f.x + f.y * f.y;
      }
    }
    red[0] += c[0];
    red[1] += c[1];
    red[2] += c[2];
  }
  if (RESTART) {
    double v1[1] = {red[0]};
    grid_reduce<1, BLAS_THREADS>(v1, ra, &st->ticket[4]);
  } else {
    grid_reduce<3, BLAS_THREADS>(red, ra, &st->ticket[4]);
  }
}

// Mixed precision: x64 += x32, x32 = 0.
__global__ void __launch_bounds__(BLAS_THREADS) accum_x_kernel(double2* __restrict__ x64, float2* __restrict__ x32, long long n) {
  OK_GRID_STRIDE(i, n) {
    float2 f = x32[i];
    double2 d = x64[i];
    d.x += (double)f.x;
    d.y += (double)f.y;
    x64[i] = d;
    x32[i] = make_float2(0.f, 0.f);
  }
}

// <x, x> and <b, b> (FP64 vectors, complex-double units).
__global__ void __launch_bounds__(BLAS_THREADS) norms_kernel(const double2* __restrict__ x, const double2* __restrict__ b,
                                                             long long n, SolverState* __restrict__ st, RedArgs ra) {
  double red[2] = {0.0, 0.0};
  OK_GRID_STRIDE(i, n) {
    double2 u = x[i], v = b[i];
    red[0] += u.x * u.x + u.y * u.y;
    red[1] += v.x * v.x + v.y * v.y;
  }
  grid_reduce<2, BLAS_THREADS>(red, ra, &st->ticket[6]);
}

// FP64 -> double-float: each double d becomes (hi, lo) = (float(d), float(d - hi)).
__global__ void __launch_bounds__(BLAS_THREADS) to_df_kernel(const double2* __restrict__ in, float4* __restrict__ out,
                                                             long long n) {
  OK_GRID_STRIDE(i, n) {
    const double2 v = in[i];
    const dd re(v.x), im(v.y);
    out[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}

// ---------------------------------------------------------------------------- launchers
static int g_sms = 0;

int sm_count() {
  if (g_sms == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 132;
    g_sms = sms;
  }
  return g_sms;
}

// Upper bound of every vector kernel's grid width (sizes the reduction partials).
int blas_blocks(long long units) {
  long long need = (units + BLAS_THREADS - 1) / BLAS_THREADS;
  long long cap = (long long)sm_count() * 8;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

// Grid width for one vector kernel: one full wave of the blocks that fit on the device at once
// (from the occupancy calculator; a grid-stride loop covers the rest).  A wider grid would leave a
// partial second wave that every thread of the first must wait for: the kernels that hold more
// registers (update_xr at 48) fit 5 blocks of 256 threads per SM, not 8.
// Kernels that end in a grid reduction take at most this many blocks per multiprocessor: every
// block's partial ends in a fence and an atomic on one completion counter, and at a full wave
// (up to 8 x 152 blocks) those serialised atomics cost more than the few extra loads in flight.
#ifndef OK_RED_BLOCKS_PER_SM
#define OK_RED_BLOCKS_PER_SM 4
#endif
template <typename K>
static int wave_blocks(K kern, long long units, bool reduces = false) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> cache;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& e : cache)
      if (e.first == (const void*)kern) per_sm = e.second;
    if (per_sm == 0) {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLAS_THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
      if (per_sm > 8) per_sm = 8;
      cache.emplace_back((const void*)kern, per_sm);
    }
  }
  if (reduces && per_sm > OK_RED_BLOCKS_PER_SM) per_sm = OK_RED_BLOCKS_PER_SM;
  const long long need = (units + BLAS_THREADS - 1) / BLAS_THREADS;
  const long long cap = (long long)sm_count() * per_sm;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

template <typename R> long long units_of(long long ncomplex) { return ncomplex / Unit<R>::NC; }

template <typename R>
int launch_update_s(const cx<R>* r, const cx<R>* v, cx<R>* s, long long n, const SolverState* st, cudaStream_t strm) {
  using T = typename Unit<R>::T;
  long long nu = units_of<R>(n);
  {
    TraceScope ts(sizeof(R) == 8 ? "update_s_f64" : "update_s_f32", strm);
    update_s_kernel<R><<<wave_blocks(update_s_kernel<R>, nu), BLAS_THREADS, 0, strm>>>((const T*)r, (const T*)v, (T*)s, nu, st);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

template <typename R>
int launch_update_xr(cx<R>* x, const cx<R>* p, const cx<R>* s, const cx<R>* t, cx<R>* r, const cx<R>* rhat, long long n,
                     SolverState* st, double* part, cudaStream_t strm, const cx<R>* sx) {
  using T = typename Unit<R>::T;
  long long nu = units_of<R>(n);
  RedArgs ra{st, part, nullptr, FIN_XR};
  {
    TraceScope ts(sizeof(R) == 8 ? "update_xr_f64" : "update_xr_f32", strm);
    update_xr_kernel<R><<<wave_blocks(update_xr_kernel<R>, nu, true), BLAS_THREADS, 0, strm>>>((T*)x, (const T*)p, (const T*)s, (const T*)t, (T*)r,
                                                                  (const T*)rhat, nu, st, ra, 0, (const T*)sx);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

template <typename R>
int launch_dots(const cx<R>* a, const cx<R>* b, long long n, bool omega, SolverState* st, double* part, cudaStream_t strm) {
  using T = typename Unit<R>::T;
  long long nu = units_of<R>(n);
  RedArgs ra{st, part, nullptr, omega ? FIN_OMEGA : FIN_ALPHA};
  {
    TraceScope ts(omega ? (sizeof(R) == 8 ? "dots_ts_f64" : "dots_ts_f32") : (sizeof(R) == 8 ? "dot_rv_f64" : "dot_rv_f32"), strm);
    if (omega)
      dots_kernel<R, true><<<wave_blocks(dots_kernel<R, true>, nu, true), BLAS_THREADS, 0, strm>>>((const T*)a, (const T*)b, nu, st, ra,
                                                                                          &st->ticket[omega ? 1 : 0]);
    else
      dots_kernel<R, false><<<wave_blocks(dots_kernel<R, false>, nu, true), BLAS_THREADS, 0, strm>>>((const T*)a, (const T*)b, nu, st, ra,
                                                                                            &st->ticket[0]);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

template <typename R>
int launch_update_p(cx<R>* p, const cx<R>* r, const cx<R>* v, long long n, const SolverState* st, cudaStream_t strm) {
  using T = typename Unit<R>::T;
  long long nu = units_of<R>(n);
  {
    TraceScope ts(sizeof(R) == 8 ? "update_p_f64" : "update_p_f32", strm);
    update_p_kernel<R><<<wave_blocks(update_p_kernel<R>, nu), BLAS_THREADS, 0, strm>>>((T*)p, (const T*)r, (const T*)v, nu, st);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

template <typename R>
int launch_restart(const cx<R>* r, cx<R>* rhat, cx<R>* p, long long n, SolverState* st, double* part, cudaStream_t strm) {
  using T = typename Unit<R>::T;
  long long nu = units_of<R>(n);
  RedArgs ra{st, part, nullptr, FIN_RESTART};
  {
    TraceScope ts(sizeof(R) == 8 ? "restart_f64" : "restart_f32", strm);
    restart_kernel<R><<<wave_blocks(restart_kernel<R>, nu), BLAS_THREADS, 0, strm>>>((const T*)r, (T*)rhat, (T*)p, nu, st, ra);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

// Batched over nrhs systems (vectors [nrhs][n], states [nrhs]); reductions use part + k * pstride
// for system k, pstride >= 3 * blas_blocks(n / units).
int launch_update_s_multi(const cx<float>* r, const cx<float>* v, cx<float>* s, long long n, int nrhs, const SolverState* st,
                          cudaStream_t strm) {
  using T = Unit<float>::T;
  const long long nu = units_of<float>(n);
  {
    TraceScope ts("update_s_multi", strm);
    update_s_kernel<float><<<dim3(wave_blocks(update_s_kernel<float>, nu), nrhs), BLAS_THREADS, 0, strm>>>((const T*)r, (const T*)v, (T*)s, nu, st);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_update_xr_multi(cx<float>* x, const cx<float>* p, const cx<float>* s, const cx<float>* t, cx<float>* r,
                           const cx<float>* rhat, long long n, int nrhs, SolverState* st, double* part, long long pstride,
                           cudaStream_t strm, const cx<float>* sx) {
  using T = Unit<float>::T;
  const long long nu = units_of<float>(n);
  if (pstride < 3LL * blas_blocks(nu)) return OK_EINVAL;
  RedArgs ra{st, part, nullptr, FIN_XR};
  {
    TraceScope ts("update_xr_multi", strm);
    update_xr_kernel<float><<<dim3(wave_blocks(update_xr_kernel<float>, nu), nrhs), BLAS_THREADS, 0, strm>>>(
        (T*)x, (const T*)p, (const T*)s, (const T*)t, (T*)r, (const T*)rhat, nu, st, ra, pstride, (const T*)sx);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_update_p_multi(cx<float>* p, const cx<float>* r, const cx<float>* v, long long n, int nrhs, const SolverState* st,
                          cudaStream_t strm) {
  using T = Unit<float>::T;
  const long long nu = units_of<float>(n);
  {
    TraceScope ts("update_p_multi", strm);
    update_p_kernel<float><<<dim3(wave_blocks(update_p_kernel<float>, nu), nrhs), BLAS_THREADS, 0, strm>>>((T*)p, (const T*)r, (const T*)v, nu, st);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_demote(const cx<double>* r64, cx<float>* r32, cx<float>* rhat, cx<float>* p, long long n, bool restart,
                  SolverState* st, double* part, cudaStream_t strm) {
  if (restart) {
    const int nb = wave_blocks(demote_kernel<true>, n);
    RedArgs ra{st, part, nullptr, FIN_RESTART};
    {
    TraceScope ts("demote_restart", strm);
    demote_kernel<true><<<nb, BLAS_THREADS, 0, strm>>>((const double2*)r64, (float2*)r32, (float2*)rhat, (float2*)p, n, st, ra);
  }
  } else {
    const int nb = wave_blocks(demote_kernel<false>, n);
    RedArgs ra{st, part, nullptr, FIN_CONTINUE};
    {
    TraceScope ts("demote_continue", strm);
    demote_kernel<false><<<nb, BLAS_THREADS, 0, strm>>>((const double2*)r64, (float2*)r32, (float2*)rhat, (float2*)p, n, st, ra);
  }
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_accum_x(cx<double>* x64, cx<float>* x32, long long n, cudaStream_t strm) {
  {
    TraceScope ts("accum_x", strm);
    accum_x_kernel<<<wave_blocks(accum_x_kernel, n), BLAS_THREADS, 0, strm>>>((double2*)x64, (float2*)x32, n);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_to_df(const cx<double>* in, cx<dd>* out, long long n, cudaStream_t strm) {
  {
    TraceScope ts("to_df64", strm);
    to_df_kernel<<<wave_blocks(to_df_kernel, n), BLAS_THREADS, 0, strm>>>((const double2*)in, (float4*)out, n);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

int launch_norms(const cx<double>* x, const cx<double>* b, long long n, SolverState* st, double* part, cudaStream_t strm) {
  RedArgs ra{st, part, nullptr, FIN_RESID};
  {
    TraceScope ts("norms_f64", strm);
    norms_kernel<<<wave_blocks(norms_kernel, n), BLAS_THREADS, 0, strm>>>((const double2*)x, (const double2*)b, n, st, ra);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

template int launch_update_s<double>(const cx<double>*, const cx<double>*, cx<double>*, long long, const SolverState*, cudaStream_t);
template int launch_update_s<float>(const cx<float>*, const cx<float>*, cx<float>*, long long, const SolverState*, cudaStream_t);
template int launch_dots<float>(const cx<float>*, const cx<float>*, long long, bool, SolverState*, double*, cudaStream_t);
template int launch_dots<double>(const cx<double>*, const cx<double>*, long long, bool, SolverState*, double*, cudaStream_t);
template int launch_update_xr<double>(cx<double>*, const cx<double>*, const cx<double>*, const cx<double>*, cx<double>*, const cx<double>*, long long, SolverState*, double*, cudaStream_t, const cx<double>*);
template int launch_update_xr<float>(cx<float>*, const cx<float>*, const cx<float>*, const cx<float>*, cx<float>*, const cx<float>*, long long, SolverState*, double*, cudaStream_t, const cx<float>*);
template int launch_update_p<double>(cx<double>*, const cx<double>*, const cx<double>*, long long, const SolverState*, cudaStream_t);
template int launch_update_p<float>(cx<float>*, const cx<float>*, const cx<float>*, long long, const SolverState*, cudaStream_t);
template int launch_restart<double>(const cx<double>*, cx<double>*, cx<double>*, long long, SolverState*, double*, cudaStream_t);
template int launch_restart<float>(const cx<float>*, cx<float>*, cx<float>*, long long, SolverState*, double*, cudaStream_t);

}  // namespace okgb
