// Learned right preconditioner: P = L_K ... L_1 with gauge-covariant linear layers
//   (L psi)(x) = sum_d A_d (T_d psi)(x),   d in {0, +x, -x, +y, -y, +z, -z, +t, -t},
// T_0 = 1, (T_{+mu} psi)(x) = U_mu(x) psi(x + mu), (T_{-mu} psi)(x) = U_mu(x - mu)^dag psi(x - mu)
// (the link transport of the hopping terms of Eq. minFlopForm, with the fermion boundary sign),
// and A_d a learned 4 x 4 complex spin matrix shared by all sites.  P is linear in psi, so
// BiCGStab on M P y = b (x = P y) keeps a fixed operator; it is gauge covariant because only the
// links move colour.
//
// Kernels (FP32 fields, FP32 weights, FP32 links from the handle's OK_W_LINKS copy in the
// site-blocked layout of W):
//   layer:    one thread per site, the nine offsets unrolled; weights staged in shared memory.
//             The adjoint layer L^dag = sum_d A_d^dag T_{-d} is the same kernel with the offsets
//             reversed and the weights conjugate-transposed.
//   gradient: dloss/dA_{l,d} = 2 sum_{x, colour} g_l(x) (T_d psi_{l-1})(x)^dag, per-thread sums
//             over a grid-stride range of sites, a fixed-order block tree in FP64 and a one-block
//             final sum over the blocks (deterministic).
//   loss:     |P b - x|^2 / |x|^2 per pair with the seed g_K = (P b - x) / |x|^2.
//   Adam:     on the real and imaginary parts of every A entry.
#include "ok_net.cuh"
#include "ok_pair.cuh"

#include <cmath>
#include <cstring>
#include <vector>

struct ok_net {
  int layers = 0;
  float2* A = nullptr;      // [layers][9][4][4]
  float* m = nullptr;       // Adam moments, [layers * 288]
  float* v = nullptr;
  double* gacc = nullptr;   // gradient accumulator [layers * 288]
  double* scal = nullptr;   // [0..1] loss sums of the current pair, [2] loss accumulator
  unsigned* ticket = nullptr;
  long long adam_t = 0;
  int V = 0;                // volume the workspace is sized for
  int device = 0;
  okgb::cx<float>* acts = nullptr;  // [layers][V * 12], training only
  okgb::cx<float>* g[2] = {nullptr, nullptr};
  double* part = nullptr;     // [blocks][9][32]
  int part_blocks = 0;
};

namespace okgb {

namespace {

constexpr int NET_THREADS = 128;
constexpr int NOFF = 9;
constexpr int NPAR = NOFF * 32;  // real parameters per layer

// (direction, step) of offset d; direction -1 is the on-site term.
__host__ __device__ constexpr int off_mu(int d) { return d == 0 ? -1 : (d - 1) / 2; }
__host__ __device__ constexpr int off_step(int d) { return d == 0 ? 0 : ((d - 1) % 2 == 0 ? 1 : -1); }

__device__ __forceinline__ int neighbour(const int (&c)[4], const Geom& g, int mu, int step, bool& neg) {
  int cc[4] = {c[0], c[1], c[2], c[3]};
  int v = cc[mu] + step;
  neg = false;
  if (v < 0) { v += g.L[mu]; neg = (g.bcneg >> mu) & 1; }
  else if (v >= g.L[mu]) { v -= g.L[mu]; neg = (g.bcneg >> mu) & 1; }
  cc[mu] = v;
  return cc[0] + g.L[0] * (cc[1] + g.L[1] * (cc[2] + g.L[2] * cc[3]));
}

__device__ __forceinline__ void site_coords(int s, const Geom& g, int (&c)[4]) {
  int r = s;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
}

__device__ __forceinline__ void load_sp(const cx<float>* __restrict__ p, int site, cx<float> (&v)[4][3]) {
  const float4* q = reinterpret_cast<const float4*>(p) + (size_t)site * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float4 d = __ldg(q + k);
    v[(2 * k) / 3][(2 * k) % 3] = mk<float>(d.x, d.y);
    v[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk<float>(d.z, d.w);
  }
}

// U_mu(site) from the site-blocked FP32 link copy (element e of the 32 sites of a block is one
// contiguous row).
__device__ __forceinline__ void link(const cx<float>* __restrict__ L, int site, int mu, M3<float>& U) {
  const float2* q = reinterpret_cast<const float2*>(L) + ((size_t)(site >> 5) * 4 + mu) * 9 * LANES + (site & 31);
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    const float2 d = __ldg(q + e * LANES);
    U.e[e] = mk<float>(d.x, d.y);
  }
}

// w = (T psi)(x) for the transport of offset d (reversed when REV).
template <bool REV>
__device__ __forceinline__ void transported(const cx<float>* __restrict__ L, const cx<float>* __restrict__ in, int x,
                                            const int (&c)[4], const Geom& g, int d, cx<float> (&w)[4][3]) {
  const int mu = off_mu(d);
  if (mu < 0) { load_sp(in, x, w); return; }
  const int step = REV ? -off_step(d) : off_step(d);
  bool neg;
  const int n = neighbour(c, g, mu, step, neg);
  cx<float> v[4][3];
  load_sp(in, n, v);
  M3<float> U;
  link(L, step > 0 ? x : n, mu, U);
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    if (step > 0) mv(w[s], U, v[s]);
    else mdv(w[s], U, v[s]);
    if (neg)
#pragma unroll
      for (int a = 0; a < 3; ++a) w[s][a] = -w[s][a];
  }
}

// out = sum_d A_d T_d in   (ADJ: sum_d A_d^dag T_{-d} in, the adjoint layer).  With nrhs fields
// [nrhs][V][12] per launch, block b works on field b % nrhs and site block b / nrhs, so the blocks
// that read the same links run back to back and share them through L2.  With `halt` non-null and
// nonzero at launch the kernel does nothing.
template <bool ADJ>
__global__ void __launch_bounds__(NET_THREADS) net_layer_kernel(const cx<float>* __restrict__ L, const float2* __restrict__ A,
                                                                const cx<float>* __restrict__ in, cx<float>* __restrict__ out,
                                                                Geom g, int nrhs, const int* __restrict__ halt) {
  if (halt && *halt) return;  // a halted solver state: this layer belongs to an iteration that does nothing
  const int rhs = blockIdx.x % nrhs, sb = blockIdx.x / nrhs;
  in += (size_t)rhs * 12 * g.V;
  out += (size_t)rhs * 12 * g.V;
  // Each weight a is kept as (a.re, a.re, -a.im, a.im), so that a w adds to (re, im) as two
  // packed FP32 multiply-adds: (a.re, a.re) * (w.re, w.im) + (-a.im, a.im) * (w.im, w.re).
  __shared__ float4 sA[NOFF * 16];
  for (int i = threadIdx.x; i < NOFF * 16; i += NET_THREADS) {
    float2 a;
    if (!ADJ) {
      a = A[i];
    } else {
      const int d = i / 16, s = (i % 16) / 4, t = i % 4;
      const float2 b = A[d * 16 + t * 4 + s];
      a = make_float2(b.x, -b.y);
    }
    sA[i] = make_float4(a.x, a.x, -a.y, a.y);
  }
  __syncthreads();
  const int x = sb * NET_THREADS + threadIdx.x;
  if (x >= g.V) return;
  int c[4];
  site_coords(x, g, c);
  float2 acc[4][3];
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) acc[s][a] = make_float2(0.f, 0.f);
#pragma unroll
  for (int d = 0; d < NOFF; ++d) {
    cx<float> w[4][3];
    transported<ADJ>(L, in, x, c, g, d, w);
    float2 wv[4][3], ws[4][3];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        wv[t][k] = make_float2(w[t][k].re, w[t][k].im);
        ws[t][k] = make_float2(w[t][k].im, w[t][k].re);
      }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float4 a4 = sA[d * 16 + s * 4 + t];
        const float2 ar = make_float2(a4.x, a4.y), ai = make_float2(a4.z, a4.w);
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[s][k] = __ffma2_rn(ai, ws[t][k], __ffma2_rn(ar, wv[t][k], acc[s][k]));
      }
  }
  float4* q = reinterpret_cast<float4*>(out) + (size_t)x * 6;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 u = acc[(2 * k) / 3][(2 * k) % 3];
    const float2 v = acc[(2 * k + 1) / 3][(2 * k + 1) % 3];
    q[k] = make_float4(u.x, u.y, v.x, v.y);
  }
}

// Per block: for every offset d, sum over this block's sites of g(x)_s,c conj((T_d in)(x)_t,c)
// (16 complex = 32 values) -> part[block][d][32] in FP64.
__global__ void __launch_bounds__(NET_THREADS) net_grad_kernel(const cx<float>* __restrict__ L, const cx<float>* __restrict__ gr,
                                                               const cx<float>* __restrict__ in, Geom g,
                                                               double* __restrict__ part) {
  __shared__ double sh[NET_THREADS / 32][32];
  for (int d = 0; d < NOFF; ++d) {
    float C[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) C[k] = 0.f;
    for (int x = blockIdx.x * NET_THREADS + threadIdx.x; x < g.V; x += gridDim.x * NET_THREADS) {
      int c[4];
      site_coords(x, g, c);
      cx<float> gv[4][3], w[4][3];
      load_sp(gr, x, gv);
      transported<false>(L, in, x, c, g, d, w);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          cx<float> z = mk<float>(C[2 * (4 * s + t)], C[2 * (4 * s + t) + 1]);
#pragma unroll
          for (int a = 0; a < 3; ++a) z = fma_cj(w[t][a], gv[s][a], z);  // g conj(w)
          C[2 * (4 * s + t)] = z.re;
          C[2 * (4 * s + t) + 1] = z.im;
        }
    }
    // fixed-order block tree: warp shuffles, then the warps in order
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      double v = C[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = 0.0;
      for (int w = 0; w < NET_THREADS / 32; ++w) v += sh[w][threadIdx.x];
      part[((size_t)blockIdx.x * NOFF + d) * 32 + threadIdx.x] = v;
    }
    __syncthreads();
  }
}

// gacc[i] += 2 sum_b part[b][i] (one block, blocks in order).
__global__ void net_grad_final_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ gacc) {
  for (int i = threadIdx.x; i < NPAR; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * NPAR + i];
    gacc[i] += 2.0 * s;
  }
}

// |x|^2 and |out - x|^2 -> scal[0], scal[1]
__global__ void __launch_bounds__(256) net_loss_kernel(const float2* __restrict__ out, const float2* __restrict__ x, long long n,
                                                       double* part, double* scal, unsigned* ticket) {
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float2 a = out[i], b = x[i];
    const double er = (double)a.x - b.x, ei = (double)a.y - b.y;
    v[0] += (double)b.x * b.x + (double)b.y * b.y;
    v[1] += er * er + ei * ei;
  }
  const RedArgs ra{nullptr, part, scal, FIN_NONE};
  grid_reduce<2, 256>(v, ra, ticket);
}

// g = (out - x) / |x|^2; block 0 adds this pair's loss to scal[2].
__global__ void __launch_bounds__(256) net_seed_kernel(const float2* __restrict__ out, const float2* __restrict__ x, float2* g,
                                                       long long n, double* scal) {
  const double n2 = scal[0];
  const float inv = n2 > 0.0 ? (float)(1.0 / n2) : 0.f;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float2 a = out[i], b = x[i];
    g[i] = make_float2((a.x - b.x) * inv, (a.y - b.y) * inv);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[2] += n2 > 0.0 ? scal[1] / n2 : 0.0;
}

__global__ void net_adam_kernel(float* P, float* m, float* v, const double* gacc, int n, double scale, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gr = (float)(gacc[i] * scale);
  m[i] = b1 * m[i] + (1.f - b1) * gr;
  v[i] = b2 * v[i] + (1.f - b2) * gr * gr;
  const float mh = m[i] / c1, vh = v[i] / c2;
  P[i] -= lr * mh / (sqrtf(vh) + eps);
}

int net_blocks(int V) {
  const int need = grid_for(V, NET_THREADS);
  const int cap = sm_count() * 4;
  return need < cap ? need : cap;
}

// Scratch for a lattice of V sites: two fields (the layer ping-pong and the backward gradients),
// the reduction partials, and, for training, the activations of every layer.
int ensure_workspace(ok_net* N, int V, bool training) {
  if (N->V == V && N->g[0] && (!training || N->acts)) return OK_SUCCESS;
  const size_t n = (size_t)V * 12;
  if (N->V != V) {
    if (N->acts) cudaFree(N->acts);
    if (N->g[0]) cudaFree(N->g[0]);
    if (N->g[1]) cudaFree(N->g[1]);
    if (N->part) cudaFree(N->part);
    N->acts = nullptr; N->g[0] = N->g[1] = nullptr; N->part = nullptr; N->V = 0;
    OK_CUDA_TRY(cudaMalloc(&N->g[0], n * sizeof(cx<float>)));
    OK_CUDA_TRY(cudaMalloc(&N->g[1], n * sizeof(cx<float>)));
    N->part_blocks = net_blocks(V);
    const int lb = grid_for((long long)n, 256) < 1024 ? grid_for((long long)n, 256) : 1024;
    size_t pn = (size_t)N->part_blocks * NPAR;
    if ((size_t)lb * 2 > pn) pn = (size_t)lb * 2;
    OK_CUDA_TRY(cudaMalloc(&N->part, pn * sizeof(double)));
    N->V = V;
  }
  if (training && !N->acts) OK_CUDA_TRY(cudaMalloc(&N->acts, (size_t)N->layers * n * sizeof(cx<float>)));
  return OK_SUCCESS;
}

int layer(const ok_net* N, const ok_W* W, int l, bool adj, const cx<float>* in, cx<float>* out, cudaStream_t st,
          int nrhs = 1, const int* halt = nullptr) {
  const Geom& g = W->g;
  const long long nb = (long long)grid_for(g.V, NET_THREADS) * nrhs;
  if (nb > 0x7fffffffLL) return OK_EINVAL;
  {
    TraceScope ts(adj ? "net_layer_adj" : "net_layer", st);
    if (adj)
      net_layer_kernel<true><<<(unsigned)nb, NET_THREADS, 0, st>>>((const cx<float>*)W->L32, N->A + (size_t)l * 144, in, out, g, nrhs, halt);
    else
      net_layer_kernel<false><<<(unsigned)nb, NET_THREADS, 0, st>>>((const cx<float>*)W->L32, N->A + (size_t)l * 144, in, out, g, nrhs, halt);
  }
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

#define NET_TRY(expr)                       \
  do {                                      \
    int _rc = (expr);                       \
    if (_rc != OK_SUCCESS) return _rc;      \
  } while (0)

// The gradient of one pair added into gacc (and its loss into scal[2]).
int pair_backprop(ok_net* N, const ok_W* W, const cx<float>* b, const cx<float>* x, cudaStream_t st) {
  const Geom& g = W->g;
  const long long n = 12LL * g.V;
  const int K = N->layers;
  const cx<float>* in = b;
  for (int l = 0; l < K; ++l) {
    cx<float>* o = N->acts + (size_t)l * n;
    NET_TRY(layer(N, W, l, false, in, o, st));
    in = o;
  }
  const int lb = grid_for(n, 256) < 1024 ? grid_for(n, 256) : 1024;
  {
    TraceScope ts("net_loss", st);
    net_loss_kernel<<<lb, 256, 0, st>>>((const float2*)in, (const float2*)x, n, N->part, N->scal, N->ticket);
  }
  OK_LAUNCH_CHECK();
  {
    TraceScope ts("net_seed", st);
    net_seed_kernel<<<lb, 256, 0, st>>>((const float2*)in, (const float2*)x, (float2*)N->g[0], n, N->scal);
  }
  OK_LAUNCH_CHECK();
  int cur = 0;
  for (int l = K - 1; l >= 0; --l) {
    const cx<float>* lin = l == 0 ? b : N->acts + (size_t)(l - 1) * n;
    {
      TraceScope ts("net_grad", st);
      net_grad_kernel<<<N->part_blocks, NET_THREADS, 0, st>>>((const cx<float>*)W->L32, N->g[cur], lin, g, N->part);
    }
    OK_LAUNCH_CHECK();
    {
      TraceScope ts("net_grad_final", st);
      net_grad_final_kernel<<<1, 288, 0, st>>>(N->part, N->part_blocks, N->gacc + (size_t)l * NPAR);
    }
    OK_LAUNCH_CHECK();
    if (l > 0) {
      NET_TRY(layer(N, W, l, true, N->g[cur], N->g[1 - cur], st));
      cur = 1 - cur;
    }
  }
  return OK_SUCCESS;
}

int check(const ok_net* N, const ok_W* W) {
  if (!N || !W || !W->L32 || N->layers < 1) return OK_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != N->device || dev != W->device) return OK_EINVAL;
  return OK_SUCCESS;
}

}  // namespace

int net_apply_unless_halted(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, const int* halt,
                           cudaStream_t st) {
  NET_TRY(check(N, W));
  NET_TRY(ensure_workspace(N, W->g.V, false));
  const cx<float>* cur = in;
  for (int l = 0; l < N->layers; ++l) {
    cx<float>* o = l == N->layers - 1 ? out : N->g[l % 2];  // ping-pong through the workspace
    NET_TRY(layer(N, W, l, false, cur, o, st, 1, halt));
    cur = o;
  }
  return OK_SUCCESS;
}

int net_apply(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, cudaStream_t st) {
  return net_apply_unless_halted(N, W, in, out, nullptr, st);
}

// out_k = P in_k for nrhs fields [nrhs][V][12] in one launch per layer, through the caller's two
// scratch fields of the same size.
int net_apply_multi(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, int nrhs, cx<float>* tmp0, cx<float>* tmp1,
                    cudaStream_t st) {
  NET_TRY(check(N, W));
  if (nrhs < 1 || nrhs > 65535 || !tmp0 || !tmp1) return OK_EINVAL;
  cx<float>* tmp[2] = {tmp0, tmp1};
  const cx<float>* cur = in;
  for (int l = 0; l < N->layers; ++l) {
    cx<float>* o = l == N->layers - 1 ? out : tmp[l % 2];
    NET_TRY(layer(N, W, l, false, cur, o, st, nrhs));
    cur = o;
  }
  return OK_SUCCESS;
}

int net_loss_grad(ok_net* N, const ok_W* W, const cx<float>* b, const cx<float>* x, double* loss, double* grad, cudaStream_t st) {
  NET_TRY(check(N, W));
  NET_TRY(ensure_workspace(N, W->g.V, true));
  OK_CUDA_TRY(cudaMemsetAsync(N->gacc, 0, sizeof(double) * NPAR * N->layers, st));
  OK_CUDA_TRY(cudaMemsetAsync(N->scal, 0, sizeof(double) * 4, st));
  NET_TRY(pair_backprop(N, W, b, x, st));
  double s[4];
  OK_CUDA_TRY(cudaMemcpyAsync(s, N->scal, sizeof(s), cudaMemcpyDeviceToHost, st));
  if (grad) OK_CUDA_TRY(cudaMemcpyAsync(grad, N->gacc, sizeof(double) * NPAR * N->layers, cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = s[2];
  return OK_SUCCESS;
}

int net_train_step(ok_net* N, const ok_W* W, int nb, const cx<float>* b, const cx<float>* x, double lr, double* loss,
                   cudaStream_t st) {
  NET_TRY(check(N, W));
  if (nb < 1 || !b || !x || !(lr > 0.0)) return OK_EINVAL;
  NET_TRY(ensure_workspace(N, W->g.V, true));
  const long long n = 12LL * W->g.V;
  OK_CUDA_TRY(cudaMemsetAsync(N->gacc, 0, sizeof(double) * NPAR * N->layers, st));
  OK_CUDA_TRY(cudaMemsetAsync(N->scal, 0, sizeof(double) * 4, st));
  for (int i = 0; i < nb; ++i) NET_TRY(pair_backprop(N, W, b + (size_t)i * n, x + (size_t)i * n, st));
  N->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)N->adam_t), c2 = 1.f - powf(b2, (float)N->adam_t);
  const int np = NPAR * N->layers;
  {
    TraceScope ts("net_adam", st);
    net_adam_kernel<<<grid_for(np, 256), 256, 0, st>>>((float*)N->A, N->m, N->v, N->gacc, np, 1.0 / nb, (float)lr, b1, b2, 1e-8f,
                                                        c1, c2);
  }
  OK_LAUNCH_CHECK();
  double s[4];
  OK_CUDA_TRY(cudaMemcpyAsync(s, N->scal, sizeof(s), cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  if (loss) *loss = s[2] / nb;
  return OK_SUCCESS;
}

int net_create(int layers, const double* w, ok_net** out) {
  if (!out || layers < 1 || layers > 16) return OK_EINVAL;
  *out = nullptr;
  ok_net* N = new (std::nothrow) ok_net();
  if (!N) return OK_ENOMEM;
  N->layers = layers;
  auto fail = [&](int rc) {
    cudaFree(N->A); cudaFree(N->m); cudaFree(N->v); cudaFree(N->gacc); cudaFree(N->scal); cudaFree(N->ticket);
    delete N;
    return rc;
  };
  if (cudaGetDevice(&N->device) != cudaSuccess) return fail(OK_ECUDA);
  const size_t np = (size_t)NPAR * layers;
  if (cudaMalloc(&N->A, np * sizeof(float)) != cudaSuccess || cudaMalloc(&N->m, np * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&N->v, np * sizeof(float)) != cudaSuccess || cudaMalloc(&N->gacc, np * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&N->scal, 4 * sizeof(double)) != cudaSuccess || cudaMalloc(&N->ticket, sizeof(unsigned)) != cudaSuccess)
    return fail(OK_ENOMEM);
  if (cudaMemset(N->m, 0, np * sizeof(float)) != cudaSuccess || cudaMemset(N->v, 0, np * sizeof(float)) != cudaSuccess ||
      cudaMemset(N->ticket, 0, sizeof(unsigned)) != cudaSuccess)
    return fail(OK_ECUDA);
  std::vector<float> h(np, 0.f);
  for (size_t i = 0; i < np; ++i) h[i] = w ? (float)w[i] : 0.f;
  if (!w)
    for (int l = 0; l < layers; ++l)
      for (int s = 0; s < 4; ++s) h[(size_t)l * NPAR + 2 * (4 * s + s)] = 1.f;  // A_0 = 1: P = identity
  if (cudaMemcpy(N->A, h.data(), np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return fail(OK_ECUDA);
  *out = N;
  return OK_SUCCESS;
}

void net_free(ok_net* N) {
  if (!N) return;
  cudaFree(N->A); cudaFree(N->m); cudaFree(N->v); cudaFree(N->gacc); cudaFree(N->scal); cudaFree(N->ticket);
  cudaFree(N->acts); cudaFree(N->g[0]); cudaFree(N->g[1]); cudaFree(N->part);
  delete N;
}

int net_weights(ok_net* N, double* get, const double* set) {
  if (!N) return OK_EINVAL;
  const size_t np = (size_t)NPAR * N->layers;
  std::vector<float> h(np);
  if (set) {
    for (size_t i = 0; i < np; ++i) {
      if (!std::isfinite(set[i])) return OK_EINVAL;
      h[i] = (float)set[i];
    }
    OK_CUDA_TRY(cudaMemcpy(N->A, h.data(), np * sizeof(float), cudaMemcpyHostToDevice));
    OK_CUDA_TRY(cudaMemset(N->m, 0, np * sizeof(float)));
    OK_CUDA_TRY(cudaMemset(N->v, 0, np * sizeof(float)));
    N->adam_t = 0;
  }
  if (get) {
    OK_CUDA_TRY(cudaMemcpy(h.data(), N->A, np * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < np; ++i) get[i] = h[i];
  }
  return OK_SUCCESS;
}

int net_layers(const ok_net* N) { return N ? N->layers : 0; }

}  // namespace okgb
