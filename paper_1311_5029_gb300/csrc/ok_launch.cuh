// Declarations of the kernel launchers shared between translation units.
#pragma once

#include "ok_reduce.cuh"

namespace okgb {

// Fused epilogues of the apply kernel.
enum : int {
  EPI_NONE = 0,   // out = M psi
  EPI_DOT = 1,    // out = M psi; reduce <rhat, out>
  EPI_TS = 2,     // out = M psi; reduce <out, psi>, <out, out>
  EPI_RESID = 3,  // out = b - M psi; reduce <out, out>, <b, b>
};

template <typename R> struct EpiArgs {
  const cx<R>* rhat;   // EPI_DOT; EPI_TS (split kernel): if set, the y of <out, y> instead of psi
  const cx<R>* b;      // EPI_RESID
  RedArgs ra;
  unsigned* ticket;
  const int* halt;     // if non-null and nonzero at launch, the kernel does nothing
};

template <typename R>
int launch_apply(const ok_W* W, const cx<R>* psi, cx<R>* out, int epi, const EpiArgs<R>& ep, cudaStream_t st);
int apply_blocks_needed(const ok_W* W);
// FP32 fields and arithmetic with the half-precision W copy (all epilogues).
int launch_apply_w16(const ok_W* W, const cx<float>* psi, cx<float>* out, int epi, const EpiArgs<float>& ep, cudaStream_t st);
// out = M psi in FP32 with every W matrix rebuilt from the handle's FP32 links and clover fields
// (OK_W_OTF) inside the apply; OK_EINVAL without them.
int launch_apply_otf(const ok_W* W, const cx<float>* psi, cx<float>* out, cudaStream_t st);
// Bounded device waits that gave up (the kernel's result is then invalid); optionally reset.
int read_wait_timeouts(unsigned* n, bool reset);
int set_stage_test_bytes(unsigned bytes);  // failure injection for the bounded waits
// Multi right-hand side apply (ok_mrhs.cu): FP32 fields [nrhs][V][12], W32 or W16 (w16).
struct MultiEpi {
  const cx<float>* rhat;  // EPI_DOT: [nrhs][V][12]; EPI_TS: if set, the y of <out, y> instead of psi
  SolverState* st;        // [nrhs]; EPI_DOT / EPI_TS reduce into st[k] (skipped while st[k].halt)
  double* part;           // partials of system k at part + k * pstride (pstride >= 3 * grid width)
  long long pstride;
  int fin;                // FIN_ALPHA (EPI_DOT) or FIN_OMEGA (EPI_TS)
  int slot;               // ticket index in each state
};
struct MultiShape {
  int nr;        // right-hand sides per thread, 1..4, dividing nrhs
  int blocks_x;  // blocks per grid row (0: as many as fit on the device)
};
int launch_apply_multi(const ok_W* W, bool w16, const cx<float>* psi, cx<float>* out, int nrhs, int epi, const MultiEpi& ep,
                       const MultiShape& shape, cudaStream_t st);
int mrhs_blocks_needed(const ok_W* W);  // upper bound of the grid width
MultiShape multi_shape(const ok_W* W, bool w16, int nrhs);  // tuned or default
// Tensor-core multi right-hand side apply (ok_tc.cu).  Fields in the tensor-core layout: float4 unit
// ((site * 2 + b) * nrhs + r) * 3 + c holds the projection h_b (b = +, -) of right-hand side r at
// colour c, spins 0 and 1; nrhs <= 16.
struct TcEpi {
  const float4* y;     // EPI_DOT: rhat (<y, out>); EPI_TS: the y of <out, y> (null: the input)
  SolverState* st;     // [nrhs]
  double* part;        // partials of right-hand side r at part + r * pstride (pstride >= 3 * grid)
  long long pstride;
  unsigned* ticket;    // grid completion counter (zero between launches)
  int fin;             // FIN_ALPHA (EPI_DOT) or FIN_OMEGA (EPI_TS)
  const float* inv_scale;  // [nrhs] 1 / sigma of the FP16 inputs; null: from each system's |r| (st)
};
int launch_tc_build(const ok_W* W, const cx<double>* W64, const WScalars* dsc, cudaStream_t st);
size_t tc_record_bytes();
int launch_tc_expand(const ok_W* W, int kind, cx<double>* out, cudaStream_t st);
int tc_blocks_needed(const ok_W* W);
int tc_vec_blocks(int nrhs);
int launch_apply_tc(const ok_W* W, const void* in16, cx<float>* out, int nrhs, int epi, const TcEpi& ep, cudaStream_t st);
// canonical complex64 [nrhs][V][4][3] -> FP16 tensor-core layout with a power-of-two scale per right-hand
// side (amax: nrhs words of scratch; inv_scale: nrhs floats out, 1 / sigma); FP32 tensor-core layout -> canonical.
size_t tc_in16_bytes(int V);  // the FP16 input layout of the tensor-core apply (1 KB per site)
int launch_to_tc16(const cx<float>* in, void* out16, int V, int nrhs, unsigned* amax, float* inv_scale, cudaStream_t st);
int launch_from_tc(const cx<float>* in, cx<float>* out, int V, int nrhs, cudaStream_t st);
int launch_tc_update_s(const cx<float>* r, const cx<float>* v, cx<float>* s, void* s16, int V, int nrhs, const SolverState* st,
                       cudaStream_t strm);
int launch_tc_update_p(cx<float>* p, void* p16, const cx<float>* r, const cx<float>* v, int V, int nrhs, const SolverState* st,
                       int only, cudaStream_t strm);
int launch_tc_half(const cx<float>* p, void* p16, int V, int nrhs, const SolverState* st, int only, cudaStream_t strm);
int launch_tc_update_xr(cx<float>* x, const void* p16, const cx<float>* s, const void* s16, const cx<float>* t, cx<float>* r,
                        const cx<float>* rhat, int V, int nrhs, SolverState* st, double* part, long long pstride,
                        unsigned* ticket, cudaStream_t strm);
int launch_tc_demote(const cx<double>* r64, cx<float>* r, cx<float>* rhat, cx<float>* p, int V, int nrhs, int k, bool restart,
                     SolverState* st, double* part, cudaStream_t strm);
int launch_tc_accum(cx<double>* x64, cx<float>* x, int V, int nrhs, int k, cudaStream_t strm);
// FP64 complex -> double-float complex (n complex numbers).
int launch_to_df(const cx<double>* in, cx<dd>* out, long long n, cudaStream_t st);

int blas_blocks(long long units);
int sm_count();  // multiprocessors of the current device (cached)
template <typename R>
int launch_update_s(const cx<R>* r, const cx<R>* v, cx<R>* s, long long n, const SolverState* st, cudaStream_t strm);
template <typename R>
int launch_update_xr(cx<R>* x, const cx<R>* p, const cx<R>* s, const cx<R>* t, cx<R>* r, const cx<R>* rhat, long long n,
                     SolverState* st, double* part, cudaStream_t strm, const cx<R>* sx = nullptr);
template <typename R>
int launch_update_p(cx<R>* p, const cx<R>* r, const cx<R>* v, long long n, const SolverState* st, cudaStream_t strm);
// <a, b> -> FIN_ALPHA (a = rhat, b = v), or with omega <a, b>, <a, a> -> FIN_OMEGA (a = t, b = s).
template <typename R>
int launch_dots(const cx<R>* a, const cx<R>* b, long long n, bool omega, SolverState* st, double* part, cudaStream_t strm);
template <typename R>
int launch_restart(const cx<R>* r, cx<R>* rhat, cx<R>* p, long long n, SolverState* st, double* part, cudaStream_t strm);
int launch_demote(const cx<double>* r64, cx<float>* r32, cx<float>* rhat, cx<float>* p, long long n, bool restart,
                  SolverState* st, double* part, cudaStream_t strm);
int launch_accum_x(cx<double>* x64, cx<float>* x32, long long n, cudaStream_t strm);
// Batched iteration kernels over nrhs systems (FP32 vectors [nrhs][n], states [nrhs]).
int launch_update_s_multi(const cx<float>* r, const cx<float>* v, cx<float>* s, long long n, int nrhs, const SolverState* st,
                          cudaStream_t strm);
int launch_update_xr_multi(cx<float>* x, const cx<float>* p, const cx<float>* s, const cx<float>* t, cx<float>* r,
                           const cx<float>* rhat, long long n, int nrhs, SolverState* st, double* part, long long pstride,
                           cudaStream_t strm, const cx<float>* sx = nullptr);
int launch_update_p_multi(cx<float>* p, const cx<float>* r, const cx<float>* v, long long n, int nrhs, const SolverState* st,
                          cudaStream_t strm);
// <x, x> and <b, b> in FP64 -> FIN_RESID (state bb = <b, b>, aux = the two sums)
int launch_norms(const cx<double>* x, const cx<double>* b, long long n, SolverState* st, double* part, cudaStream_t strm);

// ok_precompute.cu
int geom_from_lattice(const ok_lattice* lat, Geom* g);
int precompute(const ok_lattice* lat, const void* links, ok_prec links_prec, const ok_coeffs* c, int precs,
               cudaStream_t st, ok_W** W_out);
int expand(const ok_W* W, ok_prec prec, int kind, void* out, cudaStream_t st);

// ok_solver.cu
int bicgstab(const ok_W* W, const cx<double>* b, cx<double>* x, const ok_solve_params* prm, ok_solve_info* info,
             cudaStream_t st);
int true_residual(const ok_W* W, const cx<double>* b, const cx<double>* x, double* relres, cudaStream_t st);
int apply_reduce(const ok_W* W, ok_prec prec, int kind, const void* psi, const void* y, void* out, double* sums,
                 cudaStream_t st);
int bicgstab_multi(const ok_W* W, int nrhs, const cx<double>* b, cx<double>* x, const ok_solve_params* prm, ok_solve_info* info,
                   cudaStream_t st, ok_net* net = nullptr);

// ok_net.cu (learned right preconditioner)
int net_create(int layers, const double* w, ok_net** out);
void net_free(ok_net* N);
int net_weights(ok_net* N, double* get, const double* set);
int net_layers(const ok_net* N);
int net_apply(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, cudaStream_t st);
int net_apply_multi(ok_net* N, const ok_W* W, const cx<float>* in, cx<float>* out, int nrhs, cx<float>* tmp0, cx<float>* tmp1,
                    cudaStream_t st);
int net_loss_grad(ok_net* N, const ok_W* W, const cx<float>* b, const cx<float>* x, double* loss, double* grad, cudaStream_t st);
int net_train_step(ok_net* N, const ok_W* W, int nb, const cx<float>* b, const cx<float>* x, double lr, double* loss,
                   cudaStream_t st);
int bicgstab_net(const ok_W* W, ok_net* net, const cx<double>* b, cx<double>* x, const ok_solve_params* prm,
                 ok_solve_info* info, cudaStream_t st);

// ok_tune.cu
int autotune(ok_W* W, ok_prec prec, int nrhs, int* choice, double* best_us, cudaStream_t st);

}  // namespace okgb
