// BiCGStab driver (the paper's bi-stabilized CG, Sec. 2.3; van der Vorst 1992) on one stream.
//
// One iteration is five kernels whose scalars live on the device:
//   v = M p            (apply, fused <rhat, v>       -> alpha = rho / <rhat, v>)
//   s = r - alpha v
//   t = M s            (apply, fused <t, s>, <t, t>  -> omega)
//   x += alpha p + omega s,  r = s - omega t  (fused <rhat, r>, <r, r> -> beta, convergence)
//   p = r + beta (p - omega v)
// The host enqueues `check_every` iterations at a time and then reads the state once; kernels
// enqueued after the state halted do nothing.
//
// Plain mode: everything FP64.  On convergence of the iterated residual, the true residual
// b - M x is recomputed; if it is still above tol the method restarts from it (also after a
// breakdown), at most max_restarts times.
//
// Mixed mode: the iteration runs in FP32 on the FP32 copy of W with its own solution increment
// x32; x and the true residual stay FP64.  When the FP32 residual has dropped by delta against its
// maximum since the last update (or reaches tol), a reliable update folds x32 into x, recomputes
// r = b - M x with the FP64 W (the true residual) and continues from it with the same search
// direction (Sleijpen and van der Vorst, "Reliable updated residuals in hybrid Bi-CG methods",
// Computing 56 (1996) 141).  The iteration stops when the FP64 true residual is below tol.
#include "ok_launch.cuh"

#include <chrono>
#include <cstring>

namespace okgb {

namespace {

struct Workspace {
  cudaStream_t st = nullptr;
  void* mem[12] = {};
  int n = 0;
  ~Workspace() {
    for (int k = 0; k < n; ++k)
      if (mem[k]) cudaFreeAsync(mem[k], st);
  }
  template <typename T> T* get(size_t count, cudaError_t* err) {
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), st);
    if (e != cudaSuccess) { *err = e; return nullptr; }
    mem[n++] = p;
    return (T*)p;
  }
};

struct HostState {
  SolverState* h = nullptr;
  HostState() { if (cudaMallocHost((void**)&h, sizeof(SolverState)) != cudaSuccess) h = nullptr; }
  ~HostState() { if (h) cudaFreeHost(h); }
};

int read_state(SolverState* d, SolverState* h, cudaStream_t st) {
  OK_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  return OK_SUCCESS;
}

// Fields the host sets between phases.
int write_state(SolverState* d, const SolverState* h, cudaStream_t st) {
  OK_CUDA_TRY(cudaMemcpyAsync(d, h, sizeof(SolverState), cudaMemcpyHostToDevice, st));
  return OK_SUCCESS;
}

#define OK_TRY(expr)            \
  do {                          \
    int _rc = (expr);           \
    if (_rc != OK_SUCCESS) return _rc; \
  } while (0)

template <typename R>
struct IterBufs {
  cx<R>* x; cx<R>* r; cx<R>* rhat; cx<R>* p; cx<R>* v; cx<R>* s; cx<R>* t;
};

// One application of M inside the iteration: with the half-precision W copy when `w16` is set
// (FP32 fields and arithmetic), else with the copy of the iteration's precision.
template <typename R>
int apply_iter(const ok_W* W, const cx<R>* psi, cx<R>* out, int epi, const EpiArgs<R>& ep, bool w16, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (w16) return launch_apply_w16(W, psi, out, epi, ep, st);
  }
  return launch_apply<R>(W, psi, out, epi, ep, st);
}

template <typename R>
int iterate(const ok_W* W, const IterBufs<R>& b, long long n, SolverState* dst, double* part, bool w16, cudaStream_t st) {
  EpiArgs<R> e1{b.rhat, nullptr, RedArgs{dst, part, nullptr, FIN_ALPHA}, &dst->ticket[0], &dst->halt};
  OK_TRY(apply_iter<R>(W, b.p, b.v, EPI_DOT, e1, w16, st));
  OK_TRY(launch_update_s<R>(b.r, b.v, b.s, n, dst, st));
  EpiArgs<R> e2{nullptr, nullptr, RedArgs{dst, part, nullptr, FIN_OMEGA}, &dst->ticket[1], &dst->halt};
  OK_TRY(apply_iter<R>(W, b.s, b.t, EPI_TS, e2, w16, st));
  OK_TRY(launch_update_xr<R>(b.x, b.p, b.s, b.t, b.r, b.rhat, n, dst, part, st));
  OK_TRY(launch_update_p<R>(b.p, b.r, b.v, n, dst, st));
  return OK_SUCCESS;
}

// out = b - M x in FP64 with |out|^2 in state aux[0] and |b|^2 in state bb (and aux[1]).  With the
// native FP64 W copy when the handle has one, else with the double-float copy (x converted first
// into `xdf`, n complex double-floats of scratch).
int residual64(const ok_W* W, const cx<double>* bvec, const cx<double>* x, cx<double>* out, SolverState* dst, double* part,
               cx<dd>* xdf, cudaStream_t st) {
  if (W->W64) {
    EpiArgs<double> e{nullptr, bvec, RedArgs{dst, part, nullptr, FIN_RESID}, &dst->ticket[5], nullptr};
    return launch_apply<double>(W, x, out, EPI_RESID, e, st);
  }
  if (!W->Wdf || !xdf) return OK_EINVAL;
  OK_TRY(launch_to_df(x, xdf, 12LL * W->g.V, st));
  EpiArgs<dd> e{nullptr, reinterpret_cast<const cx<dd>*>(bvec), RedArgs{dst, part, nullptr, FIN_RESID}, &dst->ticket[5],
                nullptr};
  return launch_apply_df(W, xdf, out, EPI_RESID, e, st);
}

}  // namespace

int bicgstab(const ok_W* W, const cx<double>* bvec, cx<double>* x, const ok_solve_params* prm, ok_solve_info* info,
             cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  if (!W || !bvec || !x || !prm) return OK_EINVAL;
  if (!(prm->tol > 0.0) || prm->maxiter < 1 || prm->max_restarts < 0 || prm->check_every < 1) return OK_EINVAL;
  int mode = prm->mode;
  const bool has64 = W->W64 || W->Wdf;  // an FP64-accurate copy for the true residual
  if (mode == OK_SOLVE_AUTO) mode = (W->W32 && has64) ? OK_SOLVE_MIXED : OK_SOLVE_F64;
  if (mode != OK_SOLVE_F64 && mode != OK_SOLVE_MIXED && mode != OK_SOLVE_MIXED16) return OK_EINVAL;
  const bool w16 = mode == OK_SOLVE_MIXED16;
  if (w16) {
    if (!W->W16) return OK_EINVAL;
    mode = OK_SOLVE_MIXED;  // same algorithm; the FP32 iteration reads the half-precision W
  } else if (mode == OK_SOLVE_MIXED && !W->W32) {
    return OK_EINVAL;
  }
  if (mode == OK_SOLVE_F64 && !W->W64) return OK_EINVAL;  // the plain FP64 iteration uses native FP64
  if (!has64) return OK_EINVAL;
  if (mode == OK_SOLVE_MIXED && !(prm->delta > 0.0 && prm->delta < 1.0)) return OK_EINVAL;
  if ((const void*)bvec == (const void*)x) return OK_EINVAL;

  const long long n = 12LL * W->g.V;
  ok_solve_info inf;
  std::memset(&inf, 0, sizeof(inf));
  Workspace ws;
  ws.st = st;
  cudaError_t err = cudaSuccess;
  int maxblocks = apply_blocks_needed(W);
  int bb2 = blas_blocks(n);
  if (bb2 > maxblocks) maxblocks = bb2;
  double* part = ws.get<double>((size_t)maxblocks * 4, &err);
  SolverState* dst = ws.get<SolverState>(1, &err);
  HostState hs;
  if (!part || !dst || !hs.h) { if (err != cudaSuccess) set_cuda_error(err); return OK_ENOMEM; }
  SolverState* h = hs.h;
  std::memset(h, 0, sizeof(SolverState));
  h->tol2 = prm->tol * prm->tol;
  h->delta2 = mode == OK_SOLVE_MIXED ? prm->delta * prm->delta : 0.0;
  h->maxiter = prm->maxiter;
  OK_TRY(write_state(dst, h, st));

  IterBufs<double> b64{};
  IterBufs<float> b32{};
  cx<double>* r64 = ws.get<cx<double>>(n, &err);
  if (!r64) { set_cuda_error(err); return OK_ENOMEM; }
  cx<dd>* xdf = nullptr;
  if (!W->W64) {
    xdf = ws.get<cx<dd>>(n, &err);
    if (!xdf) { set_cuda_error(err); return OK_ENOMEM; }
  }
  if (mode == OK_SOLVE_F64) {
    b64.x = x; b64.r = r64;
    b64.rhat = ws.get<cx<double>>(n, &err); b64.p = ws.get<cx<double>>(n, &err); b64.v = ws.get<cx<double>>(n, &err);
    b64.s = ws.get<cx<double>>(n, &err); b64.t = ws.get<cx<double>>(n, &err);
    if (!b64.rhat || !b64.p || !b64.v || !b64.s || !b64.t) { set_cuda_error(err); return OK_ENOMEM; }
  } else {
    b32.x = ws.get<cx<float>>(n, &err); b32.r = ws.get<cx<float>>(n, &err); b32.rhat = ws.get<cx<float>>(n, &err);
    b32.p = ws.get<cx<float>>(n, &err); b32.v = ws.get<cx<float>>(n, &err); b32.s = ws.get<cx<float>>(n, &err);
    b32.t = ws.get<cx<float>>(n, &err);
    if (!b32.x || !b32.r || !b32.rhat || !b32.p || !b32.v || !b32.s || !b32.t) { set_cuda_error(err); return OK_ENOMEM; }
    OK_CUDA_TRY(cudaMemsetAsync(b32.x, 0, n * sizeof(cx<float>), st));
  }

  auto finish = [&](int rc, double rr_true) {
    inf.true_relres = h->bb > 0.0 ? sqrt(rr_true / h->bb) : sqrt(rr_true);
    inf.iter_relres = h->bb > 0.0 ? sqrt(h->rr / h->bb) : sqrt(h->rr);
    inf.iters = h->iter;
    inf.time_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
  };

  // r = b - M x (FP64), then start the iteration from it.  A zero initial guess (checked with one
  // pass over x and b) gives r = b without applying M.
  OK_TRY(launch_norms(x, bvec, n, dst, part, st));
  OK_TRY(read_state(dst, h, st));
  if (h->aux[0] == 0.0) {
    OK_CUDA_TRY(cudaMemcpyAsync(r64, bvec, n * sizeof(cx<double>), cudaMemcpyDeviceToDevice, st));
    h->aux[0] = h->bb;
  } else {
    OK_TRY(residual64(W, bvec, x, r64, dst, part, xdf, st));
    inf.fp64_applies++;
  }
  if (mode == OK_SOLVE_F64) OK_TRY(launch_restart<double>(r64, b64.rhat, b64.p, n, dst, part, st));
  else OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, true, dst, part, st));
  OK_TRY(read_state(dst, h, st));
  double rr_true = h->aux[0];
  if (h->halt == HALT_NONFINITE) return finish(OK_ENONFINITE, rr_true);
  if (h->bb == 0.0) {  // b = 0: the solution is x = 0
    OK_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(cx<double>), st));
    OK_CUDA_TRY(cudaStreamSynchronize(st));
    return finish(OK_SUCCESS, 0.0);
  }
  if (h->rr < h->tol2 * h->bb) return finish(OK_SUCCESS, rr_true);

  for (;;) {
    for (int k = 0; k < prm->check_every; ++k) {
      if (mode == OK_SOLVE_F64) OK_TRY(iterate<double>(W, b64, n, dst, part, false, st));
      else OK_TRY(iterate<float>(W, b32, n, dst, part, w16, st));
    }
    OK_TRY(read_state(dst, h, st));
    int halt = h->halt;
    if (halt == HALT_NONE) continue;
    if (halt == HALT_NONFINITE) return finish(OK_ENONFINITE, rr_true);
    // true residual
    if (mode == OK_SOLVE_MIXED) OK_TRY(launch_accum_x(x, b32.x, n, st));
    OK_TRY(residual64(W, bvec, x, r64, dst, part, xdf, st));
    inf.fp64_applies++;
    OK_TRY(read_state(dst, h, st));
    rr_true = h->aux[0];
    if (!isfinite(rr_true)) return finish(OK_ENONFINITE, rr_true);
    if (rr_true < h->tol2 * h->bb) return finish(OK_SUCCESS, rr_true);
    if (halt == HALT_MAXITER || h->iter >= prm->maxiter) return finish(OK_ENOCONV, rr_true);
    if (mode == OK_SOLVE_MIXED && halt == HALT_UPDATE) {
      // reliable update: continue from the FP64 residual with the same search direction
      inf.reliable_updates++;
      OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, false, dst, part, st));
      OK_TRY(launch_update_p<float>(b32.p, b32.r, b32.v, n, dst, st));
      continue;
    }
    // converged iterated residual that the true residual does not confirm, or a breakdown:
    // restart from the true residual
    if (inf.restarts >= prm->max_restarts)
      return finish(halt == HALT_BREAKDOWN ? OK_EBREAKDOWN : OK_ENOCONV, rr_true);
    inf.restarts++;
    if (mode == OK_SOLVE_F64) OK_TRY(launch_restart<double>(r64, b64.rhat, b64.p, n, dst, part, st));
    else OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, true, dst, part, st));
  }
}

int true_residual(const ok_W* W, const cx<double>* bvec, const cx<double>* x, double* relres, cudaStream_t st) {
  if (!W || !bvec || !x || !relres || !(W->W64 || W->Wdf)) return OK_EINVAL;
  const long long n = 12LL * W->g.V;
  Workspace ws;
  ws.st = st;
  cudaError_t err = cudaSuccess;
  double* part = ws.get<double>((size_t)apply_blocks_needed(W) * 4, &err);
  SolverState* dst = ws.get<SolverState>(1, &err);
  cx<double>* r = ws.get<cx<double>>(n, &err);
  cx<dd>* xdf = W->W64 ? nullptr : ws.get<cx<dd>>(n, &err);
  HostState hs;
  if (!part || !dst || !r || !hs.h || (!W->W64 && !xdf)) { if (err != cudaSuccess) set_cuda_error(err); return OK_ENOMEM; }
  OK_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(SolverState), st));
  OK_TRY(residual64(W, bvec, x, r, dst, part, xdf, st));
  OK_TRY(read_state(dst, hs.h, st));
  double rr = hs.h->aux[0], bb = hs.h->aux[1];
  *relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
  return OK_SUCCESS;
}

}  // namespace okgb
