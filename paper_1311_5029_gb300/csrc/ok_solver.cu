// BiCGStab driver (the paper's bi-stabilized CG, Sec. 2.3; van der Vorst 1992) on one stream.
//
// One iteration is five kernels whose scalars live on the device:
//   v = M p            (apply, fused <rhat, v>       -> alpha = rho / <rhat, v>)
//   s = r - alpha v
//   t = M s            (apply, fused <t, s>, <t, t>  -> omega)
//   x += alpha p + omega s,  r = s - omega t  (fused <rhat, r>, <r, r> -> beta, convergence)
//   p = r + beta (p - omega v)
// The host enqueues `check_every` iterations at a time and then reads the state once, with one
// more iteration enqueued behind the read; kernels enqueued after the state halted do nothing.
//
// Plain mode: everything FP64.  On convergence of the iterated residual, the true residual
// b - M x is recomputed; if it is still above tol the method restarts from it (also after a
// breakdown), at most max_restarts times.
//
// Mixed mode: the iteration runs in FP32 on the FP32 copy of W with its own solution increment
// x32; x and the true residual stay FP64.  When the FP32 residual has dropped by delta against its
// maximum since the last update (or reaches tol), a reliable update folds x32 into x, recomputes
// r = b - M x with an FP64-accurate W (the true residual: the double-float copy when the handle has
// one, else the native FP64 copy) and continues from it with the same search
// direction (Sleijpen and van der Vorst, "Reliable updated residuals in hybrid Bi-CG methods",
// Computing 56 (1996) 141).  The iteration stops when the FP64 true residual is below tol.
#include "ok_dd.cuh"
#include "ok_launch.cuh"
#include "ok_net.cuh"

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

namespace okgb {

namespace {

struct Workspace {
  static constexpr int CAP = 32;
  cudaStream_t st = nullptr;
  void* mem[CAP] = {};
  int n = 0;
  ~Workspace() {
    for (int k = 0; k < n; ++k)
      if (mem[k]) cudaFreeAsync(mem[k], st);
  }
  // Stream-ordered allocation released with the workspace; null (with *err set) on failure or
  // when the workspace's CAP buffers are taken.
  template <typename T> T* get(size_t count, cudaError_t* err) {
    if (n >= CAP) { *err = cudaErrorMemoryAllocation; return nullptr; }
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

// Right preconditioner of the FP32 iteration (null: none) and its two direction buffers.
struct Precond {
  ok_net* net = nullptr;
  cx<float>* zp = nullptr;  // P p
  cx<float>* zs = nullptr;  // P s
  const int* halt = nullptr;  // the solver state's halt flag: no network work once it is set
};

// A timing-free CUDA event owned for the scope.
struct Event {
  cudaEvent_t e = nullptr;
  ~Event() { if (e) cudaEventDestroy(e); }
  cudaError_t create() { return cudaEventCreateWithFlags(&e, cudaEventDisableTiming); }
};

// One BiCGStab iteration.  With a right preconditioner P the operator is M P:  v = M (P p),
// t = M (P s) with <t, s> taken against the unpreconditioned s, and the solution increment is
// alpha P p + omega P s, so x stays in the original variables.
template <typename R>
int iterate(const ok_W* W, const IterBufs<R>& b, long long n, SolverState* dst, double* part, bool w16, const Precond& pc,
            cudaStream_t st) {
  const cx<R>* pin = b.p;
  const cx<R>* sin = b.s;
  bool pre = false;
  if constexpr (sizeof(R) == 4) {
    if (pc.net) {
      pre = true;
      OK_TRY(net_apply_unless_halted(pc.net, W, b.p, pc.zp, pc.halt, st));
      pin = pc.zp;
    }
  }
  // FP32: plain applications, their inner products in separate passes (cheaper than the fused
  // epilogue in this kernel); FP64: the epilogue is fused (the FP64 pipe bounds that kernel).
  constexpr bool fused = sizeof(R) == 8;
  EpiArgs<R> e1{b.rhat, nullptr, RedArgs{dst, part, nullptr, FIN_ALPHA}, &dst->ticket[0], &dst->halt};
  OK_TRY(apply_iter<R>(W, pin, b.v, fused ? EPI_DOT : EPI_NONE, e1, w16, st));
  if (!fused) OK_TRY(launch_dots<R>(b.rhat, b.v, n, false, dst, part, st));
  OK_TRY(launch_update_s<R>(b.r, b.v, b.s, n, dst, st));
  if constexpr (sizeof(R) == 4) {
    if (pre) {
      OK_TRY(net_apply_unless_halted(pc.net, W, b.s, pc.zs, pc.halt, st));
      sin = pc.zs;
    }
  }
  EpiArgs<R> e2{pre ? b.s : nullptr, nullptr, RedArgs{dst, part, nullptr, FIN_OMEGA}, &dst->ticket[1], &dst->halt};
  OK_TRY(apply_iter<R>(W, sin, b.t, fused ? EPI_TS : EPI_NONE, e2, w16, st));
  if (!fused) OK_TRY(launch_dots<R>(b.t, b.s, n, true, dst, part, st));
  OK_TRY(launch_update_xr<R>(b.x, pin, b.s, b.t, b.r, b.rhat, n, dst, part, st, pre ? sin : nullptr));
  OK_TRY(launch_update_p<R>(b.p, b.r, b.v, n, dst, st));
  return OK_SUCCESS;
}

// out = b - M x in FP64 with |out|^2 in state aux[0] and |b|^2 in state bb (and aux[1]).  With the
// double-float copy when the handle has one (x converted first into `xdf`, n complex double-floats
// of scratch): on the FP32 pipes it is faster than the native FP64 copy, which is used otherwise.
int residual64(const ok_W* W, const cx<double>* bvec, const cx<double>* x, cx<double>* out, SolverState* dst, double* part,
               cx<dd>* xdf, cudaStream_t st) {
  if (W->Wdf) {
    if (!xdf) return OK_EINVAL;
    OK_TRY(launch_to_df(x, xdf, 12LL * W->g.V, st));
    EpiArgs<dd> e{nullptr, reinterpret_cast<const cx<dd>*>(bvec), RedArgs{dst, part, nullptr, FIN_RESID}, &dst->ticket[5],
                  nullptr};
    return launch_apply_dd(W, xdf, out, EPI_RESID, e, st);
  }
  if (!W->W64) return OK_EINVAL;
  EpiArgs<double> e{nullptr, bvec, RedArgs{dst, part, nullptr, FIN_RESID}, &dst->ticket[5], nullptr};
  return launch_apply<double>(W, x, out, EPI_RESID, e, st);
}

}  // namespace

namespace {

int bicgstab_impl(const ok_W* W, const cx<double>* bvec, cx<double>* x, const ok_solve_params* prm, ok_solve_info* info,
                  cudaStream_t st, ok_net* net) {
  auto t0 = std::chrono::steady_clock::now();
  if (!W || !bvec || !x || !prm) return OK_EINVAL;
  if (!(prm->tol > 0.0) || prm->maxiter < 1 || prm->max_restarts < 0 || prm->check_every < 1) return OK_EINVAL;
  int mode = prm->mode & ~OK_SOLVE_DEFECT;
  const bool defect = (prm->mode & OK_SOLVE_DEFECT) != 0;  // outer defect correction (restart at each update)
  const bool has64 = W->W64 || W->Wdf;  // an FP64-accurate copy for the true residual
  if (mode == OK_SOLVE_AUTO) mode = (W->W32 && has64) ? OK_SOLVE_MIXED : OK_SOLVE_F64;
  if (mode != OK_SOLVE_F64 && mode != OK_SOLVE_MIXED && mode != OK_SOLVE_MIXED16) return OK_EINVAL;
  if (defect && mode == OK_SOLVE_F64) return OK_EINVAL;  // defect correction needs a low-precision iteration
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
  if (net && (mode != OK_SOLVE_MIXED || !W->L32)) return OK_EINVAL;  // the network runs in the FP32 iteration

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
  if (W->Wdf) {
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
  Precond pc;
  if (net) {
    pc.net = net;
    pc.zp = ws.get<cx<float>>(n, &err);
    pc.zs = ws.get<cx<float>>(n, &err);
    pc.halt = &dst->halt;
    if (!pc.zp || !pc.zs) { set_cuda_error(err); return OK_ENOMEM; }
  }

  auto finish = [&](int rc, double rr_true) {
    cudaStreamSynchronize(st);  // the iteration enqueued ahead of the last check (it does nothing)
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

  // Blocks of check_every iterations with a state read after each.  The read overlaps one more
  // iteration, which the host enqueues before it waits for the read, so that the GPU does not idle
  // through the host's round trip; when the read shows a halt, every kernel of that iteration finds
  // the halt flag set and does nothing, and the state stays as read.
  auto enqueue = [&](int iters) -> int {
    for (int k = 0; k < iters; ++k) {
      if (mode == OK_SOLVE_F64) OK_TRY(iterate<double>(W, b64, n, dst, part, false, Precond{}, st));
      else OK_TRY(iterate<float>(W, b32, n, dst, part, w16, pc, st));
    }
    return OK_SUCCESS;
  };
  Event snap;
  OK_CUDA_TRY(snap.create());
  OK_TRY(enqueue(prm->check_every));
  for (;;) {
    OK_CUDA_TRY(cudaMemcpyAsync(h, dst, sizeof(SolverState), cudaMemcpyDeviceToHost, st));
    OK_CUDA_TRY(cudaEventRecord(snap.e, st));
    OK_TRY(enqueue(1));
    OK_CUDA_TRY(cudaEventSynchronize(snap.e));
    int halt = h->halt;
    if (halt == HALT_NONE) {
      OK_TRY(enqueue(prm->check_every - 1));
      continue;
    }
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
      inf.reliable_updates++;
      if (defect) {
        // outer defect correction: a fresh inner BiCGStab on M e = r from the FP64 residual
        OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, true, dst, part, st));
      } else {
        // reliable update: continue from the FP64 residual with the same search direction
        OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, false, dst, part, st));
        OK_TRY(launch_update_p<float>(b32.p, b32.r, b32.v, n, dst, st));
      }
      OK_TRY(enqueue(prm->check_every));
      continue;
    }
    // converged iterated residual that the true residual does not confirm, or a breakdown:
    // restart from the true residual
    if (inf.restarts >= prm->max_restarts)
      return finish(halt == HALT_BREAKDOWN ? OK_EBREAKDOWN : OK_ENOCONV, rr_true);
    inf.restarts++;
    if (mode == OK_SOLVE_F64) OK_TRY(launch_restart<double>(r64, b64.rhat, b64.p, n, dst, part, st));
    else OK_TRY(launch_demote(r64, b32.r, b32.rhat, b32.p, n, true, dst, part, st));
    OK_TRY(enqueue(prm->check_every));
  }
}

}  // namespace

int bicgstab(const ok_W* W, const cx<double>* bvec, cx<double>* x, const ok_solve_params* prm, ok_solve_info* info,
             cudaStream_t st) {
  return bicgstab_impl(W, bvec, x, prm, info, st, nullptr);
}

int bicgstab_net(const ok_W* W, ok_net* net, const cx<double>* bvec, cx<double>* x, const ok_solve_params* prm,
                 ok_solve_info* info, cudaStream_t st) {
  if (!net) return OK_EINVAL;
  return bicgstab_impl(W, bvec, x, prm, info, st, net);
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
  cx<dd>* xdf = W->Wdf ? ws.get<cx<dd>>(n, &err) : nullptr;
  HostState hs;
  if (!part || !dst || !r || !hs.h || (W->Wdf && !xdf)) { if (err != cudaSuccess) set_cuda_error(err); return OK_ENOMEM; }
  OK_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(SolverState), st));
  OK_TRY(residual64(W, bvec, x, r, dst, part, xdf, st));
  OK_TRY(read_state(dst, hs.h, st));
  double rr = hs.h->aux[0], bb = hs.h->aux[1];
  *relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
  return OK_SUCCESS;
}

// One application with the fused reduction of a BiCGStab half-iteration (inspection entry
// ok_apply_M_reduce): kind 1 = EPI_DOT (<y, M psi>), kind 2 = EPI_TS (<M psi, y>, |M psi|^2).
int apply_reduce(const ok_W* W, ok_prec prec, int kind, const void* psi, const void* y, void* out, double* sums,
                 cudaStream_t st) {
  if (!W || !psi || !y || !out || !sums || (kind != 1 && kind != 2)) return OK_EINVAL;
  if (prec != OK_F64 && prec != OK_F32 && prec != OK_F32_W16) return OK_EINVAL;
  // The one-thread-per-site FP64 kernel forms <M psi, psi> only.
  if (prec == OK_F64 && kind == 2 && y != psi) return OK_EINVAL;
  const int epi = kind == 1 ? EPI_DOT : EPI_TS;
  Workspace ws;
  ws.st = st;
  cudaError_t err = cudaSuccess;
  double* part = ws.get<double>((size_t)apply_blocks_needed(W) * 4, &err);
  SolverState* dst = ws.get<SolverState>(1, &err);
  HostState hs;
  if (!part || !dst || !hs.h) { if (err != cudaSuccess) set_cuda_error(err); return OK_ENOMEM; }
  OK_CUDA_TRY(cudaMemsetAsync(dst, 0, sizeof(SolverState), st));
  const RedArgs ra{dst, part, nullptr, FIN_NONE};
  if (prec == OK_F64) {
    EpiArgs<double> e{(const cx<double>*)y, nullptr, ra, &dst->ticket[0], nullptr};
    OK_TRY(launch_apply<double>(W, (const cx<double>*)psi, (cx<double>*)out, epi, e, st));
  } else {
    EpiArgs<float> e{(const cx<float>*)y, nullptr, ra, &dst->ticket[0], nullptr};
    if (prec == OK_F32) OK_TRY(launch_apply<float>(W, (const cx<float>*)psi, (cx<float>*)out, epi, e, st));
    else OK_TRY(launch_apply_w16(W, (const cx<float>*)psi, (cx<float>*)out, epi, e, st));
  }
  OK_TRY(read_state(dst, hs.h, st));
  for (int k = 0; k < 3; ++k) sums[k] = kind == 1 && k == 2 ? 0.0 : hs.h->aux[k];
  return OK_SUCCESS;
}

}  // namespace okgb

// ============================================================================ multi right-hand side
// nrhs systems M x_k = b_k solved together (the spin-colour sources of one propagator): the
// mixed-precision method above, run in lockstep.  Each iteration is five launches for all
// systems (the multi-RHS apply with per-system fused reductions, and the batched vector
// kernels), captured once into a CUDA graph that is replayed check_every iterations at a time.
// Every system keeps its own device state; a system that halts is skipped by the kernels while
// the host handles it (reliable update, restart or completion) and the others go on.
namespace okgb {

int bicgstab_multi(const ok_W* W, int nrhs, const cx<double>* bvec, cx<double>* x, const ok_solve_params* prm,
                   ok_solve_info* info, cudaStream_t st, ok_net* net) {
  auto t0 = std::chrono::steady_clock::now();
  if (!W || !bvec || !x || !prm || nrhs < 1 || nrhs > 64) return OK_EINVAL;
  if (!(prm->tol > 0.0) || prm->maxiter < 1 || prm->max_restarts < 0 || prm->check_every < 1) return OK_EINVAL;
  if (!(prm->delta > 0.0 && prm->delta < 1.0)) return OK_EINVAL;
  int mode = prm->mode & ~OK_SOLVE_DEFECT;
  const bool defect = (prm->mode & OK_SOLVE_DEFECT) != 0;  // outer defect correction (restart at each update)
  if (mode == OK_SOLVE_AUTO)
    mode = (W->Wtc && nrhs <= 16 && !net) ? OK_SOLVE_MIXED_TC : W->W16 ? OK_SOLVE_MIXED16 : OK_SOLVE_MIXED;
  if (mode != OK_SOLVE_MIXED && mode != OK_SOLVE_MIXED16 && mode != OK_SOLVE_MIXED_TC) return OK_EINVAL;
  // Tensor-core form: iteration vectors in the tensor-core layout (ok_tc.cu), applies on the
  // tensor cores; the network preconditioner works on the canonical layout and is not combined.
  const bool tcp = mode == OK_SOLVE_MIXED_TC;
  if (tcp && (!W->Wtc || nrhs > 16 || net)) return OK_EINVAL;
  const bool w16 = mode == OK_SOLVE_MIXED16;
  if ((w16 && !W->W16) || (!w16 && !tcp && !W->W32) || !(W->W64 || W->Wdf)) return OK_EINVAL;
  if ((const void*)bvec == (const void*)x) return OK_EINVAL;
  if (net && !W->L32) return OK_EINVAL;  // the network needs the handle's FP32 links

  // The solve runs on a private non-blocking stream ordered after the caller's stream (a CUDA
  // graph cannot be captured from the legacy default stream); on every return the caller's stream
  // is made to wait for it, after the workspace has been released on it.
  struct OwnStream {
    cudaStream_t user = nullptr, own = nullptr;
    ~OwnStream() {
      if (!own) return;
      cudaEvent_t e = nullptr;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(e, own);
        cudaStreamWaitEvent(user, e, 0);
        cudaEventDestroy(e);
      } else {
        cudaStreamSynchronize(own);
      }
      cudaStreamDestroy(own);
    }
  } os;
  os.user = st;
  {
    OK_CUDA_TRY(cudaStreamCreateWithFlags(&os.own, cudaStreamNonBlocking));
    cudaEvent_t e = nullptr;
    OK_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t e1 = cudaEventRecord(e, st);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(os.own, e, 0) : e1;
    cudaEventDestroy(e);
    OK_CUDA_TRY(e2);
    st = os.own;
  }
  const long long n = 12LL * W->g.V;
  const long long N = n * nrhs;
  Workspace ws;
  ws.st = st;
  cudaError_t err = cudaSuccess;
  long long maxblocks = mrhs_blocks_needed(W);
  if (blas_blocks(n) > maxblocks) maxblocks = blas_blocks(n);
  if (blas_blocks(n / 2) > maxblocks) maxblocks = blas_blocks(n / 2);
  if (tcp) {
    for (long long nb : {(long long)tc_blocks_needed(W), (long long)tc_vec_blocks(nrhs), (long long)blas_blocks(3LL * W->g.V)})
      if (nb > maxblocks) maxblocks = nb;
  }
  const long long pstride = 4 * maxblocks;
  double* part = ws.get<double>((size_t)pstride * nrhs, &err);
  SolverState* dst = ws.get<SolverState>(nrhs, &err);
  unsigned* tickets = tcp ? ws.get<unsigned>(4, &err) : nullptr;  // grid completion counters of the TC kernels
  // FP16 copies of p and s (scaled per system) that the tensor-core apply reads
  const size_t b16 = tcp ? tc_in16_bytes(W->g.V) : 0;
  unsigned char* p16 = tcp ? ws.get<unsigned char>(b16, &err) : nullptr;
  unsigned char* s16 = tcp ? ws.get<unsigned char>(b16, &err) : nullptr;
  if (tcp && (!tickets || !p16 || !s16)) { set_cuda_error(err); return OK_ENOMEM; }
  if (tcp) {  // absent right-hand sides stay zero; a halted system's copies stay finite
    OK_CUDA_TRY(cudaMemsetAsync(p16, 0, b16, st));
    OK_CUDA_TRY(cudaMemsetAsync(s16, 0, b16, st));
  }
  if (tcp) OK_CUDA_TRY(cudaMemsetAsync(tickets, 0, 4 * sizeof(unsigned), st));
  const int V = W->g.V;
  cx<double>* r64 = ws.get<cx<double>>(n, &err);
  cx<dd>* xdf = W->Wdf ? ws.get<cx<dd>>(n, &err) : nullptr;
  IterBufs<float> b{};
  b.x = ws.get<cx<float>>(N, &err); b.r = ws.get<cx<float>>(N, &err); b.rhat = ws.get<cx<float>>(N, &err);
  b.p = ws.get<cx<float>>(N, &err); b.v = ws.get<cx<float>>(N, &err); b.s = ws.get<cx<float>>(N, &err);
  b.t = ws.get<cx<float>>(N, &err);
  cx<float>* zp = net ? ws.get<cx<float>>(N, &err) : nullptr;  // P p and P s of every system
  cx<float>* zs = net ? ws.get<cx<float>>(N, &err) : nullptr;
  cx<float>* nt0 = net ? ws.get<cx<float>>(N, &err) : nullptr;  // the network's layer scratch
  cx<float>* nt1 = net ? ws.get<cx<float>>(N, &err) : nullptr;
  if (net && (!zp || !zs || !nt0 || !nt1)) { set_cuda_error(err); return OK_ENOMEM; }
  SolverState* h = nullptr;
  if (cudaMallocHost((void**)&h, sizeof(SolverState) * nrhs) != cudaSuccess) h = nullptr;
  struct HostFree { SolverState* p; ~HostFree() { if (p) cudaFreeHost(p); } } hf{h};
  if (!part || !dst || !r64 || (W->Wdf && !xdf) || !b.x || !b.r || !b.rhat || !b.p || !b.v || !b.s || !b.t || !h) {
    if (err != cudaSuccess) set_cuda_error(err);
    return OK_ENOMEM;
  }
  std::memset(h, 0, sizeof(SolverState) * nrhs);
  for (int k = 0; k < nrhs; ++k) {
    h[k].tol2 = prm->tol * prm->tol;
    h[k].delta2 = prm->delta * prm->delta;
    h[k].maxiter = prm->maxiter;
  }
  OK_CUDA_TRY(cudaMemcpyAsync(dst, h, sizeof(SolverState) * nrhs, cudaMemcpyHostToDevice, st));
  OK_CUDA_TRY(cudaMemsetAsync(b.x, 0, N * sizeof(cx<float>), st));

  std::vector<ok_solve_info> inf(nrhs);
  std::vector<int> status(nrhs, 1);  // 1 running, else the final return code (0 = converged)
  std::vector<double> rr_true(nrhs, 0.0);
  for (auto& i : inf) std::memset(&i, 0, sizeof(i));
  const int halt_done = HALT_CONVERGED;
  auto freeze = [&](int k) {  // keep system k out of further iterations
    return cudaMemcpyAsync(&dst[k].halt, &halt_done, sizeof(int), cudaMemcpyHostToDevice, st);
  };
  auto vec = [&](auto* base, int k) { return base + (size_t)k * n; };

  // Initial residuals, one system at a time (FP64), demoted into the FP32 iteration vectors.
  for (int k = 0; k < nrhs; ++k) {
    OK_TRY(launch_norms(vec(x, k), vec(bvec, k), n, &dst[k], part, st));
    OK_TRY(read_state(&dst[k], &h[k], st));
    const cx<double>* r0 = vec(bvec, k);
    if (h[k].aux[0] != 0.0) {
      OK_TRY(residual64(W, vec(bvec, k), vec(x, k), r64, &dst[k], part, xdf, st));
      inf[k].fp64_applies++;
      r0 = r64;
    }
    if (tcp) OK_TRY(launch_tc_demote(r0, b.r, b.rhat, b.p, V, nrhs, k, true, &dst[k], part, st));
    else OK_TRY(launch_demote(r0, vec(b.r, k), vec(b.rhat, k), vec(b.p, k), n, true, &dst[k], part, st));
  }
  if (tcp) OK_TRY(launch_tc_half(b.p, p16, V, nrhs, dst, -1, st));
  OK_CUDA_TRY(cudaMemcpyAsync(h, dst, sizeof(SolverState) * nrhs, cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < nrhs; ++k) {
    rr_true[k] = h[k].aux[0];
    if (h[k].halt == HALT_NONFINITE) status[k] = OK_ENONFINITE;
    else if (h[k].bb == 0.0) {  // b = 0: x = 0
      OK_CUDA_TRY(cudaMemsetAsync(vec(x, k), 0, n * sizeof(cx<double>), st));
      status[k] = OK_SUCCESS;
      rr_true[k] = 0.0;
    } else if (h[k].rr < h[k].tol2 * h[k].bb) status[k] = OK_SUCCESS;
    if (status[k] != 1) OK_CUDA_TRY(freeze(k));
  }

  const MultiShape shape = multi_shape(W, w16, nrhs);
  // One iteration for every system; with a right preconditioner P (one launch per network layer
  // for all systems) the operator is M P, as in iterate() above.
  auto iterate_all = [&]() -> int {
    if (tcp) {
      const TcEpi e1{(const float4*)b.rhat, dst, part, pstride, tickets + 0, FIN_ALPHA, nullptr};
      OK_TRY(launch_apply_tc(W, p16, b.v, nrhs, EPI_DOT, e1, st));
      OK_TRY(launch_tc_update_s(b.r, b.v, b.s, s16, V, nrhs, dst, st));
      const TcEpi e2{(const float4*)b.s, dst, part, pstride, tickets + 1, FIN_OMEGA, nullptr};
      OK_TRY(launch_apply_tc(W, s16, b.t, nrhs, EPI_TS, e2, st));
      OK_TRY(launch_tc_update_xr(b.x, p16, b.s, s16, b.t, b.r, b.rhat, V, nrhs, dst, part, pstride, tickets + 2, st));
      return launch_tc_update_p(b.p, p16, b.r, b.v, V, nrhs, dst, -1, st);
    }
    const cx<float>* pin = b.p;
    const cx<float>* sin = b.s;
    if (net) {
      OK_TRY(net_apply_multi(net, W, b.p, zp, nrhs, nt0, nt1, st));
      pin = zp;
    }
    MultiEpi e1{b.rhat, dst, part, pstride, FIN_ALPHA, 0};
    OK_TRY(launch_apply_multi(W, w16, pin, b.v, nrhs, EPI_DOT, e1, shape, st));
    OK_TRY(launch_update_s_multi(b.r, b.v, b.s, n, nrhs, dst, st));
    if (net) {
      OK_TRY(net_apply_multi(net, W, b.s, zs, nrhs, nt0, nt1, st));
      sin = zs;
    }
    MultiEpi e2{net ? b.s : nullptr, dst, part, pstride, FIN_OMEGA, 1};
    OK_TRY(launch_apply_multi(W, w16, sin, b.t, nrhs, EPI_TS, e2, shape, st));
    OK_TRY(launch_update_xr_multi(b.x, pin, b.s, b.t, b.r, b.rhat, n, nrhs, dst, part, pstride, st, net ? sin : nullptr));
    OK_TRY(launch_update_p_multi(b.p, b.r, b.v, n, nrhs, dst, st));
    return OK_SUCCESS;
  };

  // The first block of iterations runs with direct launches (it also initialises every kernel's
  // launch configuration); the same block is then captured once and replayed.
  cudaGraphExec_t exec = nullptr;
  struct GraphFree { cudaGraphExec_t* e; ~GraphFree() { if (*e) cudaGraphExecDestroy(*e); } } gf{&exec};
  long long graph_kernels = 0;
  bool first = true;
  int rc_final = OK_SUCCESS;
  for (;;) {
    bool running = false;
    for (int k = 0; k < nrhs; ++k) running = running || status[k] == 1;
    if (!running) break;
    if (first || !exec) {
      for (int it = 0; it < prm->check_every; ++it) OK_TRY(iterate_all());
    } else {
      TraceScope ts("bicgstab_multi_graph", st);
      OK_CUDA_TRY(cudaGraphLaunch(exec, st));
      adjust_launches(graph_kernels);
    }
    if (first) {
      first = false;
      cudaGraph_t graph = nullptr;
      const unsigned long long before = launches();
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();  // no replay: keep launching directly
      } else {
        int rc = OK_SUCCESS;
        for (int it = 0; it < prm->check_every && rc == OK_SUCCESS; ++it) rc = iterate_all();
        const cudaError_t ce = cudaStreamEndCapture(st, &graph);
        graph_kernels = (long long)(launches() - before);
        adjust_launches(-graph_kernels);  // captured, not executed
        if (rc != OK_SUCCESS || ce != cudaSuccess || !graph ||
            cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
          exec = nullptr;  // replay unavailable: keep launching directly
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
      }
    }
    OK_CUDA_TRY(cudaMemcpyAsync(h, dst, sizeof(SolverState) * nrhs, cudaMemcpyDeviceToHost, st));
    OK_CUDA_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < nrhs; ++k) {
      if (status[k] != 1) continue;
      const int halt = h[k].halt;
      if (halt == HALT_NONE) continue;
      if (halt == HALT_NONFINITE) { status[k] = OK_ENONFINITE; continue; }
      // fold the FP32 increment into x and recompute the true residual in FP64
      if (tcp) OK_TRY(launch_tc_accum(vec(x, k), b.x, V, nrhs, k, st));
      else OK_TRY(launch_accum_x(vec(x, k), vec(b.x, k), n, st));
      OK_TRY(residual64(W, vec(bvec, k), vec(x, k), r64, &dst[k], part, xdf, st));
      inf[k].fp64_applies++;
      OK_TRY(read_state(&dst[k], &h[k], st));
      rr_true[k] = h[k].aux[0];
      if (!std::isfinite(rr_true[k])) { status[k] = OK_ENONFINITE; OK_CUDA_TRY(freeze(k)); continue; }
      if (rr_true[k] < h[k].tol2 * h[k].bb) { status[k] = OK_SUCCESS; OK_CUDA_TRY(freeze(k)); continue; }
      if (halt == HALT_MAXITER || h[k].iter >= prm->maxiter) { status[k] = OK_ENOCONV; OK_CUDA_TRY(freeze(k)); continue; }
      if (halt == HALT_UPDATE) {
        inf[k].reliable_updates++;
        if (defect) {  // outer defect correction: a fresh inner BiCGStab from the FP64 residual
          if (tcp) {
            OK_TRY(launch_tc_demote(r64, b.r, b.rhat, b.p, V, nrhs, k, true, &dst[k], part, st));
            OK_TRY(launch_tc_half(b.p, p16, V, nrhs, dst, k, st));
          } else {
            OK_TRY(launch_demote(r64, vec(b.r, k), vec(b.rhat, k), vec(b.p, k), n, true, &dst[k], part, st));
          }
        } else if (tcp) {
          OK_TRY(launch_tc_demote(r64, b.r, b.rhat, b.p, V, nrhs, k, false, &dst[k], part, st));
          OK_TRY(launch_tc_update_p(b.p, p16, b.r, b.v, V, nrhs, dst, k, st));
        } else {
          OK_TRY(launch_demote(r64, vec(b.r, k), vec(b.rhat, k), vec(b.p, k), n, false, &dst[k], part, st));
          OK_TRY(launch_update_p<float>(vec(b.p, k), vec(b.r, k), vec(b.v, k), n, &dst[k], st));
        }
        continue;
      }
      if (inf[k].restarts >= prm->max_restarts) {
        status[k] = halt == HALT_BREAKDOWN ? OK_EBREAKDOWN : OK_ENOCONV;
        OK_CUDA_TRY(freeze(k));
        continue;
      }
      inf[k].restarts++;
      if (tcp) {
        OK_TRY(launch_tc_demote(r64, b.r, b.rhat, b.p, V, nrhs, k, true, &dst[k], part, st));
        OK_TRY(launch_tc_half(b.p, p16, V, nrhs, dst, k, st));
      } else {
        OK_TRY(launch_demote(r64, vec(b.r, k), vec(b.rhat, k), vec(b.p, k), n, true, &dst[k], part, st));
      }
    }
  }
  OK_CUDA_TRY(cudaMemcpyAsync(h, dst, sizeof(SolverState) * nrhs, cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int k = 0; k < nrhs; ++k) {
    inf[k].true_relres = h[k].bb > 0.0 ? sqrt(rr_true[k] / h[k].bb) : sqrt(rr_true[k]);
    inf[k].iter_relres = h[k].bb > 0.0 ? sqrt(h[k].rr / h[k].bb) : sqrt(h[k].rr);
    inf[k].iters = h[k].iter;
    inf[k].time_ms = ms;
    if (info) info[k] = inf[k];
    if (status[k] != OK_SUCCESS && rc_final == OK_SUCCESS) rc_final = status[k];
  }
  return rc_final;
}

}  // namespace okgb
