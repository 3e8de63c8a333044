// The extern "C" boundary declared in include/ok.h: argument checks, error codes, launch count.
#include "ok_dd.cuh"
#include "ok_launch.cuh"

#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace okgb {

static std::atomic<unsigned long long> g_launches{0};
static thread_local int g_last_cuda_error = 0;

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void adjust_launches(long long n) {
  if (n >= 0) g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
  else g_launches.fetch_sub((unsigned long long)(-n), std::memory_order_relaxed);
}

// ---------------------------------------------------------------------------- tracing
namespace {
struct TraceRec {
  const char* name;
  cudaEvent_t a, b;
};
struct TraceTotals {
  unsigned long long launches = 0;
  double ms = 0.0;
};
std::atomic<int> g_trace_on{0};
std::mutex g_trace_mu;
std::vector<TraceRec> g_pending;
std::vector<cudaEvent_t> g_event_pool;
std::map<std::string, TraceTotals> g_totals;

cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

// The scope holds its own two events and hands the finished record to g_pending only in the
// destructor, so a drain (ok_trace_read / ok_trace_reset) that runs between the two calls on another
// thread neither loses the record nor sees one whose end event was never recorded.
TraceScope::TraceScope(const char* n, cudaStream_t s) : name(n), st(s), a(nullptr), b(nullptr) {
  if (!g_trace_on.load(std::memory_order_relaxed)) return;
  // Kernels recorded into a CUDA graph are not timed one by one (the graph launch is).
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  cudaEvent_t ea = take_event();
  if (!ea) return;
  cudaEvent_t eb = take_event();
  if (!eb || cudaEventRecord(ea, s) != cudaSuccess) {
    g_event_pool.push_back(ea);  // nothing is timed: both events go back to the pool
    if (eb) g_event_pool.push_back(eb);
    return;
  }
  a = ea;
  b = eb;
}

TraceScope::~TraceScope() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (cudaEventRecord(b, st) == cudaSuccess) {
    g_pending.push_back(TraceRec{name, a, b});
  } else {
    g_event_pool.push_back(a);
    g_event_pool.push_back(b);
  }
}
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }
void set_cuda_error(cudaError_t e) { g_last_cuda_error = (int)e; }

static bool coeffs_finite(const ok_coeffs* c) {
  const double v[] = {c->u0, c->am0, c->kappa, c->zeta, c->r_s, c->c_B, c->c_E, c->c_EE, c->c1, c->c2, c->c3, c->c4, c->c5};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

}  // namespace okgb

using namespace okgb;

extern "C" {

int ok_precompute_W(const ok_lattice* lat, const void* links, ok_prec links_prec, const ok_coeffs* coeffs, int W_precs,
                    void* stream, ok_W** W_out) {
  if (!coeffs || !okgb::coeffs_finite(coeffs)) return OK_EINVAL;
  return precompute(lat, links, links_prec, coeffs, W_precs, (cudaStream_t)stream, W_out);
}

void ok_free_W(ok_W* W) {
  if (!W) return;
  // Returned to the stream-ordered pool they came from, after the work already queued on the
  // legacy default stream (the caller guarantees that no work on the handle is pending).
  for (void* q : {W->W64, W->W32, W->Wdf, W->W16, W->L32, W->Wtc, W->EB32})
    if (q) cudaFreeAsync(q, 0);
  delete W;
}

double ok_W_u0(const ok_W* W) { return W ? W->sc.u0 : NAN; }

double ok_W_plaquette(const ok_W* W) { return W ? W->sc.plaq : NAN; }

int ok_W_info(const ok_W* W, ok_lattice* lat, int* W_precs, size_t* bytes) {
  if (!W) return OK_EINVAL;
  if (lat) *lat = W->lat;
  if (W_precs) *W_precs = W->precs;
  if (bytes) *bytes = W->bytes;
  return OK_SUCCESS;
}

int ok_apply_M(const ok_W* W, ok_prec prec, const void* psi, void* out, void* stream) {
  if (!W || !psi || !out) return OK_EINVAL;
  size_t es = prec == OK_F64 ? 16 : (prec == OK_F32 || prec == OK_F32_W16 || prec == OK_F32_OTF) ? 8 : 0;
  if (es == 0) return OK_EINVAL;
  size_t bytes = (size_t)W->g.V * 12 * es;
  const char* a = (const char*)psi;
  const char* b = (const char*)out;
  if (a < b + bytes && b < a + bytes) return OK_EINVAL;  // overlapping ranges
  if (((uintptr_t)psi | (uintptr_t)out) & 15) return OK_EINVAL;
  if (prec == OK_F64) {
    if (W->W64) {
      EpiArgs<double> e{};
      return launch_apply<double>(W, (const cx<double>*)psi, (cx<double>*)out, EPI_NONE, e, (cudaStream_t)stream);
    }
    if (!W->Wdf) return OK_EINVAL;
    // double-float copy: convert psi into stream-ordered scratch, apply, release the scratch
    cudaStream_t st = (cudaStream_t)stream;
    void* psi_df = nullptr;
    OK_CUDA_TRY(cudaMallocAsync(&psi_df, bytes, st));
    int rc = launch_to_df((const cx<double>*)psi, (cx<dd>*)psi_df, 12LL * W->g.V, st);
    if (rc == OK_SUCCESS) {
      EpiArgs<dd> e{};
      rc = launch_apply_dd(W, (const cx<dd>*)psi_df, (cx<double>*)out, EPI_NONE, e, st);
    }
    cudaError_t fe = cudaFreeAsync(psi_df, st);
    if (rc == OK_SUCCESS && fe != cudaSuccess) { set_cuda_error(fe); rc = OK_ECUDA; }
    return rc;
  }
  EpiArgs<float> e{};
  if (prec == OK_F32_OTF) return launch_apply_otf(W, (const cx<float>*)psi, (cx<float>*)out, (cudaStream_t)stream);
  if (prec == OK_F32_W16) {
    if (!W->W16) return OK_EINVAL;
    return launch_apply_w16(W, (const cx<float>*)psi, (cx<float>*)out, EPI_NONE, e, (cudaStream_t)stream);
  }
  if (!W->W32) return OK_EINVAL;
  return launch_apply<float>(W, (const cx<float>*)psi, (cx<float>*)out, EPI_NONE, e, (cudaStream_t)stream);
}

ok_solve_params ok_default_solve_params(double tol, int maxiter) {
  ok_solve_params p;
  p.tol = tol;
  p.maxiter = maxiter;
  p.mode = OK_SOLVE_AUTO;
  p.delta = 1e-3;
  p.max_restarts = 5;
  p.check_every = 4;
  return p;
}

int ok_bicgstab_ex(const ok_W* W, const void* src, void* x, const ok_solve_params* params, ok_solve_info* info,
                   void* stream) {
  if (!W || !src || !x || !params) return OK_EINVAL;
  if ((((uintptr_t)src) | ((uintptr_t)x)) & 15) return OK_EINVAL;
  return bicgstab(W, (const cx<double>*)src, (cx<double>*)x, params, info, (cudaStream_t)stream);
}

int ok_apply_M_multi(const ok_W* W, ok_prec prec, int nrhs, const void* psi, void* out, void* stream) {
  if (!W || !psi || !out || nrhs < 1 || (prec != OK_F32 && prec != OK_F32_W16 && prec != OK_F16_TC)) return OK_EINVAL;
  const size_t bytes = (size_t)W->g.V * 12 * 8 * nrhs;
  const char* a = (const char*)psi;
  const char* b = (const char*)out;
  if (a < b + bytes && b < a + bytes) return OK_EINVAL;
  if (((uintptr_t)psi | (uintptr_t)out) & 15) return OK_EINVAL;
  if (prec == OK_F16_TC) {
    // canonical layout -> the FP16 tensor-core layout (scaled per right-hand side), apply, and back;
    // stream-ordered scratch
    if (!W->Wtc || nrhs > 16) return OK_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)W->g.V * 12 * nrhs;  // complex numbers
    char* scratch = nullptr;
    const size_t o16 = 0, o32 = tc_in16_bytes(W->g.V), oam = o32 + n * 8, oinv = oam + 64;
    OK_CUDA_TRY(cudaMallocAsync((void**)&scratch, oinv + 64, st));
    unsigned* amax = (unsigned*)(scratch + oam);
    float* inv = (float*)(scratch + oinv);
    int rc = launch_to_tc16((const cx<float>*)psi, scratch + o16, W->g.V, nrhs, amax, inv, st);
    if (rc == OK_SUCCESS) {
      TcEpi ep{};
      ep.inv_scale = inv;
      rc = launch_apply_tc(W, scratch + o16, (cx<float>*)(scratch + o32), nrhs, EPI_NONE, ep, st);
    }
    if (rc == OK_SUCCESS) rc = launch_from_tc((const cx<float>*)(scratch + o32), (cx<float>*)out, W->g.V, nrhs, st);
    const cudaError_t fe = cudaFreeAsync(scratch, st);
    if (rc == OK_SUCCESS && fe != cudaSuccess) {
      set_cuda_error(fe);
      rc = OK_ECUDA;
    }
    return rc;
  }
  const bool w16 = prec == OK_F32_W16;
  if ((w16 && !W->W16) || (!w16 && !W->W32)) return OK_EINVAL;
  MultiEpi e{};
  return launch_apply_multi(W, w16, (const cx<float>*)psi, (cx<float>*)out, nrhs, EPI_NONE, e, multi_shape(W, w16, nrhs),
                            (cudaStream_t)stream);
}

int ok_bicgstab_multi(const ok_W* W, int nrhs, const void* src, void* x, const ok_solve_params* params, ok_solve_info* info,
                      void* stream) {
  if (!W || !src || !x || !params || nrhs < 1) return OK_EINVAL;
  if ((((uintptr_t)src) | ((uintptr_t)x)) & 15) return OK_EINVAL;
  const size_t bytes = (size_t)W->g.V * 12 * 16 * nrhs;
  const char* a = (const char*)src;
  const char* b = (const char*)x;
  if (a < b + bytes && b < a + bytes) return OK_EINVAL;
  return bicgstab_multi(W, nrhs, (const cx<double>*)src, (cx<double>*)x, params, info, (cudaStream_t)stream);
}

int ok_bicgstab_multi_net(const ok_W* W, ok_net* net, int nrhs, const void* src, void* x, const ok_solve_params* params,
                          ok_solve_info* info, void* stream) {
  if (!W || !net || !src || !x || !params || nrhs < 1) return OK_EINVAL;
  if ((((uintptr_t)src) | ((uintptr_t)x)) & 15) return OK_EINVAL;
  const size_t bytes = (size_t)W->g.V * 12 * 16 * nrhs;
  const char* a = (const char*)src;
  const char* b = (const char*)x;
  if (a < b + bytes && b < a + bytes) return OK_EINVAL;
  return bicgstab_multi(W, nrhs, (const cx<double>*)src, (cx<double>*)x, params, info, (cudaStream_t)stream, net);
}

int ok_autotune(ok_W* W, ok_prec prec, int nrhs, int* choice, double* best_us, void* stream) {
  return autotune(W, prec, nrhs, choice, best_us, (cudaStream_t)stream);
}

int ok_net_create(int layers, const double* weights, ok_net** net) { return net_create(layers, weights, net); }

void ok_net_free(ok_net* net) { net_free(net); }

int ok_net_layers(const ok_net* net) { return net_layers(net); }

int ok_net_get_weights(ok_net* net, double* weights) {
  if (!net || !weights) return OK_EINVAL;
  return net_weights(net, weights, nullptr);
}

int ok_net_set_weights(ok_net* net, const double* weights) {
  if (!net || !weights) return OK_EINVAL;
  return net_weights(net, nullptr, weights);
}

static bool net_fields_ok(const ok_W* W, const void* a, const void* b, size_t count) {
  if (!W || !a || !b || (((uintptr_t)a | (uintptr_t)b) & 15)) return false;
  const size_t bytes = (size_t)W->g.V * 12 * 8 * count;
  const char* p = (const char*)a;
  const char* q = (const char*)b;
  return !(p < q + bytes && q < p + bytes);
}

int ok_net_apply(ok_net* net, const ok_W* W, const void* psi, void* out, void* stream) {
  if (!net || !net_fields_ok(W, psi, out, 1)) return OK_EINVAL;
  return net_apply(net, W, (const cx<float>*)psi, (cx<float>*)out, (cudaStream_t)stream);
}

int ok_net_loss_grad(ok_net* net, const ok_W* W, const void* b, const void* x, double* loss, double* grad, void* stream) {
  if (!net || !W || !b || !x || ((((uintptr_t)b) | ((uintptr_t)x)) & 15)) return OK_EINVAL;
  return net_loss_grad(net, W, (const cx<float>*)b, (const cx<float>*)x, loss, grad, (cudaStream_t)stream);
}

int ok_net_train_step(ok_net* net, const ok_W* W, int nb, const void* b, const void* x, double lr, double* loss, void* stream) {
  if (!net || !W || !b || !x || nb < 1 || ((((uintptr_t)b) | ((uintptr_t)x)) & 15)) return OK_EINVAL;
  return net_train_step(net, W, nb, (const cx<float>*)b, (const cx<float>*)x, lr, loss, (cudaStream_t)stream);
}

int ok_bicgstab_net(const ok_W* W, ok_net* net, const void* src, void* x, const ok_solve_params* params, ok_solve_info* info,
                    void* stream) {
  if (!W || !net || !src || !x || !params) return OK_EINVAL;
  if ((((uintptr_t)src) | ((uintptr_t)x)) & 15) return OK_EINVAL;
  return bicgstab_net(W, net, (const cx<double>*)src, (cx<double>*)x, params, info, (cudaStream_t)stream);
}

int ok_set_launch_shape(ok_W* W, ok_prec prec, int staged, int nr, int blocks_x) {
  if (!W || (prec != OK_F32 && prec != OK_F32_W16)) return OK_EINVAL;
  if ((staged != 0 && staged != 1) || (nr != 0 && nr != 1 && nr != 2 && nr != 4) || blocks_x < 0 || blocks_x > (1 << 20))
    return OK_EINVAL;
  const int k = prec == OK_F32_W16 ? 1 : 0;
  W->tune.staged[k] = staged;
  W->tune.mr_nr[k] = nr;
  W->tune.mr_bx[k] = blocks_x;
  return OK_SUCCESS;
}

int ok_bicgstab(const ok_W* W, const void* src, void* x, double tol, int maxiter, ok_solve_info* info, void* stream) {
  ok_solve_params p = ok_default_solve_params(tol, maxiter);
  return ok_bicgstab_ex(W, src, x, &p, info, stream);
}

int ok_true_residual(const ok_W* W, const void* b, const void* x, double* relres, void* stream) {
  return true_residual(W, (const cx<double>*)b, (const cx<double>*)x, relres, (cudaStream_t)stream);
}

int ok_apply_M_reduce(const ok_W* W, ok_prec prec, int kind, const void* psi, const void* y, void* out, double* sums,
                      void* stream) {
  if (!W || !psi || !y || !out || !sums) return OK_EINVAL;
  const size_t es = prec == OK_F64 ? 16 : (prec == OK_F32 || prec == OK_F32_W16) ? 8 : 0;
  if (es == 0) return OK_EINVAL;
  const size_t bytes = (size_t)W->g.V * 12 * es;
  const char* o = (const char*)out;
  for (const void* in : {psi, y}) {
    const char* a = (const char*)in;
    if (a < o + bytes && o < a + bytes) return OK_EINVAL;
  }
  if (((uintptr_t)psi | (uintptr_t)y | (uintptr_t)out) & 15) return OK_EINVAL;
  return apply_reduce(W, prec, kind, psi, y, out, sums, (cudaStream_t)stream);
}

int ok_W_expand(const ok_W* W, ok_prec prec, int kind, void* out, void* stream) {
  return expand(W, prec, kind, out, (cudaStream_t)stream);
}

unsigned long long ok_launch_count(void) { return launches(); }

int ok_inject_wait_timeout(unsigned extra_bytes) { return okgb::set_stage_test_bytes(extra_bytes); }

int ok_wait_timeouts(unsigned* n, int reset) {
  if (!n) return OK_EINVAL;
  return okgb::read_wait_timeouts(n, reset != 0);
}

void ok_trace_enable(int on) { g_trace_on.store(on ? 1 : 0); }

int ok_trace_read(ok_trace_stat* stats, int max, int* n) {
  if (!stats || !n || max < 0) return OK_EINVAL;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  int rc = OK_SUCCESS;
  for (TraceRec& r : g_pending) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
    if (e != cudaSuccess) { set_cuda_error(e); rc = OK_ECUDA; continue; }
    TraceTotals& t = g_totals[r.name];
    t.launches += 1;
    t.ms += ms;
  }
  g_pending.clear();
  int k = 0;
  for (auto& kv : g_totals) {
    if (k < max) {
      std::memset(stats[k].name, 0, sizeof(stats[k].name));
      std::strncpy(stats[k].name, kv.first.c_str(), sizeof(stats[k].name) - 1);
      stats[k].launches = kv.second.launches;
      stats[k].total_ms = kv.second.ms;
    }
    ++k;
  }
  *n = k;
  return rc;
}

void ok_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (TraceRec& r : g_pending) {
    cudaEventSynchronize(r.b);
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_pending.clear();
  g_totals.clear();
}

int ok_last_cuda_error(void) { return g_last_cuda_error; }

const char* ok_strerror(int status) {
  switch (status) {
    case OK_SUCCESS: return "success";
    case OK_EINVAL: return "invalid argument";
    case OK_ENOMEM: return "out of memory";
    case OK_ECUDA: return "CUDA error";
    case OK_ENOCONV: return "solver did not converge";
    case OK_EBREAKDOWN: return "BiCGStab breakdown";
    case OK_ENONFINITE: return "non-finite value in the solver";
    case OK_EINTERNAL: return "internal error";
    default: return "unknown status";
  }
}

}  // extern "C"
