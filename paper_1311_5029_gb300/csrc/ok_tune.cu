// Autotuner: picks launch shapes for a handle by timing the candidates on scratch fields.
//   one right-hand side: the split kernel with the forward W read by ordinary loads or streamed
//     into shared memory by TMA (which wins depends on the lattice and on L1 pressure);
//   several right-hand sides: right-hand sides per thread NR (1, 2 or 4, dividing nrhs) and the
//     width of the persistent grid (as many blocks as fit, or half of that).
// Each candidate is launched twice untimed and then timed over five launches with CUDA events on
// the caller's stream; the fastest is stored in the handle's tuning record.
#include "ok_launch.cuh"

namespace okgb {

namespace {

struct Scratch {
  cudaStream_t st;
  void* p[2] = {nullptr, nullptr};
  ~Scratch() {
    for (void* q : p)
      if (q) cudaFreeAsync(q, st);
  }
};

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

template <typename F>
int time_us(F&& launch, cudaStream_t st, Events& ev, double* us) {
  for (int k = 0; k < 2; ++k) {
    int rc = launch();
    if (rc != OK_SUCCESS) return rc;
  }
  OK_CUDA_TRY(cudaEventRecord(ev.a, st));
  constexpr int reps = 5;
  for (int k = 0; k < reps; ++k) {
    int rc = launch();
    if (rc != OK_SUCCESS) return rc;
  }
  OK_CUDA_TRY(cudaEventRecord(ev.b, st));
  OK_CUDA_TRY(cudaEventSynchronize(ev.b));
  float ms = 0.f;
  OK_CUDA_TRY(cudaEventElapsedTime(&ms, ev.a, ev.b));
  *us = 1e3 * ms / reps;
  return OK_SUCCESS;
}

}  // namespace

int autotune(ok_W* W, ok_prec prec, int nrhs, int* choice, double* best_us, cudaStream_t st) {
  if (!W || nrhs < 1 || nrhs > 64 || (prec != OK_F32 && prec != OK_F32_W16)) return OK_EINVAL;
  const bool w16 = prec == OK_F32_W16;
  if ((w16 && !W->W16) || (!w16 && !W->W32)) return OK_EINVAL;
  const int k = w16 ? 1 : 0;
  const size_t bytes = (size_t)W->g.V * 12 * sizeof(cx<float>) * nrhs;
  Scratch sc{st};
  OK_CUDA_TRY(cudaMallocAsync(&sc.p[0], bytes, st));
  OK_CUDA_TRY(cudaMallocAsync(&sc.p[1], bytes, st));
  OK_CUDA_TRY(cudaMemsetAsync(sc.p[0], 0, bytes, st));
  const cx<float>* psi = (const cx<float>*)sc.p[0];
  cx<float>* out = (cx<float>*)sc.p[1];
  Events ev;
  OK_CUDA_TRY(cudaEventCreate(&ev.a));
  OK_CUDA_TRY(cudaEventCreate(&ev.b));
  double best = 1e300;
  int pick = 0;
  if (nrhs == 1) {
    const Tune saved = W->tune;
    for (int staged = 0; staged <= 1; ++staged) {
      W->tune.staged[k] = staged;
      double us = 0.0;
      EpiArgs<float> e{};
      int rc = time_us([&] { return w16 ? launch_apply_w16(W, psi, out, EPI_NONE, e, st)
                                         : launch_apply<float>(W, psi, out, EPI_NONE, e, st); }, st, ev, &us);
      if (rc != OK_SUCCESS) { W->tune = saved; return rc; }
      if (us < best) { best = us; pick = staged; }
    }
    W->tune.staged[k] = pick;
  } else {
    int best_nr = 0, best_bx = 0;
    for (int nr : {1, 2, 4}) {
      if (nrhs % nr != 0) continue;
      // 0 = as many blocks per row as fit (resident blocks per SM as in the kernel's launch
      // bounds), or half that width, each block then walking twice as many tiles
      const int fit = sm_count() * (nr <= 2 ? 4 : 2) / (nrhs / nr);
      const int half = fit / 2 > 0 ? fit / 2 : 1;
      for (int width : {0, half}) {
        const MultiShape use{nr, width};
        const MultiEpi e{};
        double us = 0.0;
        int rc = time_us([&] { return launch_apply_multi(W, w16, psi, out, nrhs, EPI_NONE, e, use, st); }, st, ev, &us);
        if (rc != OK_SUCCESS) return rc;
        if (us < best) { best = us; best_nr = nr; best_bx = width; }
      }
    }
    W->tune.mr_nr[k] = best_nr;
    W->tune.mr_bx[k] = best_bx;
    pick = best_nr;
  }
  if (choice) *choice = pick;
  if (best_us) *best_us = best;
  return OK_SUCCESS;
}

}  // namespace okgb
