// Allocation-free variant of the FP64 true residual (see ok_true_residual_static in include/ok.h).
//
// The reduction scratch (per-block partial sums, the completion ticket and the final sums) lives
// in one file-scope __device__ array of fixed size instead of memory obtained from cudaMalloc.
// Every GPU that loads this library holds the array until the process exits.  Host code cannot
// use the array's name as a device address, so every call looks the address up with
// cudaGetSymbolAddress, with the caller's device current, and passes it to the kernel.  The
// lookup allocates nothing; doing it on every call (rather than caching it per device ordinal)
// keeps the address right after a device reset or when another context has loaded the module at
// a different address.  The first call on a device may load the module there, so it should come
// before any stream capture.
#include "ok_launch.cuh"

#include <cmath>
#include <cstring>

namespace okgb {
namespace {

// Layout of the scratch array: the solver-state record (ticket, sums) first, rounded up to 256
// bytes, then the per-block partial sums of the apply kernel's residual epilogue (2 doubles per
// block, at most one block per 32 sites for any apply variant).
constexpr size_t kStateBytes = (sizeof(SolverState) + 255) / 256 * 256;
constexpr size_t kPartialDoubles = (size_t)(OK_STATIC_MAX_SITES / 32) * 2;
constexpr size_t kScratchBytes = kStateBytes + kPartialDoubles * sizeof(double);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch in the current context.
int scratch_address(void** out) {
  void* p = nullptr;
  OK_CUDA_TRY(cudaGetSymbolAddress(&p, g_scratch));
  *out = p;
  return OK_SUCCESS;
}

}  // namespace
}  // namespace okgb

using namespace okgb;

extern "C" int ok_true_residual_static(const ok_W* W, const void* b, const void* x, void* r, double* relres,
                                       void* stream) {
  if (!W || !b || !x || !r || !relres || !W->W64) return OK_EINVAL;
  if (W->g.V > OK_STATIC_MAX_SITES) return OK_EINVAL;
  if ((size_t)apply_blocks_needed(W) * 2 > kPartialDoubles) return OK_EINVAL;
  if ((((uintptr_t)b) | ((uintptr_t)x) | ((uintptr_t)r)) & 15) return OK_EINVAL;
  const size_t bytes = (size_t)W->g.V * 12 * sizeof(cx<double>);
  const char* rb = (const char*)r;
  for (const void* in : {b, x}) {
    const char* ib = (const char*)in;
    if (rb < ib + bytes && ib < rb + bytes) return OK_EINVAL;  // r must not overlap an input
  }
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != OK_SUCCESS) return rc;
  SolverState* state = (SolverState*)base;
  double* part = (double*)((char*)base + kStateBytes);
  // The array keeps the previous call's contents: clear the ticket and sums first.
  OK_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(SolverState), st));
  EpiArgs<double> e{nullptr, (const cx<double>*)b, RedArgs{state, part, nullptr, FIN_RESID}, &state->ticket[5], nullptr};
  rc = launch_apply<double>(W, (const cx<double>*)x, (cx<double>*)r, EPI_RESID, e, st);
  if (rc != OK_SUCCESS) return rc;
  double sums[2] = {0.0, 0.0};
  OK_CUDA_TRY(cudaMemcpyAsync(sums, (const char*)state + offsetof(SolverState, aux), sizeof(sums),
                              cudaMemcpyDeviceToHost, st));
  OK_CUDA_TRY(cudaStreamSynchronize(st));
  *relres = sums[1] > 0.0 ? std::sqrt(sums[0] / sums[1]) : std::sqrt(sums[0]);
  return OK_SUCCESS;
}
