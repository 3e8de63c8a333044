// Multi-right-hand-side application: launchers (FP32 W kernels instantiated here, FP16 W kernels
// in ok_mrhs16.cu).
#include "ok_mrhs.cuh"

namespace okgb {

namespace mrhs {
template int launch_wt<float>(const ok_W*, const cx<float>*, const cx<float>*, cx<float>*, int, int, const MultiEpi&,
                              const MultiShape&, cudaStream_t);
extern template int launch_wt<__half>(const ok_W*, const cx<__half>*, const cx<float>*, cx<float>*, int, int,
                                      const MultiEpi&, const MultiShape&, cudaStream_t);
}  // namespace mrhs

int mrhs_blocks_needed(const ok_W* W) { return grid_for(W->g.V, mrhs::MR_SITES); }

MultiShape multi_shape(const ok_W* W, bool w16, int nrhs) {
  const int k = w16 ? 1 : 0;
  MultiShape s{W->tune.mr_nr[k], W->tune.mr_bx[k]};
  if ((s.nr != 1 && s.nr != 2 && s.nr != 4) || nrhs % s.nr != 0) {
    s.nr = nrhs % 2 == 0 ? 2 : 1;  // until ok_autotune has measured this handle
    s.blocks_x = 0;
  }
  return s;
}

int launch_apply_multi(const ok_W* Wh, bool w16, const cx<float>* psi, cx<float>* out, int nrhs, int epi, const MultiEpi& ep,
                       const MultiShape& shape, cudaStream_t st) {
  if (!Wh || !psi || !out || nrhs < 1) return OK_EINVAL;
  const int nr = shape.nr;
  if ((nr != 1 && nr != 2 && nr != 4) || nrhs % nr != 0) return OK_EINVAL;
  if (epi != EPI_NONE && epi != EPI_DOT && epi != EPI_TS) return OK_EINVAL;
  if (epi != EPI_NONE && (!ep.st || !ep.part || (epi == EPI_DOT && !ep.rhat))) return OK_EINVAL;
  static const char* n32[3] = {"apply_multi_f32", "apply_multi_f32_dot", "apply_multi_f32_ts"};
  static const char* n16[3] = {"apply_multi_w16", "apply_multi_w16_dot", "apply_multi_w16_ts"};
  int rc = OK_EINVAL;
  {
    TraceScope ts(w16 ? n16[epi] : n32[epi], st);
    if (w16) {
      const cx<__half>* W = (const cx<__half>*)Wh->W16;
      if (!W) return OK_EINVAL;
      rc = mrhs::launch_wt<__half>(Wh, W, psi, out, nrhs, epi, ep, shape, st);
    } else {
      const cx<float>* W = (const cx<float>*)Wh->W32;
      if (!W) return OK_EINVAL;
      rc = mrhs::launch_wt<float>(Wh, W, psi, out, nrhs, epi, ep, shape, st);
    }
  }
  if (rc != OK_SUCCESS) return rc;
  OK_LAUNCH_CHECK();
  return OK_SUCCESS;
}

}  // namespace okgb
