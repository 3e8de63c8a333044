// Multi-right-hand-side application: the kernels reading the half-precision W copy.
#include "ok_mrhs.cuh"

namespace okgb {
namespace mrhs {
template int launch_wt<__half>(const ok_W*, const cx<__half>*, const cx<float>*, cx<float>*, int, int, const MultiEpi&,
                               const MultiShape&, cudaStream_t);
}  // namespace mrhs
}  // namespace okgb
