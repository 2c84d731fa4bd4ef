// tree.cu -- placeholder until the octree kernels land.
#include "tree.h"

namespace gs {
cudaError_t tree_setup() { return cudaSuccess; }
gs_status tree_reserve(TreeWork&, int64_t, bool, cudaStream_t) { return GS_ERR_UNSUPPORTED; }
void tree_release(TreeWork&) {}
gs_status bh_forward(TreeWork&, const BHStep&, const FwdEpi&, int*, int64_t*, cudaStream_t) {
  return GS_ERR_UNSUPPORTED;
}
gs_status bh_adjoint(TreeWork&, const BHStep&, const float4*, const AdjEpi&, int*, int64_t*,
                     cudaStream_t) {
  return GS_ERR_UNSUPPORTED;
}
void bh_counts(TreeWork&, int64_t* cnt) { cnt[0] = cnt[1] = 0; }
const char* bh_last_error() { return "Barnes-Hut mode not built"; }
}  // namespace gs

extern "C" gs_status gs_tree(gs_ctx*, const double*, int64_t, uint32_t*, int32_t*, int32_t*,
                             float*, int64_t, int64_t*, void*) {
  return GS_ERR_UNSUPPORTED;
}
extern "C" gs_status gs_shoot_batched(gs_ctx*, int32_t, const int64_t*, const double*,
                                      const double*, const double*, const gs_params*, double*,
                                      double*, void*) {
  return GS_ERR_UNSUPPORTED;
}
