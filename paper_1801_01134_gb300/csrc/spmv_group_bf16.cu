// beta(r,c) SpMV with G lanes per interval (variants 24-29), BF16 values, all twelve shapes.
#include "spmv_group.cuh"

namespace spc5 {

cudaError_t launch_group_bf16(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials) {
  return dispatch_grp<BF16>(h, x, y, acc, partials, s);
}

}  // namespace spc5
