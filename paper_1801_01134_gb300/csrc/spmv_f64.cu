// beta(r,c) SpMV instantiations for the F64 value type (all twelve shapes).
#include "spmv_beta.cuh"

namespace spc5 {

cudaError_t launch_spmv_f64(const spc5_matrix* h, const void* x, void* y, bool acc, cudaStream_t s, void* partials) {
  void* part = partials ? partials : h->partials;
  if (group_variant(h->variant) || stream_variant(h->variant)) return launch_group_f64(h, x, y, acc, s, part);
  return dispatch_beta<F64>(h, x, y, acc, part, s);
}

}  // namespace spc5
