// Instantiations of the persistent forward kernel for the fused op.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

const void* fwd_kernel_fused(int block, int items, int occ) {
  return fwd_kernel<OPF_EVAL | OPF_SAMPLE>(block, items, occ);
}

}  // namespace bysdf
