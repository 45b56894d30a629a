// Instantiations of the persistent forward kernel for the eval op.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

const void* fwd_kernel_eval(int block, int items, int occ) {
  return fwd_kernel<OPF_EVAL>(block, items, occ);
}

}  // namespace bysdf
