// Instantiations of the persistent forward kernel for the sample op.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

const void* fwd_kernel_sample(int block, int items, int occ) {
  return fwd_kernel<OPF_SAMPLE>(block, items, occ);
}

}  // namespace bysdf
