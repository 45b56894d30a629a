// Instantiations of the persistent forward kernel for the pdf op.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

const void* fwd_kernel_pdf(int block, int items, int occ) {
  return fwd_kernel<OPF_PDF>(block, items, occ);
}

}  // namespace bysdf
