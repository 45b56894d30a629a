// Forward dispatch of libbysdf (launch, occupancy, shared-memory limit of the
// persistent kernels) and the plain per-material form.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

template <int OP>
__global__ void __launch_bounds__(256, 2) k_plain(const KArgs a, int mat, int64_t begin, int64_t end) {
#ifdef BYSDF_DEBUG_BOUNDS
  // no workspace here: failed checks only clamp
  if (threadIdx.x == 0) g_bounds_word = nullptr;
  __syncthreads();
#endif
  const int64_t i = begin + (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= end) return;
  const MatDev* m = reinterpret_cast<const MatDev*>(a.table + (size_t)mat * a.stride);
  Record q;
  load_record(a, i, (OP & (OPF_EVAL | OPF_PDF)) != 0, (OP & OPF_SAMPLE) != 0, q);
  q.mat = mat;
  forward_record<OP>(a, *m, reinterpret_cast<const float2*>(m + 1), i, q);
}

// ------------------------------------------------------------------ launch --
static const void* fwd_fn(int op, int block, int items, int occ) {
  if (op & OPF_STOCH) return fwd_kernel_stoch(op, block, items, occ);
  switch (op) {
    case OPF_EVAL: return fwd_kernel_eval(block, items, occ);
    case OPF_SAMPLE: return fwd_kernel_sample(block, items, occ);
    case OPF_PDF: return fwd_kernel_pdf(block, items, occ);
    case OPF_EVAL | OPF_SAMPLE: return fwd_kernel_fused(block, items, occ);
  }
  return nullptr;
}

cudaError_t set_forward_smem_limit(int op, int block, int items, int occ, size_t smem) {
  const void* f = fwd_fn(op, block, items, occ);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t forward_occupancy(int op, int block, int items, int occ, size_t smem, int* ctas) {
  const void* f = fwd_fn(op, block, items, occ);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block, smem);
}

cudaError_t launch_forward(int op, const KArgs& a, int block, int occ, int grid, size_t smem,
                           cudaStream_t st) {
  const void* f = fwd_fn(op, block, a.tile / 32, occ);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<KArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t launch_plain(int op, const KArgs& a, int mat, int64_t begin, int64_t end,
                         cudaStream_t st) {
  if (end <= begin) return cudaSuccess;
  const unsigned grid = (unsigned)((end - begin + 255) / 256);
  switch (op) {
    case OPF_EVAL: k_plain<OPF_EVAL><<<grid, 256, 0, st>>>(a, mat, begin, end); break;
    case OPF_SAMPLE: k_plain<OPF_SAMPLE><<<grid, 256, 0, st>>>(a, mat, begin, end); break;
    case OPF_PDF: k_plain<OPF_PDF><<<grid, 256, 0, st>>>(a, mat, begin, end); break;
    case OPF_EVAL | OPF_SAMPLE:
      k_plain<OPF_EVAL | OPF_SAMPLE><<<grid, 256, 0, st>>>(a, mat, begin, end);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bysdf
