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

// The float path's approximations evaluated on given arguments, beside the
// CUDA functions they stand in for, in a unit built with the forward's
// flags (approximate division and square root, denormals flushed): 0
// xatan2(y, x), 1 atan2f(y, x), 2 / 3 sine / cosine of xsincos(x), 4 / 5
// sinf(x) / cosf(x).
__global__ void k_test_math(int fn, const float* x, const float* y, int64_t n, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = x[i], b = y ? y[i] : 0.f;
  float r = 0.f, s, c;
  switch (fn) {
    case 0: r = xatan2(b, a); break;
    case 1: r = atan2f(b, a); break;
    case 2: xsincos(a, &s, &c); r = s; break;
    case 3: xsincos(a, &s, &c); r = c; break;
    case 4: r = sinf(a); break;
    case 5: r = cosf(a); break;
  }
  out[i] = r;
}

cudaError_t launch_test_math(int fn, const float* x, const float* y, int64_t n, float* out,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_test_math<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(fn, x, y, n, out);
  return cudaGetLastError();
}

}  // namespace bysdf
