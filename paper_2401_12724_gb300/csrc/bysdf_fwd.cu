// Forward kernels of libbysdf: the persistent material-table-in-shared-memory
// kernel (eval / sample / pdf / fused) and the plain per-material form.
#include "bysdf_launch.h"

namespace bysdf {

template <int OP, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_forward(const KArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[BLOCK / 32];
  constexpr bool kWo = (OP & (OPF_EVAL | OPF_PDF)) != 0;
  constexpr bool kU = (OP & OPF_SAMPLE) != 0;
  persistent_loop<BLOCK>(a, smem, bars,
                         [&](int64_t begin, int64_t end, int mat, uint8_t* slot, int lane, int) {
    for (int64_t i = begin + lane; i < end; i += 32) {
      Record q;
      load_record(a, i, kWo, kU, q);
      const MatDev* m;
      if (mat >= 0) {
        q.mat = mat;
        m = reinterpret_cast<const MatDev*>(slot);
      } else {
        q.mat = a.mat_id ? __ldg(a.mat_id + i) : 0;
        const int mm = (q.mat >= 0 && q.mat < a.n_mat) ? q.mat : 0;
        m = reinterpret_cast<const MatDev*>(smem + (size_t)mm * a.stride);
      }
      forward_record<OP>(a, *m, reinterpret_cast<const float2*>(m + 1), i, q);
    }
  });
}

template <int OP>
__global__ void __launch_bounds__(256) k_plain(const KArgs a, int mat, int64_t begin, int64_t end) {
  const int64_t i = begin + (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= end) return;
  const MatDev* m = reinterpret_cast<const MatDev*>(a.table + (size_t)mat * a.stride);
  Record q;
  load_record(a, i, (OP & (OPF_EVAL | OPF_PDF)) != 0, (OP & OPF_SAMPLE) != 0, q);
  q.mat = mat;
  forward_record<OP>(a, *m, reinterpret_cast<const float2*>(m + 1), i, q);
}

// ------------------------------------------------------------------ launch --
template <int OP>
static const void* fwd_fn(int block) {
  switch (block) {
    case 128: return (const void*)k_forward<OP, 128>;
    case 256: return (const void*)k_forward<OP, 256>;
    case 512: return (const void*)k_forward<OP, 512>;
  }
  return nullptr;
}
static const void* fwd_fn(int op, int block) {
  switch (op) {
    case OPF_EVAL: return fwd_fn<OPF_EVAL>(block);
    case OPF_SAMPLE: return fwd_fn<OPF_SAMPLE>(block);
    case OPF_PDF: return fwd_fn<OPF_PDF>(block);
    case OPF_EVAL | OPF_SAMPLE: return fwd_fn<OPF_EVAL | OPF_SAMPLE>(block);
  }
  return nullptr;
}

cudaError_t set_forward_smem_limit(int op, int block, size_t smem) {
  const void* f = fwd_fn(op, block);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t forward_occupancy(int op, int block, size_t smem, int* ctas) {
  const void* f = fwd_fn(op, block);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block, smem);
}

cudaError_t launch_forward(int op, const KArgs& a, int block, int grid, size_t smem,
                           cudaStream_t st) {
  const void* f = fwd_fn(op, block);
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
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bysdf
