// Launchers shared between the translation units of libbysdf (internal).
#pragma once

#include <cuda_runtime.h>

#include "bysdf.h"
#include "bysdf_kernels.cuh"

namespace bysdf {

// camera rays -> hit records (bysdf_trace_yarns)
struct TraceArgs {
  const float *o, *d, *o1, *d1, *o2, *d2;
  int64_t n;
  float light[3];
  float *h, *u, *v, *wi, *wo, *ratio, *t_hit;
  int32_t *mat_id, *yarn_id;
};
constexpr int kMaxYarnPieces = 2048;  // 64 bytes each in shared memory
cudaError_t launch_trace_yarns(const bysdf_yarn* yarns, int n_yarns, const TraceArgs& a,
                               int grid, cudaStream_t st);

// op: OPF_* bit set (EVAL, SAMPLE, PDF, EVAL|SAMPLE).  Returns the launch error.
cudaError_t launch_forward(int op, const KArgs& a, int block, int occ, int grid, size_t smem,
                           cudaStream_t st);
cudaError_t launch_plain(int op, const KArgs& a, int mat, int64_t begin, int64_t end,
                         cudaStream_t st);
// kind: KB_BASIC (8 columns), KB_EXT (15), KB_L2 (8 + the loss column); a.n_param
// must be the accumulated column count (8, 15, 9)
cudaError_t launch_backward(const KArgs& a, int block, int occ, int kind, int grid, size_t smem,
                            cudaStream_t st);
cudaError_t launch_reduce_partials(const KArgs& a, cudaStream_t st);
cudaError_t set_forward_smem_limit(int op, int block, int items, int occ, size_t smem);
cudaError_t set_backward_smem_limit(int block, int occ, int kind, size_t smem);
cudaError_t forward_occupancy(int op, int block, int items, int occ, size_t smem, int* ctas);
cudaError_t backward_occupancy(int block, int occ, int kind, size_t smem, int* ctas);
// direction vector-Jacobian products (a.grad_wi / a.grad_wo)
cudaError_t set_dirgrad_smem_limit(int block, size_t smem);
cudaError_t dirgrad_occupancy(int block, size_t smem, int* ctas);
cudaError_t launch_dirgrad(const KArgs& a, int block, int grid, size_t smem, cudaStream_t st);
// test hook: the float path's own approximations beside CUDA's functions
cudaError_t launch_test_math(int fn, const float* x, const float* y, int64_t n, float* out,
                             cudaStream_t st);

}  // namespace bysdf
