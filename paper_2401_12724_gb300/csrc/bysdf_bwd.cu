// Backward kernel of libbysdf: recomputes the forward pass of each record in
// forward-mode dual numbers (one tangent per differentiable parameter) and
// reduces sum_c g_c df_c/dtheta per material -- warp shuffles over a
// single-material warp tile, then one atomic (or one fixed-order partial) per
// tile; with unsorted records, shared-memory accumulators per CTA.
#include "bysdf_launch.h"

namespace bysdf {

template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_backward(const KArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[BLOCK / 32];
  // MODE_ALL_SMEM: per-CTA accumulators behind the tables
  float* sacc = reinterpret_cast<float*>(smem + (size_t)a.n_mat * a.stride);
  if (a.mode == MODE_ALL_SMEM) {
    for (int k = threadIdx.x; k < a.n_mat * 8; k += BLOCK) sacc[k] = 0.f;
  }
  persistent_loop<BLOCK>(a, smem, bars,
                             [&](int64_t begin, int64_t end, int mat, uint8_t* slot, int lane,
                                 int tile) {
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    for (int64_t i = begin + lane; i < end; i += 32) {
      Record q;
      load_record(a, i, true, false, q);
      // one call site of the (large, dual-number) record body for both
      // scheduling modes keeps the kernel's code small
      int mm;
      const uint8_t* tb;
      if (mat >= 0) {
        q.mat = mat;
        mm = mat;
        tb = slot;
      } else {
        q.mat = a.mat_id ? __ldg(a.mat_id + i) : 0;
        mm = (q.mat >= 0 && q.mat < a.n_mat) ? q.mat : 0;
        tb = smem + (size_t)mm * a.stride;
      }
      const MatDev* m = reinterpret_cast<const MatDev*>(tb);
      float g[8];
      backward_record(a, *m, reinterpret_cast<const float2*>(m + 1), i, q, g);
      if (mat >= 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += g[k];
      } else if (q.mat == mm) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (g[k] != 0.f) atomicAdd(&sacc[mm * 8 + k], g[k]);
      }
    }
    if (mat >= 0) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[k] = v;
      }
      if (lane == 0) {
        if (a.partials) {
#pragma unroll
          for (int k = 0; k < 8; ++k) a.partials[(size_t)tile * 8 + k] = acc[k];
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) atomicAdd(a.grad_params + (size_t)mat * 8 + k, acc[k]);
        }
      }
    }
  });
  if (a.mode == MODE_ALL_SMEM) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_mat * 8; k += BLOCK)
      if (sacc[k] != 0.f) atomicAdd(a.grad_params + k, sacc[k]);
  }
}

// Fixed-order reduction of per-tile partials: one warp per material sums its
// tiles lane-strided, then a shuffle tree (deterministic for a given launch
// shape).
__global__ void k_reduce_partials(const KArgs a) {
  const int m = blockIdx.x, lane = threadIdx.x;
  const int t0 = a.tile_start[m], t1 = a.tile_start[m + 1];
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
  for (int t = t0 + lane; t < t1; t += 32) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] += a.partials[(size_t)t * 8 + k];
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) a.grad_params[(size_t)m * 8 + k] = v;
  }
}

// occupancy 0: registers as needed (8 warps per SM at 256 threads);
// occupancy 1: at most 128 registers (16 warps per SM; the rest spills).
static const void* bwd_fn(int block, int occ) {
  switch (block) {
    case 128: return occ ? (const void*)k_backward<128, 4> : (const void*)k_backward<128, 1>;
    case 256: return occ ? (const void*)k_backward<256, 2> : (const void*)k_backward<256, 1>;
    case 512: return (const void*)k_backward<512, 1>;
  }
  return nullptr;
}

cudaError_t set_backward_smem_limit(int block, int occ, size_t smem) {
  const void* f = bwd_fn(block, occ);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t backward_occupancy(int block, int occ, size_t smem, int* ctas) {
  const void* f = bwd_fn(block, occ);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block, smem);
}

cudaError_t launch_backward(const KArgs& a, int block, int occ, int grid, size_t smem,
                            cudaStream_t st) {
  const void* f = bwd_fn(block, occ);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<KArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t launch_reduce_partials(const KArgs& a, cudaStream_t st) {
  k_reduce_partials<<<a.n_mat, 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bysdf
