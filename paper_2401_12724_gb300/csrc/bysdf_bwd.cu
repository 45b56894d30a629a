// Backward kernels of libbysdf.
//
// k_backward: per-material parameter gradients.  Recomputes the forward pass
// of each record with the helix angles as dual-number tangents (the other
// parameters in closed form) and reduces sum_c g_c df_c/dtheta per material --
// warp shuffles over a single-material warp tile, then one atomic (or one
// fixed-order partial) per tile; with unsorted records, shared-memory
// accumulators per CTA.  KIND: the 8-column basic set, the 15-column
// extended set, or the basic set with the upstream gradient of an L2 loss
// (its value a ninth accumulated column, flushed to the per-material loss).
//
// k_dirgrad: per-record vector-Jacobian products with respect to the record's
// directions, forward mode with 6 tangents (wi, wo); no reduction.
#include "bysdf_launch.h"

namespace bysdf {

template <int BLOCK, int MINB, int KIND>
__global__ void __launch_bounds__(BLOCK, MINB) k_backward(const KArgs a) {
  constexpr int NP = KbCols<KIND>::acc;      // accumulated columns
  constexpr int NG = KbCols<KIND>::grad;     // gradient columns of grad_params
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2 * (BLOCK / 32)];
  // MODE_ALL_SMEM: per-CTA accumulators behind the tables
  float* sacc = reinterpret_cast<float*>(smem + (size_t)a.n_mat * a.sstride);
  if (a.mode == MODE_ALL_SMEM) {
    for (int k = threadIdx.x; k < a.n_mat * NP; k += BLOCK) sacc[k] = 0.f;
  }
  persistent_loop<BLOCK>(a, smem, bars,
                             [&](int64_t begin, int64_t end, int mat, uint8_t* slot, int lane,
                                 int tile) {
    float acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.f;
    // rolled: one copy of the (large) record body
#pragma unroll 1
    for (int64_t i = begin + lane; i < end; i += 32) {
      if (!bounds_ok(i >= 0 && i < a.n)) continue;
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
        q.mat = a.mat_id ? __ldcg(a.mat_id + i) : 0;
        mm = (q.mat >= 0 && q.mat < a.n_mat) ? q.mat : 0;
        tb = smem + (size_t)mm * a.sstride;
      }
      const MatDev* m = reinterpret_cast<const MatDev*>(tb);
      float g[NP];
      backward_record<KIND>(a, *m, reinterpret_cast<const float2*>(m + 1), i, q, g);
      if (mat >= 0) {
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[k] += g[k];
      } else if (q.mat == mm) {
#pragma unroll
        for (int k = 0; k < NP; ++k)
          if (g[k] != 0.f) atomicAdd(&sacc[mm * NP + k], g[k]);
      }
    }
    if (mat >= 0) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        float v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[k] = v;
      }
      if (lane == 0) {
        if (a.partials) {
#pragma unroll
          for (int k = 0; k < NP; ++k) a.partials[(size_t)tile * NP + k] = acc[k];
        } else {
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            if (k < NG) atomicAdd(a.grad_params + (size_t)mat * NG + k, acc[k]);
            else if (a.loss_mat) atomicAdd(a.loss_mat + mat, acc[k]);
          }
        }
      }
    }
  });
  if (a.mode == MODE_ALL_SMEM) {
    __syncthreads();
    for (int k = threadIdx.x; k < a.n_mat * NP; k += BLOCK) {
      if (sacc[k] == 0.f) continue;
      const int mm = k / NP, c = k - mm * NP;
      if (c < NG) atomicAdd(a.grad_params + (size_t)mm * NG + c, sacc[k]);
      else if (a.loss_mat) atomicAdd(a.loss_mat + mm, sacc[k]);
    }
  }
}

// Fixed-order reduction of per-tile partials: one warp per material sums its
// tiles lane-strided, then a shuffle tree (deterministic for a given launch
// shape).
__global__ void k_reduce_partials(const KArgs a) {
  const int m = blockIdx.x, lane = threadIdx.x;
  const int np = a.n_param;
  const int t0 = a.tile_start[m], t1 = a.tile_start[m + 1];
  float acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) acc[k] = 0.f;
  for (int t = t0 + lane; t < t1; t += 32) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < np) acc[k] += a.partials[(size_t)t * np + k];
  }
  // gradient columns to grad_params; the L2 backward's loss column to loss_mat
  const int ng = a.target ? np - 1 : np;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    float v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && k < ng) a.grad_params[(size_t)m * ng + k] = v;
    if (lane == 0 && k == ng && k < np && a.loss_mat) a.loss_mat[m] = v;
  }
}

enum { DD_WI = 0, DD_WO = 3, NDD = 6 };

// A shading state with omega_i's three tangents as one with all six (the
// omega_o tangents zero).
template <class D, class DI>
__device__ __forceinline__ D widen_di(const DI& x) {
  D r(x.v);
#pragma unroll
  for (int k = 0; k < 3; ++k) r.d[DD_WI + k] = x.d[k];
  return r;
}
template <class D, class DI>
__device__ __forceinline__ V3<D> widen_di3(const V3<DI>& x) {
  return mk3<D>(widen_di<D>(x.x), widen_di<D>(x.y), widen_di<D>(x.z));
}
template <class D, class DI>
__device__ __forceinline__ Shade<D> widen_shade(const Shade<DI>& x) {
  Shade<D> r;
  r.t = widen_di3<D>(x.t);
  r.b = widen_di3<D>(x.b);
  r.n = widen_di3<D>(x.n);
  r.wi = widen_di3<D>(x.wi);
  r.mui = widen_di<D>(x.mui);
  r.g = widen_di<D>(x.g);
  r.fr = widen_di<D>(x.fr);
  r.at = x.at;
  r.ab = x.ab;
  r.at_free = x.at_free;
  r.ab_free = x.ab_free;
  r.body_x0 = widen_di<D>(x.body_x0);
  r.body_y0 = widen_di<D>(x.body_y0);
  r.ni_sy = x.ni_sy;
  r.tt_ok = x.tt_ok;
  r.iy = widen_di3<D>(x.iy);
  r.by = widen_di3<D>(x.by);
  r.ny = widen_di3<D>(x.ny);
  r.tx = widen_di<D>(x.tx);
  r.tau = widen_di<D>(x.tau);
  return r;
}

// Direction vector-Jacobian products of one record: sum_c g_c df_c/dwi and
// df_c/dwo.  Tangents 0..2: wi, 3..5: wo.  The material's helix angles carry
// no tangent here; the float pre-pass of the geometry picks each node's ply.
__device__ __forceinline__ void dirgrad_record(const KArgs& a, const MatDev& m,
                                               const float2* map, int64_t i, Record& q,
                                               float gwi[3], float gwo[3]) {
  typedef DualF<NDD> D;
  typedef DualF<3> DI;   // omega_i's tangents alone
#pragma unroll
  for (int c = 0; c < 3; ++c) gwi[c] = gwo[c] = 0.f;
  if (!record_valid(q, a.n_mat, true, a.ratio != nullptr, false)) return;
  // omega_o enters only the lobes: the geometry and the shading frame carry
  // omega_i's three tangents, and are widened to all six for the lobes
  const MatVars<DI> mv = mat_vars<DI>(m, false);
  V3<DI> wi = lift3<DI>(q.wi[0], q.wi[1], q.wi[2]);
  wi.x.d[0] = 1.f;
  wi.y.d[1] = 1.f;
  wi.z.d[2] = 1.f;
  Geo<DI> G;
  geometry_k<1, DI, DI>(m, map, mv, q, wi, G);
  if (G.status != ST_OK) return;
  Shade<DI> si;
  make_shade(m, mv, G, wi, si);
  const Shade<D> s = widen_shade<D>(si);
  V3<D> wo = lift3<D>(q.wo[0], q.wo[1], q.wo[2]);
  wo.x.d[DD_WO + 0] = 1.f;
  wo.y.d[DD_WO + 1] = 1.f;
  wo.z.d[DD_WO + 2] = 1.f;
  LobeVals<D> L;
  eval_lobes(m, s, wo, L);
  const int64_t n = a.n;
  const float g0 = __ldg(a.grad_f + i), g1 = __ldg(a.grad_f + n + i),
              g2 = __ldg(a.grad_f + 2 * n + i);
  const float* kb = L.refl ? m.alb : m.alb_y;
  const float gs = g0 + g1 + g2;
  const float gb = g0 * kb[0] + g1 * kb[1] + g2 * kb[2];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    gwi[c] = gs * L.spec.d[DD_WI + c] + gb * L.body.d[DD_WI + c];
    gwo[c] = gs * L.spec.d[DD_WO + c] + gb * L.body.d[DD_WO + c];
  }
}

template <int BLOCK, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_dirgrad(const KArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2 * (BLOCK / 32)];
  persistent_loop<BLOCK>(a, smem, bars,
                             [&](int64_t begin, int64_t end, int mat, uint8_t* slot, int lane,
                                 int) {
#pragma unroll 1
    for (int64_t i = begin + lane; i < end; i += 32) {
      if (!bounds_ok(i >= 0 && i < a.n)) continue;
      Record q;
      load_record(a, i, true, false, q);
      const uint8_t* tb;
      if (mat >= 0) {
        q.mat = mat;
        tb = slot;
      } else {
        q.mat = a.mat_id ? __ldcg(a.mat_id + i) : 0;
        const int mm = (q.mat >= 0 && q.mat < a.n_mat) ? q.mat : 0;
        tb = smem + (size_t)mm * a.sstride;
      }
      const MatDev* m = reinterpret_cast<const MatDev*>(tb);
      float gwi[3], gwo[3];
      dirgrad_record(a, *m, reinterpret_cast<const float2*>(m + 1), i, q, gwi, gwo);
      const int64_t n = a.n;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (a.grad_wi) __stcs(a.grad_wi + c * n + i, gwi[c]);
        if (a.grad_wo) __stcs(a.grad_wo + c * n + i, gwo[c]);
      }
    }
  });
}

// occupancy 0: registers as needed (8 warps per SM at 256 threads);
// occupancy 1: at most 128 registers (16 warps per SM; the rest spills).
template <int KIND>
static const void* bwd_fn_t(int block, int occ) {
  switch (block) {
    case 128: return occ ? (const void*)k_backward<128, 4, KIND> : (const void*)k_backward<128, 1, KIND>;
    case 256: return occ ? (const void*)k_backward<256, 2, KIND> : (const void*)k_backward<256, 1, KIND>;
    case 512: return (const void*)k_backward<512, 1, KIND>;
  }
  return nullptr;
}
static const void* bwd_fn(int block, int occ, int kind) {
  switch (kind) {
    case KB_BASIC: return bwd_fn_t<KB_BASIC>(block, occ);
    case KB_EXT: return bwd_fn_t<KB_EXT>(block, occ);
    case KB_L2: return bwd_fn_t<KB_L2>(block, occ);
  }
  return nullptr;
}
static const void* dir_fn(int block) {
  switch (block) {
    case 128: return (const void*)k_dirgrad<128, 1>;
    case 256: return (const void*)k_dirgrad<256, 1>;
    case 512: return (const void*)k_dirgrad<512, 1>;
  }
  return nullptr;
}

cudaError_t set_backward_smem_limit(int block, int occ, int kind, size_t smem) {
  const void* f = bwd_fn(block, occ, kind);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t backward_occupancy(int block, int occ, int kind, size_t smem, int* ctas) {
  const void* f = bwd_fn(block, occ, kind);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block, smem);
}

cudaError_t launch_backward(const KArgs& a, int block, int occ, int kind, int grid, size_t smem,
                            cudaStream_t st) {
  const void* f = bwd_fn(block, occ, kind);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<KArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, st);
}

cudaError_t launch_reduce_partials(const KArgs& a, cudaStream_t st) {
  k_reduce_partials<<<a.n_mat, 32, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t set_dirgrad_smem_limit(int block, size_t smem) {
  const void* f = dir_fn(block);
  if (!f) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t dirgrad_occupancy(int block, size_t smem, int* ctas) {
  const void* f = dir_fn(block);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block, smem);
}

cudaError_t launch_dirgrad(const KArgs& a, int block, int grid, size_t smem, cudaStream_t st) {
  const void* f = dir_fn(block);
  if (!f) return cudaErrorInvalidValue;
  void* args[] = {const_cast<KArgs*>(&a)};
  return cudaLaunchKernel(f, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace bysdf
