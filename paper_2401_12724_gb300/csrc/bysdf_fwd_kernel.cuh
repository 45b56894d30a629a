// The persistent forward kernel template (eval / sample / pdf / fused) and the
// table of its instantiations; each op's instantiations compile in their own
// translation unit (bysdf_fwd_<op>.cu).
#pragma once

#include "bysdf_launch.h"

namespace bysdf {

template <int OP, int BLOCK, int ITEMS, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB) k_forward(const KArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2 * (BLOCK / 32)];
  // each warp's order list (32 * ITEMS entries) and bucket counts (32)
  // behind the tables
  uint32_t* list = reinterpret_cast<uint32_t*>(smem + a.order_off) +
                   (threadIdx.x >> 5) * (32 * ITEMS + kOrderBuckets);
  uint32_t* hist = list + 32 * ITEMS;
  persistent_loop<BLOCK>(a, smem, bars,
                         [&](int64_t begin, int64_t end, int mat, uint8_t* slot, int lane, int) {
    // records with a footprint in bucket order (each lane reads back only
    // its own slots of the list, written before the warp's last
    // synchronisation); near-field records in plain order
    const bool ordered = a.ratio != nullptr;
    if (ordered) tile_order<ITEMS>(a, smem, begin, end, mat, slot, lane, list, hist);
#pragma unroll 1
    for (int j = 0; j < ITEMS; ++j) {
      uint32_t e = (uint32_t)(j * 32 + lane);
      if (ordered) {
        e = list[j * 32 + lane];
      } else if (begin + e >= end) {
        e = 0xffffffffu;
      }
      if (e == 0xffffffffu) continue;
      const int64_t i = begin + (e & 0xffu);
      if (!bounds_ok(i >= begin && i < end)) continue;
      Record q;
      load_record(a, i, (OP & (OPF_EVAL | OPF_PDF)) != 0, (OP & OPF_SAMPLE) != 0, q);
      const MatDev* m;
      if (mat >= 0) {
        q.mat = mat;
        m = reinterpret_cast<const MatDev*>(slot);
      } else {
        q.mat = a.mat_id ? __ldcg(a.mat_id + i) : 0;
        const int mm = (q.mat >= 0 && q.mat < a.n_mat) ? q.mat : 0;
        if (!bounds_ok((size_t)mm * a.sstride + a.stride <= (size_t)a.order_off)) continue;
        m = reinterpret_cast<const MatDev*>(smem + (size_t)mm * a.sstride);
      }
      // two plies side by side in the trace when registers allow (<= 128)
      forward_record<OP, (BLOCK * MINB <= 512 ? 2 : 1)>(
          a, *m, reinterpret_cast<const float2*>(m + 1), i, q);
    }
    __syncwarp();   // the list is rewritten by the next tile
  });
}

// Register budget per launch shape: occupancy 0 caps registers so that 16
// warps fit on an SM (128 per thread), occupancy 1 so that 24 fit (80 per
// thread; the rest spills to L1).
template <int BLOCK, int OCC>
struct MinBlocks {
  static constexpr int value = OCC == 1 ? (BLOCK == 128 ? 6 : (BLOCK == 256 ? 3 : 1))
                                        : (BLOCK >= 512 ? 1 : 512 / BLOCK);
};

template <int OP, int BLOCK, int ITEMS>
const void* fwd_kernel_bi(int occ) {
  if (occ == 1 && BLOCK < 512)
    return (const void*)k_forward<OP, BLOCK, ITEMS, MinBlocks<BLOCK, 1>::value>;
  return (const void*)k_forward<OP, BLOCK, ITEMS, MinBlocks<BLOCK, 0>::value>;
}

template <int OP, int BLOCK>
const void* fwd_kernel_b(int items, int occ) {
  switch (items) {
    case 1: return fwd_kernel_bi<OP, BLOCK, 1>(occ);
    case 2: return fwd_kernel_bi<OP, BLOCK, 2>(occ);
    case 4: return fwd_kernel_bi<OP, BLOCK, 4>(occ);
    case 8: return fwd_kernel_bi<OP, BLOCK, 8>(occ);
  }
  return nullptr;
}

template <int OP>
const void* fwd_kernel(int block, int items, int occ) {
  switch (block) {
    case 128: return fwd_kernel_b<OP, 128>(items, occ);
    case 256: return fwd_kernel_b<OP, 256>(items, occ);
    case 512: return fwd_kernel_b<OP, 512>(items, occ);
  }
  return nullptr;
}

// one definition per op, in bysdf_fwd_<op>.cu
const void* fwd_kernel_eval(int block, int items, int occ);
const void* fwd_kernel_sample(int block, int items, int occ);
const void* fwd_kernel_pdf(int block, int items, int occ);
const void* fwd_kernel_fused(int block, int items, int occ);
// the stochastic estimators (op with OPF_STOCH), in bysdf_fwd_stoch.cu
const void* fwd_kernel_stoch(int op, int block, int items, int occ);

}  // namespace bysdf
