// Instantiations of the persistent forward kernel for the stochastic
// estimators (eval + pdf, and the fused op): every block size at up to 128
// registers per thread, and blocks of 128 and 256 threads in the tighter
// budget of 24 warps per SM (occupancy 1).
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

template <int OP, int BLOCK, int MINB>
static const void* stoch_bm(int items) {
  switch (items) {
    case 1: return (const void*)k_forward<OP, BLOCK, 1, MINB>;
    case 2: return (const void*)k_forward<OP, BLOCK, 2, MINB>;
    case 4: return (const void*)k_forward<OP, BLOCK, 4, MINB>;
    case 8: return (const void*)k_forward<OP, BLOCK, 8, MINB>;
  }
  return nullptr;
}

template <int OP, int BLOCK>
static const void* stoch_b(int items, int occ) {
  if (occ == 1 && BLOCK < 512) return stoch_bm<OP, BLOCK, MinBlocks<BLOCK, 1>::value>(items);
  return stoch_bm<OP, BLOCK, MinBlocks<BLOCK, 0>::value>(items);
}

template <int OP>
static const void* stoch_op(int block, int items, int occ) {
  switch (block) {
    case 128: return stoch_b<OP, 128>(items, occ);
    case 256: return stoch_b<OP, 256>(items, occ);
    case 512: return stoch_b<OP, 512>(items, occ);
  }
  return nullptr;
}

const void* fwd_kernel_stoch(int op, int block, int items, int occ) {
  switch (op) {
    case OPF_EVAL | OPF_STOCH: return stoch_op<OPF_EVAL | OPF_STOCH>(block, items, occ);
    case OPF_EVAL | OPF_SAMPLE | OPF_STOCH:
      return stoch_op<OPF_EVAL | OPF_SAMPLE | OPF_STOCH>(block, items, occ);
  }
  return nullptr;
}

}  // namespace bysdf
