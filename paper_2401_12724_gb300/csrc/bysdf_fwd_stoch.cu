// Instantiations of the persistent forward kernel for the stochastic
// estimators (eval + pdf, and the fused op), in the launch shapes that keep
// up to 128 registers per thread.
#include "bysdf_fwd_kernel.cuh"

namespace bysdf {

template <int OP, int BLOCK>
static const void* stoch_b(int items) {
  constexpr int MINB = MinBlocks<BLOCK, 0>::value;
  switch (items) {
    case 1: return (const void*)k_forward<OP, BLOCK, 1, MINB>;
    case 2: return (const void*)k_forward<OP, BLOCK, 2, MINB>;
    case 4: return (const void*)k_forward<OP, BLOCK, 4, MINB>;
    case 8: return (const void*)k_forward<OP, BLOCK, 8, MINB>;
  }
  return nullptr;
}

template <int OP>
static const void* stoch_op(int block, int items) {
  switch (block) {
    case 128: return stoch_b<OP, 128>(items);
    case 256: return stoch_b<OP, 256>(items);
    case 512: return stoch_b<OP, 512>(items);
  }
  return nullptr;
}

const void* fwd_kernel_stoch(int op, int block, int items) {
  switch (op) {
    case OPF_EVAL | OPF_STOCH: return stoch_op<OPF_EVAL | OPF_STOCH>(block, items);
    case OPF_EVAL | OPF_SAMPLE | OPF_STOCH:
      return stoch_op<OPF_EVAL | OPF_SAMPLE | OPF_STOCH>(block, items);
  }
  return nullptr;
}

}  // namespace bysdf
