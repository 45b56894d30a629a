// Kernel-side plumbing of libbysdf: launch arguments, TMA bulk copies of the
// material table into shared memory with bounded mbarrier waits, record
// loads, the warp-granular tile queue, and the per-record drivers.
#pragma once

#include "bysdf_model.cuh"

namespace bysdf {

// OPF_STOCH: the stochastic estimators (jittered nodes, GGX-sampled entry)
enum : int { OPF_EVAL = 1, OPF_SAMPLE = 2, OPF_PDF = 4, OPF_STOCH = 8 };
enum : int { MODE_ALL_SMEM = 0, MODE_SORTED = 1 };
enum : uint32_t { ERR_TABLE_WAIT = 1u, ERR_TABLE_INFLIGHT = 2u };

// Workspace layout (bytes): [0, 256) control words, then tile_start[n_mat + 1]
// (int32), then per-tile gradient partials (deterministic backward).
//
// Control words.  Every launch gets an epoch e from the host (40 bits,
// never 0).  err_word = e << 24 | error bits, e the epoch of the launch that
// last claimed it.  At its start each CTA claims the error word for its
// launch: a word holding another epoch (a previous launch's, the contents
// of a fresh allocation, or 0 after bysdf_workspace_error read it) is set
// to e << 24.  The bits stay until bysdf_workspace_error reads them; a
// captured launch replayed with its one epoch adds to the bits of its
// earlier replays until then.
//
// tile_word counts the warp-tile draws.  For records in any order with
// fewer than 2^24 draws (claim_tiles) the CTAs claim it the same way and
// the draws count from e << 24; the launch's last draw sets it to 0, so the
// next launch (a replay with the same epoch too) claims it again, and no
// reset kernel runs.  Otherwise the host launches k_plan first, which sets
// tile_word to 0 and err_word to e << 24 (and, for material-sorted records,
// computes the first tile of every material).
constexpr size_t kWsCtl = 256;
constexpr int kEpochShift = 24;
struct WsCtl {
  unsigned long long tile_word;
  unsigned long long err_word;
  int32_t pad[60];
};

struct KArgs {
  const uint8_t* table;  // device material table (n_mat blocks of `stride` bytes)
  int32_t n_mat;
  int32_t stride;        // bytes of one material's table (global memory)
  int32_t sstride;       // MODE_ALL_SMEM: bytes between materials' tables in shared memory
  int32_t mode;
  int32_t tile;          // records per warp tile (32 * items)
  int64_t n;
  int64_t n_tiles;
  const float *h, *u, *v, *wi, *wo, *ratio, *u0, *u1;
  const int32_t* mat_id;
  const int64_t* seg;
  float *f_rgb, *pdf;
  uint8_t* status;
  float *wo_s, *weight_s, *pdf_s;
  uint8_t* lstat_s;
  const float* grad_f;
  float* grad_params;
  float* partials;       // deterministic backward: [n_tiles][n_param]
  const float* target;   // L2 backward: target radiance (3 planes); NULL otherwise
  const float* weight;   // L2 backward: per-record loss weights, or NULL (1)
  float* loss_mat;       // L2 backward: per-material loss, or NULL
  int32_t n_param;       // gradient columns: 8, or 15 (extended set)
  int32_t order_off;      // forward: byte offset of the warps' sort keys in shared memory
  float *grad_wi, *grad_wo;  // direction backward: 3 planes each, or NULL
  uint64_t stoch_seed;       // stochastic estimators: generator key word 0,
  int64_t stoch_index0;      //   global index of record 0,
  uint32_t stoch_flags;      //   STOCH_* bits
  uint32_t wait_limit;       // polls of a table-copy wait before it gives up
  uint32_t test_stall;       // test hook: table waits poll a barrier nothing arrives on
  uint32_t claim_tiles;      // the tile count starts at epoch << 24 (no k_plan launched)
  uint64_t epoch;            // this launch's epoch (control words)
  WsCtl* ctl;
  const int32_t* tile_start;
};

// ------------------------------------------------------ TMA + mbarrier ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> shared (TMA), completion signalled on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Sets `word` to epoch << 24 unless it already carries this epoch.  The
// first compare-and-swap guesses 0 (a claimed tile word returns to 0 at the
// end of its launch), the next ones the value the last one found.  Writers
// of another epoch cannot run at the same time (the calls that share a
// workspace are stream-ordered), so at most one compare-and-swap of the
// CTAs of a launch succeeds and the loop ends after a few turns; it is
// bounded all the same.
__device__ __forceinline__ void claim_word(unsigned long long* word, uint64_t epoch) {
  const unsigned long long mine = (unsigned long long)epoch << kEpochShift;
  unsigned long long cur = 0ull;
  for (int it = 0; it < 64; ++it) {
    const unsigned long long prev = atomicCAS(word, cur, mine);
    if (prev == cur || (prev >> kEpochShift) == epoch) break;
    cur = prev;
  }
}

// Error bits of this launch (after the CTA claimed the word).
__device__ __forceinline__ void set_error(WsCtl* ctl, uint32_t code) {
  atomicOr(&ctl->err_word, (unsigned long long)code);
}

// Bounded wait: gives up after `limit` polls (each poll may itself suspend
// for a hardware-defined interval), records the failure and returns false.
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, WsCtl* ctl,
                                                  uint32_t code, uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  set_error(ctl, code);
  return false;
}

// ------------------------------------------------------------ record IO ----
// Record planes are read once per record and cached in L2 only (ld.global.cg),
// which leaves L1 to the tables' spill-over and the register spills of the
// tighter launch shapes.
__device__ __forceinline__ void load_record(const KArgs& a, int64_t i, bool need_wo,
                                            bool need_u, Record& q) {
  const int64_t n = a.n;
  q.h = __ldcg(a.h + i);
  q.u = __ldcg(a.u + i);
  q.v = __ldcg(a.v + i);
  q.wi[0] = __ldcg(a.wi + i);
  q.wi[1] = __ldcg(a.wi + n + i);
  q.wi[2] = __ldcg(a.wi + 2 * n + i);
  if (need_wo) {
    q.wo[0] = __ldcg(a.wo + i);
    q.wo[1] = __ldcg(a.wo + n + i);
    q.wo[2] = __ldcg(a.wo + 2 * n + i);
  } else {
    q.wo[0] = q.wo[1] = q.wo[2] = 0.f;
  }
  q.ratio = a.ratio ? __ldcg(a.ratio + i) : 0.f;
  if (need_u) {
    q.u0 = __ldcg(a.u0 + i);
    q.u1 = __ldcg(a.u1 + i);
  } else {
    q.u0 = q.u1 = 0.f;
  }
}

// Forward pass of one record: eval/pdf at hits->wo and/or one sample.
template <int OP, int PLIES = 2>
__device__ __forceinline__ void forward_record(const KArgs& a, const MatDev& m,
                                               const float2* map, int64_t i, Record& q) {
  constexpr bool kEval = (OP & (OPF_EVAL | OPF_PDF)) != 0;
  constexpr bool kSample = (OP & OPF_SAMPLE) != 0;
  const int64_t n = a.n;
  // eval needs a valid omega_o, sampling valid random numbers; in the fused
  // op an invalid one invalidates only its own half
  const bool base = base_valid(q, a.n_mat, a.ratio != nullptr);
  const bool eval_ok = base && (!kEval || unit_ok(q.wo));
  const bool samp_ok = base && (!kSample || u_valid(q));
  int st = ST_INVALID;
  Geo<float> G;
  Shade<float> s;
  if (eval_ok || samp_ok) {
    const MatVars<float> mv = mat_vars<float>(m);
    if constexpr ((OP & OPF_STOCH) != 0) {
      const StochCtx sc{a.stoch_flags, a.stoch_seed, (uint64_t)(a.stoch_index0 + i)};
      const V3<float> wi = mk3<float>(q.wi[0], q.wi[1], q.wi[2]);
      geometry_k<PLIES, float, float>(m, map, mv, q, wi, G, &sc);
      st = G.status;
      if (st == ST_OK) make_shade(m, mv, G, wi, s, &sc);
    } else {
      geometry<PLIES>(m, map, mv, q, G);
      st = G.status;
      if (st == ST_OK) make_shade(m, mv, G, q, s);
    }
  }
  if constexpr (kEval) {
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, p = 0.f;
    const int est = eval_ok ? st : ST_INVALID;
    if (est == ST_OK) {
      LobeVals<float> L;
      eval_lobes(m, s, mk3<float>(q.wo[0], q.wo[1], q.wo[2]), L);
      const float* kb = L.refl ? m.alb : m.alb_y;  // k^B_x (Eq. 5) or k^B_y (Eq. 6)
      f0 = L.spec + kb[0] * L.body;
      f1 = L.spec + kb[1] * L.body;
      f2 = L.spec + kb[2] * L.body;
      p = total_pdf(m, s, L);
    }
    if (OP & OPF_EVAL) {
      __stcs(a.f_rgb + i, f0);
      __stcs(a.f_rgb + n + i, f1);
      __stcs(a.f_rgb + 2 * n + i, f2);
    }
    if (a.pdf) __stcs(a.pdf + i, p);
    a.status[i] = (uint8_t)est;
  }
  if constexpr (kSample) {
    float w0 = 0.f, w1 = 0.f, w2 = 0.f, ww0 = 0.f, ww1 = 0.f, ww2 = 0.f, p = 0.f;
    int sst = samp_ok ? st : ST_INVALID, lobe = 0;
    if (sst == ST_NO_HIT) {
      w0 = -q.wi[0];
      w1 = -q.wi[1];
      w2 = -q.wi[2];
      ww0 = ww1 = ww2 = 1.f;
    } else if (sst == ST_OK) {
      V3<float> wo;
      sst = ST_BAD_SAMPLE;
      if (sample_dir(m, s, q.u0, q.u1, &wo, &lobe)) {
        w0 = wo.x;
        w1 = wo.y;
        w2 = wo.z;
        LobeVals<float> L;
        eval_lobes(m, s, wo, L);
        const float pt = total_pdf(m, s, L);
        if (pt > 0.f) {
          const float ip = 1.0f / pt;
          const float* kb = L.refl ? m.alb : m.alb_y;
          ww0 = (L.spec + kb[0] * L.body) * ip;
          ww1 = (L.spec + kb[1] * L.body) * ip;
          ww2 = (L.spec + kb[2] * L.body) * ip;
          p = pt;
          sst = ST_OK;
        }
      }
    }
    __stcs(a.wo_s + i, w0);
    __stcs(a.wo_s + n + i, w1);
    __stcs(a.wo_s + 2 * n + i, w2);
    __stcs(a.weight_s + i, ww0);
    __stcs(a.weight_s + n + i, ww1);
    __stcs(a.weight_s + 2 * n + i, ww2);
    __stcs(a.pdf_s + i, p);
    a.lstat_s[i] = (uint8_t)(sst | (lobe << 4));
  }
}

// Kinds of the backward: the 8 parameters of the basic set, the 15 of the
// extended set, and the basic set with the upstream gradient taken from an
// L2 loss against target radiance, whose value is a ninth column.
enum { KB_BASIC = 0, KB_EXT = 1, KB_L2 = 2 };
template <int KIND> struct KbCols {
  static constexpr int grad = KIND == KB_EXT ? 15 : 8;            // gradient columns
  static constexpr int acc = KIND == KB_L2 ? 9 : grad;             // accumulated columns
};

// Gradient of sum_c g_c f_c of one record w.r.t. the material parameters:
// the 8 of the basic set ([0..2] moves both body colours), or the 15 of the
// extended set (KB_EXT; layout of bysdf_set_params_ext).  KB_L2: g_c =
// 2 w (f_c - target_c) from the record's own f (Sec. 5.2 fitting of an L2
// loss), gout[8] = w sum_c (f_c - target_c)^2, and f is written to
// a.f_rgb when given (0 where the record has no valid evaluation).
template <int KIND>
__device__ __forceinline__ void backward_record(const KArgs& a, const MatDev& m,
                                                const float2* map, int64_t i, Record& q,
                                                float* gout) {
  typedef DualF<ND> D;
  constexpr bool EXT = KIND == KB_EXT;
  constexpr int NA = KbCols<KIND>::acc;
#pragma unroll
  for (int k = 0; k < NA; ++k) gout[k] = 0.f;
  if constexpr (KIND == KB_L2) {
    if (a.f_rgb) {
      a.f_rgb[i] = 0.f;
      a.f_rgb[a.n + i] = 0.f;
      a.f_rgb[2 * a.n + i] = 0.f;
    }
  }
  if (!record_valid(q, a.n_mat, true, a.ratio != nullptr, false)) return;
  const MatVars<D> mv = mat_vars<D>(m);
  Geo<D> G;
  // one ply per pass in the float pick pass: fewer live registers at the
  // backward's 128 (2.6% faster than two)
  geometry<1>(m, map, mv, q, G);
  if (G.status != ST_OK) return;
  Shade<D> s;
  make_shade(m, mv, G, q, s);
  LobeVals<D> L;
  float dln_a[2] = {0.f, 0.f};
  eval_lobes(m, s, mk3<float>(q.wo[0], q.wo[1], q.wo[2]), L, dln_a);
  const int64_t n = a.n;
  // f_c = spec + k^B_c body, with k^B = k^B_x (reflection side) or k^B_y
  const float* kb = L.refl ? m.alb : m.alb_y;
  float g0, g1, g2;
  if constexpr (KIND == KB_L2) {
    const float f0 = L.spec.v + kb[0] * L.body.v, f1 = L.spec.v + kb[1] * L.body.v,
                f2 = L.spec.v + kb[2] * L.body.v;
    if (a.f_rgb) {
      a.f_rgb[i] = f0;
      a.f_rgb[n + i] = f1;
      a.f_rgb[2 * n + i] = f2;
    }
    const float w = a.weight ? __ldcg(a.weight + i) : 1.0f;
    const float d0 = f0 - __ldcg(a.target + i), d1 = f1 - __ldcg(a.target + n + i),
                d2 = f2 - __ldcg(a.target + 2 * n + i);
    g0 = 2.0f * w * d0;
    g1 = 2.0f * w * d1;
    g2 = 2.0f * w * d2;
    gout[8] = w * (d0 * d0 + d1 * d1 + d2 * d2);
  } else {
    g0 = __ldcg(a.grad_f + i);
    g1 = __ldcg(a.grad_f + n + i);
    g2 = __ldcg(a.grad_f + 2 * n + i);
  }
  const float gs = g0 + g1 + g2;
  const float gb = g0 * kb[0] + g1 * kb[1] + g2 * kb[2];
  const float body = L.body.v;
  const int c0 = (EXT && !L.refl) ? 9 : 0;
  gout[c0 + 0] = g0 * body;
  gout[c0 + 1] = g1 * body;
  gout[c0 + 2] = g2 * body;
  // roughness: d spec / d beta = spec * d ln spec / d alpha (alpha = beta +
  // footprint term, unless clamped)
  gout[3] = s.at_free ? gs * L.spec.v * dln_a[0] : 0.f;
  gout[4] = s.ab_free ? gs * L.spec.v * dln_a[1] : 0.f;
  // helix angles: the dual tangents
  gout[5] = gs * L.spec.d[D_ALPHA_P] + gb * L.body.d[D_ALPHA_P];
  gout[6] = gs * L.spec.d[D_ALPHA_F] + gb * L.body.d[D_ALPHA_F];
  // shadow density: the body lobes are proportional to G
  const float Gv = G.g.v;
  gout[7] = Gv > 0.f ? gb * body * (G.dg_dsig / Gv) : 0.f;
  if constexpr (EXT) {
    // body = r B body_w (reflection side) or (1 - r) B body_w; spec = (1 - B)
    // k_spec spec_u; the transmission lobe carries tau = exp(-sigma_t N_i
    // |x - y|) (Eq. 4)
    const float bw = L.body_w.v, su = L.spec_u.v;
    gout[8] = gb * (L.refl ? m.B : -m.B) * bw;
    gout[12] = L.refl ? 0.f : gs * L.spec.v * (-s.ni_sy);
    gout[13] = gb * (L.refl ? m.r : 1.0f - m.r) * bw - gs * m.k_spec * su;
    gout[14] = gs * (1.0f - m.B) * su;
  }
}

// Records of a tile no warp could evaluate (a table wait gave up): every
// per-record output gets a defined value, status ST_ABORTED and zeros, so a
// caller never reads a previous call's contents as this call's results.
__device__ __forceinline__ void abort_tile(const KArgs& a, int64_t begin, int64_t end, int lane) {
  const int64_t n = a.n;
  for (int64_t i = begin + lane; i < end; i += 32) {
    if (a.status) a.status[i] = (uint8_t)ST_ABORTED;
    if (a.lstat_s) a.lstat_s[i] = (uint8_t)ST_ABORTED;
    if (a.pdf) a.pdf[i] = 0.f;
    if (a.pdf_s) a.pdf_s[i] = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (a.f_rgb) a.f_rgb[c * n + i] = 0.f;
      if (a.wo_s) a.wo_s[c * n + i] = 0.f;
      if (a.weight_s) a.weight_s[c * n + i] = 0.f;
      if (a.grad_wi) a.grad_wi[c * n + i] = 0.f;
      if (a.grad_wo) a.grad_wo[c * n + i] = 0.f;
    }
  }
}

// Shared-memory staging of the material tables and the warp tile loop, common
// to the forward and backward persistent kernels.
//
// MODE_ALL_SMEM: every table is copied once per CTA by one TMA bulk copy;
//   records may come in any material order.
// MODE_SORTED:   records are grouped by material; each warp owns one table
//   slot and refills it (TMA bulk copy) when its tile's material changes.
// Work is handed out one warp tile (32 * items records) at a time from an
// atomic counter, so warps that drew cheap records take more tiles.
//
// Every wait on a table copy is bounded.  When one gives up, the error word
// records it, the copy is waited for once more (so that none is in flight
// when the CTA exits), and the warps keep taking tiles but only mark their
// records ST_ABORTED.  bars holds 2 * BLOCK / 32 barriers: the second half
// are the barriers of the test hook (a.test_stall), which nothing arrives on.
template <int BLOCK, class Body>
__device__ __forceinline__ void persistent_loop(const KArgs& a, uint8_t* smem, uint64_t* bars,
                                                Body&& body) {
  static_assert(BLOCK >= 64 && BLOCK % 32 == 0, "thread 32 claims the tile word");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#ifdef BYSDF_DEBUG_BOUNDS
  if (threadIdx.x == 0) g_bounds_word = &a.ctl->err_word;
  __syncthreads();
#endif
  uint64_t* stall = bars + BLOCK / 32;
  const uint32_t limit = a.wait_limit ? a.wait_limit : kWaitLimit;
  __shared__ int s_ok;
  bool aborted = false;
  // with claim_tiles the CTA claims the control words for its launch (else
  // k_plan set them): thread 0 the error word, before it can set an error
  // bit, and thread 32 the tile word, both while the table copies are in
  // flight; no warp draws a tile before the barrier after them
  if (a.mode == MODE_ALL_SMEM) {
    if (threadIdx.x == 32 && a.claim_tiles) {
      claim_word(&a.ctl->tile_word, a.epoch);
      __threadfence();
    }
    if (threadIdx.x == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&stall[0], 1);
      fence_mbar_init();
      // one bulk copy per table, each placed sstride bytes after the last:
      // the padding shifts every table's header to other banks, so lanes of
      // one round that read the same field of different materials' tables
      // do not collide in one bank
      mbar_arrive_tx(&bars[0], (uint32_t)a.n_mat * (uint32_t)a.stride);
      for (int k = 0; k < a.n_mat; ++k)
        bulk_g2s(smem + (size_t)k * a.sstride, a.table + (size_t)k * a.stride,
                 (uint32_t)a.stride, &bars[0]);
      if (a.claim_tiles) claim_word(&a.ctl->err_word, a.epoch);
      int ok = mbar_wait_bounded(a.test_stall ? &stall[0] : &bars[0], 0, a.ctl, ERR_TABLE_WAIT,
                                 limit);
      if (!ok) mbar_wait_bounded(&bars[0], 0, a.ctl, ERR_TABLE_INFLIGHT);
      s_ok = ok;
    }
    __syncthreads();
    aborted = !s_ok;
  } else {
    if (a.claim_tiles) {
      if (threadIdx.x == 0) {
        claim_word(&a.ctl->err_word, a.epoch);
        claim_word(&a.ctl->tile_word, a.epoch);
        __threadfence();
      }
      __syncthreads();
    }
    if (lane == 0) {
      mbar_init(&bars[warp], 1);
      mbar_init(&stall[warp], 1);
      fence_mbar_init();
    }
    __syncwarp();
  }
  const int64_t n_tiles = a.mode == MODE_SORTED ? (int64_t)__ldg(a.tile_start + a.n_mat)
                                                : a.n_tiles;
#ifdef BYSDF_DEBUG_BOUNDS
  {
    // the staged tables (all of them, or one slot per warp) lie inside the
    // launch's dynamic shared memory
    uint32_t dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const size_t need = a.mode == MODE_ALL_SMEM ? (size_t)a.n_mat * a.sstride
                                                : (size_t)(BLOCK / 32) * a.stride;
    if (threadIdx.x == 0) BY_BOUNDS(need <= dyn, (void)0);
  }
#endif
  uint8_t* slot = smem + (size_t)warp * a.stride;
  uint32_t parity = 0;
  int cur = -1;
  // Every warp draws until it gets a tile past the end, so a launch makes
  // exactly n_tiles + (its warps) draws.  With claim_tiles the warp that
  // makes the last one sets the word to 0, the state in which every launch
  // (a replay of a captured launch with the same epoch too) reclaims it.
  const unsigned long long tile_base =
      a.claim_tiles ? (unsigned long long)a.epoch << kEpochShift : 0ull;
  const unsigned long long last_draw =
      a.claim_tiles ? (unsigned long long)n_tiles + gridDim.x * (BLOCK / 32) - 1 : ~0ull;
  for (;;) {
    int tile = 0;
    if (lane == 0) {
      const unsigned long long t = atomicAdd(&a.ctl->tile_word, 1ull) - tile_base;
      if (t == last_draw) atomicExch(&a.ctl->tile_word, 0ull);
      tile = (int)t;
    }
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= n_tiles) break;
    int64_t begin, end;
    int mat = -1;
    if (a.mode == MODE_ALL_SMEM) {
      begin = (int64_t)tile * a.tile;
      end = begin + a.tile < a.n ? begin + a.tile : a.n;
    } else {
      int lo = 0, hi = a.n_mat;  // last material whose first tile <= tile
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(a.tile_start + mid) <= tile) lo = mid; else hi = mid;
      }
      mat = lo;
      BY_BOUNDS(mat >= 0 && mat < a.n_mat, mat = 0);
      // offsets outside [0, n] are clamped: no access outside the records
      int64_t s0 = __ldg(a.seg + mat), s1 = __ldg(a.seg + mat + 1);
      s0 = s0 < 0 ? 0 : s0;
      s1 = s1 > a.n ? a.n : s1;
      begin = s0 + (int64_t)(tile - __ldg(a.tile_start + mat)) * a.tile;
      end = begin + a.tile < s1 ? begin + a.tile : s1;
      if (end < begin) end = begin;
      if (!aborted && mat != cur) {
        __syncwarp();
        if (lane == 0) {
          fence_proxy_async();
          mbar_arrive_tx(&bars[warp], (uint32_t)a.stride);
          bulk_g2s(slot, a.table + (size_t)mat * a.stride, (uint32_t)a.stride, &bars[warp]);
        }
        bool ok = mbar_wait_bounded(a.test_stall ? &stall[warp] : &bars[warp], parity, a.ctl,
                                    ERR_TABLE_WAIT, limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (lane == 0) mbar_wait_bounded(&bars[warp], parity, a.ctl, ERR_TABLE_INFLIGHT);
          __syncwarp();
          aborted = true;
        } else {
          parity ^= 1u;
          cur = mat;
        }
      }
    }
    BY_BOUNDS(begin >= 0 && end <= a.n && begin <= end, begin = end = 0);
    if (aborted) {
      abort_tile(a, begin, end, lane);
      continue;
    }
    body(begin, end, mat, slot, lane, tile);
  }
}

// ---------------------------------------------------- work order in a tile --
// Lanes of a warp run in lock step, so a round costs as much as its most
// expensive record (most plies, most footprint nodes).  Records with a
// footprint (up to 16 geometry nodes each) are therefore taken in order of
// their loop structure: each record gets a bucket in [0, 32) and the tile is
// split into its buckets in ascending order.  Near-field records are taken
// in plain order: on them the order cost more than the uniform rounds gained
// (1.5% on 8 materials of 2 to 5 plies).  The split is a counting sort across the warp: lanes
// holding the same bucket are found by a match, one leader per group adds
// the group to the bucket's count in shared memory, a warp scan of the
// counts gives each bucket's start, and every record is written to its
// place in the warp's order list (element e = j * 32 + lane is item j of
// lane `lane`; ITEMS items per lane; records past the tile's end are
// listed as empty).
constexpr int kOrderBuckets = 32;

// Bucket of a record with a footprint: footprint nodes K (up to 16 told
// apart), then N_p above or below 4.
__device__ __forceinline__ uint32_t record_bucket(int K, int np) {
  return (uint32_t)(((K < 16 ? K : 16) - 1) * 2 + (np > 3 ? 1 : 0));
}

template <int ITEMS>
__device__ __forceinline__ void tile_order(const KArgs& a, const uint8_t* smem, int64_t begin,
                                           int64_t end, int mat, const uint8_t* slot, int lane,
                                           uint32_t* list, uint32_t* hist) {
  uint32_t b[ITEMS];
  bool valid[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const int idx = j * 32 + lane;
    const int64_t i = begin + idx;
    b[j] = kOrderBuckets - 1;
    valid[j] = i < end;
    if (valid[j]) {
      const MatDev* m;
      int mm = 0;
      if (mat >= 0) {
        m = reinterpret_cast<const MatDev*>(slot);
      } else {
        mm = a.mat_id ? __ldcg(a.mat_id + i) : 0;
        mm = (mm >= 0 && mm < a.n_mat) ? mm : 0;
        m = reinterpret_cast<const MatDev*>(smem + (size_t)mm * a.sstride);
      }
      const int K = footprint(__ldcg(a.h + i), __ldcg(a.ratio + i), m->kmax).K;
      b[j] = record_bucket(K, m->np);
    }
  }
  hist[lane] = 0u;
  __syncwarp();
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t rank[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t peers = __match_any_sync(0xffffffffu, b[j]);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&hist[b[j]], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    rank[j] = base + (uint32_t)__popc(peers & lt);
  }
  __syncwarp();
  // exclusive scan of the bucket counts (lane = bucket)
  const uint32_t h = hist[lane];
  uint32_t incl = h;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t start = incl - h;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t pos = __shfl_sync(0xffffffffu, start, (int)b[j]) + rank[j];
    list[pos] = valid[j] ? (uint32_t)(j * 32 + lane) : 0xffffffffu;
  }
  __syncwarp();
}

}  // namespace bysdf
