// Host side of libbysdf: the C ABI of include/bysdf.h.  Descriptor
// validation, the material table builder (layout, derived constants and the
// 1D fiber maps, computed in double on the host), workspace planning, kernel
// dispatch, the plain per-material form and the launch-shape autotuner.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "bysdf.h"
#include "bysdf_launch.h"

using namespace bysdf;

struct bysdf_materials {
  int device = 0;
  int n_mat = 0;
  int t_max = 0;
  int stride = 0;
  int sm_count = 0;
  size_t smem_optin = 0;
  uint8_t* d_table = nullptr;
  std::vector<bysdf_material_desc> desc;
  bysdf_launch_config cfg[BYSDF_NOPS];
  bool cfg_set[BYSDF_NOPS] = {};  // chosen by the caller or by bysdf_autotune
  // resident CTAs per SM of the forward launch shapes met so far, keyed by
  // (op bits, block, items, occupancy, dynamic shared memory): the query is
  // host time that a small batch would otherwise pay on every call
  struct OccEntry {
    int bits, block, items, occ;
    size_t smem;
    int ctas;
  };
  mutable std::mutex occ_mu;
  mutable std::vector<OccEntry> occ_cache;
  // test hook (bysdf_test_stall_table_waits): table waits of later calls poll
  // a barrier nothing arrives on and give up after this many polls; 0 = off
  uint32_t test_stall_polls = 0;
};

namespace {

constexpr double kPiD = 3.14159265358979323846;
// Tables up to this size are staged whole into each CTA's shared memory.
constexpr size_t kAllSmemMax = 48 * 1024;

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// Every device allocation of the library goes through dev_alloc.  Test hook
// (bysdf_test_fail_allocations): while g_fail_allocs > 0, an allocation
// takes one off it and fails as an exhausted device would, without calling
// cudaMalloc.
std::atomic<int32_t> g_fail_allocs{0};
cudaError_t dev_alloc(void** p, size_t bytes) {
  int32_t k = g_fail_allocs.load();
  while (k > 0)
    if (g_fail_allocs.compare_exchange_weak(k, k - 1)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

#define BY_CU(x)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess)                                                          \
      return fail(BYSDF_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));   \
  } while (0)

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// ------------------------------------------------------------- layout ----
// Reading of Sec. 3.4 / 3.5 (the paper gives no layout): N_p equal ply discs
// inscribed in the yarn circle and touching their neighbours; N_f fibers of
// one radius filling `packing` of a ply disc; the outer ring holds the fewest
// fibers whose circles close it.
struct HostLayout {
  double R, Rp, Rc, rf, Rfc;
  int M;
  int K;                   // migration map pairs (1: none)
  double Rfc_m[4];         // ring radius and fiber count of each map
  int M_m[4];
};

bool host_layout(const bysdf_material_desc& d, HostLayout* L, std::string* why) {
  auto bad = [&](const char* s) {
    *why = s;
    return false;
  };
  auto fin = [](double x) { return std::isfinite(x); };
  if (d.n_plies < 1 || d.n_plies > kMaxPlies) return bad("n_plies outside [1, 8]");
  if (d.fibers_per_ply < 4 || d.fibers_per_ply > 4096) return bad("fibers_per_ply outside [4, 4096]");
  if (d.map_texels < 4 || d.map_texels > kMaxTexels) return bad("map_texels outside [4, 1024]");
  if (d.trace_iters < 1 || d.trace_iters > 64) return bad("trace_iters outside [1, 64]");
  if (d.k_max < 1 || d.k_max > 64) return bad("k_max outside [1, 64]");
  if (!(d.yarn_radius > 0.f) || !fin(d.yarn_radius)) return bad("yarn_radius must be > 0");
  if (!(d.eta > 1.f) || !fin(d.eta)) return bad("eta must be > 1");
  if (!(d.packing > 0.f && d.packing <= 1.f)) return bad("packing outside (0, 1]");
  if (!(d.body_B >= 0.f && d.body_B <= 1.f)) return bad("body_B outside [0, 1]");
  if (!(d.body_r >= 0.f && d.body_r <= 1.f)) return bad("body_r outside [0, 1]");
  if (!(d.k_spec >= 0.f) || !fin(d.k_spec)) return bad("k_spec must be >= 0");
  if (!(d.sigma_t >= 0.f) || !fin(d.sigma_t)) return bad("sigma_t must be >= 0");
  if (!(d.shadow_density >= 0.f) || !fin(d.shadow_density)) return bad("shadow_density must be >= 0");
  for (int c = 0; c < 3; ++c) {
    if (!fin(d.albedo[c])) return bad("albedo must be finite");
    if (!fin(d.albedo_y[c])) return bad("albedo_y must be finite (negative: equal to albedo)");
  }
  for (int c = 0; c < 2; ++c)
    if (!fin(d.beta_deg[c])) return bad("beta_deg must be finite");
  if (!fin(d.ply_twist_deg) || std::fabs(d.ply_twist_deg) >= 89.f) return bad("ply_twist_deg outside (-89, 89)");
  if (!fin(d.fiber_twist_deg) || std::fabs(d.fiber_twist_deg) >= 89.f)
    return bad("fiber_twist_deg outside (-89, 89)");
  L->R = d.yarn_radius;
  if (d.n_plies == 1) {
    L->Rp = L->R;
    L->Rc = 0.0;
  } else {
    const double s = std::sin(kPiD / d.n_plies);
    L->Rc = L->R / (1.0 + s);
    L->Rp = L->Rc * s;
  }
  L->rf = L->Rp * std::sqrt((double)d.packing / (double)d.fibers_per_ply);
  L->Rfc = L->Rp - L->rf;
  if (!(L->rf < L->Rfc)) return bad("fibers too thick for the ply (raise fibers_per_ply)");
  L->M = (int)std::ceil(kPiD / std::asin(L->rf / L->Rfc));
  // fiber migration: map k is the ring sunk by k r_f / K_m
  L->K = d.migration_maps < 1 ? 1 : d.migration_maps;
  if (L->K > 4) return bad("migration_maps outside [0, 4]");
  if (L->K > 1) {
    if (!(d.migration_length > 0.f) || !fin(d.migration_length))
      return bad("migration_length must be > 0");
    if (!(d.migration_blend > 0.f && d.migration_blend <= 0.5f))
      return bad("migration_blend outside (0, 0.5]");
  }
  for (int k = 0; k < L->K; ++k) {
    L->Rfc_m[k] = L->Rfc - k * L->rf / L->K;
    if (!(L->rf < L->Rfc_m[k])) return bad("migration ring too deep for the fibers");
    L->M_m[k] = k == 0 ? L->M : (int)std::ceil(kPiD / std::asin(L->rf / L->Rfc_m[k]));
  }
  return true;
}

// Philox4x64-10 (Salmon et al. 2011) on the host: the segment table of the
// fiber migration (map index of segment s = word 0 of counter (s, 0, 0, 0),
// key (seed, 0xB15DF000F1BE0002), mod K_m).
uint64_t philox4x64_word0(uint64_t c0, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t c[4] = {c0, 0, 0, 0};
  for (int r = 0; r < 10; ++r) {
    const unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
    const unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
    const uint64_t n0 = (uint64_t)(p1 >> 64) ^ c[1] ^ k0;
    const uint64_t n2 = (uint64_t)(p0 >> 64) ^ c[3] ^ k1;
    c[1] = (uint64_t)p1;
    c[3] = (uint64_t)p0;
    c[0] = n0;
    c[2] = n2;
    k0 += W0;
    k1 += W1;
  }
  return c[0];
}

// ------------------------------------------------------------ fiber maps --
// Sec. 3.5.1: along the radial line at angular offset D from a fiber centre
// the outer fiber surface has normal tilted by delta from the radial
// direction.  Sec. 4.1.4: o_f is the share of the outward half-plane of
// directions at that point hidden by the other fibers of the ring.
double map_delta(const HostLayout& L, double D) {
  const double sd = L.Rfc * std::sin(D);
  return std::atan2(sd, std::sqrt(std::max(0.0, L.rf * L.rf - sd * sd)));
}

double map_occlusion(const HostLayout& L, double D) {
  const double sd = L.Rfc * std::sin(D);
  const double rho = L.Rfc * std::cos(D) + std::sqrt(std::max(0.0, L.rf * L.rf - sd * sd));
  const double px = rho * std::cos(D), py = rho * std::sin(D);
  const double normal_angle = std::atan2(py, px - L.Rfc);
  // sweep over interval end points ("events") inside [-pi/2, pi/2]
  std::vector<std::pair<double, int>> ev;
  for (int j = 1; j < L.M; ++j) {
    const double cj = 2.0 * kPiD * j / L.M;
    const double dx = L.Rfc * std::cos(cj) - px, dy = L.Rfc * std::sin(cj) - py;
    const double dist = std::hypot(dx, dy);
    const double half = dist > L.rf ? std::asin(L.rf / dist) : 0.5 * kPiD;
    double mid = std::remainder(std::atan2(dy, dx) - normal_angle, 2.0 * kPiD);
    for (double shift : {-2.0 * kPiD, 0.0, 2.0 * kPiD}) {
      const double a = std::max(mid + shift - half, -0.5 * kPiD);
      const double b = std::min(mid + shift + half, 0.5 * kPiD);
      if (b > a) {
        ev.push_back({a, +1});
        ev.push_back({b, -1});
      }
    }
  }
  std::sort(ev.begin(), ev.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first < y.first || (x.first == y.first && x.second > y.second);
  });
  double covered = 0.0, start = 0.0;
  int depth = 0;
  for (const auto& e : ev) {
    if (depth == 0 && e.second > 0) start = e.first;
    depth += e.second;
    if (depth == 0 && e.second < 0) covered += e.first - start;
  }
  return covered / kPiD;
}

// Derived constants from the 15 parameters of the extended set (radians),
// shared by table creation on the host and parameter updates on the device.
__host__ __device__ void split_hi_lo(double x, float* hi, float* lo) {
  *hi = (float)x;
  *lo = (float)(x - (double)*hi);
}

__host__ __device__ void derive_constants(MatDev& m, const double* p) {
  const double two_pi = 2.0 * 3.14159265358979323846;
  m.alb[0] = (float)p[0];
  m.alb[1] = (float)p[1];
  m.alb[2] = (float)p[2];
  m.beta_t = (float)p[3];
  m.beta_b = (float)p[4];
  m.alpha_p = (float)p[5];
  m.alpha_f = (float)p[6];
  m.sigma_s = (float)p[7];
  m.r = (float)p[8];
  m.alb_y[0] = (float)p[9];
  m.alb_y[1] = (float)p[10];
  m.alb_y[2] = (float)p[11];
  m.sigma_t = (float)p[12];
  m.B = (float)p[13];
  m.k_spec = (float)p[14];
  m.ks = (float)((1.0 - p[13]) * p[14]);
  if (m.np == 1) {
    m.kp_hi = m.kp_lo = 0.f;
    m.dkp = 0.f;
  } else {
    const double t = tan(p[5]);
    split_hi_lo(t / (two_pi * m.Rc_d), &m.kp_hi, &m.kp_lo);
    m.dkp = (float)((1.0 + t * t) / (two_pi * m.Rc_d));
  }
  const double tf = tan(p[6]);
  split_hi_lo(tf * m.M / (two_pi * m.Rfc_d), &m.kf_hi, &m.kf_lo);
  m.dkf = (float)((1.0 + tf * tf) * m.M / (two_pi * m.Rfc_d));
  // fiber migration maps: the same helix angle on their sunk rings
  for (int k = 1; k < m.mig_maps; ++k) {
    MigMap* mm = mig_map(m, k);
    split_hi_lo(tf * mm->M / (two_pi * mm->Rfc_d), &mm->kf_hi, &mm->kf_lo);
    mm->dkf = (float)((1.0 + tf * tf) * mm->M / (two_pi * mm->Rfc_d));
  }
  m.cos_af = (float)cos(p[6]);
  m.sin_af = (float)sin(p[6]);
}

// The 15 parameters of a table entry (the extended layout of the C ABI).
__host__ __device__ void read_params(const MatDev& m, double* p) {
  p[0] = m.alb[0];
  p[1] = m.alb[1];
  p[2] = m.alb[2];
  p[3] = m.beta_t;
  p[4] = m.beta_b;
  p[5] = m.alpha_p;
  p[6] = m.alpha_f;
  p[7] = m.sigma_s;
  p[8] = m.r;
  p[9] = m.alb_y[0];
  p[10] = m.alb_y[1];
  p[11] = m.alb_y[2];
  p[12] = m.sigma_t;
  p[13] = m.B;
  p[14] = m.k_spec;
}

// ncol 8: the first 8 parameters, k^B_y set to the albedo, the rest kept;
// ncol 15: all.
__global__ void k_update_params(uint8_t* table, int n_mat, int stride, const float* params,
                                int ncol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_mat) return;
  MatDev* m = reinterpret_cast<MatDev*>(table + (size_t)i * stride);
  double p[BYSDF_NPARAM_EXT];
  read_params(*m, p);
  for (int k = 0; k < ncol; ++k) p[k] = (double)params[(size_t)i * ncol + k];
  if (ncol == BYSDF_NPARAM) {
    p[9] = p[0];
    p[10] = p[1];
    p[11] = p[2];
  }
  derive_constants(*m, p);
}

__global__ void k_read_params(const uint8_t* table, int n_mat, int stride, float* params,
                              int ncol) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_mat) return;
  const MatDev* m = reinterpret_cast<const MatDev*>(table + (size_t)i * stride);
  double p[BYSDF_NPARAM_EXT];
  read_params(*m, p);
  for (int k = 0; k < ncol; ++k) params[(size_t)i * ncol + k] = (float)p[k];
}

// Tile plan: set the control words for the launch's epoch (tile draws
// counted from 0, no error); for material-sorted records also the first
// warp tile of every material (exclusive scan of ceil(count / tile)).
__global__ void __launch_bounds__(1024) k_plan(WsCtl* ctl, int32_t* tile_start,
                                               const int64_t* seg, int n_mat, int tile,
                                               unsigned long long epoch) {
  __shared__ int64_t part[1024];
  const int tid = threadIdx.x;
  if (seg != nullptr) {
    const int chunk = (n_mat + 1023) / 1024;
    const int b = min(tid * chunk, n_mat), e = min(b + chunk, n_mat);
    int64_t s = 0;
    for (int m = b; m < e; ++m) {
      const int64_t c = seg[m + 1] - seg[m];
      s += c > 0 ? (c + tile - 1) / tile : 0;
    }
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int64_t v = tid >= off ? part[tid - off] : 0;
      __syncthreads();
      part[tid] += v;
      __syncthreads();
    }
    int64_t run = part[tid] - s;  // exclusive prefix
    for (int m = b; m < e; ++m) {
      tile_start[m] = (int32_t)run;
      const int64_t c = seg[m + 1] - seg[m];
      run += c > 0 ? (c + tile - 1) / tile : 0;
    }
    if (tid == 1023) tile_start[n_mat] = (int32_t)part[1023];
  }
  if (tid == 0) {
    ctl->tile_word = 0ull;
    ctl->err_word = epoch << kEpochShift;
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes between two materials' tables when all of them sit in shared
// memory: the table stride plus 16, so that successive tables start four
// banks apart.
size_t smem_stride(const bysdf_materials* m) { return (size_t)m->stride + 16; }
size_t ws_tile_start_off() { return kWsCtl; }
size_t ws_partials_off(int n_mat) { return align_up(kWsCtl + 4 * (size_t)(n_mat + 1), 256); }
int64_t max_tiles(int64_t n, int n_mat) { return (n + 31) / 32 + n_mat; }

// Defaults measured on GB300 with the benchmark workloads (eval + sample +
// pdf over 2^24 records; forward + backward over 2^24 material-sorted
// records of 64 materials): 16 warps per SM in CTAs of 512; four records
// per lane per warp tile for the forward calls (two or eight within 0.3%),
// sixteen for the backward (the fused L2 pass per 2^24 records 2.25 ms,
// against 2.28 ms at eight, 2.53 ms at four and 3.12 ms at two, at the
// kernels of their times).  bysdf_autotune refines them for a given record
// set.
bysdf_launch_config default_cfg(int op) {
  bysdf_launch_config c;
  c.block = 512;
  c.items = op == BYSDF_OP_BACKWARD ? 16 : 4;
  c.ctas_per_sm = 0;  // 0: as many as fit
  c.occupancy = 0;
  return c;
}

// Records with a footprint run up to 16 geometry nodes each: their default
// shape holds more warps per SM (24, registers capped) and tiles of 256
// records, so that the sort gives each round records of equal loop counts.
bysdf_launch_config footprint_default_cfg() {
  bysdf_launch_config c;
  c.block = 256;
  c.items = 8;
  c.ctas_per_sm = 0;
  c.occupancy = 1;
  return c;
}

// The shape of a forward call: the caller's (or the tuned) one when set,
// else the default for the kind of records.
bysdf_launch_config fwd_cfg(const bysdf_materials* m, int op, const bysdf_hits* h) {
  if (m->cfg_set[op] || !h || !h->ratio) return m->cfg[op];
  return footprint_default_cfg();
}

int check_hits(const bysdf_materials* m, const bysdf_hits* h, bool need_wo, int64_t n) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  if (!h) return fail(BYSDF_E_ARG, "hits is NULL");
  if (n < 0) return fail(BYSDF_E_ARG, "n < 0");
  if (n == 0) return BYSDF_OK;
  if (n > ((int64_t)1 << 36)) return fail(BYSDF_E_ARG, "n too large");
  if (!h->h || !h->u || !h->v || !h->wi) return fail(BYSDF_E_ARG, "hits: h, u, v, wi required");
  if (need_wo && !h->wo) return fail(BYSDF_E_ARG, "hits: wo required");
  const void* ps[] = {h->h, h->u, h->v, h->wi, need_wo ? h->wo : nullptr, h->ratio, h->mat_id,
                      h->seg_offsets};
  for (const void* p : ps)
    if (p && !aligned16(p)) return fail(BYSDF_E_ARG, "hits: buffer not 16-byte aligned");
  return BYSDF_OK;
}

int check_out(const void* p, const char* name) {
  if (!p) return fail(BYSDF_E_ARG, std::string(name) + " is NULL");
  if (!aligned16(p)) return fail(BYSDF_E_ARG, std::string(name) + " not 16-byte aligned");
  return BYSDF_OK;
}

// Common preparation of a persistent launch.
int prepare(const bysdf_materials* m, const bysdf_hits* h, int64_t n, void* ws, size_t ws_bytes,
            int block, int items, KArgs* a, size_t ws_need) {
  std::memset(a, 0, sizeof(*a));
  a->table = m->d_table;
  a->n_mat = m->n_mat;
  a->stride = m->stride;
  a->sstride = smem_stride(m);
  a->n = n;
  a->tile = 32 * items;
  a->h = h->h;
  a->u = h->u;
  a->v = h->v;
  a->wi = h->wi;
  a->wo = h->wo;
  a->ratio = h->ratio;
  a->mat_id = h->mat_id;
  a->seg = h->seg_offsets;
  if (h->seg_offsets) {
    a->mode = MODE_SORTED;
  } else if ((size_t)m->n_mat * smem_stride(m) <= kAllSmemMax) {
    a->mode = MODE_ALL_SMEM;
  } else {
    return fail(BYSDF_E_UNSUPPORTED,
                "tables do not fit in shared memory: pass material-sorted records with seg_offsets");
  }
  a->n_tiles = (n + a->tile - 1) / a->tile;
  if (!ws) return fail(BYSDF_E_WORKSPACE, "workspace is NULL");
  if (!aligned16(ws)) return fail(BYSDF_E_ARG, "workspace not 16-byte aligned");
  if (ws_bytes < ws_need)
    return fail(BYSDF_E_WORKSPACE, "workspace smaller than bysdf_workspace_size()");
  a->ctl = reinterpret_cast<WsCtl*>(ws);
  a->tile_start = reinterpret_cast<const int32_t*>((uint8_t*)ws + ws_tile_start_off());
  a->wait_limit = m->test_stall_polls ? m->test_stall_polls : kWaitLimit;
  a->test_stall = m->test_stall_polls ? 1u : 0u;
  (void)block;
  return BYSDF_OK;
}

// A new epoch for every launch that uses a workspace's control words: 40
// bits, never 0, increasing through the process (it wraps after 2^40
// launches).
uint64_t next_epoch() {
  static std::atomic<uint64_t> counter{0};
  for (;;) {
    const uint64_t e = (counter.fetch_add(1, std::memory_order_relaxed) + 1) &
                       ((1ull << (64 - kEpochShift)) - 1);
    if (e) return e;
  }
}

// Gives the launch its epoch.  Records in any order, with fewer than 2^24
// tile draws (tiles plus one final draw per warp): the launch claims the
// control words itself and nothing else is launched.  Otherwise k_plan runs
// first (for material-sorted records it also computes the first tile of
// every material).
int plan(const bysdf_materials* m, KArgs& a, void* ws, cudaStream_t st, int64_t grid_warps) {
  a.epoch = next_epoch();
  a.claim_tiles = a.mode != MODE_SORTED && a.n_tiles + grid_warps < (1ll << kEpochShift);
  if (a.claim_tiles) return BYSDF_OK;
  k_plan<<<1, 1024, 0, st>>>(a.ctl, reinterpret_cast<int32_t*>((uint8_t*)ws + ws_tile_start_off()),
                             a.mode == MODE_SORTED ? a.seg : nullptr, m->n_mat, a.tile,
                             (unsigned long long)a.epoch);
  BY_CU(cudaGetLastError());
  return BYSDF_OK;
}

cudaError_t cached_forward_occupancy(const bysdf_materials* m, int bits, int block, int items,
                                     int occ, size_t smem, int* ctas) {
  std::lock_guard<std::mutex> lock(m->occ_mu);
  for (const auto& e : m->occ_cache)
    if (e.bits == bits && e.block == block && e.items == items && e.occ == occ && e.smem == smem) {
      *ctas = e.ctas;
      return cudaSuccess;
    }
  const cudaError_t err = forward_occupancy(bits, block, items, occ, smem, ctas);
  if (err == cudaSuccess) m->occ_cache.push_back({bits, block, items, occ, smem, *ctas});
  return err;
}

int grid_for(const bysdf_materials* m, const bysdf_launch_config& c, int occ) {
  int per_sm = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, std::max(occ, 1)) : std::max(occ, 1);
  return m->sm_count * per_sm;
}

int op_bits(int op) {
  switch (op) {
    case BYSDF_OP_EVAL: return OPF_EVAL;
    case BYSDF_OP_SAMPLE: return OPF_SAMPLE;
    case BYSDF_OP_PDF: return OPF_PDF;
    case BYSDF_OP_FUSED: return OPF_EVAL | OPF_SAMPLE;
  }
  return 0;
}

// sto: the stochastic estimators (flags != 0), eval and fused ops only
int run_forward(const bysdf_materials* m, int op, const bysdf_hits* h, const float* u0,
                const float* u1, int64_t n, const bysdf_outputs& o, void* ws, size_t ws_bytes,
                cudaStream_t st, const bysdf_launch_config& cfg, size_t ws_need = 0,
                const bysdf_stochastic* sto = nullptr) {
  int bits = op_bits(op);
  bysdf_launch_config c = cfg;
  if (sto && sto->flags) {
    if (sto->flags & ~(uint32_t)(BYSDF_STOCH_JITTER_NODES | BYSDF_STOCH_ROUGH_ENTRY))
      return fail(BYSDF_E_ARG, "unknown stochastic flags");
    if (op != BYSDF_OP_EVAL && op != BYSDF_OP_FUSED)
      return fail(BYSDF_E_UNSUPPORTED, "stochastic estimators: eval and the fused op only");
    bits |= OPF_STOCH;
  }
  const bool need_wo = (bits & (OPF_EVAL | OPF_PDF)) != 0;
  int rc = check_hits(m, h, need_wo, n);
  if (rc) return rc;
  if (n == 0) return BYSDF_OK;
  if (bits & OPF_EVAL) {
    if ((rc = check_out(o.f_rgb, "f_rgb"))) return rc;
  }
  if (bits & (OPF_EVAL | OPF_PDF)) {
    if ((rc = check_out(o.status, "status"))) return rc;
    if ((bits & OPF_PDF) && (rc = check_out(o.pdf, "pdf"))) return rc;
    if (o.pdf && !aligned16(o.pdf)) return fail(BYSDF_E_ARG, "pdf not 16-byte aligned");
  }
  if (bits & OPF_SAMPLE) {
    if ((rc = check_out(u0, "u0")) || (rc = check_out(u1, "u1"))) return rc;
    if ((rc = check_out(o.wo, "wo")) || (rc = check_out(o.weight, "weight")) ||
        (rc = check_out(o.pdf_s, "pdf (sample)")) || (rc = check_out(o.lobe_status, "lobe_status")))
      return rc;
  }
  KArgs a;
  if ((rc = prepare(m, h, n, ws, ws_bytes, c.block, c.items, &a,
                    ws_need ? ws_need : bysdf_workspace_size(m, n))))
    return rc;
  if (!(bits & OPF_SAMPLE) || bits == (OPF_EVAL | OPF_SAMPLE)) a.wo = h->wo;
  if (bits == OPF_SAMPLE) a.wo = nullptr;
  a.u0 = u0;
  a.u1 = u1;
  a.f_rgb = o.f_rgb;
  a.pdf = o.pdf;
  a.status = o.status;
  a.wo_s = o.wo;
  a.weight_s = o.weight;
  a.pdf_s = o.pdf_s;
  a.lstat_s = o.lobe_status;
  if (bits & OPF_STOCH) {
    a.stoch_seed = sto->seed;
    a.stoch_index0 = sto->index_offset;
    a.stoch_flags = sto->flags;
  }
  // tables, then each warp's tile order list (4 bytes per record of a tile)
  // and bucket counts
  const size_t tables = a.mode == MODE_ALL_SMEM ? (size_t)m->n_mat * a.sstride
                                                : (size_t)(c.block / 32) * m->stride;
  a.order_off = (int32_t)align_up(tables, 16);
  auto key_bytes = [&](int items) {
    return sizeof(uint32_t) * (size_t)(c.block / 32) * (32 * (size_t)items + kOrderBuckets);
  };
  size_t smem = (size_t)a.order_off + key_bytes(c.items);
  if (smem > m->smem_optin) return fail(BYSDF_E_UNSUPPORTED, "material table too large for shared memory");
  if (smem > 48 * 1024) BY_CU(set_forward_smem_limit(bits, c.block, c.items, c.occupancy, smem));
  int occ = 0;
  BY_CU(cached_forward_occupancy(m, bits, c.block, c.items, c.occupancy, smem, &occ));
  // fewer warp tiles than resident warps leaves warps idle: tiles of 32
  // records spread a small batch over twice (or four times) as many warps
  const int64_t warps = (int64_t)grid_for(m, c, occ) * (c.block / 32);
  if (c.items > 1 && a.n_tiles < warps) {
    c.items = 1;
    a.tile = 32;
    a.n_tiles = (n + 31) / 32;
    smem = (size_t)a.order_off + key_bytes(1);
    if (smem > 48 * 1024) BY_CU(set_forward_smem_limit(bits, c.block, 1, c.occupancy, smem));
    BY_CU(cached_forward_occupancy(m, bits, c.block, 1, c.occupancy, smem, &occ));
  }
  const int grid = grid_for(m, c, occ);
  if ((rc = plan(m, a, ws, st, (int64_t)grid * (c.block / 32)))) return rc;
  BY_CU(launch_forward(bits, a, c.block, c.occupancy, grid, smem, st));
  return BYSDF_OK;
}

int set_params(bysdf_materials* m, const float* params, int ncol, void* stream) {
  if (!m || !params) return fail(BYSDF_E_ARG, "materials and params must not be NULL");
  if ((uintptr_t)params & 3u) return fail(BYSDF_E_ARG, "params must be 4-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_update_params<<<(m->n_mat + 127) / 128, 128, 0, st>>>(m->d_table, m->n_mat, m->stride,
                                                          params, ncol);
  BY_CU(cudaGetLastError());
  return BYSDF_OK;
}

int get_params(const bysdf_materials* m, float* params, int ncol, void* stream) {
  if (!m || !params) return fail(BYSDF_E_ARG, "materials and params must not be NULL");
  if ((uintptr_t)params & 3u) return fail(BYSDF_E_ARG, "params must be 4-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_read_params<<<(m->n_mat + 127) / 128, 128, 0, st>>>(m->d_table, m->n_mat, m->stride,
                                                        params, ncol);
  BY_CU(cudaGetLastError());
  return BYSDF_OK;
}

// kind: KB_BASIC (8 gradient columns), KB_EXT (15) or KB_L2 (8, upstream
// gradient of the L2 loss against l2->target); grad_wi / grad_wo: direction
// vector-Jacobian products (extended call only), each optional.
struct L2Args {
  const float* target;
  const float* weight;
  float* f_rgb;
  float* loss_mat;
};
int run_backward(const bysdf_materials* m, const bysdf_hits* h, int64_t n, const float* grad_f,
                 float* grad_params, int deterministic, void* ws, size_t ws_bytes,
                 cudaStream_t st, const bysdf_launch_config& cfg, int kind = KB_BASIC,
                 float* grad_wi = nullptr, float* grad_wo = nullptr,
                 const L2Args* l2 = nullptr) {
  bysdf_launch_config c = cfg;
  const bool ext = kind == KB_EXT;
  const int ng = ext ? BYSDF_NPARAM_EXT : BYSDF_NPARAM;   // gradient columns
  const int np = kind == KB_L2 ? ng + 1 : ng;             // accumulated columns
  int rc = check_hits(m, h, true, n);
  if (rc) return rc;
  if ((rc = check_out(grad_params, "grad_params"))) return rc;
  if (kind == KB_L2) {
    if (n > 0 && (rc = check_out(l2->target, "target"))) return rc;
    if (l2->weight && !aligned16(l2->weight)) return fail(BYSDF_E_ARG, "weight not 16-byte aligned");
    if (l2->f_rgb && !aligned16(l2->f_rgb)) return fail(BYSDF_E_ARG, "f_rgb not 16-byte aligned");
    if (l2->loss_mat && ((uintptr_t)l2->loss_mat & 3u))
      return fail(BYSDF_E_ARG, "loss_mat not 4-byte aligned");
  } else if (n > 0 && (rc = check_out(grad_f, "grad_f"))) {
    return rc;
  }
  if (grad_wi && (rc = check_out(grad_wi, "grad_wi"))) return rc;
  if (grad_wo && (rc = check_out(grad_wo, "grad_wo"))) return rc;
  if (deterministic && !h->seg_offsets)
    return fail(BYSDF_E_UNSUPPORTED, "deterministic backward needs material-sorted records");
  if (kind == KB_L2 && l2->loss_mat && (n == 0 || !deterministic))
    BY_CU(cudaMemsetAsync(l2->loss_mat, 0, sizeof(float) * m->n_mat, st));
  if (n == 0) {
    BY_CU(cudaMemsetAsync(grad_params, 0, sizeof(float) * ng * m->n_mat, st));
    return BYSDF_OK;
  }
  KArgs a;
  if ((rc = prepare(m, h, n, ws, ws_bytes, c.block, c.items, &a, bysdf_workspace_size(m, n))))
    return rc;
  a.grad_f = grad_f;
  a.grad_params = grad_params;
  a.n_param = np;
  if (kind == KB_L2) {
    a.target = l2->target;
    a.weight = l2->weight;
    a.f_rgb = l2->f_rgb;
    a.loss_mat = l2->loss_mat;
  }
  a.partials = deterministic ? reinterpret_cast<float*>((uint8_t*)ws + ws_partials_off(m->n_mat))
                             : nullptr;
  const size_t smem = a.mode == MODE_ALL_SMEM
                          ? (size_t)m->n_mat * a.sstride + sizeof(float) * np * m->n_mat
                          : (size_t)(c.block / 32) * m->stride;
  if (smem > m->smem_optin) return fail(BYSDF_E_UNSUPPORTED, "material table too large for shared memory");
  if (smem > 48 * 1024) BY_CU(set_backward_smem_limit(c.block, c.occupancy, kind, smem));
  int occ = 0;
  BY_CU(backward_occupancy(c.block, c.occupancy, kind, smem, &occ));
  if (!deterministic) BY_CU(cudaMemsetAsync(grad_params, 0, sizeof(float) * ng * m->n_mat, st));
  const int grid = grid_for(m, c, occ);
  // fewer warp tiles than resident warps leaves warps idle: the tile is
  // halved until the batch covers them (n / tile tiles for records in any
  // order; material-sorted records have at least as many)
  const int64_t warps = (int64_t)grid * (c.block / 32);
  while (c.items > 1 && (n + 32 * c.items - 1) / (32 * c.items) < warps) c.items /= 2;
  a.tile = 32 * c.items;
  a.n_tiles = (n + a.tile - 1) / a.tile;
  if ((rc = plan(m, a, ws, st, warps))) return rc;
  BY_CU(launch_backward(a, c.block, c.occupancy, kind, grid, smem, st));
  if (deterministic) BY_CU(launch_reduce_partials(a, st));
  if (grad_wi || grad_wo) {
    // second pass: the direction products (its own tile plan)
    a.grad_wi = grad_wi;
    a.grad_wo = grad_wo;
    const size_t smem_d = a.mode == MODE_ALL_SMEM ? (size_t)m->n_mat * a.sstride
                                                  : (size_t)(c.block / 32) * m->stride;
    if (smem_d > 48 * 1024) BY_CU(set_dirgrad_smem_limit(c.block, smem_d));
    int occ_d = 0;
    BY_CU(dirgrad_occupancy(c.block, smem_d, &occ_d));
    const int grid_d = grid_for(m, c, occ_d);
    if ((rc = plan(m, a, ws, st, (int64_t)grid_d * (c.block / 32)))) return rc;
    BY_CU(launch_dirgrad(a, c.block, grid_d, smem_d, st));
  }
  return BYSDF_OK;
}

}  // namespace

// Scratch of bysdf_eval_noalloc: one fixed array per device that loads the
// library (kept until the process exits).  Host code must not use its name
// as an address: the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) uint8_t g_noalloc_scratch[BYSDF_NOALLOC_SCRATCH_BYTES];

namespace {
// Tables of at most this many materials fit the scratch: the control words
// and one first-tile entry per material (plus the end entry).
constexpr int kNoallocMaxMaterials =
    (int)((BYSDF_NOALLOC_SCRATCH_BYTES - kWsCtl) / sizeof(int32_t)) - 1;
static_assert(BYSDF_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch in whole 256-byte units");
static_assert(kNoallocMaxMaterials == BYSDF_NOALLOC_MAX_MATERIALS,
              "bysdf.h states the material limit of the no-allocation call");

// Device address of the scratch array on the current device, looked up on
// every call with that device current (after a device reset the module, and
// so the array, may sit elsewhere).
int noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return fail(BYSDF_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  *out = p;
  return BYSDF_OK;
}
}  // namespace

// =================================================================== C ABI ==
extern "C" {

const char* bysdf_version(void) { return "libbysdf 0.1 (sm_103a)"; }

const char* bysdf_last_error(void) { return g_err.c_str(); }

int bysdf_create_materials(const bysdf_material_desc* desc, int32_t n, void* stream,
                           bysdf_materials** out) {
  if (!desc || !out) return fail(BYSDF_E_ARG, "desc and out must not be NULL");
  if (n < 1 || n > 65536) return fail(BYSDF_E_ARG, "n outside [1, 65536]");
  *out = nullptr;
  std::vector<HostLayout> L(n);
  int t_max = 0;
  for (int i = 0; i < n; ++i) {
    std::string why;
    if (!host_layout(desc[i], &L[i], &why))
      return fail(BYSDF_E_ARG, "material " + std::to_string(i) + ": " + why);
    t_max = std::max(t_max, desc[i].map_texels);
  }
  size_t stride = 0;
  for (int i = 0; i < n; ++i)
    stride = std::max(stride, mat_bytes(desc[i].map_texels, L[i].K));
  stride = (stride + 15) / 16 * 16;
  std::vector<uint8_t> host(stride * n, 0);
  for (int i = 0; i < n; ++i) {
    const bysdf_material_desc& d = desc[i];
    MatDev& m = *reinterpret_cast<MatDev*>(host.data() + stride * i);
    m.np = d.n_plies;
    m.M = L[i].M;
    m.T = d.map_texels;
    m.nit = d.trace_iters;
    m.kmax = d.k_max;
    m.flags = d.flags;
    m.R = (float)L[i].R;
    m.Rp = (float)L[i].Rp;
    m.Rc = (float)L[i].Rc;
    m.Rfc = (float)L[i].Rfc;
    m.Rc_d = L[i].Rc;
    m.Rfc_d = L[i].Rfc;
    m.eta = d.eta;
    m.inv_eta = (float)(1.0 / (double)d.eta);
    m.inv_2Rp = (float)(0.5 / L[i].Rp);
    m.m_over_2pi = (float)(L[i].M / (2.0 * kPiD));
    m.inv_np = (float)(1.0 / d.n_plies);
    m.mig_maps = L[i].K;
    m.mig_seed = d.migration_seed;
    float inv_len_lo = 0.f;
    if (L[i].K > 1) {
      split_hi_lo(1.0 / (double)d.migration_length, &m.mig_inv_len, &inv_len_lo);
      m.mig_blend = d.migration_blend;
      m.mig_inv_2b = (float)(0.5 / (double)d.migration_blend);
    }
    for (int k = 1; k < L[i].K; ++k) {
      MigMap* mm = mig_map(m, k);
      mm->m_over_2pi = (float)(L[i].M_m[k] / (2.0 * kPiD));
      mm->Rfc_d = L[i].Rfc_m[k];
      mm->M = (float)L[i].M_m[k];
      mm->aux = k == 1 ? inv_len_lo : 0.f;
    }
    if (L[i].K > 1) {
      uint8_t* tab = const_cast<uint8_t*>(mig_table(m));
      for (int sg = 0; sg < kMigPeriod; ++sg)
        tab[sg] = (uint8_t)(philox4x64_word0((uint64_t)sg, (uint64_t)(uint32_t)d.migration_seed,
                                             kMigKey1) % (uint64_t)L[i].K);
    }
    for (int j = 0; j < kMaxPlies; ++j) {
      m.rot_c[j] = (float)std::cos(2.0 * kPiD * j / d.n_plies);
      m.rot_s[j] = (float)std::sin(2.0 * kPiD * j / d.n_plies);
    }
    const double deg = kPiD / 180.0;
    double p[BYSDF_NPARAM_EXT] = {d.albedo[0], d.albedo[1], d.albedo[2], d.beta_deg[0] * deg,
                                  d.beta_deg[1] * deg, d.ply_twist_deg * deg,
                                  d.fiber_twist_deg * deg, d.shadow_density, d.body_r,
                                  d.albedo[0], d.albedo[1], d.albedo[2], d.sigma_t, d.body_B,
                                  d.k_spec};
    for (int c = 0; c < 3; ++c)
      if (d.albedo_y[c] >= 0.f) p[9 + c] = d.albedo_y[c];
    derive_constants(m, p);
    float2* map = reinterpret_cast<float2*>(&m + 1);
    for (int t = 0; t < d.map_texels; ++t) {
      if (d.flags & 1) {
        map[t] = make_float2(0.f, 0.f);
        continue;
      }
      const double D = ((t + 0.5) / d.map_texels - 0.5) * 2.0 * kPiD / L[i].M;
      map[t] = make_float2((float)map_delta(L[i], D), (float)map_occlusion(L[i], D));
    }
    for (int k = 1; k < L[i].K; ++k) {
      HostLayout Lk = L[i];
      Lk.Rfc = L[i].Rfc_m[k];
      Lk.M = L[i].M_m[k];
      float2* mk = reinterpret_cast<float2*>(mig_map(m, k) + 1);
      for (int t = 0; t < d.map_texels; ++t) {
        if (d.flags & 1) {
          mk[t] = make_float2(0.f, 0.f);
          continue;
        }
        const double D = ((t + 0.5) / d.map_texels - 0.5) * 2.0 * kPiD / Lk.M;
        mk[t] = make_float2((float)map_delta(Lk, D), (float)map_occlusion(Lk, D));
      }
    }
  }
  bysdf_materials* M = new bysdf_materials();
  M->n_mat = n;
  M->t_max = t_max;
  M->stride = (int)stride;
  M->desc.assign(desc, desc + n);
  for (int k = 0; k < BYSDF_NOPS; ++k) M->cfg[k] = default_cfg(k);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  auto cleanup = [&](int rc) {
    if (M->d_table) cudaFree(M->d_table);
    delete M;
    return rc;
  };
  cudaError_t e;
  if ((e = cudaGetDevice(&M->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&M->sm_count, cudaDevAttrMultiProcessorCount, M->device)) !=
          cudaSuccess)
    return cleanup(fail(BYSDF_E_CUDA, std::string("device query: ") + cudaGetErrorString(e)));
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, M->device);
  M->smem_optin = (size_t)optin;
  if ((e = dev_alloc(reinterpret_cast<void**>(&M->d_table), host.size())) != cudaSuccess)
    return cleanup(fail(BYSDF_E_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e)));
  if ((e = cudaMemcpyAsync(M->d_table, host.data(), host.size(), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cleanup(fail(BYSDF_E_CUDA, std::string("table upload: ") + cudaGetErrorString(e)));
  *out = M;
  return BYSDF_OK;
}

int bysdf_destroy_materials(bysdf_materials* m) {
  if (!m) return BYSDF_OK;
  cudaDeviceSynchronize();
  if (m->d_table) cudaFree(m->d_table);
  delete m;
  return BYSDF_OK;
}

int32_t bysdf_num_materials(const bysdf_materials* m) { return m ? m->n_mat : 0; }

int bysdf_set_params(bysdf_materials* m, const float* params, void* stream) {
  return set_params(m, params, BYSDF_NPARAM, stream);
}

int bysdf_get_params(const bysdf_materials* m, float* params, void* stream) {
  return get_params(m, params, BYSDF_NPARAM, stream);
}

int bysdf_set_params_ext(bysdf_materials* m, const float* params, void* stream) {
  return set_params(m, params, BYSDF_NPARAM_EXT, stream);
}

int bysdf_get_params_ext(const bysdf_materials* m, float* params, void* stream) {
  return get_params(m, params, BYSDF_NPARAM_EXT, stream);
}

size_t bysdf_workspace_size(const bysdf_materials* m, int64_t n) {
  if (!m) return 0;
  // per-tile partials of the deterministic backward, up to 15 columns
  return ws_partials_off(m->n_mat) + sizeof(float) * 16 * (size_t)max_tiles(n, m->n_mat);
}

int bysdf_eval(const bysdf_materials* m, const bysdf_hits* hits, int64_t n, float* f_rgb,
               float* pdf, uint8_t* status, void* workspace, size_t workspace_bytes,
               void* stream) {
  bysdf_outputs o{};
  o.f_rgb = f_rgb;
  o.pdf = pdf;
  o.status = status;
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_forward(m, BYSDF_OP_EVAL, hits, nullptr, nullptr, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_EVAL, hits));
}

int bysdf_eval_noalloc(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                       float* f_rgb, float* pdf, uint8_t* status, void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  // the forward kernels need the control words and one first-tile entry per
  // material; no per-record scratch
  if (m->n_mat > kNoallocMaxMaterials)
    return fail(BYSDF_E_WORKSPACE, "bysdf_eval_noalloc: more materials than its fixed scratch "
                                   "holds (at most " + std::to_string(kNoallocMaxMaterials) + ")");
  const size_t need = ws_partials_off(m->n_mat);
  int rc = check_hits(m, hits, true, n);
  if (rc) return rc;
  if (n == 0) return BYSDF_OK;
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the previous call's contents stay in the array: every launch claims
  // the control words (tile draws, error word) for its own epoch, and the
  // per-material entries of material-sorted records are rewritten by the
  // tile plan launched before it
  bysdf_outputs o{};
  o.f_rgb = f_rgb;
  o.pdf = pdf;
  o.status = status;
  return run_forward(m, BYSDF_OP_EVAL, hits, nullptr, nullptr, n, o, scratch,
                     BYSDF_NOALLOC_SCRATCH_BYTES, st, fwd_cfg(m, BYSDF_OP_EVAL, hits), need);
}

// ------------------------------------------------------ host pipeline -----
struct bysdf_host_pipeline {
  // Three slots: the copy-in of chunk c + 3 waits only for the copy-out of
  // chunk c, so with the link busy both ways the copy-ins run back to back
  // (with two, every second copy-in waited for a copy-out).
  static constexpr int kSlots = 3;
  const bysdf_materials* m = nullptr;
  int64_t chunk = 0;
  bool with_ratio = false;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr, in_done[kSlots] = {}, run_done[kSlots] = {},
              out_done[kSlots] = {};
  bool out_pending[kSlots] = {};
  uint8_t* dev = nullptr;   // all slots
  size_t slot_bytes = 0, ws_bytes = 0;
  size_t max_pitch = 0;     // of strided copies (cudaDevAttrMaxPitch)
};

namespace {
// Slot layout (bytes, 256-aligned): inputs h u v wi(3) wo(3) u0 u1 mat_id
// ratio, outputs f(3) pdf wo_s(3) weight(3) pdf_s status lobe_status, then
// the workspace.
struct SlotPtrs {
  float *h, *u, *v, *wi, *wo, *u0, *u1, *ratio;
  int32_t* mat;
  float *f, *pdf, *wo_s, *weight, *pdf_s;
  uint8_t *status, *lstat;
  void* ws;
};
size_t slot_layout(int64_t c, size_t ws_bytes, uint8_t* base, SlotPtrs* p) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    uint8_t* q = base ? base + off : nullptr;
    off = align_up(off + bytes, 256);
    return q;
  };
  const size_t f1 = sizeof(float) * (size_t)c, f3 = 3 * f1;
  SlotPtrs t;
  t.h = (float*)take(f1); t.u = (float*)take(f1); t.v = (float*)take(f1);
  t.wi = (float*)take(f3); t.wo = (float*)take(f3); t.u0 = (float*)take(f1);
  t.u1 = (float*)take(f1); t.ratio = (float*)take(f1); t.mat = (int32_t*)take(f1);
  t.f = (float*)take(f3); t.pdf = (float*)take(f1); t.wo_s = (float*)take(f3);
  t.weight = (float*)take(f3); t.pdf_s = (float*)take(f1);
  t.status = take((size_t)c); t.lstat = take((size_t)c);
  t.ws = take(ws_bytes);
  if (p) *p = t;
  return off;
}
}  // namespace

int bysdf_host_pipeline_create(const bysdf_materials* m, int64_t chunk, int with_ratio,
                               bysdf_host_pipeline** out) {
  if (!m || !out) return fail(BYSDF_E_ARG, "NULL argument");
  if (chunk < 1024 || chunk > ((int64_t)1 << 28)) return fail(BYSDF_E_ARG, "chunk outside [1024, 2^28]");
  if ((size_t)m->n_mat * smem_stride(m) > kAllSmemMax)
    return fail(BYSDF_E_UNSUPPORTED, "host pipeline: tables must fit in shared memory");
  *out = nullptr;
  bysdf_host_pipeline* p = new bysdf_host_pipeline();
  p->m = m;
  p->chunk = chunk;
  p->with_ratio = with_ratio != 0;
  p->ws_bytes = bysdf_workspace_size(m, chunk);
  p->slot_bytes = slot_layout(chunk, p->ws_bytes, nullptr, nullptr);
  auto bad = [&](cudaError_t e, const char* what) {
    bysdf_host_pipeline_destroy(p);
    return fail(BYSDF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = dev_alloc(reinterpret_cast<void**>(&p->dev), bysdf_host_pipeline::kSlots * p->slot_bytes)) !=
      cudaSuccess)
    return bad(e, "cudaMalloc");
  int dev = 0, pitch = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&pitch, cudaDevAttrMaxPitch, dev)) != cudaSuccess)
    return bad(e, "cudaDeviceGetAttribute");
  p->max_pitch = (size_t)pitch;
  if ((e = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&p->s_run, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking)) != cudaSuccess)
    return bad(e, "cudaStreamCreate");
  if ((e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming)) != cudaSuccess)
    return bad(e, "cudaEventCreate");
  for (int k = 0; k < bysdf_host_pipeline::kSlots; ++k)
    if ((e = cudaEventCreateWithFlags(&p->in_done[k], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->run_done[k], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->out_done[k], cudaEventDisableTiming)) != cudaSuccess)
      return bad(e, "cudaEventCreate");
  *out = p;
  return BYSDF_OK;
}

int bysdf_host_pipeline_destroy(bysdf_host_pipeline* p) {
  if (!p) return BYSDF_OK;
  if (p->s_in) cudaStreamSynchronize(p->s_in);
  if (p->s_run) cudaStreamSynchronize(p->s_run);
  if (p->s_out) cudaStreamSynchronize(p->s_out);
  for (int k = 0; k < bysdf_host_pipeline::kSlots; ++k) {
    if (p->in_done[k]) cudaEventDestroy(p->in_done[k]);
    if (p->run_done[k]) cudaEventDestroy(p->run_done[k]);
    if (p->out_done[k]) cudaEventDestroy(p->out_done[k]);
  }
  if (p->start) cudaEventDestroy(p->start);
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_run) cudaStreamDestroy(p->s_run);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  if (p->dev) cudaFree(p->dev);
  delete p;
  return BYSDF_OK;
}

int bysdf_eval_sample_pdf_host(bysdf_host_pipeline* p, const bysdf_hits* hits, const float* u0,
                               const float* u1, int64_t n, float* f_rgb, float* pdf,
                               uint8_t* status, float* wo_s, float* weight_s, float* pdf_s,
                               uint8_t* lobe_status_s, void* stream) {
  if (!p || !hits) return fail(BYSDF_E_ARG, "NULL argument");
  if (n < 0) return fail(BYSDF_E_ARG, "n < 0");
  if (n == 0) return BYSDF_OK;
  if (!hits->h || !hits->u || !hits->v || !hits->wi || !hits->wo || !u0 || !u1 || !f_rgb ||
      !pdf || !status || !wo_s || !weight_s || !pdf_s || !lobe_status_s)
    return fail(BYSDF_E_ARG, "host pipeline: a required buffer is NULL");
  if (hits->seg_offsets) return fail(BYSDF_E_UNSUPPORTED, "host pipeline: seg_offsets not supported");
  if ((hits->ratio != nullptr) != p->with_ratio)
    return fail(BYSDF_E_ARG, "host pipeline: ratio given / not given unlike at creation");
  cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
  BY_CU(cudaEventRecord(p->start, caller));
  BY_CU(cudaStreamWaitEvent(p->s_in, p->start, 0));
  const cudaMemcpyKind H2D = cudaMemcpyHostToDevice, D2H = cudaMemcpyDeviceToHost;
  for (int64_t a = 0, c = 0; a < n; a += p->chunk, ++c) {
    const int64_t mcount = std::min(p->chunk, n - a);
    const int k = (int)(c % bysdf_host_pipeline::kSlots);
    SlotPtrs s;
    slot_layout(p->chunk, p->ws_bytes, p->dev + (size_t)k * p->slot_bytes, &s);
    // the slot's previous results must be copied out before it is refilled
    if (p->out_pending[k]) BY_CU(cudaStreamWaitEvent(p->s_in, p->out_done[k], 0));
    const size_t b1 = sizeof(float) * (size_t)mcount;
    auto in1 = [&](float* d, const float* h) {
      return cudaMemcpyAsync(d, h + a, b1, H2D, p->s_in);
    };
    // a 3-plane array in one strided copy (rows of b1 bytes, host pitch n,
    // slot pitch mcount) while the host pitch is within the copy engine's
    // limit, else plane by plane
    const size_t hp = sizeof(float) * (size_t)n;
    const bool strided = hp <= p->max_pitch;
    auto in3 = [&](float* d, const float* h) {
      if (strided) return cudaMemcpy2DAsync(d, b1, h + a, hp, b1, 3, H2D, p->s_in);
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(d + q * mcount, h + (size_t)q * n + a, b1, H2D, p->s_in);
      return e;
    };
    BY_CU(in1(s.h, hits->h));
    BY_CU(in1(s.u, hits->u));
    BY_CU(in1(s.v, hits->v));
    BY_CU(in3(s.wi, hits->wi));
    BY_CU(in3(s.wo, hits->wo));
    BY_CU(in1(s.u0, u0));
    BY_CU(in1(s.u1, u1));
    if (hits->ratio) BY_CU(in1(s.ratio, hits->ratio));
    if (hits->mat_id)
      BY_CU(cudaMemcpyAsync(s.mat, hits->mat_id + a, sizeof(int32_t) * mcount, H2D, p->s_in));
    BY_CU(cudaEventRecord(p->in_done[k], p->s_in));
    BY_CU(cudaStreamWaitEvent(p->s_run, p->in_done[k], 0));
    bysdf_hits dh{};
    dh.h = s.h;
    dh.u = s.u;
    dh.v = s.v;
    dh.wi = s.wi;
    dh.wo = s.wo;
    dh.ratio = hits->ratio ? s.ratio : nullptr;
    dh.mat_id = hits->mat_id ? s.mat : nullptr;
    bysdf_outputs o{};
    o.f_rgb = s.f;
    o.pdf = s.pdf;
    o.status = s.status;
    o.wo = s.wo_s;
    o.weight = s.weight;
    o.pdf_s = s.pdf_s;
    o.lobe_status = s.lstat;
    int rc = run_forward(p->m, BYSDF_OP_FUSED, &dh, s.u0, s.u1, mcount, o, s.ws, p->ws_bytes,
                         p->s_run, fwd_cfg(p->m, BYSDF_OP_FUSED, &dh));
    if (rc) return rc;
    BY_CU(cudaEventRecord(p->run_done[k], p->s_run));
    BY_CU(cudaStreamWaitEvent(p->s_out, p->run_done[k], 0));
    auto out1 = [&](float* h, const float* d) {
      return cudaMemcpyAsync(h + a, d, b1, D2H, p->s_out);
    };
    auto out3 = [&](float* h, const float* d) {
      if (strided) return cudaMemcpy2DAsync(h + a, hp, d, b1, b1, 3, D2H, p->s_out);
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < 3 && e == cudaSuccess; ++q)
        e = cudaMemcpyAsync(h + (size_t)q * n + a, d + q * mcount, b1, D2H, p->s_out);
      return e;
    };
    BY_CU(out3(f_rgb, s.f));
    BY_CU(out1(pdf, s.pdf));
    BY_CU(cudaMemcpyAsync(status + a, s.status, (size_t)mcount, D2H, p->s_out));
    BY_CU(out3(wo_s, s.wo_s));
    BY_CU(out3(weight_s, s.weight));
    BY_CU(out1(pdf_s, s.pdf_s));
    BY_CU(cudaMemcpyAsync(lobe_status_s + a, s.lstat, (size_t)mcount, D2H, p->s_out));
    BY_CU(cudaEventRecord(p->out_done[k], p->s_out));
    p->out_pending[k] = true;
  }
  // later work on the caller's stream waits for the results
  for (int k = 0; k < bysdf_host_pipeline::kSlots; ++k)
    if (p->out_pending[k]) BY_CU(cudaStreamWaitEvent(caller, p->out_done[k], 0));
  return BYSDF_OK;
}

int bysdf_sample(const bysdf_materials* m, const bysdf_hits* hits, const float* u0,
                 const float* u1, int64_t n, float* wo, float* weight, float* pdf,
                 uint8_t* lobe_status, void* workspace, size_t workspace_bytes, void* stream) {
  bysdf_outputs o{};
  o.wo = wo;
  o.weight = weight;
  o.pdf_s = pdf;
  o.lobe_status = lobe_status;
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_forward(m, BYSDF_OP_SAMPLE, hits, u0, u1, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_SAMPLE, hits));
}

int bysdf_pdf(const bysdf_materials* m, const bysdf_hits* hits, int64_t n, float* pdf,
              uint8_t* status, void* workspace, size_t workspace_bytes, void* stream) {
  bysdf_outputs o{};
  o.pdf = pdf;
  o.status = status;
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_forward(m, BYSDF_OP_PDF, hits, nullptr, nullptr, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_PDF, hits));
}

int bysdf_eval_sample_pdf(const bysdf_materials* m, const bysdf_hits* hits, const float* u0,
                          const float* u1, int64_t n, float* f_rgb, float* pdf,
                          uint8_t* status, float* wo_s, float* weight_s, float* pdf_s,
                          uint8_t* lobe_status_s, void* workspace, size_t workspace_bytes,
                          void* stream) {
  bysdf_outputs o{};
  o.f_rgb = f_rgb;
  o.pdf = pdf;
  o.status = status;
  o.wo = wo_s;
  o.weight = weight_s;
  o.pdf_s = pdf_s;
  o.lobe_status = lobe_status_s;
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_forward(m, BYSDF_OP_FUSED, hits, u0, u1, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_FUSED, hits));
}

int bysdf_trace_yarns(const bysdf_yarn* yarns, int32_t n_yarns, const bysdf_rays* rays,
                      int64_t n, const float light[3], float* h, float* u, float* v,
                      float* wi, float* wo, float* ratio, int32_t* mat_id, int32_t* yarn_id,
                      float* t_hit, void* stream) {
  if (!yarns || !rays || !light) return fail(BYSDF_E_ARG, "yarns, rays and light are required");
  if (n_yarns < 1 || n_yarns > kMaxYarnPieces) return fail(BYSDF_E_ARG, "n_yarns outside [1, 2048]");
  if (n < 0 || n > ((int64_t)1 << 36)) return fail(BYSDF_E_ARG, "n out of range");
  if (n == 0) return BYSDF_OK;
  if (!rays->o || !rays->d) return fail(BYSDF_E_ARG, "rays: o and d required");
  const bool diff = rays->o1 || rays->d1 || rays->o2 || rays->d2;
  if (diff && !(rays->o1 && rays->d1 && rays->o2 && rays->d2))
    return fail(BYSDF_E_ARG, "rays: give all four differential planes or none");
  const void* ins[] = {rays->o, rays->d, rays->o1, rays->d1, rays->o2, rays->d2};
  for (const void* p : ins)
    if (p && !aligned16(p)) return fail(BYSDF_E_ARG, "rays: buffer not 16-byte aligned");
  int rc;
  if ((rc = check_out(h, "h")) || (rc = check_out(u, "u")) || (rc = check_out(v, "v")) ||
      (rc = check_out(wi, "wi")) || (rc = check_out(wo, "wo")) || (rc = check_out(mat_id, "mat_id")))
    return rc;
  if (ratio && !aligned16(ratio)) return fail(BYSDF_E_ARG, "ratio not 16-byte aligned");
  const float ln = std::sqrt(light[0] * light[0] + light[1] * light[1] + light[2] * light[2]);
  if (!(std::fabs(ln - 1.0f) <= 1e-3f)) return fail(BYSDF_E_ARG, "light must be a unit vector");
  TraceArgs a{};
  a.o = rays->o;
  a.d = rays->d;
  a.o1 = rays->o1;
  a.d1 = rays->d1;
  a.o2 = rays->o2;
  a.d2 = rays->d2;
  a.n = n;
  for (int c = 0; c < 3; ++c) a.light[c] = light[c];
  a.h = h;
  a.u = u;
  a.v = v;
  a.wi = wi;
  a.wo = wo;
  a.ratio = ratio;
  a.t_hit = t_hit;
  a.mat_id = mat_id;
  a.yarn_id = yarn_id;
  int dev = 0, sms = 0;
  BY_CU(cudaGetDevice(&dev));
  BY_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t blocks = (n + 255) / 256;
  const int grid = (int)std::min<int64_t>(blocks, (int64_t)sms * 8);
  BY_CU(launch_trace_yarns(yarns, n_yarns, a, grid, reinterpret_cast<cudaStream_t>(stream)));
  return BYSDF_OK;
}

int bysdf_eval_stochastic(const bysdf_materials* m, const bysdf_hits* hits,
                          const bysdf_stochastic* sto, int64_t n, float* f_rgb, float* pdf,
                          uint8_t* status, void* workspace, size_t workspace_bytes,
                          void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  if (!sto) return fail(BYSDF_E_ARG, "stochastic options are NULL");
  bysdf_outputs o{};
  o.f_rgb = f_rgb;
  o.pdf = pdf;
  o.status = status;
  return run_forward(m, BYSDF_OP_EVAL, hits, nullptr, nullptr, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_EVAL, hits), 0,
                     sto);
}

int bysdf_eval_sample_pdf_stochastic(const bysdf_materials* m, const bysdf_hits* hits,
                                     const bysdf_stochastic* sto, const float* u0,
                                     const float* u1, int64_t n, float* f_rgb, float* pdf,
                                     uint8_t* status, float* wo_s, float* weight_s,
                                     float* pdf_s, uint8_t* lobe_status_s, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  if (!sto) return fail(BYSDF_E_ARG, "stochastic options are NULL");
  bysdf_outputs o{};
  o.f_rgb = f_rgb;
  o.pdf = pdf;
  o.status = status;
  o.wo = wo_s;
  o.weight = weight_s;
  o.pdf_s = pdf_s;
  o.lobe_status = lobe_status_s;
  return run_forward(m, BYSDF_OP_FUSED, hits, u0, u1, n, o, workspace, workspace_bytes,
                     reinterpret_cast<cudaStream_t>(stream), fwd_cfg(m, BYSDF_OP_FUSED, hits), 0,
                     sto);
}

int bysdf_eval_backward(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                        const float* grad_f, float* grad_params, int deterministic,
                        void* workspace, size_t workspace_bytes, void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_backward(m, hits, n, grad_f, grad_params, deterministic, workspace,
                      workspace_bytes, reinterpret_cast<cudaStream_t>(stream),
                      m->cfg[BYSDF_OP_BACKWARD]);
}

int bysdf_eval_backward_ext(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                            const float* grad_f, float* grad_params, float* grad_wi,
                            float* grad_wo, int deterministic, void* workspace,
                            size_t workspace_bytes, void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  return run_backward(m, hits, n, grad_f, grad_params, deterministic, workspace,
                      workspace_bytes, reinterpret_cast<cudaStream_t>(stream),
                      m->cfg[BYSDF_OP_BACKWARD], KB_EXT, grad_wi, grad_wo);
}

int bysdf_eval_l2_backward(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                           const float* target_rgb, const float* weight, float* f_rgb,
                           float* loss_mat, float* grad_params, int deterministic,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  L2Args l2{target_rgb, weight, f_rgb, loss_mat};
  return run_backward(m, hits, n, nullptr, grad_params, deterministic, workspace,
                      workspace_bytes, reinterpret_cast<cudaStream_t>(stream),
                      m->cfg[BYSDF_OP_BACKWARD], KB_L2, nullptr, nullptr, &l2);
}

int bysdf_plain(int op, const bysdf_materials* m, const bysdf_hits* hits,
                const int64_t* seg_offsets_host, const float* u0, const float* u1, int64_t n,
                float* f_rgb, float* wo, float* weight, float* pdf, uint8_t* status,
                void* stream) {
  const int bits = op_bits(op);
  if (bits != OPF_EVAL && bits != OPF_SAMPLE && bits != OPF_PDF)
    return fail(BYSDF_E_ARG, "bysdf_plain: op must be EVAL, SAMPLE or PDF");
  int rc = check_hits(m, hits, bits != OPF_SAMPLE, n);
  if (rc) return rc;
  if (n == 0) return BYSDF_OK;
  if (!seg_offsets_host) return fail(BYSDF_E_ARG, "seg_offsets_host is NULL");
  if (seg_offsets_host[0] != 0 || seg_offsets_host[m->n_mat] != n)
    return fail(BYSDF_E_ARG, "seg_offsets_host must run from 0 to n");
  for (int i = 0; i < m->n_mat; ++i)
    if (seg_offsets_host[i + 1] < seg_offsets_host[i])
      return fail(BYSDF_E_ARG, "seg_offsets_host must be non-decreasing");
  if ((rc = check_out(status, "status"))) return rc;
  if (bits == OPF_EVAL && (rc = check_out(f_rgb, "f_rgb"))) return rc;
  if (bits != OPF_EVAL && (rc = check_out(pdf, "pdf"))) return rc;
  if (bits == OPF_SAMPLE) {
    if ((rc = check_out(u0, "u0")) || (rc = check_out(u1, "u1")) || (rc = check_out(wo, "wo")) ||
        (rc = check_out(weight, "weight")))
      return rc;
  }
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.table = m->d_table;
  a.n_mat = m->n_mat;
  a.stride = m->stride;
  a.n = n;
  a.h = hits->h;
  a.u = hits->u;
  a.v = hits->v;
  a.wi = hits->wi;
  a.wo = bits == OPF_SAMPLE ? nullptr : hits->wo;
  a.ratio = hits->ratio;
  a.u0 = u0;
  a.u1 = u1;
  a.f_rgb = f_rgb;
  a.pdf = pdf;
  a.status = status;
  a.wo_s = wo;
  a.weight_s = weight;
  a.pdf_s = pdf;
  a.lstat_s = status;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < m->n_mat; ++i)
    BY_CU(launch_plain(bits, a, i, seg_offsets_host[i], seg_offsets_host[i + 1], st));
  return BYSDF_OK;
}

int bysdf_plain_fused(const bysdf_materials* m, const bysdf_hits* hits,
                      const int64_t* seg_offsets_host, const float* u0, const float* u1,
                      int64_t n, const bysdf_outputs* out, void* stream) {
  int rc = check_hits(m, hits, true, n);
  if (rc) return rc;
  if (!out) return fail(BYSDF_E_ARG, "out is NULL");
  if (n == 0) return BYSDF_OK;
  if (!seg_offsets_host) return fail(BYSDF_E_ARG, "seg_offsets_host is NULL");
  if (seg_offsets_host[0] != 0 || seg_offsets_host[m->n_mat] != n)
    return fail(BYSDF_E_ARG, "seg_offsets_host must run from 0 to n");
  for (int i = 0; i < m->n_mat; ++i)
    if (seg_offsets_host[i + 1] < seg_offsets_host[i])
      return fail(BYSDF_E_ARG, "seg_offsets_host must be non-decreasing");
  if ((rc = check_out(out->f_rgb, "f_rgb")) || (rc = check_out(out->status, "status")) ||
      (rc = check_out(u0, "u0")) || (rc = check_out(u1, "u1")) ||
      (rc = check_out(out->wo, "wo")) || (rc = check_out(out->weight, "weight")) ||
      (rc = check_out(out->pdf_s, "pdf (sample)")) ||
      (rc = check_out(out->lobe_status, "lobe_status")))
    return rc;
  if (out->pdf && !aligned16(out->pdf)) return fail(BYSDF_E_ARG, "pdf not 16-byte aligned");
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.table = m->d_table;
  a.n_mat = m->n_mat;
  a.stride = m->stride;
  a.n = n;
  a.h = hits->h;
  a.u = hits->u;
  a.v = hits->v;
  a.wi = hits->wi;
  a.wo = hits->wo;
  a.ratio = hits->ratio;
  a.u0 = u0;
  a.u1 = u1;
  a.f_rgb = out->f_rgb;
  a.pdf = out->pdf;
  a.status = out->status;
  a.wo_s = out->wo;
  a.weight_s = out->weight;
  a.pdf_s = out->pdf_s;
  a.lstat_s = out->lobe_status;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < m->n_mat; ++i)
    BY_CU(launch_plain(OPF_EVAL | OPF_SAMPLE, a, i, seg_offsets_host[i], seg_offsets_host[i + 1],
                       st));
  return BYSDF_OK;
}

int bysdf_set_launch_config(bysdf_materials* m, int op, const bysdf_launch_config* cfg) {
  if (!m || !cfg) return fail(BYSDF_E_ARG, "NULL argument");
  if (op < 0 || op >= BYSDF_NOPS) return fail(BYSDF_E_ARG, "bad op");
  if (cfg->block != 128 && cfg->block != 256 && cfg->block != 512)
    return fail(BYSDF_E_ARG, "block must be 128, 256 or 512");
  const bool items_ok = cfg->items == 1 || cfg->items == 2 || cfg->items == 4 ||
                        cfg->items == 8 || (op == BYSDF_OP_BACKWARD && cfg->items == 16);
  if (!items_ok) return fail(BYSDF_E_ARG, "items must be 1, 2, 4 or 8 (16 for the backward)");
  if (cfg->ctas_per_sm < 0) return fail(BYSDF_E_ARG, "ctas_per_sm < 0");
  if (cfg->occupancy != 0 && cfg->occupancy != 1) return fail(BYSDF_E_ARG, "occupancy must be 0 or 1");
  m->cfg[op] = *cfg;
  m->cfg_set[op] = true;
  return BYSDF_OK;
}

int bysdf_get_launch_config(const bysdf_materials* m, int op, bysdf_launch_config* cfg) {
  if (!m || !cfg) return fail(BYSDF_E_ARG, "NULL argument");
  if (op < 0 || op >= BYSDF_NOPS) return fail(BYSDF_E_ARG, "bad op");
  *cfg = m->cfg[op];
  return BYSDF_OK;
}

int bysdf_autotune(bysdf_materials* m, int op, const bysdf_hits* hits, const float* u0,
                   const float* u1, const float* grad_f, int64_t n, const bysdf_outputs* out,
                   void* workspace, size_t workspace_bytes, void* stream,
                   bysdf_launch_config* best) {
  if (!m || !out || !best) return fail(BYSDF_E_ARG, "NULL argument");
  if (op < 0 || op >= BYSDF_NOPS) return fail(BYSDF_E_ARG, "bad op");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  BY_CU(cudaEventCreate(&e0));
  BY_CU(cudaEventCreate(&e1));
  auto run = [&](const bysdf_launch_config& c) {
    if (op == BYSDF_OP_BACKWARD)
      return run_backward(m, hits, n, grad_f, out->grad_params, 0, workspace, workspace_bytes,
                          st, c);
    return run_forward(m, op, hits, u0, u1, n, *out, workspace, workspace_bytes, st, c);
  };
  float best_ms = 1e30f;
  bysdf_launch_config best_c = m->cfg[op];
  int rc = BYSDF_OK;
  for (int block : {128, 256, 512}) {
    for (int items : {1, 2, 4, 8, 16}) {
      if (items == 16 && op != BYSDF_OP_BACKWARD) continue;  // forward kernels: up to 8
      for (int occ_mode : {0, 1}) {
        if (occ_mode == 1 && block == 512) continue;
        bysdf_launch_config c{block, items, 0, occ_mode};
        if ((rc = run(c))) break;  // warm-up (and validation)
        cudaEventRecord(e0, st);
        for (int r = 0; r < 3 && rc == BYSDF_OK; ++r) rc = run(c);
        cudaEventRecord(e1, st);
        if (rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          rc = fail(BYSDF_E_CUDA, "autotune: kernel failed");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best_c = c;
        }
      }
      if (rc) break;
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  m->cfg[op] = best_c;
  m->cfg_set[op] = true;
  *best = best_c;
  return BYSDF_OK;
}

int bysdf_noalloc_error(void* stream, uint32_t* err) {
  if (!err) return fail(BYSDF_E_ARG, "NULL argument");
  void* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  return bysdf_workspace_error(scratch, stream, err);
}

int bysdf_test_stall_table_waits(bysdf_materials* m, uint32_t polls) {
  if (!m) return fail(BYSDF_E_ARG, "materials is NULL");
  m->test_stall_polls = polls;
  return BYSDF_OK;
}

int bysdf_test_math(int32_t fn, const float* x, const float* y, int64_t n, float* out,
                    void* stream) {
  if (fn < 0 || fn > 5) return fail(BYSDF_E_ARG, "fn outside [0, 5]");
  if (n < 0) return fail(BYSDF_E_ARG, "n < 0");
  if (n > 0 && (!x || !out || ((fn == 0 || fn == 1) && !y)))
    return fail(BYSDF_E_ARG, "NULL argument");
  BY_CU(launch_test_math(fn, x, y, n, out, reinterpret_cast<cudaStream_t>(stream)));
  return BYSDF_OK;
}

int bysdf_test_fail_allocations(int32_t count) {
  if (count < 0) return fail(BYSDF_E_ARG, "count < 0");
  g_fail_allocs.store(count);
  return BYSDF_OK;
}

int bysdf_workspace_error(const void* workspace, void* stream, uint32_t* err) {
  if (!workspace || !err) return fail(BYSDF_E_ARG, "NULL argument");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the word is epoch << 24 | error bits (the epoch of the last launch)
  const uint8_t* p = reinterpret_cast<const uint8_t*>(workspace) + offsetof(WsCtl, err_word);
  unsigned long long word = 0;
  BY_CU(cudaMemcpyAsync(&word, p, sizeof(word), cudaMemcpyDeviceToHost, st));
  BY_CU(cudaStreamSynchronize(st));
  BY_CU(cudaMemsetAsync(const_cast<uint8_t*>(p), 0, sizeof(word), st));
  *err = (uint32_t)(word & ((1ull << kEpochShift) - 1));
  return BYSDF_OK;
}

}  // extern "C"
