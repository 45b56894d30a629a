/*
 * FP64 CPU oracle of the yarn-level BYSDF ("A Multi-scale Yarn Appearance Model
 * with Fiber Details", Khattar et al.).  TEST INFRASTRUCTURE ONLY: the tests,
 * the smoke check and the CPU-baseline leg of the benchmark call it; the CUDA
 * product path never does.  It shares no code with the CUDA library.
 *
 * Every function computes the paper's model in double precision, step by step:
 *   Sec. 3.4 (implicit plies), Sec. 3.5 (implicit fibers, 1D maps),
 *   Sec. 4.1.2 Eqs. 2-4 (specular lobes, attenuation), Sec. 4.1.3 Eqs. 5-6
 *   (body lobes), Sec. 4.1.4 (shadowing), Sec. 4.1.5 (importance sampling),
 *   Sec. 4.2 Eqs. 7-11 (far-field / multi-scale aggregation).
 * Inputs are the float32 values the GPU path receives, widened exactly.
 * Where the paper is silent or garbled the oracle takes the readings listed in
 * the repository's design notes; each is named at the point of use.
 */
#ifndef BYSDF_ORACLE_H
#define BYSDF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Material description (same fields and units as the product descriptor). */
typedef struct orc_material {
  int32_t n_plies;         /* N_p >= 1 */
  int32_t fibers_per_ply;  /* N_f >= 4 */
  int32_t map_texels;      /* T, texels per fiber period of the 1D maps */
  int32_t trace_iters;     /* N_it, cross-section updates of the ply trace */
  int32_t k_max;           /* K_max, largest number of h nodes (multi-scale) */
  int32_t flags;           /* bit 0: no fiber detail (delta = 0, o_f = 0) */
  double yarn_radius;      /* R */
  double ply_twist_deg;    /* alpha_p, helix angle of the ply centre lines */
  double fiber_twist_deg;  /* alpha_f, helix angle of the fibers about the ply */
  double eta;              /* refractive index */
  double albedo[3];        /* k^B (RGB) */
  double k_spec;           /* specular albedo scale, k^S = (1 - B) k_spec */
  double beta_deg[2];      /* GGX roughness along t_f, b_f (degrees) */
  double body_B;           /* B: body share of the energy */
  double body_r;           /* r: reflected share of the body energy */
  double sigma_t;          /* extinction coefficient (per unit length) */
  double shadow_density;   /* sigma_s of the shadowing terms */
  double packing;          /* fiber area fraction of a ply cross-section */
  double albedo_y[3];      /* k^B_y (RGB) of the transmission body lobe (Eq. 6);
                              negative: equal to albedo */
  /* Fiber migration (Sec. 3.5, reading): migration_maps K_m in [1, 4] 1D map
   * pairs; map 0 is the regular outer ring, map k >= 1 the ring sunk by
   * k r_f / K_m (fewer fibers fit).  The yarn is cut into segments of
   * migration_length along v; segment s uses map (word 0 of Philox4x64-10
   * with counter (s mod 256, 0, 0, 0), key (migration_seed, ORC_MIG_KEY1))
   * mod K_m -- the choice repeats every 256 segments -- and blends linearly
   * with its neighbour within migration_blend (in (0, 0.5]) of the length
   * from each boundary.  K_m = 1: no migration. */
  int32_t migration_maps;
  int32_t migration_seed;
  double migration_length;
  double migration_blend;
} orc_material;

/* Structure-of-arrays hit records; wi/wo are [3][n] planes (x, y, z). */
typedef struct orc_records {
  const float* h;
  const float* u;
  const float* v;
  const float* wi;
  const float* wo;       /* NULL for sampling */
  const float* ratio;    /* NULL -> near field */
  const float* u0;       /* sampling random numbers, NULL otherwise */
  const float* u1;
  const int32_t* mat_id; /* NULL -> material 0 */
} orc_records;

/* Status codes (per record). */
enum { ORC_OK = 0, ORC_NO_HIT = 1, ORC_INVALID = 2, ORC_BAD_SAMPLE = 3 };

/* Index of the differentiable per-material parameters. */
enum {
  ORC_P_ALB_R = 0, ORC_P_ALB_G, ORC_P_ALB_B, ORC_P_BETA_T, ORC_P_BETA_B,
  ORC_P_ALPHA_P, ORC_P_ALPHA_F, ORC_P_SIGMA_S, ORC_NPARAM,
  /* the paper's fitting set (Sec. 5.2): body reflection share r, the body
   * colours k^B_x (= ALB above) and k^B_y, attenuation sigma_t (Eq. 4); and
   * the body fraction B and specular scale k_spec.  In the 8-parameter set
   * ALB moves k^B_x and k^B_y together. */
  ORC_P_BODY_R = ORC_NPARAM, ORC_P_ALBY_R, ORC_P_ALBY_G, ORC_P_ALBY_B, ORC_P_SIGMA_T,
  ORC_P_BODY_B, ORC_P_K_SPEC, ORC_NPARAM_EXT
};

/* Batched entry points.  Return 0, or -1 on a bad material description. */
int orc_eval(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
             double* f_rgb, double* pdf, uint8_t* status, int n_threads);
int orc_pdf(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
            double* pdf, uint8_t* status, int n_threads);
int orc_sample(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
               double* wo, double* weight, double* pdf, uint8_t* lobe_status,
               int n_threads);
/* Gradient of sum_i sum_c g[c][i] * f[c][i] with respect to the 8 parameters
 * (radians for angles) of every material, exact forward-mode AD in FP64.
 * grad: [n_mat][8]; jac (optional): [n][3][8]; f_rgb (optional) as orc_eval. */
int orc_grad(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
             const double* g_rgb, double* grad, double* jac, double* f_rgb,
             int n_threads);
/* As orc_grad for the 15 parameters of ORC_NPARAM_EXT (grad: [n_mat][15]),
 * plus, per record, the vector-Jacobian products with respect to the record's
 * directions: g_wi[c][i] = sum_k g[k][i] df_k/d wi_c and likewise g_wo
 * ([3][n] each, optional), the partial derivatives of f as a function of the
 * three components as given (no renormalisation).  jac (optional):
 * [n][3][21] = 15 parameters, then wi, then wo. */
int orc_grad_ext(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                 const double* g_rgb, double* grad, double* g_wi, double* g_wo,
                 double* jac, double* f_rgb, int n_threads);
/* Stochastic estimators of the paper's integrals, with random numbers from
 * Philox4x64-10 (Salmon et al. 2011) keyed by (seed, ORC_STOCH_KEY1) and
 * counted by the record's global index index_offset + i:
 *   ORC_STOCH_JITTER_NODES: the K footprint nodes at uniform points of their
 *     strata (Sec. 4.2, stratified sampling of h) instead of the midpoints;
 *     node j uses word j % 4 of counter (index, j / 4, 0, 0);
 *   ORC_STOCH_ROUGH_ENTRY: the entry refraction through a GGX visible normal
 *     (one sample of Eq. 1's Omega_y integral), words 0, 1 of (index, 16, 0, 0).
 * Outputs as orc_eval / orc_sample. */
#define ORC_STOCH_JITTER_NODES 1u
#define ORC_STOCH_ROUGH_ENTRY 2u
#define ORC_STOCH_KEY1 0xB15DF0005EED0001ull
#define ORC_MIG_KEY1 0xB15DF000F1BE0002ull /* key word 1 of the migration map choice */
int orc_eval_stochastic(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                        uint64_t seed, int64_t index_offset, uint32_t flags, double* f_rgb,
                        double* pdf, uint8_t* status, int n_threads);
int orc_sample_stochastic(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                          uint64_t seed, int64_t index_offset, uint32_t flags, double* wo,
                          double* weight, double* pdf, uint8_t* lobe_status, int n_threads);
/* Discontinuity margins (parity tests).  For each record, the evaluation of
 * op 0 (eval and pdf at omega_o) or op 1 (one sample from u0, u1) -- with the
 * stochastic estimators when flags != 0 -- notes at every branch point of the
 * model, and at the steep spots where the result moves faster than float32
 * rounding can be followed, how far the deciding quantity is from its
 * threshold, in that quantity's own units:
 *   0 ply trace: R_p - |perp| of the in-plane ray at every update (hit/miss)
 *   1 closest ply: distance gap to the next hit ply
 *   2 fiber maps: distance in fiber periods to the cusp texel interval
 *   3 in-plane length of omega_i (rays along the yarn axis)
 *   4 omega_i . n and omega_o . n at the shading normal (hemisphere side)
 *   5 transmission: entry and exit side tests, total internal reflection at y
 *   6 lobe choice: u0 against the cumulative lobe probabilities
 *   7 sampled direction: side tests, the sampler's disk frame
 *   8 ply shadowing: the shadow ray grazing another ply's circle
 *   9 fiber maps: distance in fiber periods to the nearest texel centre, where
 *     the interpolant's slope (and so every derivative) changes
 * out: [n][ORC_MG_N], the smallest distance per class (+inf where a record
 * never reaches the class; the row stays +inf for invalid records). */
#define ORC_MG_N 10
int orc_margins(const orc_material* m, int n_mat, const orc_records* r, int64_t n, int op,
                uint64_t seed, int64_t index_offset, uint32_t flags, double* out,
                int n_threads);
/* Test hook of the parity tests' conditioning measure: add dt to the in-plane
 * hit distance of every footprint node and du_ply (radians) to its ply
 * azimuth (and so to the fiber phase), as a float32 evaluation's rounding of
 * these two quantities would.  Process-wide; set it between evaluations and
 * back to (0, 0) afterwards. */
void orc_set_internal_offsets(double dt, double du_ply);
/* The jittered node positions h_j of one record (returns K; h_out[K]). */
int orc_stoch_nodes(double h0, int has_ratio, double ratio, int k_max, uint64_t seed,
                    uint64_t index, double* h_out);
/* Fiber migration introspection: ring radius and fiber count of map k and the
 * map index of segment seg (out[3]); the T texels (delta, o_f) of map k. */
int orc_migration_info(const orc_material* m, int k, int64_t seg, double* out);
int orc_migration_texels(const orc_material* m, int k, double* delta, double* of);
/* One Philox4x64-10 block (the generator behind the stochastic estimators). */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
/* Operation counts of one evaluation per record.  op: 0 eval (with pdf),
 * 1 sample, 3 the geometry and shading state that eval and sample share.
 * counts: [n][6] = add/sub, mul, div, sqrt, transcendental, compare. */
int orc_count_ops(const orc_material* m, int n_mat, const orc_records* r,
                  int64_t n, int op, double* counts);

/* ---- single-record introspection (tests) ---- */
typedef struct orc_geo {
  int32_t status;      /* 0 hit, 1 no hit, 2 invalid */
  int32_t n_nodes;     /* K */
  int32_t n_hit_nodes;
  int32_t ply;         /* closest ply of node 0 */
  double h1, h2;       /* footprint range */
  double ni_mean;      /* mean N_i over hit nodes */
  double t_ply[8];     /* in-plane distance to each ply of node 0 (-1: miss) */
  double x[3];         /* aggregated hit point */
  double n_p[3], t_p[3];   /* ply frame of node 0 */
  double n_f[3], t_f[3];   /* aggregated fiber frame (before the side flip) */
  double g_p, g_f;         /* shadowing of node 0 */
  double g_mean;           /* aggregated G_p * G_f */
  double u_ply, delta, o_f;/* node 0 fiber-map query */
  double residual;         /* | |x - c_k(z_x)| - R_p | of node 0 */
} orc_geo;
int orc_geometry(const orc_material* m, float h, float u, float v,
                 const float wi[3], float ratio, orc_geo* out);

/* Layout: out = {R_p, R_c, r_f, R_fc, M, omega_p, omega_f}. */
int orc_layout(const orc_material* m, double* out);
/* Analytic fiber maps at offset D from a fiber crown: {delta, o_f}. */
int orc_fiber_map(const orc_material* m, double D, double* out);
/* Tabulated (periodic, linearly interpolated) maps at fiber phase theta. */
int orc_fiber_map_tab(const orc_material* m, double theta, double* out);
/* In-plane occlusion o_p of a point x on ply k (cross-section at height z),
 * along the in-plane direction w (Sec. 4.1.4). */
double orc_ply_occlusion(const orc_material* m, int k, double z,
                         const double x[2], const double w[2]);

/* Microfacet building blocks in a local frame (t, b, n) = (x, y, z). */
double orc_fresnel(double cos_i, double eta);
double orc_ggx_d(const double m[3], double at, double ab);
double orc_ggx_g1(const double w[3], const double m[3], double at, double ab);
void orc_vndf_sample(const double w[3], double at, double ab, double u0,
                     double u1, double m_out[3]);
double orc_vndf_pdf(const double w[3], const double m[3], double at, double ab);
/* The four lobes for a given shading state (lobe tests, reciprocity):
 * frame = {t, b, n} rows, out = {R, TT, xB(rgb), yB(rgb)} cosine-weighted. */
int orc_lobes(const orc_material* m, const double frame[9], const double x[3],
              double g, double ni, double width, const double wi[3],
              const double wo[3], double out[8]);
/* Walter rough-dielectric transmission f_t(i, o) with eta_i, eta_o (no
 * cosine), in a local frame with normal z (generalised reciprocity test). */
double orc_btdf(const double i[3], const double o[3], double eta_i,
                double eta_o, double at, double ab);

#ifdef __cplusplus
}
#endif
#endif
