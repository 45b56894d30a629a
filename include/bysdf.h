/*
 * libbysdf -- batched yarn-level BYSDF on the GPU (sm_103a).
 *
 * The bidirectional yarn scattering distribution function of "A Multi-scale
 * Yarn Appearance Model with Fiber Details" (Khattar et al.), evaluated,
 * sampled and differentiated at ray--yarn hit records:
 *   - implicit ply geometry by the iterated cross-section trace (Sec. 3.4),
 *   - implicit fibers from 1D maps (Sec. 3.5.1),
 *   - ply and fiber shadowing G_p, G_f (Sec. 4.1.4),
 *   - the four lobes f_x^S, f_y^S, f_x^B, f_y^B (Sec. 4.1, Eqs. 1-6) with the
 *     attenuation tau^{N_i} (Eq. 4),
 *   - importance sampling and its pdf (Sec. 4.1.5),
 *   - near / multi-scale / far-field selection by pixel coverage
 *     (Sec. 4.2, Eqs. 7-11; Sec. 5.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * Frame: yarn-local at the hit; x = reference normal, y = T x N_ref, z = yarn
 * tangent.  Lengths in units of the yarn radius of the material.  Directions
 * are unit float32 3-vectors pointing AWAY from the hit; omega_i is the
 * camera-side direction.  Outputs f are cosine-weighted, f(wi, wo) |wo . n|,
 * with n the shading normal at the hit, so that a renderer multiplies them by
 * the incident radiance directly; pdf is a solid-angle density of wo.
 *
 * Buffers: every per-record buffer is DEVICE memory owned by the caller,
 * float32 (int32 ids, uint8 status), structure-of-arrays: a 3-vector plane
 * argument points to 3*n floats laid out [x[0..n), y[0..n), z[0..n)].  Every
 * buffer must be 16-byte aligned.  Calls are asynchronous on `stream`
 * (a cudaStream_t; NULL = legacy default stream) and allocate no memory: the
 * caller provides a workspace of at least bysdf_workspace_size() bytes, which
 * must not be shared by calls that may run concurrently.  Its contents need
 * no initialisation: each launch claims the workspace's control words for
 * itself (they carry the launch's epoch) before it uses them.
 *
 * Per-record status (uint8): 0 ok; 1 no ply hit (the ray passes through the
 * yarn, f = 0, pdf = 0); 2 invalid input (non-finite value, |h| > 1, a
 * direction whose squared norm is off by more than 1e-3, material id out of
 * range, negative ratio, random number outside [0, 1)); 3 invalid sample
 * (the sampled direction left the lobe's support, e.g. total internal
 * reflection); 4 not evaluated (a bounded device-side wait on a material
 * table copy gave up; the workspace's error word says so, see
 * bysdf_workspace_error; the record's other outputs are 0).  Sampling writes
 * lobe << 4 | status, lobe 0 = f_x^S (reflection), 1 = f_y^S
 * (transmission), 2 = f_x^B, 3 = f_y^B.
 *
 * Return codes: 0 ok; negative on a host-side error, in which case nothing
 * was launched (bysdf_last_error() describes it).
 */
#ifndef BYSDF_H
#define BYSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BYSDF_OK 0
#define BYSDF_E_ARG (-1)         /* null/misaligned pointer, bad size, bad descriptor */
#define BYSDF_E_CUDA (-2)        /* a CUDA runtime call failed */
#define BYSDF_E_UNSUPPORTED (-3) /* a combination this build does not run */
#define BYSDF_E_WORKSPACE (-4)   /* workspace missing or too small */

#define BYSDF_NPARAM 8      /* differentiable parameters per material, see below */
#define BYSDF_NPARAM_EXT 15 /* the extended set of bysdf_set_params_ext          */

/* Material descriptor (host).  Sec. 3.4 / 3.5 geometry, Sec. 4.1 appearance.
 * Readings of quantities the paper leaves open are documented with each
 * field; all angles in degrees. */
typedef struct bysdf_material_desc {
  int32_t n_plies;        /* N_p in [1, 8]; plies are equal discs inscribed in
                             the yarn circle, touching it and each other     */
  int32_t fibers_per_ply; /* N_f in [4, 4096]; fibers fill `packing` of a ply */
  int32_t map_texels;     /* T in [4, 1024]: texels per fiber period of the 1D
                             fiber maps (Sec. 3.5.1); 256 by default          */
  int32_t trace_iters;    /* N_it in [1, 64]: cross-section updates of the ply
                             trace (Sec. 3.4: "3-5 steps"); 5 by default      */
  int32_t k_max;          /* K_max in [1, 64]: h nodes of a footprint that
                             covers the yarn (Sec. 4.2); 16 by default        */
  int32_t flags;          /* bit 0: no fiber detail (flat ply surface)        */
  float yarn_radius;      /* R > 0                                            */
  float ply_twist_deg;    /* helix angle of the ply centre lines              */
  float fiber_twist_deg;  /* helix angle of the fibers about the ply axis     */
  float eta;              /* refractive index > 1                             */
  float albedo[3];        /* body albedo k^B (RGB), Eqs. 5-6                  */
  float k_spec;           /* specular albedo scale: k^S = (1 - B) k_spec      */
  float beta_deg[2];      /* GGX roughness along t_f and b_f (Eq. 2)          */
  float body_B;           /* B in [0, 1]: body share of the energy (Sec. 4.1.5)*/
  float body_r;           /* r in [0, 1]: reflected share of the body energy  */
  float sigma_t;          /* extinction coefficient of Eq. 4 (per length)     */
  float shadow_density;   /* sigma_s: G = exp(-sigma_s * occlusion) (Sec 4.1.4)*/
  float packing;          /* fiber area fraction of a ply disc (0, 1]         */
  float albedo_y[3];      /* k^B_y (RGB) of the transmission body lobe, Eq. 6;
                             negative: equal to albedo (one body colour for
                             both lobes, the default reading)               */
  /* Fiber migration (Sec. 3.5, reading): K_m = migration_maps in [1, 4] map
   * pairs; map 0 is the regular outer ring, map k >= 1 the ring sunk by
   * k r_f / K_m (as many fibers as fit on it).  The yarn is cut into
   * segments of migration_length along v; segment s uses map
   * (word 0 of Philox4x64-10 with counter (s, 0, 0, 0) and key
   * (migration_seed, 0xB15DF000F1BE0002)) mod K_m and blends linearly with
   * its neighbour within migration_blend (in (0, 0.5]) of the length from
   * each boundary.  K_m = 1 (or 0): no migration; the other fields are then
   * ignored.  Each extra map adds 32 + 8 T bytes to the material's table. */
  int32_t migration_maps;
  int32_t migration_seed;
  float migration_length;
  float migration_blend;
} bysdf_material_desc;

/* Opaque material table: per-material constants and the 1D fiber normal and
 * fiber shadowing maps, resident in device memory (Sec. 3.5.1, 4.1.4). */
typedef struct bysdf_materials bysdf_materials;

/* Hit records (device pointers; see conventions above). */
typedef struct bysdf_hits {
  const float* h;       /* azimuthal offset in [-1, 1] (Sec. 3.3)            */
  const float* u;       /* azimuthal phase of the hit, radians (Sec. 3.3)    */
  const float* v;       /* longitudinal length of the hit (Sec. 3.3)         */
  const float* wi;      /* omega_i, 3 planes                                  */
  const float* wo;      /* omega_o, 3 planes (eval/pdf/backward; NULL when
                           sampling)                                          */
  const float* ratio;   /* pixel-footprint / yarn-width ratio (Sec. 5.3):
                           the half-width of [h1, h2] in h units; NULL or 0 =
                           near field, >= 1 + |h| = far field (Eq. 7)         */
  const int32_t* mat_id;     /* material of each record; NULL = material 0    */
  const int64_t* seg_offsets;/* NULL, or n_mat + 1 offsets: records are sorted
                                by material and material m owns
                                [seg_offsets[m], seg_offsets[m+1]); required
                                when the tables do not fit in shared memory.
                                Expected: seg_offsets[0] = 0, nondecreasing,
                                seg_offsets[n_mat] = n; offsets outside
                                [0, n] are clamped (records outside a
                                material's clamped range are not written)  */
} bysdf_hits;

/* Launch shape of the persistent kernels (chosen by bysdf_autotune). */
typedef struct bysdf_launch_config {
  int32_t block;          /* threads per CTA: 128, 256 or 512               */
  int32_t items;          /* records per lane per warp tile: 1, 2, 4 or 8
                             (the backward also 16); a batch of fewer tiles
                             than the grid's resident warps takes smaller
                             tiles, so that more warps get work              */
  int32_t ctas_per_sm;    /* resident CTAs per SM the grid is sized for
                             (0: as many as fit)                             */
  int32_t occupancy;      /* register budget: 0 the default, 1 a tighter cap
                             for more resident warps (forward: 16 vs 24
                             warps per SM; backward: uncapped vs 16 warps;
                             blocks of 128 or 256; spills go to L1)         */
} bysdf_launch_config;

enum { BYSDF_OP_EVAL = 0, BYSDF_OP_SAMPLE = 1, BYSDF_OP_PDF = 2, BYSDF_OP_FUSED = 3,
       BYSDF_OP_BACKWARD = 4, BYSDF_NOPS = 5 };

/* Version string of the library. */
const char* bysdf_version(void);

/* Description of the last host-side error of the calling thread. */
const char* bysdf_last_error(void);

/* Build the material table for n descriptors on the current device and
 * upload it with stream-ordered copies on `stream`.  The library allocates
 * and owns the table; release it with bysdf_destroy_materials.  The table is
 * read-only for every call except bysdf_set_params, so it may be shared by
 * calls on several streams.  Errors: BYSDF_E_ARG (null pointer, n < 1 or
 * n > 65536, a descriptor field out of range), BYSDF_E_CUDA. */
int bysdf_create_materials(const bysdf_material_desc* desc, int32_t n, void* stream,
                           bysdf_materials** out);

/* Release the table (synchronises the device first). */
int bysdf_destroy_materials(bysdf_materials* m);

/* Number of materials in the table. */
int32_t bysdf_num_materials(const bysdf_materials* m);

/* Replace the differentiable parameters of every material from a DEVICE
 * array params[n_mat][8] (float32), stream-ordered:
 *   [0..2] albedo k^B (RGB), [3] beta_t, [4] beta_b (GGX roughness, radians),
 *   [5] ply helix angle alpha_p (radians), [6] fiber helix angle alpha_f
 *   (radians), [7] shadow density sigma_s.
 * The derived constants (helix rates, fiber phase rates) are recomputed on
 * the device.  Not safe while other calls read the table. */
int bysdf_set_params(bysdf_materials* m, const float* params, void* stream);

/* Copy the current parameters to a DEVICE array [n_mat][8] (same layout). */
int bysdf_get_params(const bysdf_materials* m, float* params, void* stream);

/* The extended parameter set: the 8 above (where [0..2] is now k^B_x, the
 * reflection body colour of Eq. 5), then the rest of the paper's fitting set
 * (Sec. 5.2: r, k^B_x, k^B_y, sigma_t) and the two energy weights:
 *   [8] r (body reflect share), [9..11] k^B_y (RGB, Eq. 6), [12] sigma_t
 *   (Eq. 4), [13] B (body share), [14] k_spec (k^S = (1 - B) k_spec).
 * DEVICE array params[n_mat][15], stream-ordered.  bysdf_set_params (8
 * columns) sets k^B_x and k^B_y to the same albedo and keeps [8], [12..14].
 * Values are not range-checked on the device: B and r outside [0, 1] or
 * negative colours give meaningless results. */
int bysdf_set_params_ext(bysdf_materials* m, const float* params, void* stream);
int bysdf_get_params_ext(const bysdf_materials* m, float* params, void* stream);

/* Workspace bytes the calls below need for n records. */
size_t bysdf_workspace_size(const bysdf_materials* m, int64_t n);

/* Evaluate f(wi, wo) |wo . n| (RGB, 3 planes into f_rgb) and, when pdf is
 * not NULL, the sampling density of wo (Sec. 4.1 Eqs. 1-6, Sec. 4.2 Eq. 8).
 * status is required.  One persistent launch. */
int bysdf_eval(const bysdf_materials* m, const bysdf_hits* hits, int64_t n, float* f_rgb,
               float* pdf, uint8_t* status, void* workspace, size_t workspace_bytes,
               void* stream);

/* Importance-sample wo from two uniform numbers per record (Sec. 4.1.5):
 * writes wo (3 planes), weight = f |wo . n| / pdf (3 planes), pdf and
 * lobe << 4 | status.  hits->wo is ignored.  A record without a ply hit
 * passes through: wo = -wi, weight = 1, pdf = 0, status 1. */
int bysdf_sample(const bysdf_materials* m, const bysdf_hits* hits, const float* u0,
                 const float* u1, int64_t n, float* wo, float* weight, float* pdf,
                 uint8_t* lobe_status, void* workspace, size_t workspace_bytes, void* stream);

/* Sampling density of hits->wo (Sec. 4.1.5). */
int bysdf_pdf(const bysdf_materials* m, const bysdf_hits* hits, int64_t n, float* pdf,
              uint8_t* status, void* workspace, size_t workspace_bytes, void* stream);

/* Eval + pdf at hits->wo and a sample from (u0, u1) in one pass over the
 * geometry, which the three results share.  Outputs as the three calls. */
int bysdf_eval_sample_pdf(const bysdf_materials* m, const bysdf_hits* hits, const float* u0,
                          const float* u1, int64_t n, float* f_rgb, float* pdf,
                          uint8_t* status, float* wo_s, float* weight_s, float* pdf_s,
                          uint8_t* lobe_status_s, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Stochastic estimators of the paper's integrals, as options of eval and the
 * fused op (the deterministic calls above take midpoints and the smooth
 * entry):
 *   BYSDF_STOCH_JITTER_NODES: the K footprint nodes at uniform points of
 *     their strata of [h1, h2] (Sec. 4.2: stratified Monte Carlo sampling of
 *     h) instead of the midpoints; the near field (no footprint) is unchanged;
 *   BYSDF_STOCH_ROUGH_ENTRY: one sample of the Omega_y integral of Eq. 1: the
 *     camera ray refracts into the yarn through a GGX visible normal m at x
 *     (roughness of the shading point) instead of n; the entry transmittance
 *     is 1 - F(omega_i . m); a ray refracted outward gives no transmission.
 * Random numbers: Philox4x64-10 (Salmon et al. 2011), key (seed,
 * 0xB15DF0005EED0001), counter (index_offset + i, block, 0, 0) for record i:
 * node j uses word j % 4 of block j / 4; the entry microfacet words 0 and 1
 * of block 16; a word w gives (w >> 40) * 2^-24.  The same seed and index
 * draw the same nodes and entry in eval and in the fused op, so a sample's
 * pdf is the stochastic eval's pdf at the sampled direction.  Launches use
 * the op's launch shape, as the deterministic calls do.  Other arguments and
 * errors as bysdf_eval / bysdf_eval_sample_pdf; NULL options: BYSDF_E_ARG;
 * unknown flag bits: BYSDF_E_ARG. */
#define BYSDF_STOCH_JITTER_NODES 1u
#define BYSDF_STOCH_ROUGH_ENTRY 2u
typedef struct bysdf_stochastic {
  uint64_t seed;         /* generator key word 0 */
  int64_t index_offset;  /* global index of record 0 (e.g. a shard's first) */
  uint32_t flags;        /* BYSDF_STOCH_* bits; 0 = the deterministic estimate */
  uint32_t reserved;     /* 0 */
} bysdf_stochastic;

int bysdf_eval_stochastic(const bysdf_materials* m, const bysdf_hits* hits,
                          const bysdf_stochastic* options, int64_t n, float* f_rgb, float* pdf,
                          uint8_t* status, void* workspace, size_t workspace_bytes,
                          void* stream);
int bysdf_eval_sample_pdf_stochastic(const bysdf_materials* m, const bysdf_hits* hits,
                                     const bysdf_stochastic* options, const float* u0,
                                     const float* u1, int64_t n, float* f_rgb, float* pdf,
                                     uint8_t* status, float* wo_s, float* weight_s,
                                     float* pdf_s, uint8_t* lobe_status_s, void* workspace,
                                     size_t workspace_bytes, void* stream);

/* ---- The step upstream of the BYSDF: rays against explicit yarns ----
 * Yarns (Sec. 3.3) are curves cut into straight pieces; a straight piece's
 * rotation-minimising frame is constant, so each piece carries its reference
 * normal.  bysdf_trace_yarns finds, per camera ray, the closest entry into
 * the lateral surface of any piece (end caps are not surfaces; a ray
 * starting inside a piece sees none of that piece) and writes the BYSDF hit
 * record in the piece's frame (x = reference normal, y = tangent x normal,
 * z = tangent):
 *   u  azimuth of the surface normal at the hit, [0, 2 pi);
 *   h  the azimuthal offset: the ray's signed distance from the axis in the
 *      cross-section over R, in [-1, 1];
 *   v  v0 + position along the piece;
 *   wi = -d, wo = the light direction, in the frame (3 planes each);
 *   ratio (optional): with the two differential rays (Sec. 5.3), the larger
 *      |h_k - h| of their own azimuthal offsets about the same axis (hit or
 *      not), i.e. the pixel footprint's half-width in h (2 for a ray along
 *      the axis); without them 0 (near field);
 *   mat_id: the piece's material; -1 where no piece is hit (the other
 *      outputs are then 0; the BYSDF reports such records as invalid).
 * Each piece's frame is made orthonormal (t / |t|, then n_ref without its t
 * component, normalised).  The pieces are staged in shared memory (at most
 * 2048) and grouped in eights in the order given, each group and each piece
 * with a bounding sphere: giving the pieces of a yarn consecutively keeps the
 * groups tight.  A warp of 32 consecutive rays skips the groups and pieces
 * that no ray of it can reach, so the cost follows the pieces near the rays
 * when neighbouring rays are coherent (camera rays in pixel order); the
 * result is that of testing every piece.  A ray with a zero or non-finite
 * direction, or a non-finite origin, hits nothing (mat_id -1). */
typedef struct bysdf_yarn {
  float p0[3];       /* root of the piece */
  float tangent[3];  /* along the piece (unit) */
  float n_ref[3];    /* reference normal, perpendicular to the tangent */
  float length;      /* of the piece */
  float radius;      /* R */
  float v0;          /* length along the yarn at the root */
  int32_t mat_id;    /* material of the piece */
  int32_t pad[3];
} bysdf_yarn;

typedef struct bysdf_rays {
  const float* o;    /* ray origins, 3 planes */
  const float* d;    /* ray directions (unit), 3 planes */
  const float* o1;   /* differential rays: NULL for none */
  const float* d1;
  const float* o2;
  const float* d2;
} bysdf_rays;

/* yarns: DEVICE array of n_yarns pieces (1..2048); rays and outputs: DEVICE
 * planes of n rays (16-byte aligned); light: HOST, 3 floats (unit, world).
 * ratio, yarn_id (piece index or -1) and t_hit (ray parameter) may be NULL.
 * Stream-ordered; returns BYSDF_E_ARG on bad sizes or pointers. */
int bysdf_trace_yarns(const bysdf_yarn* yarns, int32_t n_yarns, const bysdf_rays* rays,
                      int64_t n, const float light[3], float* h, float* u, float* v,
                      float* wi, float* wo, float* ratio, int32_t* mat_id, int32_t* yarn_id,
                      float* t_hit, void* stream);

/* Gradient of sum_i sum_c grad_f[c][i] * f_c(record i) with respect to the 8
 * parameters of each material (layout of bysdf_set_params), accumulated
 * into grad_params[n_mat][8] (DEVICE, zeroed by this call).  The forward pass
 * is recomputed, not stored.  Records with status != 0 contribute nothing.
 * deterministic != 0 reduces in a fixed order (material-sorted records with
 * seg_offsets only; otherwise BYSDF_E_UNSUPPORTED). */
int bysdf_eval_backward(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                        const float* grad_f, float* grad_params, int deterministic,
                        void* workspace, size_t workspace_bytes, void* stream);

/* As bysdf_eval_backward for the 15 parameters of bysdf_set_params_ext
 * (grad_params[n_mat][15], DEVICE, zeroed by this call; [0..2] and [9..11]
 * are the separate derivatives in k^B_x and k^B_y), and optionally, per
 * record, the vector-Jacobian products with respect to the record's
 * directions (inverse rendering):
 *   grad_wi[c][i] = sum_k grad_f[k][i] d f_k / d wi_c, likewise grad_wo,
 * 3 DEVICE planes each or NULL, written for every record (0 where the
 * status != 0).  The derivatives are the partials of f as a function of the
 * three components as given (f does not renormalise them).  The direction
 * products run as a second kernel (forward-mode, 6 tangents) only when one
 * of them is requested.  workspace: bysdf_workspace_size(). */
int bysdf_eval_backward_ext(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                            const float* grad_f, float* grad_params, float* grad_wi,
                            float* grad_wo, int deterministic, void* workspace,
                            size_t workspace_bytes, void* stream);

/* The plain form, for comparison: one launch per material over
 * material-sorted records, one thread per record, tables read from global
 * memory, no persistent scheduling.  seg_offsets_host: n_mat + 1 HOST
 * offsets.  op: BYSDF_OP_EVAL, _SAMPLE or _PDF (pointers as in the calls
 * above; unused ones may be NULL). */
int bysdf_plain(int op, const bysdf_materials* m, const bysdf_hits* hits,
                const int64_t* seg_offsets_host, const float* u0, const float* u1,
                int64_t n, float* f_rgb, float* wo, float* weight, float* pdf,
                uint8_t* status, void* stream);

/* Launch shape used for op (BYSDF_OP_*), per table.  Until one is set here
 * or by bysdf_autotune, the forward calls take 512 x 4 at occupancy 0 for
 * records without a footprint and 256 x 8 at occupancy 1 for records with a
 * ratio plane (up to 16 geometry nodes each); once set, the shape serves
 * both kinds.  get returns the set shape, else the first default. */
int bysdf_set_launch_config(bysdf_materials* m, int op, const bysdf_launch_config* cfg);
int bysdf_get_launch_config(const bysdf_materials* m, int op, bysdf_launch_config* cfg);

/* Output buffers of one op, for bysdf_autotune (unused ones may be NULL). */
typedef struct bysdf_outputs {
  float* f_rgb;          /* eval: 3 planes                                  */
  float* pdf;            /* eval / pdf                                      */
  uint8_t* status;       /* eval / pdf                                      */
  float* wo;             /* sample: 3 planes                                */
  float* weight;         /* sample: 3 planes                                */
  float* pdf_s;          /* sample                                          */
  uint8_t* lobe_status;  /* sample                                          */
  float* grad_params;    /* backward: [n_mat][8]                            */
} bysdf_outputs;

/* Forward, L2 loss and its parameter gradient in one pass (the fitting of
 * Sec. 5.2 as a loss against target radiance; the backward of
 * bysdf_eval_backward with the upstream gradient 2 w (f - target) formed
 * from each record's own f, so the forward is not run twice):
 *   loss_mat[k] = sum over the records of material k with status 0 of
 *                 w_i sum_c (f_c(i) - target_c(i))^2,
 *   grad_params = d (sum_k loss_mat[k]) / d params, [n_mat][8] as in
 *                 bysdf_eval_backward (written by the callee).
 * target_rgb: 3 planes, required; weight: per-record w_i, NULL = 1; f_rgb
 * (nullable): the forward values, 0 where a record has no valid
 * evaluation; loss_mat (nullable, 4-byte aligned): [n_mat].  Deterministic
 * mode as bysdf_eval_backward.  Errors as bysdf_eval_backward; a NULL target
 * with n > 0: BYSDF_E_ARG. */
int bysdf_eval_l2_backward(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                           const float* target_rgb, const float* weight, float* f_rgb,
                           float* loss_mat, float* grad_params, int deterministic,
                           void* workspace, size_t workspace_bytes, void* stream);

/* The plain per-material form of the fused op (bysdf_eval_sample_pdf): one
 * launch per material over its sorted record range, one thread per record,
 * tables read from global memory; eval at hits->wo and one sample from u0,
 * u1 per record, outputs as bysdf_eval_sample_pdf (out->f_rgb, pdf, status,
 * wo, weight, pdf_s, lobe_status; grad_params unused).  The comparison form
 * of the fused persistent kernel.  seg_offsets_host: n_mat + 1 HOST offsets
 * from 0 to n, non-decreasing. */
int bysdf_plain_fused(const bysdf_materials* m, const bysdf_hits* hits,
                      const int64_t* seg_offsets_host, const float* u0, const float* u1,
                      int64_t n, const bysdf_outputs* out, void* stream);

/* Time every supported launch shape of op (BYSDF_OP_EVAL, _SAMPLE, _PDF,
 * _FUSED, _BACKWARD) on these records with CUDA events on `stream`, keep the
 * fastest in the table for later calls and return it in *best.  Writes the
 * op's outputs (several times).  Synchronises the stream; not capturable. */
int bysdf_autotune(bysdf_materials* m, int op, const bysdf_hits* hits, const float* u0,
                   const float* u1, const float* grad_f, int64_t n, const bysdf_outputs* out,
                   void* workspace, size_t workspace_bytes, void* stream,
                   bysdf_launch_config* best);

/* ---- records in host memory ----------------------------------------------
 * A pipeline streams records held in host memory (pinned, for overlap)
 * through the fused eval + sample kernel in chunks: the copy of chunk c+1 to
 * the device, the kernel on chunk c and the copy of chunk c-1's results back
 * run concurrently on three streams owned by the pipeline.  The pipeline
 * allocates its device slots (three chunks of records, outputs and
 * workspace: the copy-in of chunk c + 3 waits only for the copy-out of chunk
 * c) and streams once, at creation; calls allocate nothing.  Host buffers use
 * the plane layout of the device calls with plane stride n.  The call is
 * asynchronous on `stream` (it starts after the work queued there and work
 * queued there afterwards waits for it); the host buffers must stay valid
 * until it completes.  One call at a time per pipeline. */
typedef struct bysdf_host_pipeline bysdf_host_pipeline;
int bysdf_host_pipeline_create(const bysdf_materials* m, int64_t chunk, int with_ratio,
                               bysdf_host_pipeline** out);
int bysdf_host_pipeline_destroy(bysdf_host_pipeline* p);
/* hits: HOST pointers (seg_offsets must be NULL: chunks of unsorted records,
 * so the tables must fit in shared memory); outputs: HOST pointers as in
 * bysdf_eval_sample_pdf. */
int bysdf_eval_sample_pdf_host(bysdf_host_pipeline* p, const bysdf_hits* hits, const float* u0,
                               const float* u1, int64_t n, float* f_rgb, float* pdf,
                               uint8_t* status, float* wo_s, float* weight_s, float* pdf_s,
                               uint8_t* lobe_status_s, void* stream);

/* Eval without a caller-provided workspace: the same computation and
 * outputs as bysdf_eval, for callers that are not allowed to allocate device
 * memory (for example a renderer plug-in whose host application owns every
 * allocation, or code running where an allocation could synchronise the
 * device or fail).  The paper has no counterpart; this is a library-level
 * convenience.
 *
 * Scratch: a fixed array of BYSDF_NOALLOC_SCRATCH_BYTES in device memory,
 * defined in the library, which every GPU that loads the library holds until
 * the process exits.  It fits the tables of up to
 * (BYSDF_NOALLOC_SCRATCH_BYTES - 256) / 4 - 1 = BYSDF_NOALLOC_MAX_MATERIALS
 * materials; larger tables return BYSDF_E_WORKSPACE.  The call allocates
 * nothing.  Each call looks up the array's device address
 * (cudaGetSymbolAddress) on the current device, so it stays right after a
 * device reset; the first lookup on a device may load the library's module,
 * so make the first call before any stream capture.  Every call on a device
 * shares the one array and sets the part that must start at zero; calls
 * that may overlap on the GPU (other streams, other host threads) race on
 * it and must be serialised by the caller.  bysdf_noalloc_error reads the
 * array's error word. */
#define BYSDF_NOALLOC_SCRATCH_BYTES 16384
#define BYSDF_NOALLOC_MAX_MATERIALS 4031
int bysdf_eval_noalloc(const bysdf_materials* m, const bysdf_hits* hits, int64_t n,
                       float* f_rgb, float* pdf, uint8_t* status, void* stream);

/* Device-side error word of a workspace, as left by the last call that used
 * it (each call clears it first): 0 = none; bit 0: a bounded wait on a
 * shared-memory table copy gave up (the records of the tiles that could not
 * be evaluated have status 4); bit 1: a copy was still in flight after a
 * second bounded wait; bit 2 (index-checking build only, libbysdf_bounds.so
 * built with -DBYSDF_DEBUG_BOUNDS): an index checked on the device was out
 * of range and was clamped.  Synchronises the stream, then clears the word. */
int bysdf_workspace_error(const void* workspace, void* stream, uint32_t* err);

/* The error word of bysdf_eval_noalloc's fixed scratch on the current
 * device, as bysdf_workspace_error reads a workspace's.  Synchronises
 * the stream. */
int bysdf_noalloc_error(void* stream, uint32_t* err);

/* Test hook of the device-side error path (no counterpart in the paper):
 * from now on, every wait on a material-table copy in the persistent kernels
 * of `m` polls a barrier that nothing arrives on and gives up after `polls`
 * polls, as a wait on a copy that never completes would; the real copy is
 * then waited for (so none is in flight at exit), the error word gets bit
 * 0 and the records get status 4.  polls = 0 switches the hook off.  No
 * fault, no hang: every wait stays bounded. */
int bysdf_test_stall_table_waits(bysdf_materials* m, uint32_t polls);

/* Test hook of the host-side allocation-failure path (no counterpart in the
 * paper): the next `count` device allocations of the library (the material
 * table of bysdf_create_materials, the device slots of
 * bysdf_host_pipeline_create) fail as on an exhausted device, without calling
 * cudaMalloc: the call returns BYSDF_E_CUDA ("cudaMalloc: out of memory"),
 * writes no handle and frees what it had taken.  count = 0 switches the hook
 * off; every other entry point allocates nothing and is unaffected.
 * Process-wide.  Returns BYSDF_E_ARG for count < 0. */
int bysdf_test_fail_allocations(int32_t count);

/* Test hook of the float path's own approximations (no counterpart in the
 * paper): out[i] = f(x[i], y[i]) for fn 0 the polynomial atan2(y, x) of the
 * kernels, 1 CUDA's atan2f(y, x), 2 / 3 the sine / cosine the kernels take
 * of the fiber normal's deviation, 4 / 5 CUDA's sinf / cosf; computed in a
 * unit built with the kernels' flags.  x, y (fn 0 and 1 only), out: device
 * arrays of n floats.  Asynchronous on stream; BYSDF_E_ARG on a bad fn, n or
 * pointer. */
int bysdf_test_math(int32_t fn, const float* x, const float* y, int64_t n, float* out,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BYSDF_H */
