/*
 * FP64 CPU oracle of the step upstream of the BYSDF: camera rays against
 * explicit yarns, producing the hit records the BYSDF takes (Sec. 3.3
 * "Explicit Yarns"; Sec. 5.3 ray differentials).  TEST INFRASTRUCTURE ONLY:
 * the tests and the smoke check call it; the CUDA product path never does.
 *
 * Yarns are straight cylinder segments (the pieces a curve is cut into); the
 * rotation-minimising reference frame of a straight piece is constant, so a
 * piece carries its reference normal (the frame is made orthonormal: t / |t|,
 * then n_ref without its t component, normalised).  Per ray: the closest
 * entry into the lateral surface of any piece (flat end caps are not
 * surfaces; rays starting inside a yarn see none of it),
 * then in the piece's frame (x = reference normal, y = tangent x normal,
 * z = tangent):
 *   u  azimuth of the surface normal at the hit from the reference normal,
 *      in [0, 2 pi);
 *   h  the azimuthal offset: the ray's signed distance from the axis in the
 *      cross-section over R, n_u x e for the unit in-plane direction e;
 *   v  length from the yarn's root (v0 + position along the piece);
 *   wi = -d and wo = the light direction, in the frame;
 *   ratio (pixel footprint / yarn width): with differential rays, the
 *      largest |h_k - h| of their azimuthal offsets about the same axis
 *      (their own signed distance over R, hit or not); else 0 (near field).
 */
#ifndef YARN_TRACE_ORACLE_H
#define YARN_TRACE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_yarn {
  double p0[3];     /* root of the piece */
  double t[3];      /* unit tangent */
  double n_ref[3];  /* unit reference normal, perpendicular to t */
  double length;    /* of the piece */
  double radius;    /* R */
  double v0;        /* length along the yarn at the root */
  int32_t mat_id;
  int32_t pad;
} orc_yarn;

/* [3][n] planes (x, y, z) of float32 rays; o1/d1/o2/d2 may be NULL. */
typedef struct orc_rays {
  const float* o;
  const float* d;
  const float* o1;
  const float* d1;
  const float* o2;
  const float* d2;
} orc_rays;

/* Outputs per ray (n): h, u, v, ratio, t_hit (ray parameter), yarn index
 * (-1: no hit; the other outputs are then 0 and mat_id -1), mat_id; wi, wo
 * as [3][n].  light: world direction towards the light (unit).  Returns 0. */
int orc_trace_yarns(const orc_yarn* y, int n_yarn, const orc_rays* r, int64_t n,
                    const double light[3], double* h, double* u, double* v, double* wi,
                    double* wo, double* ratio, double* t_hit, int32_t* yarn,
                    int32_t* mat_id, int n_threads);

#ifdef __cplusplus
}
#endif
#endif
