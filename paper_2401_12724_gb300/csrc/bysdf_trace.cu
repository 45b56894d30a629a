// The step upstream of the BYSDF: camera rays against explicit yarns (Sec. 3.3)
// and their ray differentials (Sec. 5.3), producing BYSDF hit records.
//
// Yarns are straight pieces of yarn curves staged in shared memory (a
// piece's rotation-minimising frame is constant, so it carries its reference
// normal).  One thread per ray tests every piece: a conservative bounding-
// sphere distance test first, then the lateral surface about the ray's point
// of closest approach to the axis, where the square root is taken of R^2
// minus a small distance (no cancellation between terms of the camera
// distance squared).
#include "bysdf_launch.h"

namespace bysdf {

namespace {

// one piece in shared memory: 4 x float4
//   a = (p0, length), b = (t, R), c = (n_ref, v0), d = (centre, r_sphere^2)
struct PieceS {
  float4 a, b, c, d;
};

__device__ __forceinline__ float dot3(float ax, float ay, float az, float bx, float by, float bz) {
  return fmaf(ax, bx, fmaf(ay, by, az * bz));
}

// signed distance of the line (o, d) from the piece's axis in its
// cross-section, over R (the azimuthal offset); +inf along the axis
__device__ __forceinline__ float line_offset(const PieceS& p, float bx, float by, float bz,
                                             float ox, float oy, float oz, float dx, float dy,
                                             float dz) {
  const float qx = ox - p.a.x, qy = oy - p.a.y, qz = oz - p.a.z;
  const float q_n = dot3(qx, qy, qz, p.c.x, p.c.y, p.c.z);
  const float q_b = dot3(qx, qy, qz, bx, by, bz);
  const float d_n = dot3(dx, dy, dz, p.c.x, p.c.y, p.c.z);
  const float d_b = dot3(dx, dy, dz, bx, by, bz);
  const float l = sqrtf(d_n * d_n + d_b * d_b);
  if (!(l > 0.f)) return __int_as_float(0x7f800000);
  return (q_n * d_b - q_b * d_n) / (l * p.b.w);
}

}  // namespace

__global__ void __launch_bounds__(256) k_trace_yarns(const bysdf_yarn* __restrict__ yarns,
                                                     int n_yarns, TraceArgs a) {
  extern __shared__ float4 smem_pieces[];
  PieceS* ps = reinterpret_cast<PieceS*>(smem_pieces);
  // stage the pieces with an orthonormal frame: t / |t|, then n_ref without
  // its t component, normalised; bounding sphere about the piece's centre
  for (int k = threadIdx.x; k < n_yarns; k += blockDim.x) {
    const bysdf_yarn y = yarns[k];
    float tx = y.tangent[0], ty = y.tangent[1], tz = y.tangent[2];
    const float it = rsqrtf(dot3(tx, ty, tz, tx, ty, tz));
    tx *= it;
    ty *= it;
    tz *= it;
    const float nt = dot3(y.n_ref[0], y.n_ref[1], y.n_ref[2], tx, ty, tz);
    float nx = y.n_ref[0] - nt * tx, ny = y.n_ref[1] - nt * ty, nz = y.n_ref[2] - nt * tz;
    const float in = rsqrtf(dot3(nx, ny, nz, nx, ny, nz));
    nx *= in;
    ny *= in;
    nz *= in;
    const float hl = 0.5f * y.length;
    const float rs = sqrtf(hl * hl + y.radius * y.radius);
    PieceS p;
    p.a = make_float4(y.p0[0], y.p0[1], y.p0[2], y.length);
    p.b = make_float4(tx, ty, tz, y.radius);
    p.c = make_float4(nx, ny, nz, y.v0);
    // margin: 1e-4 relative plus 1e-4 absolute covers the float rounding of
    // the distance test below
    const float rm = rs * 1.0001f + 1e-4f;
    p.d = make_float4(y.p0[0] + hl * tx, y.p0[1] + hl * ty, y.p0[2] + hl * tz, rm * rm);
    ps[k] = p;
  }
  __syncthreads();
  const int64_t n = a.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float ox = __ldg(a.o + i), oy = __ldg(a.o + n + i), oz = __ldg(a.o + 2 * n + i);
    const float dx = __ldg(a.d + i), dy = __ldg(a.d + n + i), dz = __ldg(a.d + 2 * n + i);
    const float idd = 1.0f / dot3(dx, dy, dz, dx, dy, dz);
    int best = -1;
    float sbest = 0.f;
    for (int k = 0; k < n_yarns; ++k) {
      const float4 sd = ps[k].d;
      // bounding sphere: distance of the centre from the ray line
      const float mx = ox - sd.x, my = oy - sd.y, mz = oz - sd.z;
      const float mb = dot3(mx, my, mz, dx, dy, dz) * idd;
      const float px = fmaf(-mb, dx, mx), py = fmaf(-mb, dy, my), pz = fmaf(-mb, dz, mz);
      if (dot3(px, py, pz, px, py, pz) > sd.w) continue;
      const float4 pa = ps[k].a, pb = ps[k].b;
      // lateral surface about the ray's closest approach to the axis
      const float qx = ox - pa.x, qy = oy - pa.y, qz = oz - pa.z;
      const float qt = dot3(qx, qy, qz, pb.x, pb.y, pb.z);
      const float dt = dot3(dx, dy, dz, pb.x, pb.y, pb.z);
      const float qpx = fmaf(-qt, pb.x, qx), qpy = fmaf(-qt, pb.y, qy), qpz = fmaf(-qt, pb.z, qz);
      const float dpx = fmaf(-dt, pb.x, dx), dpy = fmaf(-dt, pb.y, dy), dpz = fmaf(-dt, pb.z, dz);
      const float aa = dot3(dpx, dpy, dpz, dpx, dpy, dpz);
      if (!(aa > 1e-20f)) continue;
      const float R2 = pb.w * pb.w;
      if (!(dot3(qpx, qpy, qpz, qpx, qpy, qpz) > R2)) continue;  // starts inside
      const float sc = -dot3(qpx, qpy, qpz, dpx, dpy, dpz) / aa;
      const float mpx = fmaf(sc, dpx, qpx), mpy = fmaf(sc, dpy, qpy), mpz = fmaf(sc, dpz, qpz);
      const float e2 = R2 - dot3(mpx, mpy, mpz, mpx, mpy, mpz);
      if (e2 < 0.f) continue;
      const float s = sc - sqrtf(e2 / aa);
      if (!(s > 0.f) || (best >= 0 && !(s < sbest))) continue;
      const float w = fmaf(s, dt, qt);
      if (w < 0.f || w > pa.w) continue;
      best = k;
      sbest = s;
    }
    if (a.yarn_id) a.yarn_id[i] = best;
    if (a.t_hit) a.t_hit[i] = best >= 0 ? sbest : 0.f;
    if (best < 0) {
      a.h[i] = a.u[i] = a.v[i] = 0.f;
      if (a.ratio) a.ratio[i] = 0.f;
      for (int c = 0; c < 3; ++c) a.wi[c * n + i] = a.wo[c * n + i] = 0.f;
      a.mat_id[i] = -1;
      continue;
    }
    const PieceS p = ps[best];
    const float bx = p.b.y * p.c.z - p.b.z * p.c.y;  // b_ref = t x n_ref
    const float by = p.b.z * p.c.x - p.b.x * p.c.z;
    const float bz = p.b.x * p.c.y - p.b.y * p.c.x;
    // hit relative to the root: the camera distance enters only through one
    // fused multiply-add per coordinate
    const float qx = ox - p.a.x, qy = oy - p.a.y, qz = oz - p.a.z;
    const float xx = fmaf(sbest, dx, qx), xy = fmaf(sbest, dy, qy), xz = fmaf(sbest, dz, qz);
    const float w = dot3(xx, xy, xz, p.b.x, p.b.y, p.b.z);
    const float x_n = dot3(xx, xy, xz, p.c.x, p.c.y, p.c.z);
    const float x_b = dot3(xx, xy, xz, bx, by, bz);
    float u = atan2f(x_b, x_n);
    if (u < 0.f) u += 2.0f * kPi;
    if (u >= 2.0f * kPi) u = 0.f;
    // the azimuthal offset: signed distance of the ray from the axis over R
    const float h0 = fminf(fmaxf(line_offset(p, bx, by, bz, ox, oy, oz, dx, dy, dz), -1.f), 1.f);
    a.h[i] = h0;
    a.u[i] = u;
    a.v[i] = p.c.w + w;
    a.wi[i] = -dot3(dx, dy, dz, p.c.x, p.c.y, p.c.z);
    a.wi[n + i] = -dot3(dx, dy, dz, bx, by, bz);
    a.wi[2 * n + i] = -dot3(dx, dy, dz, p.b.x, p.b.y, p.b.z);
    a.wo[i] = dot3(a.light[0], a.light[1], a.light[2], p.c.x, p.c.y, p.c.z);
    a.wo[n + i] = dot3(a.light[0], a.light[1], a.light[2], bx, by, bz);
    a.wo[2 * n + i] = dot3(a.light[0], a.light[1], a.light[2], p.b.x, p.b.y, p.b.z);
    a.mat_id[i] = yarns[best].mat_id;
    if (a.ratio) {
      // Sec. 5.3: the differential rays' offsets about the same axis bound
      // the footprint; the record carries its half-width in h
      float r = 0.f;
      if (a.o1 && a.d1 && a.o2 && a.d2) {
        const float h1 = line_offset(p, bx, by, bz, __ldg(a.o1 + i), __ldg(a.o1 + n + i),
                                     __ldg(a.o1 + 2 * n + i), __ldg(a.d1 + i),
                                     __ldg(a.d1 + n + i), __ldg(a.d1 + 2 * n + i));
        const float h2 = line_offset(p, bx, by, bz, __ldg(a.o2 + i), __ldg(a.o2 + n + i),
                                     __ldg(a.o2 + 2 * n + i), __ldg(a.d2 + i),
                                     __ldg(a.d2 + n + i), __ldg(a.d2 + 2 * n + i));
        const float w1 = fabsf(h1 - h0), w2 = fabsf(h2 - h0);
        r = (isfinite(w1) && isfinite(w2)) ? fmaxf(w1, w2) : 2.0f;
      }
      a.ratio[i] = r;
    }
  }
}

cudaError_t launch_trace_yarns(const bysdf_yarn* yarns, int n_yarns, const TraceArgs& a,
                               int grid, cudaStream_t st) {
  const size_t smem = sizeof(PieceS) * (size_t)n_yarns;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_trace_yarns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_trace_yarns<<<grid, 256, smem, st>>>(yarns, n_yarns, a);
  return cudaGetLastError();
}

}  // namespace bysdf
