// The step upstream of the BYSDF: camera rays against explicit yarns (Sec. 3.3)
// and their ray differentials (Sec. 5.3), producing BYSDF hit records.
//
// Yarns are straight pieces of yarn curves staged in shared memory (a
// piece's rotation-minimising frame is constant, so it carries its reference
// normal).  One thread per ray; pieces carry a bounding sphere, and so do
// groups of kGroupPieces consecutive pieces (neighbours along a yarn, in the
// caller's order).  The rays of a warp are neighbouring pixels, so the warp
// culls against a bound on all 32 rays at once: it tests 32 groups at a time,
// one per lane, then the pieces of up to four kept groups at a time, one per
// lane, and keeps the ballot of the pieces some ray may reach.  Each ray then
// tests the kept pieces in ascending order: a conservative bounding-sphere
// distance test, then the lateral surface about the ray's point of closest
// approach to the axis, where the square root is taken of R^2 minus a small
// distance (no cancellation between terms of the camera distance squared).
// The culling only skips pieces that no ray of the warp can hit: the result
// is that of testing every piece.
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

constexpr int kGroupPieces = 8;
// the piece rounds give each of four groups 8 lanes (lane >> 3, lane & 7)
static_assert(kGroupPieces == 8, "the piece rounds assume groups of 8 pieces");

// The line of a ray with origin o_i and unit direction u_i lies at least
// dist(C, axis) - ro - (|C - oc| + ro) * del from a point C, where the axis
// is (oc, ua), ro >= |o_i - oc| and del >= |u_i - ua|: a sphere (C, r^2)
// farther than r plus that slack from the axis is missed by every ray of the
// bundle.  A bound that is not finite (a degenerate ray) keeps the sphere.
__device__ __forceinline__ bool bundle_reaches(float4 sph, float ocx, float ocy, float ocz,
                                               float uax, float uay, float uaz, float ro,
                                               float del) {
  const float vx = sph.x - ocx, vy = sph.y - ocy, vz = sph.z - ocz;
  const float tv = dot3(vx, vy, vz, uax, uay, uaz);
  const float px = fmaf(-tv, uax, vx), py = fmaf(-tv, uay, vy), pz = fmaf(-tv, uaz, vz);
  const float thr =
      fmaf(sqrtf(dot3(vx, vy, vz, vx, vy, vz)) + ro, del, sqrtf(sph.w) + ro) * 1.0001f + 1e-4f;
  return !(dot3(px, py, pz, px, py, pz) > thr * thr);
}

}  // namespace

// (256, 1): 72 registers without spills, 3 CTAs per SM; held to 64, the
// differential rays loaded ahead of the culling would spill
__global__ void __launch_bounds__(256, 1) k_trace_yarns(const bysdf_yarn* __restrict__ yarns,
                                                     int n_yarns, TraceArgs a) {
  extern __shared__ float4 smem_pieces[];
  PieceS* ps = reinterpret_cast<PieceS*>(smem_pieces);
  const int n_grp = (n_yarns + kGroupPieces - 1) / kGroupPieces;
  float4* grp = smem_pieces + 4 * n_yarns;  // (centre, squared radius) per group
  int32_t* smat = reinterpret_cast<int32_t*>(grp + n_grp);  // material per piece
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
    smat[k] = y.mat_id;
  }
  __syncthreads();
  // group spheres: the box around the pieces' spheres, then the largest
  // reach from its centre, widened like the piece spheres
  for (int c = threadIdx.x; c < n_grp; c += blockDim.x) {
    const int k0 = c * kGroupPieces, k1 = min(k0 + kGroupPieces, n_yarns);
    float lx = 3.4e38f, ly = 3.4e38f, lz = 3.4e38f, hx = -3.4e38f, hy = -3.4e38f, hz = -3.4e38f;
    for (int k = k0; k < k1; ++k) {
      const float4 d = ps[k].d;
      const float r = sqrtf(d.w);
      lx = fminf(lx, d.x - r);
      ly = fminf(ly, d.y - r);
      lz = fminf(lz, d.z - r);
      hx = fmaxf(hx, d.x + r);
      hy = fmaxf(hy, d.y + r);
      hz = fmaxf(hz, d.z + r);
    }
    const float cx = 0.5f * (lx + hx), cy = 0.5f * (ly + hy), cz = 0.5f * (lz + hz);
    float R = 0.f;
    for (int k = k0; k < k1; ++k) {
      const float4 d = ps[k].d;
      const float ex = d.x - cx, ey = d.y - cy, ez = d.z - cz;
      R = fmaxf(R, sqrtf(dot3(ex, ey, ez, ex, ey, ez)) + sqrtf(d.w));
    }
    R = R * 1.0001f + 1e-4f;
    grp[c] = make_float4(cx, cy, cz, R * R);
  }
  __syncthreads();
  const int64_t n = a.n;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // whole warps step through the rays (lanes past the end take part in the
  // ballots with a dummy ray and write nothing); each lane loads its next ray
  // while the current one is culled
  int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  float nox = 0.f, noy = 0.f, noz = 0.f, ndx = 0.f, ndy = 0.f, ndz = 1.f;
  if (i0 + lane < n) {
    const int64_t j = i0 + lane;
    nox = __ldg(a.o + j), noy = __ldg(a.o + n + j), noz = __ldg(a.o + 2 * n + j);
    ndx = __ldg(a.d + j), ndy = __ldg(a.d + n + j), ndz = __ldg(a.d + 2 * n + j);
  }
  for (; i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const bool act = i < n;
    const float ox = nox, oy = noy, oz = noz, dx = ndx, dy = ndy, dz = ndz;
    if (i + stride < n) {
      const int64_t j = i + stride;
      nox = __ldg(a.o + j), noy = __ldg(a.o + n + j), noz = __ldg(a.o + 2 * n + j);
      ndx = __ldg(a.d + j), ndy = __ldg(a.d + n + j), ndz = __ldg(a.d + 2 * n + j);
    }
    // the differential rays, loaded while the warp culls
    const bool diff = a.ratio && a.o1 && a.d1 && a.o2 && a.d2;
    float o1x = 0.f, o1y = 0.f, o1z = 0.f, d1x = 0.f, d1y = 0.f, d1z = 0.f;
    float o2x = 0.f, o2y = 0.f, o2z = 0.f, d2x = 0.f, d2y = 0.f, d2z = 0.f;
    if (act && diff) {
      o1x = __ldg(a.o1 + i), o1y = __ldg(a.o1 + n + i), o1z = __ldg(a.o1 + 2 * n + i);
      d1x = __ldg(a.d1 + i), d1y = __ldg(a.d1 + n + i), d1z = __ldg(a.d1 + 2 * n + i);
      o2x = __ldg(a.o2 + i), o2y = __ldg(a.o2 + n + i), o2z = __ldg(a.o2 + 2 * n + i);
      d2x = __ldg(a.d2 + i), d2y = __ldg(a.d2 + n + i), d2z = __ldg(a.d2 + 2 * n + i);
    }
    const float idd = 1.0f / dot3(dx, dy, dz, dx, dy, dz);
    const float ild = sqrtf(idd);
    // the warp's bundle: origin oc and unit direction ua of its middle active
    // lane, ro = max |o_i - oc|, del = max |d_i / |d_i| - ua|
    const unsigned am = __ballot_sync(0xffffffffu, act);
    const int src = (__popc(am) - 1) >> 1;  // active lanes are 0 .. popc - 1
    const float ux = dx * ild, uy = dy * ild, uz = dz * ild;
    const float ocx = __shfl_sync(0xffffffffu, ox, src), ocy = __shfl_sync(0xffffffffu, oy, src),
                ocz = __shfl_sync(0xffffffffu, oz, src);
    const float uax = __shfl_sync(0xffffffffu, ux, src), uay = __shfl_sync(0xffffffffu, uy, src),
                uaz = __shfl_sync(0xffffffffu, uz, src);
    float ro = 0.f, del = 0.f;
    if (act) {
      const float ex = ox - ocx, ey = oy - ocy, ez = oz - ocz;
      const float fx = ux - uax, fy = uy - uay, fz = uz - uaz;
      ro = sqrtf(dot3(ex, ey, ez, ex, ey, ez));
      del = sqrtf(dot3(fx, fy, fz, fx, fy, fz));
    }
    // non-negative floats order like their bit patterns
    ro = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(ro)));
    del = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(del)));
    int best = -1;
    float sbest = 0.f;
    for (int c0 = 0; c0 < n_grp; c0 += 32) {
      unsigned gm = __ballot_sync(
          0xffffffffu, c0 + lane < n_grp && bundle_reaches(grp[c0 + lane], ocx, ocy, ocz, uax,
                                                           uay, uaz, ro, del));
      while (gm) {
        // the next four kept groups (offsets in c0, 0xff for none) in bytes
        uint32_t four = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          four |= (gm ? (uint32_t)(__ffs(gm) - 1) : 0xffu) << (8 * q);
          gm &= gm - 1;
        }
        const uint32_t gq = (four >> (8 * (lane >> 3))) & 0xffu;
        const int kl = (c0 + (int)gq) * kGroupPieces + (lane & 7);
        unsigned pm = __ballot_sync(
            0xffffffffu, gq != 0xffu && kl < n_yarns &&
                             bundle_reaches(ps[kl].d, ocx, ocy, ocz, uax, uay, uaz, ro, del));
        while (pm) {
          const int b = __ffs(pm) - 1;
          pm &= pm - 1;
          const int k = (c0 + (int)((four >> (8 * (b >> 3))) & 0xffu)) * kGroupPieces + (b & 7);
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
      }
    }
    if (!act) continue;
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
    a.mat_id[i] = smat[best];
    if (a.ratio) {
      // Sec. 5.3: the differential rays' offsets about the same axis bound
      // the footprint; the record carries its half-width in h
      float r = 0.f;
      if (diff) {
        const float h1 = line_offset(p, bx, by, bz, o1x, o1y, o1z, d1x, d1y, d1z);
        const float h2 = line_offset(p, bx, by, bz, o2x, o2y, o2z, d2x, d2y, d2z);
        const float w1 = fabsf(h1 - h0), w2 = fabsf(h2 - h0);
        r = (isfinite(w1) && isfinite(w2)) ? fmaxf(w1, w2) : 2.0f;
      }
      a.ratio[i] = r;
    }
  }
}

cudaError_t launch_trace_yarns(const bysdf_yarn* yarns, int n_yarns, const TraceArgs& a,
                               int grid, cudaStream_t st) {
  const int n_grp = (n_yarns + kGroupPieces - 1) / kGroupPieces;
  const size_t smem = sizeof(PieceS) * (size_t)n_yarns + sizeof(float4) * (size_t)n_grp +
                      sizeof(int32_t) * (size_t)n_yarns;
  cudaError_t e;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_trace_yarns, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
  }
  // one resident wave: every CTA stages the pieces once
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_yarns, 256, smem)) !=
          cudaSuccess)
    return e;
  if (per_sm > 0 && grid > sms * per_sm) grid = sms * per_sm;
  k_trace_yarns<<<grid, 256, smem, st>>>(yarns, n_yarns, a);
  return cudaGetLastError();
}

}  // namespace bysdf
