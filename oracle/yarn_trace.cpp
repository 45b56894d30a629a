// FP64 oracle of camera rays against explicit yarn pieces (Sec. 3.3, 5.3).
// TEST INFRASTRUCTURE ONLY; shares no code with the CUDA library.
#include "yarn_trace.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace {

const double PI = 3.14159265358979323846;

struct V {
  double x, y, z;
};
V operator+(V a, V b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V operator-(V a, V b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V operator*(V a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dot(V a, V b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V cross(V a, V b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V load(const double* p) { return {p[0], p[1], p[2]}; }
V plane(const float* p, int64_t i, int64_t n) {
  return {(double)p[i], (double)p[n + i], (double)p[2 * n + i]};
}

// component of a perpendicular to the unit axis t
V perp(V a, V t) { return a - t * dot(a, t); }

// signed distance of the line (o, d) from the axis (p0, t), over R, measured
// in the cross-section: (q_perp x e) . t / R with e the unit in-plane
// direction; +-inf for a ray along the axis
double offset(const orc_yarn& y, V o, V d) {
  const V t = load(y.t);
  const V q = perp(o - load(y.p0), t);
  const V dp = perp(d, t);
  const double l = std::sqrt(dot(dp, dp));
  if (!(l > 0.0)) return HUGE_VAL;
  return dot(cross(q, dp * (1.0 / l)), t) / y.radius;
}

// entry of the ray into the lateral surface of piece y: ray parameter, or
// -1 when the ray misses it, runs along its axis, or starts inside it
double entry(const orc_yarn& y, V o, V d) {
  const V t = load(y.t);
  const V q = o - load(y.p0);
  const V qp = perp(q, t), dp = perp(d, t);
  const double a = dot(dp, dp);
  if (!(a > 1e-24)) return -1.0;
  const double b = dot(qp, dp), c = dot(qp, qp) - y.radius * y.radius;
  if (!(c > 0.0)) return -1.0;  // origin inside (or on) the cylinder
  const double disc = b * b - a * c;
  if (disc < 0.0) return -1.0;
  const double s = (-b - std::sqrt(disc)) / a;
  if (!(s > 0.0)) return -1.0;
  const double w = dot(q + d * s, t);
  if (w < 0.0 || w > y.length) return -1.0;
  return s;
}

// the piece with its frame made orthonormal: t / |t|, then n_ref without
// its t component, normalised (the inputs are unit to float32 precision)
orc_yarn frame(const orc_yarn& y) {
  orc_yarn o = y;
  V t = load(y.t);
  t = t * (1.0 / std::sqrt(dot(t, t)));
  V n = perp(load(y.n_ref), t);
  n = n * (1.0 / std::sqrt(dot(n, n)));
  o.t[0] = t.x; o.t[1] = t.y; o.t[2] = t.z;
  o.n_ref[0] = n.x; o.n_ref[1] = n.y; o.n_ref[2] = n.z;
  return o;
}

template <class F>
void parallel_for(int64_t n, int n_threads, F&& body) {
  if (n_threads <= 1 || n < 1024) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + n_threads - 1) / n_threads;
  for (int k = 0; k < n_threads; ++k) {
    const int64_t b = k * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([&, b, e] { body(b, e); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

extern "C" int orc_trace_yarns(const orc_yarn* ys, int n_yarn, const orc_rays* r, int64_t n,
                               const double light[3], double* h, double* u, double* v,
                               double* wi, double* wo, double* ratio, double* t_hit,
                               int32_t* yarn, int32_t* mat_id, int n_threads) {
  const V L = {light[0], light[1], light[2]};
  std::vector<orc_yarn> yv(n_yarn);
  for (int k = 0; k < n_yarn; ++k) yv[k] = frame(ys[k]);
  const orc_yarn* yy = yv.data();
  parallel_for(n, n_threads, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      const V o = plane(r->o, i, n), d = plane(r->d, i, n);
      int best = -1;
      double sb = 0.0;
      for (int k = 0; k < n_yarn; ++k) {
        const double s = entry(yy[k], o, d);
        if (s > 0.0 && (best < 0 || s < sb)) {
          best = k;
          sb = s;
        }
      }
      yarn[i] = best;
      h[i] = u[i] = v[i] = ratio[i] = t_hit[i] = 0.0;
      for (int c = 0; c < 3; ++c) wi[c * n + i] = wo[c * n + i] = 0.0;
      mat_id[i] = -1;
      if (best < 0) continue;
      const orc_yarn& y = yy[best];
      const V t = load(y.t), nr = load(y.n_ref), br = cross(t, nr);
      const V x = o + d * sb;
      const double w = dot(x - load(y.p0), t);
      const V xp = x - load(y.p0) - t * w;
      const V nu = xp * (1.0 / std::sqrt(dot(xp, xp)));
      double uu = std::atan2(dot(nu, br), dot(nu, nr));
      if (uu < 0.0) uu += 2.0 * PI;
      const V dp = perp(d, t);
      const V ep = dp * (1.0 / std::sqrt(dot(dp, dp)));
      const double ex = dot(ep, nr), ey = dot(ep, br);
      const double nx = std::cos(uu), ny = std::sin(uu);
      double hh = nx * ey - ny * ex;
      hh = std::max(-1.0, std::min(1.0, hh));
      h[i] = hh;
      u[i] = uu;
      v[i] = y.v0 + w;
      t_hit[i] = sb;
      mat_id[i] = y.mat_id;
      const V mwi = d * -1.0;
      wi[i] = dot(mwi, nr);
      wi[n + i] = dot(mwi, br);
      wi[2 * n + i] = dot(mwi, t);
      wo[i] = dot(L, nr);
      wo[n + i] = dot(L, br);
      wo[2 * n + i] = dot(L, t);
      // Sec. 5.3: the differential rays' azimuthal offsets about the same
      // axis bound the footprint [h1, h2]; the record carries its half-width
      if (r->o1 && r->d1 && r->o2 && r->d2) {
        const double h1 = offset(y, plane(r->o1, i, n), plane(r->d1, i, n));
        const double h2 = offset(y, plane(r->o2, i, n), plane(r->d2, i, n));
        const double w1 = std::fabs(h1 - hh), w2 = std::fabs(h2 - hh);
        ratio[i] = std::isfinite(w1) && std::isfinite(w2) ? std::max(w1, w2) : 2.0;
      }
    }
  });
  return 0;
}
