// FP64 oracle of the yarn-level BYSDF.  TEST INFRASTRUCTURE ONLY (see header).
//
// The model is written once, generic in the scalar type S:
//   S = double      -> values,
//   S = Dual<8>     -> exact forward-mode derivatives w.r.t. the 8 material
//                      parameters (albedo RGB, beta_t, beta_b, alpha_p,
//                      alpha_f, sigma_s),
//   S = Cnt         -> operation counts of one evaluation.
// No blocking, fusion or reordering: each function is one step of the paper.
#include "bysdf_oracle.h"

#include <algorithm>
#include <cmath>
#include <thread>
#include <utility>
#include <vector>

namespace {

constexpr double PI = 3.14159265358979323846;

// ------------------------------------------------------------------ scalars --
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
  Dual(double x) : v(x) { for (int k = 0; k < N; ++k) d[k] = 0.0; }
};
template <int N>
Dual<N> chain(const Dual<N>& a, double fv, double dfda) {
  Dual<N> r(fv);
  for (int k = 0; k < N; ++k) r.d[k] = dfda * a.d[k];
  return r;
}
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v);
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v);
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v);
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  const double q = a.v / b.v;
  Dual<N> r(q);
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - q * b.d[k]) / b.v;
  return r;
}
template <int N> Dual<N> operator-(const Dual<N>& a) { return chain(a, -a.v, -1.0); }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> bool operator<(const Dual<N>& a, double b) { return a.v < b; }
template <int N> bool operator<(double a, const Dual<N>& b) { return a < b.v; }
template <int N> bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> bool operator>(const Dual<N>& a, double b) { return a.v > b; }
template <int N> bool operator>(double a, const Dual<N>& b) { return a > b.v; }
template <int N> bool operator<=(const Dual<N>& a, double b) { return a.v <= b; }
template <int N> bool operator>=(const Dual<N>& a, double b) { return a.v >= b; }
template <int N> Dual<N> sqrt(const Dual<N>& a) {
  const double s = std::sqrt(a.v);
  return chain(a, s, s > 0.0 ? 0.5 / s : 0.0);
}
template <int N> Dual<N> sin(const Dual<N>& a) { return chain(a, std::sin(a.v), std::cos(a.v)); }
template <int N> Dual<N> cos(const Dual<N>& a) { return chain(a, std::cos(a.v), -std::sin(a.v)); }
template <int N> Dual<N> tan(const Dual<N>& a) {
  const double t = std::tan(a.v);
  return chain(a, t, 1.0 + t * t);
}
template <int N> Dual<N> exp(const Dual<N>& a) {
  const double e = std::exp(a.v);
  return chain(a, e, e);
}
template <int N> Dual<N> log(const Dual<N>& a) { return chain(a, std::log(a.v), 1.0 / a.v); }
template <int N> Dual<N> asin(const Dual<N>& a) {
  return chain(a, std::asin(a.v), 1.0 / std::sqrt(1.0 - a.v * a.v));
}
template <int N> Dual<N> atan2(const Dual<N>& y, const Dual<N>& x) {
  const double r2 = x.v * x.v + y.v * y.v;
  Dual<N> r(std::atan2(y.v, x.v));
  for (int k = 0; k < N; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) / r2;
  return r;
}

// Operation-counting scalar: counters indexed add, mul, div, sqrt, trans, cmp.
thread_local double g_ops[6];
struct Cnt {
  double v;
  Cnt(double x = 0.0) : v(x) {}
};
inline Cnt cnt(int k, double v) { g_ops[k] += 1.0; return Cnt(v); }
inline Cnt operator+(Cnt a, Cnt b) { return cnt(0, a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { return cnt(0, a.v - b.v); }
inline Cnt operator*(Cnt a, Cnt b) { return cnt(1, a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { return cnt(2, a.v / b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator+(Cnt a, double b) { return a + Cnt(b); }
inline Cnt operator+(double a, Cnt b) { return Cnt(a) + b; }
inline Cnt operator-(Cnt a, double b) { return a - Cnt(b); }
inline Cnt operator-(double a, Cnt b) { return Cnt(a) - b; }
inline Cnt operator*(Cnt a, double b) { return a * Cnt(b); }
inline Cnt operator*(double a, Cnt b) { return Cnt(a) * b; }
inline Cnt operator/(Cnt a, double b) { return a / Cnt(b); }
inline Cnt operator/(double a, Cnt b) { return Cnt(a) / b; }
inline bool cmpc(bool r) { g_ops[5] += 1.0; return r; }
inline bool operator<(Cnt a, Cnt b) { return cmpc(a.v < b.v); }
inline bool operator<(Cnt a, double b) { return cmpc(a.v < b); }
inline bool operator<(double a, Cnt b) { return cmpc(a < b.v); }
inline bool operator>(Cnt a, Cnt b) { return cmpc(a.v > b.v); }
inline bool operator>(Cnt a, double b) { return cmpc(a.v > b); }
inline bool operator>(double a, Cnt b) { return cmpc(a > b.v); }
inline bool operator<=(Cnt a, double b) { return cmpc(a.v <= b); }
inline bool operator>=(Cnt a, double b) { return cmpc(a.v >= b); }
inline Cnt sqrt(Cnt a) { return cnt(3, std::sqrt(a.v)); }
inline Cnt sin(Cnt a) { return cnt(4, std::sin(a.v)); }
inline Cnt cos(Cnt a) { return cnt(4, std::cos(a.v)); }
inline Cnt tan(Cnt a) { return cnt(4, std::tan(a.v)); }
inline Cnt exp(Cnt a) { return cnt(4, std::exp(a.v)); }
inline Cnt log(Cnt a) { return cnt(4, std::log(a.v)); }
inline Cnt asin(Cnt a) { return cnt(4, std::asin(a.v)); }
inline Cnt atan2(Cnt y, Cnt x) { return cnt(4, std::atan2(y.v, x.v)); }

// Discontinuity margins (for the parity tests): at each branch point of the
// model -- and at the steep spots where a result changes faster than rounding
// can be controlled -- the evaluation notes how far the deciding quantity is
// from its threshold, in the quantity's own units (lengths in yarn radii,
// cosines, fiber periods, probabilities).  A record's margin in class k is the
// smallest distance noted in that class.  Only evaluations with a margin
// buffer set (orc_margins) note anything.
enum {
  MG_GRAZE = 0,   // ply trace: ray vs ply circle tangent, every update (Sec. 3.4)
  MG_GAP,         // closest ply: gap to the next hit ply's distance (Sec. 3.4)
  MG_CUSP,        // fiber maps: distance to the cusp texel interval (Sec. 3.5.1)
  MG_AXIS,        // in-plane length of omega_i (rays along the yarn axis)
  MG_HEMI,        // hemisphere side of omega_i / omega_o at the shading normal
  MG_EXIT,        // transmission: entry / exit sides, total internal reflection (Sec. 4.1.2)
  MG_LOBE,        // lobe choice by u0 (Sec. 4.1.5)
  MG_SAMPLE,      // validity of the sampled direction, sampler frame
  MG_SHADOW,      // ply shadowing: shadow ray vs another ply's circle (Sec. 4.1.4)
  MG_KINK,        // fiber maps: distance to a texel centre, where the slope changes
  MG_N = 10
};
thread_local double* g_mg = nullptr;
inline void mg(int k, double dist) {
  if (g_mg) g_mg[k] = std::min(g_mg[k], std::fabs(dist));
}
// Offsets of two internal quantities (for the parity tests' conditioning
// measure, which asks how far the result moves when they carry the rounding
// of a float32 evaluation): the in-plane hit distance t of every node and
// the ply azimuth u_ply that sets the fiber phase.  Zero except between
// orc_set_internal_offsets calls; process-wide, set between evaluations.
double g_off_t = 0.0, g_off_uply = 0.0;

inline double val(double x) { return x; }
template <int N> double val(const Dual<N>& x) { return x.v; }
inline double val(const Cnt& x) { return x.v; }

template <class S> S smax(const S& a, const S& b) { return (a < b) ? b : a; }
template <class S> S smin(const S& a, const S& b) { return (b < a) ? b : a; }
template <class S> S sabs(const S& a) { return (a < 0.0) ? -a : a; }
template <class S> S sqr(const S& a) { return a * a; }

// ------------------------------------------------------------------ vectors --
template <class S>
struct V3 {
  S x, y, z;
};
template <class S> V3<S> mk(const S& x, const S& y, const S& z) { return V3<S>{x, y, z}; }
template <class S> V3<S> operator+(const V3<S>& a, const V3<S>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class S> V3<S> operator-(const V3<S>& a, const V3<S>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class S> V3<S> operator-(const V3<S>& a) { return {-a.x, -a.y, -a.z}; }
template <class S, class T> V3<S> operator*(const V3<S>& a, const T& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class S> S dot(const V3<S>& a, const V3<S>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class S> V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class S> S norm(const V3<S>& a) { using std::sqrt; return sqrt(dot(a, a)); }
template <class S> V3<S> normalize(const V3<S>& a) { return a * (S(1.0) / norm(a)); }
template <class S> V3<S> lift(const double* p) { return {S(p[0]), S(p[1]), S(p[2])}; }
// dot product of the values (margin notes: not part of the counted work)
template <class S> double dotv(const V3<S>& a, const V3<S>& b) {
  return val(a.x) * val(b.x) + val(a.y) * val(b.y) + val(a.z) * val(b.z);
}

// ---------------------------------------------------------------- material --
// Ply and fiber layout.  The paper gives no layout (Sec. 3.4, 3.5); reading:
// N_p equal ply discs inscribed in the yarn circle, touching it and their
// neighbours; N_f fibers of equal radius filling a fraction `packing` of a
// ply disc; the outer ring has M = ceil(pi / asin(r_f / R_fc)) fibers, the
// fewest whose circles close the ring.
struct Layout {
  bool ok = false;
  double R = 1, Rp = 1, Rc = 0, rf = 0, Rfc = 0;
  int M = 0;
};

Layout make_layout(const orc_material& d) {
  Layout L;
  if (d.n_plies < 1 || d.n_plies > 8 || d.fibers_per_ply < 4 ||
      d.fibers_per_ply > 4096 || !(d.packing > 0.0 && d.packing <= 1.0) ||
      !(d.yarn_radius > 0.0) || d.map_texels < 4 || d.map_texels > 4096 ||
      d.trace_iters < 1 || d.trace_iters > 64 || d.k_max < 1 || d.k_max > 64 ||
      !(d.eta > 1.0) || !(d.body_B >= 0.0 && d.body_B <= 1.0) ||
      !(d.body_r >= 0.0 && d.body_r <= 1.0) || !std::isfinite(d.albedo_y[0]) ||
      !std::isfinite(d.albedo_y[1]) || !std::isfinite(d.albedo_y[2]))
    return L;
  L.R = d.yarn_radius;
  if (d.n_plies == 1) {
    L.Rp = L.R;
    L.Rc = 0.0;
  } else {
    const double s = std::sin(PI / d.n_plies);
    L.Rp = L.R * s / (1.0 + s);
    L.Rc = L.R / (1.0 + s);
  }
  L.rf = L.Rp * std::sqrt(d.packing / d.fibers_per_ply);
  L.Rfc = L.Rp - L.rf;
  if (!(L.rf < L.Rfc)) return L;
  L.M = (int)std::ceil(PI / std::asin(L.rf / L.Rfc));
  L.ok = true;
  return L;
}

// Sec. 3.5.1: the outer fibers of a ply cross-section seen along the radial
// direction.  D is the angular offset of the radial line from a fiber centre.
// The radial line meets that fiber at rho = R_fc cos D + sqrt(r_f^2 - R_fc^2
// sin^2 D); delta is the angle of the fiber normal from the radial direction.
double fiber_delta(const Layout& L, double D) {
  const double s = L.Rfc * std::sin(D);
  const double c2 = std::max(L.rf * L.rf - s * s, 0.0);
  return std::atan2(s, std::sqrt(c2));
}

// Sec. 4.1.4 (fiber shadowing): fraction of the outward half-plane of
// directions at the fiber surface point that the other outer-ring fibers block
// (union of the angular intervals they subtend), a value in [0, 1].
double fiber_occlusion(const Layout& L, double D) {
  const double s = L.Rfc * std::sin(D);
  const double c2 = std::max(L.rf * L.rf - s * s, 0.0);
  const double rho = L.Rfc * std::cos(D) + std::sqrt(c2);
  const double px = rho * std::cos(D), py = rho * std::sin(D);
  const double nx = (px - L.Rfc) / L.rf, ny = py / L.rf;
  const double phin = std::atan2(ny, nx);
  std::vector<std::pair<double, double>> iv;
  for (int j = 1; j < L.M; ++j) {
    const double a = 2.0 * PI * j / L.M;
    const double wx = L.Rfc * std::cos(a) - px, wy = L.Rfc * std::sin(a) - py;
    const double dist = std::sqrt(wx * wx + wy * wy);
    const double half = dist <= L.rf ? PI / 2 : std::asin(L.rf / dist);
    double c = std::atan2(wy, wx) - phin;
    while (c > PI) c -= 2 * PI;
    while (c <= -PI) c += 2 * PI;
    for (int w = -1; w <= 1; ++w) {
      const double lo = std::max(c - half + 2 * PI * w, -PI / 2);
      const double hi = std::min(c + half + 2 * PI * w, PI / 2);
      if (hi > lo) iv.push_back({lo, hi});
    }
  }
  std::sort(iv.begin(), iv.end());
  double meas = 0.0, cur_lo = 0.0, cur_hi = 0.0;
  bool open = false;
  for (auto& p : iv) {
    if (!open) {
      cur_lo = p.first; cur_hi = p.second; open = true;
    } else if (p.first <= cur_hi) {
      cur_hi = std::max(cur_hi, p.second);
    } else {
      meas += cur_hi - cur_lo;
      cur_lo = p.first; cur_hi = p.second;
    }
  }
  if (open) meas += cur_hi - cur_lo;
  return meas / PI;
}

// Material-constant part: layout and the two 1D maps, tabulated at T texel
// centres over one fiber period (Sec. 3.5.1 "1D texture"; Sec. 4.1.4).
struct MatStatic {
  orc_material d;
  Layout L;
  std::vector<double> tab_delta, tab_of;
  // fiber migration: layouts and maps of the sunk rings k = 1 .. K_m - 1
  // (index 0 repeats the regular ring's)
  std::vector<Layout> Lm;
  std::vector<std::vector<double>> mig_delta, mig_of;
};

// Map k of a migrating ply (reading): the outer ring sunk by k r_f / K_m,
// holding as many fibers as fit on it.
Layout migration_layout(const Layout& L, int k, int K) {
  Layout Lk = L;
  Lk.Rfc = L.Rfc - k * L.rf / K;
  Lk.ok = L.rf < Lk.Rfc;
  if (Lk.ok) Lk.M = (int)std::ceil(PI / std::asin(L.rf / Lk.Rfc));
  return Lk;
}

void tabulate(const Layout& L, int T, bool flat, std::vector<double>& dl,
              std::vector<double>& of) {
  dl.assign(T, 0.0);
  of.assign(T, 0.0);
  if (flat) return;
  for (int i = 0; i < T; ++i) {
    const double D = ((i + 0.5) / T - 0.5) * 2.0 * PI / L.M;
    dl[i] = fiber_delta(L, D);
    of[i] = fiber_occlusion(L, D);
  }
}

bool build_static(const orc_material& d, MatStatic& st) {
  st.d = d;
  st.L = make_layout(d);
  if (!st.L.ok) return false;
  const int T = d.map_texels;
  const bool flat = (d.flags & 1) != 0;
  tabulate(st.L, T, flat, st.tab_delta, st.tab_of);
  const int K = d.migration_maps;
  if (K < 1 || K > 4) return false;
  if (K > 1 && !(d.migration_length > 0.0 && std::isfinite(d.migration_length) &&
                 d.migration_blend > 0.0 && d.migration_blend <= 0.5))
    return false;
  st.Lm.assign(K, st.L);
  st.mig_delta.assign(K, st.tab_delta);
  st.mig_of.assign(K, st.tab_of);
  for (int k = 1; k < K; ++k) {
    st.Lm[k] = migration_layout(st.L, k, K);
    if (!st.Lm[k].ok) return false;
    tabulate(st.Lm[k], T, flat, st.mig_delta[k], st.mig_of[k]);
  }
  return true;
}

template <class S>
struct Mat {
  const MatStatic* st;
  S alb[3], beta_t, beta_b, alpha_p, alpha_f, sigma_s;
  S omega_p, omega_f;  // angular rates of the ply and fiber helices (rad / length)
  // Sec. 4.1.3 / 4.1.5 weights and Eq. 4 attenuation (the paper's fitting set)
  S body_r, body_B, sigma_t, k_spec;
  S alb_y[3];  // k^B_y of Eq. 6 (equal to alb unless the material sets it)
  S omega_fm[4];  // fiber phase rates of the migration maps' rings
};

template <class S> void seed(S&, int) {}
template <int N> void seed(Dual<N>& x, int k) {
  if (k < N) x.d[k] = 1.0;
}

// ext: seed the 15 parameters of ORC_NPARAM_EXT; otherwise the 8 of
// ORC_NPARAM, where the albedo tangent moves k^B_x and k^B_y together
template <class S>
Mat<S> make_mat(const MatStatic& st, bool with_tangents, bool ext = false) {
  using std::tan;
  Mat<S> m;
  m.st = &st;
  const orc_material& d = st.d;
  for (int c = 0; c < 3; ++c) m.alb[c] = S(d.albedo[c]);
  m.beta_t = S(d.beta_deg[0] * PI / 180.0);
  m.beta_b = S(d.beta_deg[1] * PI / 180.0);
  m.alpha_p = S(d.ply_twist_deg * PI / 180.0);
  m.alpha_f = S(d.fiber_twist_deg * PI / 180.0);
  m.sigma_s = S(d.shadow_density);
  m.body_r = S(d.body_r);
  m.body_B = S(d.body_B);
  m.sigma_t = S(d.sigma_t);
  m.k_spec = S(d.k_spec);
  for (int c = 0; c < 3; ++c) m.alb_y[c] = S(d.albedo_y[c] < 0.0 ? d.albedo[c] : d.albedo_y[c]);
  if (with_tangents) {
    for (int c = 0; c < 3; ++c) {
      seed(m.alb[c], ORC_P_ALB_R + c);
      seed(m.alb_y[c], ext ? ORC_P_ALBY_R + c : ORC_P_ALB_R + c);
    }
    seed(m.beta_t, ORC_P_BETA_T);
    seed(m.beta_b, ORC_P_BETA_B);
    seed(m.alpha_p, ORC_P_ALPHA_P);
    seed(m.alpha_f, ORC_P_ALPHA_F);
    seed(m.sigma_s, ORC_P_SIGMA_S);
    seed(m.body_r, ORC_P_BODY_R);
    seed(m.body_B, ORC_P_BODY_B);
    seed(m.sigma_t, ORC_P_SIGMA_T);
    seed(m.k_spec, ORC_P_K_SPEC);
  }
  // Helix about the yarn axis at radius R_c with helix angle alpha_p; a single
  // ply sits on the axis and does not wind (Sec. 3.4).
  m.omega_p = d.n_plies == 1 ? S(0.0) : tan(m.alpha_p) / st.L.Rc;
  m.omega_f = tan(m.alpha_f) / st.L.Rfc;
  for (size_t k = 0; k < st.Lm.size(); ++k) m.omega_fm[k] = tan(m.alpha_f) / st.Lm[k].Rfc;
  return m;
}

// ----------------------------------------------------------------- records --
struct Rec {
  double h, u, v, wi[3], wo[3], ratio, u0, u1;
  bool has_ratio;
  int mat;
};

Rec read_rec(const orc_records* r, int64_t i, int64_t n) {
  Rec q{};
  q.h = r->h[i];
  q.u = r->u[i];
  q.v = r->v[i];
  for (int c = 0; c < 3; ++c) {
    q.wi[c] = r->wi[c * n + i];
    q.wo[c] = r->wo ? (double)r->wo[c * n + i] : 0.0;
  }
  q.has_ratio = r->ratio != nullptr;
  q.ratio = q.has_ratio ? (double)r->ratio[i] : 0.0;
  q.u0 = r->u0 ? (double)r->u0[i] : 0.0;
  q.u1 = r->u1 ? (double)r->u1[i] : 0.0;
  q.mat = r->mat_id ? r->mat_id[i] : 0;
  return q;
}

// Input validation (status 2): non-finite values, |h| > 1, direction norms off
// by more than 1e-3, a material id out of range, a negative ratio, random
// numbers outside [0, 1).
bool valid_rec(const Rec& q, int n_mat, bool need_wo, bool need_u) {
  auto fin = [](double x) { return std::isfinite(x); };
  if (!fin(q.h) || !fin(q.u) || !fin(q.v)) return false;
  for (int c = 0; c < 3; ++c)
    if (!fin(q.wi[c]) || (need_wo && !fin(q.wo[c]))) return false;
  if (std::fabs(q.h) > 1.0) return false;
  const double ni = q.wi[0] * q.wi[0] + q.wi[1] * q.wi[1] + q.wi[2] * q.wi[2];
  if (std::fabs(ni - 1.0) > 1e-3) return false;
  if (need_wo) {
    const double no = q.wo[0] * q.wo[0] + q.wo[1] * q.wo[1] + q.wo[2] * q.wo[2];
    if (std::fabs(no - 1.0) > 1e-3) return false;
  }
  if (q.mat < 0 || q.mat >= n_mat) return false;
  if (q.has_ratio && !(q.ratio >= 0.0)) return false;
  if (q.has_ratio && !std::isfinite(q.ratio)) return false;
  if (need_u && !(q.u0 >= 0.0 && q.u0 < 1.0 && q.u1 >= 0.0 && q.u1 < 1.0)) return false;
  return true;
}

// ------------------------------------------------------------- randomness --
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC 2011): ten rounds of two 64x64 -> 128-bit multiplies
// of the counter words, key bumped by the Weyl constants between rounds.
struct Philox4x64 {
  uint64_t w[4];
};
Philox4x64 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                      uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  uint64_t c[4] = {c0, c1, c2, c3};
  for (int r = 0; r < 10; ++r) {
    const unsigned __int128 p0 = (unsigned __int128)M0 * c[0];
    const unsigned __int128 p1 = (unsigned __int128)M1 * c[2];
    const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
  return Philox4x64{{c[0], c[1], c[2], c[3]}};
}
// 24 high bits of a word as a float in [0, 1)
double unit24(uint64_t w) { return (double)(w >> 40) * (1.0 / 16777216.0); }

// Stochastic estimators (Sec. 4.2 stratified h nodes; Eq. 1's Omega_y
// integral with a GGX-sampled refraction).  Record index `index`: node j's
// jitter is word j % 4 of the block with counter (index, j / 4, 0, 0); the
// entry microfacet takes words 0 and 1 of block (index, 16, 0, 0); key
// (seed, ORC_STOCH_KEY1).
struct Stoch {
  bool jitter = false, rough = false;
  uint64_t seed = 0;
  uint64_t index = 0;
  double xi(int j) const {
    const Philox4x64 r = philox4x64(index, (uint64_t)(j / 4), 0, 0, seed, ORC_STOCH_KEY1);
    return unit24(r.w[j % 4]);
  }
  void entry(double* v0, double* v1) const {
    const Philox4x64 r = philox4x64(index, 16, 0, 0, seed, ORC_STOCH_KEY1);
    *v0 = unit24(r.w[0]);
    *v1 = unit24(r.w[1]);
  }
};

// --------------------------------------------------------------- geometry --
// One node of the implicit geometry: the camera ray entering the yarn at
// in-plane point X0 with in-plane unit direction e and longitudinal slope
// kappa (dz per unit in-plane distance).
template <class S>
struct Node {
  bool hit = false;
  int ni = 0, k = -1;
  V3<S> x, np, tp, nf, tf;
  S gp = S(1.0), gf = S(1.0);
  S u_ply = S(0.0), delta = S(0.0), of = S(0.0);
  double t_ply[8];
  double residual = 0.0;
};

// Sec. 3.5.1: periodic linear interpolation of a map tabulated at texel
// centres; theta_f is the fiber phase (radians), one period is 2 pi / M.
template <class S>
void fiber_lookup_tab(const MatStatic& st, int Mk, const std::vector<double>& tab_delta,
                      const std::vector<double>& tab_of, const S& theta_f, S* delta, S* of) {
  const int T = st.d.map_texels;
  const S w = theta_f * (Mk / (2.0 * PI));
  const S a = w + 0.5 - std::floor(val(w + 0.5));
  const S tau = a * (double)T - 0.5;
  const double fl = std::floor(val(tau));
  // margin: the interval between the last and the first texel centre holds
  // the cusp, where delta jumps across the whole fiber; distance to it in
  // fiber periods (0 inside)
  {
    const double tv = val(tau);
    mg(MG_CUSP, (tv < 0.0 || tv >= T - 1.0) ? 0.0 : std::min(tv, (T - 1.0) - tv) / T);
    // the interpolant's slope changes at every texel centre: the value is
    // continuous there, its derivatives are not
    mg(MG_KINK, (tv - std::floor(tv + 0.5)) / T);
  }
  const S f = tau - fl;
  const int i0 = (((int)fl) % T + T) % T;
  const int i1 = (i0 + 1) % T;
  *delta = (1.0 - f) * tab_delta[i0] + f * tab_delta[i1];
  *of = (1.0 - f) * tab_of[i0] + f * tab_of[i1];
}
template <class S>
void fiber_lookup(const MatStatic& st, const S& theta_f, S* delta, S* of) {
  fiber_lookup_tab(st, st.L.M, st.tab_delta, st.tab_of, theta_f, delta, of);
}

// Sec. 4.1.4 (ply shadowing), reading: occlusion of x on ply k by the other
// plies of the same cross-section, as the summed chord length of the in-plane
// ray from x towards omega_i through the other ply discs, in units of a ply
// diameter.  psi_k is the phase of ply k in that cross-section.
template <class S>
S ply_occlusion(const Mat<S>& m, int k, const S& psi_k, const S& xx, const S& xy,
                const S& wx, const S& wy) {
  using std::cos;
  using std::sin;
  using std::sqrt;
  const Layout& L = m.st->L;
  const int Np = m.st->d.n_plies;
  S occ = S(0.0);
  for (int j = 0; j < Np; ++j) {
    if (j == k) continue;
    const S psi = psi_k + 2.0 * PI * (j - k) / Np;
    const S cx = L.Rc * cos(psi), cy = L.Rc * sin(psi);
    const S qx = xx - cx, qy = xy - cy;
    const S b = qx * wx + qy * wy;
    const S cc = qx * qx + qy * qy - L.Rp * L.Rp;
    const S disc = b * b - cc;
    // margin: the shadow ray grazing ply j's circle ahead of x (the chord
    // length has an infinite slope there)
    if (val(-b) + L.Rp > 0.0)
      mg(MG_SHADOW, L.Rp - std::sqrt(std::max(L.Rp * L.Rp - val(disc), 0.0)));
    if (disc > 0.0) {
      const S sq = sqrt(disc);
      const S s1 = -b - sq, s2 = -b + sq;
      if (s2 > 0.0) occ = occ + (s2 - ((s1 > 0.0) ? s1 : S(0.0)));
    }
  }
  return occ / (2.0 * L.Rp);
}

// Sec. 3.5 fiber migration (reading): the map of segment `seg` along the
// yarn; the choice repeats every 256 segments ("periodically and randomly")
int migration_map(const MatStatic& st, int64_t seg) {
  const uint64_t s256 = (uint64_t)(((seg % 256) + 256) % 256);
  const Philox4x64 r = philox4x64(s256, 0, 0, 0, (uint64_t)(uint32_t)st.d.migration_seed,
                                  ORC_MIG_KEY1);
  return (int)(r.w[0] % (uint64_t)st.d.migration_maps);
}

// delta and o_f at ply azimuth u_ply and height z of a migrating ply: the
// segment's map, blended linearly with the neighbour's within the blend
// fraction of the segment length from a boundary (weight 1/2 at the
// boundary, so the maps switch continuously)
template <class S>
void migration_lookup(const Mat<S>& m, const S& u_ply, const S& z, S* delta, S* of) {
  using std::floor;
  const MatStatic& st = *m.st;
  const double L = st.d.migration_length, b = st.d.migration_blend;
  const S q = z / L;
  const double sf = std::floor(val(q));
  const S t = q - sf;
  const int64_t seg = (int64_t)sf;
  S w = S(0.0);
  int64_t nb = seg;
  if (val(t) < b) {
    w = 0.5 - t / (2.0 * b);
    nb = seg - 1;
  } else if (val(t) > 1.0 - b) {
    w = 0.5 - (1.0 - t) / (2.0 * b);
    nb = seg + 1;
  }
  const int k0 = migration_map(st, seg);
  S d0, o0;
  fiber_lookup_tab(st, st.Lm[k0].M, st.mig_delta[k0], st.mig_of[k0],
                   u_ply - m.omega_fm[k0] * z, &d0, &o0);
  if (!(val(w) > 0.0)) {
    *delta = d0;
    *of = o0;
    return;
  }
  const int k1 = migration_map(st, nb);
  S d1, o1;
  fiber_lookup_tab(st, st.Lm[k1].M, st.mig_delta[k1], st.mig_of[k1],
                   u_ply - m.omega_fm[k1] * z, &d1, &o1);
  *delta = (1.0 - w) * d0 + w * d1;
  *of = (1.0 - w) * o0 + w * o1;
}

template <class S>
Node<S> node_geometry(const Mat<S>& m, double X0x, double X0y, double ex,
                      double ey, double v, const S& kappa, const V3<S>& wi) {
  using std::atan2;
  using std::cos;
  using std::exp;
  using std::sin;
  using std::sqrt;
  const MatStatic& st = *m.st;
  const Layout& L = st.L;
  const int Np = st.d.n_plies;
  Node<S> g;
  for (int k = 0; k < 8; ++k) g.t_ply[k] = -1.0;
  // Sec. 3.4: per ply, start in the cross-section at the yarn hit, intersect
  // the in-plane ray with the ply circle there, move to the cross-section of
  // that intersection and repeat (N_it updates).  A step whose circle the ray
  // misses means the ply is not hit.
  int best = -1;
  S best_t = S(0.0), best_cx = S(0.0), best_cy = S(0.0), best_psi = S(0.0);
  for (int k = 0; k < Np; ++k) {
    S t = S(0.0), cx = S(0.0), cy = S(0.0), psi = S(0.0);
    bool hit = true;
    for (int n = 0; n < st.d.trace_iters; ++n) {
      const S z = v + kappa * t;
      psi = 2.0 * PI * k / Np + m.omega_p * z;
      cx = L.Rc * cos(psi);
      cy = L.Rc * sin(psi);
      const S qx = X0x - cx, qy = X0y - cy;
      const S b = qx * ex + qy * ey;
      const S cc = qx * qx + qy * qy - L.Rp * L.Rp;
      const S disc = b * b - cc;
      // margin: distance of the in-plane ray from the ply circle's edge,
      // R_p - |perp| with perp^2 = R_p^2 - disc
      mg(MG_GRAZE, L.Rp - std::sqrt(std::max(L.Rp * L.Rp - val(disc), 0.0)));
      if (disc < 0.0) {
        hit = false;
        break;
      }
      S tn = -b - sqrt(disc);
      if (tn < 0.0) tn = S(0.0);
      t = tn;
    }
    if (!hit) continue;
    g.t_ply[k] = val(t);
    g.ni += 1;
    if (best < 0 || t < best_t) {
      best = k;
      best_t = t;
      best_cx = cx;
      best_cy = cy;
      best_psi = psi;
    }
  }
  if (best < 0) return g;  // Sec. 3.4: no ply hit, the ray passes through.
  // margin: the closest ply changes where another hit ply is as near
  for (int k = 0; k < Np; ++k)
    if (k != best && g.t_ply[k] >= 0.0) mg(MG_GAP, g.t_ply[k] - val(best_t));
  g.hit = true;
  g.k = best;
  // Sec. 3.4: hit point, ply normal (away from the ply centre in the circular
  // cross-section) and ply tangent (derivative of the helix through x).
  if (g_off_t != 0.0) best_t = best_t + g_off_t;
  const S xx = X0x + best_t * ex, xy = X0y + best_t * ey;
  const S zx = v + kappa * best_t;
  g.x = mk<S>(xx, xy, zx);
  const S dx = xx - best_cx, dy = xy - best_cy;
  const S dl = sqrt(dx * dx + dy * dy);
  g.residual = std::fabs(val(dl) - L.Rp);
  g.np = mk<S>(dx / dl, dy / dl, S(0.0));
  const V3<S> traw = mk<S>(-m.omega_p * xy, m.omega_p * xx, S(1.0));
  g.tp = normalize(traw - g.np * dot(traw, g.np));
  const V3<S> ep = cross(g.tp, g.np);
  // Sec. 3.5.1: ply azimuth u_ply of the hit about the ply centre, measured
  // from the ply centre's radial direction; fiber phase and 1D maps.
  const S ecx = cos(best_psi), ecy = sin(best_psi);
  g.u_ply = atan2(ecx * g.np.y - ecy * g.np.x, ecx * g.np.x + ecy * g.np.y);
  if (g_off_uply != 0.0) g.u_ply = g.u_ply + g_off_uply;
  const S theta_f = g.u_ply - m.omega_f * zx;
  if (st.d.migration_maps > 1)
    migration_lookup(m, g.u_ply, zx, &g.delta, &g.of);
  else
    fiber_lookup(st, theta_f, &g.delta, &g.of);
  // n_f = n'(R(n_p)), t_f = t'(R(t_p)): R tilts the tangent by the fiber
  // helix angle about n_p; n' tilts the normal by delta about t_f.
  g.tf = g.tp * cos(m.alpha_f) + ep * sin(m.alpha_f);
  g.nf = g.np * cos(g.delta) + cross(g.tf, g.np) * sin(g.delta);
  // Sec. 4.1.4: shadowing terms G = exp(-sigma_s * occlusion).
  const S wl = sqrt(wi.x * wi.x + wi.y * wi.y);
  S op = S(0.0);
  if (val(wl) > 1e-7) op = ply_occlusion(m, best, best_psi, xx, xy, wi.x / wl, wi.y / wl);
  g.gp = exp(-m.sigma_s * op);
  g.gf = exp(-m.sigma_s * g.of);
  return g;
}

// Multi-scale footprint (Sec. 4.2, 5.3).  Reading: ratio is the pixel
// footprint over the yarn width, i.e. the half-width of [h1, h2] in h units;
// the node count grows with the range, K = ceil(K_max (h2 - h1) / 2).  This
// integer decision is taken in float32 arithmetic, as the GPU path takes it.
struct Footprint {
  float h1, h2, width;
  int K;
};
Footprint footprint(double h0d, bool has_ratio, double ratiod, int kmax) {
  Footprint fp;
  const float h0 = (float)h0d;
  const float ratio = has_ratio ? (float)ratiod : 0.0f;
  volatile float a = h0 - ratio;
  volatile float b = h0 + ratio;
  fp.h1 = a < -1.0f ? -1.0f : (float)a;
  fp.h2 = b > 1.0f ? 1.0f : (float)b;
  volatile float w = fp.h2 - fp.h1;
  fp.width = w;
  volatile float kf = ((float)kmax * 0.5f) * fp.width;
  int K = (int)std::ceil((float)kf);
  fp.K = std::max(1, std::min(K, kmax));
  return fp;
}

template <class S>
struct Geo {
  int status = ORC_NO_HIT;
  Footprint fp{};
  int nhit = 0;
  V3<S> n, t, x;   // aggregated fiber normal / tangent (unflipped) and point
  S g = S(1.0);    // aggregated G_p G_f
  S ni = S(0.0);   // mean number of intersected plies
  Node<S> node0;
};

// Sec. 4.2 Eqs. 8-11 with W = 1: K midpoint nodes h_j over [h1, h2]; each
// node is the same ray direction entering at offset h_j; hit nodes are
// averaged (normal, tangent, shadowing, hit point, N_i), nodes without a ply
// hit are dropped.  K = 1 at h0 is the near field (Sec. 4.1).
template <class S>
Geo<S> geometry(const Mat<S>& m, const Rec& q, const V3<S>& wi, const Stoch* sc = nullptr) {
  using std::sqrt;
  const MatStatic& st = *m.st;
  Geo<S> G;
  G.fp = footprint(q.h, q.has_ratio, q.ratio, st.d.k_max);
  // Sec. 3.3 / reading: entry azimuth u, in-plane angle asin(h) from -n_u,
  // longitudinal slope from omega_i . T.
  const double g0 = std::asin(q.h);
  const double ex = -std::cos(q.u - g0), ey = -std::sin(q.u - g0);
  const S Lxy = sqrt(wi.x * wi.x + wi.y * wi.y);
  mg(MG_AXIS, val(Lxy));
  if (val(Lxy) < 1e-7) return G;
  const S kappa = -wi.z / Lxy;
  V3<S> ns = mk<S>(S(0.0), S(0.0), S(0.0)), ts = ns, xs = ns;
  S gs = S(0.0), nis = S(0.0);
  const int K = G.fp.K;
  for (int j = 0; j < K; ++j) {
    // midpoint of stratum j, or a uniform point in it (stratified jitter)
    const double xj = (sc && sc->jitter) ? sc->xi(j) : 0.5;
    const double hj = (double)G.fp.h1 + ((j + xj) * (double)G.fp.width) / K;
    const double uj = (q.u - g0) + std::asin(hj);
    const double X0x = st.L.R * std::cos(uj), X0y = st.L.R * std::sin(uj);
    Node<S> nd = node_geometry(m, X0x, X0y, ex, ey, q.v, kappa, wi);
    if (j == 0) G.node0 = nd;
    if (!nd.hit) continue;
    G.nhit += 1;
    ns = ns + nd.nf;
    ts = ts + nd.tf;
    xs = xs + nd.x;
    gs = gs + nd.gp * nd.gf;
    nis = nis + S((double)nd.ni);
  }
  if (G.nhit == 0) return G;
  const double inv = 1.0 / G.nhit;
  const S nl = norm(ns);
  if (!(nl > 1e-9 * G.nhit)) return G;
  G.n = ns * (S(1.0) / nl);
  const V3<S> tperp = ts - G.n * dot(ts, G.n);
  const S tl = norm(tperp);
  if (!(tl > 1e-9 * G.nhit)) return G;
  G.t = tperp * (S(1.0) / tl);
  G.x = xs * inv;
  G.g = gs * inv;
  G.ni = nis * inv;
  G.status = ORC_OK;
  return G;
}
template <class S>
Geo<S> geometry(const Mat<S>& m, const Rec& q, const Stoch* sc = nullptr) {
  return geometry(m, q, lift<S>(q.wi), sc);
}

// -------------------------------------------------------------- microfacet --
// Unpolarised dielectric Fresnel reflectance; eta = eta_t / eta_i, cos_i >= 0.
template <class S>
S fresnel(const S& cosi, double eta) {
  using std::sqrt;
  const S s2t = (1.0 - cosi * cosi) / (eta * eta);
  if (s2t >= 1.0) return S(1.0);
  const S cost = sqrt(1.0 - s2t);
  const S rs = (cosi - eta * cost) / (cosi + eta * cost);
  const S rp = (eta * cosi - cost) / (eta * cosi + cost);
  return 0.5 * (rs * rs + rp * rp);
}

// Anisotropic GGX normal distribution and Smith G1 (Heitz 2014), local frame.
template <class S>
S ggx_d(const V3<S>& m, const S& at, const S& ab) {
  if (!(m.z > 0.0)) return S(0.0);
  const S q = m.x * m.x / (at * at) + m.y * m.y / (ab * ab) + m.z * m.z;
  return 1.0 / (PI * at * ab * q * q);
}
template <class S>
S ggx_g1(const V3<S>& w, const S& wdotm, const S& at, const S& ab) {
  using std::sqrt;
  if (!(wdotm * w.z > 0.0)) return S(0.0);
  const S an = sabs(w.z);
  const S r = sqrt(an * an + at * at * w.x * w.x + ab * ab * w.y * w.y);
  return 2.0 * an / (an + r);
}
// Visible-normal sampling of GGX (Heitz 2018, "Sampling the GGX Distribution
// of Visible Normals"), local frame, w.z > 0.
template <class S>
V3<S> vndf_sample(const V3<S>& w, const S& at, const S& ab, double u0, double u1) {
  using std::cos;
  using std::sin;
  using std::sqrt;
  const V3<S> V = normalize(mk<S>(at * w.x, ab * w.y, w.z));
  const S lensq = V.x * V.x + V.y * V.y;
  V3<S> T1 = mk<S>(S(1.0), S(0.0), S(0.0));
  mg(MG_SAMPLE, std::sqrt(val(lensq)));  // margin: the disk frame turns with V
  if (lensq > 0.0) {
    const S il = 1.0 / sqrt(lensq);
    T1 = mk<S>(-V.y * il, V.x * il, S(0.0));
  }
  const V3<S> T2 = cross(V, T1);
  const double r = std::sqrt(u0), phi = 2.0 * PI * u1;
  const S t1 = S(r * std::cos(phi));
  S t2 = S(r * std::sin(phi));
  const S s = 0.5 * (1.0 + V.z);
  t2 = (1.0 - s) * sqrt(1.0 - t1 * t1) + s * t2;
  const S tz = sqrt(smax(S(0.0), 1.0 - t1 * t1 - t2 * t2));
  const V3<S> Nh = T1 * t1 + T2 * t2 + V * tz;
  return normalize(mk<S>(at * Nh.x, ab * Nh.y, smax(S(0.0), Nh.z)));
}

// ------------------------------------------------------------------ shading --
template <class S>
V3<S> to_local(const V3<S>& w, const V3<S>& t, const V3<S>& b, const V3<S>& n) {
  return mk<S>(dot(w, t), dot(w, b), dot(w, n));
}

template <class S>
struct Shade {
  V3<S> t, b, n, wi;
  S mui, at, ab, ks, g, alb[3], alb_y[3];
  double eta;
  S B = S(0.0), r = S(0.0);
  // transmission path through the yarn (TT lobe)
  bool tt_ok = false;
  V3<S> iy, ty, by, ny;
  S tx = S(0.0), tau = S(0.0), path = S(0.0);
  S fr = S(0.0);  // F(mu_i), lobe selection
};

template <class S>
S clamp_alpha(const S& a) {
  if (a < 1e-3) return S(1e-3);
  if (a > 1.5) return S(1.5);
  return a;
}

template <class S>
Shade<S> make_shade(const Mat<S>& m, const Geo<S>& G, const V3<S>& wi,
                    const Stoch* sc = nullptr) {
  using std::exp;
  using std::sqrt;
  const orc_material& d = m.st->d;
  Shade<S> s;
  s.wi = wi;
  s.n = G.n;
  s.t = G.t;
  s.b = cross(s.n, s.t);
  // Reading: two-sided shading, the side of omega_i is "outside" at x.
  if (dot(s.wi, s.n) < 0.0) {
    s.n = -s.n;
    s.b = -s.b;
  }
  s.mui = dot(s.wi, s.n);
  mg(MG_HEMI, val(s.mui));  // margin: the side of omega_i decides the flip
  // Sec. 4.2: beta_multi = beta + (h2 - h1) / 2 (reading of the normaliser);
  // GGX alpha = beta in radians, clamped to [1e-3, 1.5].
  const double half_w = 0.5 * (double)G.fp.width;
  s.at = clamp_alpha(m.beta_t + half_w);
  s.ab = clamp_alpha(m.beta_b + half_w);
  s.eta = d.eta;
  s.B = m.body_B;
  s.r = m.body_r;
  s.ks = (1.0 - m.body_B) * m.k_spec;
  s.g = G.g;
  for (int c = 0; c < 3; ++c) {
    s.alb[c] = m.alb[c];
    s.alb_y[c] = m.alb_y[c];
  }
  s.fr = fresnel(s.mui, d.eta);
  // Sec. 4.1.1, reading: the camera ray refracts smoothly into the yarn at x
  // (transmittance 1 - F), travels straight to the yarn surface y, and is
  // attenuated by tau^{N_i} (Eq. 4).
  // Rough entry (Eq. 1, the Omega_y integral, reading): the refracting
  // normal is a GGX visible normal m about n instead of n itself; the entry
  // transmittance is 1 - F(omega_i . m); a ray refracted outward carries no
  // transmission.
  V3<S> mn = s.n;
  S ci = s.mui;
  if (sc && sc->rough && s.mui > 0.0) {
    double v0, v1;
    sc->entry(&v0, &v1);
    const V3<S> ml = vndf_sample(to_local(s.wi, s.t, s.b, s.n), s.at, s.ab, v0, v1);
    mn = s.t * ml.x + s.b * ml.y + s.n * ml.z;
    ci = dot(s.wi, mn);
    mg(MG_EXIT, val(ci));
  }
  const S s2t = (1.0 - ci * ci) / (d.eta * d.eta);
  mg(MG_EXIT, std::sqrt(std::fabs(1.0 - val(s2t))));  // refraction edge, as a cosine
  if (!(s.mui > 0.0) || !(ci > 0.0) || s2t >= 1.0) return s;
  const S cost = sqrt(1.0 - s2t);
  const V3<S> din = s.wi * (-1.0 / d.eta) + mn * (ci / d.eta - cost);
  mg(MG_EXIT, dotv(din, s.n));
  if (!(dot(din, s.n) < 0.0)) return s;
  const S a = din.x * din.x + din.y * din.y;
  mg(MG_EXIT, std::sqrt(val(a)));
  if (!(a > 1e-12)) return s;
  const S bq = G.x.x * din.x + G.x.y * din.y;
  const S c = G.x.x * G.x.x + G.x.y * G.x.y - d.yarn_radius * d.yarn_radius;
  S disc = bq * bq - a * c;
  if (disc < 0.0) disc = S(0.0);
  S sy = (-bq + sqrt(disc)) / a;
  if (sy < 0.0) sy = S(0.0);
  const V3<S> y = G.x + din * sy;
  s.ny = normalize(mk<S>(y.x, y.y, S(0.0)));
  s.ty = mk<S>(S(0.0), S(0.0), S(1.0));
  s.by = cross(s.ny, s.ty);
  s.iy = -din;
  s.path = sy;
  s.tau = exp(-(m.sigma_t * G.ni * sy));
  s.tx = 1.0 - ((sc && sc->rough) ? fresnel(ci, d.eta) : s.fr);
  s.tt_ok = true;
  return s;
}
template <class S>
Shade<S> make_shade(const Mat<S>& m, const Geo<S>& G, const double* wi) {
  return make_shade(m, G, lift<S>(wi));
}

// The four lobes at omega_o, cosine-weighted (f |omega_o . n|), and the
// densities of the four sampling strategies.
template <class S>
struct Lobes {
  S fR = S(0.0), fT = S(0.0), fxb[3], fyb[3];
  S pR = S(0.0), pT = S(0.0), pxb = S(0.0), pyb = S(0.0);
};

template <class S>
Lobes<S> eval_lobes(const Shade<S>& s, const V3<S>& wo) {
  using std::log;
  using std::sqrt;
  Lobes<S> L;
  for (int c = 0; c < 3; ++c) L.fxb[c] = L.fyb[c] = S(0.0);
  const S muo = dot(wo, s.n);
  if (!(s.mui > 0.0)) return L;
  mg(MG_HEMI, val(muo));  // margin: the side of omega_o picks the lobes
  if (muo > 0.0) {
    // Eq. 2, first case (reflection, Walter et al. 2007 with GGX).
    const V3<S> h = normalize(s.wi + wo);
    const S wih = dot(s.wi, h), woh = dot(wo, h);
    const V3<S> hl = to_local(h, s.t, s.b, s.n);
    const V3<S> il = to_local(s.wi, s.t, s.b, s.n);
    const V3<S> ol = to_local(wo, s.t, s.b, s.n);
    const S D = ggx_d(hl, s.at, s.ab);
    const S g1i = ggx_g1(il, wih, s.at, s.ab);
    const S g1o = ggx_g1(ol, woh, s.at, s.ab);
    const S F = fresnel(wih, s.eta);
    L.fR = s.ks * F * g1i * g1o * D / (4.0 * s.mui);
    L.pR = g1i * D / (4.0 * s.mui);
    // Eq. 5 with the Lommel-Seeliger term LS = 1/(4 pi (mu_i + mu_o)); the
    // bracket is divided by its hemispherical albedo 1 + a(mu_i) so that the
    // lobe's albedo is r B G k^B (Sec. 4.3, each component normalised).
    const S aLS = 0.5 * (1.0 - s.mui * log(1.0 + 1.0 / s.mui));
    const S br = (1.0 / (4.0 * PI * (s.mui + muo)) + 1.0 / PI) / (1.0 + aLS);
    for (int c = 0; c < 3; ++c) L.fxb[c] = s.r * s.B * s.g * s.alb[c] * br * muo;
    L.pxb = muo / PI;
  } else if (muo < 0.0) {
    // Eq. 6: forward body, Lambertian on the far side.
    for (int c = 0; c < 3; ++c) L.fyb[c] = (1.0 - s.r) * s.B * s.g * s.alb_y[c] / PI * (-muo);
    L.pyb = -muo / PI;
    // Eq. 3 (third case times the second, Walter's transmission term), at the
    // exit point y from inside (eta) to outside (1), times tau^{N_i}.
    if (s.tt_ok) {
      const S ion = dot(s.iy, s.ny), oon = dot(wo, s.ny);
      mg(MG_EXIT, val(ion));
      mg(MG_EXIT, val(oon));
      if (ion < 0.0 && oon > 0.0) {
        V3<S> ht = normalize(-(s.iy * s.eta + wo));
        mg(MG_EXIT, dotv(ht, s.ny));
        if (dot(ht, s.ny) < 0.0) ht = -ht;
        const S ih = dot(s.iy, ht), oh = dot(wo, ht);
        mg(MG_EXIT, val(ih));
        mg(MG_EXIT, val(oh));
        // margin: total internal reflection at y (F_y = 1 beyond it), as the
        // refraction edge, as a cosine
        mg(MG_EXIT, std::sqrt(std::fabs(1.0 - (1.0 - val(ih) * val(ih)) * s.eta * s.eta)));
        if (ih < 0.0 && oh > 0.0) {
          const S den = s.eta * ih + oh;
          const V3<S> hl = to_local(ht, s.ty, s.by, s.ny);
          const V3<S> il = to_local(s.iy, s.ty, s.by, s.ny);
          const V3<S> ol = to_local(wo, s.ty, s.by, s.ny);
          const S D = ggx_d(hl, s.at, s.ab);
          const S g1i = ggx_g1(il, ih, s.at, s.ab);
          const S g1o = ggx_g1(ol, oh, s.at, s.ab);
          const S Fy = fresnel(-ih, 1.0 / s.eta);
          L.fT = s.ks * s.tx * s.tau * (-ih) * oh * (1.0 - Fy) * g1i * g1o * D /
                 ((-ion) * den * den);
          L.pT = g1i * (-ih) * D / (-ion) * oh / (den * den);
        }
      }
    }
  }
  return L;
}

// Sec. 4.1.5: lobe selection probabilities (specular 1 - B split by F(mu_i)
// into reflection / transmission; body B split by r).
template <class S>
void lobe_probs(const Shade<S>& s, double* P) {
  const double fr = val(s.fr), B = val(s.B), r = val(s.r);
  P[0] = (1.0 - B) * fr;
  P[1] = (1.0 - B) * (1.0 - fr);
  P[2] = B * r;
  P[3] = B * (1.0 - r);
}

template <class S>
void total(const Shade<S>& s, const Lobes<S>& L, S* f, S* pdf) {
  for (int c = 0; c < 3; ++c) f[c] = L.fR + L.fT + L.fxb[c] + L.fyb[c];
  const S fr = s.fr;
  const S PR = (1.0 - s.B) * fr, PT = (1.0 - s.B) * (1.0 - fr);
  *pdf = PR * L.pR + PT * L.pT + (s.B * s.r) * L.pxb + (s.B * (1.0 - s.r)) * L.pyb;
}

// -------------------------------------------------------------- entry points --
template <class S>
struct Out {
  int status = ORC_INVALID;
  S f[3];
  S pdf = S(0.0);
  double wo[3] = {0, 0, 0};
  S weight[3];
  int lobe = 0;
  Out() { for (int c = 0; c < 3; ++c) f[c] = weight[c] = S(0.0); }
};

// wi, wo: the record's directions as scalars of type S (seeded for
// derivatives with respect to them)
template <class S>
Out<S> eval_one(const Mat<S>& m, const Rec& q, const V3<S>& wi, const V3<S>& wo,
                const Stoch* sc = nullptr) {
  Out<S> o;
  const Geo<S> G = geometry(m, q, wi, sc);
  if (G.status != ORC_OK) {
    o.status = ORC_NO_HIT;
    return o;
  }
  const Shade<S> s = make_shade(m, G, wi, sc);
  const Lobes<S> L = eval_lobes(s, wo);
  total(s, L, o.f, &o.pdf);
  o.status = ORC_OK;
  return o;
}
template <class S>
Out<S> eval_one(const Mat<S>& m, const Rec& q, const Stoch* sc = nullptr) {
  return eval_one(m, q, lift<S>(q.wi), lift<S>(q.wo), sc);
}

template <class S>
Out<S> sample_one(const Mat<S>& m, const Rec& q, const Stoch* sc = nullptr) {
  using std::sqrt;
  Out<S> o;
  const Geo<S> G = geometry(m, q, sc);
  if (G.status != ORC_OK) {
    // Reading: no ply hit is a pass-through, a delta in direction -omega_i.
    o.status = ORC_NO_HIT;
    for (int c = 0; c < 3; ++c) {
      o.wo[c] = -q.wi[c];
      o.weight[c] = S(1.0);
    }
    return o;
  }
  const Shade<S> s = make_shade(m, G, lift<S>(q.wi), sc);
  double P[4];
  lobe_probs(s, P);
  // Sec. 4.1.5: one random number picks the lobe and is rescaled for reuse.
  double u0 = q.u0;
  {
    double cum = 0.0;  // margin: u0 at a boundary of the lobe choice
    for (int k = 0; k < 3; ++k) mg(MG_LOBE, u0 - (cum += P[k]));
  }
  int lobe = 3;
  double lo = 0.0;
  for (int k = 0; k < 3; ++k) {
    if (u0 < lo + P[k]) {
      lobe = k;
      break;
    }
    lo += P[k];
  }
  double ur = P[lobe] > 0.0 ? (u0 - lo) / P[lobe] : 0.0;
  ur = std::min(std::max(ur, 0.0), 1.0 - 1e-12);
  o.lobe = lobe;
  V3<S> wo;
  bool ok = true;
  if (lobe == 0) {
    // GGX visible-normal sample about n, mirror reflection.
    const V3<S> il = to_local(s.wi, s.t, s.b, s.n);
    const V3<S> ml = vndf_sample(il, s.at, s.ab, ur, q.u1);
    const V3<S> mw = s.t * ml.x + s.b * ml.y + s.n * ml.z;
    wo = mw * (2.0 * dot(s.wi, mw)) - s.wi;
    mg(MG_SAMPLE, dotv(wo, s.n));
    ok = dot(wo, s.n) > 0.0;
  } else if (lobe == 1) {
    // GGX visible-normal sample at y about the inner normal, refraction out.
    ok = s.tt_ok;
    if (ok) {
      const V3<S> Nn = -s.ny, Tn = s.ty, Bn = cross(Nn, Tn);
      const V3<S> il = to_local(s.iy, Tn, Bn, Nn);
      const V3<S> ml = vndf_sample(il, s.at, s.ab, ur, q.u1);
      const V3<S> mw = Tn * ml.x + Bn * ml.y + Nn * ml.z;
      const S c = dot(s.iy, mw);
      const S s2t = s.eta * s.eta * (1.0 - c * c);
      mg(MG_SAMPLE, val(c));
      mg(MG_SAMPLE, std::sqrt(std::fabs(1.0 - val(s2t))));
      if (!(c > 0.0) || s2t >= 1.0) {
        ok = false;
      } else {
        wo = normalize(s.iy * (-s.eta) + mw * (s.eta * c - sqrt(1.0 - s2t)));
        mg(MG_SAMPLE, dotv(wo, s.ny));
        mg(MG_SAMPLE, dotv(wo, s.n));
        ok = dot(wo, s.ny) > 0.0 && dot(wo, s.n) < 0.0;
      }
    }
  } else {
    // Cosine-weighted hemisphere about +n (lobe 2) or -n (lobe 3).
    const double r = std::sqrt(ur), phi = 2.0 * PI * q.u1;
    const double zc = std::sqrt(std::max(0.0, 1.0 - ur)) * (lobe == 2 ? 1.0 : -1.0);
    wo = s.t * (r * std::cos(phi)) + s.b * (r * std::sin(phi)) + s.n * zc;
  }
  if (ok) {
    for (int c = 0; c < 3; ++c) o.wo[c] = val(c == 0 ? wo.x : c == 1 ? wo.y : wo.z);
    const Lobes<S> L = eval_lobes(s, wo);
    S f[3];
    total(s, L, f, &o.pdf);
    if (o.pdf > 0.0) {
      for (int c = 0; c < 3; ++c) o.weight[c] = f[c] / o.pdf;
      o.status = ORC_OK;
      return o;
    }
  }
  o.pdf = S(0.0);
  o.status = ORC_BAD_SAMPLE;
  return o;
}

// ---------------------------------------------------------------- batching --
struct Batch {
  std::vector<MatStatic> st;
  bool ok = true;
};
Batch make_batch(const orc_material* m, int n_mat) {
  Batch b;
  b.st.resize(n_mat);
  for (int i = 0; i < n_mat; ++i)
    if (!build_static(m[i], b.st[i])) b.ok = false;
  return b;
}

template <class F>
void parallel_for(int64_t n, int n_threads, F&& body) {
  if (n_threads <= 1 || n < 1024) {
    body(0, n, 0);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + n_threads - 1) / n_threads;
  for (int t = 0; t < n_threads; ++t) {
    const int64_t b = t * chunk, e = std::min(n, b + chunk);
    if (b >= e) break;
    th.emplace_back([&, b, e, t] { body(b, e, t); });
  }
  for (auto& x : th) x.join();
}

}  // namespace

// ================================================================ C entry ===
extern "C" {

int orc_eval(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
             double* f_rgb, double* pdf, uint8_t* status, int n_threads) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      Out<double> o;
      if (valid_rec(q, n_mat, true, false)) o = eval_one(mats[q.mat], q);
      for (int c = 0; c < 3; ++c) f_rgb[c * n + i] = o.f[c];
      if (pdf) pdf[i] = o.pdf;
      status[i] = (uint8_t)o.status;
    }
  });
  return 0;
}

int orc_pdf(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
            double* pdf, uint8_t* status, int n_threads) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      Out<double> o;
      if (valid_rec(q, n_mat, true, false)) o = eval_one(mats[q.mat], q);
      pdf[i] = o.pdf;
      status[i] = (uint8_t)o.status;
    }
  });
  return 0;
}

int orc_sample(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
               double* wo, double* weight, double* pdf, uint8_t* lobe_status,
               int n_threads) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      Out<double> o;
      if (valid_rec(q, n_mat, false, true)) o = sample_one(mats[q.mat], q);
      for (int c = 0; c < 3; ++c) {
        wo[c * n + i] = o.wo[c];
        weight[c * n + i] = o.weight[c];
      }
      pdf[i] = o.pdf;
      lobe_status[i] = (uint8_t)(o.status | (o.lobe << 4));
    }
  });
  return 0;
}

int orc_grad(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
             const double* g_rgb, double* grad, double* jac, double* f_rgb,
             int n_threads) {
  typedef Dual<ORC_NPARAM> D8;
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  const int nt = std::max(1, n_threads);
  std::vector<double> partial((size_t)nt * n_mat * ORC_NPARAM, 0.0);
  parallel_for(n, nt, [&](int64_t b, int64_t e, int tid) {
    std::vector<Mat<D8>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<D8>(st, true));
    double* acc = partial.data() + (size_t)tid * n_mat * ORC_NPARAM;
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      Out<D8> o;
      if (valid_rec(q, n_mat, true, false)) o = eval_one(mats[q.mat], q);
      for (int c = 0; c < 3; ++c) {
        if (f_rgb) f_rgb[c * n + i] = o.f[c].v;
        for (int k = 0; k < ORC_NPARAM; ++k) {
          if (jac) jac[(i * 3 + c) * ORC_NPARAM + k] = o.f[c].d[k];
          if (o.status == ORC_OK)
            acc[q.mat * ORC_NPARAM + k] += g_rgb[c * n + i] * o.f[c].d[k];
        }
      }
    }
  });
  for (int k = 0; k < n_mat * ORC_NPARAM; ++k) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += partial[(size_t)t * n_mat * ORC_NPARAM + k];
    grad[k] = s;
  }
  return 0;
}

int orc_grad_ext(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                 const double* g_rgb, double* grad, double* g_wi, double* g_wo,
                 double* jac, double* f_rgb, int n_threads) {
  constexpr int NP = ORC_NPARAM_EXT, NT = NP + 6;  // 15 parameters, wi, wo
  typedef Dual<NT> D;
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  const int nt = std::max(1, n_threads);
  std::vector<double> partial((size_t)nt * n_mat * NP, 0.0);
  parallel_for(n, nt, [&](int64_t b, int64_t e, int tid) {
    std::vector<Mat<D>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<D>(st, true, true));
    double* acc = partial.data() + (size_t)tid * n_mat * NP;
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      V3<D> wi = lift<D>(q.wi), wo = lift<D>(q.wo);
      seed(wi.x, NP + 0);
      seed(wi.y, NP + 1);
      seed(wi.z, NP + 2);
      seed(wo.x, NP + 3);
      seed(wo.y, NP + 4);
      seed(wo.z, NP + 5);
      Out<D> o;
      if (valid_rec(q, n_mat, true, false)) o = eval_one(mats[q.mat], q, wi, wo);
      double vw[6] = {0, 0, 0, 0, 0, 0};
      for (int c = 0; c < 3; ++c) {
        const double g = g_rgb[c * n + i];
        if (f_rgb) f_rgb[c * n + i] = o.f[c].v;
        for (int k = 0; k < NT; ++k) {
          if (jac) jac[(i * 3 + c) * NT + k] = o.f[c].d[k];
          if (o.status != ORC_OK) continue;
          if (k < NP) acc[q.mat * NP + k] += g * o.f[c].d[k];
          else vw[k - NP] += g * o.f[c].d[k];
        }
      }
      for (int c = 0; c < 3; ++c) {
        if (g_wi) g_wi[c * n + i] = vw[c];
        if (g_wo) g_wo[c * n + i] = vw[3 + c];
      }
    }
  });
  for (int k = 0; k < n_mat * NP; ++k) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += partial[(size_t)t * n_mat * NP + k];
    grad[k] = s;
  }
  return 0;
}

int orc_eval_stochastic(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                        uint64_t seed, int64_t index_offset, uint32_t flags, double* f_rgb,
                        double* pdf, uint8_t* status, int n_threads) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    Stoch sc;
    sc.jitter = (flags & ORC_STOCH_JITTER_NODES) != 0;
    sc.rough = (flags & ORC_STOCH_ROUGH_ENTRY) != 0;
    sc.seed = seed;
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      sc.index = (uint64_t)(index_offset + i);
      Out<double> o;
      if (valid_rec(q, n_mat, true, false)) o = eval_one(mats[q.mat], q, &sc);
      for (int c = 0; c < 3; ++c) f_rgb[c * n + i] = o.f[c];
      if (pdf) pdf[i] = o.pdf;
      status[i] = (uint8_t)o.status;
    }
  });
  return 0;
}

int orc_sample_stochastic(const orc_material* m, int n_mat, const orc_records* r, int64_t n,
                          uint64_t seed, int64_t index_offset, uint32_t flags, double* wo,
                          double* weight, double* pdf, uint8_t* lobe_status, int n_threads) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    Stoch sc;
    sc.jitter = (flags & ORC_STOCH_JITTER_NODES) != 0;
    sc.rough = (flags & ORC_STOCH_ROUGH_ENTRY) != 0;
    sc.seed = seed;
    for (int64_t i = b; i < e; ++i) {
      const Rec q = read_rec(r, i, n);
      sc.index = (uint64_t)(index_offset + i);
      Out<double> o;
      if (valid_rec(q, n_mat, false, true)) o = sample_one(mats[q.mat], q, &sc);
      for (int c = 0; c < 3; ++c) {
        wo[c * n + i] = o.wo[c];
        weight[c * n + i] = o.weight[c];
      }
      pdf[i] = o.pdf;
      lobe_status[i] = (uint8_t)(o.status | (o.lobe << 4));
    }
  });
  return 0;
}

int orc_margins(const orc_material* m, int n_mat, const orc_records* r, int64_t n, int op,
                uint64_t seed, int64_t index_offset, uint32_t flags, double* out,
                int n_threads) {
  static_assert(MG_N == ORC_MG_N, "margin classes");
  Batch B = make_batch(m, n_mat);
  if (!B.ok || op < 0 || op > 1) return -1;
  parallel_for(n, n_threads, [&](int64_t b, int64_t e, int) {
    std::vector<Mat<double>> mats;
    for (auto& st : B.st) mats.push_back(make_mat<double>(st, false));
    Stoch sc;
    sc.jitter = (flags & ORC_STOCH_JITTER_NODES) != 0;
    sc.rough = (flags & ORC_STOCH_ROUGH_ENTRY) != 0;
    sc.seed = seed;
    for (int64_t i = b; i < e; ++i) {
      double* row = out + i * MG_N;
      for (int k = 0; k < MG_N; ++k) row[k] = HUGE_VAL;
      const Rec q = read_rec(r, i, n);
      sc.index = (uint64_t)(index_offset + i);
      const Stoch* scp = flags ? &sc : nullptr;
      if (!valid_rec(q, n_mat, op == 0, op == 1)) continue;
      g_mg = row;
      if (op == 0)
        eval_one(mats[q.mat], q, scp);
      else
        sample_one(mats[q.mat], q, scp);
      g_mg = nullptr;
    }
  });
  return 0;
}

void orc_set_internal_offsets(double dt, double du_ply) {
  g_off_t = dt;
  g_off_uply = du_ply;
}

int orc_stoch_nodes(double h0, int has_ratio, double ratio, int k_max, uint64_t seed,
                    uint64_t index, double* h_out) {
  const Footprint fp = footprint(h0, has_ratio != 0, ratio, k_max);
  Stoch sc;
  sc.jitter = true;
  sc.seed = seed;
  sc.index = index;
  for (int j = 0; j < fp.K; ++j)
    h_out[j] = (double)fp.h1 + ((j + sc.xi(j)) * (double)fp.width) / fp.K;
  return fp.K;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const Philox4x64 r = philox4x64(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1]);
  for (int k = 0; k < 4; ++k) out[k] = r.w[k];
}

int orc_count_ops(const orc_material* m, int n_mat, const orc_records* r,
                  int64_t n, int op, double* counts) {
  Batch B = make_batch(m, n_mat);
  if (!B.ok) return -1;
  std::vector<Mat<Cnt>> mats;
  for (auto& st : B.st) mats.push_back(make_mat<Cnt>(st, false));
  for (int64_t i = 0; i < n; ++i) {
    const Rec q = read_rec(r, i, n);
    for (int k = 0; k < 6; ++k) g_ops[k] = 0.0;
    if (valid_rec(q, n_mat, op != 1 && op != 3, op == 1)) {
      if (op == 1) {
        sample_one(mats[q.mat], q);
      } else if (op == 3) {
        // the part eval and sample share: geometry and shading state
        const Geo<Cnt> G = geometry(mats[q.mat], q);
        if (G.status == ORC_OK) make_shade(mats[q.mat], G, q.wi);
      } else {
        eval_one(mats[q.mat], q);
      }
    }
    for (int k = 0; k < 6; ++k) counts[i * 6 + k] = g_ops[k];
  }
  return 0;
}

int orc_geometry(const orc_material* m, float h, float u, float v,
                 const float wi[3], float ratio, orc_geo* out) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  const Mat<double> mat = make_mat<double>(st, false);
  Rec q{};
  q.h = h;
  q.u = u;
  q.v = v;
  for (int c = 0; c < 3; ++c) q.wi[c] = wi[c];
  q.has_ratio = ratio >= 0.0f;
  q.ratio = q.has_ratio ? ratio : 0.0;
  *out = orc_geo{};
  if (!valid_rec(q, 1, false, false)) {
    out->status = ORC_INVALID;
    return 0;
  }
  const Geo<double> G = geometry(mat, q);
  out->status = G.status;
  out->n_nodes = G.fp.K;
  out->n_hit_nodes = G.nhit;
  out->h1 = G.fp.h1;
  out->h2 = G.fp.h2;
  const Node<double>& nd = G.node0;
  out->ply = nd.k;
  for (int k = 0; k < 8; ++k) out->t_ply[k] = nd.t_ply[k];
  out->n_p[0] = nd.np.x; out->n_p[1] = nd.np.y; out->n_p[2] = nd.np.z;
  out->t_p[0] = nd.tp.x; out->t_p[1] = nd.tp.y; out->t_p[2] = nd.tp.z;
  out->g_p = nd.gp;
  out->g_f = nd.gf;
  out->u_ply = nd.u_ply;
  out->delta = nd.delta;
  out->o_f = nd.of;
  out->residual = nd.residual;
  if (G.status == ORC_OK) {
    out->ni_mean = G.ni;
    out->x[0] = G.x.x; out->x[1] = G.x.y; out->x[2] = G.x.z;
    out->n_f[0] = G.n.x; out->n_f[1] = G.n.y; out->n_f[2] = G.n.z;
    out->t_f[0] = G.t.x; out->t_f[1] = G.t.y; out->t_f[2] = G.t.z;
    out->g_mean = G.g;
  }
  return 0;
}

int orc_layout(const orc_material* m, double* out) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  const Mat<double> mat = make_mat<double>(st, false);
  out[0] = st.L.Rp;
  out[1] = st.L.Rc;
  out[2] = st.L.rf;
  out[3] = st.L.Rfc;
  out[4] = st.L.M;
  out[5] = mat.omega_p;
  out[6] = mat.omega_f;
  return 0;
}

int orc_migration_info(const orc_material* m, int k, int64_t seg, double* out) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  if (k < 0 || k >= (int)st.Lm.size()) return -1;
  out[0] = st.Lm[k].Rfc;
  out[1] = st.Lm[k].M;
  out[2] = st.d.migration_maps > 1 ? migration_map(st, seg) : 0;
  return 0;
}

int orc_migration_texels(const orc_material* m, int k, double* delta, double* of) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  if (k < 0 || k >= (int)st.Lm.size()) return -1;
  for (int t = 0; t < st.d.map_texels; ++t) {
    delta[t] = st.mig_delta[k][t];
    of[t] = st.mig_of[k][t];
  }
  return 0;
}

int orc_fiber_map(const orc_material* m, double D, double* out) {
  const Layout L = make_layout(*m);
  if (!L.ok) return -1;
  out[0] = fiber_delta(L, D);
  out[1] = fiber_occlusion(L, D);
  return 0;
}

int orc_fiber_map_tab(const orc_material* m, double theta, double* out) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  double d, o;
  fiber_lookup(st, theta, &d, &o);
  out[0] = d;
  out[1] = o;
  return 0;
}

double orc_ply_occlusion(const orc_material* m, int k, double z,
                         const double x[2], const double w[2]) {
  MatStatic st;
  if (!build_static(*m, st)) return -1.0;
  const Mat<double> mat = make_mat<double>(st, false);
  const double psi = 2.0 * PI * k / m->n_plies + mat.omega_p * z;
  const double wl = std::sqrt(w[0] * w[0] + w[1] * w[1]);
  return ply_occlusion(mat, k, psi, x[0], x[1], w[0] / wl, w[1] / wl);
}

double orc_fresnel(double cos_i, double eta) { return fresnel(cos_i, eta); }

double orc_ggx_d(const double m[3], double at, double ab) {
  return ggx_d(V3<double>{m[0], m[1], m[2]}, at, ab);
}
double orc_ggx_g1(const double w[3], const double m[3], double at, double ab) {
  const V3<double> wv{w[0], w[1], w[2]}, mv{m[0], m[1], m[2]};
  return ggx_g1(wv, dot(wv, mv), at, ab);
}
void orc_vndf_sample(const double w[3], double at, double ab, double u0,
                     double u1, double m_out[3]) {
  const V3<double> m = vndf_sample(V3<double>{w[0], w[1], w[2]}, at, ab, u0, u1);
  m_out[0] = m.x;
  m_out[1] = m.y;
  m_out[2] = m.z;
}
double orc_vndf_pdf(const double w[3], const double m[3], double at, double ab) {
  const V3<double> wv{w[0], w[1], w[2]}, mv{m[0], m[1], m[2]};
  const double wm = dot(wv, mv);
  if (!(wm > 0.0) || !(wv.z > 0.0)) return 0.0;
  return ggx_g1(wv, wm, at, ab) * wm * ggx_d(mv, at, ab) / wv.z;
}

int orc_lobes(const orc_material* m, const double frame[9], const double x[3],
              double g, double ni, double width, const double wi[3],
              const double wo[3], double out[8]) {
  MatStatic st;
  if (!build_static(*m, st)) return -1;
  const Mat<double> mat = make_mat<double>(st, false);
  Geo<double> G;
  G.status = ORC_OK;
  G.fp.width = (float)width;
  G.t = V3<double>{frame[0], frame[1], frame[2]};
  G.n = V3<double>{frame[6], frame[7], frame[8]};
  G.x = V3<double>{x[0], x[1], x[2]};
  G.g = g;
  G.ni = ni;
  const Shade<double> s = make_shade(mat, G, wi);
  const Lobes<double> L = eval_lobes(s, V3<double>{wo[0], wo[1], wo[2]});
  out[0] = L.fR;
  out[1] = L.fT;
  for (int c = 0; c < 3; ++c) {
    out[2 + c] = L.fxb[c];
    out[5 + c] = L.fyb[c];
  }
  return 0;
}

double orc_btdf(const double i[3], const double o[3], double eta_i,
                double eta_o, double at, double ab) {
  // Walter et al. 2007 Eq. 21 with GGX: i in medium eta_i, o in eta_o.
  const V3<double> iv{i[0], i[1], i[2]}, ov{o[0], o[1], o[2]};
  if (!(iv.z * ov.z < 0.0)) return 0.0;
  V3<double> h = normalize(-(iv * eta_i + ov * eta_o));
  if (h.z < 0.0) h = -h;
  const double ih = dot(iv, h), oh = dot(ov, h);
  if (!(ih * oh < 0.0)) return 0.0;
  const double den = eta_i * ih + eta_o * oh;
  const double F = fresnel(std::fabs(ih), eta_o / eta_i);
  const double D = ggx_d(h, at, ab);
  const double g1 = ggx_g1(iv, ih, at, ab) * ggx_g1(ov, oh, at, ab);
  return std::fabs(ih) * std::fabs(oh) / (std::fabs(iv.z) * std::fabs(ov.z)) *
         eta_o * eta_o * (1.0 - F) * g1 * D / (den * den);
}

}  // extern "C"
