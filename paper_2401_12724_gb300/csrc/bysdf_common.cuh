// Shared device definitions of libbysdf: the per-material table layout, a
// forward-mode dual number for the backward kernels, and small vector math.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace bysdf {

constexpr float kPi = 3.14159265358979323846f;
constexpr int kMaxPlies = 8;
constexpr int kMaxTexels = 1024;

// Per-material constants, 256 bytes, followed in memory by `T` float2 texels
// (delta, o_f) of the 1D fiber maps (Sec. 3.5.1: fiber normal tilt delta;
// Sec. 4.1.4: fiber self-occlusion o_f), one fiber period at texel centres.
struct alignas(16) MatDev {
  int32_t np, M, T, nit;      // plies, outer-ring fibers, texels, trace updates
  int32_t kmax, flags;
  int32_t mig_maps, mig_seed;  // fiber migration: map pairs K_m (1 = none), seed
  float R, Rp, Rc, Rfc;       // yarn / ply radius, ply-centre radius, fiber ring radius
  float eta, inv_eta, B, r;   // refractive index, body share, body reflect share
  float ks, sigma_t, sigma_s, inv_2Rp;  // (1 - B) k_spec, extinction, shadow density
  float alb[3], m_over_2pi;   // k^B_x, reflection body colour (Eq. 5); M / (2 pi)
  float beta_t, beta_b, alpha_p, alpha_f;  // differentiable angles (radians)
  float kp_hi, kp_lo;         // ply helix rate in turns per length, split hi + lo
  float kf_hi, kf_lo;         // fiber phase rate in map periods per length, split
  float cos_af, sin_af;       // fiber helix angle
  float dkp, dkf;             // d kp / d alpha_p, d kf / d alpha_f
  float inv_np;
  float mig_inv_len, mig_blend, mig_inv_2b;  // 1 / segment length (high part), b, 1 / (2 b)
  float rot_c[kMaxPlies], rot_s[kMaxPlies];  // cos, sin of 2 pi j / N_p
  double Rc_d, Rfc_d;         // layout radii in double (derived-constant updates)
  float alb_y[3];             // k^B_y, transmission body colour (Eq. 6)
  float k_spec;               // specular scale (ks = (1 - B) k_spec)
};
static_assert(sizeof(MatDev) == 256, "MatDev must be 256 bytes");

// Fiber migration map k >= 1 (Sec. 3.5): a 32-byte header, then T texels.
// Map 0 is the regular ring whose constants live in MatDev.
struct alignas(16) MigMap {
  float m_over_2pi;     // M_k / (2 pi)
  float kf_hi, kf_lo;   // fiber phase rate in map periods per length, split
  float dkf;            // d kf / d alpha_f
  double Rfc_d;         // ring radius of the sunk ring
  float M;              // fibers on it
  float aux;            // map 1 only: low part of 1 / segment length
};
static_assert(sizeof(MigMap) == 32, "MigMap must be 32 bytes");

// Bytes of one material: header, map 0, K_m - 1 migration maps, and (when
// migrating) the map index of each of 256 consecutive segments.
constexpr int kMigPeriod = 256;
__host__ __device__ inline size_t mat_bytes(int T, int K) {
  return sizeof(MatDev) + sizeof(float2) * (size_t)T +
         (size_t)(K - 1) * (sizeof(MigMap) + sizeof(float2) * (size_t)T) +
         (K > 1 ? (size_t)kMigPeriod : 0);
}
__host__ __device__ inline const MigMap* mig_map(const MatDev& m, int k) {
  const uint8_t* base = reinterpret_cast<const uint8_t*>(&m) + sizeof(MatDev) +
                        sizeof(float2) * (size_t)m.T;
  return reinterpret_cast<const MigMap*>(base + (size_t)(k - 1) *
                                                    (sizeof(MigMap) + sizeof(float2) * (size_t)m.T));
}
__host__ __device__ inline MigMap* mig_map(MatDev& m, int k) {
  return const_cast<MigMap*>(mig_map(static_cast<const MatDev&>(m), k));
}
// the segment table: map index of segment s is table[s mod 256]
__host__ __device__ inline const uint8_t* mig_table(const MatDev& m) {
  return reinterpret_cast<const uint8_t*>(mig_map(m, m.mig_maps));
}
// key word 1 of the migration map choice
constexpr uint64_t kMigKey1 = 0xB15DF000F1BE0002ull;

// Parameter slots carried by the dual numbers of the backward kernel: the two
// helix angles, which move the whole geometry.  Albedo (linear), shadow
// density (only through G = exp(-sigma_s occlusion)) and roughness (only
// through GGX D and Smith G1) are differentiated in closed form.
enum { D_ALPHA_P = 0, D_ALPHA_F = 1, ND = 2 };

// ------------------------------------------------------------- randomness --
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 64 x 64 -> 128-bit products of the counter words, the key bumped by the
// Weyl constants between rounds.  Drives the stochastic estimators.
struct U64x4 {
  uint64_t w[4];
};
__device__ __forceinline__ U64x4 philox4x64(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                            uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  return U64x4{{c0, c1, c2, c3}};
}
// 24 high bits of a word as a float in [0, 1) (exact)
__device__ __forceinline__ float unit24(uint64_t w) {
  return (float)(uint32_t)(w >> 40) * (1.0f / 16777216.0f);
}
// key word 1 of the stochastic estimators' generator
constexpr uint64_t kStochKey1 = 0xB15DF0005EED0001ull;
enum : uint32_t { STOCH_JITTER_NODES = 1u, STOCH_ROUGH_ENTRY = 2u };
// Per record: node j's jitter is word j % 4 of counter (index, j / 4, 0, 0);
// the entry microfacet takes words 0, 1 of (index, 16, 0, 0); key (seed,
// kStochKey1).
struct StochCtx {
  uint32_t flags;
  uint64_t seed, index;
};

// ------------------------------------------------------------ dual numbers --
template <int N>
struct DualF {
  float v;
  float d[N];
  DualF() = default;
  __device__ __forceinline__ DualF(float x) : v(x) {
#pragma unroll
    for (int k = 0; k < N; ++k) d[k] = 0.f;
  }
};

template <class S> struct is_dual { static constexpr bool value = false; };
template <int N> struct is_dual<DualF<N>> { static constexpr bool value = true; };

__device__ __forceinline__ float vf(float x) { return x; }
template <int N> __device__ __forceinline__ float vf(const DualF<N>& x) { return x.v; }

#define BY_DF template <int N> __device__ __forceinline__ DualF<N>
BY_DF operator+(const DualF<N>& a, const DualF<N>& b) {
  DualF<N> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
BY_DF operator-(const DualF<N>& a, const DualF<N>& b) {
  DualF<N> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
BY_DF operator-(const DualF<N>& a) {
  DualF<N> r;
  r.v = -a.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -a.d[k];
  return r;
}
BY_DF operator*(const DualF<N>& a, const DualF<N>& b) {
  DualF<N> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
BY_DF operator/(const DualF<N>& a, const DualF<N>& b) {
  DualF<N> r;
  const float inv = 1.0f / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
  return r;
}
BY_DF operator+(const DualF<N>& a, float b) {
  DualF<N> r = a;
  r.v += b;
  return r;
}
BY_DF operator+(float a, const DualF<N>& b) { return b + a; }
BY_DF operator-(const DualF<N>& a, float b) {
  DualF<N> r = a;
  r.v -= b;
  return r;
}
BY_DF operator-(float a, const DualF<N>& b) {
  DualF<N> r;
  r.v = a - b.v;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = -b.d[k];
  return r;
}
BY_DF operator*(const DualF<N>& a, float b) {
  DualF<N> r;
  r.v = a.v * b;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = a.d[k] * b;
  return r;
}
BY_DF operator*(float a, const DualF<N>& b) { return b * a; }
BY_DF operator/(const DualF<N>& a, float b) { return a * (1.0f / b); }
BY_DF operator/(float a, const DualF<N>& b) {
  DualF<N> r;
  const float inv = 1.0f / b.v;
  r.v = a * inv;
  const float g = -r.v * inv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = g * b.d[k];
  return r;
}
template <int N>
__device__ __forceinline__ DualF<N> dchain(const DualF<N>& a, float fv, float g) {
  DualF<N> r;
  r.v = fv;
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = g * a.d[k];
  return r;
}

// ------------------------------------------------------- math, float + dual --
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
BY_DF xsqrt(const DualF<N>& a) {
  const float s = sqrtf(a.v);
  return dchain(a, s, s > 0.f ? 0.5f / s : 0.f);
}
// 1 / sqrt(x).  Floats: the square root and the division (measured 1%
// faster in the forward kernels than rsqrtf).  Duals: the hardware
// reciprocal square root and the chain rule (the backward 2.7% faster than
// with a square root and a division).
__device__ __forceinline__ float xrsqrt(float x) { return 1.0f / sqrtf(x); }
BY_DF xrsqrt(const DualF<N>& a) {
  const float r = rsqrtf(a.v);
  return dchain(a, r, -0.5f * r * r * r);
}
// hardware exp2 / log2 based (relative error ~1e-7 for the arguments here,
// |x| < ~20), for floats and for the values of duals alike
__device__ __forceinline__ float xexp(float x) { return __expf(x); }
BY_DF xexp(const DualF<N>& a) {
  const float e = __expf(a.v);
  return dchain(a, e, e);
}
__device__ __forceinline__ float xlog(float x) { return __logf(x); }
BY_DF xlog(const DualF<N>& a) { return dchain(a, __logf(a.v), 1.0f / a.v); }
// atan2 for the float path: the octant's ratio a = min(|x|, |y|) / max(|x|,
// |y|) in [0, 1], atan(a) = a P(a^2) with P of degree 8 (coefficients fitted
// here by weighted least squares on Chebyshev nodes of [0, 1]; maximum
// error 5e-8 rad before rounding), then the octant's reflections.  Absolute
// error a few 1e-7 rad, as the library's atan2f, at a quarter of its cost,
// for arguments below 2^126 in magnitude (the approximate division of the
// ratio returns 0 beyond; the kernels pass components of unit vectors).
// atan2(0, 0) = 0.
__device__ __forceinline__ float xatan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  const float a = mx > 0.f ? mn / mx : 0.f;
  const float a2 = a * a;
  float p = fmaf(a2, 0.002903702901676297f, -0.016283642500638962f);
  p = fmaf(a2, p, 0.04304046556353569f);
  p = fmaf(a2, p, -0.07533776760101318f);
  p = fmaf(a2, p, 0.10654730349779129f);
  p = fmaf(a2, p, -0.14207148551940918f);
  p = fmaf(a2, p, 0.1999305635690689f);
  p = fmaf(a2, p, -0.3333309292793274f);
  p = fmaf(a2, p, 1.0f);
  float r = a * p;
  if (ay > ax) r = 1.5707963705062866f - r;
  if (x < 0.f) r = 3.1415927410125732f - r;
  return y < 0.f ? -r : r;
}
template <int N>
__device__ __forceinline__ DualF<N> xatan2(const DualF<N>& y, const DualF<N>& x) {
  DualF<N> r;
  r.v = xatan2(y.v, x.v);
  const float inv = 1.0f / (x.v * x.v + y.v * y.v);
#pragma unroll
  for (int k = 0; k < N; ++k) r.d[k] = (x.v * y.d[k] - y.v * x.d[k]) * inv;
  return r;
}
// Sine and cosine of an angle of at most pi/2 in magnitude (the fiber
// normal's deviation from the ply normal): the Taylor series of sin to
// x^13 / 13! and of cos to x^14 / 14!, in Horner form in x^2.  The first
// omitted terms are below 7e-10 on [-pi/2, pi/2], so the error is the
// evaluation's float rounding (a few 1e-8 absolute; cos keeps an absolute,
// not a relative, bound next to pi/2).  Larger arguments take sincosf.
__device__ __forceinline__ void xsincos(float x, float* s, float* c) {
  if (!(fabsf(x) <= 1.57079637f)) {
    sincosf(x, s, c);
    return;
  }
  const float x2 = x * x;
  float ps = fmaf(x2, 1.6059044e-10f, -2.5052108e-8f);   // 1/13!, -1/11!
  ps = fmaf(x2, ps, 2.7557319e-6f);                       // 1/9!
  ps = fmaf(x2, ps, -1.9841270e-4f);                      // -1/7!
  ps = fmaf(x2, ps, 8.3333333e-3f);                       // 1/5!
  ps = fmaf(x2, ps, -0.16666667f);                        // -1/3!
  float pc = fmaf(x2, -1.1470746e-11f, 2.0876757e-9f);   // -1/14!, 1/12!
  pc = fmaf(x2, pc, -2.7557319e-7f);                      // -1/10!
  pc = fmaf(x2, pc, 2.4801587e-5f);                       // 1/8!
  pc = fmaf(x2, pc, -1.3888889e-3f);                      // -1/6!
  pc = fmaf(x2, pc, 4.1666668e-2f);                       // 1/4!
  pc = fmaf(x2, pc, -0.5f);                               // -1/2!
  *s = fmaf(x * x2, ps, x);
  *c = fmaf(x2, pc, 1.0f);
}
template <int N>
__device__ __forceinline__ void xsincos(const DualF<N>& x, DualF<N>* s, DualF<N>* c) {
  float sv, cv;
  xsincos(x.v, &sv, &cv);
  *s = dchain(x, sv, cv);
  *c = dchain(x, cv, -sv);
}
// sin and cos of 2 pi t (t in turns); the pi-scaled form reduces exactly.
__device__ __forceinline__ void xsincos_turns(float t, float* s, float* c) {
  sincospif(2.0f * t, s, c);
}
template <int N>
__device__ __forceinline__ void xsincos_turns(const DualF<N>& t, DualF<N>* s, DualF<N>* c) {
  float sv, cv;
  sincospif(2.0f * t.v, &sv, &cv);
  *s = dchain(t, sv, 2.0f * kPi * cv);
  *c = dchain(t, cv, -2.0f * kPi * sv);
}
// sin and cos of 2 pi t for the small per-step phase advances of the ply
// trace: t is reduced to [-1/2, 1/2] exactly and the hardware
// approximations are taken (absolute error ~5e-7); the tangents follow from
// those values.
__device__ __forceinline__ void xsincos_turns_fast(float t, float* s, float* c) {
  const float r = t - rintf(t);
  __sincosf((2.0f * kPi) * r, s, c);
}
template <int N>
__device__ __forceinline__ void xsincos_turns_fast(const DualF<N>& t, DualF<N>* s, DualF<N>* c) {
  float sv, cv;
  xsincos_turns_fast(t.v, &sv, &cv);
  *s = dchain(t, sv, 2.0f * kPi * cv);
  *c = dchain(t, cv, -2.0f * kPi * sv);
}
template <class S> __device__ __forceinline__ S xmax0(const S& a) { return vf(a) < 0.f ? S(0.f) : a; }

// ----------------------------------------------------------- index checks --
// The index-checking build (-DBYSDF_DEBUG_BOUNDS, a separate library, the
// stand-in for a memory checker): a checked index out of range sets bit 2
// (ERR_BOUNDS) of the launch's error word and is clamped, so the access
// stays in bounds.  Each kernel that reaches a check stores the word's
// address (or NULL) in g_bounds_word before any check runs.  Compiled out of
// the product build.
enum : uint32_t { ERR_BOUNDS = 4u };
#ifdef BYSDF_DEBUG_BOUNDS
__shared__ unsigned long long* g_bounds_word;
__device__ __forceinline__ void bounds_fail() {
  if (g_bounds_word) atomicOr(g_bounds_word, (unsigned long long)ERR_BOUNDS);
}
#define BY_BOUNDS(ok, fix) \
  do {                     \
    if (!(ok)) {           \
      bounds_fail();       \
      fix;                 \
    }                      \
  } while (0)
#else
#define BY_BOUNDS(ok, fix) \
  do {                     \
  } while (0)
#endif
// the check as a value: false (after recording it) when the index is out of
// range, so the caller can skip the access; always true in the product build
__device__ __forceinline__ bool bounds_ok(bool ok) {
#ifdef BYSDF_DEBUG_BOUNDS
  if (!ok) bounds_fail();
  return ok;
#else
  (void)ok;
  return true;
#endif
}

// ----------------------------------------------------------------- vectors --
template <class S>
struct V3 {
  S x, y, z;
};
template <class S> __device__ __forceinline__ V3<S> mk3(const S& x, const S& y, const S& z) {
  V3<S> r;
  r.x = x; r.y = y; r.z = z;
  return r;
}
template <class S> __device__ __forceinline__ V3<S> lift3(float x, float y, float z) {
  return mk3<S>(S(x), S(y), S(z));
}
template <class S> __device__ __forceinline__ V3<S> operator+(const V3<S>& a, const V3<S>& b) {
  return mk3<S>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <class S> __device__ __forceinline__ V3<S> operator-(const V3<S>& a, const V3<S>& b) {
  return mk3<S>(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <class S> __device__ __forceinline__ V3<S> operator-(const V3<S>& a) {
  return mk3<S>(-a.x, -a.y, -a.z);
}
template <class S, class T> __device__ __forceinline__ V3<S> operator*(const V3<S>& a, const T& s) {
  return mk3<S>(a.x * s, a.y * s, a.z * s);
}
// a float vector may meet a dual one (a direction without tangents against
// the frame): the products then carry only the dual side's tangents
template <class A, class B> __device__ __forceinline__ auto dot(const V3<A>& a, const V3<B>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <int N>
__device__ __forceinline__ V3<DualF<N>> operator+(const V3<DualF<N>>& a, const V3<float>& b) {
  return mk3<DualF<N>>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <int N>
__device__ __forceinline__ V3<DualF<N>> operator+(const V3<float>& a, const V3<DualF<N>>& b) {
  return mk3<DualF<N>>(a.x + b.x, a.y + b.y, a.z + b.z);
}
// a float vector as S (no tangents), or the vector itself
template <class S, class W> __device__ __forceinline__ V3<S> as3(const V3<W>& w) {
  if constexpr (std::is_same<S, W>::value) {
    return w;
  } else {
    return mk3<S>(S(w.x), S(w.y), S(w.z));
  }
}
template <class S> __device__ __forceinline__ V3<S> cross(const V3<S>& a, const V3<S>& b) {
  return mk3<S>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class S> __device__ __forceinline__ V3<S> normalize(const V3<S>& a) {
  return a * xrsqrt(dot(a, a));
}

}  // namespace bysdf
