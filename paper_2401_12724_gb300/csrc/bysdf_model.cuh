// Per-record yarn BYSDF model (device).  One implementation, generic in the
// scalar type S: float for eval / sample / pdf, DualF<ND> for the backward.
//
// Steps (Khattar et al.):
//   entry ray from (h, u, omega_i)          Sec. 3.3 (reading: in-plane angle
//                                           asin h from -n_u, slope from omega_i)
//   implicit ply trace, N_it updates         Sec. 3.4
//   ply frame, fiber frame from 1D maps      Sec. 3.4, 3.5.1
//   G_p (in-plane chords through the other   Sec. 4.1.4
//   plies), G_f (fiber map)
//   footprint nodes and aggregation          Sec. 4.2 Eqs. 8-11, Sec. 5.3
//   lobes f_x^S, f_y^S, f_x^B, f_y^B         Sec. 4.1 Eqs. 1-6, tau^{N_i} Eq. 4
//   sampling, pdf                            Sec. 4.1.5
#pragma once

#include "bysdf_common.cuh"

namespace bysdf {

// ST_ABORTED: not evaluated, a device-side wait gave up (see the error word)
enum { ST_OK = 0, ST_NO_HIT = 1, ST_INVALID = 2, ST_BAD_SAMPLE = 3, ST_ABORTED = 4 };

struct Record {
  float h, u, v, ratio;
  float wi[3], wo[3];
  float u0, u1;
  int mat;
};

// frac(k * v) for a rate k = hi + lo held as two floats: the product is
// formed exactly (FMA residual) before the integer part is dropped, so a
// phase of hundreds of turns keeps float precision in its fraction.
__device__ __forceinline__ float frac_prod(float hi, float lo, float v) {
  const float p = __fmul_rn(hi, v);
  float e = fmaf(hi, v, -p);
  e = fmaf(lo, v, e);
  return __fadd_rn(__fsub_rn(p, rintf(p)), e);
}

// Differentiable per-material quantities.
template <class S>
struct MatVars {
  S kp, kf;             // ply turns / length, fiber map periods / length
  S cos_af, sin_af;     // fiber helix angle
  float sigma_s;        // shadow density (closed-form derivative)
  float beta_t, beta_b; // GGX roughness, radians (closed-form derivatives)
  bool seeded;          // helix-angle tangents carried (parameter backward)
};

template <class S>
// seed_params: carry the helix-angle tangents (the parameter backward);
// false for dual numbers that carry other tangents (the direction backward)
__device__ __forceinline__ MatVars<S> mat_vars(const MatDev& m, bool seed_params = true) {
  MatVars<S> q;
  q.kp = S(m.kp_hi + m.kp_lo);
  q.kf = S(m.kf_hi + m.kf_lo);
  q.cos_af = S(m.cos_af);
  q.sin_af = S(m.sin_af);
  q.sigma_s = m.sigma_s;
  q.beta_t = m.beta_t;
  q.beta_b = m.beta_b;
  q.seeded = false;
  if constexpr (is_dual<S>::value) {
    if (!seed_params) return q;
    q.seeded = true;
    q.kp.d[D_ALPHA_P] = m.dkp;
    q.kf.d[D_ALPHA_F] = m.dkf;
    q.cos_af.d[D_ALPHA_F] = -m.sin_af;
    q.sin_af.d[D_ALPHA_F] = m.cos_af;
  }
  return q;
}

// frac(k v) with the tangent of k v (the value is the compensated one).
template <class S>
__device__ __forceinline__ S frac_prod_s(const S& k, float hi, float lo, float v) {
  if constexpr (is_dual<S>::value) {
    S r = k * v;
    r.v = frac_prod(hi, lo, v);
    return r;
  } else {
    return frac_prod(hi, lo, v);
  }
}

// ------------------------------------------------------------ validation --
__device__ __forceinline__ bool finitef(float x) { return isfinite(x); }

// The checks are combined without early exits (one branch per record, not
// one per input: 1.7% of the fused kernel's time).  A direction is unit
// within 1e-3 only if its components are finite (a non-finite component
// makes the squared norm NaN or infinite).
__device__ __forceinline__ bool unit_ok(const float* w) {
  const float nn = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
  return fabsf(nn - 1.0f) <= 1e-3f;
}
// Inputs every op needs: (h, u, v, omega_i, material id, ratio).
__device__ __forceinline__ bool base_valid(const Record& q, int n_mat, bool has_ratio) {
  const bool ratio_ok = !has_ratio || (q.ratio >= 0.0f && q.ratio < INFINITY);
  return (fabsf(q.h) <= 1.0f) & finitef(q.u) & finitef(q.v) & unit_ok(q.wi) &
         (q.mat >= 0) & (q.mat < n_mat) & ratio_ok;
}
__device__ __forceinline__ bool u_valid(const Record& q) {
  return (q.u0 >= 0.0f) & (q.u0 < 1.0f) & (q.u1 >= 0.0f) & (q.u1 < 1.0f);
}
__device__ __forceinline__ bool record_valid(const Record& q, int n_mat, bool need_wo,
                                             bool has_ratio, bool need_u) {
  return base_valid(q, n_mat, has_ratio) && (!need_wo || unit_ok(q.wo)) &&
         (!need_u || u_valid(q));
}

// ------------------------------------------------------------- footprint --
// Sec. 4.2 / 5.3 (reading): ratio is the half-width of [h1, h2] in h units;
// K = ceil(K_max (h2 - h1) / 2) midpoint nodes.  Decided in float with
// explicitly rounded operations (no contraction), as the oracle decides it.
struct Footprint {
  float h1, width;
  int K;
};
__device__ __forceinline__ Footprint footprint(float h0, float ratio, int kmax) {
  Footprint f;
  const float a = __fsub_rn(h0, ratio);
  const float b = __fadd_rn(h0, ratio);
  f.h1 = a < -1.0f ? -1.0f : a;
  const float h2 = b > 1.0f ? 1.0f : b;
  f.width = __fsub_rn(h2, f.h1);
  const float kf = __fmul_rn((float)kmax * 0.5f, f.width);
  int K = (int)ceilf(kf);
  f.K = K < 1 ? 1 : (K > kmax ? kmax : K);
  return f;
}

// ------------------------------------------------------------- geometry --
template <class S>
struct NodeGeo {
  bool hit;
  int ni;
  int ply;  // closest ply
  V3<S> x, nf, tf;
  S g;            // G_p * G_f
  float dg_dsig;  // d(G_p G_f) / d sigma_s (value)
};

// Sec. 3.5.1: periodic linear interpolation of the tabulated maps; w is the
// fiber phase in map periods.
template <class S>
__device__ __forceinline__ void fiber_lookup(const float2* map, int T, const S& w, S* delta,
                                             S* of) {
  const float wv = vf(w) + 0.5f;
  const S a = w + (0.5f - floorf(wv));
  const S tau = a * (float)T - 0.5f;
  const float fl = floorf(vf(tau));
  const S f = tau - fl;
  int i0 = (int)fl;
  i0 = i0 < 0 ? i0 + T : (i0 >= T ? i0 - T : i0);
  BY_BOUNDS(i0 >= 0 && i0 < T, i0 = 0);
  const int i1 = i0 + 1 == T ? 0 : i0 + 1;
  const float2 t0 = map[i0], t1 = map[i1];
  *delta = t0.x + f * (t1.x - t0.x);
  *of = t0.y + f * (t1.y - t0.y);
}

// Sec. 3.5 fiber migration (reading): the yarn is cut into segments of
// length L along v; segment s uses map table[s mod 256] (the host fills the
// table from a Philox4x64-10 word per segment) and blends linearly with its
// neighbour within b L of a boundary (weight 1/2 at the boundary).  Map
// k >= 1 is the ring sunk by k r_f / K_m, with its own fiber count and phase
// rate.  Picks the map and phase of the hit's segment (*mp, *wv) and, in a
// blend zone, the neighbour's (*mp1, *wv1) with its weight *wgt (else 0).
// u_ply: ply azimuth (radians); v: the record's height; dz: the hit's
// height above it; w0: map 0's phase (periods).
template <class S>
__device__ __forceinline__ void migration_maps(const MatDev& m, const float2* map0,
                                               const MatVars<S>& mv, const S& u_ply, float v,
                                               const S& dz, const S& w0, const float2** mp,
                                               S* wv, const float2** mp1, S* wv1, S* wgt) {
  // t = frac((v + dz) / L) and the segment, with 1 / L as hi + lo and the
  // product's rounding error recovered exactly
  const MigMap* m1 = mig_map(m, 1);
  const float ph = v * m.mig_inv_len;
  const float pe = fmaf(v, m.mig_inv_len, -ph) + v * m1->aux;
  float nf = floorf(ph);
  S t = dz * m.mig_inv_len + ((ph - nf) + pe);
  const float kf2 = floorf(vf(t));
  t = t - kf2;
  nf += kf2;
  const int seg = (int)(((int64_t)nf % kMigPeriod + kMigPeriod) % kMigPeriod);
  int nb = seg;
  *wgt = S(0.f);
  if (vf(t) < m.mig_blend) {
    *wgt = 0.5f - t * m.mig_inv_2b;
    nb = seg == 0 ? kMigPeriod - 1 : seg - 1;
  } else if (vf(t) > 1.0f - m.mig_blend) {
    *wgt = 0.5f - (1.0f - t) * m.mig_inv_2b;
    nb = seg == kMigPeriod - 1 ? 0 : seg + 1;
  }
  const uint8_t* tab = mig_table(m);
  auto pick = [&](int sg, const float2** p, S* wk) {
    BY_BOUNDS(sg >= 0 && sg < kMigPeriod, sg = 0);
    int k = tab[sg];
    BY_BOUNDS(k < m.mig_maps, k = 0);
    if (k == 0) {
      *p = map0;
      *wk = w0;
      return;
    }
    const MigMap* mk = mig_map(m, k);
    S kf = S(mk->kf_hi + mk->kf_lo);
    if constexpr (is_dual<S>::value) {
      if (mv.seeded) kf.d[D_ALPHA_F] = mk->dkf;
    }
    *p = reinterpret_cast<const float2*>(mk + 1);
    *wk = u_ply * mk->m_over_2pi - frac_prod_s(kf, mk->kf_hi, mk->kf_lo, v) - kf * dz;
  };
  pick(seg, mp, wv);
  if (vf(*wgt) > 0.f) pick(nb, mp1, wv1);
}

// Scalar of the ply trace (see node_geometry): the parameter backward's
// two-tangent dual numbers (alpha_p, alpha_f) with float directions trace
// with alpha_p alone; every other scalar traces as itself.
template <class S, class K>
struct TraceScalar {
  using type = S;
};
template <>
struct TraceScalar<DualF<ND>, float> {
  using type = DualF<1>;
};
template <class P, class S>
__device__ __forceinline__ P narrow(const S& x) {
  if constexpr (std::is_same<P, S>::value) {
    return x;
  } else {
    P r;
    r.v = x.v;
    r.d[0] = x.d[D_ALPHA_P];
    return r;
  }
}
template <class S, class P>
__device__ __forceinline__ S widen(const P& x) {
  if constexpr (std::is_same<P, S>::value) {
    return x;
  } else {
    S r(x.v);
    r.d[D_ALPHA_P] = x.d[0];
    return r;
  }
}
template <class S, class P>
__device__ __forceinline__ V3<S> widen3(const V3<P>& x) {
  return mk3<S>(widen<S>(x.x), widen<S>(x.y), widen<S>(x.z));
}

template <class S, int PLIES = 2, class K = float>
__device__ __forceinline__ void node_geometry(const MatDev& m, const float2* map,
                                              const MatVars<S>& mv, float X0x, float X0y,
                                              float ex, float ey, float v, const K& kappa,
                                              const K& wx, const K& wy, const S& s0v,
                                              const S& c0v, const S& phase_f_v,
                                              NodeGeo<S>& out, int only_ply = -1,
                                              int ni_known = 0, bool trace_only = false,
                                              bool coarse = false) {
  const float Rp = m.Rp, Rc = m.Rc;
  out.hit = false;
  out.ni = 0;
  // Per ply: start in the cross-section at the yarn hit (t = 0), intersect
  // the in-plane ray with the ply circle there, move to the cross-section of
  // that intersection and repeat, N_it updates; an update whose circle the
  // ray misses marks the ply "not hit".
  const int n_re = m.nit < 1 ? m.nit : 1;
  int best = -1, n_upd = m.nit;
  float t_start = 0.f;
  if (only_ply >= 0) {
    // the closest ply and N_i are known already (from a float pass over all
    // plies): trace that ply alone, all N_it updates in S
    best = only_ply;
    out.ni = ni_known;
  } else {
    // Float pass over all plies, to pick the closest ply and count N_i.  The
    // ply centre c = R_c (cos, sin)(psi_k + 2 pi kp kappa t) enters an update
    // only through b = (X0 - c).e and perp = (X0 - c) x e, which are linear
    // in (cos, sin) of the phase advance: with A_k = R_c (cos psi_k, sin
    // psi_k).e and B_k = R_c (cos psi_k, sin psi_k) x e, an update is 4 FMAs
    // and one hardware sin/cos.  Every ply runs all N_it updates (a miss is
    // a flag, not a break), so the lanes of a warp -- one material, hence one
    // N_p, after the tile sort -- never diverge here.  The closest ply's last
    // update (n_re = 1) is run again below with the correctly rounded
    // sin/cos, so the hit carries float32 rounding and the earlier updates'
    // hardware sin/cos error damped by the contraction of the map (two
    // exact updates measured the same parity and cost 1.3% more on
    // near-field records, 4% on footprint records).
    const float kk = vf(mv.kp) * vf(kappa);
    const float bx0 = X0x * ex + X0y * ey, px0 = X0x * ey - X0y * ex;
    const float c0 = vf(c0v), s0 = vf(s0v);
    const float A0 = Rc * (c0 * ex + s0 * ey), B0 = Rc * (c0 * ey - s0 * ex);
    const float Rp2 = Rp * Rp;
    float best_t = 0.f;
    auto consider = [&](int k, bool hit, float t, float t_re) {
      if (hit) {
        out.ni += 1;
        if (best < 0 || t < best_t) {
          best = k;
          best_t = t;
          t_start = t_re;
        }
      }
    };
    // Update 0 starts in the hit's cross-section (no phase advance, no
    // sin/cos): a ply whose circle the ray misses there is not hit whatever
    // the later updates give, so only the plies that pass it are iterated.
    uint32_t todo = 0;
#pragma unroll 1
    for (int k = 0; k < m.np; ++k) {
      const float perp = px0 - (B0 * m.rot_c[k] - A0 * m.rot_s[k]);
      if (fmaf(-perp, perp, Rp2) >= 0.f) todo |= 1u << k;
    }
    // updates 1 .. N_it - 1; t at the entry of update N_it - n_re is where
    // the exact re-run starts.  The update loops (like the update-0 mask,
    // node and shadowing loops) stay rolled: unrolled copies of these bodies cost more
    // in instruction fetch (the kernels are large, and their warps spread
    // over them) than they save in branches.
    const int n_mid = m.nit - n_re > 1 ? m.nit - n_re : 1;
    if constexpr (PLIES == 1) {
      while (todo) {
        const int k = __ffs(todo) - 1;
        todo &= todo - 1;
        const float A = A0 * m.rot_c[k] + B0 * m.rot_s[k];
        const float Bk = B0 * m.rot_c[k] - A0 * m.rot_s[k];
        const float p0 = px0 - Bk;
        float t = fmaxf(-(bx0 - A) - sqrtf(fmaxf(fmaf(-p0, p0, Rp2), 0.f)), 0.f);
        bool hit = true;
        auto update = [&]() {
          float sd, cd;
          xsincos_turns_fast(kk * t, &sd, &cd);
          const float bb = fmaf(-sd, Bk, fmaf(-cd, A, bx0));
          const float perp = fmaf(sd, A, fmaf(-cd, Bk, px0));
          const float disc = fmaf(-perp, perp, Rp2);
          hit = hit && disc >= 0.f;
          // a miss gives sqrt(disc < 0) = NaN and fmaxf(NaN, 0) = 0; the
          // ply is flagged and its t no longer used
          t = fmaxf(-bb - sqrtf(disc), 0.f);
        };
#pragma unroll 1
        for (int n = 1; n < n_mid; ++n) update();
        const float t_re = m.nit > n_re ? t : 0.f;
#pragma unroll 1
        for (int n = n_mid; n < m.nit; ++n) update();
        consider(k, hit, t, t_re);
      }
    } else {
      // two plies per pass: two independent dependency chains per lane
      while (todo) {
        const int ka = __ffs(todo) - 1;
        todo &= todo - 1;
        const bool two = todo != 0;
        const int kb = two ? __ffs(todo) - 1 : ka;
        todo &= todo - 1;
        const float Aa = A0 * m.rot_c[ka] + B0 * m.rot_s[ka];
        const float Ba = B0 * m.rot_c[ka] - A0 * m.rot_s[ka];
        const float Ab = A0 * m.rot_c[kb] + B0 * m.rot_s[kb];
        const float Bb = B0 * m.rot_c[kb] - A0 * m.rot_s[kb];
        const float pa0 = px0 - Ba, pb0 = px0 - Bb;
        float ta = fmaxf(-(bx0 - Aa) - sqrtf(fmaxf(fmaf(-pa0, pa0, Rp2), 0.f)), 0.f);
        float tb = fmaxf(-(bx0 - Ab) - sqrtf(fmaxf(fmaf(-pb0, pb0, Rp2), 0.f)), 0.f);
        bool ha = true, hb = true;
        auto update = [&]() {
          float sa, ca, sb, cb;
          xsincos_turns_fast(kk * ta, &sa, &ca);
          xsincos_turns_fast(kk * tb, &sb, &cb);
          const float ba = fmaf(-sa, Ba, fmaf(-ca, Aa, bx0));
          const float bb = fmaf(-sb, Bb, fmaf(-cb, Ab, bx0));
          const float pa = fmaf(sa, Aa, fmaf(-ca, Ba, px0));
          const float pb = fmaf(sb, Ab, fmaf(-cb, Bb, px0));
          const float da = fmaf(-pa, pa, Rp2);
          const float db = fmaf(-pb, pb, Rp2);
          ha = ha && da >= 0.f;
          hb = hb && db >= 0.f;
          // a miss gives sqrt(d < 0) = NaN and fmaxf(NaN, 0) = 0; the ply
          // is flagged and its t no longer used
          ta = fmaxf(-ba - sqrtf(da), 0.f);
          tb = fmaxf(-bb - sqrtf(db), 0.f);
        };
#pragma unroll 1
        for (int n = 1; n < n_mid; ++n) update();
        const float ta_re = m.nit > n_re ? ta : 0.f, tb_re = m.nit > n_re ? tb : 0.f;
#pragma unroll 1
        for (int n = n_mid; n < m.nit; ++n) update();
        consider(ka, ha, ta, ta_re);
        if (two) consider(kb, hb, tb, tb_re);
      }
    }
    if (best < 0) return;
    n_upd = n_re;
  }
  out.hit = true;
  out.ply = best;
  if (trace_only) return;
  // the closest ply's updates with sincospif: ply centre, its phase and the
  // intersection distance of the last one.  In the parameter backward (two
  // tangents, alpha_p and alpha_f, and float directions) only alpha_p moves
  // the trace, the ply frame, the ply azimuth and the ply shadowing: that
  // part runs in P, which carries alpha_p alone (P = S otherwise).
  using P = typename TraceScalar<S, K>::type;
  const P kp = narrow<P>(mv.kp);
  const P c0p = narrow<P>(c0v), s0p = narrow<P>(s0v);
  const P ck = c0p * m.rot_c[best] - s0p * m.rot_s[best];
  const P sk = s0p * m.rot_c[best] + c0p * m.rot_s[best];
  P best_t = P(t_start), best_cx = P(0.f), best_cy = P(0.f), best_s = P(0.f), best_c = P(1.f);
  bool grazed = false;
#pragma unroll 1
  for (int i = 0; i < n_upd; ++i) {
    // the dual pass traces its ply's N_it updates like the float pass: the
    // hardware sin/cos, the last update correctly rounded
    P sd, cd;
    if (i + 1 < n_upd || coarse) {
      xsincos_turns_fast(kp * (kappa * best_t), &sd, &cd);
    } else {
      xsincos_turns(kp * (kappa * best_t), &sd, &cd);
    }
    best_c = ck * cd - sk * sd;
    best_s = sk * cd + ck * sd;
    best_cx = Rc * best_c;
    best_cy = Rc * best_s;
    const P qx = X0x - best_cx, qy = X0y - best_cy;
    const P b = qx * ex + qy * ey;
    const P perp = qx * ey - qy * ex;
    const P disc = (Rp - perp) * (Rp + perp);
    grazed = grazed || !(vf(disc) > 0.f);
    best_t = xmax0(-b - xsqrt(xmax0(disc)));
  }
  if (grazed) {
    // the ray grazes the ply within rounding: the dual pass has no
    // derivative there (the node is dropped, as when its trace misses); the
    // float pass keeps the tangent point
    if constexpr (is_dual<S>::value) {
      out.hit = false;
      return;
    }
  }
  // Sec. 3.4: hit point, ply normal (from the ply centre, in the circular
  // cross-section), ply tangent (derivative of the helix through x)
  const P xx = X0x + best_t * ex, xy = X0y + best_t * ey;
  const P dz = kappa * best_t;
  out.x = mk3<S>(widen<S>(xx), widen<S>(xy), widen<S>(v + dz));
  const P dx = xx - best_cx, dy = xy - best_cy;
  const P inv_dl = xrsqrt(dx * dx + dy * dy);
  const V3<P> np = mk3<P>(dx * inv_dl, dy * inv_dl, P(0.f));
  const P wp = (2.0f * kPi) * kp;
  const V3<P> traw = mk3<P>(-(wp * xy), wp * xx, P(1.f));
  const V3<P> tp = normalize(traw - np * dot(traw, np));
  const V3<P> ep = cross(tp, np);
  // Sec. 3.5.1: ply azimuth of the hit about the ply centre, from the ply
  // centre's radial direction; fiber phase in map periods; 1D map lookup
  const S u_ply =
      widen<S>(xatan2(best_c * np.y - best_s * np.x, best_c * np.x + best_s * np.y));
  const S dzs = widen<S>(dz);
  const S w = u_ply * m.m_over_2pi - phase_f_v - mv.kf * dzs;
  // map 0, or the migration maps of the hit's segment (Sec. 3.5)
  S delta, of;
  if (m.mig_maps > 1) {
    const float2* mp = map;
    const float2* mp1 = map;
    S wv = w, wv1 = w, wgt = S(0.f);
    migration_maps(m, map, mv, u_ply, v, dzs, w, &mp, &wv, &mp1, &wv1, &wgt);
    fiber_lookup(mp, m.T, wv, &delta, &of);
    if (vf(wgt) > 0.f) {
      S d1, o1;
      fiber_lookup(mp1, m.T, wv1, &d1, &o1);
      delta = delta + wgt * (d1 - delta);
      of = of + wgt * (o1 - of);
    }
  } else {
    fiber_lookup(map, m.T, w, &delta, &of);
  }
  // n_f = n'(R(n_p)), t_f = t'(R(t_p))
  const V3<S> nps = widen3<S>(np);
  out.tf = widen3<S>(tp) * mv.cos_af + widen3<S>(ep) * mv.sin_af;
  S sd, cd;
  if constexpr (!is_dual<S>::value) {
    // a node of a multi-node aggregate: the hardware sin/cos (|delta| <=
    // pi/2, absolute error ~5e-7)
    if (coarse) {
      __sincosf(delta, &sd, &cd);
    } else {
      xsincos(delta, &sd, &cd);
    }
  } else {
    xsincos(delta, &sd, &cd);
  }
  out.nf = nps * cd + cross(out.tf, nps) * sd;
  // Sec. 4.1.4: ply shadowing by the in-plane chords through the other
  // plies of this cross-section; fiber shadowing from the map
  P occ = P(0.f);
#pragma unroll 1
  for (int j = 1; j < m.np; ++j) {
    int r = j;
    const float rc = m.rot_c[r], rs = m.rot_s[r];
    const P cjx = best_cx * rc - best_cy * rs, cjy = best_cx * rs + best_cy * rc;
    const P qx = xx - cjx, qy = xy - cjy;
    const P b = qx * wx + qy * wy;
    const P perp = qx * wy - qy * wx;
    const P disc = (Rp - perp) * (Rp + perp);
    if constexpr (is_dual<P>::value) {
      if (vf(disc) > 0.f) {
        const P sq = xsqrt(disc);
        const P s2 = sq - b;
        if (vf(s2) > 0.f) occ = occ + (s2 - xmax0(-b - sq));
      }
    } else {
      // predicated (no branch): the chord from its near end max(-b - sq, 0)
      // to its far end s2 = sq - b, where the ray meets the disc ahead
      const float sq = sqrtf(fmaxf(disc, 0.f));
      const float s2 = sq - b;
      const float chord = s2 - fmaxf(-b - sq, 0.f);
      occ += (disc > 0.f && s2 > 0.f) ? chord : 0.f;
    }
  }
  const S occ_all = widen<S>(occ) * m.inv_2Rp + of;
  out.g = xexp(-(mv.sigma_s * occ_all));
  out.dg_dsig = -vf(occ_all) * vf(out.g);
}

// Aggregated geometry of a record (Sec. 4.2 Eqs. 8-11, W = 1).
template <class S>
struct Geo {
  int status;
  float width;
  V3<S> n, t, x;
  S g, ni;
  float dg_dsig;
};

// PLIES: plies traced side by side in the float pass of the ply trace (2
// gives each lane two independent dependency chains and costs ~5 registers)
// sc: the stochastic estimators' state (jittered nodes), or NULL
template <int PLIES = 2, class S, class K>
__device__ __forceinline__ void geometry_k(const MatDev& m, const float2* map,
                                           const MatVars<S>& mv, const Record& q,
                                           const V3<K>& wi, Geo<S>& G,
                                           const StochCtx* sc = nullptr) {
  G.status = ST_NO_HIT;
  const Footprint fp = footprint(q.h, q.ratio, m.kmax);
  G.width = fp.width;
  // (sin, cos) of u and, by the angle-difference identity, of the in-plane
  // ray's azimuth u_rel = u - asin(h): one sine / cosine and one square root
  float sU, cU;
  sincosf(q.u, &sU, &cU);
  const float ch = sqrtf(fmaxf(0.f, 1.0f - q.h * q.h));
  const float su = fmaf(sU, ch, -cU * q.h), cu = fmaf(cU, ch, sU * q.h);
  const float ex = -cu, ey = -su;
  const K lxy = xsqrt(wi.x * wi.x + wi.y * wi.y);
  if (!(vf(lxy) >= 1e-7f)) return;
  const K inv_l = 1.0f / lxy;
  const K kappa = -wi.z * inv_l;
  const K wx = wi.x * inv_l, wy = wi.y * inv_l;
  // ply 0's phase at the hit's cross-section, and the fiber phase there
  const S turns_v = frac_prod_s(mv.kp, m.kp_hi, m.kp_lo, q.v);
  S s0v, c0v;
  xsincos_turns(turns_v, &s0v, &c0v);
  const S phase_f_v = frac_prod_s(mv.kf, m.kf_hi, m.kf_lo, q.v);
  // derivatives follow the branch the values take: a float pass picks the
  // closest ply and N_i of each node, the dual pass re-traces that ply only
  MatVars<float> mvf;
  float s0f = 0.f, c0f = 1.f, pff = 0.f;
  if constexpr (is_dual<S>::value) {
    mvf = mat_vars<float>(m);
    s0f = s0v.v;
    c0f = c0v.v;
    pff = phase_f_v.v;
  }
  V3<S> ns = lift3<S>(0.f, 0.f, 0.f), ts = ns, xs = ns;
  S gs = S(0.f);
  float dgs = 0.f;
  int nis = 0, nhit = 0;
  const bool near = fp.K == 1 && fp.width == 0.0f;
  const bool jitter = sc != nullptr && (sc->flags & STOCH_JITTER_NODES) != 0;
  U64x4 rnd = {{0, 0, 0, 0}};
#pragma unroll 1
  for (int j = 0; j < fp.K; ++j) {
    float X0x, X0y;
    if (near) {
      X0x = cU;
      X0y = sU;
    } else {
      // midpoint of stratum j, or a uniform point in it (Sec. 4.2, stratified
      // sampling of h)
      float xj = 0.5f;
      if (jitter) {
        if ((j & 3) == 0) rnd = philox4x64(sc->index, (uint64_t)(j >> 2), 0, 0, sc->seed, kStochKey1);
        xj = unit24(rnd.w[j & 3]);
      }
      const float hj = fp.h1 + ((float)j + xj) * fp.width / (float)fp.K;
      // entry azimuth u_rel + asin(hj) by the angle-sum identity from the
      // record's (sin, cos)(u_rel): one square root per node instead of an
      // arcsine and a range-reduced sine / cosine
      const float cj = sqrtf(fmaxf(0.f, 1.0f - hj * hj));
      X0x = fmaf(cu, cj, -su * hj);
      X0y = fmaf(su, cj, cu * hj);
    }
    X0x *= m.R;
    X0y *= m.R;
    NodeGeo<S> nd;
    if constexpr (is_dual<S>::value) {
      NodeGeo<float> pick;
      node_geometry<float, PLIES, float>(m, map, mvf, X0x, X0y, ex, ey, q.v, vf(kappa), vf(wx),
                                         vf(wy), s0f, c0f, pff, pick, -1, 0, true);
      if (!pick.hit) continue;
      node_geometry<S, PLIES, K>(m, map, mv, X0x, X0y, ex, ey, q.v, kappa, wx, wy, s0v, c0v,
                                 phase_f_v, nd, pick.ply, pick.ni);
    } else {
      // a node of several: its last update takes the hardware sin/cos too
      // (the aggregate averages the nodes' frames)
      node_geometry<S, PLIES, K>(m, map, mv, X0x, X0y, ex, ey, q.v, kappa, wx, wy, s0v, c0v,
                                 phase_f_v, nd, -1, 0, false, !near);
    }
    if (!nd.hit) continue;
    nhit += 1;
    nis += nd.ni;
    ns = ns + nd.nf;
    ts = ts + nd.tf;
    xs = xs + nd.x;
    gs = gs + nd.g;
    dgs += nd.dg_dsig;
  }
  if (nhit == 0) return;
  const float inv = 1.0f / (float)nhit;
  const S nl = xsqrt(dot(ns, ns));
  if (!(vf(nl) > 1e-9f * (float)nhit)) return;
  G.n = ns * (1.0f / nl);
  const V3<S> tperp = ts - G.n * dot(ts, G.n);
  const S tl = xsqrt(dot(tperp, tperp));
  if (!(vf(tl) > 1e-9f * (float)nhit)) return;
  G.t = tperp * (1.0f / tl);
  G.x = xs * inv;
  G.g = gs * inv;
  G.dg_dsig = dgs * inv;
  G.ni = S((float)nis * inv);
  G.status = ST_OK;
}
// the record's own (float) incoming direction
template <int PLIES = 2, class S>
__device__ __forceinline__ void geometry(const MatDev& m, const float2* map,
                                         const MatVars<S>& mv, const Record& q, Geo<S>& G) {
  geometry_k<PLIES, S, float>(m, map, mv, q, mk3<float>(q.wi[0], q.wi[1], q.wi[2]), G);
}

// ------------------------------------------------------------ microfacet --
// Unpolarised dielectric Fresnel reflectance, eta = eta_t / eta_i, cos >= 0.
// fresnel_ct takes the cosine of the transmitted direction as well.
template <class S>
__device__ __forceinline__ S fresnel_ct(const S& ci, const S& ct, float eta) {
  const S rs = (ci - eta * ct) / (ci + eta * ct);
  const S rp = (eta * ci - ct) / (eta * ci + ct);
  return 0.5f * (rs * rs + rp * rp);
}
template <class S>
__device__ __forceinline__ S fresnel(const S& ci, float eta) {
  const S s2t = (1.0f - ci * ci) * (1.0f / (eta * eta));
  if (!(vf(s2t) < 1.0f)) return S(1.f);
  return fresnel_ct(ci, xsqrt(1.0f - s2t), eta);
}
// Anisotropic GGX (Heitz 2014) in a local frame (x = t, y = b, z = n).
template <class S>
__device__ __forceinline__ S ggx_d(const V3<S>& m, float at, float ab) {
  if (!(vf(m.z) > 0.f)) return S(0.f);
  const S mx = m.x / at, my = m.y / ab;
  const S q = mx * mx + my * my + m.z * m.z;
  return S(1.0f / kPi) / (at * ab * q * q);
}
template <class S>
__device__ __forceinline__ S ggx_g1(const V3<S>& w, const S& wm, float at, float ab) {
  if (!(vf(wm) * vf(w.z) > 0.f)) return S(0.f);
  const S an = vf(w.z) < 0.f ? -w.z : w.z;
  const S ax = at * w.x, ay = ab * w.y;
  return 2.0f * an / (an + xsqrt(an * an + ax * ax + ay * ay));
}
// G1(w) / |w.z| in closed form: the lobes divide G1 of the incoming
// direction by its own cosine, which near grazing is a ratio of two small
// numbers rounded apart; the quotient is formed without them
template <class S>
__device__ __forceinline__ S ggx_g1_over_cos(const V3<S>& w, const S& wm, float at,
                                             float ab) {
  if (!(vf(wm) * vf(w.z) > 0.f)) return S(0.f);
  const S an = vf(w.z) < 0.f ? -w.z : w.z;
  const S ax = at * w.x, ay = ab * w.y;
  return 2.0f / (an + xsqrt(an * an + ax * ax + ay * ay));
}
// GGX visible-normal sample (Heitz 2018), local frame, w.z > 0; the disk
// point is (r cos phi, r sin phi) with r = sqrt(u0), phi = 2 pi u1.
template <class S>
__device__ __forceinline__ V3<S> vndf_sample(const V3<S>& w, float at, float ab, float r,
                                             float sphi, float cphi) {
  const V3<S> V = normalize(mk3<S>(at * w.x, ab * w.y, w.z));
  const S lensq = V.x * V.x + V.y * V.y;
  V3<S> T1 = lift3<S>(1.f, 0.f, 0.f);
  if (vf(lensq) > 0.f) {
    const S il = xrsqrt(lensq);
    T1 = mk3<S>(-(V.y * il), V.x * il, S(0.f));
  }
  const V3<S> T2 = cross(V, T1);
  const float t1 = r * cphi;
  const S s = 0.5f * (1.0f + V.z);
  const S t2 = (1.0f - s) * sqrtf(1.0f - t1 * t1) + s * (r * sphi);
  const S tz = xsqrt(xmax0(1.0f - t1 * t1 - t2 * t2));
  const V3<S> Nh = T1 * t1 + T2 * t2 + V * tz;
  return normalize(mk3<S>(at * Nh.x, ab * Nh.y, xmax0(Nh.z)));
}

template <class W, class S>
__device__ __forceinline__ V3<S> to_local(const V3<W>& w, const V3<S>& t, const V3<S>& b,
                                          const V3<S>& n) {
  return mk3<S>(dot(w, t), dot(w, b), dot(w, n));
}

// ---------------------------------------------------------------- shading --
template <class S>
struct Shade {
  V3<S> t, b, n, wi;
  S mui, g, fr;
  float at, ab;           // GGX roughness (no tangents: closed-form derivatives)
  bool at_free, ab_free;  // roughness not clamped (its derivative passes)
  S body_x0;  // G / (1 + a(mu_i)): f_x^B per unit r B k^B_x before its angular term
  S body_y0;  // G / pi: f_y^B per unit (1 - r) B k^B_y per unit cosine
  float ni_sy;  // N_i |x - y|: d ln tau / d sigma_t = -ni_sy
  // transmission path (f_y^S)
  bool tt_ok;
  V3<S> iy, by, ny;
  S tx, tau;
};

template <class S>
__device__ __forceinline__ S clamp_alpha(const S& a) {
  if (vf(a) < 1e-3f) return S(1e-3f);
  if (vf(a) > 1.5f) return S(1.5f);
  return a;
}

// wi: the record's incoming direction, float (no tangents) or S (seeded for
// direction tangents); sc: the stochastic estimators' state (GGX-sampled
// entry), or NULL
template <class S, class W>
__device__ __forceinline__ void make_shade(const MatDev& m, const MatVars<S>& mv,
                                           const Geo<S>& G, const V3<W>& wi, Shade<S>& s,
                                           const StochCtx* sc = nullptr) {
  s.wi = as3<S>(wi);
  s.n = G.n;
  s.t = G.t;
  s.b = cross(s.n, s.t);
  // reading: two-sided shading, the side of omega_i is outside at x
  if (vf(dot(wi, s.n)) < 0.f) {
    s.n = -s.n;
    s.b = -s.b;
  }
  s.mui = dot(wi, s.n);
  // Sec. 4.2: beta_multi = beta + (h2 - h1) / 2 (reading), GGX alpha = beta
  const float hw = 0.5f * G.width;
  s.at = clamp_alpha(mv.beta_t + hw);
  s.ab = clamp_alpha(mv.beta_b + hw);
  s.at_free = vf(s.at) == vf(mv.beta_t + hw);
  s.ab_free = vf(s.ab) == vf(mv.beta_b + hw);
  s.g = G.g;
  s.fr = fresnel(s.mui, m.eta);
  // Eq. 5: the Lommel-Seeliger + Lambert bracket divided by its albedo
  // 1 + a(mu_i), a(mu) = (1 - mu ln(1 + 1/mu)) / 2; Eq. 6: Lambert
  s.body_x0 = S(0.f);
  if (vf(s.mui) > 0.f) {
    const S aLS = 0.5f * (1.0f - s.mui * xlog(1.0f + 1.0f / s.mui));
    s.body_x0 = s.g / (1.0f + aLS);
  }
  s.body_y0 = s.g * (1.0f / kPi);
  s.ni_sy = 0.f;
  s.tt_ok = false;
  // Sec. 4.1.1 (reading): smooth refraction into the yarn at x, straight path
  // to the yarn surface y, attenuation tau^{N_i} (Eq. 4)
  // Rough entry (Eq. 1's Omega_y integral, one sample): the refracting normal
  // is a GGX visible normal m about n; the entry transmittance is
  // 1 - F(omega_i . m); a ray refracted outward carries no transmission
  V3<S> mn = s.n;
  S ci = s.mui;
  const bool rough = sc != nullptr && (sc->flags & STOCH_ROUGH_ENTRY) != 0;
  if (rough && vf(s.mui) > 0.f) {
    const U64x4 rnd = philox4x64(sc->index, 16, 0, 0, sc->seed, kStochKey1);
    const float v0 = unit24(rnd.w[0]), v1 = unit24(rnd.w[1]);
    float sphi, cphi;
    sincospif(2.0f * v1, &sphi, &cphi);
    const V3<S> ml = vndf_sample(to_local(wi, s.t, s.b, s.n), s.at, s.ab, sqrtf(v0), sphi, cphi);
    mn = s.t * ml.x + s.b * ml.y + s.n * ml.z;
    ci = dot(wi, mn);
  }
  const S s2t = (1.0f - ci * ci) * (m.inv_eta * m.inv_eta);
  if (!(vf(s.mui) > 0.f) || !(vf(ci) > 0.f) || !(vf(s2t) < 1.0f)) return;
  const S ct = xsqrt(1.0f - s2t);
  const V3<S> din = wi * (-m.inv_eta) + mn * (ci * m.inv_eta - ct);
  if (rough && !(vf(dot(din, s.n)) < 0.f)) return;
  const S a = din.x * din.x + din.y * din.y;
  if (!(vf(a) > 1e-12f)) return;
  const S bq = G.x.x * din.x + G.x.y * din.y;
  const S c = G.x.x * G.x.x + G.x.y * G.x.y - m.R * m.R;
  const S disc = xmax0(bq * bq - a * c);
  const S sy = xmax0((xsqrt(disc) - bq) / a);
  const S yx = G.x.x + din.x * sy, yy = G.x.y + din.y * sy;
  const S il = xrsqrt(yx * yx + yy * yy);
  s.ny = mk3<S>(yx * il, yy * il, S(0.f));
  s.by = mk3<S>(s.ny.y, -s.ny.x, S(0.f));  // n_y x z
  s.iy = -din;
  s.tau = xexp(-(m.sigma_t * G.ni * sy));
  s.ni_sy = vf(G.ni) * vf(sy);
  s.tx = 1.0f - (rough ? fresnel(ci, m.eta) : s.fr);
  s.tt_ok = true;
}
template <class S>
__device__ __forceinline__ void make_shade(const MatDev& m, const MatVars<S>& mv,
                                           const Geo<S>& G, const Record& q, Shade<S>& s) {
  make_shade(m, mv, G, mk3<float>(q.wi[0], q.wi[1], q.wi[2]), s);
}

// f |wo.n| of the four lobes at wo; spec = f_x^S + f_y^S (grey), body = the
// body lobe per unit colour (k^B_x if refl, else k^B_y); pdf terms of the four
// sampling strategies.  spec_u = spec / k^S and body_w = body / (r B) (refl)
// or body / ((1 - r) B) carry the closed-form derivatives in k_spec, B, r.
template <class S>
struct LobeVals {
  S spec, body, pR, pT, pxb, pyb;
  S spec_u, body_w;
  bool refl;
};

template <class S>
__device__ __forceinline__ V3<S> vsel(bool c, const V3<S>& a, const V3<S>& b) {
  return c ? a : b;
}

// Closed-form d ln / d alpha of GGX D and Smith G1 (local frames, values).
__device__ __forceinline__ void dln_ggx_d(float hx, float hy, float hz, float at, float ab,
                                          float* dt, float* db) {
  const float q = hx * hx / (at * at) + hy * hy / (ab * ab) + hz * hz;
  *dt = -1.0f / at + 4.0f * hx * hx / (at * at * at * q);
  *db = -1.0f / ab + 4.0f * hy * hy / (ab * ab * ab * q);
}
__device__ __forceinline__ void dln_ggx_g1(float wx, float wy, float wz, float at, float ab,
                                           float* dt, float* db) {
  const float an = fabsf(wz);
  const float r = sqrtf(an * an + at * at * wx * wx + ab * ab * wy * wy);
  const float k = 1.0f / (r * (an + r));
  *dt = -at * wx * wx * k;
  *db = -ab * wy * wy * k;
}

// wo: float (no tangents) or S (seeded for direction tangents)
template <class S, class W>
__device__ __forceinline__ void eval_lobes(const MatDev& m, const Shade<S>& s, const V3<W>& wo,
                                           LobeVals<S>& L, float* dln_alpha = nullptr) {
  L.spec = S(0.f);
  L.body = S(0.f);
  L.pR = S(0.f);
  L.pT = S(0.f);
  L.pxb = S(0.f);
  L.pyb = S(0.f);
  L.spec_u = S(0.f);
  L.body_w = S(0.f);
  L.refl = true;
  if (!(vf(s.mui) > 0.f)) return;
  const S muo = dot(wo, s.n);
  const bool refl = vf(muo) > 0.f;
  L.refl = refl;
  if (!refl && !(vf(muo) < 0.f)) return;
  // Eqs. 5-6: body lobes, per unit colour
  if (refl) {
    L.body_w = s.body_x0 * (S(1.0f / (4.0f * kPi)) / (s.mui + muo) + 1.0f / kPi) * muo;
    L.body = (m.r * m.B) * L.body_w;
    L.pxb = muo * (1.0f / kPi);
  } else {
    L.body_w = s.body_y0 * (-muo);
    L.body = ((1.0f - m.r) * m.B) * L.body_w;
    L.pyb = -muo * (1.0f / kPi);
  }
  // Eq. 2 (reflection at x, Walter et al. 2007 with GGX) and Eq. 3 (exit BTDF
  // at y from inside (eta) to outside (1), times the entry transmittance and
  // tau^{N_i}) share one microfacet evaluation: GGX D at the half vector,
  // Smith G1 of both directions, Fresnel -- in the frame of the lobe that
  // applies to this omega_o
  S ion = S(0.f);
  if (!refl) {
    if (!s.tt_ok) return;
    ion = dot(s.iy, s.ny);
    const S oon = dot(wo, s.ny);
    if (!(vf(ion) < 0.f && vf(oon) > 0.f)) return;
  }
  const V3<S> fz = lift3<S>(0.f, 0.f, 1.f);
  const V3<S> fn = vsel(refl, s.n, s.ny);
  const V3<S> ft = vsel(refl, s.t, fz);
  const V3<S> fb = vsel(refl, s.b, s.by);
  const V3<S> vi = vsel(refl, s.wi, s.iy);
  V3<S> h = normalize(refl ? s.wi + wo : -(s.iy * m.eta + wo));
  if (vf(dot(h, fn)) < 0.f) h = -h;
  const S ih = dot(vi, h), oh = dot(wo, h);
  if (!refl && !(vf(ih) < 0.f && vf(oh) > 0.f)) return;
  const V3<S> hl = to_local(h, ft, fb, fn), il = to_local(vi, ft, fb, fn),
              ol = to_local(wo, ft, fb, fn);
  const S D = ggx_d(hl, s.at, s.ab);
  const S g1i_c = ggx_g1_over_cos(il, ih, s.at, s.ab);  // G1(i) / |i.n|
  const S g1o = ggx_g1(ol, oh, s.at, s.ab);
  if (dln_alpha) {
    // the specular value is a product with D, G1(i), G1(o): its log
    // derivative in the roughness is the sum of theirs
    const float at = vf(s.at), ab = vf(s.ab);
    float a0, a1, b0, b1, c0, c1;
    dln_ggx_d(vf(hl.x), vf(hl.y), vf(hl.z), at, ab, &a0, &a1);
    dln_ggx_g1(vf(il.x), vf(il.y), vf(il.z), at, ab, &b0, &b1);
    dln_ggx_g1(vf(ol.x), vf(ol.y), vf(ol.z), at, ab, &c0, &c1);
    dln_alpha[0] = a0 + b0 + c0;
    dln_alpha[1] = a1 + b1 + c1;
  }
  // at the exit the generalised half vector of two unit vectors gives
  // eta^2 (1 - (i.h)^2) = 1 - (o.h)^2 exactly, so the float path takes o.h as
  // the transmitted cosine (no cancellation next to total internal
  // reflection); dual numbers keep the general form, whose partial
  // derivatives in omega_o's components also hold off the unit sphere
  S F;
  if (refl) {
    F = fresnel(ih, m.eta);
  } else if constexpr (is_dual<S>::value) {
    F = fresnel(-ih, m.inv_eta);
  } else {
    F = fresnel_ct(-ih, oh, m.inv_eta);
  }
  if (refl) {
    const S q = g1i_c * D * 0.25f;
    L.spec_u = F * g1o * q;
    L.pR = q;
  } else {
    const S den = m.eta * ih + oh;
    const S q = g1i_c * (-ih) * D * oh / (den * den);
    L.spec_u = s.tx * s.tau * (1.0f - F) * g1o * q;
    L.pT = q;
  }
  L.spec = m.ks * L.spec_u;
}

// Sec. 4.1.5: lobe probabilities (1 - B) F(mu_i), (1 - B)(1 - F), B r, B (1 - r).
template <class S>
__device__ __forceinline__ S total_pdf(const MatDev& m, const Shade<S>& s, const LobeVals<S>& L) {
  const S PR = (1.0f - m.B) * s.fr;
  const S PT = (1.0f - m.B) - PR;
  return PR * L.pR + PT * L.pT + (m.B * m.r) * L.pxb + (m.B * (1.0f - m.r)) * L.pyb;
}

// Draw wo (Sec. 4.1.5).  Returns false when the sample leaves the lobe.
__device__ __forceinline__ bool sample_dir(const MatDev& m, const Shade<float>& s, float u0,
                                           float u1, V3<float>* wo, int* lobe) {
  const float P[4] = {(1.0f - m.B) * s.fr, (1.0f - m.B) * (1.0f - s.fr), m.B * m.r,
                      m.B * (1.0f - m.r)};
  int k = 3;
  float lo = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (k == 3 && u0 < lo + P[j]) {
      k = j;
    } else if (k == 3) {
      lo += P[j];
    }
  }
  *lobe = k;
  float ur = P[k] > 0.f ? (u0 - lo) / P[k] : 0.f;
  ur = fminf(fmaxf(ur, 0.0f), 0.99999994f);
  // both samplers map (ur, u1) to the unit disk the same way
  float sphi, cphi;
  sincospif(2.0f * u1, &sphi, &cphi);
  const float r = sqrtf(ur);
  if (k <= 1) {
    // GGX visible normals (Heitz 2018): about n at x for reflection, about
    // the inner normal at y for transmission -- one sampler, frame per lane
    const bool refl = k == 0;
    if (!refl && !s.tt_ok) return false;
    const V3<float> N = refl ? s.n : -s.ny;
    const V3<float> T = refl ? s.t : mk3<float>(0.f, 0.f, 1.f);
    const V3<float> B = refl ? s.b : cross(N, T);
    const V3<float> view = refl ? s.wi : s.iy;
    const V3<float> ml = vndf_sample(to_local(view, T, B, N), s.at, s.ab, r, sphi, cphi);
    const V3<float> mw = T * ml.x + B * ml.y + N * ml.z;
    const float c = dot(view, mw);
    if (refl) {
      *wo = mw * (2.0f * c) - s.wi;
      return dot(*wo, s.n) > 0.f;
    }
    const float s2t = m.eta * m.eta * (1.0f - c * c);
    if (!(c > 0.f) || !(s2t < 1.0f)) return false;
    *wo = normalize(s.iy * (-m.eta) + mw * (m.eta * c - sqrtf(1.0f - s2t)));
    return dot(*wo, s.ny) > 0.f && dot(*wo, s.n) < 0.f;
  }
  const float zc = sqrtf(fmaxf(0.f, 1.0f - ur)) * (k == 2 ? 1.0f : -1.0f);
  *wo = s.t * (r * cphi) + s.b * (r * sphi) + s.n * zc;
  return true;
}

}  // namespace bysdf
