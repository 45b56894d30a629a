"""Writes closed_forms.json: textbook values the oracle must reproduce.

The paper prints no per-evaluation value, so these fixtures are closed forms of
special cases, derived by hand from the definitions and evaluated here with
plain `math` (this script imports neither the oracle nor the CUDA path):

* Fresnel reflectance at normal incidence ((eta-1)/(eta+1))^2 and the critical
  angle asin(1/eta) of the exit interface (Sec. 4.1.2, Eqs. 2-3, F).
* Inscribed ply layout (reading of Sec. 3.4): N_p discs touching the yarn
  circle and each other: R_c + R_p = R, R_c sin(pi/N_p) = R_p.
* Worked BYSDF values (Eqs. 2, 3, 5, 6) for a one-ply yarn without fiber
  detail, seen head-on (h = 0, omega_i along the yarn normal), where the
  geometry collapses to a flat GGX interface with normal n_u.

Run:  python tests/golden/make_closed_forms.py
"""
import json
import math
import os

out = {}
out["fresnel_normal"] = {str(e): ((e - 1) / (e + 1)) ** 2 for e in (1.33, 1.5, 1.55, 2.0)}
out["critical_angle_deg_1.55"] = math.degrees(math.asin(1 / 1.55))

lay = {}
for n in range(2, 6):
    s = math.sin(math.pi / n)
    rc = 1.0 / (1.0 + s)
    lay[str(n)] = {"Rp": rc * s, "Rc": rc}
out["ply_layout_R1"] = lay

# worked examples: material (float32-exact values)
eta, beta_deg, B, r, ks, sig_t = 1.5, 10.0, 0.5, 0.5, 1.0, 0.5
alb = [0.25, 0.5, 0.75]
a = math.radians(beta_deg)
F0 = ((eta - 1) / (eta + 1)) ** 2
kS = (1 - B) * ks


def ggx_d_iso(cos_m, alpha):
    t2 = (1 - cos_m ** 2) / cos_m ** 2
    return 1.0 / (math.pi * alpha ** 2 * cos_m ** 4 * (1 + t2 / alpha ** 2) ** 2)


def g1_iso(cos_w, alpha):   # Walter et al. 2007, GGX Smith G1 in angle form
    t2 = (1 - cos_w ** 2) / cos_w ** 2
    return 2.0 / (1.0 + math.sqrt(1.0 + alpha ** 2 * t2))


def fresnel_angles(ti, eta):  # Fresnel equations in angle form (Hecht)
    if ti == 0.0:
        return ((eta - 1) / (eta + 1)) ** 2
    tt = math.asin(math.sin(ti) / eta)
    rs = math.sin(ti - tt) ** 2 / math.sin(ti + tt) ** 2
    rp = math.tan(ti - tt) ** 2 / math.tan(ti + tt) ** 2
    return 0.5 * (rs + rp)


def body_x(mu_i, mu_o, k):
    a_ls = 0.5 * (1 - mu_i * math.log(1 + 1 / mu_i))
    return r * B * k * (1 / (4 * math.pi * (mu_i + mu_o)) + 1 / math.pi) / (1 + a_ls) * mu_o


cases = []
# (1) retro-reflection along the normal: R lobe at the NDF peak + backward body
fR = kS * F0 * ggx_d_iso(1.0, a) / 4.0
pdf = (1 - B) * F0 * ggx_d_iso(1.0, a) / 4.0 + B * r / math.pi
cases.append({"name": "retro", "wi": [1, 0, 0], "wo": [1, 0, 0],
              "f": [fR + body_x(1.0, 1.0, k) for k in alb], "pdf": pdf})
# (2) off-specular reflection in the cross-section plane, theta_o = 50 deg
th = math.radians(50.0)
wo = [math.cos(th), math.sin(th), 0.0]
half = th / 2
fR = kS * fresnel_angles(half, eta) * g1_iso(1.0, a) * g1_iso(math.cos(th), a) * \
    ggx_d_iso(math.cos(half), a) / 4.0
pdfR = g1_iso(1.0, a) * ggx_d_iso(math.cos(half), a) / 4.0
pdf = (1 - B) * F0 * pdfR + B * r * math.cos(th) / math.pi
cases.append({"name": "off_specular_50", "wi": [1, 0, 0], "wo": wo,
              "f": [fR + body_x(1.0, math.cos(th), k) for k in alb], "pdf": pdf})
# (3) straight transmission through the yarn (chord 2R, one ply crossed)
tau = math.exp(-sig_t * 1 * 2.0)
fT = kS * (1 - F0) * tau * (1 - F0) * ggx_d_iso(1.0, a) / (eta - 1) ** 2
pdfT = ggx_d_iso(1.0, a) / (eta - 1) ** 2
pdf = (1 - B) * (1 - F0) * pdfT + B * (1 - r) / math.pi
cases.append({"name": "straight_through", "wi": [1, 0, 0], "wo": [-1, 0, 0],
              "f": [fT + (1 - r) * B * k / math.pi for k in alb], "pdf": pdf})
# (4) oblique exit: the internal ray leaves y along the normal's reverse and
# refracts out at theta_o = 30 deg (exit BTDF from eta to 1, Walter et al.)
th = math.radians(30.0)
H = math.sqrt(eta * eta - 2 * eta * math.cos(th) + 1)
cos_m = (eta - math.cos(th)) / H          # microfacet normal vs exit normal
ih, oh = cos_m, (eta * math.cos(th) - 1) / H
ti = math.acos(ih)                        # incidence angle inside, on the facet
tt = math.asin(math.sin(ti) * eta)        # refraction angle outside
Fy = 0.5 * (math.sin(ti - tt) ** 2 / math.sin(ti + tt) ** 2 +
            math.tan(ti - tt) ** 2 / math.tan(ti + tt) ** 2)
D = ggx_d_iso(cos_m, a)
fT = kS * (1 - F0) * tau * ih * oh * (1 - Fy) * g1_iso(math.cos(th), a) * D / H ** 2
pdfT = ih * D * oh / H ** 2
wo = [-math.cos(th), math.sin(th), 0.0]
pdf = (1 - B) * (1 - F0) * pdfT + B * (1 - r) * math.cos(th) / math.pi
cases.append({"name": "oblique_exit_30", "wi": [1, 0, 0], "wo": wo,
              "f": [fT + (1 - r) * B * k / math.pi * math.cos(th) for k in alb], "pdf": pdf})
# (5, 6) footprints symmetric about h0 = 0: by symmetry the aggregated normal
# stays n_u, and the roughness grows to beta + (h2 - h1)/2 (Sec. 4.2 reading)
for name, ratio in (("multi_retro_0.5", 0.5), ("far_retro", 100.0)):
    width = min(ratio, 1.0) * 2
    a_m = a + width / 2
    fR = kS * F0 * ggx_d_iso(1.0, a_m) / 4.0
    pdf = (1 - B) * F0 * ggx_d_iso(1.0, a_m) / 4.0 + B * r / math.pi
    cases.append({"name": name, "wi": [1, 0, 0], "wo": [1, 0, 0], "ratio": ratio,
                  "f": [fR + body_x(1.0, 1.0, k) for k in alb], "pdf": pdf})
out["worked_material"] = dict(n_plies=1, fibers_per_ply=64, map_texels=256, trace_iters=5,
                              k_max=16, flags=1, yarn_radius=1.0, ply_twist_deg=0.0,
                              fiber_twist_deg=0.0, eta=eta, albedo=alb, k_spec=ks,
                              beta_deg=[beta_deg, beta_deg], body_B=B, body_r=r,
                              sigma_t=sig_t, shadow_density=0.0, packing=0.8)
out["worked_record"] = {"h": 0.0, "u": 0.0, "v": 3.0}
out["worked_cases"] = cases

path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "closed_forms.json")
with open(path, "w") as fh:
    json.dump(out, fh, indent=1)
print("wrote", path)
