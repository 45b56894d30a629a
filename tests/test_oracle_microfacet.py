"""Pins of the oracle's microfacet building blocks (Sec. 4.1.2: rough
dielectric BSDF with GGX, Fresnel, uncorrelated Smith G2) against textbook
identities, evaluated by quadrature, and of the whole BYSDF chain against
closed-form worked examples (tests/golden/closed_forms.json)."""
import json
import math
import os

import numpy as np
import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def _hemisphere_grid(n_t=400, n_p=400):
    # midpoint rule in (s, phi) with theta = (pi/2) s^2, which packs nodes near
    # the pole where narrow lobes peak: d omega = sin(theta) pi s ds dphi
    s = (np.arange(n_t) + 0.5) / n_t
    th = 0.5 * math.pi * s * s
    p = (np.arange(n_p) + 0.5) / n_p * 2 * math.pi
    T, P = np.meshgrid(th, p, indexing="ij")
    W = np.meshgrid(np.sin(th) * math.pi * s / n_t, p, indexing="ij")[0] * (2 * math.pi / n_p)
    dirs = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    return dirs, W.reshape(-1)


def test_fresnel_normal_incidence_and_tir(orc):
    for eta, want in GOLD["fresnel_normal"].items():
        assert orc.fresnel(1.0, float(eta)) == pytest.approx(want, rel=1e-14)
    # exit interface (1.55 -> 1): total internal reflection beyond asin(1/eta)
    crit = math.radians(GOLD["critical_angle_deg_1.55"])
    assert orc.fresnel(math.cos(crit + 1e-6), 1 / 1.55) == 1.0
    assert orc.fresnel(math.cos(crit - 1e-3), 1 / 1.55) < 1.0
    assert orc.fresnel(math.cos(crit - 1e-9), 1 / 1.55) == pytest.approx(1.0, abs=1e-3)
    # grazing incidence reflects everything
    assert orc.fresnel(1e-9, 1.55) == pytest.approx(1.0, abs=1e-6)


@pytest.mark.parametrize("eta", [1.33, 1.55, 2.0, 1 / 1.55])
def test_fresnel_matches_angle_form(orc, eta):
    # Fresnel equations written with angles (Hecht): a different closed form
    for ti in np.linspace(0.05, 1.5, 30):
        st = math.sin(ti) / eta
        if st >= 1:
            continue
        tt = math.asin(st)
        rs = math.sin(ti - tt) ** 2 / math.sin(ti + tt) ** 2
        rp = math.tan(ti - tt) ** 2 / math.tan(ti + tt) ** 2
        assert orc.fresnel(math.cos(ti), eta) == pytest.approx(0.5 * (rs + rp), rel=1e-10)


@pytest.mark.parametrize("at,ab", [(0.1, 0.1), (0.3, 0.3), (0.1, 0.4), (0.8, 0.25)])
def test_ggx_normalisation(orc, at, ab):
    # projected-area normalisation of the NDF: int D(m) (m.n) dm = 1
    dirs, dw = _hemisphere_grid(1200, 240)
    d = np.array([orc.ggx_d(m, at, ab) for m in dirs])
    assert (d * dirs[:, 2] * dw).sum() == pytest.approx(1.0, abs=1e-4)


def test_ggx_g1_isotropic_angle_form(orc):
    # isotropic Smith G1 (Walter et al. 2007): 2 / (1 + sqrt(1 + a^2 tan^2))
    for a in (0.05, 0.2, 0.7):
        for th in np.linspace(0.0, 1.5, 16):
            w = np.array([math.sin(th), 0.0, math.cos(th)])
            want = 2.0 / (1.0 + math.sqrt(1.0 + a * a * math.tan(th) ** 2))
            assert orc.ggx_g1(w, [0, 0, 1], a, a) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("at,ab", [(0.15, 0.15), (0.1, 0.5)])
def test_visible_normal_identities(orc, at, ab):
    # projected-area identity int G1(w,m) <w,m>+ D(m) dm = w.n, i.e. the VNDF
    # integrates to one (Heitz 2014 / 2018)
    dirs, dw = _hemisphere_grid(1200, 240)
    for th, ph in ((0.3, 0.4), (1.0, 2.0), (1.4, -0.7)):
        w = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        s = sum(orc.vndf_pdf(w, m, at, ab) * q for m, q in zip(dirs, dw))
        assert s == pytest.approx(1.0, abs=1e-4)


def test_vndf_sampler_matches_its_density(orc):
    # the VNDF sampler's histogram over (cos, phi) bins follows the VNDF pdf
    at, ab = 0.3, 0.15
    w = np.array([math.sin(0.9) * math.cos(0.5), math.sin(0.9) * math.sin(0.5), math.cos(0.9)])
    rng = np.random.default_rng(3)
    n = 60000
    u = rng.random((n, 2))
    ms = np.array([orc.vndf_sample(w, at, ab, a, b) for a, b in u])
    assert np.allclose(np.linalg.norm(ms, axis=1), 1.0, atol=1e-12)
    nb_c, nb_p = 8, 8
    ci = np.minimum((ms[:, 2] * nb_c).astype(int), nb_c - 1)
    pi = (np.mod(np.arctan2(ms[:, 1], ms[:, 0]), 2 * math.pi) / (2 * math.pi) * nb_p).astype(int)
    pi = np.minimum(pi, nb_p - 1)
    hist = np.zeros((nb_c, nb_p))
    np.add.at(hist, (ci, pi), 1)
    dirs, dw = _hemisphere_grid(400, 400)
    pd = np.array([orc.vndf_pdf(w, m, at, ab) for m in dirs]) * dw
    dci = np.minimum((dirs[:, 2] * nb_c).astype(int), nb_c - 1)
    dpi = np.minimum((np.mod(np.arctan2(dirs[:, 1], dirs[:, 0]), 2 * math.pi)
                      / (2 * math.pi) * nb_p).astype(int), nb_p - 1)
    exp = np.zeros((nb_c, nb_p))
    np.add.at(exp, (dci, dpi), pd)
    exp *= n
    m = exp > 20
    chi2 = (((hist - exp) ** 2)[m] / exp[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_btdf_generalised_reciprocity(orc):
    # Walter et al. 2007: f_t(i,o) / eta_o^2 = f_t(o,i) / eta_i^2
    rng = np.random.default_rng(5)
    n_ok = 0
    for _ in range(300):
        i = rng.normal(size=3); i /= np.linalg.norm(i); i[2] = -abs(i[2])
        o = rng.normal(size=3); o /= np.linalg.norm(o); o[2] = abs(o[2])
        a = orc.btdf(i, o, 1.55, 1.0, 0.3, 0.2)
        b = orc.btdf(o, i, 1.0, 1.55, 0.3, 0.2)
        if a > 0:
            n_ok += 1
        assert a / 1.0 ** 2 == pytest.approx(b / 1.55 ** 2, rel=1e-10, abs=1e-300)
    assert n_ok > 50


def _worked(orc):
    mat = GOLD["worked_material"]
    rec0 = GOLD["worked_record"]
    cases = GOLD["worked_cases"]
    n = len(cases)
    rec = dict(h=np.full(n, rec0["h"], np.float32), u=np.full(n, rec0["u"], np.float32),
               v=np.full(n, rec0["v"], np.float32),
               wi=np.array([c["wi"] for c in cases], np.float32).T.copy(),
               wo=np.array([c["wo"] for c in cases], np.float32).T.copy(),
               mat_id=np.zeros(n, np.int32),
               ratio=np.array([c.get("ratio", 0.0) for c in cases], np.float32))
    return mat, rec, cases


def test_worked_examples_eval_and_pdf(orc):
    mat, rec, cases = _worked(orc)
    f, pdf, st = orc.eval_records([mat], rec)
    assert (st == 0).all()
    for j, c in enumerate(cases):
        np.testing.assert_allclose(f[:, j], c["f"], rtol=1e-6, err_msg=c["name"])
        assert pdf[j] == pytest.approx(c["pdf"], rel=1e-6), c["name"]


def test_attenuation_power_of_plies_crossed(orc):
    # Eq. 4 with the N_i exponent: tau^{N_i} = exp(-sigma_t N_i |x - y|); on the
    # head-on single-ply geometry the internal chord is the yarn diameter 2R
    mat = dict(GOLD["worked_material"])
    frame = [0, 0, 1, 0, -1, 0, 1, 0, 0]      # t = z, b = n x t, n = x
    x = [1.0, 0.0, 0.0]
    wi, wo = [1.0, 0.0, 0.0], [-1.0, 0.0, 0.0]
    tt = [orc.lobes(mat, frame, x, 1.0, ni, 0.0, wi, wo)["TT"] for ni in (0.0, 1.0, 2.5)]
    sig = float(np.float32(mat["sigma_t"]))
    assert tt[1] / tt[0] == pytest.approx(math.exp(-sig * 2.0), rel=1e-12)
    assert tt[2] / tt[0] == pytest.approx(math.exp(-sig * 2.5 * 2.0), rel=1e-12)
