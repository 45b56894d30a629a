"""Pins of the oracle's implicit geometry (Sec. 3.4 implicit plies, Sec. 3.5
implicit fibers, Sec. 4.1.4 shadowing) against brute force on explicit ply
helices and fiber circles, closed forms and invariants."""
import json
import math
import os

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def mat(**kw):
    return I.material(**kw)


# ------------------------------------------------------------------- layout --
@pytest.mark.parametrize("n_p", [2, 3, 4, 5])
def test_ply_layout_inscribed(orc, n_p):
    L = orc.layout(mat(n_plies=n_p))
    g = GOLD["ply_layout_R1"][str(n_p)]
    assert L["Rp"] == pytest.approx(g["Rp"], rel=1e-14)
    assert L["Rc"] == pytest.approx(g["Rc"], rel=1e-14)
    # invariants: plies touch the yarn circle and their neighbours
    assert L["Rc"] + L["Rp"] == pytest.approx(1.0, rel=1e-14)
    gap = 2 * L["Rc"] * math.sin(math.pi / n_p)
    assert gap == pytest.approx(2 * L["Rp"], rel=1e-12)


@pytest.mark.parametrize("n_f", [32, 64, 100, 128])
def test_fiber_ring_closes(orc, n_f):
    L = orc.layout(mat(fibers_per_ply=n_f))
    # packing: N_f fibers of radius r_f fill 80% of the ply disc
    pk = float(np.float32(0.8))   # descriptors are float32
    assert n_f * L["rf"] ** 2 == pytest.approx(pk * L["Rp"] ** 2, rel=1e-12)
    assert L["Rfc"] + L["rf"] == pytest.approx(L["Rp"], rel=1e-14)
    # M is the fewest fibers whose circles close the ring: neighbours at angle
    # 2 pi / M overlap (or touch), with M - 1 they would leave a gap
    half = math.asin(L["rf"] / L["Rfc"])
    M = L["M"]
    assert math.pi / M <= half + 1e-15
    assert math.pi / (M - 1) > half
    assert (n_f, M) in ((32, 17), (64, 25), (100, 32), (128, 37))


def test_helix_rates(orc):
    m = mat(n_plies=4, ply_twist_deg=25.0, fiber_twist_deg=35.0)
    L = orc.layout(m)
    # helix at radius R_c with helix angle alpha: d(psi)/dz R_c = tan(alpha)
    assert L["omega_p"] * L["Rc"] == pytest.approx(math.tan(math.radians(25.0)), rel=1e-6)
    assert L["omega_f"] * L["Rfc"] == pytest.approx(math.tan(math.radians(35.0)), rel=1e-6)
    assert orc.layout(mat(n_plies=1))["omega_p"] == 0.0


# -------------------------------------------------------------- ply trace --
def consistent_wi(h, u, wz):
    """omega_i whose in-plane part points back along the entering ray."""
    g = math.asin(h)
    L = math.sqrt(1 - wz * wz)
    return np.array([L * math.cos(u - g), L * math.sin(u - g), wz], np.float32)


def helix_centre(L, k, n_p, z):
    psi = 2 * math.pi * k / n_p + L["omega_p"] * z
    return np.array([L["Rc"] * math.cos(psi), L["Rc"] * math.sin(psi)])


def brute_crossings(m, h, u, v, wi, step=2e-4):
    """Per ply, the first in-plane distance t at which the camera ray enters
    the ply tube (disc of radius R_p about the explicit helix centre in the
    yarn-perpendicular plane at the ray's height), or None; by marching along
    the chord and bisection."""
    import oracle as orc
    L = orc.layout(m)
    n_p = m["n_plies"]
    wi = np.asarray(wi, np.float64)
    g = math.asin(h)
    X0 = np.array([math.cos(u), math.sin(u)])
    e = -np.array([math.cos(u - g), math.sin(u - g)])
    kap = -wi[2] / math.hypot(wi[0], wi[1])
    chord = 2 * math.cos(g)
    t = np.arange(0, chord + step, step)
    out = []
    for k in range(n_p):
        z = v + kap * t
        psi = 2 * math.pi * k / n_p + L["omega_p"] * z
        dx = X0[0] + t * e[0] - L["Rc"] * np.cos(psi)
        dy = X0[1] + t * e[1] - L["Rc"] * np.sin(psi)
        F = np.hypot(dx, dy) - L["Rp"]
        idx = np.nonzero(F <= 0)[0]
        if len(idx) == 0:
            out.append(None)
            continue
        i = idx[0]
        if i == 0:
            out.append(0.0)
            continue
        lo, hi = t[i - 1], t[i]

        def Fk(tt):
            c = helix_centre(L, k, n_p, v + kap * tt)
            return math.hypot(X0[0] + tt * e[0] - c[0], X0[1] + tt * e[1] - c[1]) - L["Rp"]
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if Fk(mid) > 0:
                lo = mid
            else:
                hi = mid
        out.append(0.5 * (lo + hi))
    return out


def brute_first_hit(m, h, u, v, wi, step=2e-4):
    cr = brute_crossings(m, h, u, v, wi, step)
    hits = [(t, k) for k, t in enumerate(cr) if t is not None]
    return min(hits) if hits else None


def test_untwisted_plies_closed_form(orc):
    # alpha_p = 0: ply centres do not move along z, one cross-section update is
    # exact and equals the 2D ray/circle intersection
    m1 = mat(n_plies=4, ply_twist_deg=0.0, trace_iters=1)
    m5 = mat(n_plies=4, ply_twist_deg=0.0, trace_iters=5)
    L = orc.layout(m1)
    rng = np.random.default_rng(1)
    for _ in range(200):
        h, u, v = rng.uniform(-1, 1), rng.uniform(0, 6.28), rng.uniform(0, 100)
        h, u, v = float(np.float32(h)), float(np.float32(u)), float(np.float32(v))
        wi = consistent_wi(h, u, rng.uniform(-0.9, 0.9))
        g1 = orc.geometry(m1, h, u, v, wi)
        g5 = orc.geometry(m5, h, u, v, wi)
        assert np.array_equal(g1["t_ply"], g5["t_ply"])
        g = math.asin(h)
        X0 = np.array([math.cos(u), math.sin(u)])
        e = -np.array([math.cos(u - g), math.sin(u - g)])
        for k in range(4):
            c = helix_centre(L, k, 4, 0.0)
            q = X0 - c
            b = q @ e
            disc = b * b - (q @ q - L["Rp"] ** 2)
            if disc < 0:
                assert g1["t_ply"][k] == -1.0
            else:
                assert g1["t_ply"][k] == pytest.approx(max(-b - math.sqrt(disc), 0.0), abs=1e-12)


def test_perpendicular_ray_one_step(orc):
    # omega_i perpendicular to the yarn: the ray stays in one cross-section
    m1 = mat(n_plies=3, trace_iters=1)
    m8 = mat(n_plies=3, trace_iters=8)
    rng = np.random.default_rng(2)
    for _ in range(100):
        h, u, v = (float(np.float32(x)) for x in (rng.uniform(-1, 1), rng.uniform(0, 6.28),
                                                    rng.uniform(0, 100)))
        wi = consistent_wi(h, u, 0.0)
        a = orc.geometry(m1, h, u, v, wi)
        b = orc.geometry(m8, h, u, v, wi)
        np.testing.assert_allclose(a["t_ply"], b["t_ply"], atol=1e-13)


def test_trace_matches_brute_force_march(orc):
    # a converged implicit trace is the first entry into the explicit helix
    # tube, ply by ply, for moderately oblique consistent rays; where every
    # ply agrees, N_i is the number of tubes the straight chord crosses
    m = mat(n_plies=3, ply_twist_deg=30.0, trace_iters=64)
    L = orc.layout(m)
    rng = np.random.default_rng(3)
    agree = total = full = 0
    for _ in range(150):
        h, u, v = (float(np.float32(x)) for x in (rng.uniform(-0.95, 0.95),
                                                    rng.uniform(0, 6.28), rng.uniform(0, 100)))
        wi = consistent_wi(h, u, rng.uniform(-0.45, 0.45))
        g = orc.geometry(m, h, u, v, wi)
        cr = brute_crossings(m, h, u, v, wi)
        ok_all = True
        for k in range(3):
            total += 1
            tk = g["t_ply"][k]
            if cr[k] is None:
                good = tk == -1.0
            else:
                good = tk >= 0 and abs(tk - cr[k]) < 1e-9
            agree += good
            ok_all &= good
        if not ok_all:
            continue
        full += 1
        crossed = sum(c is not None for c in cr)
        if crossed == 0:
            assert g["status"] == 1
            continue
        assert g["ni_mean"] == crossed
        first = min((c, k) for k, c in enumerate(cr) if c is not None)
        assert g["ply"] == first[1]
        # residual invariant at convergence: the hit lies on its ply tube
        c = helix_centre(L, g["ply"], 3, g["x"][2])
        assert abs(math.hypot(g["x"][0] - c[0], g["x"][1] - c[1]) - L["Rp"]) < 1e-12
    assert agree >= 0.95 * total, (agree, total)
    assert full >= 0.85 * 150, full


def test_elliptical_beats_circular_at_oblique_view(orc):
    # Sec. 3.4: at oblique views the cross-section at the yarn hit (one update,
    # "circular") misplaces the ply hit; iterating ("elliptical") fixes it
    m_c = mat(n_plies=3, ply_twist_deg=30.0, trace_iters=1)
    m_e = mat(n_plies=3, ply_twist_deg=30.0, trace_iters=5)
    rng = np.random.default_rng(4)
    err_c, err_e = [], []
    wz = math.cos(math.radians(60.0))   # ray 60 degrees off the yarn normal plane
    for _ in range(120):
        h, u, v = (float(np.float32(x)) for x in (rng.uniform(-0.9, 0.9),
                                                    rng.uniform(0, 6.28), rng.uniform(0, 100)))
        wi = consistent_wi(h, u, wz * rng.choice([-1, 1]))
        bf = brute_first_hit(m_e, h, u, v, wi)
        gc = orc.geometry(m_c, h, u, v, wi)
        ge = orc.geometry(m_e, h, u, v, wi)
        if bf is None or gc["status"] or ge["status"]:
            continue
        err_c.append(abs(gc["t_ply"][gc["ply"]] - bf[0]))
        err_e.append(abs(ge["t_ply"][ge["ply"]] - bf[0]))
    assert len(err_c) > 50
    assert np.median(err_e) < 0.2 * np.median(err_c)


def test_single_ply_hits_at_yarn_surface(orc):
    m = mat(n_plies=1, flags=1)
    g = orc.geometry(m, 0.3, 1.0, 5.0, consistent_wi(0.3, 1.0, 0.2))
    assert g["status"] == 0 and g["t_ply"][0] == pytest.approx(0.0, abs=1e-12)
    np.testing.assert_allclose(g["n_p"], [math.cos(1.0), math.sin(1.0), 0.0], atol=1e-12)
    np.testing.assert_allclose(g["t_p"], [0, 0, 1], atol=1e-12)


def test_frames_orthonormal(orc):
    m = mat(n_plies=4, ply_twist_deg=40.0, fiber_twist_deg=30.0)
    rng = np.random.default_rng(6)
    n = 0
    for _ in range(100):
        h, u, v = rng.uniform(-1, 1), rng.uniform(0, 6.28), rng.uniform(0, 100)
        wi = rng.normal(size=3)
        wi = (wi / np.linalg.norm(wi)).astype(np.float32)
        g = orc.geometry(m, h, u, v, wi)
        if g["status"]:
            continue
        n += 1
        for a in ("n_p", "t_p", "n_f", "t_f"):
            assert np.linalg.norm(g[a]) == pytest.approx(1.0, abs=1e-12)
        assert abs(g["n_p"] @ g["t_p"]) < 1e-12
        assert abs(g["n_f"] @ g["t_f"]) < 1e-12
        assert g["n_p"][2] == 0.0
        assert 1 <= g["ni_mean"] <= 4
    assert n > 50


# ------------------------------------------------------------- fiber maps --
def brute_fiber_normal(L, D):
    """Outermost point of the fiber ring along the radial line at angle D
    (fiber 0 centred at angle 0), over all M fibers, and its normal angle."""
    d = np.array([math.cos(D), math.sin(D)])
    best = (-1.0, None)
    for j in range(L["M"]):
        a = 2 * math.pi * j / L["M"]
        C = L["Rfc"] * np.array([math.cos(a), math.sin(a)])
        cd = C @ d
        disc = L["rf"] ** 2 - C @ C + cd * cd
        if disc < 0:
            continue
        rho = cd + math.sqrt(disc)
        if rho > best[0]:
            best = (rho, C)
    P = best[0] * d
    nrm = (P - best[1]) / L["rf"]
    return math.atan2(d[0] * nrm[1] - d[1] * nrm[0], d @ nrm), P, nrm


@pytest.mark.parametrize("n_f", [32, 64, 128])
def test_fiber_normal_map_brute_force(orc, n_f):
    m = mat(fibers_per_ply=n_f)
    L = orc.layout(m)
    P = 2 * math.pi / L["M"]
    for D in np.linspace(-0.499 * P, 0.499 * P, 41):
        dlt, _ = orc.fiber_map(m, D)
        want, _, _ = brute_fiber_normal(L, D)
        assert dlt == pytest.approx(want, abs=1e-12)
    assert orc.fiber_map(m, 0.0)[0] == 0.0
    for D in (0.1 * P, 0.37 * P):
        assert orc.fiber_map(m, -D)[0] == pytest.approx(-orc.fiber_map(m, D)[0], abs=1e-15)


@pytest.mark.parametrize("n_f", [32, 64])
def test_fiber_occlusion_brute_force(orc, n_f):
    m = mat(fibers_per_ply=n_f)
    L = orc.layout(m)
    P = 2 * math.pi / L["M"]
    centres = [L["Rfc"] * np.array([math.cos(2 * math.pi * j / L["M"]),
                                    math.sin(2 * math.pi * j / L["M"])]) for j in range(1, L["M"])]
    n_dir = 4000
    phis = (np.arange(n_dir) + 0.5) / n_dir * math.pi - math.pi / 2
    for D in (0.0, 0.2 * P, -0.35 * P, 0.45 * P, 0.499 * P):
        _, Pt, nrm = brute_fiber_normal(L, D)
        base = math.atan2(nrm[1], nrm[0])
        blocked = 0
        for ph in phis:
            w = np.array([math.cos(base + ph), math.sin(base + ph)])
            hit = False
            for C in centres:
                q = Pt - C
                b = q @ w
                disc = b * b - (q @ q - L["rf"] ** 2)
                if disc >= 0 and -b + math.sqrt(disc) > 1e-12:
                    hit = True
                    break
            blocked += hit
        _, of = orc.fiber_map(m, D)
        assert of == pytest.approx(blocked / n_dir, abs=2.0 / n_dir + 1e-9), D
    assert orc.fiber_map(m, 0.0)[1] == 0.0   # a fiber crown sees the whole sky


def test_tabulated_maps_interpolate_linearly(orc):
    m = mat(fibers_per_ply=64, map_texels=64)
    L = orc.layout(m)
    P = 2 * math.pi / L["M"]
    T = 64
    centre = lambda i: ((i + 0.5) / T - 0.5) * P   # noqa: E731
    for i in (0, 5, 31, 63):
        a = orc.fiber_map(m, centre(i))
        b = orc.fiber_map_tab(m, centre(i) + 7 * P)   # periodic in the fiber phase
        assert b[0] == pytest.approx(a[0], abs=1e-12) and b[1] == pytest.approx(a[1], abs=1e-12)
    for i in (3, 40):
        mid = orc.fiber_map_tab(m, 0.5 * (centre(i) + centre(i + 1)))
        lo, hi = orc.fiber_map(m, centre(i)), orc.fiber_map(m, centre(i + 1))
        assert mid[0] == pytest.approx(0.5 * (lo[0] + hi[0]), abs=1e-12)
    # the wrap from the last texel to the first crosses the cusp linearly
    w = orc.fiber_map_tab(m, 0.5 * P)
    assert abs(w[0]) < 1e-12
    # no fiber detail
    assert orc.fiber_map_tab(mat(flags=1), 0.3) == (0.0, 0.0)


# --------------------------------------------------------------- shadowing --
@pytest.mark.parametrize("n_p", [2, 3, 5])
def test_ply_occlusion_brute_force(orc, n_p):
    m = mat(n_plies=n_p)
    L = orc.layout(m)
    rng = np.random.default_rng(7)
    ds = 1e-5
    s = np.arange(0.5, 2 / ds) * ds
    for _ in range(40):
        k, z = int(rng.integers(0, n_p)), float(rng.uniform(0, 50))
        a = rng.uniform(0, 2 * math.pi)
        c = helix_centre(L, k, n_p, z)
        x = c + L["Rp"] * np.array([math.cos(a), math.sin(a)])
        w = rng.normal(size=2)
        w /= np.linalg.norm(w)
        inside = np.zeros_like(s, dtype=bool)
        for j in range(n_p):
            if j == k:
                continue
            cj = helix_centre(L, j, n_p, z)
            px, py = x[0] + s * w[0] - cj[0], x[1] + s * w[1] - cj[1]
            inside |= px * px + py * py < L["Rp"] ** 2
        want = inside.sum() * ds / (2 * L["Rp"])
        got = orc.ply_occlusion(m, k, z, x, w)
        assert got == pytest.approx(want, abs=3 * ds)


def test_shadowing_limits(orc):
    rng = np.random.default_rng(8)
    recs = I.random_records(400, seed=8)
    for sig in (0.0, 1.0, 1e6):
        m = mat(n_plies=4, shadow_density=sig)
        for i in range(0, 400, 4):
            g = orc.geometry(m, recs["h"][i], recs["u"][i], recs["v"][i], recs["wi"][:, i])
            if g["status"]:
                continue
            for key in ("g_p", "g_f", "g_mean"):
                assert 0.0 <= g[key] <= 1.0
            if sig == 0.0:
                assert g["g_p"] == 1.0 and g["g_f"] == 1.0
            if sig == 1e6:
                # hard visibility: 0 when anything occludes, else 1
                assert g["g_p"] in (0.0, 1.0) or g["g_p"] < 1e-30
    del rng


def test_fiber_tangent_follows_fiber_helix(orc):
    # Sec. 3.5: t_f = R(t_p) tilts the ply tangent by the fiber helix angle in
    # the sense in which the fiber pattern advances along the ply; compare with
    # the tangent of the explicit fiber helix through the hit point
    rng = np.random.default_rng(9)
    for tw_f in (15.0, 35.0):
        m = mat(n_plies=3, ply_twist_deg=20.0, fiber_twist_deg=tw_f)
        L = orc.layout(m)
        errs = []
        for _ in range(60):
            h, u, v = (float(np.float32(x)) for x in (rng.uniform(-0.9, 0.9),
                                                        rng.uniform(0, 6.28), rng.uniform(0, 50)))
            wi = consistent_wi(h, u, rng.uniform(-0.3, 0.3))
            g = orc.geometry(m, h, u, v, wi)
            if g["status"]:
                continue
            k, zx = g["ply"], g["x"][2]

            def fiber_point(z, k=k, zx=zx, g=g):
                # explicit helix: ply centre c_k(z) plus R_p at the angle that
                # advances with the ply phase and the fiber phase
                c = helix_centre(L, k, 3, z)
                c0 = helix_centre(L, k, 3, zx)
                phi0 = math.atan2(g["x"][1] - c0[1], g["x"][0] - c0[0])
                phi = phi0 + (L["omega_p"] + L["omega_f"]) * (z - zx)
                return np.array([c[0] + L["Rp"] * math.cos(phi), c[1] + L["Rp"] * math.sin(phi), z])
            d = (fiber_point(zx + 1e-6) - fiber_point(zx - 1e-6)) / 2e-6
            # the implicit model keeps n_p in the cross-section (Sec. 3.4), so
            # compare within the plane it treats as tangent
            d -= (d @ g["n_p"]) * g["n_p"]
            d /= np.linalg.norm(d)
            errs.append(math.acos(min(1.0, abs(d @ g["t_f"]))))
        # the implicit frame approximates the explicit helix closely; the
        # opposite twist sense would be off by about twice the fiber angle
        assert np.median(errs) < 0.45 * math.radians(tw_f), (tw_f, np.median(errs))
        assert max(errs) < 0.9 * math.radians(tw_f), (tw_f, max(errs))
