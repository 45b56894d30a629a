"""Pins of the oracle's ray-yarn step (Sec. 3.3 explicit yarns, Sec. 5.3 ray
differentials): closed forms, a brute-force march, reconstruction of the hit
from the record, and consistency with the BYSDF's reading of (u, h, omega_i).
"""
import math

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

LIGHT = np.array([0.3, -0.4, math.sqrt(1 - 0.25)])


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def one_yarn(R=1.0):
    # along z from z = -10, reference normal x
    return [dict(p0=[0.0, 0.0, -10.0], t=[0.0, 0.0, 1.0], n_ref=[1.0, 0.0, 0.0], length=20.0,
                 radius=R, v0=3.0, mat_id=5)]


def rays_of(o, d):
    o = np.asarray(o, np.float32).reshape(-1, 3).T.copy()
    d = np.asarray(d, np.float32).reshape(-1, 3).T.copy()
    return dict(o=o, d=d)


def test_closed_forms_single_yarn(orc):
    # through the axis from +x, perpendicular: h = 0, u = 0, hit at x = R
    out = orc.trace_yarns(one_yarn(), rays_of([[5.0, 0.0, 1.0]], [[-1.0, 0.0, 0.0]]), LIGHT)
    assert out["yarn"][0] == 0 and out["mat_id"][0] == 5
    assert out["h"][0] == pytest.approx(0.0, abs=1e-15)
    assert out["u"][0] == pytest.approx(0.0, abs=1e-15)
    assert out["t_hit"][0] == pytest.approx(4.0, abs=1e-12)
    assert out["v"][0] == pytest.approx(3.0 + 11.0, abs=1e-12)
    np.testing.assert_allclose(out["wi"][:, 0], [1.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(out["wo"][:, 0], LIGHT, atol=1e-7)
    # from +y: u = pi / 2 (the frame's y = t x n_ref)
    out = orc.trace_yarns(one_yarn(), rays_of([[0.0, 5.0, 0.0]], [[0.0, -1.0, 0.0]]), LIGHT)
    assert out["u"][0] == pytest.approx(math.pi / 2, abs=1e-12)
    # offset by b in the cross-section: |h| = b / R, hit at the chord's entry
    b, R = 0.6, 2.0
    out = orc.trace_yarns(one_yarn(R), rays_of([[5.0, b, 0.0]], [[-1.0, 0.0, 0.0]]), LIGHT)
    assert abs(out["h"][0]) == pytest.approx(b / R, abs=1e-7)
    assert out["t_hit"][0] == pytest.approx(5.0 - math.sqrt(R * R - b * b), abs=1e-6)
    # a slanted ray: h and u see only the in-plane part; wi keeps the slope
    d = np.array([-1.0, 0.0, 0.5]) / math.sqrt(1.25)
    out = orc.trace_yarns(one_yarn(), rays_of([[5.0, 0.0, 0.0]], [d]), LIGHT)
    assert out["h"][0] == pytest.approx(0.0, abs=1e-7)
    assert out["wi"][2, 0] == pytest.approx(-0.5 / math.sqrt(1.25), abs=1e-7)
    # misses: past the radius, along the axis, beyond the piece's ends
    out = orc.trace_yarns(one_yarn(), rays_of([[5.0, 1.5, 0.0], [0.0, 0.0, -30.0],
                                               [5.0, 0.0, 12.0]],
                                              [[-1.0, 0.0, 0.0], [0.0, 0.0, 1.0],
                                               [-1.0, 0.0, 0.0]]), LIGHT)
    assert np.all(out["yarn"] == -1) and np.all(out["mat_id"] == -1)


def test_ray_starting_inside_sees_no_surface_of_that_yarn(orc):
    out = orc.trace_yarns(one_yarn(), rays_of([[0.2, 0.0, 0.0]], [[1.0, 0.0, 0.0]]), LIGHT)
    assert out["yarn"][0] == -1


def _scene():
    sc = I.woven_scene(6, 6)
    rays = I.camera_rays(48, 40, extent=6 * 2.5, jitter_seed=3)
    return sc, rays


def frame32(y):
    """The piece as the tracer reads it: float32 values, orthonormal frame."""
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    t = f(y["t"]); t /= np.linalg.norm(t)
    nr = f(y["n_ref"]); nr -= t * (nr @ t); nr /= np.linalg.norm(nr)
    return f(y["p0"]), t, nr, float(np.float32(y["radius"])), float(np.float32(y["v0"]))


def test_hit_reconstructs_from_the_record(orc):
    sc, rays = _scene()
    out = orc.trace_yarns(sc, rays, LIGHT, threads=4)
    hit = np.nonzero(out["yarn"] >= 0)[0]
    assert len(hit) > 0.8 * out["yarn"].size
    for i in hit[::7]:
        p0, t, nr, R, v0 = frame32(sc[out["yarn"][i]])
        br = np.cross(t, nr)
        u, v = out["u"][i], out["v"][i]
        x = p0 + (v - v0) * t + R * (math.cos(u) * nr + math.sin(u) * br)
        xr = rays["o"][:, i].astype(np.float64) + out["t_hit"][i] * rays["d"][:, i].astype(np.float64)
        np.testing.assert_allclose(x, xr, atol=1e-9)
        # the ray enters: wi on the outside of the surface normal
        n_u = math.cos(u) * np.array([1, 0, 0]) + math.sin(u) * np.array([0, 1, 0])
        assert out["wi"][:, i] @ n_u > 0


def test_brute_force_march_finds_the_same_first_entry(orc):
    # march each ray from the camera; an entry is a step from outside to
    # inside a piece's infinite cylinder whose axial coordinate lies on the
    # piece (its lateral surface; end caps are not surfaces)
    sc, rays = _scene()
    out = orc.trace_yarns(sc, rays, LIGHT, threads=4)
    fr = [frame32(y) for y in sc]
    P0 = np.array([x[0] for x in fr]); T = np.array([x[1] for x in fr])
    R = np.array([x[3] for x in fr]); Lk = np.array([float(np.float32(y["length"])) for y in sc])
    step = 2e-3
    for i in range(0, out["yarn"].size, 97):
        o = rays["o"][:, i].astype(np.float64); d = rays["d"][:, i].astype(np.float64)
        s_end = out["t_hit"][i] + 0.5 if out["yarn"][i] >= 0 else 250.0
        s = np.arange(0.0, s_end, step)
        q = (o[None, :] + s[:, None] * d[None, :])[:, None, :] - P0[None, :, :]
        w = np.einsum("skc,kc->sk", q, T)
        inside = (np.einsum("skc,skc->sk", q, q) - w * w) < R[None, :] ** 2
        enter = inside[1:] & ~inside[:-1] & (w[1:] >= 0) & (w[1:] <= Lk[None, :])
        steps, pieces = np.nonzero(enter)
        if out["yarn"][i] < 0:
            assert steps.size == 0
            continue
        k = np.argmin(steps)
        assert abs(s[steps[k] + 1] - out["t_hit"][i]) <= step
        assert pieces[k] == out["yarn"][i] or abs(s[steps[k] + 1] - out["t_hit"][i]) < 1e-9


def test_record_matches_the_bysdf_reading_of_u_h_and_wi(orc):
    # the BYSDF takes the in-plane ray direction from (u, h): -(cos(u - asin
    # h), sin(u - asin h)); for a traced hit it must be the in-plane part of
    # -wi
    sc, rays = _scene()
    out = orc.trace_yarns(sc, rays, LIGHT, threads=4)
    hit = out["yarn"] >= 0
    u, h, wi = out["u"][hit], out["h"][hit], out["wi"][:, hit]
    e_rec = -np.stack([np.cos(u - np.arcsin(h)), np.sin(u - np.arcsin(h))])
    e_ray = -wi[:2] / np.linalg.norm(wi[:2], axis=0)
    np.testing.assert_allclose(e_rec, e_ray, atol=1e-9)
    np.testing.assert_allclose(np.linalg.norm(wi, axis=0), 1.0, atol=1e-6)


def test_differential_rays_give_the_footprint(orc):
    # parallel rays shifted by +-delta across the axis: h = +-delta / R about
    # the centre ray, half-width delta / R
    R, delta = 2.0, 0.3
    o = np.array([[5.0, 0.1, 0.0]], np.float32).T
    d = np.array([[-1.0, 0.0, 0.0]], np.float32).T
    rays = dict(o=o, d=d, o1=o + np.array([[0], [delta], [0]], np.float32), d1=d,
                o2=o - np.array([[0], [delta], [0]], np.float32), d2=d)
    out = orc.trace_yarns(one_yarn(R), rays, LIGHT)
    assert out["ratio"][0] == pytest.approx(delta / R, abs=1e-7)
    # identical differential rays: no footprint
    rays.update(o1=o, o2=o)
    assert orc.trace_yarns(one_yarn(R), rays, LIGHT)["ratio"][0] == pytest.approx(0.0, abs=1e-12)
    # a distant camera: the footprint grows with the pixel size
    sc = I.woven_scene(4, 4)
    r1 = orc.trace_yarns(sc, I.camera_rays(32, 32, extent=10.0), LIGHT)
    r2 = orc.trace_yarns(sc, I.camera_rays(128, 128, extent=10.0), LIGHT)
    m1 = np.median(r1["ratio"][r1["yarn"] >= 0]); m2 = np.median(r2["ratio"][r2["yarn"] >= 0])
    assert m1 == pytest.approx(4 * m2, rel=0.15)


def test_scene_reference_normals_are_rotation_minimising(orc):
    # double reflection keeps n_ref perpendicular to each piece and turns it
    # only as much as the tangent turns (no twist about the yarn)
    sc = I.woven_scene(3, 10)
    for k in range(len(sc) - 1):
        a, b = sc[k], sc[k + 1]
        ta, tb = np.array(a["t"]), np.array(b["t"])
        na, nb = np.array(a["n_ref"]), np.array(b["n_ref"])
        assert abs(na @ ta) < 1e-12 and abs(np.linalg.norm(na) - 1) < 1e-12
        if b["v0"] == 0.0:            # next yarn
            continue
        # the frame rotation equals the tangent rotation (angle between
        # normals = angle between tangents for a planar polyline)
        ang_t = math.acos(np.clip(ta @ tb, -1, 1))
        ang_n = math.acos(np.clip(na @ nb, -1, 1))
        assert ang_n == pytest.approx(ang_t, abs=1e-9)
