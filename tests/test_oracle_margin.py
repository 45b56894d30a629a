"""Pins of the oracle's discontinuity margins (the parity rule's record
classification): records placed exactly on a branch point of the model get a
zero margin in the right class, closed forms where the geometry gives one,
the measure of the fiber-map cusp interval, and -- tying the parity rule's
classification to the model's behaviour rather than to its own code --
well-conditioned records keep their oracle value under random moves of all
inputs at once, and records whose value jumps are never well-conditioned."""
import math

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

CL = {c: k for k, c in enumerate(("graze", "gap", "cusp", "axis", "hemi", "exit", "lobe",
                                   "sample", "shadow"))}


def one(**kw):
    """A single record as planes."""
    rec = dict(h=np.array([kw.get("h", 0.2)], np.float32),
               u=np.array([kw.get("u", 0.7)], np.float32),
               v=np.array([kw.get("v", 3.0)], np.float32),
               wi=np.asarray(kw["wi"], np.float32).reshape(3, 1),
               wo=np.asarray(kw.get("wo", [0.0, 0.6, 0.8]), np.float32).reshape(3, 1),
               mat_id=np.zeros(1, np.int32))
    for k in ("u0", "u1", "ratio"):
        if k in kw:
            rec[k] = np.array([kw[k]], np.float32)
    return rec


def consistent_wi(h, u, wz):
    g = math.asin(h)
    L = math.sqrt(1 - wz * wz)
    return [L * math.cos(u - g), L * math.sin(u - g), wz]


def test_single_ply_graze_is_distance_to_the_rim(orc):
    # one ply = the yarn itself, centred on the axis: the in-plane ray enters
    # at offset h, so its distance from the circle's edge is R (1 - |h|) at
    # every update
    m = [I.material(n_plies=1, fibers_per_ply=64)]
    for h in (0.0, 0.3, -0.77, 0.999):
        rec = one(h=h, u=1.1, wi=consistent_wi(h, 1.1, 0.3))
        g = orc.margins(m, rec, "eval")[CL["graze"], 0]
        assert g == pytest.approx(1.0 - abs(float(np.float32(h))), abs=1e-6)


def test_ray_through_the_contact_point_of_two_plies(orc):
    # two plies touch at the yarn axis; at v = 0 their centres lie on the x
    # axis.  A ray perpendicular to the yarn entering at u = pi/2 with h = 0
    # runs down the y axis, tangent to both ply circles at the contact
    # point: both plies are grazed and hit at the same distance
    m = [I.material(n_plies=2, ply_twist_deg=20.0)]
    rec = one(h=0.0, u=math.pi / 2, v=0.0, wi=[0.0, 1.0, 0.0])
    mg = orc.margins(m, rec, "eval")[:, 0]
    assert mg[CL["graze"]] < 1e-6
    # a ray off the axis by 0.1 misses the contact: both margins open up
    rec = one(h=0.1, u=math.pi / 2, v=0.0, wi=consistent_wi(0.1, math.pi / 2, 0.0))
    mg = orc.margins(m, rec, "eval")[:, 0]
    assert mg[CL["graze"]] > 1e-3


def test_outgoing_direction_in_the_tangent_plane(orc):
    m = [I.material()]
    h, u = 0.35, 0.9
    wi = consistent_wi(h, u, 0.2)
    geo = orc.geometry(m[0], h, u, 3.0, np.array(wi, np.float32))
    n = np.array(geo["n_f"])
    if np.dot(n, wi) < 0:
        n = -n
    t = np.cross(n, [0.0, 0.0, 1.0])
    t /= np.linalg.norm(t)
    for tilt in (0.0, 1e-3, 0.05):
        wo = t * math.cos(tilt) + n * math.sin(tilt)
        mg = orc.margins(m, one(h=h, u=u, wi=wi, wo=wo), "eval")[:, 0]
        assert mg[CL["hemi"]] == pytest.approx(math.sin(tilt), abs=2e-7)


def test_u0_on_a_lobe_boundary(orc):
    # the first lobe boundary is (1 - B) F(mu_i)
    m = [I.material()]
    h, u = -0.2, 2.0
    wi = consistent_wi(h, u, -0.1)
    geo = orc.geometry(m[0], h, u, 3.0, np.array(wi, np.float32))
    mui = abs(float(np.dot(geo["n_f"], wi)))
    p0 = (1.0 - m[0]["body_B"]) * orc.fresnel(mui, float(np.float32(m[0]["eta"])))
    for off in (0.0, 0.01):
        rec = one(h=h, u=u, wi=wi, u0=p0 + off, u1=0.3)
        mg = orc.margins(m, rec, "sample")[:, 0]
        assert mg[CL["lobe"]] == pytest.approx(off, abs=1e-7)
    # the eval op never reaches the lobe choice
    assert np.isinf(orc.margins(m, one(h=h, u=u, wi=wi), "eval")[CL["lobe"], 0])


def test_ray_along_the_axis(orc):
    m = [I.material()]
    mg = orc.margins(m, one(wi=[0.0, 0.0, 1.0]), "eval")[:, 0]
    assert mg[CL["axis"]] == 0.0
    mg = orc.margins(m, one(wi=[0.6, 0.0, 0.8]), "eval")[:, 0]
    assert mg[CL["axis"]] == pytest.approx(0.6, rel=1e-6)


def test_invalid_records_have_no_margin(orc):
    m = [I.material()]
    mg = orc.margins(m, one(h=1.5, wi=[1.0, 0.0, 0.0]), "eval")
    assert np.isinf(mg).all()


def test_cusp_interval_has_its_measure(orc):
    # the fiber phase of a near-field hit is spread evenly over the fiber
    # period, so the share of lookups in the cusp interval is 1 / T and the
    # share within x periods of it 1 / T + 2 x
    m = [I.material(map_texels=64)]
    rec = I.random_records(60000, seed=5, wi_mode="cosine")
    f, p, st = orc.eval_records(m, rec, threads=8)
    c = orc.margins(m, rec, "eval", threads=8)[CL["cusp"], st == 0]
    n = c.size
    for x, expect in ((0.0, 1 / 64), (0.005, 1 / 64 + 0.01)):
        share = (c <= x).mean()
        assert abs(share - expect) < 4 * math.sqrt(expect / n) + 1e-3, (x, share, expect)


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_well_conditioned_records_are_stable(orc, cfg):
    """The parity rule's classification against the model's behaviour under
    moves it did not use: random moves of all inputs at once, half as long
    as the rule's axis moves, change a well-conditioned record's value by no
    more than the rule allows (a quarter of the tolerance, by linearity at
    most half that), and records whose value jumps by ten tolerances under
    such moves are never classed well-conditioned."""
    from oracle import parity as PU
    mats = I.materials(cfg)
    rec = I.records(cfg, 0, 6000)
    fn = lambda r: orc.eval_records(mats, r, threads=8)  # noqa: E731
    view = PU.oracle_view(orc, fn, mats, rec, n_random=0)
    base = view.base
    dev = np.zeros(len(rec["h"]))
    for k in range(6):
        e = PU.SIGMA / 2
        o = fn(PU.perturb(rec, 500 + k, eps_geo=e, eps_dir=e))
        d = np.maximum(PU.dev(o[0], base[0]), PU.dev(o[1], base[1]))
        d[o[2] != base[2]] = np.inf
        dev = np.maximum(dev, d)
    assert view.stable.mean() > 0.4
    assert dev[view.stable].max() <= 2 * PU.COND_MAX, np.sort(dev[view.stable])[-5:]
    assert not (view.stable & (dev > 10)).any()
    assert (dev > 10).any()          # the workload does have such records
