"""Pins of the oracle's fiber migration (Sec. 3.5, "Adding fiber migration").

Reading: a migrating ply carries K_m map pairs; map 0 is the regular outer
ring, map k >= 1 the ring sunk by k r_f / K_m (holding as many fibers as fit
there).  Segments of `migration_length` along the yarn pick a map by a
Philox4x64-10 word of the segment index mod 256; maps blend linearly near
segment boundaries.
"""
import math

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

MIG_KEY1 = 0xB15DF000F1BE0002


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def mig(**kw):
    d = dict(migration_maps=3, migration_seed=7, migration_length=0.8, migration_blend=0.25)
    d.update(kw)
    return I.material(**d)


def numpy_word(seg, seed):
    # counter (seg mod 256, 0, 0, 0); NumPy advances it before its block
    v = ((seg % 256) - 1) % 2 ** 256
    c = np.array([(v >> (64 * j)) & (2 ** 64 - 1) for j in range(4)], dtype=np.uint64)
    k = np.array([seed, MIG_KEY1], dtype=np.uint64)
    return int(np.random.Philox(counter=c, key=k).random_raw(1)[0])


def brute_ring_normal(Rfc, rf, M, D):
    """Outermost point of a ring of M circles (radius rf, centres at radius
    Rfc, fiber 0 at angle 0) along the radial line at angle D; the angle of
    the circle's normal there from the radial direction."""
    d = np.array([math.cos(D), math.sin(D)])
    best = (-1.0, None)
    for j in range(M):
        a = 2 * math.pi * j / M
        C = Rfc * np.array([math.cos(a), math.sin(a)])
        cd = C @ d
        disc = rf ** 2 - C @ C + cd * cd
        if disc >= 0 and cd + math.sqrt(disc) > best[0]:
            best = (cd + math.sqrt(disc), C)
    nrm = (best[0] * d - best[1]) / rf
    return math.atan2(d[0] * nrm[1] - d[1] * nrm[0], d @ nrm)


def test_one_map_is_no_migration(orc):
    rec = I.random_records(3000, seed=91, wi_mode="cosine", v_max=20.0)
    f0, p0, s0 = orc.eval_records([I.material()], rec)
    f1, p1, s1 = orc.eval_records([mig(migration_maps=1)], rec)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(s0, s1)


def test_sunk_rings_and_their_maps(orc):
    m = mig(migration_maps=4, fibers_per_ply=64)
    L = orc.layout(m)
    T = m["map_texels"]
    prev_M = None
    for k in range(4):
        info = orc.migration_info(m, k)
        assert info["Rfc"] == pytest.approx(L["Rfc"] - k * L["rf"] / 4, abs=1e-14)
        # as many fibers as fit on the ring: ceil(pi / asin(r_f / R_fc))
        assert info["M"] == math.ceil(math.pi / math.asin(L["rf"] / info["Rfc"]))
        if prev_M is not None:
            assert info["M"] <= prev_M           # a deeper ring holds no more fibers
        prev_M = info["M"]
        dl, of = orc.migration_texels(m, k)
        P = 2 * math.pi / info["M"]
        for t in range(0, T, 17):
            D = ((t + 0.5) / T - 0.5) * P
            assert dl[t] == pytest.approx(brute_ring_normal(info["Rfc"], L["rf"], info["M"], D),
                                          abs=1e-12)
        assert np.all((of >= 0) & (of <= 1))
    # map 0 is the regular ring's
    dl0, of0 = orc.migration_texels(m, 0)
    D = ((np.arange(T) + 0.5) / T - 0.5) * 2 * math.pi / L["M"]
    np.testing.assert_allclose(dl0, [orc.fiber_map(m, x)[0] for x in D], atol=1e-15)


def test_segment_maps_follow_the_generator(orc):
    m = mig(migration_maps=3, migration_seed=1234)
    seen = set()
    for seg in list(range(-5, 60)) + [10 ** 6, -(10 ** 6)]:
        k = orc.migration_info(m, 0, seg)["map_of_segment"]
        assert k == numpy_word(seg, 1234) % 3
        # the choice repeats every 256 segments
        assert k == orc.migration_info(m, 0, seg + 256 * 7)["map_of_segment"]
        seen.add(k)
    assert seen == {0, 1, 2}


def test_migration_is_continuous_along_the_yarn(orc):
    # one ply (no twist about the axis) and straight fibers: f depends on v
    # only through the migration maps.  With blending the maps switch over
    # 2 b L of yarn, so no step between neighbouring samples comes near the
    # total change (a hard switch would jump by about all of it)
    m = mig(n_plies=1, migration_maps=3, migration_length=0.5, migration_blend=0.2,
            fibers_per_ply=32, fiber_twist_deg=0.0)
    n = 4001
    rec = I.random_records(1, seed=92, wi_mode="cosine")
    rec = {k: np.repeat(v, n, axis=-1) for k, v in rec.items()}
    rec["h"][:] = 0.35
    rec["v"] = np.linspace(0.0, 4.0, n).astype(np.float32)
    f, _, st = orc.eval_records([m], rec)
    assert np.all(st == 0)
    span = f[0].max() - f[0].min()
    assert span > 1e-4                       # the maps differ
    assert np.abs(np.diff(f[0])).max() < 0.05 * span
    # inside a segment, away from the blend zones, f is constant
    t = (rec["v"] / 0.5) % 1.0
    inner = (t > 0.25) & (t < 0.75) & (np.floor(rec["v"] / 0.5) == 3)
    assert np.ptp(f[0, inner]) == 0.0


def test_migration_changes_the_fiber_detail(orc):
    rec = I.random_records(4000, seed=93, wi_mode="cosine", v_max=20.0)
    f0, _, s0 = orc.eval_records([I.material()], rec)
    f1, _, s1 = orc.eval_records([mig()], rec)
    ok = (s0 == 0) & (s1 == 0)
    changed = (np.abs(f1 - f0) > 1e-6 * (1 + np.abs(f0))).any(axis=0)[ok]
    # records whose hit lies in a segment (or blend zone) using a sunk map
    assert 0.2 < changed.mean() < 1.0


def test_migration_gradient_matches_finite_differences(orc, monkeypatch):
    # the helix angles move the hit height, hence the blend weights and the
    # maps' phases: exact derivatives against central differences
    import oracle.oracle as O
    from test_oracle_bysdf import _material_f64, perturbed
    monkeypatch.setattr(O, "_material", _material_f64(O))
    m = mig(n_plies=3, ply_twist_deg=28.0, fiber_twist_deg=20.0, migration_length=0.6)
    rec = I.random_records(200, seed=94, wi_mode="cosine", v_max=3.0)
    g = np.random.default_rng(94).uniform(-1, 1, (3, 200))
    _, _, J = orc.grad_records([m], rec, g, jac=True)
    for k in (5, 6):
        eps = 1e-6
        fd = (orc.eval_records([perturbed(m, k, eps)], rec)[0]
              - orc.eval_records([perturbed(m, k, -eps)], rec)[0]) / (2 * eps)
        fd2 = (orc.eval_records([perturbed(m, k, 2 * eps)], rec)[0]
               - orc.eval_records([perturbed(m, k, -2 * eps)], rec)[0]) / (4 * eps)
        smooth = np.abs(fd - fd2) <= 1e-6 * (1 + np.abs(fd))
        assert smooth.mean() > 0.8
        for c in range(3):
            s = smooth[c]
            np.testing.assert_allclose(J[s, c, k], fd[c, s], rtol=1e-5, atol=1e-7)
