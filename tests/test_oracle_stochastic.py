"""Pins of the oracle's stochastic estimators (Sec. 4.2 stratified h nodes;
Eq. 1's Omega_y integral with a GGX-sampled entry refraction).

The random numbers come from Philox4x64-10; the oracle's implementation is
checked bit for bit against NumPy's independent one.  The node positions are
recomputed here from NumPy's generator and the stratum formula.
"""
import math

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

KEY1 = 0xB15DF0005EED0001
JITTER, ROUGH = 1, 2


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def numpy_block(ctr, key):
    # NumPy's Philox advances the counter before its first block; counter and
    # key go in as uint64 arrays (a list of Python ints passes through float64)
    v = sum(int(x) << (64 * j) for j, x in enumerate(ctr)) - 1   # 256-bit counter - 1
    c = np.array([(v >> (64 * j)) & (2 ** 64 - 1) for j in range(4)], dtype=np.uint64)
    k = np.array([int(x) for x in key], dtype=np.uint64)
    return np.random.Philox(counter=c, key=k).random_raw(4)


def test_philox_matches_numpy(orc):
    rng = np.random.default_rng(5)
    for _ in range(50):
        ctr = rng.integers(1, 2 ** 63, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        np.testing.assert_array_equal(orc.philox4x64(ctr, key), numpy_block(ctr, key))
    # the counter words the estimators use (small indices, block 0 and 16)
    for ctr in ([1, 0, 0, 0], [12345, 3, 0, 0], [7, 16, 0, 0]):
        np.testing.assert_array_equal(orc.philox4x64(ctr, [9, KEY1]), numpy_block(ctr, [9, KEY1]))


def test_jittered_nodes_lie_in_their_strata(orc):
    rng = np.random.default_rng(6)
    for _ in range(40):
        h0 = float(np.float32(rng.uniform(-0.9, 0.9)))
        ratio = float(np.float32(rng.uniform(0.05, 0.6)))
        seed, index = int(rng.integers(0, 2 ** 40)), int(rng.integers(1, 2 ** 40))
        h = orc.stoch_nodes(h0, ratio, 16, seed, index)
        K = len(h)
        h1 = max(np.float32(h0) - np.float32(ratio), np.float32(-1.0))
        h2 = min(np.float32(h0) + np.float32(ratio), np.float32(1.0))
        w = float(np.float32(h2 - h1))
        assert K == max(1, math.ceil(np.float32(8.0) * np.float32(w)))
        for j in range(K):
            word = numpy_block([index, j // 4, 0, 0], [seed, KEY1])[j % 4]
            xi = int(word >> np.uint64(40)) / 2.0 ** 24
            assert h[j] == pytest.approx(float(h1) + (j + xi) * w / K, abs=1e-15)
            assert float(h1) + j * w / K <= h[j] < float(h1) + (j + 1) * w / K


def test_jitter_is_uniform_within_the_stratum(orc):
    # the fractional positions over many record indices are uniform (KS test)
    xs = []
    for index in range(1, 4001):
        h = orc.stoch_nodes(0.0, 0.25, 16, 123, index)
        K = len(h)
        xs.append((h[1] - (-0.25 + 0.5 / K)) / (0.5 / K))
    xs = np.sort(np.asarray(xs))
    d = np.max(np.abs(xs - (np.arange(1, len(xs) + 1) - 0.5) / len(xs)))
    assert d < 1.63 / math.sqrt(len(xs))   # 1% critical value


def test_no_flags_reproduce_the_deterministic_estimates(orc):
    mats = I.materials(3)
    rec = I.records(3, 0, 3000)
    f0, p0, s0 = orc.eval_records(mats, rec, threads=4)
    f1, p1, s1 = orc.eval_stochastic_records(mats, rec, seed=5, flags=0, threads=4)
    np.testing.assert_array_equal(f0, f1)
    np.testing.assert_array_equal(p0, p1)
    np.testing.assert_array_equal(s0, s1)
    a = orc.sample_records(mats, rec, threads=4)
    b = orc.sample_stochastic_records(mats, rec, seed=5, flags=0, threads=4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_jitter_leaves_the_near_field_alone(orc):
    # no footprint: one node at the record's own h, nothing to jitter
    mats = I.materials(1)
    rec = I.records(1, 0, 2000)
    f0, _, _ = orc.eval_records(mats, rec)
    f1, _, _ = orc.eval_stochastic_records(mats, rec, seed=11, flags=JITTER)
    np.testing.assert_array_equal(f0, f1)


def test_single_jittered_node_is_the_deterministic_node_moved(orc):
    # with K_max = 1 the one node sits at h1 + xi (h2 - h1); the same value is
    # the deterministic estimate of a record centred there with the entry
    # azimuth shifted so that the ray is unchanged
    m = I.material(k_max=1)
    rec = I.random_records(400, seed=81, wi_mode="cosine", v_max=5.0)
    rec["h"] = np.random.default_rng(82).uniform(-0.5, 0.5, 400).astype(np.float32)
    rec["ratio"] = np.full(400, 0.25, np.float32)
    seed = 77
    f_j, _, s_j = orc.eval_stochastic_records([m], rec, seed=seed, flags=JITTER)
    moved = {k: np.array(v, copy=True) for k, v in rec.items()}
    for i in range(400):
        word = numpy_block([i, 0, 0, 0], [seed, KEY1])[0]
        xi = int(word >> np.uint64(40)) / 2.0 ** 24
        h0 = np.float32(rec["h"][i])
        hj = float(h0 - np.float32(0.25)) + xi * float(np.float32(h0 + np.float32(0.25))
                                                       - np.float32(h0 - np.float32(0.25)))
        moved["h"][i] = np.float32(hj)
        moved["u"][i] = np.float32(float(rec["u"][i]) - math.asin(float(h0)) + math.asin(hj))
    f_d, _, s_d = orc.eval_records([m], moved)
    same = (s_j == 0) & (s_d == 0)
    assert same.mean() > 0.6
    # float32 rounding of the moved record (h, u, the footprint width) only;
    # where the fiber phase is steep that rounding alone moves f further
    close = np.isclose(f_j[:, same], f_d[:, same], rtol=2e-3, atol=1e-6).all(axis=0)
    assert close.mean() >= 0.99, close.mean()


def test_rough_entry_changes_only_the_transmission_lobe(orc):
    mats = I.materials(2)
    rec = I.records(2, 0, 4000)
    f0, _, s0 = orc.eval_records(mats, rec, threads=4)
    f1, _, s1 = orc.eval_stochastic_records(mats, rec, seed=3, flags=ROUGH, threads=4)
    np.testing.assert_array_equal(s0, s1)
    # omega_o on the camera side of the shading normal: reflection and f_x^B
    # only, untouched by the entry refraction; the far side differs
    frames = [orc.geometry(mats[int(rec["mat_id"][i])], rec["h"][i], rec["u"][i], rec["v"][i],
                           rec["wi"][:, i]) for i in range(400)]
    same_side = []
    for i, g in enumerate(frames):
        if g["status"] != 0:
            continue
        n = np.asarray(g["n_f"])
        wi, wo = rec["wi"][:, i], rec["wo"][:, i]
        same_side.append(i) if np.sign(n @ wi) == np.sign(n @ wo) else None
    same_side = np.asarray(same_side)
    assert len(same_side) > 50
    np.testing.assert_array_equal(f0[:, same_side], f1[:, same_side])
    assert np.any(f0 != f1)


def test_rough_entry_tends_to_the_smooth_entry(orc):
    # GGX roughness at its 1e-3 rad floor: the entry microfacet stays within
    # ~1e-3 rad of n, so the transmission lobe moves by O(1e-3) away from its
    # peak
    m = I.material(beta_deg=[0.01, 0.01])
    rec = I.random_records(3000, seed=83, wi_mode="cosine", v_max=5.0)
    f0, _, s0 = orc.eval_records([m], rec)
    f1, _, s1 = orc.eval_stochastic_records([m], rec, seed=9, flags=ROUGH)
    ok = (s0 == 0) & (s1 == 0) & (f0[0] > 1e-6)
    rel = np.abs(f1[0, ok] - f0[0, ok]) / f0[0, ok]
    assert np.median(rel) < 1e-3
    assert np.quantile(rel, 0.9) < 2e-2


def test_stochastic_sample_is_consistent_with_stochastic_eval(orc):
    # one seed and index draw the same nodes and entry for the sample and the
    # eval: the sample's pdf and weight are the eval's at the sampled omega_o
    mats = I.materials(3)
    rec = I.records(3, 0, 2000)
    flags = JITTER | ROUGH
    wo, w, pdf, st, lobe = orc.sample_stochastic_records(mats, rec, seed=21, flags=flags,
                                                        threads=4)
    r2 = dict(rec)
    r2["wo"] = wo.astype(np.float32)
    f, p, s = orc.eval_stochastic_records(mats, r2, seed=21, flags=flags, threads=4)
    ok = (st == 0) & (s == 0)
    assert ok.mean() > 0.5
    np.testing.assert_allclose(p[ok], pdf[ok], rtol=2e-4)
    np.testing.assert_allclose(f[:, ok] / p[ok], w[:, ok], rtol=2e-4)


def test_rough_entry_energy_bound(orc):
    # hemispherical albedo of the rough-entry BYSDF by importance sampling
    # (mean sample weight) stays within 1 for a white material
    m = I.material(albedo=[1.0, 1.0, 1.0], k_spec=1.0, sigma_t=0.0)
    n = 20000
    rec = I.random_records(n, seed=84, wi_mode="cosine", sample=True, v_max=5.0)
    rec["h"][:] = 0.3
    rec["u"][:] = 0.7
    rec["v"][:] = 1.1
    rec["wi"][:] = rec["wi"][:, :1]
    _, w, _, st, _ = orc.sample_stochastic_records([m], rec, seed=31, flags=ROUGH, threads=4)
    assert np.all(w[:, st == 0] >= 0)
    albedo = w[:, st == 0].sum(axis=1) / n
    assert np.all(albedo <= 1.0 + 3e-2), albedo
