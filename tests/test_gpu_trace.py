"""GPU parity of the ray-yarn step (bysdf_trace_yarns) against the oracle, and
the traced records fed end to end into the BYSDF kernels."""
import math

import numpy as np
import pytest

import parity_util as PU
from paper_2401_12724_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LIGHT = (0.3, -0.4, math.sqrt(0.75))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12724_gb300 import api as A
    return A


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def np_(t):
    return t.detach().cpu().numpy()


def traced(api, orc, n_yarns=6, pieces=6, w=96, h=80, keep=None):
    sc = I.woven_scene(n_yarns, pieces)
    if keep is not None:
        sc = sc[:keep]
    rays = I.camera_rays(w, h, extent=pieces * 2.5, jitter_seed=5)
    Y = api.yarns_to_device(sc)
    rd = {k: torch.from_numpy(v).cuda() for k, v in rays.items()}
    g = {k: np_(v) for k, v in api.trace_yarns(Y, rd, LIGHT).items()}
    o = orc.trace_yarns(sc, rays, np.array(LIGHT), threads=8)
    return sc, rays, g, o


def check_trace(g, o, min_hit=0.8, extent=15.0):
    # float32 hit positions carry a few ulp of the camera distance, which the
    # camera sets in proportion to the patch extent: the tolerances of the
    # position-derived outputs (u, h, v) grow with it (2e-5 at extent 15)
    tol = 2e-5 * extent / 15.0
    same = g["yarn_id"] == o["yarn"]
    # ties between pieces meeting at a joint, and grazing rays, may go either
    # way in float32
    assert same.mean() >= 0.995, same.mean()
    hit = same & (o["yarn"] >= 0)
    assert hit.mean() > min_hit, hit.mean()
    assert np.all(g["mat_id"][hit] == o["mat_id"][hit])
    du = np.abs(np.angle(np.exp(1j * (g["u"][hit] - o["u"][hit]))))
    assert np.quantile(du, 0.999) < tol and du.max() < 1e-3, (np.quantile(du, 0.999), du.max())
    dh = np.abs(g["h"][hit] - o["h"][hit])
    assert np.quantile(dh, 0.999) < tol and dh.max() < 1e-3, (np.quantile(dh, 0.999), dh.max())
    np.testing.assert_allclose(g["v"][hit], o["v"][hit], rtol=1e-6, atol=tol)
    np.testing.assert_allclose(g["wi"][:, hit], o["wi"][:, hit], atol=2e-6)
    np.testing.assert_allclose(g["wo"][:, hit], o["wo"][:, hit], atol=2e-6)
    np.testing.assert_allclose(g["t_hit"][hit], o["t_hit"][hit], rtol=1e-5)
    dr = np.abs(g["ratio"][hit] - o["ratio"][hit])
    assert np.quantile(dr, 0.999) < 1e-4 + 1e-3 * np.quantile(o["ratio"][hit], 0.999)
    miss = same & (o["yarn"] < 0)
    assert np.all(g["mat_id"][miss] == -1)


def test_trace_matches_oracle(api, orc):
    sc, rays, g, o = traced(api, orc)
    PU.dump("trace", **{"g_" + k: v for k, v in g.items()}, **{"o_" + k: v for k, v in o.items()})
    check_trace(g, o)


@pytest.mark.parametrize("keep", [2048, 1001])
def test_trace_max_and_ragged_piece_counts(api, orc, keep):
    # the largest scene the kernel takes (2048 pieces: 8 rounds of 32 groups)
    # and a count that ends in a partial group and a partial round of groups
    sc, rays, g, o = traced(api, orc, n_yarns=32, pieces=32, w=72, h=64, keep=keep)
    assert len(sc) == keep
    # the first 1001 pieces are warp yarns only: gaps between them
    check_trace(g, o, min_hit=0.8 if keep == 2048 else 0.3, extent=32 * 2.5)


def test_traced_records_feed_the_bysdf(api, orc):
    # GPU trace -> GPU fused eval + sample, against the oracle BYSDF on the
    # same (GPU-traced) records
    sc, rays, g, _ = traced(api, orc, w=128, h=96)
    mats = I.materials(2)
    n = g["h"].size
    rng = np.random.default_rng(7)
    rec = dict(h=g["h"], u=g["u"], v=g["v"], wi=g["wi"], wo=g["wo"], ratio=g["ratio"],
               mat_id=g["mat_id"],
               u0=np.minimum(rng.random(n), 1 - 2 ** -24).astype(np.float32),
               u1=np.minimum(rng.random(n), 1 - 2 ** -24).astype(np.float32))
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda")
    out = api.eval_sample_pdf(M, d)
    f, p, st = np_(out["f"]), np_(out["pdf"]), np_(out["status"])
    assert np.all(st[g["mat_id"] < 0] == 2)
    fn = lambda r: orc.eval_records(mats, r, threads=8)  # noqa: E731
    view = PU.oracle_view(orc, fn, mats, rec)
    PU.assert_status(st, view, "trace.status")
    PU.assert_parity(f, view, 0, "trace.f", gpu_status=st)
    PU.assert_parity(p, view, 1, "trace.pdf", gpu_status=st)
    assert (st == 0).mean() > 0.5


def test_degenerate_rays_do_not_disturb_their_warp(api):
    # rays with a zero or non-finite direction or origin miss, and the other
    # rays of their warps (which share a culling bound with them) keep the
    # result they have without them, bit for bit
    sc = I.woven_scene(6, 6)
    rays = I.camera_rays(64, 48, extent=15.0, jitter_seed=2)
    Y = api.yarns_to_device(sc)
    base = {k: np_(v) for k, v in
            api.trace_yarns(Y, {k: torch.from_numpy(v).cuda() for k, v in rays.items()},
                            LIGHT).items()}
    bad = dict((k, v.copy()) for k, v in rays.items())
    idx = np.array([5, 37, 38, 700, 1501, 64 * 48 - 1])
    bad["d"][:, idx[:2]] = 0.0
    bad["d"][0, idx[2]] = np.nan
    bad["d"][1, idx[3]] = np.inf
    bad["o"][2, idx[4]] = np.nan
    bad["o"][:, idx[5]] = -np.inf
    got = {k: np_(v) for k, v in
           api.trace_yarns(Y, {k: torch.from_numpy(v).cuda() for k, v in bad.items()},
                           LIGHT).items()}
    assert np.all(got["mat_id"][idx] == -1)
    keep = np.ones(64 * 48, bool)
    keep[idx] = False
    assert (base["mat_id"][keep] >= 0).mean() > 0.5
    for k in base:
        np.testing.assert_array_equal(got[k][..., keep], base[k][..., keep], err_msg=k)


def test_trace_argument_errors(api):
    sc = I.woven_scene(2, 2)
    Y = api.yarns_to_device(sc)
    rays = {k: torch.from_numpy(v).cuda() for k, v in I.camera_rays(8, 8, 5.0).items()}
    with pytest.raises(RuntimeError, match="unit"):
        api.trace_yarns(Y, rays, (1.0, 1.0, 0.0))
    with pytest.raises(RuntimeError, match="yarns"):
        api.trace_yarns(Y[:0], rays, LIGHT)
    big = api.yarns_to_device(I.woven_scene(32, 33))
    with pytest.raises(RuntimeError, match="2048"):
        api.trace_yarns(big[:2049], rays, LIGHT)
    partial = dict(rays)
    partial.pop("d2")
    with pytest.raises(RuntimeError, match="differential"):
        api.trace_yarns(Y, partial, LIGHT)
