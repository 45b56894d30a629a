"""Pins of the oracle's BYSDF (Sec. 4.1 Eqs. 1-6, Sec. 4.1.5 sampling, Sec.
4.2 Eqs. 7-11 multi-scale, Sec. 4.3 energy) by invariants: reciprocity,
closed-form albedos, the white furnace, the energy bound, chi-square tests of
the sampler against the pdf, the multi-scale limits, and finite differences of
the exact gradients."""
import math

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I


def mat(**kw):
    return I.material(**kw)


def rand_dir(rng, n=None):
    v = rng.normal(size=(3,) if n is None else (3, n))
    return v / np.linalg.norm(v, axis=0)


def rand_frame(rng):
    n = rand_dir(rng)
    t = rand_dir(rng)
    t -= n * (t @ n)
    t /= np.linalg.norm(t)
    return np.concatenate([t, np.cross(n, t), n])


def broadcast(rec, i, wo):
    """Record i repeated for every outgoing direction in wo (3, m)."""
    m = wo.shape[1]
    out = {k: np.repeat(rec[k][..., i:i + 1], m, axis=-1) for k in rec if k not in ("wo",)}
    out["wo"] = wo.astype(np.float32)
    return out


def sphere_grid(n_c, n_p):
    c = (np.arange(n_c) + 0.5) / n_c * 2 - 1
    p = (np.arange(n_p) + 0.5) / n_p * 2 * math.pi
    C, P = np.meshgrid(c, p, indexing="ij")
    S = np.sqrt(1 - C * C)
    dirs = np.stack([S * np.cos(P), S * np.sin(P), C]).reshape(3, -1)
    return dirs, 4 * math.pi / (n_c * n_p)


# ----------------------------------------------------------------- lobes --
def test_reflection_lobe_reciprocal(orc):
    # Eq. 2 first case: f_x^S(wi, wo) = f_x^S(wo, wi); outputs are f |wo.n|
    rng = np.random.default_rng(11)
    m = mat(beta_deg=[8.0, 14.0])
    n_ok = 0
    for _ in range(400):
        fr = rand_frame(rng)
        n = fr[6:]
        wi, wo = rand_dir(rng), rand_dir(rng)
        if (wi @ n) * (wo @ n) <= 0:
            continue
        a = orc.lobes(m, fr, [0.1, 0.2, 0.0], 0.7, 2.0, 0.0, wi, wo)["R"] / abs(wo @ n)
        b = orc.lobes(m, fr, [0.1, 0.2, 0.0], 0.7, 2.0, 0.0, wo, wi)["R"] / abs(wi @ n)
        assert a == pytest.approx(b, rel=1e-11, abs=1e-300)
        n_ok += a > 0
    assert n_ok > 100


def test_body_albedos_closed_form(orc):
    # Eqs. 5-6 with the normalised LS term: hemispherical albedos are exactly
    # r B G k^B (backward) and (1 - r) B G k^B (forward)
    rng = np.random.default_rng(12)
    m = mat(k_spec=0.0, body_B=0.6, body_r=0.3, albedo=[0.2, 0.5, 0.9], flags=1)
    dirs, dw = sphere_grid(1000, 48)
    for _ in range(3):
        fr = rand_frame(rng)
        n = fr[6:]
        wi = rand_dir(rng)
        if wi @ n < 0.05:
            wi = wi - 2 * (wi @ n) * n + 0.1 * n
            wi /= np.linalg.norm(wi)
        G = rng.uniform(0.2, 1.0)
        sx = np.zeros(3)
        sy = np.zeros(3)
        for k in range(dirs.shape[1]):
            o = orc.lobes(m, fr, [0, 0, 0], G, 1.0, 0.0, wi, dirs[:, k])
            sx += o["xB"]
            sy += o["yB"]
        alb = np.array([0.2, 0.5, 0.9])
        B, r = m["body_B"], m["body_r"]
        np.testing.assert_allclose(sx * dw, r * B * G * np.float32(alb), rtol=2e-3)
        np.testing.assert_allclose(sy * dw, (1 - r) * B * G * np.float32(alb), rtol=2e-3)


def _albedo_by_sampling(orc, mats, rec, i, n_side=64):
    """int f |cos| d(wo) of record i, as the mean sampling weight over a
    stratified (u0, u1) grid (weight = f / pdf, unbiased where pdf > 0)."""
    g = (np.arange(n_side) + 0.5) / n_side
    U0, U1 = np.meshgrid(g, g, indexing="ij")
    m = n_side * n_side
    r = {k: np.repeat(rec[k][..., i:i + 1], m, axis=-1) for k in rec if k != "wo"}
    r["u0"] = U0.reshape(-1).astype(np.float32)
    r["u1"] = U1.reshape(-1).astype(np.float32)
    wo, w, pdf, st, lobe = orc.sample_records(mats, r)
    return w.mean(axis=1), st


def test_white_furnace_and_energy_bound(orc):
    # Sec. 4.3: with albedos 1, sigma_t = 0 and no shadowing the body part
    # returns exactly B; specular reflection + transmission lose a little
    # (no internal reflection, single scattering), so the total is in [B, 1]
    rec = I.random_records(64, seed=13, wi_mode="cosine", sample=True)
    white = mat(albedo=[1.0, 1.0, 1.0], sigma_t=0.0, shadow_density=0.0, k_spec=1.0)
    body_only = dict(white, k_spec=0.0)
    seen = 0
    for i in range(0, 64, 4):
        tot, st = _albedo_by_sampling(orc, [white], rec, i)
        if (st == 1).all():
            continue
        seen += 1
        body, _ = _albedo_by_sampling(orc, [body_only], rec, i)
        np.testing.assert_allclose(body, 0.5, rtol=2e-2)
        assert (tot <= 1.0 + 2e-2).all()
        assert (tot >= 0.5 - 1e-2).all()
    assert seen >= 10
    # every workload material conserves energy for random records
    for cfg in (2,):
        mats = I.materials(cfg)
        rec = I.records(cfg, 0, 48)
        for i in range(48):
            tot, st = _albedo_by_sampling(orc, mats, rec, i, n_side=48)
            if (st == 1).all():
                continue
            assert (tot <= 1.0 + 2e-2).all(), (i, tot)


# -------------------------------------------------------------- sampling --
@pytest.mark.parametrize("seed", [21, 22, 23])
def test_sampler_chi_square_against_pdf(orc, seed):
    m = mat(n_plies=3, beta_deg=[18.0, 18.0], sigma_t=0.3)
    rec = I.random_records(40, seed=seed, wi_mode="cosine", sample=True)
    i = next(j for j in range(40)
             if orc.eval_records([m], {k: v[..., j:j + 1] for k, v in rec.items()})[2][0] == 0)
    n = 200_000
    rng = np.random.default_rng(seed)
    r = {k: np.repeat(rec[k][..., i:i + 1], n, axis=-1) for k in rec if k != "wo"}
    r["u0"] = np.minimum(rng.random(n), 1 - 2 ** -24).astype(np.float32)
    r["u1"] = np.minimum(rng.random(n), 1 - 2 ** -24).astype(np.float32)
    wo, w, pdf, st, lobe = orc.sample_records([m], r, threads=8)
    # pdf reported by the sampler equals the pdf of the sampled direction
    ok = st == 0
    q = {k: v[..., ok][..., :3000] for k, v in r.items()}
    q["wo"] = wo[:, ok][:, :3000].astype(np.float32)
    pdf2, st2 = orc.pdf_records([m], q)
    f2, _, _ = orc.eval_records([m], q)
    np.testing.assert_allclose(pdf2, pdf[ok][:3000], rtol=1e-5)
    np.testing.assert_allclose(f2 / pdf2, w[:, ok][:, :3000], rtol=1e-5)
    # histogram over (cos theta, phi) bins of the yarn frame + an invalid bin
    nc, nph = 12, 24
    def binof(d):
        ci = np.minimum(((d[2] + 1) / 2 * nc).astype(int), nc - 1)
        pi = np.minimum((np.mod(np.arctan2(d[1], d[0]), 2 * math.pi) / (2 * math.pi) * nph)
                        .astype(int), nph - 1)
        return ci * nph + pi
    hist = np.bincount(binof(wo[:, ok]), minlength=nc * nph).astype(float)
    dirs, dw = sphere_grid(1200, 1200)
    qq = broadcast({k: v[..., i:i + 1] for k, v in rec.items()}, 0, dirs)
    pd, _ = orc.pdf_records([m], qq, threads=8)
    expd = np.bincount(binof(dirs), weights=pd * dw, minlength=nc * nph) * n
    p_valid = (pd * dw).sum()
    assert p_valid <= 1.0 + 1e-3
    assert ok.mean() == pytest.approx(p_valid, abs=5e-3)
    sel = expd > 30
    chi2 = ((hist[sel] - expd[sel]) ** 2 / expd[sel]).sum()
    dof = sel.sum()
    assert chi2 < dof + 6 * math.sqrt(2 * dof), (chi2, dof)


# ----------------------------------------------------------- multi-scale --
def test_multiscale_limits(orc):
    mats = [mat(n_plies=4)]
    rec = I.random_records(300, seed=31, wi_mode="cosine")
    f_near, p_near, s_near = orc.eval_records(mats, rec)
    r0 = dict(rec, ratio=np.zeros(300, np.float32))
    f0, p0, s0 = orc.eval_records(mats, r0)
    assert np.array_equal(f_near, f0) and np.array_equal(s_near, s0)
    # a vanishing footprint tends to the near field (Sec. 4.2)
    r1 = dict(rec, ratio=np.full(300, 1e-6, np.float32))
    f1, p1, s1 = orc.eval_records(mats, r1)
    same = (s1 == s_near) & (s_near == 0)
    np.testing.assert_allclose(f1[:, same], f_near[:, same], rtol=2e-3, atol=1e-9)
    # a footprint covering the yarn is the far field: one value for any ratio
    # beyond 1 + |h0| (Eq. 7 over [-1, 1])
    h = rec["h"]
    ra = dict(rec, ratio=(1.0 + np.abs(h)).astype(np.float32) + np.float32(1e-3))
    rb = dict(rec, ratio=np.full(300, 100.0, np.float32))
    fa, _, sa = orc.eval_records(mats, ra)
    fb, _, sb = orc.eval_records(mats, rb)
    assert np.array_equal(fa, fb) and np.array_equal(sa, sb)


def test_far_field_ignores_hit_offset(orc):
    # Eq. 7 has no h0: the same ray direction gives the same far field
    m = mat(n_plies=3)
    rng = np.random.default_rng(32)
    for _ in range(20):
        c = rng.uniform(0, 2 * math.pi)
        wi = rand_dir(rng).astype(np.float32)
        wo = rand_dir(rng).astype(np.float32)
        vals = []
        for h0 in (-0.6, 0.1, 0.8):
            u = np.float32(c + math.asin(np.float32(h0)))
            r = dict(h=np.array([h0], np.float32), u=np.array([u]), v=np.array([7.0], np.float32),
                     wi=wi[:, None].copy(), wo=wo[:, None].copy(), ratio=np.array([50.0], np.float32),
                     mat_id=np.zeros(1, np.int32))
            vals.append(orc.eval_records([m], r)[0][:, 0])
        np.testing.assert_allclose(vals[0], vals[1], rtol=1e-4, atol=1e-9)
        np.testing.assert_allclose(vals[0], vals[2], rtol=1e-4, atol=1e-9)


def test_node_count_grows_with_footprint(orc):
    m = mat(k_max=16)
    for h0, ratio, K in ((0.0, 0.0, 1), (0.0, 0.05, 1), (0.0, 0.07, 2), (0.2, 0.5, 8),
                         (0.9, 0.5, 5), (0.0, 1.0, 16), (0.5, 3.0, 16)):
        g = orc.geometry(m, h0, 0.3, 1.0, np.array([1.0, 0.0, 0.0], np.float32), ratio)
        h1, h2 = max(h0 - ratio, -1.0), min(h0 + ratio, 1.0)
        assert g["n_nodes"] == max(1, math.ceil(16 * (h2 - h1) / 2 - 1e-6)) == K


def test_multiscale_roughness_and_aggregate(orc):
    # a wide footprint averages normals over the cross-section: the aggregate
    # normal turns towards the viewer and the lobe widens (beta_multi)
    m = mat(n_plies=1, flags=1, shadow_density=0.0)
    wi = np.array([1.0, 0.0, 0.0], np.float32)
    g = orc.geometry(m, 0.0, 0.0, 1.0, wi, 100.0)
    assert g["n_nodes"] == 16 and g["n_hit_nodes"] == 16
    np.testing.assert_allclose(g["n_f"], [1.0, 0.0, 0.0], atol=1e-12)


# ------------------------------------------------------------- gradients --
PARAM_FIELDS = [("albedo", 0, 1.0), ("albedo", 1, 1.0), ("albedo", 2, 1.0),
                ("beta_deg", 0, 180 / math.pi), ("beta_deg", 1, 180 / math.pi),
                ("ply_twist_deg", None, 180 / math.pi), ("fiber_twist_deg", None, 180 / math.pi),
                ("shadow_density", None, 1.0)]


def perturbed(m, k, eps):
    d = {kk: (list(vv) if isinstance(vv, list) else vv) for kk, vv in m.items()}
    field, idx, scale = PARAM_FIELDS[k]
    if idx is None:
        d[field] = d[field] + eps * scale
    else:
        d[field][idx] = d[field][idx] + eps * scale
    return d


def test_gradient_matches_finite_differences(orc, monkeypatch):
    # exact forward-mode AD of the oracle vs central differences in FP64; the
    # descriptor is widened from float32, so differences use a float64 path
    import oracle.oracle as O
    monkeypatch.setattr(O, "_material", _material_f64(O))
    m = mat(n_plies=3, ply_twist_deg=28.0, fiber_twist_deg=20.0, beta_deg=[12.0, 9.0],
            albedo=[0.3, 0.6, 0.8], shadow_density=0.7)
    rec = I.random_records(200, seed=41, wi_mode="cosine", v_max=3.0)
    rec["ratio"] = np.where(np.arange(200) % 2 == 0, 0.0, 0.3).astype(np.float32)
    rng = np.random.default_rng(41)
    g = rng.uniform(-1, 1, (3, 200))
    _, f, J = orc.grad_records([m], rec, g, jac=True)
    checked = 0
    for k in range(8):
        for eps in (1e-6,):
            fp = orc.eval_records([perturbed(m, k, eps)], rec)[0]
            fm = orc.eval_records([perturbed(m, k, -eps)], rec)[0]
            fp2 = orc.eval_records([perturbed(m, k, 2 * eps)], rec)[0]
            fm2 = orc.eval_records([perturbed(m, k, -2 * eps)], rec)[0]
            fd = (fp - fm) / (2 * eps)
            fd2 = (fp2 - fm2) / (4 * eps)
            # skip records whose difference quotient straddles a branch
            smooth = np.abs(fd - fd2) <= 1e-6 * (1 + np.abs(fd))
            for c in range(3):
                s = smooth[c]
                checked += s.sum()
                np.testing.assert_allclose(J[s, c, k], fd[c, s], rtol=1e-5, atol=1e-7)
    assert checked > 0.9 * 200 * 3 * 8 * 0.8


def _material_f64(O):
    def mk(d):
        m = O.Material()
        for f, t in O.Material._fields_:
            if f in ("albedo",):
                for c in range(3):
                    m.albedo[c] = float(d["albedo"][c])
            elif f == "albedo_y":
                for c in range(3):
                    m.albedo_y[c] = float(d["albedo_y"][c]) if "albedo_y" in d else -1.0
            elif f == "beta_deg":
                for c in range(2):
                    m.beta_deg[c] = float(d["beta_deg"][c])
            elif f == "flags":
                m.flags = int(d.get("flags", 0))
            elif f.startswith("migration_"):
                dflt = dict(migration_maps=1, migration_seed=0, migration_length=1.0,
                            migration_blend=0.25)[f]
                setattr(m, f, type(dflt)(d.get(f, dflt)))
            else:
                setattr(m, f, d[f] if t.__name__.startswith("c_int") else float(d[f]))
        return m
    return mk


# Extended parameter set (the paper's fitting set, Sec. 5.2: r, k^B_x, k^B_y,
# sigma_t; plus B and k_spec) and the record's directions.
PARAM_FIELDS_EXT = PARAM_FIELDS + [("body_r", None, 1.0), ("albedo_y", 0, 1.0),
                                   ("albedo_y", 1, 1.0), ("albedo_y", 2, 1.0),
                                   ("sigma_t", None, 1.0), ("body_B", None, 1.0),
                                   ("k_spec", None, 1.0)]


def perturbed_ext(m, k, eps):
    d = {kk: (list(vv) if isinstance(vv, list) else vv) for kk, vv in m.items()}
    field, idx, scale = PARAM_FIELDS_EXT[k]
    if idx is None:
        d[field] = d[field] + eps * scale
    else:
        d[field][idx] = d[field][idx] + eps * scale
    return d


def _ext_case():
    m = mat(n_plies=3, ply_twist_deg=28.0, fiber_twist_deg=20.0, beta_deg=[12.0, 9.0],
            albedo=[0.3, 0.6, 0.8], albedo_y=[0.45, 0.35, 0.7], shadow_density=0.7,
            body_r=0.4, body_B=0.6, sigma_t=0.8, k_spec=0.9)
    rec = I.random_records(240, seed=43, wi_mode="cosine", v_max=3.0)
    rec["ratio"] = np.where(np.arange(240) % 2 == 0, 0.0, 0.3).astype(np.float32)
    g = np.random.default_rng(43).uniform(-1, 1, (3, 240))
    return m, rec, g


def test_extended_gradient_matches_finite_differences(orc, monkeypatch):
    # the 15 material parameters: central differences on the float64
    # descriptor path, branch straddles skipped by a step-halving check
    import oracle.oracle as O
    monkeypatch.setattr(O, "_material", _material_f64(O))
    m, rec, g = _ext_case()
    _, _, _, f, J = orc.grad_ext_records([m], rec, g, jac=True)
    assert J.shape == (240, 3, 21)
    for k in range(15):
        eps = 1e-6
        fd = (orc.eval_records([perturbed_ext(m, k, eps)], rec)[0]
              - orc.eval_records([perturbed_ext(m, k, -eps)], rec)[0]) / (2 * eps)
        fd2 = (orc.eval_records([perturbed_ext(m, k, 2 * eps)], rec)[0]
               - orc.eval_records([perturbed_ext(m, k, -2 * eps)], rec)[0]) / (4 * eps)
        smooth = np.abs(fd - fd2) <= 1e-6 * (1 + np.abs(fd))
        assert smooth.mean() > 0.8, k
        for c in range(3):
            s = smooth[c]
            np.testing.assert_allclose(J[s, c, k], fd[c, s], rtol=1e-5, atol=1e-7,
                                       err_msg=f"parameter {k}")
    # each new parameter moves f somewhere (a dropped dependence fails here)
    for k in range(8, 15):
        assert np.abs(J[:, :, k]).max() > 1e-3, k


def test_extended_gradient_direction_partials(orc):
    # d f / d wi_c and d f / d wo_c against central differences of the
    # oracle's value: the records are float32, so each step is the exact
    # float32 difference (the value itself is evaluated in float64)
    m, rec, g = _ext_case()
    _, gwi, gwo, f, J = orc.grad_ext_records([m], rec, g, jac=True)
    # small enough not to cross texels of the piecewise-linear fiber maps
    # (the fiber phase is steep in wi), large against the float32 spacing
    step = 2.0 ** -20
    for key, base in (("wi", 15), ("wo", 18)):
        for c in range(3):
            def fdiff(h):
                rp = {k: np.array(v, copy=True) for k, v in rec.items()}
                rm = {k: np.array(v, copy=True) for k, v in rec.items()}
                rp[key][c] = (rec[key][c].astype(np.float64) + h).astype(np.float32)
                rm[key][c] = (rec[key][c].astype(np.float64) - h).astype(np.float32)
                den = rp[key][c].astype(np.float64) - rm[key][c].astype(np.float64)
                fp, _, sp = orc.eval_records([m], rp)
                fm, _, sm = orc.eval_records([m], rm)
                return (fp - fm) / den, (sp == 0) & (sm == 0)
            fd, ok1 = fdiff(step)
            fd2, ok2 = fdiff(2 * step)
            smooth = (np.abs(fd - fd2) <= 2e-4 * (1 + np.abs(fd))) & ok1 & ok2
            assert smooth.mean() > 0.6, (key, c)
            for cc in range(3):
                s = smooth[cc]
                np.testing.assert_allclose(J[s, cc, base + c], fd[cc, s], rtol=1e-3, atol=1e-5,
                                           err_msg=f"{key}[{c}]")
    # the vector-Jacobian products are the Jacobian contracted with g
    np.testing.assert_allclose(gwi, np.einsum("ck,kcd->dk", g, J[:, :, 15:18]), rtol=1e-12,
                               atol=1e-12)
    np.testing.assert_allclose(gwo, np.einsum("ck,kcd->dk", g, J[:, :, 18:21]), rtol=1e-12,
                               atol=1e-12)


def test_extended_gradient_agrees_with_eight_parameter_set(orc):
    # with k^B_y tied to the albedo, the 8-parameter albedo derivative moves
    # both body colours: it is the sum of the two separate ones
    m, rec, g = _ext_case()
    m = {k: v for k, v in m.items() if k != "albedo_y"}
    grad8, f8 = orc.grad_records([m], rec, g)
    grad15, _, _, f15 = orc.grad_ext_records([m], rec, g)
    np.testing.assert_array_equal(f8, f15)
    np.testing.assert_allclose(grad8[:, 0:3], grad15[:, 0:3] + grad15[:, 9:12], rtol=1e-12,
                               atol=1e-12)
    np.testing.assert_allclose(grad8[:, 3:8], grad15[:, 3:8], rtol=1e-12, atol=1e-12)



def test_l2_loss_is_multimodal_in_the_helix_angles(orc):
    """Why the fitting tests leave the helix angles alone: within 4% of the
    true angles, over a stretch of yarn only two radii long, the L2 loss
    against the true radiance already has several local minima in each
    angle -- the ply and fiber phases, and the fiber pattern under the hit
    point, cycle as the angles move -- so gradient steps from a start a few
    percent off need not reach the true values (their gradients are still
    checked against finite differences and against the GPU)."""
    mats0 = I.materials(5)[:4]
    rec = I.random_records(4096, n_mat=4, seed=65, wi_mode="cosine", sorted_ids=True, v_max=2.0)
    tgt, _, st = orc.eval_records(mats0, rec, threads=8)
    for key in ("ply_twist_deg", "fiber_twist_deg"):
        loss = []
        for e in np.linspace(-0.04, 0.04, 81):
            mats = [dict(m, **{key: m[key] * (1 + e)}) for m in mats0]
            f, _, _ = orc.eval_records(mats, rec, threads=8)
            loss.append((((f - tgt) ** 2) * (st == 0)).sum())
        d = np.diff(np.array(loss))
        minima = int(((d[:-1] < 0) & (d[1:] > 0)).sum())
        assert minima >= 3, (key, minima)


def test_l2_loss_gradient_matches_finite_differences(orc, monkeypatch):
    # the objective of the fused L2 pass, L = sum_i w_i sum_c (f_c - t_c)^2
    # over the valid records, differentiated with the oracle's exact
    # gradient at g = 2 w (f - t), against central differences of L itself
    # (float64 descriptors so that the steps are not rounded away)
    import oracle.oracle as O
    monkeypatch.setattr(O, "_material", _material_f64(O))
    m = mat(n_plies=3, ply_twist_deg=28.0, fiber_twist_deg=20.0, beta_deg=[12.0, 9.0],
            albedo=[0.3, 0.6, 0.8], shadow_density=0.7)
    rec = I.random_records(300, seed=47, wi_mode="cosine", v_max=3.0)
    rng = np.random.default_rng(48)
    f0, _, st = orc.eval_records([m], rec)
    target = f0 * rng.uniform(0.6, 1.4, f0.shape)
    w = rng.uniform(0.5, 1.5, 300) * (st == 0)

    def loss(mm):
        f, _, _ = orc.eval_records([mm], rec)
        return float((w * ((f - target) ** 2).sum(0)).sum())

    g = 2.0 * w * (f0 - target)
    grad, _ = orc.grad_records([m], rec, g)
    checked = 0
    for k in range(8):
        eps = 1e-6
        fd = (loss(perturbed(m, k, eps)) - loss(perturbed(m, k, -eps))) / (2 * eps)
        fd2 = (loss(perturbed(m, k, 2 * eps)) - loss(perturbed(m, k, -2 * eps))) / (4 * eps)
        if abs(fd - fd2) > 1e-5 * (1 + abs(fd)):
            continue              # a record on a branch within the step
        checked += 1
        np.testing.assert_allclose(grad[0, k], fd, rtol=1e-5, atol=1e-6)
    assert checked >= 6
