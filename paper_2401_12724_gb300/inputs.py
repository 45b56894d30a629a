"""Seeded synthetic workloads (material descriptors and hit records).

This module holds no arithmetic of the BYSDF itself: it only draws inputs.
Both the CUDA path and the FP64 oracle consume what it produces.

The paper renders Mitsuba scenes from yarn datasets that are not available
here; these generators stand in for its ray--yarn hit records with the shapes
and parameter ranges of five benchmark workloads:

  1  near-field eval, 1 material, 65,536 records
  2  eval + sample + pdf, 8 materials, 2^24 records, ids uniform
  3  as 2 plus a pixel-footprint / yarn-width ratio, log-uniform [0.01, 100]
  4  256 materials, Zipf(1.1) record counts totalling 2^26, material-sorted
  5  64 materials, 2^24 material-sorted records, upstream gradients (fitting)

Random numbers come from NumPy's Philox-4x64-10 (a counter-based generator),
keyed by (seed, workload); records are drawn in chunks of 2^16 so that any
sub-range is reproducible on its own.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0xB15DF
CHUNK = 1 << 16

DEFAULTS = dict(
    yarn_radius=1.0, eta=1.55, k_spec=1.0, body_B=0.5, body_r=0.5, sigma_t=0.5,
    shadow_density=1.0, packing=0.8, map_texels=256, trace_iters=5, k_max=16, flags=0,
)

N_RECORDS = {1: 1 << 16, 2: 1 << 24, 3: 1 << 24, 4: 1 << 26, 5: 1 << 24}
N_MATERIALS = {1: 1, 2: 8, 3: 8, 4: 256, 5: 64}
WORKLOAD_NAME = {
    1: "near-eval-1mat-65536",
    2: "eval+sample+pdf-8mat-2^24",
    3: "multiscale-8mat-2^24",
    4: "batched-256mat-zipf1.1-2^26",
    5: "fwd+bwd-64mat-2^24",
}


def _key(cfg: int, seed: int | None = None):
    return [SEED_BASE + cfg if seed is None else seed, cfg]


def _gen(cfg: int, stream: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=_key(cfg, seed)).jumped(stream))


def material(**over) -> dict:
    """One material descriptor with the documented defaults."""
    d = dict(DEFAULTS)
    d.update(n_plies=3, fibers_per_ply=64, ply_twist_deg=30.0, fiber_twist_deg=15.0,
             beta_deg=[10.0, 10.0], albedo=[0.5, 0.5, 0.5])
    d.update(over)
    return d


def materials(cfg: int, seed: int | None = None) -> list[dict]:
    g = _gen(cfg, 0, seed)
    if cfg == 1:
        alb = g.uniform(0.2, 0.9, 3)
        return [material(albedo=[float(np.float32(a)) for a in alb])]
    out = []
    for _ in range(N_MATERIALS[cfg]):
        n_p = int(g.integers(2, 6))
        n_f = int(g.integers(32, 129))
        tw_p, tw_f = (float(np.float32(x)) for x in g.uniform(10.0, 45.0, 2))
        beta = float(np.float32(g.uniform(5.0, 20.0)))
        alb = [float(np.float32(a)) for a in g.uniform(0.1, 0.95, 3)]
        out.append(material(n_plies=n_p, fibers_per_ply=n_f, ply_twist_deg=tw_p,
                            fiber_twist_deg=tw_f, beta_deg=[beta, beta], albedo=alb))
    return out


def counts(cfg: int, seed: int | None = None) -> np.ndarray | None:
    """Per-material record counts of the material-sorted workloads."""
    n, m = N_RECORDS[cfg], N_MATERIALS[cfg]
    g = _gen(cfg, 1 << 20, seed)
    if cfg == 4:
        w = 1.0 / np.arange(1, m + 1, dtype=np.float64) ** 1.1
        perm = g.permutation(m)
        exact = w / w.sum() * n
        base = np.floor(exact).astype(np.int64)
        rem = n - int(base.sum())
        order = np.argsort(-(exact - base), kind="stable")
        base[order[:rem]] += 1
        c = np.zeros(m, np.int64)
        c[perm] = base
        return c
    if cfg == 5:
        return g.multinomial(n, [1.0 / m] * m).astype(np.int64)
    return None


def seg_offsets(cfg: int, seed: int | None = None) -> np.ndarray | None:
    c = counts(cfg, seed)
    if c is None:
        return None
    return np.concatenate([[0], np.cumsum(c)]).astype(np.int64)


def _uniform_sphere(g, n):
    z = 1.0 - 2.0 * g.random(n)
    phi = 2.0 * math.pi * g.random(n)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z])


def _cosine_about_yarn_normal(g, u, n):
    a = g.random(n)
    phi = 2.0 * math.pi * g.random(n)
    lt, lb, ln = np.sqrt(a) * np.cos(phi), np.sqrt(a) * np.sin(phi), np.sqrt(1.0 - a)
    cu, su = np.cos(u), np.sin(u)
    # frame at azimuth u: yarn normal (cu, su, 0), binormal (-su, cu, 0), tangent z
    return np.stack([ln * cu - lb * su, ln * su + lb * cu, lt])


def _chunk(cfg: int, c: int, n_chunk: int, offs, seed):
    g = _gen(cfg, c + 1, seed)
    out = {}
    h = g.uniform(-1.0, 1.0, n_chunk)
    u = g.uniform(0.0, 2.0 * math.pi, n_chunk)
    v = g.uniform(0.0, 100.0, n_chunk)
    if cfg == 1:
        wi = _uniform_sphere(g, n_chunk)
    else:
        wi = _cosine_about_yarn_normal(g, u.astype(np.float32).astype(np.float64), n_chunk)
    wo = _uniform_sphere(g, n_chunk)
    out["h"] = h.astype(np.float32)
    out["u"] = u.astype(np.float32)
    out["v"] = v.astype(np.float32)
    out["wi"] = wi.astype(np.float32)
    out["wo"] = wo.astype(np.float32)
    if cfg in (2, 3, 4):
        out["u0"] = g.random(n_chunk).astype(np.float32)
        out["u1"] = g.random(n_chunk).astype(np.float32)
        np.minimum(out["u0"], np.float32(1.0 - 2.0 ** -24), out=out["u0"])
        np.minimum(out["u1"], np.float32(1.0 - 2.0 ** -24), out=out["u1"])
    if cfg == 3:
        out["ratio"] = np.exp(g.uniform(math.log(0.01), math.log(100.0), n_chunk)).astype(np.float32)
    if cfg == 5:
        out["g"] = g.uniform(-1.0, 1.0, (3, n_chunk)).astype(np.float32)
    if offs is None:
        out["mat_id"] = g.integers(0, N_MATERIALS[cfg], n_chunk).astype(np.int32)
    return out


def records(cfg: int, start: int = 0, count: int | None = None, seed: int | None = None) -> dict:
    """Records [start, start + count) of workload `cfg` as float32/int32 planes.

    Keys: h, u, v (n), wi, wo (3, n), mat_id (n), and depending on the workload
    u0, u1 (sampling), ratio (footprint), g (upstream gradient, (3, n)).
    """
    n_total = N_RECORDS[cfg]
    if count is None:
        count = n_total - start
    assert 0 <= start and start + count <= n_total
    offs = seg_offsets(cfg, seed)
    parts = []
    c0, c1 = start // CHUNK, (start + count + CHUNK - 1) // CHUNK
    for c in range(c0, c1):
        n_chunk = min(CHUNK, n_total - c * CHUNK)
        parts.append(_chunk(cfg, c, n_chunk, offs, seed))
    out = {}
    lo = start - c0 * CHUNK
    for k in parts[0]:
        axis = -1
        cat = np.concatenate([p[k] for p in parts], axis=axis)
        out[k] = np.ascontiguousarray(cat[..., lo:lo + count])
    if offs is not None:
        idx = np.arange(start, start + count, dtype=np.int64)
        out["mat_id"] = (np.searchsorted(offs, idx, side="right") - 1).astype(np.int32)
    return out


def sample_indices(cfg: int, k: int, seed: int = 7) -> np.ndarray:
    """k sorted record indices spread over the whole workload (for spot checks)."""
    g = np.random.Generator(np.random.Philox(key=[SEED_BASE + 1000 + cfg, seed]))
    return np.sort(g.choice(N_RECORDS[cfg], size=k, replace=False))


def gather(cfg: int, idx: np.ndarray, seed: int | None = None) -> dict:
    """Records at arbitrary indices (chunk-wise, without drawing the whole set)."""
    idx = np.asarray(idx, dtype=np.int64)
    chunks = np.unique(idx // CHUNK)
    offs = seg_offsets(cfg, seed)
    cache = {}
    for c in chunks:
        n_chunk = min(CHUNK, N_RECORDS[cfg] - int(c) * CHUNK)
        cache[int(c)] = _chunk(cfg, int(c), n_chunk, offs, seed)
    keys = list(next(iter(cache.values())).keys())
    out = {}
    for k in keys:
        vals = [cache[int(i // CHUNK)][k][..., int(i % CHUNK)] for i in idx]
        out[k] = np.ascontiguousarray(np.stack(vals, axis=-1))
    if offs is not None:
        out["mat_id"] = (np.searchsorted(offs, idx, side="right") - 1).astype(np.int32)
    return out


def random_records(n: int, n_mat: int = 1, seed: int = 1, wi_mode: str = "sphere",
                   ratio: str | None = None, sample: bool = False, v_max: float = 100.0,
                   sorted_ids: bool = False) -> dict:
    """Small ad-hoc record sets for tests (same distributions as the workloads)."""
    g = np.random.Generator(np.random.Philox(key=[SEED_BASE + 99, seed]))
    u = g.uniform(0.0, 2.0 * math.pi, n).astype(np.float32)
    out = dict(h=g.uniform(-1.0, 1.0, n).astype(np.float32), u=u,
               v=g.uniform(0.0, v_max, n).astype(np.float32))
    if wi_mode == "sphere":
        wi = _uniform_sphere(g, n)
    else:
        wi = _cosine_about_yarn_normal(g, u.astype(np.float64), n)
    out["wi"] = wi.astype(np.float32)
    out["wo"] = _uniform_sphere(g, n).astype(np.float32)
    ids = g.integers(0, n_mat, n).astype(np.int32)
    out["mat_id"] = np.sort(ids) if sorted_ids else ids
    if ratio == "loguniform":
        out["ratio"] = np.exp(g.uniform(math.log(0.01), math.log(100.0), n)).astype(np.float32)
    elif ratio is not None:
        out["ratio"] = np.full(n, float(ratio), np.float32)
    if sample:
        out["u0"] = np.minimum(g.random(n), 1.0 - 2.0 ** -24).astype(np.float32)
        out["u1"] = np.minimum(g.random(n), 1.0 - 2.0 ** -24).astype(np.float32)
    return out


def seg_offsets_from_ids(mat_id: np.ndarray, n_mat: int) -> np.ndarray:
    c = np.bincount(np.asarray(mat_id), minlength=n_mat)
    return np.concatenate([[0], np.cumsum(c)]).astype(np.int64)


# ----------------------------------------------------------------- scenes --
def _rmf_normals(points: np.ndarray, n0: np.ndarray) -> np.ndarray:
    """Reference normals of the pieces of a polyline, carried from n0 by the
    double-reflection rule for rotation-minimising frames (Wang, Juettler,
    Zheng, Liu 2008): reflect across the plane bisecting consecutive piece
    starts, then across the plane bisecting the two tangents."""
    t = np.diff(points, axis=0)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    out = np.zeros_like(t)
    r = n0 - t[0] * (n0 @ t[0])
    out[0] = r / np.linalg.norm(r)
    for k in range(len(t) - 1):
        v1 = points[k + 1] - points[k]
        c1 = v1 @ v1
        rl = out[k] - (2.0 / c1) * (v1 @ out[k]) * v1
        tl = t[k] - (2.0 / c1) * (v1 @ t[k]) * v1
        v2 = t[k + 1] - tl
        c2 = v2 @ v2
        rn = rl - (2.0 / c2) * (v2 @ rl) * v2 if c2 > 1e-30 else rl
        rn -= t[k + 1] * (rn @ t[k + 1])
        out[k + 1] = rn / np.linalg.norm(rn)
    return out


def woven_scene(n_yarns: int = 16, pieces: int = 16, radius: float = 1.0,
                spacing: float = 2.5, lift: float = 0.6, n_mat: int = 8,
                seed: int = 0) -> list[dict]:
    """A plain-weave patch: n_yarns warp yarns along x and n_yarns weft yarns
    along y, each a polyline of straight pieces alternating over (+lift) and
    under (-lift) at the crossings; materials drawn per yarn.  Returns the
    pieces as dicts (p0, t, n_ref, length, radius, v0, mat_id)."""
    g = np.random.Generator(np.random.Philox(key=[SEED_BASE + 500, seed]))
    ids = g.integers(0, n_mat, 2 * n_yarns)
    out = []
    span = np.arange(pieces + 1) * spacing
    for axis in (0, 1):
        for j in range(n_yarns):
            z = np.where((np.arange(pieces + 1) + j + axis) % 2 == 0, lift, -lift)
            pts = np.zeros((pieces + 1, 3))
            pts[:, axis] = span
            pts[:, 1 - axis] = (j + 0.5) * spacing
            pts[:, 2] = z
            nref = _rmf_normals(pts, np.array([0.0, 0.0, 1.0]))
            v0 = 0.0
            for k in range(pieces):
                d = pts[k + 1] - pts[k]
                L = float(np.linalg.norm(d))
                out.append(dict(p0=pts[k].tolist(), t=(d / L).tolist(), n_ref=nref[k].tolist(),
                                length=L, radius=radius, v0=v0,
                                mat_id=int(ids[axis * n_yarns + j])))
                v0 += L
    return out


def camera_rays(width: int, height: int, extent: float, elevation_deg: float = 55.0,
                distance: float | None = None, fov_deg: float = 30.0,
                jitter_seed: int | None = None) -> dict:
    """Pinhole camera over a square patch [0, extent]^2 at z = 0, looking at
    its centre from the given elevation (by default from the distance at
    which the patch's inner 80% fills the image width); rays o, d as float32
    [3, n] planes (row-major pixels) and two differential rays through the
    pixel's opposite corners (o1, d1, o2, d2)."""
    c = np.array([extent / 2, extent / 2, 0.0])
    if distance is None:
        distance = 0.4 * extent / math.tan(math.radians(fov_deg) / 2)
    el = math.radians(elevation_deg)
    eye = c + distance * np.array([0.0, -math.cos(el), math.sin(el)])
    fwd = (c - eye) / np.linalg.norm(c - eye)
    right = np.cross(fwd, [0.0, 0.0, 1.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    tan_h = math.tan(math.radians(fov_deg) / 2)
    ys, xs = np.mgrid[0:height, 0:width]
    px, py = xs.ravel().astype(np.float64), ys.ravel().astype(np.float64)
    if jitter_seed is not None:
        g = np.random.Generator(np.random.Philox(key=[SEED_BASE + 501, jitter_seed]))
        px = px + g.random(px.size) - 0.5
        py = py + g.random(py.size) - 0.5

    def dirs(ox, oy):
        sx = ((px + 0.5 + ox) / width * 2 - 1) * tan_h
        sy = (1 - (py + 0.5 + oy) / height * 2) * tan_h * height / width
        d = fwd[:, None] + right[:, None] * sx + up[:, None] * sy
        return (d / np.linalg.norm(d, axis=0)).astype(np.float32)
    n = px.size
    o = np.repeat(eye[:, None], n, axis=1).astype(np.float32)
    return dict(o=o, d=dirs(0.0, 0.0), o1=o, d1=dirs(0.5, 0.5), o2=o, d2=dirs(-0.5, -0.5))
