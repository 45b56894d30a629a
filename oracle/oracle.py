"""ctypes binding of the FP64 oracle (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bysdf_oracle.cpp")
_HDR = os.path.join(_HERE, "bysdf_oracle.h")
_SRC_TRACE = os.path.join(_HERE, "yarn_trace.cpp")
_HDR_TRACE = os.path.join(_HERE, "yarn_trace.h")
_LIB = os.path.join(_HERE, "liboracle.so")
NPARAM = 8
NPARAM_EXT = 15   # NPARAM, then r, k^B_y (RGB), sigma_t, B, k_spec
_lock = threading.Lock()
_lib = None


class Material(C.Structure):
    _fields_ = [
        ("n_plies", C.c_int32),
        ("fibers_per_ply", C.c_int32),
        ("map_texels", C.c_int32),
        ("trace_iters", C.c_int32),
        ("k_max", C.c_int32),
        ("flags", C.c_int32),
        ("yarn_radius", C.c_double),
        ("ply_twist_deg", C.c_double),
        ("fiber_twist_deg", C.c_double),
        ("eta", C.c_double),
        ("albedo", C.c_double * 3),
        ("k_spec", C.c_double),
        ("beta_deg", C.c_double * 2),
        ("body_B", C.c_double),
        ("body_r", C.c_double),
        ("sigma_t", C.c_double),
        ("shadow_density", C.c_double),
        ("packing", C.c_double),
        ("albedo_y", C.c_double * 3),
        ("migration_maps", C.c_int32),
        ("migration_seed", C.c_int32),
        ("migration_length", C.c_double),
        ("migration_blend", C.c_double),
    ]


class Yarn(C.Structure):
    _fields_ = [("p0", C.c_double * 3), ("t", C.c_double * 3), ("n_ref", C.c_double * 3),
                ("length", C.c_double), ("radius", C.c_double), ("v0", C.c_double),
                ("mat_id", C.c_int32), ("pad", C.c_int32)]


class RayPlanes(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("o", "d", "o1", "d1", "o2", "d2")]


class Records(C.Structure):
    _fields_ = [
        ("h", C.c_void_p),
        ("u", C.c_void_p),
        ("v", C.c_void_p),
        ("wi", C.c_void_p),
        ("wo", C.c_void_p),
        ("ratio", C.c_void_p),
        ("u0", C.c_void_p),
        ("u1", C.c_void_p),
        ("mat_id", C.c_void_p),
    ]


class Geo(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("n_nodes", C.c_int32),
        ("n_hit_nodes", C.c_int32),
        ("ply", C.c_int32),
        ("h1", C.c_double),
        ("h2", C.c_double),
        ("ni_mean", C.c_double),
        ("t_ply", C.c_double * 8),
        ("x", C.c_double * 3),
        ("n_p", C.c_double * 3),
        ("t_p", C.c_double * 3),
        ("n_f", C.c_double * 3),
        ("t_f", C.c_double * 3),
        ("g_p", C.c_double),
        ("g_f", C.c_double),
        ("g_mean", C.c_double),
        ("u_ply", C.c_double),
        ("delta", C.c_double),
        ("o_f", C.c_double),
        ("residual", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (IEEE double, no FMA contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or any(
            os.path.getmtime(p) > os.path.getmtime(_LIB)
            for p in (_SRC, _HDR, _SRC_TRACE, _HDR_TRACE))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call([
                "g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC",
                "-shared", "-o", tmp, _SRC, _SRC_TRACE, "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        MP = C.POINTER(Material)
        RP = C.POINTER(Records)
        L.orc_eval.argtypes = [MP, C.c_int, RP, C.c_int64, P, P, P, C.c_int]
        L.orc_pdf.argtypes = [MP, C.c_int, RP, C.c_int64, P, P, C.c_int]
        L.orc_sample.argtypes = [MP, C.c_int, RP, C.c_int64, P, P, P, P, C.c_int]
        L.orc_grad.argtypes = [MP, C.c_int, RP, C.c_int64, P, P, P, P, C.c_int]
        L.orc_grad_ext.argtypes = [MP, C.c_int, RP, C.c_int64, P, P, P, P, P, P, C.c_int]
        L.orc_eval_stochastic.argtypes = [MP, C.c_int, RP, C.c_int64, C.c_uint64, C.c_int64,
                                          C.c_uint32, P, P, P, C.c_int]
        L.orc_sample_stochastic.argtypes = [MP, C.c_int, RP, C.c_int64, C.c_uint64, C.c_int64,
                                            C.c_uint32, P, P, P, P, C.c_int]
        L.orc_stoch_nodes.argtypes = [C.c_double, C.c_int, C.c_double, C.c_int, C.c_uint64,
                                      C.c_uint64, P]
        L.orc_philox4x64.argtypes = [P, P, P]
        L.orc_set_internal_offsets.argtypes = [C.c_double, C.c_double]
        L.orc_set_internal_offsets.restype = None
        L.orc_margins.argtypes = [MP, C.c_int, RP, C.c_int64, C.c_int, C.c_uint64, C.c_int64,
                                  C.c_uint32, P, C.c_int]
        L.orc_trace_yarns.argtypes = [P, C.c_int, C.POINTER(RayPlanes), C.c_int64, P, P, P, P,
                                      P, P, P, P, P, P, C.c_int]
        L.orc_migration_info.argtypes = [MP, C.c_int, C.c_int64, P]
        L.orc_migration_texels.argtypes = [MP, C.c_int, P, P]
        L.orc_philox4x64.restype = None
        L.orc_count_ops.argtypes = [MP, C.c_int, RP, C.c_int64, C.c_int, P]
        L.orc_geometry.argtypes = [MP, C.c_float, C.c_float, C.c_float, P, C.c_float,
                                   C.POINTER(Geo)]
        L.orc_layout.argtypes = [MP, P]
        L.orc_fiber_map.argtypes = [MP, C.c_double, P]
        L.orc_fiber_map_tab.argtypes = [MP, C.c_double, P]
        L.orc_ply_occlusion.argtypes = [MP, C.c_int, C.c_double, P, P]
        L.orc_ply_occlusion.restype = C.c_double
        L.orc_fresnel.argtypes = [C.c_double, C.c_double]
        L.orc_fresnel.restype = C.c_double
        L.orc_ggx_d.argtypes = [P, C.c_double, C.c_double]
        L.orc_ggx_d.restype = C.c_double
        L.orc_ggx_g1.argtypes = [P, P, C.c_double, C.c_double]
        L.orc_ggx_g1.restype = C.c_double
        L.orc_vndf_sample.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double, P]
        L.orc_vndf_pdf.argtypes = [P, P, C.c_double, C.c_double]
        L.orc_vndf_pdf.restype = C.c_double
        L.orc_lobes.argtypes = [MP, P, P, C.c_double, C.c_double, C.c_double, P, P, P]
        L.orc_btdf.argtypes = [P, P, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_btdf.restype = C.c_double
        _lib = L
    return _lib


# ----------------------------------------------------------------- marshalling
def _material(d: dict) -> Material:
    m = Material()
    m.n_plies = int(d["n_plies"])
    m.fibers_per_ply = int(d["fibers_per_ply"])
    m.map_texels = int(d["map_texels"])
    m.trace_iters = int(d["trace_iters"])
    m.k_max = int(d["k_max"])
    m.flags = int(d.get("flags", 0))
    # float32 descriptor values widened exactly, as the GPU path receives them
    f = lambda k: float(np.float32(d[k]))  # noqa: E731
    m.yarn_radius = f("yarn_radius")
    m.ply_twist_deg = f("ply_twist_deg")
    m.fiber_twist_deg = f("fiber_twist_deg")
    m.eta = f("eta")
    for c in range(3):
        m.albedo[c] = float(np.float32(d["albedo"][c]))
    m.k_spec = f("k_spec")
    for c in range(2):
        m.beta_deg[c] = float(np.float32(d["beta_deg"][c]))
    m.body_B = f("body_B")
    m.body_r = f("body_r")
    m.sigma_t = f("sigma_t")
    m.shadow_density = f("shadow_density")
    m.packing = f("packing")
    ay = d.get("albedo_y")
    for c in range(3):
        m.albedo_y[c] = -1.0 if ay is None else float(np.float32(ay[c]))
    m.migration_maps = int(d.get("migration_maps", 1))
    m.migration_seed = int(d.get("migration_seed", 0))
    m.migration_length = float(np.float32(d.get("migration_length", 1.0)))
    m.migration_blend = float(np.float32(d.get("migration_blend", 0.25)))
    return m


def _materials(mats):
    arr = (Material * len(mats))()
    for i, d in enumerate(mats):
        arr[i] = _material(d)
    return arr


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _records(rec: dict, keep: list):
    """Records dict (numpy planes) -> ctypes struct; `keep` pins the arrays."""
    r = Records()
    n = len(rec["h"])
    for k in ("h", "u", "v"):
        a = _f32(rec[k]); keep.append(a); setattr(r, k, a.ctypes.data)
    for k in ("wi", "wo"):
        a = rec.get(k)
        if a is not None:
            a = _f32(a).reshape(3, n); keep.append(a); setattr(r, k, a.ctypes.data)
    for k in ("ratio", "u0", "u1"):
        a = rec.get(k)
        if a is not None:
            a = _f32(a); keep.append(a); setattr(r, k, a.ctypes.data)
    mid = rec.get("mat_id")
    if mid is not None:
        mid = np.ascontiguousarray(mid, dtype=np.int32); keep.append(mid)
        r.mat_id = mid.ctypes.data
    return r, n


def eval_records(mats, rec, threads: int = 1):
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    f = np.zeros((3, n)); pdf = np.zeros(n); st = np.zeros(n, np.uint8)
    rc = lib().orc_eval(M, len(mats), C.byref(r), n, f.ctypes.data, pdf.ctypes.data,
                        st.ctypes.data, threads)
    if rc:
        raise ValueError("oracle: bad material description")
    return f, pdf, st


def pdf_records(mats, rec, threads: int = 1):
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    pdf = np.zeros(n); st = np.zeros(n, np.uint8)
    if lib().orc_pdf(M, len(mats), C.byref(r), n, pdf.ctypes.data, st.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return pdf, st


def sample_records(mats, rec, threads: int = 1):
    keep = []
    M = _materials(mats)
    rec = dict(rec); rec.pop("wo", None)
    r, n = _records(rec, keep)
    wo = np.zeros((3, n)); w = np.zeros((3, n)); pdf = np.zeros(n)
    ls = np.zeros(n, np.uint8)
    if lib().orc_sample(M, len(mats), C.byref(r), n, wo.ctypes.data, w.ctypes.data,
                        pdf.ctypes.data, ls.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return wo, w, pdf, ls & 15, ls >> 4


def grad_records(mats, rec, g_rgb, threads: int = 1, jac: bool = False):
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    g = np.ascontiguousarray(g_rgb, dtype=np.float64).reshape(3, n)
    grad = np.zeros((len(mats), NPARAM)); f = np.zeros((3, n))
    J = np.zeros((n, 3, NPARAM)) if jac else None
    if lib().orc_grad(M, len(mats), C.byref(r), n, g.ctypes.data, grad.ctypes.data,
                      None if J is None else J.ctypes.data, f.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return (grad, f, J) if jac else (grad, f)


def grad_ext_records(mats, rec, g_rgb, threads: int = 1, jac: bool = False):
    """15 parameter gradients [n_mat, 15], the direction vector-Jacobian
    products g_wi, g_wo [3, n], f [3, n] (and jac [n, 3, 21])."""
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    g = np.ascontiguousarray(g_rgb, dtype=np.float64).reshape(3, n)
    grad = np.zeros((len(mats), NPARAM_EXT)); f = np.zeros((3, n))
    gwi = np.zeros((3, n)); gwo = np.zeros((3, n))
    J = np.zeros((n, 3, NPARAM_EXT + 6)) if jac else None
    if lib().orc_grad_ext(M, len(mats), C.byref(r), n, g.ctypes.data, grad.ctypes.data,
                          gwi.ctypes.data, gwo.ctypes.data,
                          None if J is None else J.ctypes.data, f.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return (grad, gwi, gwo, f, J) if jac else (grad, gwi, gwo, f)


STOCH_JITTER_NODES, STOCH_ROUGH_ENTRY = 1, 2


def eval_stochastic_records(mats, rec, seed: int, flags: int, index_offset: int = 0,
                            threads: int = 1):
    """Stochastic estimators (jittered nodes, rough entry): f, pdf, status."""
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    f = np.zeros((3, n)); pdf = np.zeros(n); st = np.zeros(n, np.uint8)
    if lib().orc_eval_stochastic(M, len(mats), C.byref(r), n, seed, index_offset, flags,
                                 f.ctypes.data, pdf.ctypes.data, st.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return f, pdf, st


def sample_stochastic_records(mats, rec, seed: int, flags: int, index_offset: int = 0,
                              threads: int = 1):
    keep = []
    M = _materials(mats)
    rec = dict(rec); rec.pop("wo", None)
    r, n = _records(rec, keep)
    wo = np.zeros((3, n)); w = np.zeros((3, n)); pdf = np.zeros(n)
    ls = np.zeros(n, np.uint8)
    if lib().orc_sample_stochastic(M, len(mats), C.byref(r), n, seed, index_offset, flags,
                                   wo.ctypes.data, w.ctypes.data, pdf.ctypes.data,
                                   ls.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return wo, w, pdf, ls & 15, ls >> 4


MG_N = 10
MARGIN_CLASSES = ("graze", "gap", "cusp", "axis", "hemi", "exit", "lobe", "sample", "shadow",
                  "kink")


def margins(mats, rec, op: str = "eval", seed: int = 0, flags: int = 0, index_offset: int = 0,
            threads: int = 1) -> np.ndarray:
    """Discontinuity margins of each record (bysdf_oracle.h, orc_margins):
    [ORC_MG_N, n], the smallest distance of a deciding quantity from its
    branch threshold per class (MARGIN_CLASSES order; +inf where a record
    never reaches the class).  op: "eval" (f and pdf at omega_o) or "sample"
    (one sample from u0, u1); flags != 0 follows the stochastic estimators."""
    keep = []
    M = _materials(mats)
    rec = dict(rec)
    if op == "sample":
        rec.pop("wo", None)
    r, n = _records(rec, keep)
    out = np.zeros((n, MG_N))
    if lib().orc_margins(M, len(mats), C.byref(r), n, 0 if op == "eval" else 1, seed,
                         index_offset, flags, out.ctypes.data, threads):
        raise ValueError("oracle: bad material description")
    return np.ascontiguousarray(out.T)


class internal_offsets:
    """Context manager: evaluations inside it see the in-plane hit distance
    moved by dt and the ply azimuth by du_ply radians (orc_set_internal_offsets)."""

    def __init__(self, dt: float = 0.0, du_ply: float = 0.0):
        self.dt, self.du = dt, du_ply

    def __enter__(self):
        lib().orc_set_internal_offsets(self.dt, self.du)
        return self

    def __exit__(self, *exc):
        lib().orc_set_internal_offsets(0.0, 0.0)
        return False


def margin(mats, rec, op: str = "eval", **kw) -> np.ndarray:
    """The smallest margin over all classes, per record."""
    return margins(mats, rec, op, **kw).min(axis=0)


def stoch_nodes(h0, ratio, k_max, seed, index):
    out = np.zeros(64)
    K = lib().orc_stoch_nodes(float(np.float32(h0)), 1, float(np.float32(ratio)), k_max,
                              seed, index, out.ctypes.data)
    return out[:K]


def migration_info(mat, k: int, seg: int = 0):
    out = np.zeros(3)
    if lib().orc_migration_info(C.byref(_material(mat)), k, seg, out.ctypes.data):
        raise ValueError("oracle: bad material description or map index")
    return dict(Rfc=out[0], M=int(out[1]), map_of_segment=int(out[2]))


def migration_texels(mat, k: int):
    T = int(mat["map_texels"])
    dl = np.zeros(T); of = np.zeros(T)
    if lib().orc_migration_texels(C.byref(_material(mat)), k, dl.ctypes.data, of.ctypes.data):
        raise ValueError("oracle: bad material description or map index")
    return dl, of


def trace_yarns(yarns, rays: dict, light, threads: int = 1) -> dict:
    """Camera rays against yarn pieces (yarn_trace.h).  yarns: list of dicts
    (p0, t, n_ref, length, radius, v0, mat_id); rays: float32 [3, n] planes
    o, d and optionally o1, d1, o2, d2."""
    arr = (Yarn * len(yarns))()
    for k, yd in enumerate(yarns):
        for f in ("p0", "t", "n_ref"):
            for c in range(3):
                getattr(arr[k], f)[c] = float(np.float32(yd[f][c]))
        arr[k].length = float(np.float32(yd["length"]))
        arr[k].radius = float(np.float32(yd["radius"]))
        arr[k].v0 = float(np.float32(yd["v0"]))
        arr[k].mat_id = int(yd["mat_id"])
    keep = []
    rp = RayPlanes()
    n = int(np.asarray(rays["o"]).shape[1])
    for k in ("o", "d", "o1", "d1", "o2", "d2"):
        if rays.get(k) is not None:
            a = np.ascontiguousarray(rays[k], dtype=np.float32).reshape(3, n)
            keep.append(a)
            setattr(rp, k, a.ctypes.data)
    out = {k: np.zeros(n) for k in ("h", "u", "v", "ratio", "t_hit")}
    out["wi"] = np.zeros((3, n)); out["wo"] = np.zeros((3, n))
    out["yarn"] = np.zeros(n, np.int32); out["mat_id"] = np.zeros(n, np.int32)
    lt = np.ascontiguousarray(light, dtype=np.float64)
    lib().orc_trace_yarns(arr, len(yarns), C.byref(rp), n, lt.ctypes.data,
                          *(out[k].ctypes.data for k in ("h", "u", "v", "wi", "wo", "ratio",
                                                         "t_hit", "yarn", "mat_id")), threads)
    return out


def philox4x64(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def count_ops(mats, rec, op: int = 0):
    keep = []
    M = _materials(mats)
    r, n = _records(rec, keep)
    out = np.zeros((n, 6))
    if lib().orc_count_ops(M, len(mats), C.byref(r), n, op, out.ctypes.data):
        raise ValueError("oracle: bad material description")
    return out


def geometry(mat, h, u, v, wi, ratio=-1.0):
    g = Geo()
    wi = np.ascontiguousarray(wi, dtype=np.float32)
    if lib().orc_geometry(C.byref(_material(mat)), h, u, v, wi.ctypes.data, ratio, C.byref(g)):
        raise ValueError("oracle: bad material description")
    return {k: (np.array(getattr(g, k)) if isinstance(getattr(g, k), C.Array) else getattr(g, k))
            for k, _ in Geo._fields_}


def layout(mat):
    out = np.zeros(7)
    if lib().orc_layout(C.byref(_material(mat)), out.ctypes.data):
        raise ValueError("oracle: bad material description")
    return dict(Rp=out[0], Rc=out[1], rf=out[2], Rfc=out[3], M=int(out[4]),
                omega_p=out[5], omega_f=out[6])


def fiber_map(mat, D):
    out = np.zeros(2)
    if lib().orc_fiber_map(C.byref(_material(mat)), float(D), out.ctypes.data):
        raise ValueError("oracle: bad material description")
    return out[0], out[1]


def fiber_map_tab(mat, theta):
    out = np.zeros(2)
    if lib().orc_fiber_map_tab(C.byref(_material(mat)), float(theta), out.ctypes.data):
        raise ValueError("oracle: bad material description")
    return out[0], out[1]


def ply_occlusion(mat, k, z, x, w):
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_ply_occlusion(C.byref(_material(mat)), int(k), float(z), x.ctypes.data,
                                   w.ctypes.data)


def fresnel(cos_i, eta):
    return lib().orc_fresnel(float(cos_i), float(eta))


def _v(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def ggx_d(m, at, ab):
    m = _v(m)
    return lib().orc_ggx_d(m.ctypes.data, at, ab)


def ggx_g1(w, m, at, ab):
    w = _v(w); m = _v(m)
    return lib().orc_ggx_g1(w.ctypes.data, m.ctypes.data, at, ab)


def vndf_sample(w, at, ab, u0, u1):
    w = _v(w); out = np.zeros(3)
    lib().orc_vndf_sample(w.ctypes.data, at, ab, u0, u1, out.ctypes.data)
    return out


def vndf_pdf(w, m, at, ab):
    w = _v(w); m = _v(m)
    return lib().orc_vndf_pdf(w.ctypes.data, m.ctypes.data, at, ab)


def lobes(mat, frame, x, g, ni, width, wi, wo):
    fr = _v(frame).reshape(9); x = _v(x); wi = _v(wi); wo = _v(wo); out = np.zeros(8)
    if lib().orc_lobes(C.byref(_material(mat)), fr.ctypes.data, x.ctypes.data, g, ni, width,
                       wi.ctypes.data, wo.ctypes.data, out.ctypes.data):
        raise ValueError("oracle: bad material description")
    return dict(R=out[0], TT=out[1], xB=out[2:5].copy(), yB=out[5:8].copy())


def btdf(i, o, eta_i, eta_o, at, ab):
    i = _v(i); o = _v(o)
    return lib().orc_btdf(i.ctypes.data, o.ctypes.data, eta_i, eta_o, at, ab)
