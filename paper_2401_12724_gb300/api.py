"""PyTorch-facing binding of libbysdf.

Argument marshalling only: tensors are passed to the C ABI as raw device
pointers and every step of the BYSDF runs in the library's CUDA kernels.
Records are a dict of CUDA tensors: h, u, v (n,), wi, wo (3, n) float32,
optional mat_id (n,) int32, ratio (n,) float32, seg_offsets (n_mat + 1,)
int64.  Outputs are allocated here with torch (device memory is plumbing).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _native as N

PARAM_NAMES = ("albedo_r", "albedo_g", "albedo_b", "beta_t", "beta_b", "alpha_p", "alpha_f",
               "sigma_s")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def desc_struct(d: dict) -> N.MaterialDesc:
    s = N.MaterialDesc()
    for k in ("n_plies", "fibers_per_ply", "map_texels", "trace_iters", "k_max"):
        setattr(s, k, int(d[k]))
    s.flags = int(d.get("flags", 0))
    for k in ("yarn_radius", "ply_twist_deg", "fiber_twist_deg", "eta", "k_spec", "body_B",
              "body_r", "sigma_t", "shadow_density", "packing"):
        setattr(s, k, float(d[k]))
    for c in range(3):
        s.albedo[c] = float(d["albedo"][c])
    for c in range(2):
        s.beta_deg[c] = float(d["beta_deg"][c])
    ay = d.get("albedo_y")
    for c in range(3):
        s.albedo_y[c] = -1.0 if ay is None else float(ay[c])
    s.migration_maps = int(d.get("migration_maps", 1))
    s.migration_seed = int(d.get("migration_seed", 0))
    s.migration_length = float(d.get("migration_length", 1.0))
    s.migration_blend = float(d.get("migration_blend", 0.25))
    return s


class Materials:
    """Device-resident material table (bysdf_create_materials)."""

    def __init__(self, descs, device=None, stream=None):
        self.lib = N.load()
        self.device = torch.device(device if device is not None else "cuda")
        self.descs = [dict(d) for d in descs]
        arr = (N.MaterialDesc * len(descs))(*[desc_struct(d) for d in descs])
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            N.check(self.lib.bysdf_create_materials(arr, len(descs), _stream(stream), C.byref(h)),
                    "bysdf_create_materials")
        self.handle = h
        self.n_mat = len(descs)
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            self.lib.bysdf_destroy_materials(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, n: int) -> torch.Tensor:
        need = int(self.lib.bysdf_workspace_size(self.handle, int(n)))
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def set_params(self, params: torch.Tensor, stream=None):
        p = params.detach().to(device=self.device, dtype=torch.float32).contiguous()
        assert p.shape == (self.n_mat, 8)
        N.check(self.lib.bysdf_set_params(self.handle, _ptr(p), _stream(stream)), "bysdf_set_params")
        self._params_keepalive = p

    def get_params(self, stream=None) -> torch.Tensor:
        p = torch.empty(self.n_mat, 8, dtype=torch.float32, device=self.device)
        N.check(self.lib.bysdf_get_params(self.handle, _ptr(p), _stream(stream)), "bysdf_get_params")
        return p

    def set_params_ext(self, params: torch.Tensor, stream=None):
        """The 15 parameters of the extended set (bysdf_set_params_ext)."""
        p = params.detach().to(device=self.device, dtype=torch.float32).contiguous()
        assert p.shape == (self.n_mat, N.NPARAM_EXT)
        N.check(self.lib.bysdf_set_params_ext(self.handle, _ptr(p), _stream(stream)),
                "bysdf_set_params_ext")
        self._params_keepalive = p

    def get_params_ext(self, stream=None) -> torch.Tensor:
        p = torch.empty(self.n_mat, N.NPARAM_EXT, dtype=torch.float32, device=self.device)
        N.check(self.lib.bysdf_get_params_ext(self.handle, _ptr(p), _stream(stream)),
                "bysdf_get_params_ext")
        return p

    def set_launch_config(self, op: int, block: int, items: int, ctas_per_sm: int = 0,
                          occupancy: int = 0):
        c = N.LaunchConfig(block, items, ctas_per_sm, occupancy)
        N.check(self.lib.bysdf_set_launch_config(self.handle, op, C.byref(c)), "set_launch_config")

    def launch_config(self, op: int) -> dict:
        c = N.LaunchConfig()
        N.check(self.lib.bysdf_get_launch_config(self.handle, op, C.byref(c)), "get_launch_config")
        return dict(block=c.block, items=c.items, ctas_per_sm=c.ctas_per_sm,
                    occupancy=c.occupancy)

    def test_stall_table_waits(self, polls: int):
        """Test hook of the device-side error path (bysdf_test_stall_table_waits):
        table waits give up after `polls` polls; 0 switches it off."""
        N.check(self.lib.bysdf_test_stall_table_waits(self.handle, int(polls)),
                "bysdf_test_stall_table_waits")

    def workspace_error(self, stream=None) -> int:
        err = C.c_uint32(0)
        ws = self.workspace(0)
        N.check(self.lib.bysdf_workspace_error(_ptr(ws), _stream(stream), C.byref(err)),
                "bysdf_workspace_error")
        return int(err.value)


def hits_struct(rec: dict, sample: bool = False) -> N.Hits:
    h = N.Hits()
    h.h = _ptr(rec["h"])
    h.u = _ptr(rec["u"])
    h.v = _ptr(rec["v"])
    h.wi = _ptr(rec["wi"])
    h.wo = None if sample else _ptr(rec.get("wo"))
    h.ratio = _ptr(rec.get("ratio"))
    h.mat_id = _ptr(rec.get("mat_id"))
    h.seg_offsets = _ptr(rec.get("seg_offsets"))
    return h


def records_to_device(rec: dict, device="cuda", seg_offsets=None) -> dict:
    """numpy planes (see inputs.records) -> CUDA tensors."""
    out = {}
    for k, a in rec.items():
        t = torch.from_numpy(np.ascontiguousarray(a))
        out[k] = t.to(device)
    if seg_offsets is not None:
        out["seg_offsets"] = torch.from_numpy(np.asarray(seg_offsets, np.int64)).to(device)
    return out


def _n(rec) -> int:
    return int(rec["h"].shape[0])


def _empty(shape, dtype, dev):
    return torch.empty(shape, dtype=dtype, device=dev)


def eval(mats: Materials, rec: dict, with_pdf: bool = True, stream=None, out=None):
    """f |wo.n| (3, n), pdf (n,) and status (n,) uint8."""
    n = _n(rec)
    dev = rec["h"].device
    f = out["f"] if out else _empty((3, n), torch.float32, dev)
    pdf = (out["pdf"] if out else _empty((n,), torch.float32, dev)) if with_pdf else None
    st = out["status"] if out else _empty((n,), torch.uint8, dev)
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval(mats.handle, C.byref(hits_struct(rec)), n, _ptr(f), _ptr(pdf),
                                _ptr(st), _ptr(ws), ws.numel(), _stream(stream)), "bysdf_eval")
    return f, pdf, st


def sample(mats: Materials, rec: dict, u0=None, u1=None, stream=None, out=None):
    """wo (3, n), weight (3, n), pdf (n,), lobe << 4 | status (n,)."""
    n = _n(rec)
    dev = rec["h"].device
    u0 = rec["u0"] if u0 is None else u0
    u1 = rec["u1"] if u1 is None else u1
    if out:
        wo, w, p, ls = out["wo"], out["weight"], out["pdf"], out["lobe_status"]
    else:
        wo, w = _empty((3, n), torch.float32, dev), _empty((3, n), torch.float32, dev)
        p, ls = _empty((n,), torch.float32, dev), _empty((n,), torch.uint8, dev)
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_sample(mats.handle, C.byref(hits_struct(rec, sample=True)), _ptr(u0),
                                  _ptr(u1), n, _ptr(wo), _ptr(w), _ptr(p), _ptr(ls), _ptr(ws),
                                  ws.numel(), _stream(stream)), "bysdf_sample")
    return wo, w, p, ls


def pdf(mats: Materials, rec: dict, stream=None, out=None):
    n = _n(rec)
    dev = rec["h"].device
    p = out["pdf"] if out else _empty((n,), torch.float32, dev)
    st = out["status"] if out else _empty((n,), torch.uint8, dev)
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_pdf(mats.handle, C.byref(hits_struct(rec)), n, _ptr(p), _ptr(st),
                               _ptr(ws), ws.numel(), _stream(stream)), "bysdf_pdf")
    return p, st


def alloc_fused(n: int, dev) -> dict:
    return dict(f=_empty((3, n), torch.float32, dev), pdf=_empty((n,), torch.float32, dev),
                status=_empty((n,), torch.uint8, dev), wo=_empty((3, n), torch.float32, dev),
                weight=_empty((3, n), torch.float32, dev), pdf_s=_empty((n,), torch.float32, dev),
                lobe_status=_empty((n,), torch.uint8, dev))


def eval_sample_pdf(mats: Materials, rec: dict, u0=None, u1=None, stream=None, out=None) -> dict:
    """Fused eval + pdf at rec['wo'] and a sample from (u0, u1)."""
    n = _n(rec)
    o = out if out is not None else alloc_fused(n, rec["h"].device)
    u0 = rec["u0"] if u0 is None else u0
    u1 = rec["u1"] if u1 is None else u1
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_sample_pdf(
        mats.handle, C.byref(hits_struct(rec)), _ptr(u0), _ptr(u1), n, _ptr(o["f"]),
        _ptr(o["pdf"]), _ptr(o["status"]), _ptr(o["wo"]), _ptr(o["weight"]), _ptr(o["pdf_s"]),
        _ptr(o["lobe_status"]), _ptr(ws), ws.numel(), _stream(stream)), "bysdf_eval_sample_pdf")
    return o


def eval_stochastic(mats: Materials, rec: dict, seed: int, flags: int, index_offset: int = 0,
                    with_pdf: bool = True, stream=None, out=None):
    """The stochastic estimators (N.STOCH_* flags): f, pdf, status as eval."""
    n = _n(rec)
    dev = rec["h"].device
    f = out["f"] if out else _empty((3, n), torch.float32, dev)
    pdf = (out["pdf"] if out else _empty((n,), torch.float32, dev)) if with_pdf else None
    st = out["status"] if out else _empty((n,), torch.uint8, dev)
    opt = N.Stochastic(int(seed), int(index_offset), int(flags), 0)
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_stochastic(mats.handle, C.byref(hits_struct(rec)), C.byref(opt),
                                           n, _ptr(f), _ptr(pdf), _ptr(st), _ptr(ws), ws.numel(),
                                           _stream(stream)), "bysdf_eval_stochastic")
    return f, pdf, st


def eval_sample_pdf_stochastic(mats: Materials, rec: dict, seed: int, flags: int,
                               index_offset: int = 0, u0=None, u1=None, stream=None,
                               out=None) -> dict:
    n = _n(rec)
    o = out if out is not None else alloc_fused(n, rec["h"].device)
    u0 = rec["u0"] if u0 is None else u0
    u1 = rec["u1"] if u1 is None else u1
    opt = N.Stochastic(int(seed), int(index_offset), int(flags), 0)
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_sample_pdf_stochastic(
        mats.handle, C.byref(hits_struct(rec)), C.byref(opt), _ptr(u0), _ptr(u1), n,
        _ptr(o["f"]), _ptr(o["pdf"]), _ptr(o["status"]), _ptr(o["wo"]), _ptr(o["weight"]),
        _ptr(o["pdf_s"]), _ptr(o["lobe_status"]), _ptr(ws), ws.numel(), _stream(stream)),
        "bysdf_eval_sample_pdf_stochastic")
    return o


def yarns_to_device(pieces, device="cuda") -> torch.Tensor:
    """Yarn pieces (dicts: p0, t, n_ref, length, radius, v0, mat_id) packed as
    the bysdf_yarn struct (64 bytes each) in device memory."""
    n = len(pieces)
    f = np.zeros((n, 16), np.float32)
    for k, y in enumerate(pieces):
        f[k, 0:3] = y["p0"]
        f[k, 3:6] = y["t"]
        f[k, 6:9] = y["n_ref"]
        f[k, 9:12] = (y["length"], y["radius"], y["v0"])
    words = f.view(np.int32)
    words[:, 12] = [int(y["mat_id"]) for y in pieces]
    words[:, 13:16] = 0
    return torch.from_numpy(words.copy()).to(device)


def trace_yarns(yarns: torch.Tensor, rays: dict, light, stream=None, out=None) -> dict:
    """Camera rays (device planes o, d and optionally o1, d1, o2, d2) against
    the packed yarn pieces: the BYSDF hit records (h, u, v, wi, wo, ratio,
    mat_id) plus yarn_id and t_hit."""
    n = int(rays["o"].shape[-1])
    dev = rays["o"].device
    o = out if out is not None else dict(
        h=_empty((n,), torch.float32, dev), u=_empty((n,), torch.float32, dev),
        v=_empty((n,), torch.float32, dev), wi=_empty((3, n), torch.float32, dev),
        wo=_empty((3, n), torch.float32, dev), ratio=_empty((n,), torch.float32, dev),
        mat_id=_empty((n,), torch.int32, dev), yarn_id=_empty((n,), torch.int32, dev),
        t_hit=_empty((n,), torch.float32, dev))
    r = N.Rays(*[_ptr(rays.get(k)) for k in ("o", "d", "o1", "d1", "o2", "d2")])
    lt = (C.c_float * 3)(*[float(x) for x in light])
    lib = N.load()
    N.check(lib.bysdf_trace_yarns(_ptr(yarns), int(yarns.shape[0]), C.byref(r), n, lt,
                                  _ptr(o["h"]), _ptr(o["u"]), _ptr(o["v"]), _ptr(o["wi"]),
                                  _ptr(o["wo"]), _ptr(o.get("ratio")), _ptr(o["mat_id"]),
                                  _ptr(o.get("yarn_id")), _ptr(o.get("t_hit")), _stream(stream)),
            "bysdf_trace_yarns")
    return o


def eval_backward(mats: Materials, rec: dict, grad_f: torch.Tensor, deterministic: bool = False,
                  stream=None, out=None) -> torch.Tensor:
    """d(sum grad_f * f) / d params, shape (n_mat, 8)."""
    n = _n(rec)
    g = out if out is not None else _empty((mats.n_mat, 8), torch.float32, rec["h"].device)
    gf = grad_f.contiguous()
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_backward(mats.handle, C.byref(hits_struct(rec)), n, _ptr(gf),
                                         _ptr(g), int(deterministic), _ptr(ws), ws.numel(),
                                         _stream(stream)), "bysdf_eval_backward")
    return g


def eval_l2_backward(mats: Materials, rec: dict, target: torch.Tensor, weight=None,
                     deterministic: bool = False, stream=None, with_f: bool = True):
    """Forward, L2 loss against target (3, n) and its parameter gradient in
    one pass (bysdf_eval_l2_backward): returns grad (n_mat, 8), per-material
    loss (n_mat,) and f (3, n) (None unless with_f)."""
    n = _n(rec)
    dev = rec["h"].device
    g = _empty((mats.n_mat, 8), torch.float32, dev)
    loss = _empty((mats.n_mat,), torch.float32, dev)
    f = _empty((3, n), torch.float32, dev) if with_f else None
    t = target.contiguous()
    w = None if weight is None else weight.contiguous()
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_l2_backward(
        mats.handle, C.byref(hits_struct(rec)), n, _ptr(t), _ptr(w), _ptr(f), _ptr(loss), _ptr(g),
        int(deterministic), _ptr(ws), ws.numel(), _stream(stream)), "bysdf_eval_l2_backward")
    return g, loss, f


def eval_backward_ext(mats: Materials, rec: dict, grad_f: torch.Tensor,
                      deterministic: bool = False, dirs: bool = False, stream=None):
    """d(sum grad_f * f) / d params for the 15-column extended set, and with
    dirs=True the per-record products grad_f . df/dwi and . df/dwo (3, n)."""
    n = _n(rec)
    dev = rec["h"].device
    g = _empty((mats.n_mat, N.NPARAM_EXT), torch.float32, dev)
    gwi = _empty((3, n), torch.float32, dev) if dirs else None
    gwo = _empty((3, n), torch.float32, dev) if dirs else None
    gf = grad_f.contiguous()
    ws = mats.workspace(n)
    N.check(mats.lib.bysdf_eval_backward_ext(
        mats.handle, C.byref(hits_struct(rec)), n, _ptr(gf), _ptr(g), _ptr(gwi), _ptr(gwo),
        int(deterministic), _ptr(ws), ws.numel(), _stream(stream)), "bysdf_eval_backward_ext")
    return g, gwi, gwo


def plain(op: int, mats: Materials, rec: dict, seg_host, stream=None, out=None) -> dict:
    """The per-material-launch comparison form (records sorted by material)."""
    n = _n(rec)
    dev = rec["h"].device
    seg = np.ascontiguousarray(seg_host, dtype=np.int64)
    o = out if out is not None else dict(
        f=_empty((3, n), torch.float32, dev), wo=_empty((3, n), torch.float32, dev),
        weight=_empty((3, n), torch.float32, dev), pdf=_empty((n,), torch.float32, dev),
        status=_empty((n,), torch.uint8, dev))
    samp = op == N.OP_SAMPLE
    N.check(mats.lib.bysdf_plain(
        op, mats.handle, C.byref(hits_struct(rec, sample=samp)), seg.ctypes.data,
        _ptr(rec.get("u0")) if samp else None, _ptr(rec.get("u1")) if samp else None, n,
        _ptr(o["f"]), _ptr(o["wo"]), _ptr(o["weight"]), _ptr(o["pdf"]), _ptr(o["status"]),
        _stream(stream)), "bysdf_plain")
    return o


def plain_fused(mats: Materials, rec: dict, seg_host, u0=None, u1=None, stream=None,
                out=None) -> dict:
    """The per-material-launch form of the fused op (bysdf_plain_fused)."""
    n = _n(rec)
    seg = np.ascontiguousarray(seg_host, dtype=np.int64)
    o = out if out is not None else alloc_fused(n, rec["h"].device)
    u0 = rec["u0"] if u0 is None else u0
    u1 = rec["u1"] if u1 is None else u1
    outs = N.Outputs(_ptr(o["f"]), _ptr(o["pdf"]), _ptr(o["status"]), _ptr(o["wo"]),
                     _ptr(o["weight"]), _ptr(o["pdf_s"]), _ptr(o["lobe_status"]), None)
    N.check(mats.lib.bysdf_plain_fused(mats.handle, C.byref(hits_struct(rec)), seg.ctypes.data,
                                       _ptr(u0), _ptr(u1), n, C.byref(outs), _stream(stream)),
            "bysdf_plain_fused")
    return o


def autotune(mats: Materials, op: int, rec: dict, out: dict | None = None, grad_f=None,
             stream=None) -> dict:
    n = _n(rec)
    dev = rec["h"].device
    o = out if out is not None else alloc_fused(n, dev)
    gp = _empty((mats.n_mat, 8), torch.float32, dev)
    outs = N.Outputs(_ptr(o["f"]), _ptr(o["pdf"]), _ptr(o["status"]), _ptr(o["wo"]),
                     _ptr(o["weight"]), _ptr(o["pdf_s"]), _ptr(o["lobe_status"]), _ptr(gp))
    ws = mats.workspace(n)
    best = N.LaunchConfig()
    samp = op == N.OP_SAMPLE
    N.check(mats.lib.bysdf_autotune(
        mats.handle, op, C.byref(hits_struct(rec, sample=samp)), _ptr(rec.get("u0")),
        _ptr(rec.get("u1")), _ptr(grad_f), n, C.byref(outs), _ptr(ws), ws.numel(),
        _stream(stream), C.byref(best)), "bysdf_autotune")
    return dict(block=best.block, items=best.items, ctas_per_sm=best.ctas_per_sm,
                occupancy=best.occupancy)


def default_params(descs) -> torch.Tensor:
    """The 8 differentiable parameters of each descriptor (angles in radians)."""
    d2r = np.pi / 180.0
    rows = [[d["albedo"][0], d["albedo"][1], d["albedo"][2], d["beta_deg"][0] * d2r,
             d["beta_deg"][1] * d2r, d["ply_twist_deg"] * d2r, d["fiber_twist_deg"] * d2r,
             d["shadow_density"]] for d in descs]
    return torch.tensor(np.asarray(rows, np.float64), dtype=torch.float32)


def default_params_ext(descs) -> torch.Tensor:
    """The 15 parameters of the extended set of each descriptor."""
    base = default_params(descs).double().numpy()
    rows = []
    for d, b in zip(descs, base):
        ay = d.get("albedo_y")
        ky = [d["albedo"][c] if (ay is None or ay[c] < 0) else ay[c] for c in range(3)]
        rows.append(list(b) + [d["body_r"], *ky, d["sigma_t"], d["body_B"], d["k_spec"]])
    return torch.tensor(np.asarray(rows, np.float64), dtype=torch.float32)


class BYSDFEval(torch.autograd.Function):
    """f = BYSDF(params; records), differentiable in the per-material
    parameters; backward runs the library's recompute-and-reduce kernel."""

    @staticmethod
    def forward(ctx, params, mats, rec, deterministic=False):
        mats.set_params(params)
        f, _, st = eval(mats, rec, with_pdf=False)
        ctx.mats, ctx.rec, ctx.det = mats, rec, deterministic
        ctx.mark_non_differentiable(st)
        return f, st

    @staticmethod
    def backward(ctx, grad_f, grad_st):
        g = eval_backward(ctx.mats, ctx.rec, grad_f.float().contiguous(), ctx.det)
        return g, None, None, None


def bysdf(params: torch.Tensor, mats: Materials, rec: dict, deterministic: bool = False):
    """Differentiable evaluation: returns f (3, n) and status (n,)."""
    return BYSDFEval.apply(params, mats, rec, deterministic)


class BYSDFL2Loss(torch.autograd.Function):
    """loss = sum_i w_i sum_c (f_c(i) - target_c(i))^2 over the records with
    status 0, differentiable in the 8 parameters; forward and backward are
    one library pass (bysdf_eval_l2_backward), whose gradient is kept for
    backward."""

    @staticmethod
    def forward(ctx, params, mats, rec, target, weight=None, deterministic=False):
        mats.set_params(params)
        g, loss, _ = eval_l2_backward(mats, rec, target, weight, deterministic, with_f=False)
        ctx.save_for_backward(g)
        return loss.sum()

    @staticmethod
    def backward(ctx, grad_loss):
        (g,) = ctx.saved_tensors
        return g * grad_loss, None, None, None, None, None


def bysdf_l2_loss(params: torch.Tensor, mats: Materials, rec: dict, target: torch.Tensor,
                  weight=None, deterministic: bool = False) -> torch.Tensor:
    """Differentiable L2 loss of the BYSDF against target radiance (scalar)."""
    return BYSDFL2Loss.apply(params, mats, rec, target, weight, deterministic)


class BYSDFEvalExt(torch.autograd.Function):
    """f = BYSDF(params15, wi, wo; records): differentiable in the 15
    parameters of the extended set and in the record directions wi, wo
    (3, n) -- the latter for inverse rendering through the hit records."""

    @staticmethod
    def forward(ctx, params, wi, wo, mats, rec, deterministic=False):
        mats.set_params_ext(params)
        r = dict(rec)
        r["wi"] = wi.detach().float().contiguous()
        r["wo"] = wo.detach().float().contiguous()
        f, _, st = eval(mats, r, with_pdf=False)
        ctx.mats, ctx.rec, ctx.det = mats, r, deterministic
        ctx.mark_non_differentiable(st)
        return f, st

    @staticmethod
    def backward(ctx, grad_f, grad_st):
        dirs = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        g, gwi, gwo = eval_backward_ext(ctx.mats, ctx.rec, grad_f.float().contiguous(), ctx.det,
                                        dirs=dirs)
        return (g, gwi if ctx.needs_input_grad[1] else None,
                gwo if ctx.needs_input_grad[2] else None, None, None, None)


def bysdf_ext(params: torch.Tensor, wi: torch.Tensor, wo: torch.Tensor, mats: Materials,
              rec: dict, deterministic: bool = False):
    """Differentiable evaluation in the extended parameters and the record
    directions: returns f (3, n) and status (n,)."""
    return BYSDFEvalExt.apply(params, wi, wo, mats, rec, deterministic)


# ------------------------------------------------------------ host buffers --
_IN_KEYS = ("h", "u", "v", "wi", "wo", "u0", "u1", "mat_id", "ratio")
_OUT_KEYS = ("f", "pdf", "status", "wo", "weight", "pdf_s", "lobe_status")


def pinned_records(rec: dict) -> dict:
    """numpy planes -> pinned host tensors (for eval_sample_pdf_host)."""
    return {k: torch.from_numpy(np.ascontiguousarray(rec[k])).pin_memory()
            for k in _IN_KEYS if k in rec}


def pinned_fused_outputs(n: int) -> dict:
    o = alloc_fused(n, "cpu")
    return {k: v.pin_memory() for k, v in o.items()}


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous host tensor")
    return t.data_ptr()


class HostPipeline:
    """Records in (pinned) host memory through the fused eval + sample kernel,
    chunk by chunk, by the library's host pipeline (bysdf_eval_sample_pdf_host):
    copy-in, kernel and copy-out of consecutive chunks overlap on the
    pipeline's own streams."""

    def __init__(self, mats: Materials, chunk: int, with_ratio: bool = False):
        self.mats = mats
        h = C.c_void_p()
        N.check(mats.lib.bysdf_host_pipeline_create(mats.handle, int(chunk), int(with_ratio),
                                                    C.byref(h)), "bysdf_host_pipeline_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self.mats.lib.bysdf_host_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, host_in: dict, host_out: dict, stream=None):
        n = int(host_in["h"].shape[0])
        hs = N.Hits()
        hs.h, hs.u, hs.v = _hptr(host_in["h"]), _hptr(host_in["u"]), _hptr(host_in["v"])
        hs.wi, hs.wo = _hptr(host_in["wi"]), _hptr(host_in["wo"])
        hs.ratio = _hptr(host_in.get("ratio"))
        hs.mat_id = _hptr(host_in.get("mat_id"))
        o = host_out
        N.check(self.mats.lib.bysdf_eval_sample_pdf_host(
            self.handle, C.byref(hs), _hptr(host_in["u0"]), _hptr(host_in["u1"]), n,
            _hptr(o["f"]), _hptr(o["pdf"]), _hptr(o["status"]), _hptr(o["wo"]),
            _hptr(o["weight"]), _hptr(o["pdf_s"]), _hptr(o["lobe_status"]), _stream(stream)),
            "bysdf_eval_sample_pdf_host")

    @staticmethod
    def bytes_per_record(host_in: dict, host_out: dict):
        n = int(host_in["h"].shape[0])
        bi = sum(t.numel() * t.element_size() for t in host_in.values()) / n
        bo = sum(t.numel() * t.element_size() for t in host_out.values()) / n
        return bi, bo
