"""Element-wise parity of the CUDA path against the FP64 oracle.

Tolerance (the contract of the GPU path): |gpu - oracle| <= 1e-6 + 1e-4 |oracle|
on eval f and pdf, 1e-4 rad on sampled directions, exact status / lobe codes.

The BYSDF has branches (closest ply, ply hit or miss, fiber-map cusp ramp,
hemisphere side, total internal reflection, lobe choice by u0).  Where a record
sits within float32 rounding of a branch, several results are correct.  Each
record is therefore also evaluated by the oracle at a few copies of its inputs
perturbed by ~2^-20 relative; a record whose oracle values move by more than a
quarter of the tolerance is "ill-conditioned": its GPU value must then lie in
the range the perturbed oracle values span (plus the tolerance), and the share
of such records is bounded.  Every other record is checked strictly.
"""
from __future__ import annotations

import numpy as np

REL, ABS = 1e-4, 1e-6
ANGLE = 1e-4


def tol(ref):
    return ABS + REL * np.abs(ref)


def perturb(rec: dict, k: int, eps: float = 2.0 ** -21, sample: bool = False) -> dict:
    """A copy of the records moved by about the GPU path's own float32
    rounding of its internal quantities: entry offset h, azimuth u and the
    direction components by ~eps (absolute), the footprint ratio by eps
    (relative), u0/u1 by eps/2.  The longitudinal position v is not moved:
    the path forms its phases from v with compensated products, so its phase
    error is far below what one ulp of v would cause."""
    g = np.random.default_rng(1000 + k)
    out = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in rec.items()}
    n = len(rec["h"])

    def r(*shape):
        return g.uniform(-1.0, 1.0, shape)
    out["h"] = np.clip(rec["h"] + eps * r(n), -1, 1).astype(np.float32)
    out["u"] = (rec["u"] + eps * r(n)).astype(np.float32)
    for key in ("wi", "wo"):
        if key in rec and rec[key] is not None:
            w = rec[key].astype(np.float64) + eps * r(3, n)
            out[key] = (w / np.linalg.norm(w, axis=0)).astype(np.float32)
    if "ratio" in rec:
        out["ratio"] = (rec["ratio"] * (1 + eps * r(n))).astype(np.float32)
    if sample:
        for key in ("u0", "u1"):
            out[key] = np.clip(rec[key] + 0.5 * eps * r(n), 0.0, 1 - 2.0 ** -24).astype(np.float32)
    return out


def dump(name: str, **arrays):
    """Save raw arrays for offline analysis when BYSDF_PARITY_DUMP is set."""
    import os
    d = os.environ.get("BYSDF_PARITY_DUMP")
    if d:
        os.makedirs(d, exist_ok=True)
        np.savez_compressed(os.path.join(d, name + ".npz"),
                            **{k: np.asarray(v) for k, v in arrays.items()})


def conditioning(orc_fn, rec: dict, n_pert: int = 6, sample: bool = False):
    """Oracle outputs at the record and at n_pert perturbed copies.
    orc_fn(rec) -> tuple of arrays (last axis = record)."""
    base = orc_fn(rec)
    pert = [orc_fn(perturb(rec, k, sample=sample)) for k in range(n_pert)]
    return base, pert


def split_conditioned(base_vals, pert_vals, base_status, pert_status, frac: float = 0.25):
    """Mask of well-conditioned records: all value arrays move by at most
    frac * tol and the status never changes under the perturbations."""
    good = np.ones(base_status.shape, bool)
    for ps in pert_status:
        good &= ps == base_status
    for b, ps in zip(base_vals, zip(*pert_vals)):
        for p in ps:
            d = np.abs(p - b)
            if d.ndim > 1:
                d = d.max(axis=0)
                t = tol(np.abs(b).max(axis=0))
            else:
                t = tol(b)
            good &= d <= frac * t
    return good


def _per_record(mask):
    return mask if mask.ndim == 1 else mask.any(axis=0)


def assert_close_conditioned(gpu, base, pert, good, name, max_ill=0.03):
    """Strict on well-conditioned records; bracketed by the perturbed oracle
    values on the others; at most max_ill of the records ill-conditioned.
    Arrays have the record index on the last axis."""
    gpu = np.asarray(gpu, np.float64)
    base = np.asarray(base, np.float64)
    err = np.abs(gpu - base)
    t = tol(base)
    bad = good & _per_record(err > t)
    if np.any(bad):
        idx = np.nonzero(bad)[0][:8]
        raise AssertionError(
            f"{name}: {int(bad.sum())} well-conditioned records out of tolerance; first "
            f"{idx.tolist()}: gpu {gpu[..., idx].tolist()} oracle {base[..., idx].tolist()}")
    lo = np.minimum.reduce([base] + [np.asarray(p, np.float64) for p in pert])
    hi = np.maximum.reduce([base] + [np.asarray(p, np.float64) for p in pert])
    ill = ~good
    outside = ill & _per_record((gpu < lo - tol(lo)) | (gpu > hi + tol(hi)))
    n = good.size
    ill_frac = ill.sum() / max(n, 1)
    out_frac = outside.sum() / max(n, 1)
    assert ill_frac <= max_ill, f"{name}: {ill_frac:.4f} of records ill-conditioned"
    # a record on a branch may take one the few perturbations did not reach
    assert out_frac <= 0.002, f"{name}: {out_frac:.5f} of records outside the oracle bracket"
    rel = _per_record_max(err / t)
    return dict(ill=float(ill_frac), outside=float(out_frac),
                worst_good=float(rel[good].max()) if good.any() else 0.0)


def _per_record_max(x):
    return x if x.ndim == 1 else x.max(axis=0)


def angle_between(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c = np.clip((a * b).sum(0) / (np.linalg.norm(a, axis=0) * np.linalg.norm(b, axis=0)), -1, 1)
    return np.arccos(c)
