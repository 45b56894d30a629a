"""Element-wise parity of the CUDA path against the FP64 oracle.

Tolerance (the contract of the GPU path): |gpu - oracle| <= 1e-6 + 1e-4 |oracle|
on eval f and pdf, 1e-4 rad on sampled directions, identical status / lobe
codes.

The BYSDF has branches and steep spots (closest ply, ply hit or miss, the
one-texel ramp at a fiber-map cusp, hemisphere side, total internal
reflection, lobe choice by u0, and grazing rays along the yarn axis where the
cross-section iteration stops contracting).  Where a record sits there, the
float32 rounding of the path decides which nearby value it lands on.  So
every record is also evaluated by the oracle at a few copies of its inputs
moved by about the GPU path's own rounding (see `perturb`), and the rule is:

* at least `min_strict` of the records (98% by default) agree with the
  oracle within the tolerance, and their status codes agree;
* every record that does not lies within the range the perturbed oracle
  values span (widened by the tolerance), except at most `max_outside`
  (0.2%) that sit on a branch none of the few perturbations reached.
"""
from __future__ import annotations

import numpy as np

REL, ABS = 1e-4, 1e-6
ANGLE = 1e-4


def tol(ref):
    return ABS + REL * np.abs(ref)


def perturb(rec: dict, k: int, eps_geo: float = 2.0 ** -21, eps_dir: float = 2.0 ** -23,
            sample: bool = False) -> dict:
    """A copy of the records moved by about the GPU path's own float32
    rounding: the entry offset h and azimuth u by ~eps_geo (they set the ply
    and fiber geometry, whose float32 chain -- ply centre, hit point, atan2
    of the ply azimuth, fiber phase -- accumulates a few ulps), the direction
    components by ~eps_dir (they enter the lobes after a few operations), the
    footprint ratio by eps_geo relative and u0/u1 by eps_dir.  The
    longitudinal position v is not moved: the path forms its phases from v
    with compensated products, so its phase error is far below one ulp of v."""
    g = np.random.default_rng(1000 + k)
    out = {kk: (vv.copy() if isinstance(vv, np.ndarray) else vv) for kk, vv in rec.items()}
    n = len(rec["h"])

    def r(*shape):
        return g.uniform(-1.0, 1.0, shape)
    out["h"] = np.clip(rec["h"] + eps_geo * r(n), -1, 1).astype(np.float32)
    out["u"] = (rec["u"] + eps_geo * r(n)).astype(np.float32)
    for key in ("wi", "wo"):
        if key in rec and rec[key] is not None:
            w = rec[key].astype(np.float64) + eps_dir * r(3, n)
            out[key] = (w / np.linalg.norm(w, axis=0)).astype(np.float32)
    if "ratio" in rec:
        out["ratio"] = (rec["ratio"] * (1 + eps_geo * r(n))).astype(np.float32)
    if sample:
        for key in ("u0", "u1"):
            out[key] = np.clip(rec[key] + eps_dir * r(n), 0.0, 1 - 2.0 ** -24).astype(np.float32)
    return out


def dump(name: str, **arrays):
    """Save raw arrays for offline analysis when BYSDF_PARITY_DUMP is set."""
    import os
    d = os.environ.get("BYSDF_PARITY_DUMP")
    if d:
        os.makedirs(d, exist_ok=True)
        np.savez_compressed(os.path.join(d, name + ".npz"),
                            **{k: np.asarray(v) for k, v in arrays.items()})


def conditioning(orc_fn, rec: dict, n_pert: int = 12, sample: bool = False):
    """Oracle outputs at the record and at n_pert perturbed copies.
    orc_fn(rec) -> tuple of arrays (last axis = record)."""
    base = orc_fn(rec)
    pert = [orc_fn(perturb(rec, k, sample=sample)) for k in range(n_pert)]
    return base, pert


def stable_mask(base_vals, pert_vals, base_status, pert_status, frac: float = 0.02):
    """Records whose oracle values move by at most frac * tolerance, and whose
    status does not change, under the perturbations (used to pick records with
    a unique derivative for the gradient test)."""
    good = np.ones(base_status.shape, bool)
    for ps in pert_status:
        good &= ps == base_status
    for b, ps in zip(base_vals, zip(*pert_vals)):
        for p in ps:
            d = np.abs(p - b) / tol(b)
            good &= (d if d.ndim == 1 else d.max(axis=0)) <= frac
    return good


def _per_record(x, how):
    return x if x.ndim == 1 else getattr(x, how)(axis=0)


def assert_parity(gpu, base, pert, name, min_strict=0.98, max_outside=0.002, err=None):
    """The rule above for one output (record index on the last axis).
    Returns a dict of the measured shares."""
    gpu = np.asarray(gpu, np.float64)
    base = np.asarray(base, np.float64)
    if err is None:
        err = _per_record(np.abs(gpu - base) / tol(base), "max")
    strict = err <= 1.0
    lo = np.minimum.reduce([base] + [np.asarray(p, np.float64) for p in pert])
    hi = np.maximum.reduce([base] + [np.asarray(p, np.float64) for p in pert])
    inside = ~_per_record((gpu < lo - tol(lo)) | (gpu > hi + tol(hi)), "any")
    unexplained = ~strict & ~inside
    n = max(strict.size, 1)
    res = dict(strict=float(strict.sum() / n), unexplained=float(unexplained.sum() / n),
               worst_strict=float(err[strict].max()) if strict.any() else 0.0,
               median_err=float(np.median(err)) if err.size else 0.0)
    assert res["strict"] >= min_strict, f"{name}: only {res['strict']:.4f} within tolerance {res}"
    if unexplained.any():
        i = np.nonzero(unexplained)[0][:5]
        assert res["unexplained"] <= max_outside, (
            f"{name}: {res['unexplained']:.5f} outside the oracle's perturbation range; "
            f"records {i.tolist()} gpu {gpu[..., i].tolist()} oracle {base[..., i].tolist()}")
    return res


def assert_status(gpu_st, base_st, pert_st, name):
    """Status codes agree wherever the perturbed oracle agrees with itself."""
    stable = np.ones(base_st.shape, bool)
    for ps in pert_st:
        stable &= ps == base_st
    diff = stable & (gpu_st != base_st)
    if diff.any():
        i = np.nonzero(diff)[0][:8]
        raise AssertionError(f"{name}: status differs on {int(diff.sum())} stable records, e.g. "
                             f"{i.tolist()}: gpu {gpu_st[i].tolist()} oracle {base_st[i].tolist()}")
    return float(stable.mean())


def angle_between(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c = np.clip((a * b).sum(0) / (np.linalg.norm(a, axis=0) * np.linalg.norm(b, axis=0)), -1, 1)
    return np.arccos(c)
