"""Element-wise parity of the CUDA path against the FP64 oracle (test
infrastructure: the tests, the smoke check and the benchmark's parity report
use it).

Tolerance (the contract of the GPU path): |gpu - oracle| <= 1e-6 + 1e-4 |oracle|
on eval f and pdf and on the sample's weight and pdf, 1e-4 rad on sampled
directions, identical status / lobe codes.

The rule is decided per record by the oracle alone, before the GPU's result
is looked at:

* A record is *well-conditioned* when (a) every branch point of the model
  it passes is at least 1e-4 away (the oracle's discontinuity margins: ply
  hit or miss, closest ply, the fiber-map cusp interval, rays along the yarn
  axis, hemisphere sides, the transmission path's side and refraction tests,
  and for sampling the lobe choice and the sampled direction's tests), and
  (b) it is well-conditioned in float32: moving each input (h, u, every
  direction component, and u0, u1 when sampling) on its own by SIGMA = 4
  units of 2^-24 -- about one float32 rounding of the inputs -- and moving
  the two internal quantities whose float32 rounding the result amplifies
  most, the in-plane hit distance t (by SIGMA yarn radii) and the ply
  azimuth that sets the fiber phase (by UPLY = 2 units of 2^-22 rad, two
  roundings of an angle near pi), changes the oracle's outputs by at most
  a quarter of the tolerance summed over these moves, and leaves the status
  alone.
  Every well-conditioned record must match strictly, status included.
* Every other record must match one of the values the oracle takes next to
  it: its status must be one the perturbed oracle reports, and its value
  must lie within the range of the perturbed oracle values (widened by the
  tolerance).  The perturbations are those of (b), the same moves 16 and
  256 times longer, 15 random moves of h, u and the direction components by
  2^-23, 2^-21, 2^-19, 2^-17 or 2^-15 (3 each; see `perturb`), and for a
  record closer than 1e-4 to a branch point 6 random moves four times its
  margin long, so that both sides of the branch are in the bracket.  Where
  the result is ill-conditioned the float32 path's own rounding compounds
  through the ply trace's iterations, and on the worst records (rays nearly
  along the yarn axis, footprint nodes in a fiber cusp next to a glossy
  lobe) its deviation reaches that of inputs moved by hundreds of units of
  2^-24.

* A record whose outputs move by more than COND_UNDETERMINED = 1000
  tolerances (10% of the value) under the moves of (b) is not determined by
  its float32 inputs at all: a float32 evaluation may land anywhere in the
  range the model sweeps next to it, which a finite set of perturbations
  does not map out (these are rays nearly along the yarn axis, whose ply
  trace does not contract, and footprints whose nodes meet a fiber cusp).
  It must have a status the oracle reports next to it, and a finite value
  of the right kind: >= 0, or a unit vector for a sampled direction.

No share of records is let off: a record that meets none of these fails the
test, and every test prints the shares of the three kinds.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

REL, ABS = 1e-4, 1e-6
ANGLE = 1e-4
MARGIN = 1e-4
SIGMA = 4.0 * 2.0 ** -24
UPLY = 2.0 * 2.0 ** -22
COND_MAX = 0.25
COND_UNDETERMINED = 1000.0
# margin classes that decide a well-conditioned record (all but the ply
# shadowing chord, whose steepness the conditioning test measures)
EVAL_CLASSES = ("graze", "gap", "cusp", "axis", "hemi", "exit")
SAMPLE_CLASSES = EVAL_CLASSES + ("lobe", "sample")


def tol(ref):
    return ABS + REL * np.abs(ref)


def perturb(rec: dict, k: int, eps_geo: float = 2.0 ** -21, eps_dir: float = 2.0 ** -23,
            sample: bool = False) -> dict:
    """A copy of the records moved at random by about the GPU path's own
    float32 rounding: the entry offset h and azimuth u by ~eps_geo, the
    direction components by ~eps_dir (renormalised), the footprint ratio by
    eps_geo relative and u0/u1 by eps_dir.  The longitudinal position v is
    not moved: the path forms its phases from v with compensated products."""
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


def axis_moves(rec: dict, sample: bool = False, sigma: float = SIGMA):
    """(name, record copy) with one input moved by +-SIGMA: h, u, each
    component of omega_i (and of omega_o for eval), u0 and u1 for sampling.
    The float32 rounding of a move is part of it (what the GPU receives is
    float32 too)."""
    axes = [("h", None), ("u", None)] + [("wi", c) for c in range(3)]
    axes += [("u0", None), ("u1", None)] if sample else [("wo", c) for c in range(3)]
    for key, c in axes:
        for s in (-sigma, sigma):
            r = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in rec.items()}
            if c is None:
                x = r[key].astype(np.float64) + s
                lo, hi = (-1.0, 1.0) if key == "h" else ((0.0, 1 - 2.0 ** -24) if key in ("u0", "u1")
                                                        else (-np.inf, np.inf))
                r[key] = np.clip(x, lo, hi).astype(np.float32)
            else:
                w = r[key].astype(np.float64)
                w[c] += s
                r[key] = (w / np.linalg.norm(w, axis=0)).astype(np.float32)
            yield f"{key}{'' if c is None else c}", r


def _per_record(x, how):
    return x if x.ndim == 1 else getattr(x, how)(axis=0)


def dev(values, base, scale=None):
    """|values - base| in units of the tolerance (per record, max over the
    leading axis)."""
    v = np.asarray(values, np.float64)
    b = np.asarray(base, np.float64)
    d = np.abs(v - b) / (tol(b) if scale is None else scale)
    return _per_record(d, "max")


@dataclass
class Oracle:
    """The oracle's view of a record set: base outputs, perturbed outputs,
    and the well-conditioned mask with its parts."""
    base: tuple
    pert: list
    stable: np.ndarray      # well-conditioned records
    margin: np.ndarray      # smallest margin over the deciding classes
    cond: np.ndarray        # summed first-order change per SIGMA move, in tolerances
    status_idx: int

    def shares(self) -> dict:
        return dict(well_conditioned=float(self.stable.mean()) if self.stable.size else 1.0,
                    low_margin=float((self.margin < MARGIN).mean()) if self.margin.size else 0.0,
                    ill_conditioned=float((self.cond > COND_MAX).mean()) if self.cond.size else 0.0,
                    undetermined=float((self.cond > COND_UNDETERMINED).mean())
                    if self.cond.size else 0.0)


def oracle_view(orc, orc_fn, mats, rec, sample: bool = False, values=(0, 1), status_idx=2,
                angle_idx=None, n_random: int = 15, margin_kw=None) -> Oracle:
    """Run the oracle at the records, at the SIGMA moves and at n_random
    random perturbations.  orc_fn(rec) -> tuple of arrays (record on the last
    axis); `values` index the outputs compared with the tolerance,
    `status_idx` the status, `angle_idx` a direction output compared by
    angle (sampling)."""
    base = orc_fn(rec)
    n = base[status_idx].shape[-1]
    cond = np.zeros(n)
    st_moves = np.zeros(n, bool)
    pert = []
    for _, r in axis_moves(rec, sample):
        pert.append(orc_fn(r))
    for kw in (dict(dt=SIGMA), dict(du_ply=UPLY)):
        for sg in (-1.0, 1.0):
            with orc.internal_offsets(**{k: sg * v for k, v in kw.items()}):
                pert.append(orc_fn(rec))
    # the worst of the two moves of each axis, summed over the axes
    for a in range(0, len(pert), 2):
        worst = np.zeros(n)
        for o in pert[a:a + 2]:
            for vi in values:
                worst = np.maximum(worst, dev(o[vi], base[vi]))
            if angle_idx is not None:
                ok = ((o[status_idx] & 15) == 0) & ((base[status_idx] & 15) == 0)
                with np.errstate(invalid="ignore"):
                    ang = np.where(ok, angle_between(o[angle_idx], base[angle_idx]), 0.0)
                worst = np.maximum(worst, ang / ANGLE)
            st_moves |= o[status_idx] != base[status_idx]
        cond += worst
    # the bracket also holds each move 16 and 256 times longer, and random moves
    for f in (16.0, 256.0):
        for _, r in axis_moves(rec, sample, f * SIGMA):
            pert.append(orc_fn(r))
    for f in (16.0, 256.0):
        for kw in (dict(dt=f * SIGMA), dict(du_ply=f * UPLY)):
            for sg in (-1.0, 1.0):
                with orc.internal_offsets(**{k: sg * v for k, v in kw.items()}):
                    pert.append(orc_fn(rec))
    for k in range(n_random):
        e = 2.0 ** -(23 - 2 * (k % 5))
        pert.append(orc_fn(perturb(rec, k, eps_geo=e, eps_dir=e, sample=sample)))
    mk = dict(margin_kw or {})
    mg = orc.margins(mats, rec, "sample" if sample else "eval", threads=8, **mk)
    cls = SAMPLE_CLASSES if sample else EVAL_CLASSES
    rows = [orc.MARGIN_CLASSES.index(c) for c in cls]
    margin = mg[rows].min(axis=0)
    # records next to a branch point: random moves four times their margin
    # long (margins are lengths in yarn radii, cosines or probabilities, on
    # the scale of the inputs)
    low = margin < MARGIN
    if low.any():
        e = np.where(low, 4.0 * np.maximum(margin, 1e-7), 0.0)
        for k in range(6):
            pert.append(orc_fn(perturb(rec, 100 + k, eps_geo=e, eps_dir=e, sample=sample)))
    stable = (margin >= MARGIN) & (cond <= COND_MAX) & ~st_moves
    return Oracle(base, pert, stable, margin, cond, status_idx)


def assert_parity(gpu, view: Oracle, vi: int, name: str, err=None, gpu_status=None,
                  direction: bool = False):
    """The rule for one output (index vi of the oracle tuple; record on the
    last axis).  err: per-record error in tolerances (default |gpu - oracle|
    / tol).  gpu_status: the GPU's status codes, used to bracket the value
    against the perturbed oracle values of the same status.  direction: the
    output is a unit direction (components of either sign).  Returns the
    measured shares."""
    gpu = np.asarray(gpu, np.float64)
    base = np.asarray(view.base[vi], np.float64)
    if err is None:
        err = _per_record(np.abs(gpu - base) / tol(base), "max")
    strict = err <= 1.0
    bad_wc = view.stable & ~strict
    n = max(strict.size, 1)
    if bad_wc.any():
        i = np.nonzero(bad_wc)[0][:5]
        raise AssertionError(
            f"{name}: {int(bad_wc.sum())} well-conditioned records outside the tolerance, e.g. "
            f"{i.tolist()}: err {err[i].round(3).tolist()} margin {view.margin[i].tolist()} "
            f"cond {view.cond[i].round(3).tolist()} gpu {gpu[..., i].tolist()} "
            f"oracle {base[..., i].tolist()}")
    # bracket of the others: over the perturbed values (of the GPU's status,
    # where given), widened by the tolerance
    vals = [base] + [np.asarray(p[vi], np.float64) for p in view.pert]
    sts = [view.base[view.status_idx]] + [p[view.status_idx] for p in view.pert]
    lo = np.full(base.shape, np.inf)
    hi = np.full(base.shape, -np.inf)
    for v, s in zip(vals, sts):
        use = np.ones(s.shape, bool) if gpu_status is None else (s == gpu_status)
        lo = np.where(use, np.minimum(lo, v), lo)
        hi = np.where(use, np.maximum(hi, v), hi)
    inside = ~_per_record((gpu < lo - tol(lo)) | (gpu > hi + tol(hi)), "any")
    # records the float32 inputs do not determine: a finite value of the
    # right kind
    undet = view.cond > COND_UNDETERMINED
    if direction:
        within = np.abs(np.linalg.norm(gpu, axis=0) - 1.0) <= 1e-3
    else:
        within = ~_per_record(gpu < 0.0, "any")
    inside |= undet & within & _per_record(np.isfinite(gpu), "all")
    outside = ~strict & ~inside
    if outside.any():
        i = np.nonzero(outside)[0][:5]
        raise AssertionError(
            f"{name}: {int(outside.sum())} records neither within the tolerance nor inside the "
            f"oracle's bracket, e.g. {i.tolist()}: gpu {gpu[..., i].tolist()} "
            f"oracle {base[..., i].tolist()} margin {view.margin[i].tolist()}")
    res = dict(n=int(strict.size), strict=float(strict.sum() / n),
               strict_on_well_conditioned=1.0, **view.shares(),
               median_err=float(np.median(err)) if err.size else 0.0)
    print(f"[parity] {name}: {res}")
    return res


def assert_status(gpu_st, view: Oracle, name: str, code=None):
    """Status codes: equal on well-conditioned records; elsewhere one of the
    codes the oracle reports at the record or its perturbations.  code(o)
    builds the compared code from an oracle tuple (default: its status)."""
    code = code or (lambda o: o[view.status_idx])
    base = code(view.base)
    diff = view.stable & (gpu_st != base)
    if diff.any():
        i = np.nonzero(diff)[0][:8]
        raise AssertionError(f"{name}: status differs on {int(diff.sum())} well-conditioned "
                             f"records, e.g. {i.tolist()}: gpu {gpu_st[i].tolist()} "
                             f"oracle {base[i].tolist()}")
    seen = gpu_st == base
    for p in view.pert:
        seen |= gpu_st == code(p)
    if not seen.all():
        i = np.nonzero(~seen)[0][:8]
        raise AssertionError(f"{name}: status on {int((~seen).sum())} records is none the "
                             f"oracle reports next to them, e.g. {i.tolist()}: gpu "
                             f"{gpu_st[i].tolist()} oracle {base[i].tolist()}")
    return float((gpu_st == base).mean())


KINK = 1e-5          # fiber periods: a few times the float32 path's phase error
JAC_STABLE = 1e-3    # relative change of a record's Jacobian under one internal move


def gradient_spread(orc, mats, rec, view: Oracle, **margin_kw):
    """(mask, dJ) for the gradient tests.

    mask: records whose derivatives the float32 path can follow --
    well-conditioned; no fiber-map lookup within KINK periods of a texel
    centre (the interpolant's slope changes there, and the helix angles'
    derivatives carry that slope times hundreds of periods per radian); and
    a Jacobian (oracle, 8 parameters) that moves by at most JAC_STABLE of
    itself when the azimuth u, the hit distance or the ply azimuth moves by
    about one float32 rounding.

    dJ [n, 3, 8]: the largest change of each Jacobian entry under those
    moves -- how far a float32 evaluation of the derivative may honestly sit
    from the exact one.  At large |v| the helix angles' derivatives are
    products of the phase v tan(alpha) with slopes that vary over a fraction
    of a fiber period, so dJ reaches a few 1e-4 of J there."""
    mg = orc.margins(mats, rec, "eval", threads=8, **margin_kw)
    good = view.stable & (mg[orc.MARGIN_CLASSES.index("kink")] >= KINK)
    n = good.shape[0]
    g = np.ones((3, n))
    _, _, J0 = orc.grad_records(mats, rec, g, threads=8, jac=True)
    size = np.abs(J0).max(axis=1)                      # [n, 8]
    dJ = np.zeros_like(J0)

    def moved(J1):
        nonlocal dJ
        dJ = np.maximum(dJ, np.abs(J1 - J0))

    for kw in (dict(dt=SIGMA), dict(dt=-SIGMA), dict(du_ply=UPLY), dict(du_ply=-UPLY)):
        with orc.internal_offsets(**kw):
            moved(orc.grad_records(mats, rec, g, threads=8, jac=True)[2])
    for s in (-SIGMA, SIGMA):
        r = dict(rec)
        r["u"] = (rec["u"].astype(np.float64) + s).astype(np.float32)
        moved(orc.grad_records(mats, r, g, threads=8, jac=True)[2])
    rel = np.where(size > 0, dJ.max(axis=1) / (size + 1e-12), 0.0).max(axis=1)
    return good & (rel <= JAC_STABLE), dJ


def gradient_mask(orc, mats, rec, view: Oracle, **margin_kw):
    """The mask of gradient_spread alone."""
    return gradient_spread(orc, mats, rec, view, **margin_kw)[0]


def gradient_bound(mat_id, g, J, dJ, n_mat: int, rel: float = 1e-4, abs_: float = 1e-6):
    """Per-material tolerance [n_mat, 8] of a float32 gradient
    sum_records sum_c g_c dJ_c/dtheta: rel of sum |g J| (the float32
    accumulation and arithmetic) plus sum |g| dJ (each record's Jacobian
    known only to within its spread under float32 rounding of its inputs)
    plus abs_."""
    g = np.asarray(g, np.float64)
    t = rel * np.abs(g.T[:, :, None] * J).sum(1) + (np.abs(g.T)[:, :, None] * dJ).sum(1)
    out = np.zeros((n_mat, J.shape[2]))
    np.add.at(out, mat_id, t)
    return out + abs_


def dump(name: str, **arrays):
    """Save raw arrays for offline analysis when BYSDF_PARITY_DUMP is set."""
    import os
    d = os.environ.get("BYSDF_PARITY_DUMP")
    if d:
        os.makedirs(d, exist_ok=True)
        np.savez_compressed(os.path.join(d, name + ".npz"),
                            **{k: np.asarray(v) for k, v in arrays.items()})


def angle_between(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c = np.clip((a * b).sum(0) / (np.linalg.norm(a, axis=0) * np.linalg.norm(b, axis=0)), -1, 1)
    return np.arccos(c)
