#!/usr/bin/env python
"""Throughput of the yarn BYSDF hot path on GB300.

Default step (workload "eval+sample+pdf-8mat-2^24"): 2^24 hit records over 8
yarn materials, each record evaluated at omega_o (f and pdf) and importance
sampled from two uniform numbers (direction, weight, pdf), in the fused
persistent kernel.  value = records per second over all ranks (weak scaling:
each rank owns its own 2^24 records); inputs are larger than L2.

Also reported (same JSON line): the other workloads (near-field eval,
multi-scale, 256-material batched with a CUDA graph, forward + backward), the
plain per-material-launch form, the end-to-end rate with host buffers, the
roofline of the fused kernel, and the FP64 oracle on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2401_12724_gb300 import inputs as I  # noqa: E402

METRIC = "BYSDF evals/sec (fwd, fwd+bwd) on 1 GB300, % FP32/SFU roofline, vs plain, ≤1e-4 rel err"
UNIT = "records/s"
MAIN_CFG = 2

# Algorithmic work per record, counted by the FP64 oracle's operation-counting
# scalar on 4096 records of each workload (oracle/count_ops.py, which also
# gives the backward's count: one recompute plus one reverse sweep): FP32
# flops (adds + multiplies) and XU ops (divisions, square roots,
# transcendentals).  tests/test_op_counts.py recounts and compares.
OPS = {
    1: dict(eval=(480.3, 67.9)),
    2: dict(eval=(519.5, 73.6), fused=(700.1, 92.6)),
    3: dict(eval=(2946.4, 458.5), fused=(3133.1, 478.0)),
    4: dict(eval=(561.6, 79.7), fused=(748.7, 99.3)),
    5: dict(eval=(415.9, 58.6), backward=(1862.6, 117.2)),
}
# DRAM traffic of the fused kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch on the first 2^22 records of the
# workload, per record; the records stream through once, so traffic scales
# with the record count).  It is reported only while the kernel sources are
# the ones captured (SHA-256 of FUSED_SOURCES).
TRAFFIC_CAPTURE = dict(sources_sha256="07f29fb7cc8d35a65bad24fce53f029eea1404be7ea8e7c308d8f21570f80e8a",
                       bytes_per_record=82.51,
                       summary="profiles/k_forward_fused_eval-sample-pdf_8mat.md")
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (2 flops each)
XU_LANES_PER_SM = 16      # special-function (MUFU) lanes per SM
SM_MAX_MHZ = 2070.0


# the files that decide the fused kernel's code and its tables
FUSED_SOURCES = ("paper_2401_12724_gb300/csrc/bysdf_fwd_fused.cu",
                 "paper_2401_12724_gb300/csrc/bysdf_fwd_kernel.cuh",
                 "paper_2401_12724_gb300/csrc/bysdf_kernels.cuh",
                 "paper_2401_12724_gb300/csrc/bysdf_model.cuh",
                 "paper_2401_12724_gb300/csrc/bysdf_common.cuh",
                 "paper_2401_12724_gb300/csrc/bysdf_launch.h",
                 "paper_2401_12724_gb300/csrc/bysdf_api.cu",
                 "paper_2401_12724_gb300/build.py",
                 "include/bysdf.h")


def sources_sha256() -> str:
    """Digest of the fused kernel's sources (file names and bytes)."""
    h = hashlib.sha256()
    for rel in FUSED_SOURCES:
        h.update(rel.encode())
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def peaks(sm_count: int, mhz: float):
    return dict(fp32_tflops=sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
                xu_tops=sm_count * XU_LANES_PER_SM * mhz * 1e6 / 1e12)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6),
                              ("sw_thermal_slowdown", 7), ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ------------------------------------------------------------ distributed --
def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def dist_max(x: float) -> float:
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return x


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ------------------------------------------------------------ CPU oracle --
CHECK_RECORDS = 1 << 22   # prefix of the main workload the oracle runs on
RULE_RECORDS = 1 << 18    # prefix the tests' parity rule is applied to


def cpu_oracle_rate(cfg: int, target_s: float = 10.0, max_records: int = CHECK_RECORDS):
    """The FP64 oracle, as it stands, on this host's cores: eval at omega_o
    (with pdf) plus one sample per record, over a bounded prefix of the
    workload, repeated until about target_s of CPU time has passed.  Also
    returns the first pass's outputs (for the parity report)."""
    import oracle
    threads = os.cpu_count() or 1
    mats = I.materials(cfg)
    n = min(max_records, I.N_RECORDS[cfg])
    rec = I.records(cfg, 0, n)
    done, t0, first = 0, time.perf_counter(), None
    while True:
        ev = oracle.eval_records(mats, rec, threads=threads)
        sa = oracle.sample_records(mats, rec, threads=threads)
        if first is None:
            first = (ev, sa)
        done += n
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    # one thread, on a shorter prefix
    n1 = 1 << 15
    rec1 = I.records(cfg, 0, n1)
    t1 = time.perf_counter()
    oracle.eval_records(mats, rec1, threads=1)
    oracle.sample_records(mats, rec1, threads=1)
    dt1 = time.perf_counter() - t1
    return dict(value=done / dt, unit=UNIT, cores=threads, kind="oracle",
                sample=f"first {n} records of workload {I.WORKLOAD_NAME[cfg]}, eval(+pdf) and "
                       f"one sample each, FP64, {threads} threads, {done // n} passes",
                seconds=dt, records=done,
                single_thread=dict(value=n1 / dt1, unit=UNIT, cores=1, records=n1,
                                   seconds=dt1)), first


def parity_rule(gpu: dict, cfg: int) -> dict:
    """The parity tests' rule (oracle/parity.py) on the first RULE_RECORDS
    records of the timed outputs: strict on every record the oracle finds
    well-conditioned (margin to every branch point >= 1e-4, first-order
    change under one float32 rounding of its inputs <= a quarter of the
    tolerance), the oracle's bracket on the others."""
    import oracle
    from oracle import parity as PU
    threads = os.cpu_count() or 1
    mats = I.materials(cfg)
    m = min(RULE_RECORDS, gpu["status"].shape[0])
    rec = I.records(cfg, 0, m)
    out = dict(records=m)
    try:
        view = PU.oracle_view(oracle, lambda r: oracle.eval_records(mats, r, threads=threads),
                              mats, rec)
        st = gpu["status"][:m]
        PU.assert_status(st, view, "bench.status")
        r_f = PU.assert_parity(gpu["f"][:, :m], view, 0, "bench.f", gpu_status=st)
        r_p = PU.assert_parity(gpu["pdf"][:m], view, 1, "bench.pdf", gpu_status=st)

        def code(r):
            wo, w, p, s, lb = oracle.sample_records(mats, r, threads=threads)
            return wo, w, p, s | (lb << 4)
        sv = PU.oracle_view(oracle, code, mats, rec, sample=True, values=(1, 2), status_idx=3,
                            angle_idx=0)
        ls = gpu["lobe_status"][:m]
        PU.assert_status(ls, sv, "bench.lobe_status")
        both = ((sv.base[3] & 15) == 0) & ((ls & 15) == 0)
        with np.errstate(invalid="ignore"):
            ang = np.where(both, PU.angle_between(gpu["wo"][:, :m], sv.base[0]), 0.0)
        r_wo = PU.assert_parity(gpu["wo"][:, :m], sv, 0, "bench.wo", err=ang / PU.ANGLE,
                                gpu_status=ls, direction=True)
        r_w = PU.assert_parity(gpu["weight"][:, :m], sv, 1, "bench.weight", gpu_status=ls)
        r_ps = PU.assert_parity(gpu["pdf_s"][:m], sv, 2, "bench.pdf_s", gpu_status=ls)
        out.update(passed=True, within_tol_well_conditioned=1.0,
                   eval=dict(strict_f=r_f["strict"], strict_pdf=r_p["strict"],
                             well_conditioned=r_f["well_conditioned"],
                             low_margin=r_f["low_margin"], ill_conditioned=r_f["ill_conditioned"],
                             undetermined=r_f["undetermined"]),
                   sample=dict(strict_wo=r_wo["strict"], strict_weight=r_w["strict"],
                               strict_pdf=r_ps["strict"],
                               well_conditioned=r_w["well_conditioned"],
                               low_margin=r_w["low_margin"],
                               ill_conditioned=r_w["ill_conditioned"],
                               undetermined=r_w["undetermined"]))
    except AssertionError as e:
        out.update(passed=False, failure=str(e)[:400])
    return out


def parity_report(gpu: dict, first) -> dict:
    """The benchmark's own outputs against the oracle's on the same records:
    status agreement, the share within 1e-4 relative + 1e-6 absolute (f, pdf
    at omega_o and the sample's weight and pdf, where both report a valid
    result), and relative-error quantiles.  The maximum includes records at
    a branch boundary of the model (argmin ties, fiber cusps, grazing
    directions), where either side is correct; the parity tests bracket those
    by perturbing the inputs."""
    (fo, po, so), (wo_o, w_o, ps_o, ss_o, lb_o) = first
    n = so.shape[0]
    st, ls = gpu["status"][:n], gpu["lobe_status"][:n]
    ok = (st == 0) & (so == 0)
    oks = ((ls & 15) == 0) & (ss_o == 0) & ((ls >> 4) == lb_o)

    def rel(g, o, m):
        e = np.abs(g - o) / (np.abs(o) + 1e-6 / 1e-4)
        return e[..., m].reshape(-1) if e.ndim == 1 else e[:, m].max(axis=0)
    errs = np.concatenate([np.maximum(rel(gpu["f"][:, :n], fo, ok), rel(gpu["pdf"][:n], po, ok)),
                           np.maximum(rel(gpu["weight"][:, :n], w_o, oks),
                                      rel(gpu["pdf_s"][:n], ps_o, oks))])
    q = np.quantile(errs, [0.5, 0.99, 0.999]) if errs.size else [0.0] * 3
    return dict(records=int(n), status_equal=float((st == so).mean()),
                sample_status_equal=float((ls == (ss_o | (lb_o << 4))).mean()),
                within_tol=float((errs <= 1e-4).mean()) if errs.size else 1.0,
                rel_err_p50=float(q[0]), rel_err_p99=float(q[1]), rel_err_p999=float(q[2]),
                rel_err_max=float(errs.max()) if errs.size else 0.0,
                note="relative error |gpu - oracle| / (|oracle| + 1e-2); within_tol: share "
                     "at most 1e-4, i.e. within 1e-4 relative + 1e-6 absolute; the max includes "
                     "records at branch boundaries, where either side is correct")


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample of the workload."""
    import oracle
    threads = os.cpu_count() or 1
    cfg = MAIN_CFG
    mats = I.materials(cfg)
    n = 1 << 16
    rec = I.records(cfg, 0, n)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.eval_records(mats, rec, threads=threads)
        oracle.sample_records(mats, rec, threads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = n * len(times) / tot
    sample = (f"first {n} records of workload {I.WORKLOAD_NAME[cfg]} per step, eval(+pdf) and "
              f"one sample each, FP64, {threads} threads")
    line = dict(impl="reference", metric=METRIC, value=val, unit=UNIT, n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup, ms_per_step=1e3 * tot / len(times),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic",
                config=dict(workload=I.WORKLOAD_NAME[cfg], records_per_step=n, materials=len(mats)),
                cpu_baseline=dict(value=val, unit=UNIT, cores=threads, kind="oracle", sample=sample),
                e2e=dict(value=val, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU ----
def timed(fn, steps, warmup, stream=None):
    """Mean milliseconds per call with CUDA events on the launching stream."""
    import torch
    for _ in range(warmup):
        fn()
    st = stream or torch.cuda.current_stream()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        starts[k].record(st)
        fn()
        ends[k].record(st)
    torch.cuda.synchronize()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return sum(per) / len(per), per


def workload_device(api, cfg, rank, count=0):
    seed = None if rank == 0 else I.SEED_BASE + cfg + 1000 * rank
    rec = I.records(cfg, 0, count or None, seed=seed)
    seg = I.seg_offsets(cfg, seed=seed)
    if seg is not None and count:
        # the first `count` records of a material-sorted workload
        seg = np.minimum(seg, int(rec["h"].shape[0]))
    d = api.records_to_device(rec, "cuda", seg)
    return rec, d, seg


def sorted_copy(d, n_mat):
    """Records permuted into material order (for the plain per-material form)."""
    import torch
    order = torch.argsort(d["mat_id"], stable=True)
    out = {}
    for k, t in d.items():
        out[k] = t[..., order].contiguous() if t.shape[-1] == order.numel() else t
    counts = torch.bincount(d["mat_id"].long(), minlength=n_mat).cpu().numpy()
    seg = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return out, seg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--main-only", action="store_true", help="skip the other workloads")
    ap.add_argument("--profile", action="store_true",
                    help="main workload only, no clocks/e2e/CPU baseline (for ncu)")
    ap.add_argument("--records", type=int, default=0,
                    help="use only the first N records of the workload (profiling)")
    ap.add_argument("--profile-op", default="fused",
                    choices=["fused", "backward", "l2", "trace", "multiscale"],
                    help="with --profile: fused = eval + sample + pdf over workload 2; "
                         "backward = forward eval + backward over workload 5; l2 = forward, "
                         "L2 loss and backward in one pass over workload 5; trace = "
                         "2048 x 2048 camera rays against a 512-piece yarn patch; "
                         "multiscale = eval + sample + pdf over workload 3")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_setup()
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    from paper_2401_12724_gb300 import _native as N
    from paper_2401_12724_gb300 import api

    torch.cuda.set_device(local)
    props = torch.cuda.get_device_properties(local)
    sm_count = props.multi_processor_count

    if args.profile and args.profile_op in ("backward", "l2"):
        profile_backward(api, torch, args, rank, l2=args.profile_op == "l2")
        return
    if args.profile and args.profile_op == "multiscale":
        M = api.Materials(I.materials(3))
        _, d, _ = workload_device(api, 3, rank, args.records)
        o = api.alloc_fused(int(d["h"].shape[0]), "cuda")
        ms, _ = timed(lambda: api.eval_sample_pdf(M, d, out=o), args.steps, args.warmup)
        print(json.dumps(dict(profile="multiscale", workload=I.WORKLOAD_NAME[3],
                              records=int(d["h"].shape[0]), ms_per_step=ms)), flush=True)
        return
    if args.profile and args.profile_op == "trace":
        sc = I.woven_scene(16, 16)
        Y = api.yarns_to_device(sc)
        rays = {k: torch.from_numpy(v).cuda() for k, v in
                I.camera_rays(2048, 2048, extent=16 * 2.5).items()}
        light = (0.3, -0.4, math.sqrt(0.75))
        tr = api.trace_yarns(Y, rays, light)
        ms, _ = timed(lambda: api.trace_yarns(Y, rays, light, out=tr), args.steps, args.warmup)
        print(json.dumps(dict(profile="trace", rays=int(rays["o"].shape[1]), ms_per_step=ms)),
              flush=True)
        return

    # ---------------------------------------------- main workload (fused) --
    cfg = MAIN_CFG
    mats = I.materials(cfg)
    M = api.Materials(mats)
    rec, d, _ = workload_device(api, cfg, rank, args.records)
    n = int(d["h"].shape[0])
    out = api.alloc_fused(n, "cuda")
    step = lambda: api.eval_sample_pdf(M, d, out=out)  # noqa: E731
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if not args.profile:
        clocks.start()
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    for k in range(args.steps):
        step()
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if not args.profile else None
    per_launch = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    ms_total = ev[0].elapsed_time(ev[-1])
    ms_total = dist_max(ms_total)
    ms_step = ms_total / args.steps
    value = ws * n * args.steps / (ms_total / 1e3)
    err = M.workspace_error()
    if err:
        raise RuntimeError(f"device-side error word {err:#x} during the timed steps")

    if rank != 0:
        return
    # roofline of the fused kernel (the step is that one launch; the step
    # time bounds the kernel's time from above)
    fl, xu = OPS[cfg]["fused"]
    t_launch = sum(per_launch) / len(per_launch) / 1e3
    ach_fp32 = fl * n / t_launch / 1e12
    ach_xu = xu * n / t_launch / 1e12
    pk = peaks(sm_count, SM_MAX_MHZ)
    frac_fp32 = ach_fp32 / pk["fp32_tflops"]
    frac_xu = ach_xu / pk["xu_tops"]
    if frac_fp32 >= frac_xu:
        roof = dict(bound="alu", pipe="fp32", achieved=ach_fp32, peak=pk["fp32_tflops"],
                    unit="TFLOP/s", frac=frac_fp32)
    else:
        roof = dict(bound="alu", pipe="xu", achieved=ach_xu, peak=pk["xu_tops"], unit="Top/s",
                    frac=frac_xu)
    digest = sources_sha256()
    traffic = None
    if TRAFFIC_CAPTURE["bytes_per_record"] and TRAFFIC_CAPTURE["sources_sha256"] == digest:
        traffic = TRAFFIC_CAPTURE["bytes_per_record"] * n
    roof.update(traffic=traffic, traffic_unit="bytes per launch",
                traffic_source=(TRAFFIC_CAPTURE["summary"] if traffic else
                                "null: no ncu capture of these kernel sources"),
                sources_sha256=digest, peak_basis=f"{sm_count} SMs x lanes x {SM_MAX_MHZ:.0f} MHz",
                pipes=dict(fp32=dict(achieved_tflops=ach_fp32, frac=frac_fp32,
                                     flops_per_record=fl),
                           xu=dict(achieved_tops=ach_xu, frac=frac_xu, ops_per_record=xu)),
                algorithmic_bytes_per_record=48 + 46)
    if clk:
        pm = peaks(sm_count, clk["sm_mhz"])
        roof["frac_at_measured_clock"] = max(ach_fp32 / pm["fp32_tflops"], ach_xu / pm["xu_tops"])

    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=ws, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=I.WORKLOAD_NAME[cfg], records=n, materials=len(mats),
                            headline="the metric's quoted workload: eval + importance sample + "
                                     "pdf over 8 yarn materials, 2^24 records; the 2^26-record "
                                     "256-material batch and the other workloads are in "
                                     "'workloads'",
                            step="fused eval(+pdf at wo) + one importance sample per record",
                            l2="inputs larger than L2 (~0.8 GB of records per step)",
                            launch=M.launch_config(N.OP_FUSED),
                            parallelism=f"records sharded, {ws} rank(s)"),
                # one fused kernel per step: the records come in any order, so no
                # tile-plan kernel runs (the ncu launch list of this step shows one)
                roofline=roof, gpu_launches=args.steps)
    if clk:
        line["clocks"] = clk

    if not args.profile:
        # ------------------------------------------ end to end, host buffers --
        hin = api.pinned_records(rec)
        hout = api.pinned_fused_outputs(n)
        pipe = api.HostPipeline(M, chunk=1 << 21)   # the C ABI's host-buffer pipeline
        pipe.run(hin, hout)
        torch.cuda.synchronize()
        e2e_steps = max(3, args.steps // 4)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            pipe.run(hin, hout)
            # a step ends with its results readable in host memory
            torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        bi, bo = api.HostPipeline.bytes_per_record(hin, hout)
        line["e2e"] = dict(value=n * e2e_steps / dt, unit=UNIT,
                           h2d_bytes_per_step=int(bi * n), d2h_bytes_per_step=int(bo * n),
                           chunks=math.ceil(n / (1 << 21)))
        del hin, hout, pipe

        # ------------------------------------------ plain form, same records --
        ds, seg = sorted_copy(d, len(mats))
        po = api.alloc_fused(n, "cuda")
        plain_out = dict(f=po["f"], wo=po["wo"], weight=po["weight"], pdf=po["pdf"],
                         status=po["status"])

        def plain_step():
            api.plain(N.OP_EVAL, M, ds, seg, out=plain_out)
            api.plain(N.OP_SAMPLE, M, ds, seg, out=plain_out)
            api.plain(N.OP_PDF, M, ds, seg, out=plain_out)
        ms_plain, _ = timed(plain_step, max(3, args.steps // 2), 2)
        # like for like: the fused op in the plain per-material form, and the
        # persistent kernel on the same material-sorted records
        ms_plain_fused, _ = timed(lambda: api.plain_fused(M, ds, seg, out=po),
                                  max(3, args.steps // 2), 2)
        dss = dict(ds)
        dss["seg_offsets"] = torch.from_numpy(seg).cuda()
        ms_pers_sorted, _ = timed(lambda: api.eval_sample_pdf(M, dss, out=po),
                                  max(3, args.steps // 2), 2)
        # the same three ops as separate persistent calls (no fusion)
        sep = lambda: (api.eval(M, d, out=out), api.sample(M, d, out=dict(  # noqa: E731
            wo=out["wo"], weight=out["weight"], pdf=out["pdf_s"], lobe_status=out["lobe_status"])),
            api.pdf(M, d, out=out))
        ms_sep, _ = timed(sep, max(3, args.steps // 2), 2)
        line["vs_plain"] = dict(plain_fused_records_per_s=n / (ms_plain_fused / 1e3),
                                fused_speedup_vs_plain_fused=ms_plain_fused / ms_step,
                                note="the plain form needs its records sorted by material "
                                     "(done outside its timed region); the timed step takes "
                                     "them in any order",
                                persistent_on_sorted_records_per_s=n / (ms_pers_sorted / 1e3),
                                persistent_vs_plain_same_sorted_input=ms_plain_fused / ms_pers_sorted,
                                plain_fused_launches_per_step=len(mats),
                                plain_three_ops_records_per_s=n / (ms_plain / 1e3),
                                separate_persistent_records_per_s=n / (ms_sep / 1e3),
                                fused_speedup_vs_plain_three_ops=ms_plain / ms_step)
        del ds, dss, po, plain_out
        # the timed steps' outputs on the records the oracle checks
        m = min(CHECK_RECORDS, n)
        gpu_check = {k: (v[..., :m].cpu().numpy()) for k, v in out.items()}
        del d, out
        torch.cuda.empty_cache()

        if not args.main_only:
            line["workloads"] = other_workloads(api, N, torch, args, sm_count)
        line["cpu_baseline"], first = cpu_oracle_rate(cfg)
        line["parity"] = parity_report(gpu_check, first)
        line["parity"]["rule"] = parity_rule(gpu_check, cfg)
    print(json.dumps(line), flush=True)


def profile_backward(api, torch, args, rank, l2=False):
    """Forward eval + backward steps over workload 5 (or its first --records
    records), or (l2) the one-pass forward, L2 loss and backward, for a
    profiler; prints the mean step time."""
    M = api.Materials(I.materials(5))
    rec, d, _ = workload_device(api, 5, rank, args.records)
    n = int(d["h"].shape[0])
    gf = torch.from_numpy(np.ascontiguousarray(rec["g"])).cuda()
    f = torch.empty(3, n, device="cuda")
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    gp = torch.empty(M.n_mat, 8, device="cuda")
    target = (gf.abs() * 0.05).contiguous()

    def step():
        if l2:
            api.eval_l2_backward(M, d, target)
            return
        api.eval(M, d, with_pdf=False, out=dict(f=f, status=st))
        api.eval_backward(M, d, gf, out=gp)
    ms, _ = timed(step, args.steps, args.warmup)
    print(json.dumps(dict(profile="l2" if l2 else "backward", workload=I.WORKLOAD_NAME[5],
                          records=n, ms_per_step=ms)), flush=True)


def other_workloads(api, N, torch, args, sm_count):
    res = {}
    steps = max(3, args.steps // 2)
    # near-field eval, 1 material, 65,536 records
    mats = I.materials(1)
    M = api.Materials(mats)
    _, d, _ = workload_device(api, 1, 0)
    n = int(d["h"].shape[0])
    o = dict(f=torch.empty(3, n, device="cuda"), pdf=torch.empty(n, device="cuda"),
             status=torch.empty(n, dtype=torch.uint8, device="cuda"))
    ms, _ = timed(lambda: api.eval(M, d, out=o), steps * 4, 3)
    # the same calls replayed from a CUDA graph (16 calls per graph): the
    # device time per call without the Python binding's per-call host cost
    calls = 16
    g1 = torch.cuda.CUDAGraph()
    s1 = torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s1):
        api.eval(M, d, out=o, stream=s1)
    torch.cuda.current_stream().wait_stream(s1)
    torch.cuda.synchronize()
    with torch.cuda.graph(g1):
        for _ in range(calls):
            api.eval(M, d, out=o)
    ms_g, _ = timed(g1.replay, steps, 3)
    ms_g /= calls
    # the plain form: one launch, one thread per record
    seg1 = np.array([0, n], np.int64)
    po = dict(f=o["f"], wo=torch.empty(3, n, device="cuda"),
              weight=torch.empty(3, n, device="cuda"), pdf=o["pdf"], status=o["status"])
    ms_p, _ = timed(lambda: api.plain(N.OP_EVAL, M, d, seg1, out=po), steps * 4, 3)
    res[I.WORKLOAD_NAME[1]] = dict(records_per_s=n / (ms / 1e3), ms=ms, records=n,
                                   roofline_frac=frac(OPS[1]["eval"], n, ms, sm_count),
                                   graph_ms_per_call=ms_g,
                                   graph_records_per_s=n / (ms_g / 1e3),
                                   graph_roofline_frac=frac(OPS[1]["eval"], n, ms_g, sm_count),
                                   plain_records_per_s=n / (ms_p / 1e3))
    del g1, po
    # multi-scale: fused eval + sample
    mats = I.materials(3)
    M = api.Materials(mats)
    _, d, _ = workload_device(api, 3, 0)
    n = int(d["h"].shape[0])
    o = api.alloc_fused(n, "cuda")
    ms, _ = timed(lambda: api.eval_sample_pdf(M, d, out=o), steps, 2)
    # the stochastic estimators (jittered nodes + GGX-sampled entry)
    ms_st, _ = timed(lambda: api.eval_sample_pdf_stochastic(M, d, 1, 3, out=o),
                     max(3, steps // 4), 2)
    # the plain form of the fused op on the same records sorted by material
    # (sorted outside the timed region)
    ds, seg3 = sorted_copy(d, len(mats))
    ms_p, _ = timed(lambda: api.plain_fused(M, ds, seg3, out=o), max(3, steps // 2), 2)
    res[I.WORKLOAD_NAME[3]] = dict(records_per_s=n / (ms / 1e3), ms=ms, records=n,
                                   roofline_frac=frac(OPS[3]["fused"], n, ms, sm_count),
                                   stochastic_records_per_s=n / (ms_st / 1e3),
                                   plain_fused_records_per_s=n / (ms_p / 1e3))
    del d, o, ds
    torch.cuda.empty_cache()
    # fiber migration (Sec. 3.5): the workload-2 records and materials, each
    # material with 2 map pairs switched along the yarn (tables still fit in
    # shared memory)
    mats = I.materials(2)
    for k, dsc in enumerate(mats):
        dsc.update(migration_maps=2, migration_seed=k, migration_length=0.5,
                   migration_blend=0.25)
    M = api.Materials(mats)
    _, d, _ = workload_device(api, 2, 0)
    n = int(d["h"].shape[0])
    o = api.alloc_fused(n, "cuda")
    ms, _ = timed(lambda: api.eval_sample_pdf(M, d, out=o), max(3, steps // 2), 2)
    res["migration-2maps-" + I.WORKLOAD_NAME[2]] = dict(records_per_s=n / (ms / 1e3), ms=ms,
                                                        records=n)
    del d, o
    torch.cuda.empty_cache()
    # upstream step: 2048 x 2048 camera rays against a plain-weave patch of
    # 32 yarns cut into 512 straight pieces, then the fused BYSDF on the
    # traced records (8 materials)
    sc = I.woven_scene(16, 16)
    Y = api.yarns_to_device(sc)
    rays = {k: torch.from_numpy(v).cuda() for k, v in
            I.camera_rays(2048, 2048, extent=16 * 2.5).items()}
    n = int(rays["o"].shape[1])
    light = (0.3, -0.4, math.sqrt(0.75))
    tr = api.trace_yarns(Y, rays, light)
    rec_t = dict(h=tr["h"], u=tr["u"], v=tr["v"], wi=tr["wi"], wo=tr["wo"], ratio=tr["ratio"],
                 mat_id=tr["mat_id"], u0=torch.rand(n, device="cuda") * 0.9999,
                 u1=torch.rand(n, device="cuda") * 0.9999)
    M = api.Materials(I.materials(2))
    o = api.alloc_fused(n, "cuda")
    # traced records carry footprints of ~0.01 (one node each): the launch
    # shape is tuned once on them, outside the timed region
    tuned = api.autotune(M, N.OP_FUSED, rec_t, out=o)
    ms_tr, _ = timed(lambda: api.trace_yarns(Y, rays, light, out=tr), max(3, steps // 4), 2)

    def render_step():
        api.trace_yarns(Y, rays, light, out=tr)
        api.eval_sample_pdf(M, rec_t, out=o)
    ms_rs, _ = timed(render_step, max(3, steps // 4), 2)
    res["trace-512pieces-2048x2048+fused"] = dict(
        rays_per_s=n / (ms_rs / 1e3), ms=ms_rs, rays=n, trace_only_rays_per_s=n / (ms_tr / 1e3),
        fused_autotuned=tuned,
        trace_ms=ms_tr, hit_share=float((tr["mat_id"] >= 0).float().mean()))
    del rays, tr, rec_t, o
    torch.cuda.empty_cache()
    # batched heterogeneous: 256 materials, Zipf counts, one persistent
    # material-sorted launch per op captured in a CUDA graph, vs plain
    mats = I.materials(4)
    M = api.Materials(mats)
    rec4, d, seg = workload_device(api, 4, 0)
    del rec4
    n = int(d["h"].shape[0])
    o = api.alloc_fused(n, "cuda")
    tuned = api.autotune(M, N.OP_FUSED, d, out=o)
    api.eval_sample_pdf(M, d, out=o)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.eval_sample_pdf(M, d, out=o, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        api.eval_sample_pdf(M, d, out=o)
    ms_graph, _ = timed(g.replay, steps, 2)

    ms_plain, _ = timed(lambda: api.plain_fused(M, d, seg, out=o), max(2, steps // 2), 1)
    # the persistent fused kernel without the graph (one launch per call)
    ms_nograph, _ = timed(lambda: api.eval_sample_pdf(M, d, out=o), max(2, steps // 2), 1)
    res[I.WORKLOAD_NAME[4]] = dict(records_per_s=n / (ms_graph / 1e3), ms=ms_graph, records=n,
                                   autotuned=tuned, plain_fused_records_per_s=n / (ms_plain / 1e3),
                                   speedup_vs_plain_fused=ms_plain / ms_graph,
                                   persistent_without_graph_records_per_s=n / (ms_nograph / 1e3),
                                   roofline_frac=frac(OPS[4]["fused"], n, ms_graph, sm_count))
    del d, o, g
    torch.cuda.empty_cache()
    # forward + backward, 64 materials, material-sorted
    mats = I.materials(5)
    M = api.Materials(mats)
    rec5, d, seg = workload_device(api, 5, 0)
    n = int(d["h"].shape[0])
    gf = torch.from_numpy(rec5["g"]).cuda()
    del rec5
    f = torch.empty(3, n, device="cuda")
    st = torch.empty(n, dtype=torch.uint8, device="cuda")
    gp = torch.empty(64, 8, device="cuda")

    def fwd_bwd():
        api.eval(M, d, with_pdf=False, out=dict(f=f, status=st))
        api.eval_backward(M, d, gf, out=gp)
    ms_fb, _ = timed(fwd_bwd, max(3, steps // 2), 1)
    ms_f, _ = timed(lambda: api.eval(M, d, with_pdf=False, out=dict(f=f, status=st)), steps, 2)
    ms_b, _ = timed(lambda: api.eval_backward(M, d, gf, out=gp), max(3, steps // 2), 1)
    fwd_bwd_ops = tuple(a + b for a, b in zip(OPS[5]["eval"], OPS[5]["backward"]))
    # the fitting step of the workload: forward, L2 loss against target
    # radiance and its gradient in one pass (bysdf_eval_l2_backward), the
    # forward values written; the target is the forward at held-out
    # parameters (20% off), evaluated once outside the timed region
    theta = api.default_params(mats).cuda()
    held = theta * (1 + 0.2 * (2 * torch.rand(theta.shape, generator=torch.Generator().manual_seed(5))
                                .cuda() - 1))
    M.set_params(held)
    target = api.eval(M, d, with_pdf=False)[0].clone()
    M.set_params(theta)
    ms_l2, _ = timed(lambda: api.eval_l2_backward(M, d, target), max(3, steps // 2), 1)
    # its work: the backward's count already holds one forward evaluation;
    # the loss adds 9 flops per record
    l2_ops = (OPS[5]["backward"][0] + 9.0, OPS[5]["backward"][1])
    # the extended parameter set (15 columns), and with the per-record
    # direction products
    ms_x, _ = timed(lambda: api.eval_backward_ext(M, d, gf), max(3, steps // 4), 1)
    ms_xd, _ = timed(lambda: api.eval_backward_ext(M, d, gf, dirs=True), max(3, steps // 8), 1)
    res[I.WORKLOAD_NAME[5]] = dict(records_per_s=n / (ms_l2 / 1e3), ms=ms_l2, records=n,
                                   step="forward + L2 loss + backward in one pass",
                                   roofline_frac=frac(l2_ops, n, ms_l2, sm_count),
                                   roofline_pipe=pipe_of(l2_ops, n, ms_l2, sm_count),
                                   two_calls_records_per_s=n / (ms_fb / 1e3),
                                   two_calls_step="eval, then backward of a given "
                                                  "upstream gradient",
                                   two_calls_roofline_frac=frac(fwd_bwd_ops, n, ms_fb, sm_count),
                                   forward_only_records_per_s=n / (ms_f / 1e3),
                                   roofline_frac_forward=frac(OPS[5]["eval"], n, ms_f, sm_count),
                                   backward_only_records_per_s=n / (ms_b / 1e3),
                                   roofline_frac_backward=frac(OPS[5]["backward"], n, ms_b,
                                                               sm_count),
                                   work_per_record=dict(forward=OPS[5]["eval"],
                                                        backward=OPS[5]["backward"],
                                                        unit="(FP32 flops, XU ops)"),
                                   backward_ext15_records_per_s=n / (ms_x / 1e3),
                                   backward_ext15_dirs_records_per_s=n / (ms_xd / 1e3))
    return res


def pipe_of(ops, n, ms, sm_count):
    """The binding pipe of a roofline fraction (the larger of the two)."""
    fl, xu = ops
    pk = peaks(sm_count, SM_MAX_MHZ)
    t = ms / 1e3
    return "fp32" if fl * n / t / 1e12 / pk["fp32_tflops"] >= xu * n / t / 1e12 / pk["xu_tops"] \
        else "xu"


def frac(ops, n, ms, sm_count):
    fl, xu = ops
    pk = peaks(sm_count, SM_MAX_MHZ)
    t = ms / 1e3
    return max(fl * n / t / 1e12 / pk["fp32_tflops"], xu * n / t / 1e12 / pk["xu_tops"])


if __name__ == "__main__":
    main()
