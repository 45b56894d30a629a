"""Records per second of the FP64 oracle, as it stands, on this host's cores
(test infrastructure: a CPU reference rate for each workload, on one thread
and on all of them; nothing here is tuned).

Per workload, the oracle runs what the GPU step runs: eval at omega_o (with
pdf) for the near-field eval workload; eval plus one sample for the fused
workloads; eval plus the parameter gradient for the forward + backward
workload.  Records are bounded prefixes of the seeded workloads (for the
material-sorted 256-material batch, eight runs spread over the batch, so
that several materials are included); each measurement repeats its pass
until about `seconds` have passed.

Run:  python oracle/rates.py [--seconds S]   (prints one JSON line)
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2401_12724_gb300 import inputs as I  # noqa: E402

OPS = {1: "eval", 2: "eval+sample", 3: "eval+sample", 4: "eval+sample", 5: "eval+gradient"}


def workload_sample(cfg: int, n: int) -> dict:
    if cfg != 4:
        return I.records(cfg, 0, min(n, I.N_RECORDS[cfg]))
    total, parts = I.N_RECORDS[4], 8
    runs = [I.records(4, k * (total // parts), n // parts) for k in range(parts)]
    return {k: np.concatenate([r[k] for r in runs], axis=-1) for k in runs[0]}


def one_pass(cfg: int, mats, rec: dict, threads: int):
    if cfg == 1:
        oracle.eval_records(mats, rec, threads=threads)
    elif cfg == 5:
        oracle.eval_records(mats, rec, threads=threads)
        oracle.grad_records(mats, rec, np.asarray(rec["g"], np.float64), threads=threads)
    else:
        oracle.eval_records(mats, rec, threads=threads)
        oracle.sample_records(mats, rec, threads=threads)


def rate(cfg: int, threads: int, n: int, seconds: float) -> dict:
    mats = I.materials(cfg)
    rec = workload_sample(cfg, n)
    m = int(rec["h"].shape[0])
    done, t0 = 0, time.perf_counter()
    while True:
        one_pass(cfg, mats, rec, threads)
        done += m
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return dict(records_per_s=done / dt, records=done, seconds=dt, threads=threads)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=3.0)
    args = ap.parse_args()
    cores = os.cpu_count() or 1
    out = dict(cores=cores)
    for cfg in (1, 2, 3, 4, 5):
        out[I.WORKLOAD_NAME[cfg]] = dict(
            op=OPS[cfg],
            one_thread=rate(cfg, 1, 1 << 14, args.seconds),
            all_threads=rate(cfg, cores, 1 << 17, args.seconds))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
