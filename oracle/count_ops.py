"""Algorithmic work per hit record, counted by the oracle's operation-counting
scalar (test infrastructure; the benchmark uses the numbers it prints).

FP32 work = additions/subtractions + multiplications (flops); XU work =
divisions + square roots + transcendental calls (sin, cos, exp, log, atan2,
asin, tan); comparisons are listed apart.  Counted on 4096 records of each
workload, for eval at omega_o (which includes its pdf), for one sample (which
evaluates f and pdf at the sampled direction), and for both in one pass over
the shared geometry (eval + sample - shared part).

Run:  python oracle/count_ops.py
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2401_12724_gb300 import inputs as I  # noqa: E402


def per_record(cfg, op, n=4096):
    rec = I.records(cfg, 0, n)
    c = oracle.count_ops(I.materials(cfg), rec, op)
    add, mul, div, sq, tr, cmp_ = c.mean(0)
    return dict(flops=add + mul, xu=div + sq + tr, cmp=cmp_)


def main():
    for cfg in (1, 2, 3, 4, 5):
        ev = per_record(cfg, 0)
        line = f"workload {cfg} {I.WORKLOAD_NAME[cfg]}: eval flops {ev['flops']:.1f} xu {ev['xu']:.1f}"
        if cfg in (2, 3, 4):
            sm = per_record(cfg, 1)
            sh = per_record(cfg, 3)
            fu = {k: ev[k] + sm[k] - sh[k] for k in ev}
            line += (f" | sample flops {sm['flops']:.1f} xu {sm['xu']:.1f}"
                     f" | fused eval+sample flops {fu['flops']:.1f} xu {fu['xu']:.1f}")
        print(line)


if __name__ == "__main__":
    main()
