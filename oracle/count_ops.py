"""Algorithmic work per hit record, counted by the oracle's operation-counting
scalar (test infrastructure; the benchmark's OPS table holds what it prints,
and tests/test_op_counts.py checks that table against a fresh count).

FP32 work = additions/subtractions + multiplications (flops); XU work =
divisions + square roots + transcendental calls (sin, cos, exp, log, atan2,
asin, tan); comparisons are listed apart.  Counted on 4096 records of each
workload, for eval at omega_o (which includes its pdf), for one sample (which
evaluates f and pdf at the sampled direction), and for both in one pass over
the shared geometry (eval + sample - shared part).

Backward (gradients of the per-material parameters): one forward evaluation
(the recompute) plus one reverse sweep over it, each forward operation's
adjoint costed as in reverse-mode differentiation (Griewank and Walther,
"Evaluating Derivatives", 2008): z = a +- b: 2 adds; z = a b: 2 mul + 2
adds; z = a / b: 1 div + 1 mul + 2 adds; z = sqrt(a): 1 div + 1 mul + 1
add; z = f(a) transcendental: 1 transcendental + 1 mul + 1 add.  The cost
does not depend on how many parameters are differentiated.

Run:  python oracle/count_ops.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2401_12724_gb300 import inputs as I  # noqa: E402


def adjoint(add, mul, div, sq, tr):
    """Reverse-sweep (add, mul, xu) of a forward evaluation with these counts."""
    a = 2 * add + 2 * mul + 2 * div + sq + tr
    m = 2 * mul + div + sq + tr
    x = div + sq + tr
    return a, m, x


def per_record(cfg, op, n=4096):
    rec = I.records(cfg, 0, n)
    c = oracle.count_ops(I.materials(cfg), rec, op)
    add, mul, div, sq, tr, cmp_ = c.mean(0)
    out = dict(flops=add + mul, xu=div + sq + tr, cmp=cmp_)
    if op == 0:
        a, m, x = adjoint(add, mul, div, sq, tr)
        out["bwd_flops"] = add + mul + a + m
        out["bwd_xu"] = div + sq + tr + x
    return out


def table():
    """{workload: {op: (flops, xu)}} as the benchmark's OPS table holds it."""
    res = {}
    for cfg in (1, 2, 3, 4, 5):
        ev = per_record(cfg, 0)
        res[cfg] = dict(eval=(ev["flops"], ev["xu"]))
        if cfg in (2, 3, 4):
            sm = per_record(cfg, 1)
            sh = per_record(cfg, 3)
            res[cfg]["fused"] = (ev["flops"] + sm["flops"] - sh["flops"],
                                 ev["xu"] + sm["xu"] - sh["xu"])
        if cfg == 5:
            res[cfg]["backward"] = (ev["bwd_flops"], ev["bwd_xu"])
    return res


def main():
    for cfg, ops in table().items():
        print(f"workload {cfg} {I.WORKLOAD_NAME[cfg]}: " +
              " | ".join(f"{op} flops {fl:.1f} xu {xu:.1f}" for op, (fl, xu) in ops.items()))


if __name__ == "__main__":
    main()
