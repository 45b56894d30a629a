"""The benchmark's roofline numerator (bench.OPS, algorithmic work per
record) against a fresh count by the oracle's operation-counting scalar: a
change to the oracle's arithmetic that is not carried into the table fails
here."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load(rel, name):
    spec = importlib.util.spec_from_file_location(name, os.path.join(ROOT, rel))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_bench_op_table_matches_a_fresh_count(orc):
    bench = _load("bench.py", "bench_for_ops")
    count = _load("oracle/count_ops.py", "count_ops_for_ops")
    fresh = count.table()
    assert set(fresh) == set(bench.OPS)
    for cfg, ops in fresh.items():
        assert set(ops) == set(bench.OPS[cfg]), cfg
        for op, (fl, xu) in ops.items():
            bfl, bxu = bench.OPS[cfg][op]
            assert bfl == pytest.approx(fl, abs=0.051), (cfg, op, fl)
            assert bxu == pytest.approx(xu, abs=0.051), (cfg, op, xu)


def test_reverse_sweep_cost_model(orc):
    # one operation of each kind: the adjoint costs of the docstring
    count = _load("oracle/count_ops.py", "count_ops_for_model")
    assert count.adjoint(1, 0, 0, 0, 0) == (2, 0, 0)
    assert count.adjoint(0, 1, 0, 0, 0) == (2, 2, 0)
    assert count.adjoint(0, 0, 1, 0, 0) == (2, 1, 1)
    assert count.adjoint(0, 0, 0, 1, 0) == (1, 1, 1)
    assert count.adjoint(0, 0, 0, 0, 1) == (1, 1, 1)


def test_oracle_rate_script_measures_every_workload(orc, monkeypatch):
    # oracle/rates.py (the CPU reference rates of the measured table): one
    # short pass per workload and thread count, on small samples
    rates = _load("oracle/rates.py", "oracle_rates")
    monkeypatch.setattr(rates, "workload_sample",
                        lambda cfg, n, f=rates.workload_sample: f(cfg, min(n, 512)))
    for cfg in (1, 4, 5):
        r = rates.rate(cfg, 2, 1 << 9, 0.0)
        assert r["records"] == 512 and r["records_per_s"] > 0 and r["threads"] == 2
