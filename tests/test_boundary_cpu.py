"""The C-ABI boundary without a GPU: the library builds and loads, exports
every symbol include/bysdf.h declares, and rejects bad host-side input with
status codes before touching the device.  Also the sharded multi-rank path
(world size 2, gloo) on CPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2401_12724_gb300 import _native as N
from paper_2401_12724_gb300 import dist as D
from paper_2401_12724_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bysdf.h")


@pytest.fixture(scope="module")
def lib():
    return N.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bysdf_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    decl = declared_symbols()
    assert len(decl) >= 18
    out = subprocess.run(["nm", "-D", "--defined-only", N.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines()}
    missing = [s for s in decl if s not in exported]
    assert not missing, missing
    # and the ctypes table covers them all
    assert sorted(s for s, _, _ in N.SYMBOLS) == decl
    assert lib.bysdf_version().startswith(b"libbysdf")


def desc(**over):
    from paper_2401_12724_gb300.api import desc_struct  # torch-free path below
    return desc_struct(I.material(**over))


@pytest.mark.parametrize("field,value,msg", [
    ("n_plies", 0, "n_plies"), ("n_plies", 9, "n_plies"), ("fibers_per_ply", 3, "fibers_per_ply"),
    ("map_texels", 2048, "map_texels"), ("trace_iters", 0, "trace_iters"), ("k_max", 65, "k_max"),
    ("eta", 1.0, "eta"), ("packing", 0.0, "packing"), ("body_B", 1.5, "body_B"),
    ("body_r", -0.1, "body_r"), ("sigma_t", -1.0, "sigma_t"), ("yarn_radius", 0.0, "yarn_radius"),
    ("ply_twist_deg", 90.0, "ply_twist"), ("shadow_density", float("nan"), "shadow_density"),
])
def test_create_rejects_bad_descriptor(lib, field, value, msg):
    pytest.importorskip("torch")
    d = desc(**{field: value})
    out = C.c_void_p()
    rc = lib.bysdf_create_materials(C.byref(d), 1, None, C.byref(out))
    assert rc == -1
    assert msg in lib.bysdf_last_error().decode()
    assert out.value is None


def test_null_arguments_are_rejected(lib):
    h = N.Hits()
    assert lib.bysdf_eval(None, C.byref(h), 10, None, None, None, None, 0, None) == -1
    assert lib.bysdf_sample(None, C.byref(h), None, None, 10, None, None, None, None, None, 0,
                            None) == -1
    assert lib.bysdf_pdf(None, C.byref(h), 10, None, None, None, 0, None) == -1
    assert lib.bysdf_eval_backward(None, C.byref(h), 10, None, None, 0, None, 0, None) == -1
    assert lib.bysdf_create_materials(None, 1, None, None) == -1
    assert lib.bysdf_workspace_size(None, 100) == 0
    c = N.LaunchConfig(256, 2, 0, 0)
    assert lib.bysdf_set_launch_config(None, 0, C.byref(c)) == -1
    assert lib.bysdf_set_params(None, None, None) == -1
    err = C.c_uint32()
    assert lib.bysdf_workspace_error(None, None, C.byref(err)) == -1


def test_allocation_failure_hook_arguments(lib):
    # the hook itself is host-only: a negative count is refused, 0 switches
    # it off (its effect on the allocating calls is a GPU test)
    assert lib.bysdf_test_fail_allocations(-1) == -1
    assert "count" in lib.bysdf_last_error().decode()
    assert lib.bysdf_test_fail_allocations(3) == 0
    assert lib.bysdf_test_fail_allocations(0) == 0


def test_shard_bounds_cover_and_balance():
    for n in (0, 1, 7, 1000, 2 ** 24 + 3):
        for w in (1, 2, 3, 8):
            rs = [D.shard_bounds(n, w, r) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [e - b for b, e in rs]
            assert max(sizes) - min(sizes) <= 1
    seg = np.array([0, 5, 5, 12, 20], np.int64)
    np.testing.assert_array_equal(D.shard_segments(seg, 4, 13), [0, 1, 1, 8, 9])


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mats = I.materials(5)[:6]
    n = 3000
    rec = I.random_records(n, n_mat=6, seed=81, wi_mode="cosine", sorted_ids=True, v_max=5.0)
    g = np.random.default_rng(82).uniform(-1, 1, (3, n))
    b, e = D.shard_bounds(n, world, rank)
    part = {k: v[..., b:e] for k, v in rec.items()}
    grad, _ = oracle.grad_records(mats, part, g[:, b:e])
    t = torch.from_numpy(grad)
    D.allreduce_param_grads(t)
    q.put((rank, t.numpy()))
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce_gloo():
    """Records sharded over two gloo ranks: the all-reduced per-material
    gradients equal the single-process gradient of all records."""
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    import socket

    import oracle
    oracle.build()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    mats = I.materials(5)[:6]
    n = 3000
    rec = I.random_records(n, n_mat=6, seed=81, wi_mode="cosine", sorted_ids=True, v_max=5.0)
    g = np.random.default_rng(82).uniform(-1, 1, (3, n))
    full, _ = oracle.grad_records(mats, rec, g)
    for r in (0, 1):
        np.testing.assert_allclose(res[r], full, rtol=1e-10, atol=1e-12)
    del torch


def test_bench_parity_report_counts_planted_errors():
    # the bench's parity summary: a GPU result equal to the oracle's up to
    # float32 rounding is within tolerance; planted errors of 1% (f) and a
    # status mismatch are counted, and a record whose sampled lobe differs
    # is left out of the sample comparison
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    n = 2000
    g = np.random.default_rng(3)
    fo, po = g.random((3, n)) + 0.1, g.random(n) + 0.1
    so = np.zeros(n, np.uint8)
    so[:20] = 1
    w_o, ps_o = g.random((3, n)) + 0.1, g.random(n) + 0.1
    ss_o = np.zeros(n, np.uint8)
    lb_o = g.integers(0, 4, n).astype(np.uint8)
    gpu = dict(f=fo.astype(np.float32), pdf=po.astype(np.float32), status=so.copy(),
               weight=w_o.astype(np.float32), pdf_s=ps_o.astype(np.float32),
               lobe_status=(ss_o | (lb_o << 4)).astype(np.uint8))
    gpu["f"][1, 100] *= 1.01
    gpu["f"][0, 101] *= 1.01
    gpu["status"][5] = 0                       # status mismatch (and not compared)
    gpu["lobe_status"][7] = (lb_o[7] ^ 1) << 4  # other lobe: left out
    gpu["weight"][2, 7] *= 2.0
    r = bench.parity_report(gpu, ((fo, po, so), (None, w_o, ps_o, ss_o, lb_o)))
    assert r["records"] == n
    assert r["status_equal"] == (n - 1) / n
    assert r["sample_status_equal"] == (n - 1) / n
    n_cmp = (n - 20) + (n - 1)                 # eval records both ok + sample records kept
    assert abs(r["within_tol"] - (n_cmp - 2) / n_cmp) < 1e-12
    assert 0.009 < r["rel_err_max"] < 0.011 and r["rel_err_p50"] < 1e-6


def test_bench_reference_arm_prints_the_contract_line():
    # bench.py --impl reference: the FP64 oracle on the host cores, one JSON
    # line with the contract's keys (runs without a GPU)
    import json
    import sys
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
