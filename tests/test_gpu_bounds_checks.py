"""The index-checking build of the library (libbysdf_bounds.so, built with
-DBYSDF_DEBUG_BOUNDS; the stand-in for a memory checker): every checked
index -- texel of the fiber maps, migration segment and map, record index,
material id and table offset in shared memory, record range of a tile --
that falls out of range would set bit 2 of the launch's error word and be
clamped.  The workloads of bounds_workloads.py run under it in a child
process: no check fires (every error word reads 0), and the outputs are the
product build's on the same inputs (to within float rounding where the two
builds' code may form FMAs differently)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_index_checks_never_fire(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, HERE)
    import bounds_workloads as W
    errs = W.run(str(tmp_path / "product.npz"))
    assert not errs, errs
    env = dict(os.environ, BYSDF_BOUNDS_CHECKS="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_workloads.py"),
                        str(tmp_path / "bounds.npz")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    a = np.load(tmp_path / "product.npz")
    b = np.load(tmp_path / "bounds.npz")
    assert int(a["_bounds_library"][0]) == 0 and int(b["_bounds_library"][0]) == 1
    assert set(a.files) == set(b.files)
    for k in a.files:
        if k.startswith("_"):
            continue
        x, y = a[k], b[k]
        if x.dtype.kind in "ui":
            assert np.array_equal(x, y), k
        elif k.startswith("bwd_any"):
            # float32 atomics: the records add in another order per call
            np.testing.assert_allclose(x, y, rtol=1e-4, atol=1e-4 * (np.abs(x).max() + 1e-6),
                                       err_msg=k)
        elif k in ("ext.1", "ext.2"):
            # the direction products (six-tangent dual numbers): the two
            # builds' code differs, and where an FMA is formed may differ
            # with it; a rounding difference is amplified on the records
            # next to a branch, so the share within 1e-3 is what is checked
            tol = 1e-3 * np.abs(x) + 1e-5 * (np.abs(x).max() + 1e-6)
            share = (np.abs(x - y) <= tol).mean()
            assert share >= 0.99 and np.isfinite(y).all(), (k, share)
        else:
            np.testing.assert_allclose(x, y, rtol=1e-6, atol=1e-9, err_msg=k)
