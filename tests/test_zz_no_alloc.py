"""bysdf_eval_noalloc: eval for callers that may not allocate device memory.

Some callers cannot call cudaMalloc -- for example a plug-in whose host
application owns every device allocation, or code running where an
allocation could synchronise the device or fail.  This entry point takes no
workspace and uses a fixed scratch array inside the library instead.  The
test calls it through the C ABI and checks it against bysdf_eval (the entry
point with a caller-provided workspace), twice in a row, in both scheduling
modes (all tables in shared memory; material-sorted records), and that a
table too large for the fixed scratch is refused.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

REL, ABS = 1e-4, 1e-6   # the tolerance of the parity tests


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12724_gb300 import _native as N
    from paper_2401_12724_gb300 import api
    return api, N.load()


def noalloc_eval(api, lib, M, d):
    n = int(d["h"].shape[0])
    f = torch.full((3, n), -1.0, device="cuda")
    p = torch.full((n,), -1.0, device="cuda")
    st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    rc = lib.bysdf_eval_noalloc(M.handle, C.byref(api.hits_struct(d)), n, f.data_ptr(),
                                p.data_ptr(), st.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == 0, lib.bysdf_last_error().decode()
    torch.cuda.synchronize()
    return f.cpu().numpy(), p.cpu().numpy(), st.cpu().numpy()


def cases():
    # 8 materials, any record order: all tables staged in shared memory
    yield I.materials(2), I.records(2, 0, 7001), None
    # 64 materials, material-sorted with segment offsets (uses the scratch's
    # first-tile table)
    mats = I.materials(4)[:64]
    rec = I.random_records(5003, n_mat=64, seed=91, wi_mode="cosine", sorted_ids=True)
    yield mats, rec, I.seg_offsets_from_ids(rec["mat_id"], 64)


def test_noalloc_eval_matches_eval_twice(mods):
    api, lib = mods
    for mats, rec, seg in cases():
        M = api.Materials(mats)
        d = api.records_to_device(rec, "cuda", seg)
        f_ref, p_ref, st_ref = (t.cpu().numpy() for t in api.eval(M, d))
        for _ in range(2):
            f, p, st = noalloc_eval(api, lib, M, d)
            assert np.array_equal(st, st_ref)
            np.testing.assert_allclose(f, f_ref, rtol=REL, atol=ABS)
            np.testing.assert_allclose(p, p_ref, rtol=REL, atol=ABS)
        M.close()


def header_define(name):
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "bysdf.h")
    return int(re.search(rf"#define {name} (\d+)", open(hdr).read()).group(1))


def test_noalloc_error_word_reads_zero_after_a_normal_call(mods):
    api, lib = mods
    mats, rec, seg = next(cases())
    M = api.Materials(mats)
    noalloc_eval(api, lib, M, api.records_to_device(rec, "cuda", seg))
    err = C.c_uint32(123)
    assert lib.bysdf_noalloc_error(None, C.byref(err)) == 0
    assert err.value == 0
    M.close()


def test_noalloc_refuses_tables_beyond_its_scratch(mods):
    api, lib = mods
    # the fixed scratch holds the 256-byte control block and one 4-byte
    # first-tile entry per material plus an end entry
    limit = (header_define("BYSDF_NOALLOC_SCRATCH_BYTES") - 256) // 4 - 1
    assert limit == header_define("BYSDF_NOALLOC_MAX_MATERIALS")
    n_mat = limit + 1       # one more than the fixed scratch holds
    mats = [I.material(flags=1)] * n_mat
    M = api.Materials(mats)
    rec = I.random_records(64, seed=92, wi_mode="cosine")
    rec["mat_id"] = np.zeros(64, np.int32)
    seg = np.concatenate([[0], np.full(n_mat, 64)]).astype(np.int64)
    d = api.records_to_device(rec, "cuda", seg)
    f = torch.empty(3, 64, device="cuda")
    p = torch.empty(64, device="cuda")
    st = torch.empty(64, dtype=torch.uint8, device="cuda")
    rc = lib.bysdf_eval_noalloc(M.handle, C.byref(api.hits_struct(d)), 64, f.data_ptr(),
                                p.data_ptr(), st.data_ptr(), None)
    assert rc == -4
    assert f"at most {limit}" in lib.bysdf_last_error().decode()
    M.close()
