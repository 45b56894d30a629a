"""Host-side fault injection: device allocations made to fail through the
library's test hook (bysdf_test_fail_allocations), without exhausting the
device.  The allocating calls return BYSDF_E_CUDA, write no handle and free
what they had taken (repeated failures leave the device's free memory where
it was); the next call without the hook works; and the calls that promise to
allocate nothing (every op on a caller's workspace, the no-allocation eval)
run to the same results while every allocation would fail."""
import ctypes as C

import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12724_gb300 import _native as N
    from paper_2401_12724_gb300 import api
    lib = N.load()
    yield api, N, lib
    lib.bysdf_test_fail_allocations(0)


def create(api, N, lib, mats):
    arr = (N.MaterialDesc * len(mats))(*[api.desc_struct(d) for d in mats])
    h = C.c_void_p()
    rc = lib.bysdf_create_materials(arr, len(mats), None, C.byref(h))
    return rc, h


def test_material_table_allocation_failure(mods):
    api, N, lib = mods
    mats = I.materials(2)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(20):
        assert lib.bysdf_test_fail_allocations(1) == 0
        rc, h = create(api, N, lib, mats)
        assert rc == -2
        assert "cudaMalloc: out of memory" in lib.bysdf_last_error().decode()
        assert h.value is None
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (2 << 20)
    # the hook is used up: the next create works
    rc, h = create(api, N, lib, mats)
    assert rc == 0 and h.value is not None
    assert lib.bysdf_destroy_materials(h) == 0


def test_host_pipeline_allocation_failure(mods):
    api, N, lib = mods
    M = api.Materials(I.materials(2))
    p = C.c_void_p()
    assert lib.bysdf_test_fail_allocations(1) == 0
    assert lib.bysdf_host_pipeline_create(M.handle, 1 << 16, 0, C.byref(p)) == -2
    assert p.value is None
    assert lib.bysdf_host_pipeline_create(M.handle, 1 << 16, 0, C.byref(p)) == 0
    assert p.value is not None
    assert lib.bysdf_host_pipeline_destroy(p) == 0
    M.close()


def test_ops_allocate_nothing(mods):
    api, N, lib = mods
    mats = I.materials(2)
    rec = I.random_records(4099, n_mat=8, seed=77, wi_mode="cosine", sample=True)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", None)
    n = 4099
    g = torch.ones(3, n, device="cuda")
    ws = M.workspace(n)
    ref = [t.cpu().numpy() for t in api.eval(M, d)]
    fused_ref = {k: v.cpu().numpy() for k, v in api.eval_sample_pdf(M, d).items()}
    f_na = torch.empty(3, n, device="cuda")
    p_na = torch.empty(n, device="cuda")
    s_na = torch.empty(n, dtype=torch.uint8, device="cuda")
    try:
        # every allocation the library tried now would fail
        assert lib.bysdf_test_fail_allocations(1 << 30) == 0
        got = [t.cpu().numpy() for t in api.eval(M, d)]
        fused = {k: v.cpu().numpy() for k, v in api.eval_sample_pdf(M, d).items()}
        gp = api.eval_backward(M, d, g).cpu().numpy()
        rc = lib.bysdf_eval_noalloc(M.handle, C.byref(api.hits_struct(d)), n, f_na.data_ptr(),
                                    p_na.data_ptr(), s_na.data_ptr(), None)
        assert rc == 0, lib.bysdf_last_error().decode()
        torch.cuda.synchronize()
    finally:
        lib.bysdf_test_fail_allocations(0)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    for k in fused_ref:
        assert np.array_equal(fused[k], fused_ref[k]), k
    assert np.isfinite(gp).all() and np.abs(gp).sum() > 0
    assert np.array_equal(s_na.cpu().numpy(), ref[2])
    assert ws.data_ptr() == M.workspace(n).data_ptr()
    M.close()
