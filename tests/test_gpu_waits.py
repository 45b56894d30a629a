"""The bounded waits of the persistent kernels, made to give up through the
library's test hook (bysdf_test_stall_table_waits: every table wait polls a
barrier that nothing arrives on, a few polls long).  No fault and no hang:
the kernels wait for their real copies once more and finish.  Checks that
the workspace's error word reports it, that every record of the call gets a
defined result (status 4, zero outputs -- not a previous call's contents),
and that the next call without the hook is clean."""
import numpy as np
import pytest

from paper_2401_12724_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_12724_gb300 import api as A
    return A


@pytest.mark.parametrize("sorted_mode", [False, True])
def test_table_waits_give_up_and_mark_every_record(api, sorted_mode):
    mats = I.materials(2)
    n = 5003
    rec = I.random_records(n, n_mat=8, seed=31, wi_mode="cosine", sample=True,
                           sorted_ids=sorted_mode)
    seg = I.seg_offsets_from_ids(rec["mat_id"], 8) if sorted_mode else None
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", seg)
    good = api.eval_sample_pdf(M, d)
    good = {k: v.cpu().numpy() for k, v in good.items()}
    assert M.workspace_error() == 0
    # outputs filled with garbage first: the aborted call must overwrite them
    out = api.alloc_fused(n, "cuda")
    for k, v in out.items():
        v.fill_(7 if v.dtype == torch.uint8 else 3.0)
    M.test_stall_table_waits(64)
    api.eval_sample_pdf(M, d, out=out)
    torch.cuda.synchronize()
    err = M.workspace_error()
    assert err == 1, err              # the wait gave up; no copy left in flight
    o = {k: v.cpu().numpy() for k, v in out.items()}
    assert (o["status"] == 4).all() and (o["lobe_status"] == 4).all()
    for k in ("f", "pdf", "wo", "weight", "pdf_s"):
        assert (o[k] == 0).all(), k
    # the backward gives up the same way: gradients of nothing
    g = torch.ones(3, n, device="cuda")
    gp = api.eval_backward(M, d, g).cpu().numpy()
    assert M.workspace_error() == 1
    assert (gp == 0).all()
    # hook off: the same call is clean and gives the earlier results
    M.test_stall_table_waits(0)
    again = {k: v.cpu().numpy() for k, v in api.eval_sample_pdf(M, d, out=out).items()}
    assert M.workspace_error() == 0
    for k in good:
        assert np.array_equal(again[k], good[k]), k
    M.close()
