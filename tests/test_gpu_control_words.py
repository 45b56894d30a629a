"""The workspace's control words (tile-draw counter, error word) claimed by
each launch for its own epoch, with no reset kernel for records in any
order: a workspace full of garbage, a captured launch replayed with its one
epoch, and calls of several kinds taking turns on one workspace all give the
results of a clean call, bit for bit (the per-record arithmetic does not
depend on which warp draws which tile)."""
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


def host(t):
    return {k: v.cpu().numpy() for k, v in t.items()} if isinstance(t, dict) else \
        tuple(v.cpu().numpy() for v in t)


def same(a, b):
    if isinstance(a, dict):
        return all(np.array_equal(a[k], b[k]) for k in a)
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def setup(api, n=20011, seed=33):
    mats = I.materials(2)
    rec = I.random_records(n, n_mat=8, seed=seed, wi_mode="cosine", sample=True)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", None)
    return M, d, n


def test_garbage_workspace(api):
    M, d, n = setup(api)
    ref = host(api.eval_sample_pdf(M, d))
    ws = M.workspace(n)
    for fill in (0xFF, 0x00, 0x5A):
        ws.fill_(fill)
        assert same(host(api.eval_sample_pdf(M, d)), ref), fill
    # random bytes, and a previous launch's words left behind by a call of
    # another kind
    ws.copy_(torch.randint(0, 256, ws.shape, dtype=torch.uint8, device="cuda"))
    assert same(host(api.eval_sample_pdf(M, d)), ref)
    g = torch.ones(3, n, device="cuda")
    gp = api.eval_backward(M, d, g).cpu().numpy()
    ev = host(api.eval(M, d))
    assert same(host(api.eval_sample_pdf(M, d)), ref)
    ws.fill_(0xFF)
    # float32 atomics add the records in another order each call
    gp2 = api.eval_backward(M, d, g).cpu().numpy()
    np.testing.assert_allclose(gp2, gp, rtol=1e-4, atol=1e-4 * np.abs(gp).max())
    assert same(host(api.eval(M, d)), ev)
    assert M.workspace_error() == 0
    M.close()


def test_captured_launch_replays_with_its_epoch(api):
    M, d, n = setup(api, n=70001, seed=34)
    ref = host(api.eval_sample_pdf(M, d))
    out = api.alloc_fused(n, "cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        api.eval_sample_pdf(M, d, out=out, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):          # one launch: every replay has one epoch
        api.eval_sample_pdf(M, d, out=out)
    for _ in range(3):
        for v in out.values():
            v.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert same(host(out), ref)
    # an uncaptured call between replays, then another replay
    assert same(host(api.eval_sample_pdf(M, d)), ref)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert same(host(out), ref)
    assert M.workspace_error() == 0
    M.close()


def test_small_batches_back_to_back(api):
    # many short launches in a row on one workspace, each its own epoch,
    # sizes from one partial tile to a few waves
    M, d, n = setup(api, n=65536, seed=35)
    ref = host(api.eval(M, d))
    for m in (1, 31, 33, 4097, 65536, 7, 65536):
        sub = {k: (v[..., :m].contiguous() if isinstance(v, torch.Tensor) and v.dim() and
                   v.shape[-1] == n else v) for k, v in d.items()}
        got = host(api.eval(M, sub))
        assert same(got, tuple(r[..., :m] for r in ref)), m
    M.close()
