"""Checkpoint and resume of a fitting run (the forward + L2 loss + backward
workload's optimisation loop): the state is the parameter tensor and the
optimiser's state, saved with torch.save.  With the deterministic backward,
a run interrupted after 6 Adam steps and resumed from the checkpoint (a new
parameter tensor and optimiser loaded from it) ends bit for bit where the
uninterrupted run ends after 12, and its loss fell."""
import io

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


def test_fit_checkpoint_resume_is_exact(api):
    mats = I.materials(5)[:4]
    n = 1 << 15
    rec = I.random_records(n, n_mat=4, seed=81, wi_mode="cosine", sorted_ids=True, v_max=5.0)
    seg = I.seg_offsets_from_ids(rec["mat_id"], 4)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", seg)
    truth = api.default_params(mats).cuda()
    M.set_params(truth)
    target = api.eval(M, d, with_pdf=False)[0].clone()
    start = truth.clone()
    start[:, 0:3] *= 0.8       # albedo
    start[:, 3:5] *= 1.2       # roughness
    start[:, 7] *= 0.8         # shadow density
    mask = torch.zeros_like(start)
    mask[:, [0, 1, 2, 3, 4, 7]] = 1.0   # the helix angles stay fixed

    def run(th, opt, steps):
        losses = []
        for _ in range(steps):
            opt.zero_grad()
            L = api.bysdf_l2_loss(th, M, d, target, deterministic=True)
            L.backward()
            th.grad *= mask
            opt.step()
            losses.append(float(L.detach()))
        return losses

    th = start.clone().requires_grad_(True)
    opt = torch.optim.Adam([th], lr=0.01)
    first = run(th, opt, 6)
    buf = io.BytesIO()
    torch.save({"params": th.detach().cpu(), "opt": opt.state_dict(), "step": 6}, buf)
    rest = run(th, opt, 6)
    end_straight = th.detach().cpu().numpy()

    buf.seek(0)
    ck = torch.load(buf, weights_only=False)
    assert ck["step"] == 6
    th2 = ck["params"].cuda().requires_grad_(True)
    opt2 = torch.optim.Adam([th2], lr=0.01)
    opt2.load_state_dict(ck["opt"])
    rest2 = run(th2, opt2, 6)
    assert rest2 == rest
    assert np.array_equal(th2.detach().cpu().numpy(), end_straight)
    assert rest[-1] < first[0]
    M.close()
