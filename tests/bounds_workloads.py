"""Workloads run under both builds of the library by test_gpu_bounds_checks:
each op on ragged record counts, in both scheduling modes, with footprints,
fiber migration, the stochastic estimators, the backward kinds and invalid
records.  run(path) executes them with whichever library this process
loads, checks after every op that the workspace's error word is 0, and
saves every output to path (.npz).  Run as a script under
BYSDF_BOUNDS_CHECKS=1 it uses the index-checking build."""
import sys

import numpy as np


def run(path):
    import torch

    from paper_2401_12724_gb300 import _native as N
    from paper_2401_12724_gb300 import api
    from paper_2401_12724_gb300 import inputs as I

    out = {}
    errs = []

    def keep(name, M, res):
        e = M.workspace_error()
        if e != 0:
            errs.append((name, e))
        if isinstance(res, dict):
            for k, v in res.items():
                out[f"{name}.{k}"] = v.detach().cpu().numpy()
        else:
            for k, v in enumerate(res):
                if v is not None:
                    out[f"{name}.{k}"] = v.detach().cpu().numpy()

    # any order, all tables in shared memory; a ragged count
    mats = I.materials(2)
    rec = I.random_records(20011, n_mat=8, seed=301, wi_mode="cosine", sample=True)
    rec["h"][3] = np.nan          # invalid records on the way
    rec["mat_id"][4] = 9
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", None)
    keep("eval", M, api.eval(M, d))
    keep("sample", M, api.sample(M, d))
    keep("pdf", M, api.pdf(M, d))
    keep("fused", M, api.eval_sample_pdf(M, d))
    keep("stoch", M, api.eval_sample_pdf_stochastic(M, d, 7, 3))
    g = torch.from_numpy(np.random.default_rng(302).uniform(-1, 1, (3, 20011)).astype(np.float32)).cuda()
    gb = api.eval_backward(M, d, g)
    keep("bwd_any", M, (gb,))
    one = {k: (v[..., :1].contiguous() if torch.is_tensor(v) and v.dim() and v.shape[-1] == 20011
               else v) for k, v in d.items()}
    keep("one", M, api.eval_sample_pdf(M, one))
    M.close()
    # footprints (multi-scale nodes)
    mats = I.materials(3)
    rec = I.records(3, 0, 8191)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", None)
    keep("ms", M, api.eval_sample_pdf(M, d))
    M.close()
    # material-sorted records, 64 materials: forward and every backward kind
    mats = I.materials(5)
    rec = I.random_records(9001, n_mat=64, seed=303, wi_mode="cosine", sorted_ids=True,
                           sample=True, v_max=20.0)
    rec["ratio"] = np.where(np.arange(9001) % 3 == 0, 0.4, 0.0).astype(np.float32)
    seg = I.seg_offsets_from_ids(rec["mat_id"], 64)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", seg)
    keep("sorted", M, api.eval_sample_pdf(M, d))
    g = torch.from_numpy(np.random.default_rng(304).uniform(-1, 1, (3, 9001)).astype(np.float32)).cuda()
    keep("bwd_det", M, (api.eval_backward(M, d, g, deterministic=True),))
    target = (g.abs() * 0.05).contiguous()
    gp, loss, f = api.eval_l2_backward(M, d, target, deterministic=True)
    keep("l2", M, (gp, loss, f))
    keep("ext", M, api.eval_backward_ext(M, d, g, dirs=True, deterministic=True))
    M.close()
    # fiber migration
    mats = I.materials(2)
    for k, dsc in enumerate(mats):
        dsc.update(migration_maps=2, migration_seed=k, migration_length=0.5,
                   migration_blend=0.25)
    rec = I.random_records(5003, n_mat=8, seed=305, wi_mode="cosine", sample=True, v_max=20.0)
    M = api.Materials(mats)
    d = api.records_to_device(rec, "cuda", None)
    keep("mig", M, api.eval_sample_pdf(M, d))
    M.close()
    torch.cuda.synchronize()
    out["_bounds_library"] = np.array([int(N.bounds_checks())])
    np.savez(path, **out)
    return errs


if __name__ == "__main__":
    errs = run(sys.argv[1])
    if errs:
        print("error words:", errs)
        sys.exit(1)
