"""Batches (hgf_batch_*): many mixed-size jobs forked over internal streams, run directly and as
one captured CUDA graph, give the same results as each job prepared and aggregated alone; the
degree-3 and bfloat16 jobs also match the float64 oracle directly."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

JOBS = [dict(w=320, h=240, L=32, seed=401, degree=2, r=9),
        dict(w=160, h=120, L=12, seed=402, degree=1, r=4),
        dict(w=257, h=131, L=7, seed=403, degree=2, r=4, dtype="f16"),
        dict(w=200, h=100, L=9, seed=404, degree=3, r=9),
        dict(w=64, h=48, L=16, seed=405, degree=1, r=4),
        dict(w=300, h=220, L=20, seed=406, degree=2, r=9, dtype="bf16")]


@pytest.mark.parametrize("kernel", [0, 1])
def test_batch_equals_alone_direct_and_graph(kernel):
    """kernel = 0: every job on the internal streams (two-kernel path); kernel = 1: the RGB
    degree-1/2 jobs in one persistent single-pass launch, the others on the streams. Either way
    each job equals the same job run alone under the same tuning, bit for bit."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf, synth
    build.build()
    ctx = hgf.hgf_create(0)
    hgf.hgf_set_tuning(ctx, kernel=kernel)
    items = []
    try:
        for sp in JOBS:
            dt = sp.get("dtype", "f32")
            case = synth.make_case(sp["w"], sp["h"], sp["L"], sp["seed"], dt)
            img = torch.from_numpy(case.guidance).cuda()
            if dt == "bf16":
                cost = torch.from_numpy(case.cost.view(np.int16)).cuda().view(torch.bfloat16)
            else:
                cost = torch.from_numpy(case.cost).cuda()
            p = hgf.make_params(degree=sp["degree"], r=sp["r"], eps=1e-4)
            g = hgf.hgf_prepare(ctx, img, p)
            lab = torch.empty((sp["h"], sp["w"]), dtype=torch.int32, device="cuda")
            best = torch.empty((sp["h"], sp["w"]), device="cuda")
            hgf.hgf_aggregate(ctx, g, cost, labels=lab, best=best)
            torch.cuda.synchronize()
            hgf.hgf_guidance_release(g)
            out_l = torch.full_like(lab, -1)
            out_b = torch.full_like(best, float("nan"))
            items.append(dict(img=img, cost=cost, p=p, ref=(lab.cpu().numpy(), best.cpu().numpy()),
                              out=(out_l, out_b), case=case, spec=sp))
        jobs = [hgf.make_job(it["img"], it["cost"], it["p"], labels=it["out"][0],
                             best=it["out"][1]) for it in items]
        batch = hgf.hgf_batch_create(ctx, jobs, streams=3)
        try:
            for runner in (hgf.hgf_batch_run, hgf.hgf_batch_launch_graph,
                           hgf.hgf_batch_launch_graph):
                for it in items:
                    it["out"][0].fill_(-1)
                    it["out"][1].fill_(float("nan"))
                direct = runner is hgf.hgf_batch_run
                hgf.hgf_profile_enable(ctx, direct)   # launches in a graph are not bracketed
                runner(ctx, batch)
                torch.cuda.synchronize()
                hgf.hgf_profile_enable(ctx, False)
                if direct:
                    names = set(hgf.hgf_profile_report(ctx))
                    assert ("k_fused_batch" in names) == (kernel == 1), names
                for it in items:
                    assert np.array_equal(it["out"][0].cpu().numpy(), it["ref"][0])
                    assert np.array_equal(it["out"][1].cpu().numpy(), it["ref"][1])
            # batched results against the oracle directly: the degree-3 (n = 19) job and the
            # bfloat16 one
            from oracle import hgf_oracle as O
            from gpu_helpers import check_against_oracle
            for it in items:
                sp = it["spec"]
                if sp["degree"] == 3 or sp.get("dtype") == "bf16":
                    ref = O.centred_filter(it["case"].guidance,
                                           synth.from_dtype(it["case"].cost, sp.get("dtype", "f32")),
                                           sp["r"], 1e-4, sp["degree"])
                    check_against_oracle(None, it["out"][0].cpu().numpy(),
                                         it["out"][1].cpu().numpy(), ref)
        finally:
            hgf.hgf_batch_destroy(batch)
    finally:
        hgf.hgf_destroy(ctx)
