"""Autotuner (hgf_autotune): it times only tunings that leave results bit-identical, so the
filtered volume, labels and best costs after tuning equal those of the automatic plan; the chosen
tuning is one of the candidates and stays set on the context."""
import numpy as np
import pytest

from paper_1803_00005_gb300 import synth

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_autotune_preserves_results():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    case = synth.make_case(300, 170, 70, 37, "f32")
    ctx = hgf.hgf_create(0)
    try:
        img = torch.from_numpy(case.guidance).cuda()
        cost = torch.from_numpy(case.cost).cuda()
        g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=2, r=9, eps=1e-4))
        L, H, W = case.cost.shape

        def run():
            q = torch.empty((L, H, W), device="cuda")
            lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
            best = torch.empty((H, W), device="cuda")
            hgf.hgf_aggregate(ctx, g, cost, filtered=q, labels=lab, best=best)
            torch.cuda.synchronize()
            return q, lab, best

        before = run()
        scratch = torch.empty((H, W), dtype=torch.int32, device="cuda")
        tuning, n = hgf.hgf_autotune(ctx, g, cost, scratch, reps=2)
        assert n >= 6
        assert tuning["labels_per_pass"] in (2, 4, 8) and tuning["band_rows"] == 0
        assert tuning["chunk_labels"] in (0, 16, 64) and tuning["apply_mode"] in (1, 2)
        after = run()
        for x, y in zip(before, after):
            assert torch.equal(x, y)
        assert torch.equal(scratch, before[1])
        hgf.hgf_guidance_release(g)
    finally:
        hgf.hgf_destroy(ctx)


def test_autotune_cache_roundtrip(tmp_path):
    """autotune_cached: the first call times and stores the tuning under its key, the second is a
    hit that sets the same tuning without timing."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    case = synth.make_case(160, 120, 20, 39, "f32")
    ctx = hgf.hgf_create(0)
    try:
        img = torch.from_numpy(case.guidance).cuda()
        cost = torch.from_numpy(case.cost).cuda()
        g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=1, r=4, eps=1e-4))
        lab = torch.empty((120, 160), dtype=torch.int32, device="cuda")
        path = str(tmp_path / "tune.json")
        t1, hit1 = hgf.autotune_cached(ctx, g, cost, lab, path, reps=1)
        t2, hit2 = hgf.autotune_cached(ctx, g, cost, lab, path, reps=1)
        assert (hit1, hit2) == (False, True) and t1 == t2
        hgf.hgf_guidance_release(g)
    finally:
        hgf.hgf_destroy(ctx)
