"""Autotuner (hgf_autotune): it times the kernel paths, labels per pass, chunks and row-band
heights; the tuning it keeps is a candidate, stays set on the context, and gives results within
the oracle tolerance that repeat bit for bit; the JSON cache keyed by shape class reuses it."""
import numpy as np
import pytest

from paper_1803_00005_gb300 import synth

from gpu_helpers import check_against_oracle, oracle_case, torch_cuda

pytestmark = pytest.mark.gpu


def test_autotune_candidates_and_results():
    """The autotuner times the kernel paths, the two-kernel family and row-band heights; the tuning
    it keeps is one of those candidates, the tuned aggregation stays within the tolerance of the
    float64 oracle, repeats bit for bit, and the scratch labels it wrote equal the tuned path's."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    case, ref = oracle_case(200, 150, 12, 37, degree=2, r=9, eps=1e-4)
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

        scratch = torch.empty((H, W), dtype=torch.int32, device="cuda")
        tuning, n = hgf.hgf_autotune(ctx, g, cost, scratch, reps=1)
        assert n >= 7  # the two-kernel family, the single pass, band heights
        assert tuning["kernel"] in (1, 2)
        if tuning["kernel"] == 2:
            assert tuning["labels_per_pass"] in (2, 4, 8)
            assert tuning["chunk_labels"] in (0, 16, 64) and tuning["apply_mode"] in (1, 2)
        assert tuning["band_rows"] in (0, (H + 1) // 2, (H + 3) // 4, (H + 7) // 8)
        a, b = run(), run()
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        assert torch.equal(scratch, a[1])
        check_against_oracle(a[0].cpu().numpy(), a[1].cpu().numpy(), a[2].cpu().numpy(), ref)
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
