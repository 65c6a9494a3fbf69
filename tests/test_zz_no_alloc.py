"""hgf_aggregate_static: the aggregation entry point for callers that must not allocate device
memory while running (fixed-latency loops, where cudaMalloc can block; plugins in a program whose
allocator owns all device memory from start-up). It takes its scratch from the library's fixed
device array; this test checks, through the C ABI, that two calls in a row give what the
allocating hgf_aggregate gives on the same inputs - on the single-pass kernel (keys only in the
array) and on the two-kernel path with more labels than the array's coefficient planes hold, so
that the call runs several chunks whose WTA keys persist across them - and that an image too
large for the array is refused with a clear error instead of being processed."""
import numpy as np
import pytest

from gpu_helpers import TOL_Q, normwise, torch_cuda

pytestmark = pytest.mark.gpu


def _compare(torch, hgf, ctx, g, cost, L, H, W):
    ref_q = torch.empty((L, H, W), device="cuda")
    ref_l = torch.empty((H, W), dtype=torch.int32, device="cuda")
    ref_b = torch.empty((H, W), device="cuda")
    hgf.hgf_aggregate(ctx, g, cost, filtered=ref_q, labels=ref_l, best=ref_b)
    torch.cuda.synchronize()
    for _ in range(2):
        q = torch.full((L, H, W), float("nan"), device="cuda")
        lab = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
        bst = torch.full((H, W), float("nan"), device="cuda")
        hgf.hgf_aggregate_static(ctx, g, cost, filtered=q, labels=lab, best=bst)
        torch.cuda.synchronize()
        assert normwise(q.cpu().numpy(), ref_q.cpu().numpy()) <= TOL_Q
        assert np.array_equal(lab.cpu().numpy(), ref_l.cpu().numpy())
        np.testing.assert_allclose(bst.cpu().numpy(), ref_b.cpu().numpy(), rtol=0,
                                   atol=TOL_Q * float(ref_q.abs().max()))


def test_static_scratch_matches_allocating_path():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf, synth
    build.build()
    ctx = hgf.hgf_create(0)
    try:
        # single-pass kernel: keys and ring slots in the array
        case = synth.make_case(210, 130, 11, 77, "f32")
        L, H, W = case.cost.shape
        img = torch.from_numpy(case.guidance).cuda()
        cost = torch.from_numpy(case.cost).cuda()
        hgf.hgf_set_tuning(ctx, kernel=1)
        g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=2, r=9, eps=1e-4))
        _compare(torch, hgf, ctx, g, cost, L, H, W)
        hgf.hgf_guidance_release(g)
        hgf.hgf_set_tuning(ctx)

        # two-kernel path: 900 x 700 at n = 9 takes 25.2 MB of coefficient planes per label, so
        # the 64 MiB array holds two labels' planes next to the keys and 7 labels run in 4 chunks
        case = synth.make_case(900, 700, 7, 78, "f32")
        L, H, W = case.cost.shape
        img = torch.from_numpy(case.guidance).cuda()
        cost = torch.from_numpy(case.cost).cuda()
        hgf.hgf_set_tuning(ctx, kernel=2)
        g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=2, r=9, eps=1e-4))
        _compare(torch, hgf, ctx, g, cost, L, H, W)
        hgf.hgf_guidance_release(g)
        hgf.hgf_set_tuning(ctx)

        # more pixels than the array holds keys and planes for: refused
        big = torch.rand((1, 3000, 3000), device="cuda")
        gb = hgf.hgf_prepare(ctx, big, hgf.make_params(degree=1, r=1, eps=1e-4))
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_aggregate_static(ctx, gb, torch.rand((2, 3000, 3000), device="cuda"),
                                     labels=torch.empty((3000, 3000), dtype=torch.int32,
                                                        device="cuda"))
        assert ei.value.status == hgf.HGF_EUNSUPPORTED
        assert "static scratch" in str(ei.value)
        hgf.hgf_guidance_release(gb)
    finally:
        hgf.hgf_destroy(ctx)
