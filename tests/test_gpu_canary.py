"""Output buffers with canary padding: every entry point that writes caller-owned device memory
(aggregate, aggregate_stereo, cost_volume, refine_lr, batched_inverse, export) writes inside its
output and nowhere around it, on ragged shapes (widths that are not multiples of the strip width
or of 4). The canaries are checked after each call."""
import numpy as np
import pytest

from paper_1803_00005_gb300 import synth

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

PAD = 4099


def padded(torch, shape, dtype, fill):
    n = int(np.prod(shape))
    buf = torch.full((PAD + n + PAD,), fill, dtype=dtype, device="cuda")
    return buf, buf[PAD:PAD + n].view(*shape)


def intact(torch, buf, n, fill):
    torch.cuda.synchronize()
    return bool(torch.all(buf[:PAD] == fill)) and bool(torch.all(buf[PAD + n:] == fill))


def test_canaries_around_outputs():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    W, H, L = 227, 61, 9
    left, right, _ = synth.stereo_pair(W, H, L, 41)
    lt = torch.from_numpy(left.astype(np.float32)).cuda()
    rt = torch.from_numpy(right.astype(np.float32)).cuda()
    ctx = hgf.hgf_create(0)
    try:
        vb, vol = padded(torch, (L, H, W), torch.float32, -7.0)
        hgf.hgf_cost_volume(ctx, lt, rt, L, out=vol)
        assert intact(torch, vb, L * H * W, -7.0)
        for form in ("centred", "paper"):
            g = hgf.hgf_prepare(ctx, lt, hgf.make_params(degree=2, r=9, eps=1e-3, form=form))
            qb, q = padded(torch, (L, H, W), torch.float32, -7.0)
            lb, lab = padded(torch, (H, W), torch.int32, -7)
            bb, best = padded(torch, (H, W), torch.float32, -7.0)
            hgf.hgf_aggregate(ctx, g, vol, filtered=q, labels=lab, best=best)
            assert intact(torch, qb, L * H * W, -7.0)
            assert intact(torch, lb, H * W, -7) and intact(torch, bb, H * W, -7.0)
            hgf.hgf_aggregate_stereo(ctx, g, rt, L, filtered=q, labels=lab, best=best)
            assert intact(torch, qb, L * H * W, -7.0)
            assert intact(torch, lb, H * W, -7) and intact(torch, bb, H * W, -7.0)
            if form == "centred":
                n = 9
                mb, minv = padded(torch, (n * (n + 1) // 2, H, W), torch.float32, -7.0)
                ub, mu = padded(torch, (n, H, W), torch.float32, -7.0)
                hgf.hgf_guidance_export(ctx, g, minv, mu)
                assert intact(torch, mb, minv.numel(), -7.0) and intact(torch, ub, mu.numel(), -7.0)
            hgf.hgf_guidance_release(g)
        dl = torch.randint(0, L, (H, W), dtype=torch.int32, device="cuda")
        dr = torch.randint(0, L, (H, W), dtype=torch.int32, device="cuda")
        ob, out = padded(torch, (H, W), torch.int32, -7)
        kb, keep = padded(torch, (H, W), torch.uint8, 77)
        hgf.hgf_refine_lr(ctx, dl, dr, 1, out=out, keep=keep)
        assert intact(torch, ob, H * W, -7) and intact(torch, kb, H * W, 77)
        S = torch.from_numpy(synth.pack_upper(synth.gram_batch(301, 9))).cuda()
        sb, so = padded(torch, tuple(S.shape), torch.float64, -7.0)
        hgf.hgf_batched_inverse(ctx, S, 9, 0.5, out=so)
        assert intact(torch, sb, S.numel(), -7.0)
        assert hgf.hgf_device_status(ctx) == 0
    finally:
        hgf.hgf_destroy(ctx)
