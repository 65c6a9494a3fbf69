"""hgf_filter: one frame (guidance update, aggregation, WTA) in one call, against the oracle and
bit for bit against hgf_guidance_update followed by hgf_aggregate, including the guidance it
leaves behind, on both kernel paths and over repeated frames on one handle."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import check_against_oracle, cost_tensor, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


def _outputs(torch, L, H, W):
    return (torch.empty((L, H, W), dtype=torch.float32, device="cuda"),
            torch.empty((H, W), dtype=torch.int32, device="cuda"),
            torch.empty((H, W), dtype=torch.float32, device="cuda"))


def _export(hgf, torch, ctx, g, n, H, W):
    minv = torch.empty((n * (n + 1) // 2, H, W), dtype=torch.float32, device="cuda")
    mu = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
    hgf.hgf_guidance_export(ctx, g, minv, mu)
    return minv, mu


def filter_vs_two_calls(ctx, guid, cost, dtype, degree, r, eps, basis="monomial", tuning=None,
                        frames=1):
    """hgf_filter on a handle first prepared from another image (the mirrored one) against
    hgf_prepare + hgf_aggregate on a second handle, under the same tuning: identical outputs,
    identical exported inverse and means. Returns hgf_filter's outputs (numpy) and its plan."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    tuning = tuning or {}
    img = torch.from_numpy(np.ascontiguousarray(guid, dtype=np.float32)).cuda()
    other = torch.flip(img, dims=[2]).contiguous()
    c = cost_tensor(torch, cost, dtype)
    L, H, W = cost.shape
    params = hgf.make_params(degree=degree, r=r, eps=eps, basis=basis)
    g_ref = hgf.hgf_prepare(ctx, img, params)
    g = hgf.hgf_prepare(ctx, other, params)
    n = hgf.hgf_guidance_info(g)["n"]
    try:
        hgf.hgf_set_tuning(ctx, **tuning)
        q1, l1, b1 = _outputs(torch, L, H, W)
        hgf.hgf_aggregate(ctx, g_ref, c, filtered=q1, labels=l1, best=b1)
        for _ in range(frames):
            q2, l2, b2 = _outputs(torch, L, H, W)
            hgf.hgf_filter(ctx, g, img, c, filtered=q2, labels=l2, best=b2)
        torch.cuda.synchronize()
        plan = hgf.hgf_last_plan(ctx)
        assert torch.equal(q1, q2), float((q1 - q2).abs().max())
        assert torch.equal(l1, l2) and torch.equal(b1, b2)
        m1, u1 = _export(hgf, torch, ctx, g_ref, n, H, W)
        m2, u2 = _export(hgf, torch, ctx, g, n, H, W)
        assert torch.equal(m1, m2) and torch.equal(u1, u2)
    finally:
        hgf.hgf_set_tuning(ctx)
        hgf.hgf_guidance_release(g)
        hgf.hgf_guidance_release(g_ref)
    return q2.cpu().numpy(), l2.cpu().numpy(), b2.cpu().numpy(), plan


# W, H, L, seed, degree, r, cost dtype, tuning
CASES = [
    (300, 170, 12, 71, 2, 9, "f32", dict(kernel=1)),           # n=9: 5 strips, 3 bands
    (300, 170, 12, 71, 2, 9, "f32", dict(kernel=2)),           # the two-kernel path
    (300, 170, 7, 72, 1, 4, "bf16", dict(kernel=1)),           # n=3, bfloat16 costs
    (131, 97, 5, 73, 2, 2, "f16", dict(kernel=1, band_rows=9)),  # ragged, 11 short bands
]


@pytest.mark.parametrize("W,H,L,seed,degree,r,dtype,tuning", CASES)
def test_filter_matches_two_calls_and_oracle(ctx, W, H, L, seed, degree, r, dtype, tuning):
    case = synth.make_case(W, H, L, seed, dtype)
    q, labels, best, plan = filter_vs_two_calls(ctx, case.guidance, case.cost, dtype, degree, r,
                                                1e-4, tuning=tuning)
    assert plan["path"] == tuning["kernel"]
    ref = O.centred_filter(case.guidance, synth.from_dtype(case.cost, dtype), r, 1e-4, degree)
    check_against_oracle(q, labels, best, ref)


def test_filter_gray_powers_repeated_frames(ctx):
    """Gray guidance with the power basis (n=5), three frames in a row on one handle."""
    case = synth.make_case(150, 110, 6, 76)
    gray = case.guidance.mean(axis=0, keepdims=True).astype(np.float32)
    q, labels, best, _ = filter_vs_two_calls(ctx, gray, case.cost, "f32", 5, 7, 1e-3,
                                             basis="powers", frames=3)
    ref = O.centred_filter(gray, case.cost.astype(np.float64), 7, 1e-3, 5, "powers")
    check_against_oracle(q, labels, best, ref)


def test_filter_quarter_size_default_plan(ctx):
    """The 450x375 / 60-label / n=9 / r=9 workload under the automatic plan, two frames."""
    c = synth.CONFIG_QUARTER
    case = synth.make_case(c["width"], c["height"], c["n_labels"], c["seed"], "f32")
    _, labels, _, plan = filter_vs_two_calls(ctx, case.guidance, case.cost, "f32", c["degree"],
                                             c["r"], c["eps"], frames=2)
    assert plan["path"] == 1
    assert labels.min() >= 0 and labels.max() < c["n_labels"]
