"""Aggregation straight from a stereo pair (hgf_aggregate_stereo): the coefficient kernel
computes the cost of hgf_cost_volume as it reads it. Checked bit for bit against the two-step
path (hgf_cost_volume into a float32 volume, then hgf_aggregate), and against the oracle
(cost_volume then the centred filter, float64) at the usual tolerance, for the left and the
right view as reference."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import check_against_oracle, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


@pytest.mark.parametrize("direction,degree,r,form", [(1, 2, 9, "centred"), (-1, 1, 4, "centred"),
                                                     (1, 2, 7, "paper")])
def test_stereo_fused_equals_two_step_and_oracle(ctx, direction, degree, r, form):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    W, H, L, eps = 230, 140, 21, (1e-4 if form == "centred" else 0.05)
    left, right, _ = synth.stereo_pair(W, H, L, 23)
    ref, other = (left, right) if direction == 1 else (right, left)
    ref32, oth32 = ref.astype(np.float32), other.astype(np.float32)
    R = torch.from_numpy(ref32).cuda()
    Ot = torch.from_numpy(oth32).cuda()
    g = hgf.hgf_prepare(ctx, R, hgf.make_params(degree=degree, r=r, eps=eps, form=form))
    try:
        q1 = torch.empty((L, H, W), device="cuda")
        l1 = torch.empty((H, W), dtype=torch.int32, device="cuda")
        b1 = torch.empty((H, W), device="cuda")
        hgf.hgf_aggregate_stereo(ctx, g, Ot, L, filtered=q1, labels=l1, best=b1,
                                 direction=direction)
        vol = hgf.hgf_cost_volume(ctx, R, Ot, L, direction=direction)
        q2 = torch.empty_like(q1)
        l2 = torch.empty_like(l1)
        b2 = torch.empty_like(b1)
        hgf.hgf_aggregate(ctx, g, vol, filtered=q2, labels=l2, best=b2)
        torch.cuda.synchronize()
    finally:
        hgf.hgf_guidance_release(g)
    assert torch.equal(q1, q2) and torch.equal(l1, l2) and torch.equal(b1, b2)
    V = O.cost_volume(ref32, oth32, L, direction=direction)
    if form == "centred":
        ref_q = O.centred_filter(ref32, V, r, eps, degree)
    else:
        ref_q = O.paper_filter(ref32.astype(np.float64), V, r, eps, degree, basis="monomial")
    check_against_oracle(q1.cpu().numpy(), l1.cpu().numpy(), b1.cpu().numpy(), ref_q)
