"""Precision variants on the 1400x1100 / 256-label / n=9 / r=9 workload: cost storage float32,
bfloat16, float16 (float32 accumulation), the covariance assembly + inverse in float64 vs
float32, and Kahan-compensated running sums. Each variant's error is measured against the float64
oracle on every pixel of rectangles around the plan's band and strip boundaries (the oracle runs
on the exact crop each rectangle depends on), both against the oracle fed the same rounded costs
(the kernels' own error) and against the oracle fed the float32 costs (adding the storage
rounding). The table is printed and the bounds below are asserted."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import boundary_regions, cost_tensor, torch_cuda

pytestmark = pytest.mark.gpu

W, H, L, R, EPS, DEG = 1400, 1100, 256, 9, 1e-4, 2


@pytest.fixture(scope="module")
def workload():
    left, right, _ = synth.stereo_pair(W, H, L, 3)
    v32 = synth.cost_volume(left, right, L, "f32")
    return left.astype(np.float32), left, right, v32


def test_precision_variants(workload, capsys):
    """Every variant on the full image in the benchmark's launch configuration, checked on all
    pixels of 8x8 rectangles around band x strip boundary crossings of the plan, the corners and
    the centre. Asserted per variant: the normwise error against the oracle on the same rounded
    costs (<= 1e-4 with a float64 or double-float inverse), and labels equal to that oracle's
    wherever its winning margin exceeds 1e-3 (a mismatch prints its margin; the float32 inverse,
    a reported variant, is not held to either); label agreement with the float32-cost oracle is
    reported."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    guid, left, right, v32 = workload
    rows = []
    mismatches = []
    ctx = hgf.hgf_create(0)
    try:
        img = torch.from_numpy(guid).cuda()
        regions = None
        refs32 = None
        for dtype in ("f32", "bf16", "f16"):
            stored = synth.cost_volume(left, right, L, dtype) if dtype != "f32" else v32
            exact = synth.from_dtype(stored, dtype)
            cost = cost_tensor(torch, stored, dtype)
            refs_same = None
            for prec, comp in (("f64", False), ("df64", False), ("f32", False), ("f64", True)):
                g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=DEG, r=R, eps=EPS,
                                                              inv_precision=prec,
                                                              compensated=comp))
                q = torch.empty((L, H, W), device="cuda")
                lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
                hgf.hgf_aggregate(ctx, g, cost, filtered=q, labels=lab)
                torch.cuda.synchronize()
                hgf.hgf_guidance_release(g)
                if regions is None:
                    plan = hgf.hgf_last_plan(ctx)
                    regions = boundary_regions(plan, H, W, half=4, limit=8)
                    refs32 = [O.filter_region(guid, v32, R, EPS, DEG, *rg) for rg in regions]
                if refs_same is None:
                    refs_same = refs32 if dtype == "f32" else [
                        O.filter_region(guid, exact, R, EPS, DEG, *rg) for rg in regions]
                e_same = e_store = 0.0
                agree = []
                s_same = max(float(np.max(np.abs(rf))) for rf in refs_same)
                s32 = max(float(np.max(np.abs(rf))) for rf in refs32)
                name = prec + ("+kahan" if comp else "")
                for (y0, y1, x0, x1), rs, r32 in zip(regions, refs_same, refs32):
                    got = q[:, y0:y1, x0:x1].cpu().numpy()
                    gl = lab[y0:y1, x0:x1].cpu().numpy()
                    e_same = max(e_same, float(np.max(np.abs(got - rs))) / s_same)
                    e_store = max(e_store, float(np.max(np.abs(got - r32))) / s32)
                    ol, _, om = O.wta(rs)
                    bad = (gl != ol) & (om > 1e-3)
                    for yy, xx in zip(*np.nonzero(bad)):
                        mismatches.append((dtype, name, y0 + yy, x0 + xx, float(om[yy, xx])))
                    ol32, _, _ = O.wta(r32)
                    agree.append(gl == ol32)
                rows.append((dtype, name, e_same, e_store,
                             float(np.mean(np.concatenate([a.ravel() for a in agree])))))
                del q
    finally:
        hgf.hgf_destroy(ctx)
    npx = sum((y1 - y0) * (x1 - x0) for y0, y1, x0, x1 in regions)
    with capsys.disabled():
        print(f"\n{len(regions)} rectangles, {npx} pixels")
        print("cost   inverse+sums  err vs oracle(same costs)  err vs oracle(f32 costs)  "
              "label agreement (vs f32 oracle)")
        for d, p, a, b, c in rows:
            print(f"{d:6s} {p:12s} {a:24.2e}  {b:24.2e}  {c:8.4f}")
        for m in mismatches:
            print("label mismatch where the oracle margin > 1e-3:", m)
    assert npx >= 256
    # the float32 inverse is a reported variant (not held to the tolerance): its mismatches are
    # printed above; every other variant's labels are exact where the margin exceeds 1e-3
    held = [m for m in mismatches if not m[1].startswith("f32")]
    assert not held, held
    for d, p, a, b, c in rows:
        if p.startswith("f64") or p.startswith("df64"):
            assert a <= 1e-4, (d, p, a)       # the kernels' own error meets the tolerance
        else:
            assert a <= 5e-2, (d, p, a)       # float32 inverse: reported, larger
        if d == "f32":
            assert b == a
