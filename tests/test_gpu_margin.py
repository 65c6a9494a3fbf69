"""WTA margin (second-smallest minus smallest filtered cost per pixel) through the C ABI:
hgf_aggregate_margin (fused path, second key kept by the atomic minimum; plain path for wide
windows) and hgf_wta_margin (over a filtered volume), against the oracle's WTA (Sec. 1) and
against the GPU's own filtered volume."""
import numpy as np
import pytest

from oracle import hgf_oracle as O

from gpu_helpers import TOL_Q, cost_tensor, oracle_case, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


def _margin_from_volume(q):
    """Second-smallest minus smallest of a float32 volume along labels, in float32 (NaN as +inf,
    +inf for a single label)."""
    q = np.where(np.isnan(q), np.float32(np.inf), q).astype(np.float32)
    if q.shape[0] == 1:
        return np.full(q.shape[1:], np.inf, dtype=np.float32)
    s = np.sort(q, axis=0)
    with np.errstate(invalid="ignore"):
        return (s[1] - s[0]).astype(np.float32)


def _run(ctx, guidance, cost, dtype, degree, r, eps):
    """(filtered, labels, best) from hgf_aggregate and (labels, best, margin) from
    hgf_aggregate_margin on the same guidance handle."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    img = torch.from_numpy(np.ascontiguousarray(guidance, dtype=np.float32)).cuda()
    c = cost_tensor(torch, cost, dtype)
    L, H, W = cost.shape
    g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=degree, r=r, eps=eps))
    try:
        filt = torch.empty((L, H, W), dtype=torch.float32, device="cuda")
        lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
        best = torch.empty((H, W), dtype=torch.float32, device="cuda")
        hgf.hgf_aggregate(ctx, g, c, filtered=filt, labels=lab, best=best)
        lab2 = torch.empty_like(lab)
        best2 = torch.empty_like(best)
        marg = torch.empty_like(best)
        hgf.hgf_aggregate_margin(ctx, g, c, marg, labels=lab2, best=best2)
        torch.cuda.synchronize()
    finally:
        hgf.hgf_guidance_release(g)
    return (filt.cpu().numpy(), lab.cpu().numpy(), best.cpu().numpy(), lab2.cpu().numpy(),
            best2.cpu().numpy(), marg.cpu().numpy())


@pytest.mark.parametrize("width,height,L,degree,r", [(300, 170, 11, 2, 9), (64, 48, 16, 1, 4)])
def test_fused_margin(ctx, width, height, L, degree, r):
    """Several strips, bands and label passes with ragged tails: the margin equals the second
    minus the smallest value of the GPU's own filtered volume bit for bit, labels and best equal
    hgf_aggregate's, and the margin is within twice the filtering tolerance of the oracle's."""
    case, ref = oracle_case(width, height, L, 61, degree=degree, r=r, eps=1e-4)
    q, lab, best, lab2, best2, marg = _run(ctx, case.guidance, case.cost, "f32", degree, r, 1e-4)
    np.testing.assert_array_equal(lab2, lab)
    np.testing.assert_array_equal(best2, best)
    np.testing.assert_array_equal(marg, _margin_from_volume(q))
    _, _, om = O.wta(ref)
    scale = float(np.max(np.abs(ref)))
    assert np.all(marg >= 0)
    assert np.max(np.abs(marg.astype(np.float64) - om)) <= 2 * TOL_Q * scale


def test_single_label_margin_is_inf(ctx):
    case, ref = oracle_case(150, 40, 1, 62, degree=2, r=9, eps=1e-4)
    _, lab, _, lab2, _, marg = _run(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
    assert np.all(lab2 == 0) and np.all(lab == 0)
    assert np.all(np.isposinf(marg))
    assert np.all(np.isposinf(O.wta(ref)[2]))


def test_identical_slices_tie(ctx):
    """Three copies of one slice: the filtered values tie exactly, so every label is 0 (lowest on
    ties) and every margin is 0."""
    case, _ = oracle_case(200, 60, 1, 63, degree=2, r=9, eps=1e-4)
    cost = np.ascontiguousarray(np.repeat(case.cost, 3, axis=0))
    _, lab, _, lab2, _, marg = _run(ctx, case.guidance, cost, "f32", 2, 9, 1e-4)
    assert np.all(lab2 == 0) and np.all(lab == 0)
    assert np.all(marg == 0)


def test_wide_window_plain_path(ctx):
    """2r+1 >= 128 takes the plain kernels and the volume WTA: same margin contract."""
    case, ref = oracle_case(140, 30, 4, 64, degree=1, r=64, eps=1e-4)
    q, lab, best, lab2, best2, marg = _run(ctx, case.guidance, case.cost, "f32", 1, 64, 1e-4)
    np.testing.assert_array_equal(lab2, lab)
    np.testing.assert_array_equal(best2, best)
    np.testing.assert_array_equal(marg, _margin_from_volume(q))
    scale = float(np.max(np.abs(ref)))
    assert np.max(np.abs(marg.astype(np.float64) - O.wta(ref)[2])) <= 2 * TOL_Q * scale


@pytest.mark.parametrize("L", [1, 2, 7])
def test_volume_margin_with_nan_inf_and_ties(ctx, L):
    """hgf_wta_margin on a float32 volume with NaN, +inf, -inf and exact ties: labels and best
    equal the oracle's WTA exactly, and the margin equals the oracle's (exact in float64 for two
    float32 values) rounded once to float32; NaN where the two smallest are both +inf."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    rng = np.random.default_rng(65 + L)
    H, W = 37, 53
    q = rng.integers(0, 6, size=(L, H, W)).astype(np.float32) * np.float32(0.25)
    u = rng.random((L, H, W))
    q[u < 0.05] = np.nan
    q[(u >= 0.05) & (u < 0.08)] = np.inf
    q[(u >= 0.08) & (u < 0.09)] = -np.inf
    q[:, 0, 0] = np.nan  # a pixel whose every value is NaN (counted as +inf)
    qt = torch.from_numpy(q).cuda()
    lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
    best = torch.empty((H, W), dtype=torch.float32, device="cuda")
    marg = torch.empty((H, W), dtype=torch.float32, device="cuda")
    hgf.hgf_wta_margin(ctx, qt, marg, labels=lab, best=best)
    torch.cuda.synchronize()
    ol, ob, om = O.wta(q)
    np.testing.assert_array_equal(lab.cpu().numpy(), ol)
    np.testing.assert_array_equal(best.cpu().numpy(), ob.astype(np.float32))
    with np.errstate(invalid="ignore", over="ignore"):
        np.testing.assert_array_equal(marg.cpu().numpy(), om.astype(np.float32))


def test_null_margin_is_rejected(ctx):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    q = torch.zeros((2, 4, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(hgf.HGFError):
        hgf.hgf_wta_margin(ctx, q, None)
