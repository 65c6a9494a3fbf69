"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Sizes are chosen so that the oracle finishes in seconds while the strip kernels still see several
strips, several row bands, several label passes and ragged tails; the full 450x375 / 60-label /
n=9 workload is checked on sampled pixels (oracle on exact crops)."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import (boundary_regions, check_against_oracle, normwise, oracle_case, run_path,
                         torch_cuda, cost_tensor)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


PATHS = {"single-pass": dict(kernel=1), "two-kernel": dict(kernel=2), "plain": dict(plain=True)}


@pytest.mark.parametrize("path", list(PATHS))
def test_small_stereo_n3(ctx, path):
    """64x48, L=16, degree 1 (n=3), r=4, eps=1e-4 (the small stereo configuration), in full."""
    case, ref = oracle_case(64, 48, 16, 1, degree=1, r=4, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 1, 4, 1e-4, **PATHS[path])
    check_against_oracle(q, labels, best, ref)


@pytest.mark.parametrize("path", list(PATHS))
def test_n9_several_strips_ragged(ctx, path):
    """n=9, r=9 on 300x170 with 11 labels: several strips (the last ragged: 4 strips of 92
    output columns for the single-pass kernel, 3 of 110 for the two-kernel path), several bands,
    label passes 2+2+..+1 on the two-kernel path."""
    case, ref = oracle_case(300, 170, 11, 21, degree=2, r=9, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4, **PATHS[path])
    check_against_oracle(q, labels, best, ref)


def test_n19_degree3(ctx):
    """Degree-3 monomials (n=19), 2 labels per pass."""
    case, ref = oracle_case(140, 75, 5, 31, degree=3, r=4, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 3, 4, 1e-4)
    check_against_oracle(q, labels, best, ref)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_low_precision_costs(ctx, dtype):
    """BF16/FP16 cost storage, float32 accumulation: parity against the oracle fed the same
    rounded costs."""
    case, ref = oracle_case(200, 130, 9, 41, degree=2, r=9, eps=1e-4, dtype=dtype)
    q, labels, best = run_path(ctx, case.guidance, case.cost, dtype, 2, 9, 1e-4)
    check_against_oracle(q, labels, best, ref)


def test_combine_w3_matches(ctx):
    """Eq. HGF_w3's combination lambda^-1 E + S alpha gives the same filter (float64)."""
    case, ref = oracle_case(150, 90, 6, 51, degree=2, r=9, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4, combine="w3")
    check_against_oracle(q, labels, best, ref)


def test_float32_inverse_variant_error_is_reported(ctx):
    """The float32 assembly + recursion variant: its error against the float64 oracle is larger
    (the recursion loses digits for eps << |Sigma|); it is measured, not held to 1e-4."""
    case, ref = oracle_case(150, 90, 6, 51, degree=2, r=9, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4,
                               inv_precision="f32")
    err = normwise(q, ref)
    assert np.all(np.isfinite(q))
    assert err < 5e-2, err


def test_gray_powers_basis(ctx):
    """Gray guidance with the paper's power basis I, I^2, .., I^5 (C=1, n=5)."""
    case = synth.make_case(120, 80, 4, 61)
    gray = case.guidance.mean(axis=0, keepdims=True).astype(np.float32)
    ref = O.centred_filter(gray, case.cost.astype(np.float64), 7, 1e-3, 5, "powers")
    q, labels, best = run_path(ctx, gray, case.cost, "f32", 5, 7, 1e-3, basis="powers")
    check_against_oracle(q, labels, best, ref)


def test_powers_basis_rgb(ctx):
    """The paper's colour power basis G_{(i-1)d+j} = I_i^j with d=2 (n=6), lambda-scale eps."""
    case = synth.make_case(96, 64, 5, 62)
    ref = O.centred_filter(case.guidance, case.cost.astype(np.float64), 7, 2.2e-4, 2, "powers")
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", 2, 7, 2.2e-4,
                               basis="powers")
    check_against_oracle(q, labels, best, ref)


@pytest.mark.parametrize("W,H,L,r,degree", [(1, 1, 1, 4, 1), (1, 9, 3, 2, 2), (13, 1, 2, 3, 2),
                                            (7, 5, 2, 9, 2), (40, 30, 3, 0, 2), (5, 6, 1, 200, 1),
                                            (129, 3, 4, 1, 1), (110, 7, 5, 9, 1)])
def test_edge_shapes(ctx, W, H, L, r, degree):
    """Degenerate and ragged shapes: single pixel, single row/column, windows larger than the
    image (r >= size, clamped exactly), r = 0, a single label, strip-width boundaries."""
    g = np.random.Generator(np.random.PCG64(W * 1000 + H * 10 + r))
    guid = g.uniform(size=(3, H, W)).astype(np.float32)
    cost = (g.uniform(size=(L, H, W)) * 0.03).astype(np.float32)
    ref = O.centred_filter(guid, cost.astype(np.float64), r, 1e-3, degree)
    for path in PATHS.values():
        q, labels, best = run_path(ctx, guid, cost, "f32", degree, r, 1e-3, **path)
        check_against_oracle(q, labels, best, ref)


def test_constant_guidance_double_mean(ctx):
    """Constant guidance: q = A(A(p)) (the special case that reduces to the mean filter)."""
    H, W, L, r = 33, 47, 3, 5
    guid = np.full((3, H, W), 0.37, dtype=np.float32)
    cost = (np.random.Generator(np.random.PCG64(7)).uniform(size=(L, H, W)) * 0.03).astype(np.float32)
    N = O.window_count(H, W, r)
    ref = np.stack([O.box_sum(O.box_sum(c.astype(np.float64), r) / N, r) / N for c in cost])
    q, labels, best = run_path(ctx, guid, cost, "f32", 2, r, 1e-4)
    assert normwise(q, ref) <= 1e-5


def test_prepare_export_matches_oracle_inverse(ctx):
    """The resident inverse and means (Prop. 1 in float64) against the oracle's Cholesky-free
    closed form (lambda E + Sigma)^-1 via LAPACK, per pixel."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    case = synth.make_case(60, 40, 2, 71)
    degree, r, eps = 2, 4, 1e-4
    G, N, mu, M = O.guidance_moments(case.guidance, r, eps, degree)
    n = G.shape[0]
    img = torch.from_numpy(case.guidance).cuda()
    g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=degree, r=r, eps=eps))
    minv = torch.empty((n * (n + 1) // 2, 40, 60), device="cuda")
    mu_d = torch.empty((n, 40, 60), device="cuda")
    hgf.hgf_guidance_export(ctx, g, minv, mu_d)
    torch.cuda.synchronize()
    hgf.hgf_guidance_release(g)
    minv = minv.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(mu_d.cpu().numpy(), mu, rtol=0, atol=2e-6)
    Minv_ref = np.linalg.inv(np.moveaxis(M, (0, 1), (2, 3)))  # (H, W, n, n)
    iu = np.triu_indices(n)
    ref_packed = np.moveaxis(Minv_ref[:, :, iu[0], iu[1]], 2, 0)
    scale = np.max(np.abs(ref_packed), axis=0)
    rel = np.max(np.abs(minv - ref_packed) / scale)
    assert rel < 2e-3, rel  # float32 moments feed an inverse with condition number up to ~1e4


def test_standalone_wta_ties_and_nan(ctx):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    g = np.random.Generator(np.random.PCG64(3))
    Q = g.integers(0, 4, size=(7, 20, 30)).astype(np.float32)   # many ties
    Q[2, 0, :5] = np.nan
    Q[:, 1, 0] = np.nan
    t = torch.from_numpy(Q).cuda()
    labels = torch.empty((20, 30), dtype=torch.int32, device="cuda")
    best = torch.empty((20, 30), dtype=torch.float32, device="cuda")
    hgf.hgf_wta(ctx, t, labels, best)
    torch.cuda.synchronize()
    ol, ob, _ = O.wta(Q.astype(np.float64))
    np.testing.assert_array_equal(labels.cpu().numpy(), ol)
    np.testing.assert_array_equal(best.cpu().numpy(), ob.astype(np.float32))


def test_deterministic_repeat(ctx):
    """Two runs give bit-identical filtered volumes and labels."""
    case = synth.make_case(200, 120, 8, 81)
    a = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
    b = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_filter_host_end_to_end(ctx):
    """hgf_filter_host (host buffers in, host labels out) equals the device path."""
    from paper_1803_00005_gb300 import hgf
    case, ref = oracle_case(120, 90, 10, 91, degree=2, r=9, eps=1e-4)
    labels = np.empty((90, 120), dtype=np.int32)
    best = np.empty((90, 120), dtype=np.float32)
    params = hgf.make_params(degree=2, r=9, eps=1e-4)
    hgf.hgf_filter_host(ctx, case.guidance, case.cost, "f32", params, labels, best)
    check_against_oracle(None, labels, best, ref)
    _, l2, b2 = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
    assert np.array_equal(labels, l2) and np.array_equal(best, b2)


@pytest.mark.parametrize("path", ["two-kernel", "single-pass"])
def test_quarter_size_n9_regions(ctx, path):
    """The 450x375 / 60-label / n=9 / r=9 workload in full on the GPU, in the launch configuration
    the benchmark times (the automatic plan of each path), checked against the oracle on every
    pixel of rectangles around each crossing of a band boundary with a strip boundary that the
    plan produced, the corners and random interior points (the oracle runs on the exact crop each
    rectangle depends on); labels exact where the oracle's margin exceeds 1e-3. At full size: all
    values finite, labels index the minimum of the returned volume."""
    from paper_1803_00005_gb300 import hgf
    c = synth.CONFIG_QUARTER
    case = synth.make_case(c["width"], c["height"], c["n_labels"], c["seed"], "f32")
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", c["degree"], c["r"], c["eps"],
                               kernel=1 if path == "single-pass" else 2)
    plan = hgf.hgf_last_plan(ctx)
    assert plan["path"] == (1 if path == "single-pass" else 2)
    H, W = c["height"], c["width"]
    g = np.random.Generator(np.random.PCG64(123))
    extra = [(int(y), int(x)) for y, x in zip(g.integers(10, H - 10, 6), g.integers(10, W - 10, 6))]
    regions = boundary_regions(plan, H, W, extra=extra)
    assert len(regions) > 8, plan
    scale = max(float(np.max(np.abs(q))), 1e-30)
    npx = 0
    for y0, y1, x0, x1 in regions:
        ref = O.filter_region(case.guidance, case.cost, c["r"], c["eps"], c["degree"],
                              y0, y1, x0, x1)
        got = q[:, y0:y1, x0:x1]
        assert np.max(np.abs(got - ref)) / scale <= 1e-4, (y0, x0)
        ol, ob, om = O.wta(ref)
        gl = labels[y0:y1, x0:x1]
        sure = om > 1e-3
        assert np.array_equal(gl[sure], ol[sure]), (y0, x0)
        picked = np.take_along_axis(ref, gl[None].astype(np.int64), axis=0)[0]
        assert np.all(picked - ob <= 1e-4 * scale)
        npx += (y1 - y0) * (x1 - x0)
    assert npx >= 256, npx
    assert np.all(np.isfinite(q))
    picked = np.take_along_axis(q, labels[None].astype(np.int64), axis=0)[0]
    assert np.array_equal(picked, q.min(axis=0))
    assert np.array_equal(best, q.min(axis=0))


def test_invalid_arguments_rejected(ctx):
    """Host-side argument checks: nothing is launched for invalid calls."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    img = torch.rand((3, 8, 8), device="cuda")
    for kw in (dict(eps=0.0), dict(r=-1), dict(degree=0), dict(degree=4)):
        p = dict(degree=1, r=2, eps=1e-4)
        p.update(kw)
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_prepare(ctx, img, hgf.make_params(**p))
        assert ei.value.status in (hgf.HGF_EINVAL, hgf.HGF_EUNSUPPORTED)
    g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=1, r=2, eps=1e-4))
    with pytest.raises(hgf.HGFError):
        hgf.hgf_aggregate(ctx, g, torch.rand((2, 8, 8), device="cuda"))  # no output requested
    hgf.hgf_guidance_release(g)


def test_results_independent_of_label_chunking(ctx):
    """On the two-kernel path, label chunking (workspace size) and labels per pass do not change
    any result bit: the band boundaries of the running sums depend on the image shape only.
    (Explicit band_rows or apply_mode tuning does change the rounding, within the tolerance.)"""
    from paper_1803_00005_gb300 import hgf
    case = synth.make_case(330, 210, 23, 111)
    hgf.hgf_set_tuning(ctx, kernel=2)
    base = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
    try:
        for chunk, K in ((5, 2), (1, 2), (8, 4), (23, 4)):
            hgf.hgf_set_tuning(ctx, labels_per_pass=K, chunk_labels=chunk, kernel=2)
            got = run_path(ctx, case.guidance, case.cost, "f32", 2, 9, 1e-4)
            assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
    finally:
        hgf.hgf_set_tuning(ctx)


def test_n19_labels_per_pass_bit_identical(ctx):
    """n = 19 with one label per pass of the coefficient kernel (three CTAs per SM instead of
    two) gives the same bits as two labels per pass, and matches the oracle."""
    from paper_1803_00005_gb300 import hgf
    case, ref = oracle_case(150, 80, 5, 33, degree=3, r=4, eps=1e-4)
    hgf.hgf_set_tuning(ctx, labels_per_pass=2, kernel=2)
    try:
        a = run_path(ctx, case.guidance, case.cost, "f32", 3, 4, 1e-4)
        hgf.hgf_set_tuning(ctx, labels_per_pass=1, kernel=2)
        b = run_path(ctx, case.guidance, case.cost, "f32", 3, 4, 1e-4)
        assert hgf.hgf_last_plan(ctx)["labels_per_pass"] == 1
    finally:
        hgf.hgf_set_tuning(ctx)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    check_against_oracle(*b, ref)


@pytest.mark.parametrize("degree,r", [(2, 9), (1, 4), (3, 4)])
def test_compensated_running_sums(ctx, degree, r, capsys):
    """Kahan-compensated running sums (hgf_params.compensated): the same tolerance holds, and the
    RMS error against the float64 oracle stays that of the uncompensated path (within 20%): the
    vertical running sums are not the dominant rounding source (the prefix-scan differences and
    the float32 mat-vec are), so compensation moves the maximum error up or down by rounding
    chance and leaves the RMS error where it was. Both are printed."""
    case, ref = oracle_case(300, 170, 7, 61, degree=degree, r=r, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", degree, r, 1e-4,
                               compensated=True)
    check_against_oracle(q, labels, best, ref)
    q0, _, _ = run_path(ctx, case.guidance, case.cost, "f32", degree, r, 1e-4)
    scale = float(np.max(np.abs(ref)))
    rms = [float(np.sqrt(np.mean((x - ref) ** 2))) / scale for x in (q0, q)]
    with capsys.disabled():
        print(f"\ndegree {degree} r {r}: max {normwise(q0, ref):.2e} -> {normwise(q, ref):.2e}, "
              f"rms {rms[0]:.2e} -> {rms[1]:.2e} (plain -> compensated)")
    assert rms[1] <= 1.2 * rms[0]


@pytest.mark.parametrize("degree,r", [(2, 9), (3, 4), (1, 4)])
def test_double_float_inverse(ctx, degree, r, capsys):
    """The covariance assembly + Prop. 1 recursion in double-float (inv_precision = HGF_DF64,
    pairs of float32, about 48 bits): the same tolerance as native float64, and an error within
    10% (plus 1e-7) of the float64 path's, since both round the inverse to float32 records."""
    case, ref = oracle_case(300, 170, 7, 61, degree=degree, r=r, eps=1e-4)
    q, labels, best = run_path(ctx, case.guidance, case.cost, "f32", degree, r, 1e-4,
                               inv_precision="df64")
    check_against_oracle(q, labels, best, ref)
    q0, _, _ = run_path(ctx, case.guidance, case.cost, "f32", degree, r, 1e-4)
    with capsys.disabled():
        print(f"\ndegree {degree} r {r}: float64 {normwise(q0, ref):.2e}, "
              f"double-float {normwise(q, ref):.2e}")
    assert normwise(q, ref) <= 1.1 * normwise(q0, ref) + 1e-7
