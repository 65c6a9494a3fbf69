"""The paper's own form on the GPU (Secs. 3-4: G_0 = 1 joins the guidance, the (n+1) x (n+1)
Gram matrix of uncentred window sums and b = B(G p) are solved with lambda = eps in units of
window sums, Z = sum_i A(w_i) G_i + A(w_0)), through the C ABI, against the oracle's
paper_filter (Prop. 1 in float64, pinned against brute-force least squares on CPU).

The fused kernels solve it in shifted coordinates (the record holds T^T (lambda E + Gram)^-1 T
for the image-mean shift T, built in float64), so the float32 part sees the same centred sums as
the centred form, and the same 1e-4 normwise tolerance applies."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import TOL_Q, check_against_oracle, normwise, run_path, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


# (width, height, labels, seed, degree, r, lambda, basis, gray, combine)
CASES = [
    (64, 48, 16, 1, 1, 4, 0.05, "monomial", False, "alpha"),     # n = 3
    (300, 170, 11, 21, 2, 9, 0.05, "monomial", False, "alpha"),  # n = 9: 3 strips, ragged
    (150, 90, 6, 51, 2, 7, 0.05, "powers", False, "alpha"),      # the paper's RGB d = 2, r = 7
    (150, 90, 6, 51, 2, 7, 0.05, "powers", False, "w3"),         # Eq. HGF_w3's combination
    (140, 75, 5, 31, 3, 4, 0.5, "monomial", False, "alpha"),     # n = 19 (pixel-major records)
    (120, 100, 7, 61, 5, 3, 0.01, "powers", True, "alpha"),      # gray I..I^5 (n = 5)
    (97, 61, 4, 71, 2, 9, 5.0, "monomial", False, "alpha"),      # large lambda: heavy shrinkage
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_d{c[4]}_{c[7]}_r{c[5]}_"
                                                       f"lam{c[6]}_{c[9]}{'_gray' if c[8] else ''}")
def test_paper_form_parity(ctx, case, capsys):
    w, h, L, seed, degree, r, lam, basis, gray, combine = case
    sc = synth.make_case(w, h, L, seed, "f32")
    guid = sc.guidance.mean(axis=0, keepdims=True).astype(np.float32) if gray else sc.guidance
    ref = O.paper_filter(guid.astype(np.float64), sc.cost.astype(np.float64), r, lam, degree,
                         basis=basis, solver="hgf")
    q, labels, best = run_path(ctx, guid, sc.cost, "f32", degree, r, lam, basis=basis,
                               combine=combine, form="paper")
    with capsys.disabled():
        print(f"\npaper form {w}x{h} L={L} d={degree} {basis} r={r} lambda={lam} {combine}: "
              f"normwise error {normwise(q, ref):.2e}")
    check_against_oracle(q, labels, best, ref, tol=TOL_Q)


def test_paper_form_differs_from_centred(ctx):
    """The two forms are different filters: same inputs, visibly different outputs."""
    sc = synth.make_case(96, 64, 4, 5, "f32")
    qa, _, _ = run_path(ctx, sc.guidance, sc.cost, "f32", 1, 4, 0.05, form="centred")
    qb, _, _ = run_path(ctx, sc.guidance, sc.cost, "f32", 1, 4, 0.05, form="paper")
    assert normwise(qa, qb) > 1e-2


def test_paper_form_unsupported_routes(ctx):
    """Routes that compute the centred form only refuse the paper form."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    sc = synth.make_case(64, 48, 3, 9, "f32")
    img = torch.from_numpy(sc.guidance).cuda()
    cost = torch.from_numpy(sc.cost).cuda()
    lab = torch.empty((48, 64), dtype=torch.int32, device="cuda")
    g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=1, r=4, eps=0.05, form="paper"))
    try:
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_aggregate_plain(ctx, g, cost, labels=lab)
        assert ei.value.status == hgf.HGF_EUNSUPPORTED
        minv = torch.empty((6, 48, 64), device="cuda")
        mu = torch.empty((3, 48, 64), device="cuda")
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_guidance_export(ctx, g, minv, mu)
        assert ei.value.status == hgf.HGF_EUNSUPPORTED
    finally:
        hgf.hgf_guidance_release(g)
    # windows wider than the strip kernels (2r+1 >= 128): the plain route is centred only
    wide = synth.make_case(200, 48, 3, 9, "f32")
    img = torch.from_numpy(wide.guidance).cuda()
    cost = torch.from_numpy(wide.cost).cuda()
    lab = torch.empty((48, 200), dtype=torch.int32, device="cuda")
    g = hgf.hgf_prepare(ctx, img, hgf.make_params(degree=1, r=70, eps=0.05, form="paper"))
    try:
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_aggregate(ctx, g, cost, labels=lab)
        assert ei.value.status == hgf.HGF_EUNSUPPORTED
    finally:
        hgf.hgf_guidance_release(g)
    assert hgf.hgf_device_status(ctx) == 0
