"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and compare with the
CPU oracle on the same seeded inputs."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

# Tolerances: filtered costs normwise max|q - q*| / max|q*| <= 1e-4 (float32 path, float64
# inverse); labels bit-exact wherever the oracle's winning margin exceeds 1e-3; >= 99.9% overall.
TOL_Q = 1e-4
MARGIN = 1e-3
MIN_AGREEMENT = 0.999


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def cost_tensor(torch, cost, dtype):
    if dtype == "bf16":
        return torch.from_numpy(cost.view(np.int16)).cuda().view(torch.bfloat16)
    return torch.from_numpy(np.ascontiguousarray(cost)).cuda()


def run_path(ctx, guidance, cost, dtype, degree, r, eps, basis="monomial", plain=False,
             inv_precision="f64", combine="alpha", want_filtered=True, form="centred",
             compensated=False, kernel=0):
    """kernel: hgf_tuning.kernel for the call (0 automatic, 1 single pass, 2 two kernels)."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    img = torch.from_numpy(np.ascontiguousarray(guidance, dtype=np.float32)).cuda()
    c = cost_tensor(torch, cost, dtype)
    L, H, W = cost.shape
    params = hgf.make_params(degree=degree, r=r, eps=eps, basis=basis,
                             inv_precision=inv_precision, combine=combine, form=form,
                             compensated=compensated)
    g = hgf.hgf_prepare(ctx, img, params)
    try:
        filt = torch.empty((L, H, W), dtype=torch.float32, device="cuda") if want_filtered else None
        labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
        best = torch.empty((H, W), dtype=torch.float32, device="cuda")
        fn = hgf.hgf_aggregate_plain if plain else hgf.hgf_aggregate
        if kernel:
            hgf.hgf_set_tuning(ctx, kernel=kernel)
        try:
            fn(ctx, g, c, filtered=filt, labels=labels, best=best)
            torch.cuda.synchronize()
        finally:
            if kernel:
                hgf.hgf_set_tuning(ctx)
    finally:
        hgf.hgf_guidance_release(g)
    return (None if filt is None else filt.cpu().numpy()), labels.cpu().numpy(), best.cpu().numpy()


def normwise(q, ref):
    return float(np.max(np.abs(q - ref)) / max(np.max(np.abs(ref)), 1e-30))


def check_against_oracle(q, labels, best, ref, tol=TOL_Q, margin=MARGIN):
    """Filtered volume within tol (normwise); WTA labels exact where the oracle's margin > margin
    and >= 99.9% overall; best equals the filtered minimum."""
    if q is not None:
        err = normwise(q, ref)
        assert np.all(np.isfinite(q)), "non-finite filtered values"
        assert err <= tol, f"normwise error {err:.3e} > {tol:.1e}"
    ol, ob, om = O.wta(ref)
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    sure = om > margin
    mism = (labels != ol) & sure
    assert not mism.any(), f"{mism.sum()} labels differ where the oracle margin > {margin}"
    # every GPU label is a minimum of the oracle's volume within the filtering tolerance
    picked_ref = np.take_along_axis(ref, labels[None].astype(np.int64), axis=0)[0]
    assert np.all(picked_ref - ob <= tol * scale), "a GPU label is not a minimum within tolerance"
    # agreement over pixels whose oracle minimum is unique (exact ties, margin == 0 in float64,
    # have several correct labels: e.g. labels l >= x at the left border see identical slices)
    unique = om > 0
    agree = float(np.mean(labels[unique] == ol[unique])) if unique.any() else 1.0
    assert agree >= MIN_AGREEMENT, f"label agreement {agree:.5f} on {unique.sum()} unique pixels"
    assert np.max(np.abs(best - ob)) <= tol * scale * 1.0001
    # labels must index a minimum of the GPU's own filtered volume where it was returned
    if q is not None:
        H, W = labels.shape
        picked = np.take_along_axis(q, labels[None].astype(np.int64), axis=0)[0]
        assert np.array_equal(picked, np.min(np.where(np.isnan(q), np.inf, q), axis=0))
    return agree


def oracle_case(width, height, L, seed, degree, r, eps, dtype="f32", basis="monomial"):
    case = synth.make_case(width, height, L, seed, dtype)
    ref = O.centred_filter(case.guidance, synth.from_dtype(case.cost, dtype), r, eps, degree, basis)
    return case, ref


def boundary_regions(plan, H, W, half=3, extra=(), limit=None):
    """Rectangles of (2 half)^2 pixels centred on crossings of the band boundary rows of the plan's
    kernels (hgf_last_plan) with its strip boundary columns (at most `limit` crossings, spread
    over the image), plus the four corners, the centre and `extra` centres."""
    rows = sorted({k * b for b in (plan["band_rows"], plan["apply_band_rows"]) if b > 0
                   for k in range(1, (H + b - 1) // b) if 0 < k * b < H})
    cols = sorted({k * plan["out_strip"] for k in range(1, W) if 0 < k * plan["out_strip"] < W}
                  if plan["out_strip"] > 0 else [])
    cross = [(y, x) for y in rows for x in cols]
    if limit is not None and len(cross) > limit:
        cross = [cross[i * len(cross) // limit] for i in range(limit)]
    centres = cross + [(half, half), (half, W - half), (H - half, half), (H - half, W - half),
                       (H // 2, W // 2)] + list(extra)
    regions = []
    for y, x in centres:
        y0, x0 = min(max(0, y - half), H - 2 * half), min(max(0, x - half), W - 2 * half)
        regions.append((y0, y0 + 2 * half, x0, x0 + 2 * half))
    return sorted(set(regions))
