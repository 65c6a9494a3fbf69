"""Stereo cost volume on the GPU (hgf_cost_volume) against the oracle's cost_volume (float64,
pinned by closed forms on CPU), both directions, float32 / bfloat16 / float16 storage, a ragged
label block and a gray (C = 1) pair. The kernel computes in float32: float32 output within 1e-6
absolute (the costs are at most alpha tau_color + (1 - alpha) tau_grad < 0.03); rounded storage
within half an ulp of the stored type (plus the same 1e-6) of the float64 value."""
import numpy as np
import pytest

from oracle import hgf_oracle as O
from paper_1803_00005_gb300 import synth

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    c = hgf.hgf_create(0)
    yield c
    hgf.hgf_destroy(c)


def half_ulp(v, dtype):
    a = np.abs(v).astype(np.float32)
    if dtype == "f16":
        return 0.5 * np.spacing(a.astype(np.float16)).astype(np.float64)
    if dtype == "bf16":
        return 0.5 * np.spacing(a).astype(np.float64) * 2.0 ** 16
    return np.zeros_like(v)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("direction", [1, -1])
def test_cost_volume_parity(ctx, dtype, direction):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    left, right, _ = synth.stereo_pair(261, 77, 37, 13)
    ref, other = (left, right) if direction == 1 else (right, left)
    want = O.cost_volume(ref, other, 37, direction=direction)
    R = torch.from_numpy(ref.astype(np.float32)).cuda()
    Ot = torch.from_numpy(other.astype(np.float32)).cuda()
    out = hgf.hgf_cost_volume(ctx, R, Ot, 37, dtype=dtype, direction=direction)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64)
    # the oracle takes the float32-rounded views the kernel sees
    want = O.cost_volume(ref.astype(np.float32), other.astype(np.float32), 37,
                         direction=direction)
    err = np.abs(got - want)
    assert np.all(err <= half_ulp(want, dtype) * (1 + 1e-3) + 1e-6), float(err.max())


def test_cost_volume_gray_and_params(ctx):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    left, right, _ = synth.stereo_pair(130, 40, 9, 17)
    gl = left.mean(axis=0, keepdims=True).astype(np.float32)
    gr = right.mean(axis=0, keepdims=True).astype(np.float32)
    out = hgf.hgf_cost_volume(ctx, torch.from_numpy(gl).cuda(), torch.from_numpy(gr).cuda(), 9,
                              alpha=0.5, tau_color=0.05, tau_grad=0.02)
    torch.cuda.synchronize()
    want = O.cost_volume(gl, gr, 9, alpha=0.5, tau_color=0.05, tau_grad=0.02)
    assert np.max(np.abs(out.cpu().numpy() - want)) <= 1e-6


def test_cost_volume_argument_errors(ctx):
    torch = torch_cuda()
    from paper_1803_00005_gb300 import hgf
    a = torch.zeros((3, 4, 5), device="cuda")
    for kw in (dict(alpha=1.5), dict(tau_color=-1.0), dict(direction=2)):
        with pytest.raises(hgf.HGFError) as ei:
            hgf.hgf_cost_volume(ctx, a, a, 3, **kw)
        assert ei.value.status == hgf.HGF_EINVAL
