"""Seeded synthetic stereo / multi-label inputs shaped like the paper's workloads.

The paper evaluates on Middlebury stereo pairs (Sec. 6, Fig. 6), which are not available here.
This module stands in for them: a left view made of star-shaped polygons of constant colour at
integer disparities over a background, Gaussian texture, a right view made by backward-warping the
left view with the rendered right-view disparity, and a truncated colour + gradient matching cost
V(x, y, l) (the "cost volume" of Sec. 1), label-major.

It is input generation only: it contains none of the filter's arithmetic (no box filtering, no
moments, no inverse). Both the CUDA path and the CPU oracle consume the arrays it returns.
Everything is generated in float64 from ``numpy.random.PCG64(seed)`` and rounded to the storage
dtype at the end (round to nearest even).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "StereoCase", "stereo_pair", "cost_volume", "cost_volume_torch", "make_case", "to_dtype",
    "CONFIG_SMALL",
    "CONFIG_QUARTER", "CONFIG_LARGE", "batched_cases", "serving_requests", "gram_batch",
    "gram_batch_torch", "pack_upper",
]


@dataclasses.dataclass
class StereoCase:
    guidance: np.ndarray      # float32 (3, H, W), left view RGB in [0, 1]
    cost: np.ndarray          # (L, H, W) in the requested storage dtype (float32/float16/bf16-as-uint16)
    cost_dtype: str           # "f32", "f16" or "bf16"
    disparity: np.ndarray     # int32 (H, W) left-view ground-truth disparity (for reporting only)
    seed: int

    @property
    def shape(self):
        return self.cost.shape


def _inside_polygon(px: np.ndarray, py: np.ndarray, vx: np.ndarray, vy: np.ndarray) -> np.ndarray:
    """Even-odd rule point-in-polygon test, vectorised over the points (px, py)."""
    inside = np.zeros(px.shape, dtype=bool)
    nv = len(vx)
    j = nv - 1
    for i in range(nv):
        xi, yi, xj, yj = vx[i], vy[i], vx[j], vy[j]
        cond = (yi > py) != (yj > py)
        if yj != yi:
            xcross = (xj - xi) * (py - yi) / (yj - yi) + xi
            inside ^= cond & (px < xcross)
        j = i
    return inside


def stereo_pair(width: int, height: int, n_labels: int, seed: int, n_polygons=None):
    """Left/right views (float64, (3, H, W), clipped to [0, 1]) and the left disparity map.

    Polygons: K ~ U{6..10}, centre uniform in the image, mean radius U[0.05, 0.35]*min(H, W),
    3..8 vertices at sorted uniform angles with radius jitter x U[0.5, 1], colour U[0,1]^3, integer
    disparity U{0..L-1}; painted in increasing disparity so nearer surfaces are on top. Texture:
    iid N(0, 0.02^2) per pixel and channel. Right view: R(x, y) = L(min(x + D_R(x, y), W-1), y),
    with D_R rendered by painting every polygon shifted by -d_k in the same order.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W = int(height), int(width)
    bg = rng.uniform(0.0, 1.0, 3)
    K = int(rng.integers(6, 11)) if n_polygons is None else int(n_polygons)
    polys = []
    for _ in range(K):
        cx = rng.uniform(0.0, W)
        cy = rng.uniform(0.0, H)
        mean_r = rng.uniform(0.05, 0.35) * min(H, W)
        nv = int(rng.integers(3, 9))
        ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, nv))
        rad = mean_r * rng.uniform(0.5, 1.0, nv)
        col = rng.uniform(0.0, 1.0, 3)
        d = int(rng.integers(0, max(1, n_labels)))
        polys.append((d, cx + rad * np.cos(ang), cy + rad * np.sin(ang), col))
    polys.sort(key=lambda t: t[0])  # stable: increasing disparity, nearer on top

    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    left = np.empty((3, H, W), dtype=np.float64)
    left[:] = bg[:, None, None]
    disp = np.zeros((H, W), dtype=np.int32)
    disp_r = np.zeros((H, W), dtype=np.int32)
    for d, vx, vy, col in polys:
        m = _inside_polygon(xs, ys, vx, vy)
        left[:, m] = col[:, None]
        disp[m] = d
        mr = _inside_polygon(xs + d, ys, vx, vy)  # right-view pixel x sees left x + d
        disp_r[mr] = d
    left += rng.normal(0.0, 0.02, size=left.shape)
    np.clip(left, 0.0, 1.0, out=left)
    xsrc = np.minimum(np.arange(W)[None, :] + disp_r, W - 1)
    right = np.take_along_axis(left, np.broadcast_to(xsrc, (3, H, W)), axis=2)
    return left, right, disp


def _grad_x(gray: np.ndarray) -> np.ndarray:
    """Central difference along x with clamped borders."""
    W = gray.shape[1]
    xp = np.minimum(np.arange(W) + 1, W - 1)
    xm = np.maximum(np.arange(W) - 1, 0)
    return 0.5 * (gray[:, xp] - gray[:, xm])


def to_dtype(v64: np.ndarray, dtype: str) -> np.ndarray:
    """Round float64 values to the storage dtype (round to nearest even).

    bf16 is returned as its raw uint16 bit pattern (numpy has no bfloat16 type)."""
    if dtype == "f32":
        return v64.astype(np.float32)
    if dtype == "f16":
        return v64.astype(np.float16)
    if dtype == "bf16":
        f = v64.astype(np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
        return rounded.astype(np.uint16)
    raise ValueError(f"unknown dtype {dtype!r}")


def from_dtype(v: np.ndarray, dtype: str) -> np.ndarray:
    """Exact float64 value of stored costs."""
    if dtype == "bf16":
        return (v.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return v.astype(np.float64)


def cost_volume(left: np.ndarray, right: np.ndarray, n_labels: int, dtype: str = "f32",
                labels=None) -> np.ndarray:
    """V(x, y, l) = 0.9 min(mean_c |L_c(x,y) - R_c(max(x-l,0),y)|, 0.028)
                  + 0.1 min(|gx L(x,y) - gx R(max(x-l,0),y)|, 0.008), label-major (L, H, W)."""
    _, H, W = left.shape
    gl = _grad_x(left.mean(axis=0))
    gr = _grad_x(right.mean(axis=0))
    labels = range(n_labels) if labels is None else labels
    out = None
    x = np.arange(W)
    for k, l in enumerate(labels):
        xs = np.maximum(x - l, 0)
        col = np.abs(left - right[:, :, xs]).mean(axis=0)
        grd = np.abs(gl - gr[:, xs])
        v = 0.9 * np.minimum(col, 0.028) + 0.1 * np.minimum(grd, 0.008)
        s = to_dtype(v, dtype)
        if out is None:
            out = np.empty((len(labels), H, W), dtype=s.dtype)
        out[k] = s
    return out


def cost_volume_torch(left, right, n_labels: int, dtype: str = "bf16", device="cuda"):
    """The same V(x, y, l) as cost_volume, built with torch on `device` (for large serving
    inputs); float32 arithmetic, then rounded to the storage dtype. Returns a torch tensor."""
    import torch
    Lt = torch.as_tensor(left, dtype=torch.float32, device=device)
    Rt = torch.as_tensor(right, dtype=torch.float32, device=device)
    _, H, W = Lt.shape

    def gx(img):
        g = img.mean(dim=0)
        xp = torch.clamp(torch.arange(W, device=device) + 1, max=W - 1)
        xm = torch.clamp(torch.arange(W, device=device) - 1, min=0)
        return 0.5 * (g[:, xp] - g[:, xm])

    gl, gr = gx(Lt), gx(Rt)
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    out = torch.empty((n_labels, H, W), dtype=tdt, device=device)
    x = torch.arange(W, device=device)
    for l in range(n_labels):
        xs = torch.clamp(x - l, min=0)
        col = (Lt - Rt[:, :, xs]).abs().mean(dim=0)
        grd = (gl - gr[:, xs]).abs()
        out[l] = (0.9 * torch.clamp(col, max=0.028) + 0.1 * torch.clamp(grd, max=0.008)).to(tdt)
    return out


def make_case(width: int, height: int, n_labels: int, seed: int, dtype: str = "f32") -> StereoCase:
    left, right, disp = stereo_pair(width, height, n_labels, seed)
    cost = cost_volume(left, right, n_labels, dtype)
    return StereoCase(guidance=left.astype(np.float32), cost=cost, cost_dtype=dtype,
                      disparity=disp, seed=seed)


# Workload shapes (width x height, labels, polynomial degree, radius, eps, storage, seed).
CONFIG_SMALL = dict(width=64, height=48, n_labels=16, degree=1, r=4, eps=1e-4, dtype="f32", seed=1)
CONFIG_QUARTER = dict(width=450, height=375, n_labels=60, degree=2, r=9, eps=1e-4, dtype="f32", seed=2)
CONFIG_LARGE = dict(width=1400, height=1100, n_labels=256, degree=2, r=9, eps=1e-4, dtype="bf16", seed=3)


def batched_cases(count: int = 32, base_seed: int = 400):
    """Mixed-size batch: sizes 320x240 / 640x480 / 1024x768 / 1280x960 (count/4 each), L drawn
    from {32, 64, 128, 192}, degree 1 or 2, r in {4, 9}; item i uses seed base_seed + i."""
    sizes = [(320, 240), (640, 480), (1024, 768), (1280, 960)]
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(base_seed + i))
        w, h = sizes[i % 4]
        L = int(rng.choice([32, 64, 128, 192]))
        degree = int(rng.integers(1, 3))
        r = int(rng.choice([4, 9]))
        out.append(dict(width=w, height=h, n_labels=L, degree=degree, r=r, eps=1e-4,
                        dtype="f32", seed=base_seed + i))
    return out


def serving_requests(n_requests: int, rate_hz: float = 200.0, seed: int = 5, reuse_p: float = 0.3,
                     sizes=((640, 480), (1024, 768), (1280, 720), (1280, 960), (1920, 1080)),
                     label_range=(64, 256), degrees=(1, 2, 3), radii=(4, 9)):
    """Open-loop Poisson request stream: exponential gaps with mean 1/rate_hz seconds. With
    probability reuse_p a request reuses the guidance key (and size) of a uniformly chosen
    earlier request. Request i draws its own image seed 5000 + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        if reqs and rng.uniform() < reuse_p:
            src = reqs[int(rng.integers(0, len(reqs)))]
            spec = dict(src)
            spec.update(arrival_s=t, request=i, image_seed=5000 + i, reused=True)
        else:
            w, h = sizes[int(rng.integers(0, len(sizes)))]
            spec = dict(arrival_s=t, request=i, width=w, height=h,
                        n_labels=int(rng.integers(label_range[0], label_range[1] + 1)),
                        degree=int(rng.choice(degrees)), r=int(rng.choice(radii)), eps=1e-4,
                        guidance_key=i, image_seed=5000 + i, reused=False)
        reqs.append(spec)
    return reqs


def gram_batch(count: int, n: int, samples: int = 25, seed: int = 7) -> np.ndarray:
    """count Gram matrices S_i = sum_k x_k x_k^T of `samples` guidance vectors x_k ~ U[0,1]^n each
    (a window's worth of polynomial-guidance samples, the matrices Sec. 3's recursion inverts);
    float64, shape (count, n, n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, 1.0, size=(count, samples, n))
    return np.einsum("cki,ckj->cij", X, X)


def gram_batch_torch(count: int, n: int, samples: int = 25, seed: int = 7, device="cuda"):
    """Same recipe built on the device with torch (for large batches): float64 (count, n, n)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    X = torch.rand((count, samples, n), generator=gen, dtype=torch.float64, device=device)
    return torch.bmm(X.transpose(1, 2), X)


def pack_upper(S):
    """(count, n, n) -> packed upper triangles row by row, element-major: (n(n+1)/2, count).
    Works for numpy arrays and torch tensors."""
    n = S.shape[-1]
    rows, cols = np.triu_indices(n)
    if isinstance(S, np.ndarray):
        return S[:, rows, cols].T.copy()
    import torch
    r = torch.as_tensor(rows, device=S.device)
    c = torch.as_tensor(cols, device=S.device)
    return S[:, r, c].transpose(0, 1).contiguous()
