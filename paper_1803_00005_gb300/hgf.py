"""Thin Python binding of libhgf's C ABI (include/hgf.h): argument marshalling only.

Every function here has the name of the C entry point it calls and passes device pointers
(``torch.Tensor.data_ptr()``) and the current CUDA stream through unchanged; all computation runs
in libhgf's kernels. The library must have been built (``paper_1803_00005_gb300.build``); loading
fails loudly otherwise - there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhgf.so")

HGF_OK, HGF_EINVAL, HGF_ENOMEM, HGF_ECUDA, HGF_ETIMEOUT, HGF_EBUSY, HGF_EAGAIN, \
    HGF_EUNSUPPORTED = range(8)
STATUS_NAMES = ["HGF_OK", "HGF_EINVAL", "HGF_ENOMEM", "HGF_ECUDA", "HGF_ETIMEOUT", "HGF_EBUSY",
                "HGF_EAGAIN", "HGF_EUNSUPPORTED"]
HGF_F32, HGF_BF16, HGF_F16, HGF_F64, HGF_DF64 = range(5)
HGF_BASIS_MONOMIAL, HGF_BASIS_POWERS = range(2)
HGF_COMBINE_ALPHA, HGF_COMBINE_W3 = range(2)
HGF_FORM_CENTRED, HGF_FORM_PAPER = range(2)
HGF_INV_PROP1, HGF_INV_CHOLESKY = range(2)

DTYPE_CODES = {"f32": HGF_F32, "bf16": HGF_BF16, "f16": HGF_F16, "f64": HGF_F64,
               "df64": HGF_DF64}
BASIS_CODES = {"monomial": HGF_BASIS_MONOMIAL, "powers": HGF_BASIS_POWERS}
FORM_CODES = {"centred": HGF_FORM_CENTRED, "paper": HGF_FORM_PAPER}

# Every symbol include/hgf.h declares.
EXPORTED = [
    "hgf_create", "hgf_destroy", "hgf_last_error", "hgf_num_channels", "hgf_make_guidance",
    "hgf_prepare", "hgf_guidance_release", "hgf_guidance_info", "hgf_guidance_export",
    "hgf_aggregate", "hgf_aggregate_plain", "hgf_wta", "hgf_filter_host", "hgf_set_tuning",
    "hgf_guidance_update", "hgf_launch_count", "hgf_last_plan", "hgf_profile_enable",
    "hgf_profile_report",
    "hgf_aggregate_static", "hgf_serve_create", "hgf_serve_submit", "hgf_serve_poll",
    "hgf_serve_wait", "hgf_serve_stats", "hgf_serve_inject_alloc_failures", "hgf_serve_destroy",
    "hgf_batch_create", "hgf_batch_run", "hgf_batch_launch_graph", "hgf_batch_destroy",
    "hgf_device_status", "hgf_batched_inverse", "hgf_cost_volume", "hgf_aggregate_stereo",
    "hgf_refine_lr", "hgf_autotune", "hgf_watchdog_probe", "hgf_stereo_host",
    "hgf_aggregate_margin", "hgf_wta_margin", "hgf_filter",
]


class HGFError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


class hgf_params(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("basis", ctypes.c_int), ("r", ctypes.c_int),
                ("eps", ctypes.c_double), ("inv_precision", ctypes.c_int),
                ("combine", ctypes.c_int), ("form", ctypes.c_int),
                ("compensated", ctypes.c_int)]


class hgf_cost_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tau_color", ctypes.c_double),
                ("tau_grad", ctypes.c_double), ("direction", ctypes.c_int)]


class hgf_tuning(ctypes.Structure):
    _fields_ = [("labels_per_pass", ctypes.c_int), ("band_rows", ctypes.c_int),
                ("chunk_labels", ctypes.c_int), ("apply_mode", ctypes.c_int),
                ("kernel", ctypes.c_int)]


class hgf_request(ctypes.Structure):
    _fields_ = [("guidance_key", ctypes.c_uint64), ("img", ctypes.c_void_p), ("C", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int), ("params", hgf_params),
                ("cost", ctypes.c_void_p), ("cost_dtype", ctypes.c_int), ("L", ctypes.c_int),
                ("labels", ctypes.c_void_p), ("best", ctypes.c_void_p)]


class hgf_job(ctypes.Structure):
    _fields_ = [("img", ctypes.c_void_p), ("C", ctypes.c_int), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("params", hgf_params), ("cost", ctypes.c_void_p),
                ("cost_dtype", ctypes.c_int), ("L", ctypes.c_int), ("labels", ctypes.c_void_p),
                ("best", ctypes.c_void_p), ("filtered", ctypes.c_void_p)]


class hgf_serve_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "rejected_busy",
                                               "rejected_nomem", "cache_hits", "cache_misses",
                                               "evictions")] + \
               [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "max_ms",
                                               "mpixel_labels_per_s")] + \
               [(n, ctypes.c_size_t) for n in ("budget_bytes", "resident_bytes", "peak_bytes")] + \
               [("slots", ctypes.c_int), ("max_concurrent", ctypes.c_int)] + \
               [("queue_mean_ms", ctypes.c_double), ("queue_p99_ms", ctypes.c_double),
                ("prepare_ms_total", ctypes.c_double * 3),
                ("aggregate_ms_total", ctypes.c_double * 3),
                ("completed_by_class", ctypes.c_uint64 * 3)]

    def as_dict(self):
        out = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            out[f] = list(v) if isinstance(v, ctypes.Array) else v
        return out


_lib = None


def lib():
    """Loads libhgf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_1803_00005_gb300.build` (there is no fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, c_int, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "hgf_create": (c_int, [c_int, P(vp)]),
        "hgf_destroy": (c_int, [vp]),
        "hgf_last_error": (ctypes.c_char_p, [vp]),
        "hgf_num_channels": (c_int, [c_int, c_int, c_int]),
        "hgf_make_guidance": (c_int, [vp, vp, c_int, c_int, c_int, c_int, c_int, vp, P(c_int), vp]),
        "hgf_prepare": (c_int, [vp, vp, c_int, c_int, c_int, P(hgf_params), vp, P(vp)]),
        "hgf_guidance_release": (c_int, [vp]),
        "hgf_guidance_info": (c_int, [vp, P(c_int), P(c_int), P(c_int), P(c_int), P(c_int),
                                      P(c_double)]),
        "hgf_guidance_export": (c_int, [vp, vp, vp, vp, vp]),
        "hgf_aggregate": (c_int, [vp, vp, vp, c_int, c_int, vp, c_int, vp, vp, vp]),
        "hgf_filter": (c_int, [vp, vp, vp, vp, c_int, c_int, vp, c_int, vp, vp, vp]),
        "hgf_aggregate_plain": (c_int, [vp, vp, vp, c_int, c_int, vp, c_int, vp, vp, vp]),
        "hgf_aggregate_static": (c_int, [vp, vp, vp, c_int, c_int, vp, c_int, vp, vp, vp]),
        "hgf_serve_create": (c_int, [c_int, ctypes.c_size_t, c_int, c_int, c_int, c_int, P(vp)]),
        "hgf_serve_submit": (c_int, [vp, P(hgf_request), P(ctypes.c_uint64)]),
        "hgf_serve_poll": (c_int, [vp, ctypes.c_uint64]),
        "hgf_serve_wait": (c_int, [vp, ctypes.c_uint64, c_int]),
        "hgf_serve_stats": (c_int, [vp, P(hgf_serve_stats_t), c_int]),
        "hgf_serve_inject_alloc_failures": (c_int, [vp, c_int]),
        "hgf_serve_destroy": (c_int, [vp]),
        "hgf_batch_create": (c_int, [vp, P(hgf_job), c_int, c_int, P(vp)]),
        "hgf_batch_run": (c_int, [vp, vp]),
        "hgf_batch_launch_graph": (c_int, [vp, vp]),
        "hgf_batch_destroy": (c_int, [vp]),
        "hgf_wta": (c_int, [vp, vp, c_int, c_int, c_int, c_int, vp, vp, vp]),
        "hgf_wta_margin": (c_int, [vp, vp, c_int, c_int, c_int, c_int, vp, vp, vp, vp]),
        "hgf_aggregate_margin": (c_int, [vp, vp, vp, c_int, c_int, vp, vp, vp, vp]),
        "hgf_filter_host": (c_int, [vp, vp, c_int, c_int, c_int, P(hgf_params), vp, c_int, c_int,
                                    vp, vp, vp]),
        "hgf_set_tuning": (c_int, [vp, P(hgf_tuning)]),
        "hgf_guidance_update": (c_int, [vp, vp, vp, vp]),
        "hgf_launch_count": (c_int, [vp, P(ctypes.c_ulonglong)]),
        "hgf_last_plan": (c_int, [vp, P(c_int), c_int]),
        "hgf_device_status": (c_int, [vp, P(c_int), c_int]),
        "hgf_watchdog_probe": (c_int, [vp, c_int, vp]),
        "hgf_stereo_host": (c_int, [vp, vp, vp, c_int, c_int, c_int, c_int, P(hgf_params),
                                    P(hgf_cost_params), c_int, c_int, vp, vp]),
        "hgf_batched_inverse": (c_int, [vp, vp, c_int, c_int, c_double, c_int, c_int, vp, vp]),
        "hgf_cost_volume": (c_int, [vp, vp, vp, c_int, c_int, c_int, c_int, P(hgf_cost_params),
                                    c_int, vp, vp]),
        "hgf_aggregate_stereo": (c_int, [vp, vp, vp, c_int, P(hgf_cost_params), vp, c_int, vp,
                                         vp, vp]),
        "hgf_refine_lr": (c_int, [vp, vp, vp, c_int, c_int, c_int, vp, vp, vp]),
        "hgf_autotune": (c_int, [vp, vp, vp, c_int, c_int, vp, c_int, P(hgf_tuning), P(c_int),
                                 vp]),
        "hgf_profile_enable": (c_int, [vp, c_int]),
        "hgf_profile_report": (c_int, [vp, ctypes.c_char_p, ctypes.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(ctx, st):
    if st != HGF_OK:
        msg = lib().hgf_last_error(ctx) if ctx else b""
        raise HGFError(st, (msg or b"").decode(errors="replace"))


def _dtype_code(t):
    import torch
    return {torch.float32: HGF_F32, torch.bfloat16: HGF_BF16, torch.float16: HGF_F16,
            torch.float64: HGF_F64}[t.dtype]


def _require_cuda(t, name):
    if t is not None and (not t.is_cuda or not t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


def make_params(degree=1, r=4, eps=1e-4, basis="monomial", inv_precision="f64", combine="alpha",
                form="centred", compensated=False):
    """form: "centred" (Sec. 5.1; eps in units of window means) or "paper" (G_0 = 1, uncentred
    window sums, lambda = eps in units of window sums; Sec. 3-4). compensated: Kahan-compensated
    running sums in the strip kernels."""
    return hgf_params(degree=int(degree), basis=BASIS_CODES[basis], r=int(r), eps=float(eps),
                      inv_precision=DTYPE_CODES[inv_precision],
                      combine=HGF_COMBINE_ALPHA if combine == "alpha" else HGF_COMBINE_W3,
                      form=FORM_CODES[form], compensated=1 if compensated else 0)


# ------------------------------------------------------------------ entry points, same names
def hgf_create(device=0):
    h = ctypes.c_void_p()
    st = lib().hgf_create(int(device), ctypes.byref(h))
    if st != HGF_OK:
        raise HGFError(st, f"hgf_create(device={device}) failed")
    return h


def hgf_destroy(ctx):
    lib().hgf_destroy(ctx)


def hgf_last_error(ctx):
    return (lib().hgf_last_error(ctx) or b"").decode(errors="replace")


def hgf_num_channels(C, degree, basis="monomial"):
    return lib().hgf_num_channels(int(C), int(degree), BASIS_CODES[basis])


def hgf_make_guidance(ctx, img, degree, basis="monomial", G_out=None, stream=None):
    import torch
    _require_cuda(img, "img")
    C, H, W = img.shape
    n = hgf_num_channels(C, degree, basis)
    if G_out is None:
        G_out = torch.empty((n, H, W), dtype=torch.float32, device=img.device)
    n_out = ctypes.c_int()
    _check(ctx, lib().hgf_make_guidance(ctx, _ptr(img), C, H, W, int(degree), BASIS_CODES[basis],
                                        _ptr(G_out), ctypes.byref(n_out), _stream(stream)))
    return G_out


def hgf_prepare(ctx, img, params, stream=None):
    _require_cuda(img, "img")
    C, H, W = img.shape
    g = ctypes.c_void_p()
    _check(ctx, lib().hgf_prepare(ctx, _ptr(img), C, H, W, ctypes.byref(params), _stream(stream),
                                  ctypes.byref(g)))
    return g


def hgf_guidance_release(g):
    lib().hgf_guidance_release(g)


def hgf_guidance_info(g):
    v = [ctypes.c_int() for _ in range(5)]
    eps = ctypes.c_double()
    st = lib().hgf_guidance_info(g, *[ctypes.byref(x) for x in v], ctypes.byref(eps))
    if st != HGF_OK:
        raise HGFError(st, "hgf_guidance_info")
    C, H, W, n, r = (x.value for x in v)
    return dict(C=C, H=H, W=W, n=n, r=r, eps=eps.value)


def hgf_guidance_export(ctx, g, minv_out=None, mu_out=None, stream=None):
    _check(ctx, lib().hgf_guidance_export(ctx, g, _ptr(minv_out), _ptr(mu_out), _stream(stream)))


def hgf_aggregate(ctx, g, cost, filtered=None, labels=None, best=None, stream=None):
    for t, nm in ((cost, "cost"), (filtered, "filtered"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    L = cost.shape[0]
    _check(ctx, lib().hgf_aggregate(ctx, g, _ptr(cost), _dtype_code(cost), L, _ptr(filtered),
                                    HGF_F32, _ptr(labels), _ptr(best), _stream(stream)))


def hgf_filter(ctx, g, img, cost, filtered=None, labels=None, best=None, stream=None):
    """hgf_guidance_update(g, img) + hgf_aggregate(g, cost) in one call (see include/hgf.h)."""
    for t, nm in ((img, "img"), (cost, "cost"), (filtered, "filtered"), (labels, "labels"),
                  (best, "best")):
        _require_cuda(t, nm)
    L = cost.shape[0]
    _check(ctx, lib().hgf_filter(ctx, g, _ptr(img), _ptr(cost), _dtype_code(cost), L,
                                 _ptr(filtered), HGF_F32, _ptr(labels), _ptr(best),
                                 _stream(stream)))


def hgf_aggregate_static(ctx, g, cost, filtered=None, labels=None, best=None, stream=None):
    """hgf_aggregate without device allocation: scratch comes from the library's fixed 64 MiB
    device array (see include/hgf.h)."""
    for t, nm in ((cost, "cost"), (filtered, "filtered"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    L = cost.shape[0]
    _check(ctx, lib().hgf_aggregate_static(ctx, g, _ptr(cost), _dtype_code(cost), L,
                                           _ptr(filtered), HGF_F32, _ptr(labels), _ptr(best),
                                           _stream(stream)))


def hgf_aggregate_plain(ctx, g, cost, filtered=None, labels=None, best=None, stream=None):
    for t, nm in ((cost, "cost"), (filtered, "filtered"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    L = cost.shape[0]
    _check(ctx, lib().hgf_aggregate_plain(ctx, g, _ptr(cost), _dtype_code(cost), L,
                                          _ptr(filtered), HGF_F32, _ptr(labels), _ptr(best),
                                          _stream(stream)))


def hgf_aggregate_margin(ctx, g, cost, margin, labels=None, best=None, stream=None):
    """hgf_aggregate with the WTA margin: second-smallest minus smallest filtered cost."""
    for t, nm in ((cost, "cost"), (margin, "margin"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    L = cost.shape[0]
    _check(ctx, lib().hgf_aggregate_margin(ctx, g, _ptr(cost), _dtype_code(cost), L,
                                           _ptr(labels), _ptr(best), _ptr(margin),
                                           _stream(stream)))


def hgf_wta_margin(ctx, filtered, margin, labels=None, best=None, stream=None):
    for t, nm in ((filtered, "filtered"), (margin, "margin"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    L, H, W = filtered.shape
    _check(ctx, lib().hgf_wta_margin(ctx, _ptr(filtered), HGF_F32, L, H, W, _ptr(labels),
                                     _ptr(best), _ptr(margin), _stream(stream)))


def hgf_wta(ctx, filtered, labels=None, best=None, stream=None):
    _require_cuda(filtered, "filtered")
    L, H, W = filtered.shape
    _check(ctx, lib().hgf_wta(ctx, _ptr(filtered), HGF_F32, L, H, W, _ptr(labels), _ptr(best),
                              _stream(stream)))


def hgf_filter_host(ctx, img, cost, cost_dtype, params, labels, best=None, stream=None):
    """img: numpy float32 (C, H, W); cost: numpy (L, H, W) raw storage (float32, float16 or
    bf16 bits as uint16); labels: numpy int32 (H, W); best: numpy float32 (H, W) or None.
    Host buffers may be pinned (e.g. numpy views of pinned torch tensors)."""
    import numpy as np
    C, H, W = img.shape
    L = cost.shape[0]
    for a in (img, cost, labels, best):
        if a is not None and not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
    assert img.dtype == np.float32 and labels.dtype == np.int32
    st = lib().hgf_filter_host(ctx, ctypes.c_void_p(img.ctypes.data), C, H, W,
                               ctypes.byref(params), ctypes.c_void_p(cost.ctypes.data),
                               DTYPE_CODES[cost_dtype], L,
                               ctypes.c_void_p(labels.ctypes.data),
                               None if best is None else ctypes.c_void_p(best.ctypes.data),
                               _stream(stream))
    _check(ctx, st)


def hgf_set_tuning(ctx, labels_per_pass=0, band_rows=0, chunk_labels=0, apply_mode=0, kernel=0):
    """kernel: 0 automatic, 1 single pass (n <= 9), 2 coefficient + output kernels."""
    t = hgf_tuning(labels_per_pass=labels_per_pass, band_rows=band_rows,
                   chunk_labels=chunk_labels, apply_mode=apply_mode, kernel=kernel)
    _check(ctx, lib().hgf_set_tuning(ctx, ctypes.byref(t)))


def hgf_guidance_update(ctx, g, img, stream=None):
    _require_cuda(img, "img")
    _check(ctx, lib().hgf_guidance_update(ctx, g, _ptr(img), _stream(stream)))


def hgf_launch_count(ctx):
    v = ctypes.c_ulonglong()
    _check(ctx, lib().hgf_launch_count(ctx, ctypes.byref(v)))
    return v.value


PLAN_FIELDS = ("path", "out_strip", "coef_strip", "band_rows", "apply_band_rows",
               "labels_per_pass", "chunk", "ctas")


def hgf_last_plan(ctx):
    """The plan of ctx's last aggregation as a dict (PLAN_FIELDS; path 1 single pass, 2 two
    kernels, 3 plain)."""
    arr = (ctypes.c_int * 8)()
    _check(ctx, lib().hgf_last_plan(ctx, arr, 8))
    return dict(zip(PLAN_FIELDS, list(arr)))


def hgf_batched_inverse(ctx, S, n, lam, method="prop1", precision="f64", out=None, stream=None):
    """(lam E + S_i)^-1 for the packed, element-major float64 batch S of shape (n(n+1)/2, count)
    on the device; returns `out` (allocated like S when None)."""
    _require_cuda(S, "S")
    if S.dim() != 2 or S.shape[0] != n * (n + 1) // 2 or str(S.dtype) != "torch.float64":
        raise ValueError("S must be float64 of shape (n(n+1)/2, count)")
    if out is None:
        import torch
        out = torch.empty_like(S)
    _require_cuda(out, "out")
    count = int(S.shape[1])
    _check(ctx, lib().hgf_batched_inverse(
        ctx, _ptr(S), count, int(n), float(lam),
        HGF_INV_PROP1 if method == "prop1" else HGF_INV_CHOLESKY, DTYPE_CODES[precision],
        _ptr(out), _stream(stream)))
    return out


def hgf_cost_volume(ctx, ref, other, L, out=None, dtype="f32", alpha=0.9, tau_color=0.028,
                    tau_grad=0.008, direction=1, stream=None):
    """Stereo cost volume V (L, H, W) of the float32 (C, H, W) views `ref` and `other` on the
    device; returns `out` (allocated when None; a bfloat16/float16/float32 tensor)."""
    _require_cuda(ref, "ref")
    _require_cuda(other, "other")
    C, H, W = ref.shape
    if tuple(other.shape) != (C, H, W):
        raise ValueError("ref and other must have the same shape")
    if out is None:
        import torch
        tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[dtype]
        out = torch.empty((L, H, W), dtype=tdt, device=ref.device)
    _require_cuda(out, "out")
    p = hgf_cost_params(alpha=float(alpha), tau_color=float(tau_color), tau_grad=float(tau_grad),
                        direction=int(direction))
    _check(ctx, lib().hgf_cost_volume(ctx, _ptr(ref), _ptr(other), C, H, W, int(L),
                                      ctypes.byref(p), _dtype_code(out), _ptr(out),
                                      _stream(stream)))
    return out


def hgf_aggregate_stereo(ctx, g, other, L, filtered=None, labels=None, best=None, alpha=0.9,
                         tau_color=0.028, tau_grad=0.008, direction=1, stream=None):
    """Aggregation + WTA of the stereo cost of (guidance image, other) computed on the fly."""
    for t, nm in ((other, "other"), (filtered, "filtered"), (labels, "labels"), (best, "best")):
        _require_cuda(t, nm)
    p = hgf_cost_params(alpha=float(alpha), tau_color=float(tau_color), tau_grad=float(tau_grad),
                        direction=int(direction))
    _check(ctx, lib().hgf_aggregate_stereo(ctx, g, _ptr(other), int(L), ctypes.byref(p),
                                           _ptr(filtered), HGF_F32, _ptr(labels), _ptr(best),
                                           _stream(stream)))


def hgf_refine_lr(ctx, disp_left, disp_right, threshold=1, out=None, keep=None, stream=None):
    """Left-right consistency + hole filling of int32 (H, W) disparity maps on the device;
    returns (out, keep)."""
    import torch
    for t, nm in ((disp_left, "disp_left"), (disp_right, "disp_right")):
        _require_cuda(t, nm)
        if t.dtype != torch.int32:
            raise ValueError(f"{nm} must be int32")
    H, W = disp_left.shape
    if out is None:
        out = torch.empty_like(disp_left)
    if keep is None:
        keep = torch.empty((H, W), dtype=torch.uint8, device=disp_left.device)
    _require_cuda(out, "out")
    _require_cuda(keep, "keep")
    _check(ctx, lib().hgf_refine_lr(ctx, _ptr(disp_left), _ptr(disp_right), H, W, int(threshold),
                                    _ptr(out), _ptr(keep), _stream(stream)))
    return out, keep


def hgf_autotune(ctx, g, cost, labels, reps=3, stream=None):
    """Times every result-preserving tuning on (g, cost), keeps the fastest on ctx; returns
    (tuning dict, candidates timed)."""
    _require_cuda(cost, "cost")
    _require_cuda(labels, "labels")
    t = hgf_tuning()
    n = ctypes.c_int()
    _check(ctx, lib().hgf_autotune(ctx, g, _ptr(cost), _dtype_code(cost), cost.shape[0],
                                   _ptr(labels), int(reps), ctypes.byref(t), ctypes.byref(n),
                                   _stream(stream)))
    return dict(labels_per_pass=t.labels_per_pass, band_rows=t.band_rows,
                chunk_labels=t.chunk_labels, apply_mode=t.apply_mode, kernel=t.kernel), n.value


def autotune_cached(ctx, g, cost, labels, cache_path, reps=3, stream=None):
    """hgf_autotune behind a JSON cache file keyed by GPU name, guidance channels n, radius r,
    cost dtype and size class (H*W and L rounded up to powers of two). A hit sets the cached
    tuning on ctx without timing anything. Returns (tuning dict, hit)."""
    import json
    import os
    import torch
    info = hgf_guidance_info(g)
    pow2 = lambda v: 1 << max(0, int(v - 1).bit_length())  # noqa: E731
    key = "|".join(str(x) for x in (torch.cuda.get_device_name(cost.device), info["n"],
                                     info["r"], str(cost.dtype).replace("torch.", ""),
                                     pow2(info["H"] * info["W"]), pow2(cost.shape[0])))
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        hgf_set_tuning(ctx, **cache[key])
        return dict(cache[key]), True
    tuning, _ = hgf_autotune(ctx, g, cost, labels, reps=reps, stream=stream)
    cache[key] = tuning
    tmp = cache_path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return tuning, False


def hgf_stereo_host(ctx, left, right, L, params, refine=True, threshold=1, out=None,
                    alpha=0.9, tau_color=0.028, tau_grad=0.008, stream=None):
    """Stereo pipeline from host memory: left/right float32 (C, H, W) numpy arrays (pinned or
    pageable) in, int32 (H, W) disparity numpy array out (written into `out` when given)."""
    import numpy as np
    left = np.ascontiguousarray(left, dtype=np.float32)
    right = np.ascontiguousarray(right, dtype=np.float32)
    if left.shape != right.shape or left.ndim != 3:
        raise ValueError("left and right must be (C, H, W) arrays of the same shape")
    C, H, W = left.shape
    if out is None:
        out = np.empty((H, W), dtype=np.int32)
    if out.dtype != np.int32 or out.shape != (H, W) or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a contiguous int32 (H, W) array")
    cp = hgf_cost_params(alpha=float(alpha), tau_color=float(tau_color), tau_grad=float(tau_grad),
                         direction=1)
    _check(ctx, lib().hgf_stereo_host(ctx, left.ctypes.data, right.ctypes.data, C, H, W, int(L),
                                      ctypes.byref(params), ctypes.byref(cp),
                                      1 if refine else 0, int(threshold), out.ctypes.data,
                                      _stream(stream)))
    return out


def hgf_watchdog_probe(ctx, limit_us, stream=None):
    """Enqueues a wait that nothing completes; it times out after limit_us and sets the device
    status word (test hook for the kernels' bounded waits)."""
    _check(ctx, lib().hgf_watchdog_probe(ctx, int(limit_us), _stream(stream)))


def hgf_device_status(ctx, clear=False):
    """Watchdog word of ctx's device after all its work: 0 unless a bounded wait in a kernel ran
    out (that call's results are then incomplete)."""
    v = ctypes.c_int()
    _check(ctx, lib().hgf_device_status(ctx, ctypes.byref(v), 1 if clear else 0))
    return v.value


def hgf_profile_enable(ctx, enable=True):
    _check(ctx, lib().hgf_profile_enable(ctx, 1 if enable else 0))


def hgf_profile_report(ctx):
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(ctx, lib().hgf_profile_report(ctx, buf, len(buf)))
    return json.loads(buf.value.decode())


# ------------------------------------------------------------------------------------ serving
def hgf_serve_create(device=0, budget_bytes=8 << 30, slots=4, max_queue=256,
                     max_pixels=1920 * 1080, max_n=19):
    h = ctypes.c_void_p()
    st = lib().hgf_serve_create(int(device), int(budget_bytes), int(slots), int(max_queue),
                                int(max_pixels), int(max_n), ctypes.byref(h))
    if st != HGF_OK:
        raise HGFError(st, "hgf_serve_create failed")
    return h


def make_request(guidance_key, img, cost, params, labels, best=None):
    """Request structure for device tensors img (C, H, W), cost (L, H, W), labels (H, W)."""
    C, H, W = img.shape
    return hgf_request(guidance_key=int(guidance_key), img=img.data_ptr(), C=C, H=H, W=W,
                       params=params, cost=cost.data_ptr(), cost_dtype=_dtype_code(cost),
                       L=cost.shape[0], labels=labels.data_ptr(),
                       best=None if best is None else best.data_ptr())


def hgf_serve_submit(server, req):
    """Returns (status, id); status is HGF_OK, HGF_EBUSY, HGF_ENOMEM, ..."""
    rid = ctypes.c_uint64()
    st = lib().hgf_serve_submit(server, ctypes.byref(req), ctypes.byref(rid))
    return st, rid.value


def hgf_serve_poll(server, rid):
    return lib().hgf_serve_poll(server, ctypes.c_uint64(rid))


def hgf_serve_wait(server, rid, timeout_ms=-1):
    return lib().hgf_serve_wait(server, ctypes.c_uint64(rid), int(timeout_ms))


def hgf_serve_stats(server, reset=False):
    s = hgf_serve_stats_t()
    st = lib().hgf_serve_stats(server, ctypes.byref(s), 1 if reset else 0)
    if st != HGF_OK:
        raise HGFError(st, "hgf_serve_stats")
    return s.as_dict()


def hgf_serve_inject_alloc_failures(server, count):
    return lib().hgf_serve_inject_alloc_failures(server, int(count))


def hgf_serve_destroy(server):
    lib().hgf_serve_destroy(server)


# -------------------------------------------------------------------------------------- batches
def make_job(img, cost, params, labels=None, best=None, filtered=None):
    C, H, W = img.shape
    return hgf_job(img=img.data_ptr(), C=C, H=H, W=W, params=params, cost=cost.data_ptr(),
                   cost_dtype=_dtype_code(cost), L=cost.shape[0],
                   labels=None if labels is None else labels.data_ptr(),
                   best=None if best is None else best.data_ptr(),
                   filtered=None if filtered is None else filtered.data_ptr())


def hgf_batch_create(ctx, jobs, streams=8):
    arr = (hgf_job * len(jobs))(*jobs)
    h = ctypes.c_void_p()
    _check(ctx, lib().hgf_batch_create(ctx, arr, len(jobs), int(streams), ctypes.byref(h)))
    return h


def hgf_batch_run(ctx, batch, stream=None):
    _check(ctx, lib().hgf_batch_run(batch, _stream(stream)))


def hgf_batch_launch_graph(ctx, batch, stream=None):
    _check(ctx, lib().hgf_batch_launch_graph(batch, _stream(stream)))


def hgf_batch_destroy(batch):
    lib().hgf_batch_destroy(batch)
