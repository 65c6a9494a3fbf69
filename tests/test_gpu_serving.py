"""Serving loop (hgf_serve_*): results of requests run in a mix of concurrent requests equal the
results of the same requests run alone, and the degree-3 and bfloat16 requests match the float64
oracle directly; guidance reuse, admission by memory budget, queue limits,
bounded waits and injected allocation failures behave as documented. Failures are made on the
host (an allocation made to fail, a budget too small, a wait with a short limit): no GPU fault."""
import numpy as np
import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def make_inputs(torch, specs):
    from paper_1803_00005_gb300 import synth
    out = []
    for sp in specs:
        case = synth.make_case(sp["w"], sp["h"], sp["L"], sp["seed"], sp.get("dtype", "f32"))
        img = torch.from_numpy(case.guidance).cuda()
        if sp.get("dtype", "f32") == "bf16":
            cost = torch.from_numpy(case.cost.view(np.int16)).cuda().view(torch.bfloat16)
        else:
            cost = torch.from_numpy(case.cost).cuda()
        out.append(dict(sp, img=img, cost=cost, case=case))
    return out


def oracle_check(item, labels, best):
    """A served (or batched) result against the float64 oracle on the same (rounded) inputs."""
    from oracle import hgf_oracle as O
    from paper_1803_00005_gb300 import synth
    from gpu_helpers import check_against_oracle
    case = item["case"]
    ref = O.centred_filter(case.guidance, synth.from_dtype(case.cost, item.get("dtype", "f32")),
                           item["r"], 1e-4, item["degree"])
    check_against_oracle(None, labels, best, ref)


def alone(torch, hgf, ctx, item):
    p = hgf.make_params(degree=item["degree"], r=item["r"], eps=1e-4)
    g = hgf.hgf_prepare(ctx, item["img"], p)
    H, W = item["h"], item["w"]
    lab = torch.empty((H, W), dtype=torch.int32, device="cuda")
    best = torch.empty((H, W), device="cuda")
    hgf.hgf_aggregate(ctx, g, item["cost"], labels=lab, best=best)
    torch.cuda.synchronize()
    hgf.hgf_guidance_release(g)
    return lab.cpu().numpy(), best.cpu().numpy()


SPECS = [dict(w=320, h=240, L=32, seed=101, degree=2, r=9, key=1),
         dict(w=200, h=150, L=20, seed=102, degree=1, r=4, key=2),
         dict(w=320, h=240, L=24, seed=103, degree=2, r=9, key=1),   # same guidance key as #0
         dict(w=256, h=192, L=16, seed=104, degree=3, r=4, key=3),
         dict(w=160, h=120, L=48, seed=105, degree=2, r=4, key=4, dtype="bf16"),
         dict(w=300, h=200, L=40, seed=106, degree=1, r=9, key=5)]


def test_mix_equals_alone_and_cache_reuse():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    items = make_inputs(torch, SPECS)
    # request #2 shares #0's guidance: give it #0's image so the shared guidance is right
    items[2]["img"] = items[0]["img"]
    ctx = hgf.hgf_create(0)
    try:
        refs = [alone(torch, hgf, ctx, it) for it in items]
    finally:
        hgf.hgf_destroy(ctx)
    srv = hgf.hgf_serve_create(0, budget_bytes=6 << 30, slots=3, max_queue=64,
                               max_pixels=320 * 240, max_n=19)
    try:
        outs, ids = [], []
        for it in items:
            lab = torch.full((it["h"], it["w"]), -1, dtype=torch.int32, device="cuda")
            best = torch.full((it["h"], it["w"]), float("nan"), device="cuda")
            req = hgf.make_request(it["key"], it["img"], it["cost"],
                                   hgf.make_params(degree=it["degree"], r=it["r"], eps=1e-4),
                                   lab, best)
            st, rid = hgf.hgf_serve_submit(srv, req)
            assert st == hgf.HGF_OK
            outs.append((lab, best))
            ids.append(rid)
        for rid in ids:
            assert hgf.hgf_serve_wait(srv, rid, 60000) == hgf.HGF_OK
        for (lab, best), (rl, rb) in zip(outs, refs):
            assert np.array_equal(lab.cpu().numpy(), rl)
            assert np.array_equal(best.cpu().numpy(), rb)
        # served results against the oracle directly: the degree-3 (n = 19) request and the
        # bfloat16 one
        for k in (3, 4):
            oracle_check(items[k], outs[k][0].cpu().numpy(), outs[k][1].cpu().numpy())
        stats = hgf.hgf_serve_stats(srv)
        assert stats["completed"] == len(items)
        assert stats["cache_hits"] >= 1
        assert stats["max_concurrent"] >= 2           # requests overlapped on the device
        assert stats["p99_ms"] >= stats["p50_ms"] > 0
        assert hgf.hgf_serve_poll(srv, ids[0]) == hgf.HGF_OK
        assert hgf.hgf_serve_poll(srv, 10 ** 9) == hgf.HGF_EINVAL
    finally:
        hgf.hgf_serve_destroy(srv)


def test_admission_limits_timeouts_and_injected_failures():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    items = make_inputs(torch, [dict(w=256, h=192, L=64, seed=201, degree=2, r=9, key=7),
                                dict(w=256, h=192, L=8, seed=202, degree=1, r=4, key=8)])
    big, small = items
    p_big = hgf.make_params(degree=2, r=9, eps=1e-4)
    p_small = hgf.make_params(degree=1, r=4, eps=1e-4)

    def req(it, p, key=None):
        lab = torch.empty((it["h"], it["w"]), dtype=torch.int32, device="cuda")
        return hgf.make_request(it["key"] if key is None else key, it["img"], it["cost"], p,
                                lab), lab

    # a budget that holds the slot workspaces but no guidance: the request alone cannot fit
    srv = hgf.hgf_serve_create(0, budget_bytes=1 << 30, slots=1, max_queue=2,
                               max_pixels=256 * 192, max_n=9)
    try:
        ws = hgf.hgf_serve_stats(srv)["resident_bytes"]
    finally:
        hgf.hgf_serve_destroy(srv)
    srv = hgf.hgf_serve_create(0, budget_bytes=ws + 1024, slots=1, max_queue=2,
                               max_pixels=256 * 192, max_n=9)
    try:
        r, _ = req(small, p_small)
        st, _ = hgf.hgf_serve_submit(srv, r)
        assert st == hgf.HGF_ENOMEM
        # image larger than the slots were sized for
        r2, _ = req(dict(big, w=1024, h=768, img=torch.rand((3, 768, 1024), device="cuda"),
                         cost=torch.rand((2, 768, 1024), device="cuda")), p_small)
        st, _ = hgf.hgf_serve_submit(srv, r2)
        assert st == hgf.HGF_EUNSUPPORTED
    finally:
        hgf.hgf_serve_destroy(srv)

    srv = hgf.hgf_serve_create(0, budget_bytes=4 << 30, slots=1, max_queue=2,
                               max_pixels=256 * 192, max_n=9)
    try:
        keep = []
        # queue limit: one running + two queued at most; further submissions are refused
        statuses = []
        for i in range(8):
            r, lab = req(big, p_big, key=100 + i)
            keep.append((r, lab))
            statuses.append(hgf.hgf_serve_submit(srv, r))
        assert any(st == hgf.HGF_EBUSY for st, _ in statuses)
        accepted = [rid for st, rid in statuses if st == hgf.HGF_OK]
        assert hgf.hgf_serve_wait(srv, accepted[-1], 0) in (hgf.HGF_ETIMEOUT, hgf.HGF_OK)
        for rid in accepted:
            assert hgf.hgf_serve_wait(srv, rid, 60000) == hgf.HGF_OK
        # an allocation made to fail on the host side: that request fails, the next succeeds
        assert hgf.hgf_serve_inject_alloc_failures(srv, 1) == hgf.HGF_OK
        r1, _ = req(small, p_small, key=500)
        st1, id1 = hgf.hgf_serve_submit(srv, r1)
        r2, lab2 = req(small, p_small, key=501)
        st2, id2 = hgf.hgf_serve_submit(srv, r2)
        assert st1 == hgf.HGF_OK and st2 == hgf.HGF_OK
        assert hgf.hgf_serve_wait(srv, id1, 60000) == hgf.HGF_ENOMEM
        assert hgf.hgf_serve_wait(srv, id2, 60000) == hgf.HGF_OK
        s = hgf.hgf_serve_stats(srv)
        assert s["failed"] == 1 and s["rejected_busy"] >= 1
    finally:
        hgf.hgf_serve_destroy(srv)


def test_eviction_under_budget_keeps_results_exact():
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    items = make_inputs(torch, [dict(w=320, h=240, L=12, seed=300 + i, degree=2, r=9, key=i)
                                for i in range(4)])
    ctx = hgf.hgf_create(0)
    try:
        refs = [alone(torch, hgf, ctx, it) for it in items]
    finally:
        hgf.hgf_destroy(ctx)
    probe = hgf.hgf_serve_create(0, budget_bytes=8 << 30, slots=1, max_queue=8,
                                 max_pixels=320 * 240, max_n=9)
    ws = hgf.hgf_serve_stats(probe)["resident_bytes"]
    hgf.hgf_serve_destroy(probe)
    per_guidance = 320 * 240 * (56 + 3 + 9 + 45 + 9) * 4 + 256
    srv = hgf.hgf_serve_create(0, budget_bytes=ws + int(1.5 * per_guidance), slots=1,
                               max_queue=8, max_pixels=320 * 240, max_n=9)
    try:
        for rep in range(2):
            for it, (rl, rb) in zip(items, refs):
                lab = torch.empty((240, 320), dtype=torch.int32, device="cuda")
                r = hgf.make_request(it["key"], it["img"], it["cost"],
                                     hgf.make_params(degree=2, r=9, eps=1e-4), lab)
                st, rid = hgf.hgf_serve_submit(srv, r)
                assert st == hgf.HGF_OK
                assert hgf.hgf_serve_wait(srv, rid, 60000) == hgf.HGF_OK
                assert np.array_equal(lab.cpu().numpy(), rl)
        s = hgf.hgf_serve_stats(srv)
        assert s["evictions"] >= 3
        assert s["peak_bytes"] <= s["budget_bytes"]
    finally:
        hgf.hgf_serve_destroy(srv)


def test_degree_aware_admission_and_breakdown():
    """With two slots, requests with n = 19 hold one slot at most: a request with n = 3 queued
    behind three n = 19 requests starts in the other slot at once and completes while the second
    n = 19 request has not started. The statistics split each completed request's time into the
    queue wait and its device time (precompute on a cache miss, aggregation), by guidance size."""
    torch = torch_cuda()
    from paper_1803_00005_gb300 import build, hgf
    build.build()
    big = [dict(w=640, h=480, L=64, seed=700 + i, degree=3, r=4, key=70 + i) for i in range(3)]
    small = [dict(w=160, h=120, L=8, seed=710, degree=1, r=4, key=80)]
    items = make_inputs(torch, big + small)
    srv = hgf.hgf_serve_create(0, budget_bytes=16 << 30, slots=2, max_queue=16,
                               max_pixels=640 * 480, max_n=19)
    try:
        ids = []
        for it in items:
            lab = torch.empty((it["h"], it["w"]), dtype=torch.int32, device="cuda")
            it["lab"] = lab
            req = hgf.make_request(it["key"], it["img"], it["cost"],
                                   hgf.make_params(degree=it["degree"], r=it["r"], eps=1e-4), lab)
            st, rid = hgf.hgf_serve_submit(srv, req)
            assert st == hgf.HGF_OK
            ids.append(rid)
        assert hgf.hgf_serve_wait(srv, ids[3], 60000) == hgf.HGF_OK
        assert hgf.hgf_serve_poll(srv, ids[1]) == hgf.HGF_EAGAIN   # waits for the n = 19 slot
        for rid in ids:
            assert hgf.hgf_serve_wait(srv, rid, 60000) == hgf.HGF_OK
        s = hgf.hgf_serve_stats(srv)
        assert s["completed"] == 4
        assert list(s["completed_by_class"]) == [1, 0, 3]
        assert s["prepare_ms_total"][2] > 0 and s["aggregate_ms_total"][2] > 0
        assert s["aggregate_ms_total"][0] > 0
        assert s["queue_p99_ms"] >= s["queue_mean_ms"] >= 0
        assert s["max_concurrent"] == 2
    finally:
        hgf.hgf_serve_destroy(srv)
