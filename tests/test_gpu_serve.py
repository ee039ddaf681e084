"""Serving: batched graph path vs single renders, oracle parity, admission and failures.

A request's image must be the same alone and in a mixed batch (the batch kernels never mix
requests), equal to rgs_render_fwd's image of the same view, and within the pixel
tolerance of the FP64 oracle.  Host-side failures (oversized requests, overflowing
batches, destroy with pending work) are made on the host; nothing here faults a GPU.
"""
import numpy as np
import pytest
import torch

from _helpers import assert_all_close, image_at, oracle_opts
from oracle import oracle as O
from paper_2406_11836_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = ((320, 240), (200, 150), (640, 480), (97, 61), (480, 272), (256, 256))


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    return rgs


@pytest.fixture(scope="module")
def scene(R):
    wl = W.serving_5m(device="cuda", n=200_000)
    g = R.scene_c(wl.scene)
    kd = R.kd_partition(wl.scene, wl.depth_L)
    rng = np.random.default_rng(3)
    cams = []
    for i, (w, h) in enumerate(SIZES):
        v = rng.normal(size=3)
        v[2] = abs(v[2]) + 0.2
        v /= np.linalg.norm(v)
        cams.append(W.look_at(10.0 * v, (0, 0, 0), w, h))
    return wl, g, kd, cams


def _serve(R, scene, cams, together=True, **kw):
    """Serve `cams`; with together=True all are queued before the scheduler may start a
    batch (rgs_serve_hold), so the batching does not depend on host timing."""
    wl, g, kd, _ = scene
    srv = R.Server(kd, g, R.default_opts(), keepalive=wl.scene, **kw)
    outs = [torch.full((3, c.height, c.width), -1.0, device="cuda") for c in cams]
    try:
        if together:
            srv.hold(True)
        tickets = [srv.submit(c, o) for c, o in zip(cams, outs)]
        srv.hold(False)
        lat = [srv.wait(t, timeout_s=120) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    torch.cuda.synchronize()
    return outs, lat, st


def _alone(R, scene, cam):
    outs, _, st = _serve(R, scene, [cam], mem_budget_bytes=2 << 30, max_slots=1, lanes=1)
    assert st["completed"] == 1 and st["batches"] == 1
    return outs[0]


def test_alone_equals_mix_and_render_fwd(R, scene):
    wl, g, kd, cams = scene
    alone = [_alone(R, scene, c) for c in cams]
    mix, lat, st = _serve(R, scene, cams, mem_budget_bytes=4 << 30, max_slots=8, lanes=1)
    assert st["completed"] == len(cams) and st["failed"] == 0
    assert st["mean_batch"] > 1.0                      # the requests shared batches
    ws = R.Workspace()
    opts = R.default_opts()
    for c, a, m in zip(cams, alone, mix):
        assert torch.equal(a, m), (c.width, c.height)     # bit-identical alone and in the mix
        ref = R.render_fwd(kd, g, c, opts, ws, partials=False)["image"]
        torch.cuda.synchronize()
        assert torch.equal(ref, m), (c.width, c.height, (ref - m).abs().max().item())
        assert (m >= 0).all()                              # every pixel written
    assert all(x > 0 for x in lat)


def test_served_images_match_oracle(R, scene):
    wl, g, kd, cams = scene
    outs, _, _ = _serve(R, scene, cams[:3], mem_budget_bytes=4 << 30, max_slots=4, lanes=2)
    host = wl.scene.to("cpu")
    for c, img in zip(cams[:3], outs):
        pix = W.sample_pixels(c.width, c.height, 512, seed=23)
        ref = O.render(host, c, oracle_opts(), pix=pix)
        assert_all_close(image_at(img, pix), ref["C"], ref["flags"], f"served {c.width}x{c.height}")


def test_plain_mode_matches(R, scene):
    wl, g, kd, cams = scene
    mix, _, _ = _serve(R, scene, cams, mem_budget_bytes=4 << 30, max_slots=8, lanes=2)
    plain, _, st = _serve(R, scene, cams, mem_budget_bytes=1 << 30, plain=True, max_width=1024, max_height=1024)
    assert st["completed"] == len(cams) and st["mean_batch"] == 1.0
    for a, b in zip(mix, plain):
        assert torch.equal(a, b)


def _render_counts(R, kd, g, cam):
    """(tile instances, visible splats) of one render of cam binned in one group."""
    ws = R.Workspace()
    R.profile_enable(timing=False, counters=True)
    try:
        R.profile_read(reset=True)
        R.render_fwd(kd, g, cam, R.default_opts(group_binning=0), ws, partials=False)
        torch.cuda.synchronize()
        c = R.profile_read(reset=True)["counters"]
        return c["instances"], c["visible"]
    finally:
        R.profile_enable(timing=False, counters=False)


def test_grouped_batches_match_render_fwd(R, scene):
    """Requests that bin their subsets in two groups of view ranks (the nearest first, the
    rest only in the tiles the first left open) give rgs_render_fwd's image bit for bit,
    in batches of grouped requests only and in batches that mix grouped and one-group
    requests (the server groups a resolution once its measured instances per visible
    splat reach group_per_splat)."""
    wl, g, kd, cams = scene
    assert kd.K >= 4
    ws = R.Workspace()
    refs = []
    for c in cams:
        refs.append(R.render_fwd(kd, g, c, R.default_opts(), ws, partials=False)["image"].clone())
    torch.cuda.synchronize()
    outs, _, st = _serve(R, scene, cams, mem_budget_bytes=4 << 30, max_slots=8, lanes=1, group_per_splat=0.0,
                         group_min_instances=0.0)
    assert st["completed"] == len(cams) and st["failed"] == 0 and st["mean_batch"] > 1.0
    for c, r, o in zip(cams, refs, outs):
        assert torch.equal(r, o), (c.width, c.height, (r - o).abs().max().item())
    # a threshold between the views' ratios: the second batch mixes both kinds of request
    ratios = []
    for c in cams:
        inst, vis = _render_counts(R, kd, g, c)
        ratios.append(inst / vis)
    thr = sorted(ratios)[len(ratios) // 2]
    n_grouped = sum(r >= thr for r in ratios)
    assert 0 < n_grouped < len(cams)
    srv = R.Server(kd, g, R.default_opts(), 4 << 30, max_slots=8, lanes=1, group_per_splat=float(thr),
                   group_min_instances=0.0, keepalive=wl.scene)
    try:
        for rnd in range(2):     # the first batch measures, the second groups by the measure
            outs = [torch.full((3, c.height, c.width), -1.0, device="cuda") for c in cams]
            srv.hold(True)
            ts = [srv.submit(c, o) for c, o in zip(cams, outs)]
            srv.hold(False)
            for t in ts:
                srv.wait(t, timeout_s=120)
            torch.cuda.synchronize()
            for c, r, o in zip(cams, refs, outs):
                assert torch.equal(r, o), (rnd, c.width, c.height)
    finally:
        srv.close()


def _instances(R, kd, g, cam):
    """Tile instances of one render of cam (the library's tracing counters), binned in one
    group as the batch path bins them."""
    ws = R.Workspace()
    R.profile_enable(timing=False, counters=True)
    try:
        R.profile_read(reset=True)
        R.render_fwd(kd, g, cam, R.default_opts(group_binning=0), ws, partials=False)
        torch.cuda.synchronize()
        return R.profile_read(reset=True)["counters"]["instances"]
    finally:
        R.profile_enable(timing=False, counters=False)


def test_overflowing_batch_is_requeued(R, scene):
    wl, g, kd, cams = scene
    cam = cams[2]                                       # 640x480
    alone = _alone(R, scene, cam)
    inst = _instances(R, kd, g, cam)
    assert inst > 0
    # one lane holds 2.5 requests; a low first estimate admits all 4, the batch overflows
    # and is re-run with the exact sizes
    kw = dict(max_slots=4, max_width=640, max_height=480)
    cap = max(int(2.5 * inst), 1 << 16)
    assert 4 * inst > cap
    budget = R.serve_lane_bytes(kd, g, cap, **kw)
    outs, _, st = _serve(R, scene, [cam] * 4, mem_budget_bytes=budget, lanes=1, inst_per_pixel=0.01, **kw)
    assert st["completed"] == 4 and st["failed"] == 0
    assert st["requeued"] >= 1 and st["batches"] >= 2
    assert st["instance_capacity"] <= cap
    for o in outs:
        assert torch.equal(o, alone)


def test_request_larger_than_a_lane_fails_cleanly(R, scene):
    wl, g, kd, cams = scene
    big, small = cams[2], cams[3]                       # 640x480, 97x61
    ib, i_s = _instances(R, kd, g, big), _instances(R, kd, g, small)
    assert i_s < ib
    kw = dict(max_slots=2, max_width=640, max_height=480)
    cap = max((ib + i_s) // 2, 1 << 16)
    if cap >= ib:
        pytest.skip("the large view does not exceed the smallest lane")
    srv = R.Server(kd, g, R.default_opts(), R.serve_lane_bytes(kd, g, cap, **kw), lanes=1, keepalive=wl.scene, **kw)
    try:
        t = srv.submit(big, torch.empty(3, 480, 640, device="cuda"))
        with pytest.raises(R.RGSError) as ei:
            srv.wait(t, timeout_s=60)
        assert ei.value.code == R.RGS_EOVERFLOW
        # the server keeps serving requests that fit
        out = torch.empty(3, 61, 97, device="cuda")
        srv.wait(srv.submit(small, out), timeout_s=60)
        torch.cuda.synchronize()
        assert torch.equal(out, _alone(R, scene, small))
    finally:
        srv.close()


def test_submit_validation_and_destroy_with_pending(R, scene):
    wl, g, kd, cams = scene
    srv = R.Server(kd, g, R.default_opts(), 2 << 30, max_slots=4, lanes=2, max_width=640, max_height=480,
                   keepalive=wl.scene)
    too_big = W.look_at((10.0, 0.0, 5.0), (0, 0, 0), 800, 600)
    with pytest.raises(R.RGSError) as ei:
        srv.submit(too_big, torch.empty(3, 600, 800, device="cuda"))
    assert ei.value.code == R.RGS_EINVAL
    with pytest.raises(R.RGSError) as ei:
        srv.poll(123456789)
    assert ei.value.code == R.RGS_EINVAL
    outs = [torch.empty(3, c.height, c.width, device="cuda") for c in cams[:4]] * 8
    for c, o in zip(cams[:4] * 8, outs):
        srv.submit(c, o)
    srv.close()          # cancels what is queued, waits (bounded) for what runs
    torch.cuda.synchronize()


def test_edge_sizes_and_a_single_subset_scene(R):
    """1x1 and odd-sized requests, and a scene with one KD subset (K = 1), through the
    batched server: each equal to rgs_render_fwd's image of the same view."""
    wl = W.serving_5m(device="cuda", n=30_000)
    g = R.scene_c(wl.scene)
    for L in (0, 2):
        kd = R.kd_partition(wl.scene, L)
        cams = [W.look_at((6.0, -5.0, 4.0), (0, 0, 0), w, h) for (w, h) in ((1, 1), (17, 9), (33, 65), (16, 16))]
        srv = R.Server(kd, g, R.default_opts(), 2 << 30, max_slots=4, lanes=1, max_width=64, max_height=128,
                       keepalive=wl.scene)
        outs = [torch.full((3, c.height, c.width), -1.0, device="cuda") for c in cams]
        try:
            srv.hold(True)
            ts = [srv.submit(c, o) for c, o in zip(cams, outs)]
            srv.hold(False)
            for t in ts:
                srv.wait(t, timeout_s=60)
        finally:
            srv.close()
        torch.cuda.synchronize()
        ws = R.Workspace()
        for c, o in zip(cams, outs):
            ref = R.render_fwd(kd, g, c, R.default_opts(), ws, partials=False)["image"]
            torch.cuda.synchronize()
            assert torch.equal(ref, o), (L, c.width, c.height)
