"""GPU parity of the perpendicular-foot reading of x_i (Sec. 3.2, comparison mode).

rgs_render_fwd_foot against the FP64 oracle with opts.foot: the image against the flat
form (contributors of each ray ordered by the foot's ray parameter), the partial maps
against the literal Eq. 3-4 with the indicator of Eq. 6 at the foot.  rgs_render_bwd_foot
against the oracle's adjoint under the same reading (every sampled pixel in the loss).  The per-pixel order
buffer must not overflow on these scenes (the order is then exact), and the two readings
must really differ on each scene.

Margins: the GPU orders a pixel's contributors by s = z (fx^2 + a b + k c d), fx^2 |r_p|
times the ray parameter t, carried as a float pair from the projection's float-pair depth
and centre (a = X - cx and, for square pixels, k c = Y - cy exact), so each key is good to
about 1e-12 of its size; the oracle flags adjacent ray parameters closer than 1e-9 of
max(|R_z u_i| + |t_z|, |u_i - o|) (at least t).  The ball and plane tests at the foot run
in fp32 with errors near 1e-6 of their thresholds; they keep the depth-plane margin of
3e-6.
"""
import numpy as np
import pytest
import torch

from _helpers import (FWD_FLAGS, GRAD_RTOL, MAX_FLAGGED, PART_FLAGS, PART_MAX_FLAGGED, PIXEL_TOL, image_at,
                      oracle_opts, partials_at, rel_l2)
from oracle import oracle as O
from paper_2406_11836_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FOOT_FLAG_REL = 3e-6
FOOT_DEPTH_REL = 1e-9


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    return rgs


def foot_opts(opts=None, eps_T=0.0):
    o = oracle_opts(opts, eps_T)
    o.foot = True
    o.flag_rel = FOOT_FLAG_REL
    o.flag_depth_rel = FOOT_DEPTH_REL
    return o


def _check_foot(R, scene, cam, L, pix=None, opts=None, partials=True, differ=True, max_flagged=MAX_FLAGGED,
                part_cap=PART_MAX_FLAGGED):
    dev = scene.to("cuda")
    kd = R.kd_partition(dev, L)
    opts = opts if opts is not None else R.default_opts()
    g = R.scene_c(dev)
    out = R.render_fwd_foot(kd, g, cam, opts, R.Workspace(), partials=partials)
    torch.cuda.synchronize()
    assert out["overflow"] == 0
    pix = np.arange(cam.width * cam.height) if pix is None else pix
    flat = O.render(scene, cam, foot_opts(opts), pix=pix)
    # the foot's order key is a float pair good to ~1e-12 and its ball test differs from the
    # depth plane's: pixels the oracle flags as ambiguous are left out (at most 0.1%)
    ok = (flat["flags"] & FWD_FLAGS) == 0
    assert ok.mean() >= 1 - max_flagged, ok.mean()
    err = np.abs(image_at(out["image"], pix) - flat["C"])[ok].max()
    assert err <= PIXEL_TOL, err
    if partials:
        terr = np.abs(out["T_final"].reshape(-1).double().cpu().numpy()[pix] - flat["T"])[ok].max()
        assert terr <= PIXEL_TOL, terr
        axis, split = kd.splits()
        hier = O.render(scene, cam, foot_opts(opts, eps_T=float(np.float32(1e-6))), pix=pix, hier=True, L=L,
                        axis=axis, split=split)
        okp = (hier["flags"] & PART_FLAGS) == 0
        assert okp.mean() >= 1 - part_cap, okp.mean()
        pc, pt = partials_at(out["partial_C"], out["partial_T"], pix)
        perr = max(np.abs(pc - hier["partC"])[okp].max(), np.abs(pt - hier["partT"])[okp].max())
        assert perr <= PIXEL_TOL, perr
    if differ:
        # the depth-plane render of the same scene differs somewhere
        plane = R.render_fwd(kd, g, cam, opts, R.Workspace(), partials=False)["image"]
        torch.cuda.synchronize()
        assert float((plane - out["image"]).abs().max()) > 1e-3
    return kd, out, flat


def test_foot_tiny_full_image(R):
    """4,096 splats, 128x128, K = 2: every pixel, image and partial maps."""
    wl = W.tiny()
    _, _, flat = _check_foot(R, wl.scene, wl.cameras[0], wl.depth_L)
    assert (flat["ncontrib"] > 0).mean() > 0.3


@pytest.mark.parametrize("L", [0, 2, 3, 6])
def test_foot_partition_depths_and_ragged_image(R, L):
    """A camera inside the scene (rays cross many subspaces), 100x70 (ragged tiles), SH
    degree 3, from 1 to 64 subsets."""
    scene = W.uniform_cube_scene(3000, seed=7 + L, log_scale_mean=-3.2, sh_degree=3)
    cam = W.look_at((0.15, -0.2, 0.1), (0.3, 1.0, -0.2), 100, 70)
    _check_foot(R, scene, cam, L)


def test_foot_reorders_splats_in_thin_slabs(R):
    """Three thin slabs of splats facing the camera (depth jitter 0.01): inside a slab the
    lateral offsets decide the foot order, which differs from the depth order on most
    pixels and crowds each pixel's ray parameters into three narrow bands."""
    g = torch.Generator().manual_seed(5)
    n = 6000
    means = torch.rand(n, 3, generator=g) * 2 - 1
    slab = torch.tensor([-0.4, 0.0, 0.4])[torch.randint(0, 3, (n,), generator=g)]
    means[:, 2] = slab + 0.01 * torch.randn(n, generator=g)
    log_scales = torch.randn(n, 3, generator=g) * 0.3 - 3.4
    q = torch.randn(n, 4, generator=g)
    scene = W.Scene(means, log_scales, q / q.norm(dim=1, keepdim=True), torch.randn(n, generator=g),
                    torch.rand(n, 1, 3, generator=g), 0)
    cam = W.axis_camera((0.1, -0.05, -3.0), 640, 480)
    _check_foot(R, scene, cam, 2)


def test_foot_image_only_and_background(R):
    """Forward-only render (no partial maps) with a background colour; the merge stops at
    negligible front transmittance, which moves a pixel by less than 1e-6."""
    opts = R.default_opts(bg=(0.2, 0.4, 0.6))
    wl = W.tiny()
    _check_foot(R, wl.scene, wl.cameras[0], 3, opts=opts, partials=False)


def test_foot_edge_cases(R):
    opts = R.default_opts(bg=(0.25, 0.5, 0.75))
    # every splat behind the camera
    scene = W.uniform_cube_scene(100, seed=1)
    dev = scene.to("cuda")
    kd = R.kd_partition(dev, 2)
    out = R.render_fwd_foot(kd, R.scene_c(dev), W.axis_camera((0.0, 0.0, 5.0), 33, 17), opts, R.Workspace())
    torch.cuda.synchronize()
    img = out["image"].cpu().numpy()
    for c, v in enumerate((0.25, 0.5, 0.75)):
        assert np.all(img[c] == np.float32(v))
    assert np.all(out["partial_C"].cpu().numpy() == 0) and np.all(out["partial_T"].cpu().numpy() == 1)
    # a single splat, 1x1 image; an image smaller than one tile with straddling splats (a
    # 10 degree field: at 60 degrees each of the 7x5 pixels spans ~9 degrees, and the ray
    # parameters of a pixel's ~90 contributors interleave beyond what the order buffer holds)
    one = W.uniform_cube_scene(1, seed=2, log_scale_mean=-1.0)
    _check_foot(R, one, W.axis_camera((0.0, 0.0, -3.0), 1, 1), 0, opts=opts, differ=False)
    _check_foot(R, W.uniform_cube_scene(500, seed=5, log_scale_mean=-2.0),
                W.axis_camera((0.1, 0.0, -2.5), 7, 5, fov_x_deg=10.0), 3, differ=False, max_flagged=0.1,
                part_cap=1.0)   # 35 rays along a split plane: a few are at a plane or a threshold


def test_foot_rejects_missing_outputs(R):
    """Neither partial maps nor an image: EINVAL, nothing launched."""
    import ctypes
    wl = W.tiny()
    dev = wl.scene.to("cuda")
    kd = R.kd_partition(dev, 1)
    over = ctypes.c_uint64(0)
    rc = R.lib().rgs_render_fwd_foot(kd.handle, ctypes.byref(R.scene_c(dev)), ctypes.byref(R.camera_c(wl.cameras[0])),
                                     ctypes.byref(R.default_opts()), None, None, None, None, None, 0,
                                     ctypes.byref(over), None)
    assert rc == R.RGS_EINVAL


@pytest.mark.parametrize("name,view,n_pix,max_flagged,max_over,cull", [("object_1m", 0, 4096, MAX_FLAGGED, 0.0, 0),
                                                                       ("city_10m", 3, 1024, 0.015, 0.1, 0),
                                                                       ("city_10m", 3, 1024, 0.015, 0.0, 1)])
def test_foot_fullsize_sampled(R, name, view, n_pix, max_flagged, max_over, cull):
    """Full workload sizes in the benchmark's configuration (1M splats at 1600x1060 with
    8 subsets; 10M at 3840x2160 with 16): the whole frame on the GPU, a seeded sample of
    pixels in the oracle.  In the city view the foot's ball test, which accepts more rays
    than the depth plane's, leaves ~1.1% of the sampled pixels with a pair at a truncation
    threshold: up to 1.5% may be left out there.  The city's clusters put more than 64
    contributors within one bound window on some pixels: with every subset blended on every
    ray (cull = 0) the order buffer blends some contributors early there (counted; at most
    0.1 per pixel allowed), and the sampled pixels must still agree with the exact order to
    1e-4; with the training step's culling behind a saturated front (cull = 1) no
    contributor is blended early: the per-pixel order is exact at full size."""
    wl = getattr(W, name)(device="cuda")
    cam = wl.cameras[view]
    kd = R.kd_partition(wl.scene, wl.depth_L)
    g = R.scene_c(wl.scene)
    out = R.render_fwd_foot(kd, g, cam, R.default_opts(cull_occluded=cull), R.Workspace())
    torch.cuda.synchronize()
    pix = W.sample_pixels(cam.width, cam.height, n_pix, seed=23)
    ref = O.render(wl.scene.to("cpu"), cam, foot_opts(), pix=pix)
    ok = (ref["flags"] & FWD_FLAGS) == 0
    assert ok.mean() >= 1 - max_flagged, ok.mean()
    err = np.abs(image_at(out["image"], pix) - ref["C"])[ok].max()
    assert err <= PIXEL_TOL, err
    assert (ref["ncontrib"] > 0).mean() > 0.5
    assert out["overflow"] <= max_over * cam.width * cam.height, out["overflow"]


# --------------------------------------------------------------------------- backward
def _foot_grad_parity(R, scene, cam, L, opts=None, pix_loss=None, seed=1, differ=True):
    """L1 loss against a random target over the given pixels (none left out as ambiguous);
    dL/dC is formed from the GPU's foot-reading image and both sides get the same dL/dC.
    Per parameter tensor, the relative L2 error against the oracle's foot-reading adjoint
    must be at most GRAD_RTOL; with `differ`, the depth-plane adjoint of the same loss must
    be farther from it than that."""
    dev = scene.to("cuda")
    kd = R.kd_partition(dev, L)
    opts = opts if opts is not None else R.default_opts()
    g = R.scene_c(dev)
    ws = R.Workspace()
    img = R.render_fwd_foot(kd, g, cam, opts, ws, partials=False)["image"]
    H, Wd = cam.height, cam.width
    pix = np.arange(H * Wd) if pix_loss is None else np.asarray(pix_loss)
    target = W.target_image(Wd, H, seed=seed, device="cuda")
    mask = torch.zeros(H * Wd, device="cuda")
    mask[torch.as_tensor(pix, device="cuda")] = 1.0
    dL = (torch.sign(img - target) * mask.view(1, H, Wd) / float(len(pix))).contiguous()
    grads = [torch.zeros_like(t) for t in (dev.means, dev.log_scales, dev.quats, dev.opacity_logits, dev.sh)]
    over = R.render_bwd_foot(kd, g, cam, opts, img, dL, grads, ws)
    torch.cuda.synchronize()
    assert over == 0
    dLdC = dL.reshape(3, -1)[:, torch.as_tensor(pix, device="cuda")].T.double().cpu().numpy()
    host = scene.to("cpu")
    adj = O.adjoint(host, cam, dLdC, foot_opts(opts), pix=pix)
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    errs = {n: rel_l2(t.double().cpu().numpy(), adj[n]) for n, t in zip(names, grads)}
    for n in names:
        assert np.abs(adj[n]).max() > 0, n
        assert errs[n] <= GRAD_RTOL, errs
    if differ:
        plane = O.adjoint(host, cam, dLdC, oracle_opts(opts), pix=pix)
        assert rel_l2(plane["means"], adj["means"]) > 10 * GRAD_RTOL
    return errs


def test_foot_backward_tiny(R):
    """4,096 splats, 128x128, K = 2, every pixel in the loss."""
    wl = W.tiny()
    _foot_grad_parity(R, wl.scene, wl.cameras[0], wl.depth_L)


@pytest.mark.parametrize("L", [0, 3])
def test_foot_backward_inside_camera(R, L):
    """A camera inside the scene (rays cross many subspaces), 64x40 (ragged tiles), SH
    degree 3, a background colour."""
    scene = W.uniform_cube_scene(1500, seed=11 + L, log_scale_mean=-3.0, sh_degree=3)
    cam = W.look_at((0.1, -0.15, 0.05), (0.2, 1.0, 0.1), 64, 40)
    _foot_grad_parity(R, scene, cam, L, opts=R.default_opts(bg=(0.2, 0.4, 0.6)))


def test_foot_backward_thin_slabs(R):
    """The thin-slab scene, where the foot order differs from the depth order on most
    pixels: the gradients follow the foot's per-pixel order."""
    g = torch.Generator().manual_seed(5)
    n = 3000
    means = torch.rand(n, 3, generator=g) * 2 - 1
    slab = torch.tensor([-0.4, 0.0, 0.4])[torch.randint(0, 3, (n,), generator=g)]
    means[:, 2] = slab + 0.01 * torch.randn(n, generator=g)
    log_scales = torch.randn(n, 3, generator=g) * 0.3 - 3.0
    q = torch.randn(n, 4, generator=g)
    scene = W.Scene(means, log_scales, q / q.norm(dim=1, keepdim=True), torch.randn(n, generator=g),
                    torch.rand(n, 1, 3, generator=g), 0)
    cam = W.axis_camera((0.1, -0.05, -3.0), 160, 120)
    _foot_grad_parity(R, scene, cam, 2)


def test_foot_backward_object_1m_sampled(R):
    """The object workload at full size (1M splats, 1600x1060, K = 8): the loss on a
    seeded sample of pixels, the whole frame replayed on the GPU."""
    wl = W.object_1m(device="cuda")
    cam = wl.cameras[0]
    pix = W.sample_pixels(cam.width, cam.height, 1024, seed=29)
    _foot_grad_parity(R, wl.scene, cam, wl.depth_L, pix_loss=pix, differ=False)


def test_foot_backward_rejects_missing_image(R):
    """A NULL image: EINVAL, nothing launched."""
    import ctypes
    wl = W.tiny()
    dev = wl.scene.to("cuda")
    kd = R.kd_partition(dev, 1)
    grads = [torch.zeros_like(t) for t in (dev.means, dev.log_scales, dev.quats, dev.opacity_logits, dev.sh)]
    gg = R.GaussianGrads(*(ctypes.c_void_p(t.data_ptr()) for t in grads))
    dL = torch.zeros(3, 128, 128, device="cuda")
    rc = R.lib().rgs_render_bwd_foot(kd.handle, ctypes.byref(R.scene_c(dev)), ctypes.byref(R.camera_c(wl.cameras[0])),
                                     ctypes.byref(R.default_opts()), None, ctypes.c_void_p(dL.data_ptr()),
                                     ctypes.byref(gg), None, 0, None, None)
    assert rc == R.RGS_EINVAL
