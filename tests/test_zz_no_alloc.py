"""rgs_render_fwd_noalloc: the forward render for callers that cannot allocate device
memory (for example a real-time thread that must not block in the allocator, or a host
program that hands out all device memory from its own pool).  It must give the same
partial maps, image and depth table as rgs_render_fwd, on consecutive calls that reuse
its fixed scratch array, and refuse a render that does not fit that array, before or
after binning, leaving the next render correct.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2406_11836_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the pixel tolerance of the parity tests (the outputs are in fact bit-identical)


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    lib = rgs.lib()
    lib.rgs_render_fwd_noalloc.argtypes = [ctypes.c_void_p, ctypes.POINTER(rgs.Gaussians), ctypes.POINTER(rgs.CameraC),
                                           ctypes.POINTER(rgs.RenderOpts)] + [ctypes.c_void_p] * 6
    return rgs


def _noalloc(R, kd, g, cam, opts):
    H, Wd = cam.height, cam.width
    tiles = ((H + 15) // 16) * ((Wd + 15) // 16)
    out = {"partial_C": torch.full((kd.K, 3, H, Wd), float("nan"), device="cuda"),
           "partial_T": torch.full((kd.K, H, Wd), float("nan"), device="cuda"),
           "image": torch.full((3, H, Wd), float("nan"), device="cuda"),
           "T_final": torch.full((H, Wd), float("nan"), device="cuda"),
           "tile_depth": torch.full((tiles, kd.K), float("nan"), device="cuda")}
    c = R.camera_c(cam)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = R.lib().rgs_render_fwd_noalloc(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                        p(out["partial_C"]), p(out["partial_T"]), p(out["image"]), p(out["T_final"]),
                                        p(out["tile_depth"]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, out


def _small_scene(R):
    scene = W.uniform_cube_scene(6000, seed=61, log_scale_mean=-3.0, sh_degree=2)
    dev = scene.to("cuda")
    return R.kd_partition(dev, 2), R.scene_c(dev), dev


def _check_against_render_fwd(R, kd, g, cam, opts):
    rc, got = _noalloc(R, kd, g, cam, opts)
    assert rc == R.RGS_OK, R.lib().rgs_last_error()
    ref = R.render_fwd(kd, g, cam, opts, R.Workspace())
    torch.cuda.synchronize()
    for key in ("partial_C", "partial_T", "image", "T_final"):
        assert torch.isfinite(got[key]).all(), key
        assert (got[key] - ref[key]).abs().max().item() <= TOL, key
    assert torch.equal(got["tile_depth"], ref["tile_depth"])


def test_noalloc_matches_render_fwd_on_consecutive_calls(R):
    kd, g, _dev = _small_scene(R)
    opts = R.default_opts()
    cams = [W.look_at((0.3, -2.7, 0.4), (0, 0, 0), 120, 90), W.look_at((-1.5, 1.8, 1.2), (0.1, 0, 0), 100, 75)]
    for cam in cams:                                  # two calls in a row share the scratch array
        _check_against_render_fwd(R, kd, g, cam, opts)


def test_noalloc_rejects_a_render_beyond_its_scratch(R):
    """Before binning: the splats alone do not fit the array."""
    scene = W.uniform_cube_scene(600_000, seed=62, log_scale_mean=-3.0)
    dev = scene.to("cuda")
    kd = R.kd_partition(dev, 1)
    rc, _ = _noalloc(R, kd, R.scene_c(dev), W.axis_camera((0.0, 0.0, -3.0), 64, 64), R.default_opts())
    assert rc == R.RGS_EOVERFLOW
    err = R.lib().rgs_last_error()
    assert b"fixed scratch" in err and b"before binning" in err, err
    assert R.lib().rgs_last_required_workspace() > 64 << 20


def test_noalloc_rejects_too_many_instances_then_renders_correctly(R):
    """After binning: the splats fit, their tile instances do not.  The refused call has
    already projected into the shared array; the next call must not see its leftovers."""
    big = W.uniform_cube_scene(100_000, seed=63, log_scale_mean=-1.0)
    bdev = big.to("cuda")
    bkd = R.kd_partition(bdev, 1)
    rc, _ = _noalloc(R, bkd, R.scene_c(bdev), W.axis_camera((0.0, 0.0, -3.0), 1024, 1024), R.default_opts())
    assert rc == R.RGS_EOVERFLOW
    err = R.lib().rgs_last_error()
    assert b"fixed scratch" in err and b"tile instances" in err, err
    assert R.lib().rgs_last_required_workspace() > 64 << 20
    kd, g, _dev = _small_scene(R)
    _check_against_render_fwd(R, kd, g, W.look_at((0.3, -2.7, 0.4), (0, 0, 0), 120, 90), R.default_opts())
