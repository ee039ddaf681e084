"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every function
include/rgs.h declares, and rejects invalid arguments before any CUDA call."""
import ctypes
import math
import os
import re

import pytest

from paper_2406_11836_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    B.build()
    from paper_2406_11836_gb300 import rgs
    return rgs


def declared_functions():
    text = open(os.path.join(ROOT, "include", "rgs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rgs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(R):
    lib = R.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(R.ABI_SYMBOLS) <= set(names)


def test_defaults_and_version(R):
    o = R.default_opts()
    assert o.tile == 16 and o.trunc_mult == 3.0 and abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    assert abs(o.eps_T - 1e-6) < 1e-12 and abs(o.dilation - 0.3) < 1e-7
    assert R.lib().rgs_version() >= 100


def test_position_lr_closed_form(R):
    assert R.position_lr(0, 100) == pytest.approx(1.6e-4, rel=1e-6)
    assert R.position_lr(100, 100) == pytest.approx(1.6e-6, rel=1e-6)
    assert R.position_lr(50, 100) == pytest.approx(math.sqrt(1.6e-4 * 1.6e-6), rel=1e-6)


def test_invalid_arguments_are_rejected(R):
    lib = R.lib()
    out = ctypes.c_void_p()
    assert lib.rgs_kd_partition(None, 2, ctypes.c_float(3.0), ctypes.byref(out), None) == R.RGS_EINVAL
    assert b"kd_partition" in lib.rgs_last_error()
    fake = 1 << 20       # aligned non-NULL pointers; never dereferenced on these paths
    g = R.Gaussians(fake, fake, fake, fake, fake, 10, 5)   # sh_degree 5
    assert lib.rgs_kd_partition(ctypes.byref(g), 9, ctypes.c_float(3.0), ctypes.byref(out), None) == R.RGS_EINVAL
    g = R.Gaussians(fake, fake, fake, fake, fake, 10, 3)
    cam = R.CameraC()
    cam.width, cam.height, cam.fx, cam.fy, cam.near_z = 64, 64, 50.0, 50.0, 0.2
    cam.viewmat[0] = cam.viewmat[5] = cam.viewmat[10] = cam.viewmat[15] = 1.0
    opts = R.default_opts()
    nbytes = ctypes.c_size_t()
    # NULL kd handle
    assert lib.rgs_render_workspace_size(None, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), 0,
                                         ctypes.byref(nbytes)) == R.RGS_EINVAL
    # periodic Adam rule: its segment must exist, the period be positive
    offs = (ctypes.c_int64 * 3)(0, 8, 16)
    rates = (ctypes.c_float * 2)(1e-3, 1e-4)
    for pseg, period, head in ((2, 4, 1), (1, 0, 0), (1, 4, 5)):
        assert lib.rgs_adam_step_periodic(ctypes.c_void_p(fake), ctypes.c_void_p(fake), ctypes.c_void_p(fake),
                                          ctypes.c_void_p(fake), 16, offs, rates, 2, pseg, period, head,
                                          ctypes.c_float(1e-2), ctypes.c_float(0.9), ctypes.c_float(0.999),
                                          ctypes.c_float(1e-15), 1, 1, None) == R.RGS_EINVAL
    # foot-reading forward: no output at all, then a NULL kd handle
    over = ctypes.c_uint64()
    assert lib.rgs_render_fwd_foot(None, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), None, None, None,
                                   None, None, 0, ctypes.byref(over), None) == R.RGS_EINVAL
    assert lib.rgs_render_fwd_foot(None, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), None, None,
                                   ctypes.c_void_p(fake), None, ctypes.c_void_p(fake), 1 << 20, ctypes.byref(over),
                                   None) == R.RGS_EINVAL
    assert b"kd" in lib.rgs_last_error()
    # foot-reading backward: no image, then a NULL kd handle
    gg = R.GaussianGrads(fake, fake, fake, fake, fake)
    assert lib.rgs_render_bwd_foot(None, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), None,
                                   ctypes.c_void_p(fake), ctypes.byref(gg), None, 0, ctypes.byref(over),
                                   None) == R.RGS_EINVAL
    assert b"render_bwd_foot" in lib.rgs_last_error()
    assert lib.rgs_render_bwd_foot(None, ctypes.byref(g), ctypes.byref(cam), ctypes.byref(opts), ctypes.c_void_p(fake),
                                   ctypes.c_void_p(fake), ctypes.byref(gg), ctypes.c_void_p(fake), 1 << 20,
                                   ctypes.byref(over), None) == R.RGS_EINVAL
    assert b"kd" in lib.rgs_last_error()
    # view order needs a handle; merge needs buffers
    assert lib.rgs_merge_partials(None, None, None, 0, 1, 1, None, None, None, None) == R.RGS_EINVAL
    assert lib.rgs_adam_step(None, None, None, None, 0, None, None, 0, ctypes.c_float(0.9), ctypes.c_float(0.999),
                             ctypes.c_float(1e-15), 1, 1, None) == R.RGS_EINVAL


def test_missing_library_fails_loudly(R, monkeypatch):
    monkeypatch.setattr(R, "_lib", None)
    monkeypatch.setattr(R, "LIB_PATH", "/nonexistent/librgs.so")
    with pytest.raises(RuntimeError, match="missing"):
        R.lib()


def test_serving_arguments_are_rejected(R):
    lib = R.lib()
    cfg = R.ServeConfig()
    lib.rgs_serve_default_config(ctypes.byref(cfg))
    assert cfg.max_slots == 8 and cfg.lanes == 2 and cfg.plain == 0 and cfg.max_width == 4096
    out = ctypes.c_void_p()
    fake = 1 << 20
    g = R.Gaussians(fake, fake, fake, fake, fake, 10, 3)
    opts = R.default_opts()
    # NULL kd, NULL out: rejected before any CUDA call
    assert lib.rgs_serve_create_ex(None, ctypes.byref(g), ctypes.byref(opts), ctypes.byref(cfg),
                                   ctypes.byref(out)) == R.RGS_EINVAL
    assert lib.rgs_serve_create_ex(None, ctypes.byref(g), ctypes.byref(opts), ctypes.byref(cfg), None) == R.RGS_EINVAL
    cam = R.CameraC()
    t = ctypes.c_uint64()
    assert lib.rgs_serve_submit(None, ctypes.byref(cam), ctypes.c_void_p(fake), ctypes.byref(t)) == R.RGS_EINVAL
    done = ctypes.c_int()
    assert lib.rgs_serve_poll(None, 1, ctypes.byref(done), None) == R.RGS_EINVAL
    st = R.ServeStats()
    assert lib.rgs_serve_stats_read(None, ctypes.byref(st)) == R.RGS_EINVAL
    assert lib.rgs_serve_destroy(None) == R.RGS_OK
