"""Parity at full workload sizes, in the configuration the benchmark times.

The whole frame is rendered on the GPU; the FP64 oracle computes a seeded sample of pixels
one by one (every splat projected, every contributor of each sampled pixel blended).  The
gradient check restricts the L1 loss to the sampled pixels so that the oracle's adjoint
stays cheap, and compares every parameter tensor by relative L2 error.
"""
import numpy as np
import pytest
import torch

from _helpers import FWD_FLAGS, GRAD_FLAGS, GRAD_RTOL, MAX_FLAGGED, PIXEL_TOL, image_at, oracle_opts, rel_l2
from oracle import oracle as O
from paper_2406_11836_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    return rgs


def _fullsize(R, wl, cam, n_fwd, n_grad):
    from paper_2406_11836_gb300.render import Trainer
    tr = Trainer(wl.scene, wl.depth_L)               # the benchmark's parameter layout and path
    g = tr.gaussians()
    out = R.render_fwd(tr.kd, g, cam, tr.opts, tr.ws)
    torch.cuda.synchronize()
    host = wl.scene.to("cpu")
    H, Wd = cam.height, cam.width
    # forward on sampled pixels
    pix = W.sample_pixels(Wd, H, n_fwd, seed=17)
    ref = O.render(host, cam, oracle_opts(), pix=pix)
    ok = (ref["flags"] & FWD_FLAGS) == 0
    assert ok.mean() >= 1 - MAX_FLAGGED, ok.mean()
    err = np.abs(image_at(out["image"], pix) - ref["C"])[ok].max()
    assert err <= PIXEL_TOL, err
    assert (ref["ncontrib"] > 0).mean() > 0.5
    # gradients of an L1 loss restricted to sampled pixels
    gpix = pix[:n_grad]
    gref = O.render(host, cam, oracle_opts(), pix=gpix)
    keep = gpix[(gref["flags"] & GRAD_FLAGS) == 0]
    target = W.target_image(Wd, H, seed=3, device="cuda")
    mask = torch.zeros(H * Wd, device="cuda")
    mask[torch.as_tensor(keep, device="cuda")] = 1.0
    mask = mask.view(1, H, Wd)
    dL = torch.sign(out["image"] - target) * mask / float(len(keep))
    R.render_bwd(tr.kd, g, cam, tr.opts, out["partial_C"], out["partial_T"], dL, tr.grads(), tr.ws,
                 tile_depth=out["tile_depth"])
    torch.cuda.synchronize()
    dLdC = dL.reshape(3, -1)[:, torch.as_tensor(keep, device="cuda")].T.double().cpu().numpy()
    adj = O.adjoint(host, cam, dLdC, oracle_opts(), pix=keep)
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    for name, got in zip(names, tr.grads()):
        e = rel_l2(got.double().cpu().numpy().reshape(adj[name].shape), adj[name])
        assert np.abs(adj[name]).max() > 0, name
        assert e <= GRAD_RTOL, (name, e)


def test_fullsize_object_1m_1600x1060_k8(R):
    wl = W.object_1m(device="cuda")
    _fullsize(R, wl, wl.cameras[0], n_fwd=4096, n_grad=1024)


def test_fullsize_city_10m_3840x2160_k16(R):
    wl = W.city_10m(device="cuda")
    _fullsize(R, wl, wl.cameras[3], n_fwd=1024, n_grad=256)
