"""Parity at full workload sizes, in the configuration the benchmark times.

The whole frame is rendered on the GPU; the FP64 oracle computes a seeded sample of pixels
one by one (every splat projected, every contributor of each sampled pixel blended).  The
gradient check restricts the L1 loss to the sampled pixels so that the oracle's adjoint
stays cheap, and compares every parameter tensor by relative L2 error.
"""
import numpy as np
import pytest
import torch

from _helpers import GRAD_RTOL, assert_all_close, image_at, oracle_opts, rel_l2
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


def _relevant(scene, cam, pix, trunc_mult=3.0, chunk=10_000_000):
    """Indices of the splats that can contribute to a sampled pixel.  By the ball test of the
    truncation rule (|x_i - mu_i| <= D_i, x_i on the pixel ray at depth z_i) a contributor's
    projected centre lies within f D_i / z_i of the pixel centre; splats whose disc of that
    radius (plus 1% and 2 px) holds no sampled pixel, or that lie behind half the near
    plane, cannot contribute and cannot be flagged, so the oracle may skip them."""
    dev = scene.means.device
    H, Wd = cam.height, cam.width
    V = torch.tensor(np.asarray(cam.viewmat, np.float64), device=dev)
    Rm, t = V[:3, :3], V[:3, 3]
    ind = torch.zeros(H + 1, Wd + 1, dtype=torch.int64, device=dev)
    pt = torch.as_tensor(pix, device=dev)
    ind[pt // Wd + 1, pt % Wd + 1] = 1
    S = ind.cumsum(0).cumsum(1)
    f = float(max(cam.fx, cam.fy))
    keep = []
    for c0 in range(0, scene.n, chunk):
        mu = scene.means[c0:c0 + chunk].double()
        p = mu @ Rm.T + t
        z = p[:, 2]
        D = trunc_mult * torch.exp(scene.log_scales[c0:c0 + chunk].double().amax(dim=1))
        zc = z.clamp(min=1e-9)
        u = cam.fx * p[:, 0] / zc + cam.cx
        v = cam.fy * p[:, 1] / zc + cam.cy
        r = f * D / zc * 1.01 + 2.0
        x0 = torch.ceil(u - r - 0.5).clamp(0, Wd - 1).long()
        x1 = torch.floor(u + r - 0.5).clamp(-1, Wd - 1).long()
        y0 = torch.ceil(v - r - 0.5).clamp(0, H - 1).long()
        y1 = torch.floor(v + r - 0.5).clamp(-1, H - 1).long()
        ok = (z > 0.5 * cam.near_z) & (x0 <= x1) & (y0 <= y1)
        x1c, y1c = x1.clamp(min=0), y1.clamp(min=0)
        cnt = S[y1c + 1, x1c + 1] - S[y0, x1c + 1] - S[y1c + 1, x0] + S[y0, x0]
        keep.append(torch.nonzero(ok & (cnt > 0)).squeeze(1) + c0)
    return torch.cat(keep)


def _fullsize(R, wl, cam, n_fwd, n_grad, prefilter=False):
    from paper_2406_11836_gb300.render import Trainer
    tr = Trainer(wl.scene, wl.depth_L)               # the benchmark's parameter layout and path
    g = tr.gaussians()
    out = R.render_fwd(tr.kd, g, cam, tr.opts, tr.ws)
    torch.cuda.synchronize()
    H, Wd = cam.height, cam.width
    pix = W.sample_pixels(Wd, H, n_fwd, seed=17)
    if prefilter:
        idx = _relevant(wl.scene, cam, pix)
        host = W.Scene(*(t[idx].cpu() for t in wl.scene.tensors()), wl.scene.sh_degree)
    else:
        idx = None
        host = wl.scene.to("cpu")
    # forward on sampled pixels
    ref = O.render(host, cam, oracle_opts(), pix=pix)
    assert_all_close(image_at(out["image"], pix), ref["C"], ref["flags"], "image")
    assert (ref["ncontrib"] > 0).mean() > 0.5
    # gradients of an L1 loss restricted to sampled pixels (none left out as ambiguous)
    keep = pix[:n_grad]
    target = W.target_image(Wd, H, seed=3, device="cuda")
    mask = torch.zeros(H * Wd, device="cuda")
    mask[torch.as_tensor(keep, device="cuda")] = 1.0
    mask = mask.view(1, H, Wd)
    dL = torch.sign(out["image"] - target) * mask / float(len(keep))
    dLdC = dL.reshape(3, -1)[:, torch.as_tensor(keep, device="cuda")].T.double().cpu().numpy()
    adj = O.adjoint(host, cam, dLdC, oracle_opts(), pix=keep)
    # both backward forms against the same adjoint: the per-subset form from this forward's
    # partial maps, the flat form (the trainer's step) after an image-only forward
    R.render_bwd(tr.kd, g, cam, tr.opts, out["partial_C"], out["partial_T"], dL, tr.grads(), tr.ws,
                 tile_depth=out["tile_depth"])
    torch.cuda.synchronize()
    _check_grads(tr.grads(), adj, idx, "subsets")
    for t in tr.grads():
        t.zero_()
    img = R.render_fwd(tr.kd, g, cam, tr.opts, tr.ws, partials=False)
    R.render_bwd_flat(tr.kd, g, cam, tr.opts, img["image"], dL, tr.grads(), tr.ws, tile_depth=img["tile_depth"])
    torch.cuda.synchronize()
    assert_all_close(image_at(img["image"], pix), ref["C"], ref["flags"], "image-only forward")
    _check_grads(tr.grads(), adj, idx, "flat")


def _check_grads(grads, adj, idx, form):
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    for name, got in zip(names, grads):
        assert np.abs(adj[name]).max() > 0, name
        if idx is None:
            e = rel_l2(got.double().cpu().numpy().reshape(adj[name].shape), adj[name])
        else:
            # oracle gradients are zero outside the relevant splats: compare the subset and
            # count every other GPU gradient as error
            gs = got[idx].double().cpu().numpy().reshape(adj[name].shape)
            tot = sum(float(got[c:c + 10_000_000].double().pow(2).sum()) for c in range(0, got.shape[0], 10_000_000))
            rest = max(tot - float((gs ** 2).sum()), 0.0)
            e = np.sqrt(float(((gs - adj[name]) ** 2).sum()) + rest) / max(np.linalg.norm(adj[name]), 1e-30)
        assert e <= GRAD_RTOL, (form, name, e)


def test_fullsize_object_1m_1600x1060_k8(R):
    wl = W.object_1m(device="cuda")
    _fullsize(R, wl, wl.cameras[0], n_fwd=4096, n_grad=1024)


def test_fullsize_city_10m_3840x2160_k16(R):
    wl = W.city_10m(device="cuda")
    _fullsize(R, wl, wl.cameras[3], n_fwd=1024, n_grad=256)


def test_fullsize_city_100m_3840x2160_k64(R):
    # 100M splats, params + grads + Adam state ~94 GB; the oracle samples 64 pixels
    wl = W.city_100m(device="cuda")
    _fullsize(R, wl, wl.cameras[0], n_fwd=256, n_grad=64, prefilter=True)
