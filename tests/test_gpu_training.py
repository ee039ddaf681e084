"""Training steps over one and several views (Sec. 3.4; batches of views as the paper's
larger batch sizes): a one-view batch is the one-view step, and a batch's gradient is the
mean of its views' gradients."""
import numpy as np
import pytest
import torch

from _helpers import rel_l2
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


def _trainer(R):
    from paper_2406_11836_gb300.render import Trainer
    scene = W.uniform_cube_scene(20_000, seed=9, log_scale_mean=-2.6, sh_degree=1).to("cuda")
    return Trainer(scene, 2, device="cuda")


def test_one_view_batch_is_the_one_view_step(R):
    cam = W.look_at((0.2, -2.6, 0.3), (0, 0, 0), 96, 64)
    target = torch.rand(3, 64, 96, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    a, b = _trainer(R), _trainer(R)
    la = a.step(cam, target)
    lb = b.step_batch([cam], [target])
    torch.cuda.synchronize()
    assert torch.equal(la, lb)
    # the 2D gradients are summed with atomics, so the first moments (0.1 g) agree to rounding
    assert rel_l2(a.m.double().cpu().numpy(), b.m.double().cpu().numpy()) <= 1e-5
    # Adam's first update is lr g / (|g| + eps): only where g itself is at the rounding level
    # of those sums may the two updates differ by more than rounding
    d = (a.flat - b.flat).abs()
    big = d > 1e-6
    assert bool((a.m[big].abs() <= 1e-6 * float(a.m.abs().max())).all())
    assert a.step_count == b.step_count == 1


def test_batch_gradient_is_the_mean_of_the_views(R):
    cams = [W.look_at((0.2, -2.6, 0.3), (0, 0, 0), 96, 64), W.look_at((2.5, 0.4, 0.9), (0, 0, 0), 80, 72)]
    gen = torch.Generator(device="cuda").manual_seed(2)
    targets = [torch.rand(3, c.height, c.width, device="cuda", generator=gen) for c in cams]
    tr = _trainer(R)
    g = tr.gaussians()
    per_view = []
    for c, t in zip(cams, targets):
        tr.grad.zero_()
        tr._accumulate(g, c, t, 1.0, False)
        per_view.append(tr.grad.clone())
    tr.grad.zero_()
    for c, t in zip(cams, targets):
        tr._accumulate(g, c, t, 0.5, False)
    torch.cuda.synchronize()
    want = 0.5 * (per_view[0] + per_view[1])
    assert float(want.abs().sum()) > 0
    assert rel_l2(tr.grad.double().cpu().numpy(), want.double().cpu().numpy()) <= 1e-5
    # and a batch step applies it: the parameters move, the loss is the views' mean
    tr.grad.zero_()
    before = tr.flat.clone()
    loss = tr.step_batch(cams, targets)
    torch.cuda.synchronize()
    assert torch.isfinite(loss) and float((tr.flat - before).abs().max()) > 0


def test_batched_views_match_one_view_at_a_time(R):
    """The batched training forward (one projection, sort and blend launch sequence for all
    views) gives each view's image-only render bit for bit; its backward (one persistent
    launch over every view's tiles) gives the sum of the views' flat backwards; and after
    the workspace was used by another render it re-derives its lists."""
    from paper_2406_11836_gb300.render import Trainer
    scene = W.uniform_cube_scene(20_000, seed=9, log_scale_mean=-2.6, sh_degree=1).to("cuda")
    tr = Trainer(scene, 3, device="cuda")
    cams = [W.look_at((0.2, -2.6, 0.3), (0, 0, 0), 96, 64), W.look_at((2.5, 0.4, 0.9), (0, 0, 0), 80, 72),
            W.look_at((-1.1, 2.0, -1.4), (0.1, 0, 0), 45, 37)]
    gen = torch.Generator(device="cuda").manual_seed(4)
    targets = [torch.rand(3, c.height, c.width, device="cuda", generator=gen) for c in cams]
    g = tr.gaussians()
    imgs = R.render_batch_fwd(tr.kd, g, cams, tr.opts, tr.ws)
    torch.cuda.synchronize()
    for c, im in zip(cams, imgs):
        ref = R.render_fwd(tr.kd, g, c, tr.opts, R.Workspace(), partials=False)["image"]
        torch.cuda.synchronize()
        assert torch.equal(im, ref), (c.width, c.height, float((im - ref).abs().max()))
    dls = [torch.sign(im - t) / float(im.numel()) for im, t in zip(imgs, targets)]
    zeros = lambda: tuple(torch.zeros_like(t) for t in tr.grads())
    gb = zeros()
    R.render_batch_bwd(tr.kd, g, cams, tr.opts, imgs, dls, gb, tr.ws)
    gs = zeros()
    for c, dl in zip(cams, dls):
        ws = R.Workspace()
        out = R.render_fwd(tr.kd, g, c, tr.opts, ws, partials=False)
        R.render_bwd_flat(tr.kd, g, c, tr.opts, out["image"], dl, gs, ws, tile_depth=out["tile_depth"])
    torch.cuda.synchronize()
    assert float(sum(t.abs().sum() for t in gs)) > 0
    for a, b in zip(gb, gs):
        assert rel_l2(a.double().cpu().numpy(), b.double().cpu().numpy()) <= 1e-5
    R.render_fwd(tr.kd, g, cams[0], tr.opts, tr.ws)            # the workspace's lists are replaced
    gr = zeros()
    R.render_batch_bwd(tr.kd, g, cams, tr.opts, imgs, dls, gr, tr.ws)
    torch.cuda.synchronize()
    for a, b in zip(gr, gb):
        assert rel_l2(a.double().cpu().numpy(), b.double().cpu().numpy()) <= 1e-5


def test_batched_views_gradient_matches_oracle_adjoint(R):
    """Two views of the tiny scene through the batched step: the summed gradient against the
    oracle's adjoint of Eq. 2 for each view, added."""
    from oracle import oracle as O
    from _helpers import oracle_opts
    from paper_2406_11836_gb300.render import Trainer
    wl = W.tiny()
    tr = Trainer(wl.scene.to("cuda"), wl.depth_L, device="cuda")
    cams = [wl.cameras[0], W.look_at((1.8, -2.2, 0.6), (0, 0, 0), 64, 48)]
    g = tr.gaussians()
    imgs = R.render_batch_fwd(tr.kd, g, cams, tr.opts, tr.ws)
    gen = torch.Generator(device="cuda").manual_seed(6)
    dls = [torch.sign(im - torch.rand(im.shape, device="cuda", generator=gen)) / float(im.numel()) for im in imgs]
    grads = tuple(torch.zeros_like(t) for t in tr.grads())
    R.render_batch_bwd(tr.kd, g, cams, tr.opts, imgs, dls, grads, tr.ws)
    torch.cuda.synchronize()
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    want = {n: 0.0 for n in names}
    for c, dl in zip(cams, dls):
        pix = np.arange(c.width * c.height)
        adj = O.adjoint(wl.scene, c, dl.reshape(3, -1).T.double().cpu().numpy(), oracle_opts(), pix=pix)
        for n in names:
            want[n] = want[n] + adj[n]
    for n, got in zip(names, grads):
        assert np.abs(want[n]).max() > 0, n
        assert rel_l2(got.double().cpu().numpy().reshape(want[n].shape), want[n]) <= 1e-3, n


def test_step_batch_batched_equals_sequential(R):
    """Trainer.step_batch through the batched launch sequence and view by view: the same
    loss and the same first Adam moments (the gradient) up to the order of atomic sums."""
    from paper_2406_11836_gb300.render import Trainer
    scene = W.uniform_cube_scene(20_000, seed=9, log_scale_mean=-2.6, sh_degree=1).to("cuda")
    cams = [W.look_at((0.2, -2.6, 0.3), (0, 0, 0), 96, 64), W.look_at((2.5, 0.4, 0.9), (0, 0, 0), 80, 72)]
    gen = torch.Generator(device="cuda").manual_seed(5)
    targets = [torch.rand(3, c.height, c.width, device="cuda", generator=gen) for c in cams]
    a = Trainer(scene, 2, device="cuda", batched_views=True)
    b = Trainer(scene, 2, device="cuda", batched_views=False)
    la = a.step_batch(cams, targets)
    lb = b.step_batch(cams, targets)
    torch.cuda.synchronize()
    assert abs(float(la) - float(lb)) <= 1e-6 * max(1.0, abs(float(lb)))
    assert float(b.m.abs().sum()) > 0
    assert rel_l2(a.m.double().cpu().numpy(), b.m.double().cpu().numpy()) <= 1e-5
