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
