"""Partition balance (Sec. 3.3) and re-partitioning during training (Sec. 3.4).

The median KD splits give every subset the same number of splat centres up to one per
level; a fixed spatial grid of the same shape does not on a clustered scene.  As centres
move, an old partition drifts out of balance and re-partitioning restores it.
"""
import numpy as np
import pytest
import torch

from paper_2406_11836_gb300 import partition as Pt


def test_grid_planes_split_boxes_in_the_middle():
    axis, split = Pt.grid_splits((0, 0, 0), (8, 4, 2), 3)
    # heap order: root on x at 4; its children on y at 2; their children on z at 1
    assert list(axis) == [0, 1, 1, 2, 2, 2, 2]
    assert np.allclose(split, [4, 2, 2, 1, 1, 1, 1])
    axis, split = Pt.grid_splits((-1, -1, -1), (1, 3, 1), 4)
    assert axis[7] == 0                        # depth 3 cycles back to x
    # node 7 is the leftmost at depth 3: box x in [-1, 0], so its middle is -0.5
    assert np.isclose(split[7], -0.5)


@pytest.mark.gpu
def test_median_partition_balances_and_repartition_restores_it():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import rgs
    from paper_2406_11836_gb300 import workloads as W
    scene = W.cluster_scene(200_000, 40, seed=11, device="cuda", sh_degree=1, centre_lo=(-25, -25, 0),
                            centre_hi=(25, 25, 5), std_lo=(0.5, 0.5, 0.1), std_hi=(3.0, 3.0, 1.0))
    L = 4
    kd = rgs.kd_partition(scene, L)
    med = Pt.balance(kd, scene.means)
    assert sum(med["owned"]) == scene.n
    assert max(med["owned"]) - min(med["owned"]) <= L         # median splits: off by one per level
    assert med["overlap"] >= 0.0
    grid = Pt.balance(Pt.kd_grid(scene, L), scene.means)
    assert sum(grid["owned"]) == scene.n
    assert grid["owned_max_over_mean"] > 1.5 * med["owned_max_over_mean"]   # clusters crowd grid cells
    # the centres drift (a cluster moves): the old planes go out of balance, new ones do not
    moved = scene.means.clone()
    sel = moved[:, 0] > moved[:, 0].median()
    moved[sel] += torch.tensor([30.0, 0.0, 0.0], device="cuda")
    drifted = Pt.balance(kd, moved)
    assert max(drifted["owned"]) - min(drifted["owned"]) > L
    scene2 = W.Scene(moved, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh, scene.sh_degree)
    again = Pt.balance(rgs.kd_partition(scene2, L), moved)
    assert max(again["owned"]) - min(again["owned"]) <= L


@pytest.mark.gpu
def test_trainer_repartitions_every_n_steps():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_11836_gb300 import build as B
    B.build()
    from paper_2406_11836_gb300 import workloads as W
    from paper_2406_11836_gb300.render import Trainer
    scene = W.uniform_cube_scene(20_000, seed=5, log_scale_mean=-2.6, sh_degree=1).to("cuda")
    tr = Trainer(scene, 2, device="cuda", repartition_every=2)
    cam = W.look_at((0.2, -2.6, 0.3), (0, 0, 0), 96, 64)
    target = torch.rand(3, 64, 96, device="cuda")
    handles = []
    for _ in range(4):
        loss = tr.step(cam, target)
        assert torch.isfinite(loss)
        handles.append(tr.kd.handle.value)
    assert handles[0] != handles[1] and handles[1] == handles[2] and handles[2] != handles[3]
