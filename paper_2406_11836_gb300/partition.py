"""Partition reports and the fixed-grid alternative (Sec. 3.3 and Sec. 3.4).

The method splits the scene by median KD splits (Sec. 3.3), so every subset owns the same
number of splat centres up to one per level, and re-runs the partition during training
as the centres move (Sec. 3.4).  This module reports how balanced a partition is (the
analogue of the paper's subset-balance table) and builds the comparison partition of a
fixed spatial grid: the same KD tree shape with every node split at the middle of its
box instead of at the median.  Both are host-side bookkeeping around the library's KD
calls; nothing here is on the render path.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rgs


def grid_splits(lo, hi, depth_L: int):
    """Planes of a fixed grid in heap order: node n at depth d splits its box at the middle
    along axis d mod 3 (the axis rule of the median partition).  lo, hi: the root box."""
    lo = np.asarray(lo, np.float64).reshape(3)
    hi = np.asarray(hi, np.float64).reshape(3)
    n = (1 << depth_L) - 1
    axis = np.zeros(n, np.int32)
    split = np.zeros(n, np.float32)
    boxes = [(lo.copy(), hi.copy())]
    for node in range(n):
        d = int(np.floor(np.log2(node + 1)))
        a = d % 3
        blo, bhi = boxes[node]
        s = 0.5 * (blo[a] + bhi[a])
        axis[node] = a
        split[node] = np.float32(s)
        left_hi = bhi.copy()
        left_hi[a] = s
        right_lo = blo.copy()
        right_lo[a] = s
        boxes.append((blo.copy(), left_hi))     # child 2n + 1
        boxes.append((right_lo, bhi.copy()))    # child 2n + 2
    return axis, split


def kd_grid(scene, depth_L: int, trunc_mult: float = 3.0):
    """The fixed-grid partition of the scene's centres (box of all centres, mid splits)."""
    means = scene.means
    lo = means.min(dim=0).values.double().cpu().numpy()
    hi = means.max(dim=0).values.double().cpu().numpy()
    axis, split = grid_splits(lo, hi, depth_L)
    return rgs.kd_from_splits(scene, depth_L, axis, split, trunc_mult)


def leaf_of(means: torch.Tensor, kd) -> torch.Tensor:
    """Leaf (subset) holding each centre, by the half-open rule (right iff x >= split)."""
    axis, split = kd.splits()
    node = torch.zeros(means.shape[0], dtype=torch.int64, device=means.device)
    ax = torch.as_tensor(axis, dtype=torch.int64, device=means.device)
    sp = torch.as_tensor(split, dtype=means.dtype, device=means.device)
    for _ in range(kd.L):
        a = ax[node]
        right = (means.gather(1, a[:, None])[:, 0] >= sp[node]).long()
        node = 2 * node + 1 + right
    return node - ((1 << kd.L) - 1)


def balance(kd, means: torch.Tensor) -> dict:
    """Owned centres and subset members (with the D_i overlap) per subset, and how far the
    largest is above the mean: the load of the busiest subset relative to a perfect split."""
    K = kd.K
    owned = torch.bincount(leaf_of(means, kd), minlength=K).cpu().numpy().astype(np.int64)
    offsets, _ = kd.subsets(device=means.device)
    members = np.diff(offsets).astype(np.int64)
    n = int(means.shape[0])
    return {
        "subsets": K,
        "owned": owned.tolist(),
        "members": members.tolist(),
        "owned_max_over_mean": float(owned.max() / (n / K)),
        "owned_min_over_mean": float(owned.min() / (n / K)),
        "members_max_over_mean": float(members.max() / members.mean()),
        "overlap": float(members.sum() / n - 1.0),
    }
