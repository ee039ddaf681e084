"""Differentiable hierarchical render (autograd) and a training step (Sec. 3.4 pipeline).

``RetinaGSRender`` wraps the C ABI: its forward renders every subset's partial colour and
transmittance and merges them (Eq. 3-5); its backward routes dL/dimage through the merge
to each subset, replays each subset's blend from the stored partials over the forward's
per-tile lists (kept in the render's workspace), and pulls the 2D gradients back to means,
scales, rotations, opacity and SH.  ``Trainer`` runs the full step (render, L1 loss, backward, Adam with the position
learning-rate decay of Sec. 4) on flat parameter buffers without extra copies.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rgs


class RenderContext:
    """Non-tensor state of a render: KD partition, camera, options and workspace."""

    def __init__(self, kd: rgs.KD, cam, opts: rgs.RenderOpts | None = None, ws: rgs.Workspace | None = None,
                 sh_degree: int = 0):
        self.kd = kd
        self.cam = cam
        self.opts = opts if opts is not None else rgs.default_opts()
        self.ws = ws if ws is not None else rgs.Workspace()
        self.sh_degree = sh_degree
        self.last = None


class RetinaGSRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, rc: RenderContext):
        g = rgs.gaussians_c(means, log_scales, quats, opacity_logits, sh, rc.sh_degree)
        out = rgs.render_fwd(rc.kd, g, rc.cam, rc.opts, rc.ws, image=True)
        ctx.rc = rc
        ctx.save_for_backward(means, log_scales, quats, opacity_logits, sh, out["partial_C"], out["partial_T"],
                              out["tile_depth"])
        rc.last = out
        ctx.mark_non_differentiable(out["partial_C"], out["partial_T"], out["T_final"])
        return out["image"], out["partial_C"], out["partial_T"], out["T_final"]

    @staticmethod
    def backward(ctx, g_image, g_pc, g_pt, g_tf):
        means, log_scales, quats, opacity_logits, sh, pc, pt, td = ctx.saved_tensors
        rc = ctx.rc
        grads = tuple(torch.zeros_like(t) for t in (means, log_scales, quats, opacity_logits, sh))
        if g_image is None:
            return (*grads, None)
        g = rgs.gaussians_c(means, log_scales, quats, opacity_logits, sh, rc.sh_degree)
        rgs.render_bwd(rc.kd, g, rc.cam, rc.opts, pc, pt, g_image.contiguous(), grads, rc.ws, tile_depth=td)
        return (*grads, None)


def render(means, log_scales, quats, opacity_logits, sh, rc: RenderContext):
    """Differentiable render: returns (image [3,H,W], partial_C, partial_T, T_final)."""
    return RetinaGSRender.apply(means, log_scales, quats, opacity_logits, sh, rc)


# --------------------------------------------------------------------------- training step
class Trainer:
    """Parameters, gradients and Adam moments in flat float32 buffers (one Adam launch per
    step).  Groups, in buffer order: quats, means, log_scales, opacity_logits, sh."""

    # learning rates of the non-position groups: the paper gives only the position schedule
    # (1.6e-4 -> 1.6e-6); the others are the usual 3DGS values
    LR = {"quats": 1e-3, "log_scales": 5e-3, "opacity_logits": 5e-2, "sh_dc": 2.5e-3, "sh_rest": 2.5e-3 / 20}

    def __init__(self, scene, depth_L: int, opts: rgs.RenderOpts | None = None, max_steps: int = 60000,
                 device="cuda", repartition_every: int = 0, cull_occluded: bool = True, backward: str = "flat",
                 batched_views: bool = True):
        n = scene.n
        self.n = n
        self.sh_degree = scene.sh_degree
        self.nsh = (scene.sh_degree + 1) ** 2
        sizes = [("quats", 4 * n), ("means", 3 * n), ("log_scales", 3 * n), ("opacity_logits", n),
                 ("sh", 3 * self.nsh * n)]
        offs = np.cumsum([0] + [s for _, s in sizes])
        total = int(offs[-1])
        self.flat = torch.empty(total, dtype=torch.float32, device=device)
        self.grad = torch.zeros(total, dtype=torch.float32, device=device)
        self.m = torch.zeros(total, dtype=torch.float32, device=device)
        self.v = torch.zeros(total, dtype=torch.float32, device=device)
        src = {"quats": scene.quats, "means": scene.means, "log_scales": scene.log_scales,
               "opacity_logits": scene.opacity_logits, "sh": scene.sh}
        shapes = {"quats": (n, 4), "means": (n, 3), "log_scales": (n, 3), "opacity_logits": (n,),
                  "sh": (n, self.nsh, 3)}
        self.p, self.g = {}, {}
        for (name, _), a, b in zip(sizes, offs[:-1], offs[1:]):
            self.p[name] = self.flat[a:b].view(shapes[name])
            self.g[name] = self.grad[a:b].view(shapes[name])
            self.p[name].copy_(src[name].reshape(shapes[name]).to(device))
        # Adam segments: quats, means, log_scales, opacity, sh; inside the sh block [N, nsh, 3]
        # the degree-0 coefficients of every splat (3 of each 3 nsh) take the dc rate
        self.seg = [0, int(offs[1]), int(offs[2]), int(offs[3]), int(offs[4]), total]
        self.max_steps = max_steps
        # Sec. 3.4: the partition is re-run on the current centres every so many steps
        # (0: never); the planes change, the parameters and moments do not
        self.repartition_every = int(repartition_every)
        self.step_count = 0
        # by default a subset is not blended on rays already saturated in front of it
        # (rgs_render_opts.cull_occluded): the image moves by less than eps_T max(rgb), and
        # the backward skips those rays anyway
        self.opts = opts if opts is not None else rgs.default_opts(cull_occluded=1 if cull_occluded else 0)
        # "flat" (default, the faster on the city workload): the forward writes the image
        # only and the backward replays each pixel's concatenated list once
        # (rgs_render_bwd_flat, exact by the equality of Eq. 5 and Eq. 2); "subsets": the
        # forward writes the partial maps and the backward routes dL/dimage through the
        # merge to each subset (rgs_render_bwd)
        if backward not in ("subsets", "flat"):
            raise ValueError(f"backward must be 'subsets' or 'flat', not {backward!r}")
        self.backward = backward
        # step_batch renders its views through one launch sequence (rgs_render_batch_fwd/bwd;
        # flat backward only) rather than one after another
        self.batched_views = bool(batched_views)
        self.ws = rgs.Workspace(device)
        self.kd = rgs.kd_partition(self.gaussians(), depth_L, float(self.opts.trunc_mult))

    def gaussians(self):
        p = self.p
        return rgs.gaussians_c(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"], self.sh_degree)

    def grads(self):
        g = self.g
        return (g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"])

    def lrs(self, step):
        sh = self.LR["sh_rest"] if self.nsh > 1 else self.LR["sh_dc"]
        return [self.LR["quats"], rgs.position_lr(step, self.max_steps), self.LR["log_scales"],
                self.LR["opacity_logits"], sh]

    def sh_periodic(self):
        """The Adam rule giving the degree-0 SH coefficients of every splat the dc rate."""
        return (4, 3 * self.nsh, 3, self.LR["sh_dc"]) if self.nsh > 1 else None

    def repartition(self, depth_L: int | None = None):
        """Re-run the KD partition on the current centres (Sec. 3.4: repeated after a set
        number of epochs)."""
        self.kd = rgs.kd_partition(self.gaussians(), depth_L if depth_L is not None else self.kd.L,
                                   float(self.opts.trunc_mult))

    # ---------------------------------------------------------------- checkpoint / resume
    def checkpoint(self, device=None) -> dict:
        """Parameters, Adam moments, step count and KD splits (device copies by default)."""
        dev = device if device is not None else self.flat.device
        axis, split = self.kd.splits()
        return {"flat": self.flat.detach().to(dev, copy=True), "m": self.m.to(dev, copy=True),
                "v": self.v.to(dev, copy=True), "step": self.step_count, "seg": list(self.seg),
                "n": self.n, "sh_degree": self.sh_degree, "kd_L": self.kd.L,
                "kd_axis": torch.as_tensor(axis), "kd_split": torch.as_tensor(split)}

    def restore(self, ck: dict):
        """Resume from `checkpoint()`: parameters, moments, step and the KD partition (its
        planes, with the subsets re-formed on the restored parameters) come back exactly."""
        assert ck["n"] == self.n and ck["sh_degree"] == self.sh_degree
        self.flat.copy_(ck["flat"])
        self.m.copy_(ck["m"])
        self.v.copy_(ck["v"])
        self.grad.zero_()
        self.step_count = int(ck["step"])
        self.kd = rgs.kd_from_splits(self.gaussians(), int(ck["kd_L"]), np.asarray(ck["kd_axis"]),
                                     np.asarray(ck["kd_split"]), float(self.opts.trunc_mult))

    def save(self, path: str):
        torch.save(self.checkpoint(device="cpu"), path)

    def load(self, path: str):
        self.restore(torch.load(path, map_location="cpu"))

    def _accumulate(self, g, cam, target: torch.Tensor, weight: float, return_loss: bool):
        """Forward, L1 loss (scaled by weight) and backward of one view, adding its gradients
        to the gradient buffer; the backward follows its own forward, so it replays the
        forward's lists."""
        flat = self.backward == "flat"
        out = rgs.render_fwd(self.kd, g, cam, self.opts, self.ws, image=True, partials=not flat)
        img = out["image"]
        diff = img - target
        loss = diff.abs().mean() if return_loss else None
        dL = torch.sign(diff).div_(float(diff.numel()) / weight)
        if flat:
            rgs.render_bwd_flat(self.kd, g, cam, self.opts, img, dL, self.grads(), self.ws,
                                tile_depth=out["tile_depth"])
        else:
            rgs.render_bwd(self.kd, g, cam, self.opts, out["partial_C"], out["partial_T"], dL, self.grads(), self.ws,
                           tile_depth=out["tile_depth"])
        return loss

    def step(self, cam, target: torch.Tensor, return_loss: bool = True):
        """One training step: forward, L1 loss against `target` [3,H,W], backward, Adam.
        Returns the loss as a 0-d tensor (left on the device)."""
        loss = self._accumulate(self.gaussians(), cam, target, 1.0, return_loss)
        return self._update(loss)

    def step_batch(self, cams, targets, return_loss: bool = True):
        """One training step on several views: the mean of their L1 losses, its gradient
        summed over the views' backwards, then one Adam step.  Returns the mean loss.
        With the flat backward (and batched_views) the views go through one batched forward
        and one batched backward; otherwise one view after another."""
        g = self.gaussians()
        w = 1.0 / len(cams)
        if self.backward == "flat" and self.batched_views and 1 < len(cams) <= 16:
            imgs = rgs.render_batch_fwd(self.kd, g, cams, self.opts, self.ws)
            losses, dls = [], []
            for img, t in zip(imgs, targets):
                diff = img - t
                if return_loss:
                    losses.append(diff.abs().mean() * w)
                dls.append(torch.sign(diff).div_(float(diff.numel()) / w))
            rgs.render_batch_bwd(self.kd, g, cams, self.opts, imgs, dls, self.grads(), self.ws)
            return self._update(torch.stack(losses).sum() if return_loss else None)
        losses = [self._accumulate(g, c, t, w, return_loss) for c, t in zip(cams, targets)]
        return self._update(torch.stack(losses).mean() if return_loss else None)

    def _update(self, loss):
        self.step_count += 1
        rgs.adam_step(self.flat, self.grad, self.m, self.v, self.seg, self.lrs(self.step_count), self.step_count,
                      zero_grad=True, periodic=self.sh_periodic())
        if self.repartition_every and self.step_count % self.repartition_every == 0:
            self.repartition()
        return loss
