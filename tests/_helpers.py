"""Shared helpers of the GPU parity tests (inputs and comparisons; no method arithmetic)."""
import numpy as np
import torch

from oracle import oracle as O

FWD_FLAGS = O.FLAG_TRUNC | O.FLAG_DEPTH
PART_FLAGS = O.FLAG_TRUNC_PART | O.FLAG_DEPTH_PART | O.FLAG_SPLIT
GRAD_FLAGS = O.FLAG_TRUNC | O.FLAG_DEPTH | O.FLAG_KINK

PIXEL_TOL = 1e-4        # max abs pixel error, float32 path vs float64 oracle
GRAD_RTOL = 1e-3        # per-tensor relative L2 error of the gradients
MAX_FLAGGED = 0.001     # at most this fraction of pixels may be left out as ambiguous where a
                        # comparison leaves any out (the foot reading): the straddle policy's cap
PART_MAX_FLAGGED = 0.005  # partial maps: pixels with a contributor whose ray point lies within
                          # rounding of a split plane (or at a threshold inside a subset) may hold
                          # it in either subset; the merged image is compared on every pixel


def oracle_opts(opts=None, eps_T=0.0):
    """Oracle options equal to the library's render options."""
    if opts is None:
        return O.Opts(eps_T=eps_T)
    return O.Opts(trunc_mult=opts.trunc_mult, eps_T=eps_T, alpha_min=opts.alpha_min, alpha_max=opts.alpha_max,
                  dilation=opts.dilation, bg=tuple(opts.bg))


def image_at(img: torch.Tensor, pix: np.ndarray) -> np.ndarray:
    """[3,H,W] device image -> [P,3] float64 at flat pixel indices."""
    flat = img.reshape(3, -1).double().cpu().numpy()
    return flat[:, pix].T


def partials_at(pc: torch.Tensor, pt: torch.Tensor, pix: np.ndarray):
    K = pc.shape[0]
    c = pc.reshape(K, 3, -1).double().cpu().numpy()[:, :, pix]        # [K,3,P]
    t = pt.reshape(K, -1).double().cpu().numpy()[:, pix]              # [K,P]
    return np.transpose(c, (2, 0, 1)), t.T                            # [P,K,3], [P,K]


def rel_l2(a, b):
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / max(nb, 1e-30)


def assert_all_close(got, ref, flags=None, what="image", tol=PIXEL_TOL):
    """Max abs error over EVERY sampled pixel, flagged ones included (hierarchical blending
    equals flat blending exactly, so no pixel is left out); the number the oracle flags as
    ambiguous is only reported."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = float(np.abs(got - ref).max()) if got.size else 0.0
    nflag = int(((np.asarray(flags) & FWD_FLAGS) != 0).sum()) if flags is not None else 0
    assert err <= tol, f"{what}: max abs error {err:.3g} over all {len(got)} pixels ({nflag} flagged ambiguous)"
    return err
