"""FP64 CPU oracle for hierarchical 3D Gaussian splatting (RetinaGS, arXiv 2406.11836).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg may use this module; the product path never imports it, and it imports nothing
from the product package.  The heavy per-pixel work lives in ``rgs_oracle.c`` (plain C,
double precision, OpenMP over pixels); the merge of Eq. 5, its adjoint and the Adam
step are written here in numpy float64.

Every function states the passage it follows.  Inputs: splat parameters are float32
arrays (widened exactly to float64 before use); cameras are objects with ``viewmat``
(4x4 world->camera, OpenCV axes), ``fx, fy, cx, cy, width, height, near_z``, rounded
to float32 first because that is what the library receives.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rgs_oracle.c")
_LIB = os.path.join(_HERE, "_build", "librgs_oracle.so")

FLAG_TRUNC, FLAG_DEPTH, FLAG_SPLIT, FLAG_KINK, FLAG_DEPTH_PART, FLAG_TRUNC_PART = 1, 2, 4, 8, 16, 32


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with the host compiler (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib_handle = None


def _lib():
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = ctypes.CDLL(build())
        _lib_handle.or_subsets.restype = ctypes.c_int64
    return _lib_handle


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else ctypes.c_void_p(0)


def _np(x, dtype=None):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.asarray(x)
    if dtype is not None:
        a = a.astype(dtype)
    return np.ascontiguousarray(a)


# --------------------------------------------------------------------------- inputs
@dataclass
class Opts:
    """Render constants (the readings of the truncation rule and the blend clamps)."""
    trunc_mult: float = 3.0
    eps_T: float = 0.0          # 0: no early termination (flat mode never terminates)
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    dilation: float = 0.3
    bg: tuple = (0.0, 0.0, 0.0)
    flag_rel: float = 3e-6      # relative rounding margin of the truncation/plane ambiguity flags (~50 fp32 ulp)
    flag_depth_rel: float = 1e-11  # relative margin for two contributors at (nearly) equal depth
    foot: bool = False          # x_i = foot of the perpendicular from u_i onto the ray (comparison reading)

    def vec(self) -> np.ndarray:
        f = lambda v: float(np.float32(v))
        return np.array([f(self.trunc_mult), f(self.eps_T), f(self.alpha_min), f(self.alpha_max),
                         f(self.dilation), f(self.bg[0]), f(self.bg[1]), f(self.bg[2]), self.flag_rel,
                         self.flag_depth_rel, 1.0 if self.foot else 0.0], np.float64)


def cam_vec(cam) -> np.ndarray:
    v = np.zeros(23, np.float64)
    v[:16] = np.asarray(cam.viewmat, np.float32).astype(np.float64).reshape(16)
    v[16:20] = np.array([cam.fx, cam.fy, cam.cx, cam.cy], np.float32).astype(np.float64)
    v[20], v[21] = cam.width, cam.height
    v[22] = float(np.float32(cam.near_z))
    return v


def camera_center(cam) -> np.ndarray:
    """o = -R^T t from the float32 view matrix."""
    V = np.asarray(cam.viewmat, np.float32).astype(np.float64)
    return -V[:3, :3].T @ V[:3, 3]


def pixel_ray(cam, px, py) -> np.ndarray:
    """World direction of pixel (px,py) with unit camera-z component."""
    V = np.asarray(cam.viewmat, np.float32).astype(np.float64)
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    r = np.array([(px + 0.5 - cx) / fx, (py + 0.5 - cy) / fy, 1.0])
    return V[:3, :3].T @ r


class _Scene:
    def __init__(self, scene):
        self.means = _np(scene.means, np.float64)
        self.log_scales = _np(scene.log_scales, np.float64)
        self.quats = _np(scene.quats, np.float64)
        self.logits = _np(scene.opacity_logits, np.float64).reshape(-1)
        self.sh = _np(scene.sh, np.float64)
        self.deg = int(scene.sh_degree)
        self.n = self.means.shape[0]

    def args(self):
        return (ctypes.c_int64(self.n), _p(self.means), _p(self.log_scales), _p(self.quats), _p(self.logits),
                _p(self.sh), ctypes.c_int(self.deg))


# --------------------------------------------------------------------------- Sec. 3.3: KD tree
def kd_partition(means, L: int):
    """KD tree of depth L on the splat centres (Sec. 3.3): axis = level mod 3, median split
    (fp32 midpoint of the two middle coordinates for an even count, the median itself for an
    odd count).  Returns (axis int32[K-1], split float32[K-1]) in heap order."""
    m = _np(means, np.float32)
    K = 1 << L
    axis = np.zeros(max(K - 1, 1), np.int32)
    split = np.zeros(max(K - 1, 1), np.float32)
    rc = _lib().or_kd_partition(ctypes.c_int64(m.shape[0]), _p(m), ctypes.c_int(L), _p(axis), _p(split))
    assert rc == 0, rc
    return axis[:K - 1], split[:K - 1]


def subsets(means, log_scales, L, axis, split, trunc_mult=3.0, margin=1e-6):
    """Overlapping subsets N_k = {i : n.u_i + d <= D_i for every plane of S_k} (Sec. 3.3),
    D_i = trunc_mult * max scale.  Returns CSR (offsets int64[K+1], idx int32[M]) and a
    per-splat flag of memberships within `margin` (relative) of a split."""
    mu = _np(means, np.float64)
    ls = _np(log_scales, np.float64)
    K = 1 << L
    ax = np.ascontiguousarray(np.asarray(axis, np.int32).reshape(-1)) if K > 1 else np.zeros(1, np.int32)
    sp = np.ascontiguousarray(np.asarray(split, np.float32).reshape(-1)) if K > 1 else np.zeros(1, np.float32)
    offsets = np.zeros(K + 1, np.int64)
    amb = np.zeros(mu.shape[0], np.int32)
    lib = _lib()
    M = lib.or_subsets(ctypes.c_int64(mu.shape[0]), _p(mu), _p(ls), ctypes.c_int(L), _p(ax), _p(sp),
                       ctypes.c_double(trunc_mult), ctypes.c_double(margin), _p(offsets), None, None)
    idx = np.zeros(max(M, 1), np.int32)
    lib.or_subsets(ctypes.c_int64(mu.shape[0]), _p(mu), _p(ls), ctypes.c_int(L), _p(ax), _p(sp),
                   ctypes.c_double(trunc_mult), ctypes.c_double(margin), _p(offsets), _p(idx), _p(amb))
    return offsets, idx[:M], amb.astype(bool)


def leaf_boxes(L, axis, split):
    """Half-open boxes [lo, hi) of the K leaves (unbounded sides are +-inf)."""
    K = 1 << L
    lo = np.zeros((K, 3))
    hi = np.zeros((K, 3))
    ax = np.ascontiguousarray(np.asarray(axis, np.int32).reshape(-1)) if K > 1 else np.zeros(1, np.int32)
    sp = np.ascontiguousarray(np.asarray(split, np.float32).reshape(-1)) if K > 1 else np.zeros(1, np.float32)
    _lib().or_leaf_boxes(ctypes.c_int(L), _p(ax), _p(sp), _p(lo), _p(hi))
    return lo, hi


def ray_order(L, axis, split, o, d):
    """Order o_l of Eq. 5 for the ray o + t d: the leaves it crosses sorted by entry t, then
    the others.  Returns (order int32[K], number crossed)."""
    K = 1 << L
    ax = np.ascontiguousarray(np.asarray(axis, np.int32).reshape(-1)) if K > 1 else np.zeros(1, np.int32)
    sp = np.ascontiguousarray(np.asarray(split, np.float32).reshape(-1)) if K > 1 else np.zeros(1, np.float32)
    order = np.zeros(K, np.int32)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    nc = _lib().or_ray_order(ctypes.c_int(L), _p(ax), _p(sp), _p(o), _p(d), _p(order))
    return order, nc


# --------------------------------------------------------------------------- Sec. 3.1: projection
PROJ_FIELDS = ("visible", "z", "mean_x", "mean_y", "cov_xx", "cov_xy", "cov_yy", "conic_a", "conic_b", "conic_c",
               "alpha", "r", "g", "b", "D", "p_x", "p_y", "raw_r", "raw_g", "raw_b")


def project(scene, cam, opts: Opts = Opts()) -> dict:
    """Per-splat EWA projection (Sec. 3.1): dict of float64 arrays named by PROJ_FIELDS."""
    s = _Scene(scene)
    out = np.zeros((s.n, len(PROJ_FIELDS)))
    rc = _lib().or_project(*s.args(), _p(cam_vec(cam)), _p(opts.vec()), _p(out))
    assert rc == 0
    return {k: out[:, j] for j, k in enumerate(PROJ_FIELDS)}


def sh_basis(deg, dirs):
    """Real SH basis (Condon-Shortley phase) and its polynomial gradient at unit dirs [M,3]."""
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), np.float64)
    nsh = (deg + 1) ** 2
    Y = np.zeros((dirs.shape[0], 16))
    dY = np.zeros((dirs.shape[0], 16, 3))
    lib = _lib()
    for i in range(dirs.shape[0]):
        y = np.zeros(16)
        dy = np.zeros((16, 3))
        lib.or_sh_basis(ctypes.c_int(deg), _p(np.ascontiguousarray(dirs[i])), _p(y), _p(dy))
        Y[i], dY[i] = y, dy
    return Y[:, :nsh], dY[:, :nsh]


# --------------------------------------------------------------------------- Eq. 2 / Eq. 3-6: render
def _pix(cam, pix):
    if pix is None:
        return np.arange(cam.width * cam.height, dtype=np.int64)
    return np.ascontiguousarray(np.asarray(pix, np.int64).reshape(-1))


def render(scene, cam, opts: Opts = Opts(), pix=None, hier=False, L=0, axis=None, split=None, brute=False) -> dict:
    """Render the listed pixels (py*W+px; all when None).

    hier=False: flat blending, Eq. 2, over every splat that passes the truncation tests,
    in depth order.  hier=True: Eq. 3-4 per subset of the KD tree (axis, split) with the
    indicator of Eq. 6, merged by Eq. 5 in the order each ray crosses the subspaces.
    With opts.foot, x_i is the foot of the perpendicular from the splat centre onto the
    pixel ray (Sec. 3.2, printed reading) and the contributors are ordered by its ray
    parameter.  Returns C [P,3] (background included), T [P], flags [P], ncontrib [P] and, in
    hierarchical mode, partC [P,K,3], partT [P,K], order [P,K]."""
    s = _Scene(scene)
    p = _pix(cam, pix)
    P = p.shape[0]
    K = 1 << L if hier else 1
    ax = np.ascontiguousarray(np.asarray(axis if axis is not None else [0], np.int32).reshape(-1))
    sp = np.ascontiguousarray(np.asarray(split if split is not None else [0], np.float32).reshape(-1))
    if ax.size == 0:
        ax, sp = np.zeros(1, np.int32), np.zeros(1, np.float32)
    C = np.zeros((P, 3))
    T = np.zeros(P)
    flags = np.zeros(P, np.int32)
    nc = np.zeros(P, np.int32)
    partC = np.zeros((P, K, 3)) if hier else None
    partT = np.zeros((P, K)) if hier else None
    order = np.zeros((P, K), np.int32) if hier else None
    rc = _lib().or_render(ctypes.c_int(1 if hier else 0), *s.args(), _p(cam_vec(cam)), _p(opts.vec()),
                          ctypes.c_int(L if hier else 0), _p(ax), _p(sp), ctypes.c_int64(P), _p(p),
                          ctypes.c_int(1 if brute else 0), _p(C), _p(T), _p(flags), _p(nc), _p(partC), _p(partT),
                          _p(order))
    assert rc == 0, rc
    out = {"C": C, "T": T, "flags": flags, "ncontrib": nc}
    if hier:
        out.update(partC=partC, partT=partT, order=order)
    return out


def adjoint(scene, cam, dLdC, opts: Opts = Opts(), pix=None) -> dict:
    """Reverse mode of the flat form (Eq. 2 and the projection of Sec. 3.1), written by
    hand: given dL/dC [P,3] at the listed pixels, returns dL/d(means, log_scales, quats,
    opacity_logits, sh) in float64, and the per-splat 2D gradients g2d [N,9] =
    (mean x, mean y, conic a, b, c, alpha, r, g, b).  With opts.foot the contributors and
    their order are the foot reading's (Sec. 3.2, the perpendicular-foot reading of x_i);
    the per-pair adjoint is the same, since that reading changes only discrete decisions."""
    s = _Scene(scene)
    p = _pix(cam, pix)
    g = np.ascontiguousarray(np.asarray(dLdC, np.float64).reshape(p.shape[0], 3))
    out = {"means": np.zeros_like(s.means), "log_scales": np.zeros_like(s.log_scales),
           "quats": np.zeros_like(s.quats), "opacity_logits": np.zeros_like(s.logits), "sh": np.zeros_like(s.sh),
           "g2d": np.zeros((s.n, 9))}
    rc = _lib().or_adjoint(*s.args(), _p(cam_vec(cam)), _p(opts.vec()), ctypes.c_int64(p.shape[0]), _p(p), _p(g),
                           _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logits"]),
                           _p(out["sh"]), _p(out["g2d"]))
    assert rc == 0
    return out


def pair_signature(scene, cam, opts: Opts = Opts(), pix=None):
    """(count, checksum) of the contributing (pixel, splat) pairs, for finite differences."""
    s = _Scene(scene)
    p = _pix(cam, pix)
    cnt = ctypes.c_int64(0)
    cs = ctypes.c_double(0)
    _lib().or_pair_signature(*s.args(), _p(cam_vec(cam)), _p(opts.vec()), ctypes.c_int64(p.shape[0]), _p(p),
                             ctypes.byref(cnt), ctypes.byref(cs))
    return cnt.value, cs.value


# --------------------------------------------------------------------------- Eq. 5: merge
def merge(partC, partT, order, bg=(0.0, 0.0, 0.0)):
    """Eq. 5: C = sum_r C_{o_r} prod_{m<r} T_{o_m}, plus the background behind everything.
    partC [K,3,P], partT [K,P], order [R] (one order for every pixel) or [R,P], R <= K: the
    subsets taking part, front to back.  Returns (C [3,P], T_final [P])."""
    partC = np.asarray(partC, np.float64)
    partT = np.asarray(partT, np.float64)
    K, _, P = partC.shape
    order = np.asarray(order)
    order = order.reshape(order.shape[0], -1)
    R = order.shape[0]
    if order.shape[1] == 1:
        order = np.repeat(order, P, axis=1)
    cols = np.arange(P)
    C = np.zeros((3, P))
    Pm = np.ones(P)
    for r in range(R):
        k = order[r]
        C += partC[k, :, cols].T * Pm
        Pm = Pm * partT[k, cols]
    C += np.asarray(bg, np.float64)[:, None] * Pm
    return C, Pm


def merge_backward(partC, partT, order, gC, gT=None, bg=(0.0, 0.0, 0.0)):
    """Adjoint of Eq. 5.  With P_r = prod_{m<r} T_{o_m} and S_r the colour seen behind
    subset o_r (S_r = sum_{j>r} C_{o_j} prod_{r<m<j} T_{o_m} + bg prod_{m>r} T_{o_m}):
    dL/dC_{o_r} = g P_r, dL/dT_{o_r} = P_r <g, S_r> (+ gT * prod_{m != r} T_{o_m}).
    Returns (dL/dpartC [K,3,P], dL/dpartT [K,P])."""
    partC = np.asarray(partC, np.float64)
    partT = np.asarray(partT, np.float64)
    K, _, P = partC.shape
    order = np.asarray(order)
    order = order.reshape(order.shape[0], -1)
    R = order.shape[0]
    if order.shape[1] == 1:
        order = np.repeat(order, P, axis=1)
    cols = np.arange(P)
    gC = np.asarray(gC, np.float64)
    prefix = np.ones((R + 1, P))
    for r in range(R):
        prefix[r + 1] = prefix[r] * partT[order[r], cols]
    suffix = np.ones((R + 1, P))
    for r in range(R - 1, -1, -1):
        suffix[r] = suffix[r + 1] * partT[order[r], cols]
    S = np.zeros((R, 3, P))
    behind = np.asarray(bg, np.float64)[:, None] * np.ones((3, P))
    for r in range(R - 1, -1, -1):
        S[r] = behind
        behind = partC[order[r], :, cols].T + partT[order[r], cols] * behind
    dC = np.zeros((K, 3, P))
    dT = np.zeros((K, P))
    for r in range(R):
        k = order[r]
        dC[k, :, cols] = (gC * prefix[r]).T
        dT[k, cols] = prefix[r] * np.sum(gC * S[r], axis=0)
        if gT is not None:
            dT[k, cols] += np.asarray(gT, np.float64) * prefix[r] * suffix[r + 1]
    return dC, dT


# --------------------------------------------------------------------------- Adam (Sec. 4 details)
def position_lr(step: int, max_steps: int, lr_init=1.6e-4, lr_final=1.6e-6) -> float:
    """Exponential (log-linear) decay of the position learning rate from 1.6e-4 to 1.6e-6
    (Sec. 4, implementation details)."""
    t = min(max(step / max(max_steps, 1), 0.0), 1.0)
    return math.exp(math.log(lr_init) * (1.0 - t) + math.log(lr_final) * t)


def adam_step(param, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (Kingma & Ba), float64: returns (param, m, v) after step `step` (1-based)."""
    param = np.asarray(param, np.float64)
    grad = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1 - beta1) * grad
    v = beta2 * np.asarray(v, np.float64) + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
