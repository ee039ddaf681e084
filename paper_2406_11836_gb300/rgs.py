"""Thin Python binding of the C ABI in ``include/rgs.h`` (ctypes; argument marshalling only).

Every step of the render runs in the CUDA library ``_build/librgs.so``; PyTorch only
provides device memory and streams.  There is no CPU fallback: if the library is not
built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librgs.so")

RGS_OK, RGS_EINVAL, RGS_ENOMEM, RGS_ECUDA, RGS_EOVERFLOW, RGS_ETIMEOUT, RGS_EAGAIN = 0, -1, -2, -3, -4, -5, -6


class RGSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rgs error {code}: {msg}")
        self.code = code


class Gaussians(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("sh", c_void_p), ("n", c_int64), ("sh_degree", c_int)]


class GaussianGrads(ctypes.Structure):
    _fields_ = [("means", c_void_p), ("log_scales", c_void_p), ("quats", c_void_p), ("opacity_logits", c_void_p),
                ("sh", c_void_p)]


class CameraC(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 16), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int), ("height", c_int), ("near_z", c_float)]


class RenderOpts(ctypes.Structure):
    _fields_ = [("tile", c_int), ("trunc_mult", c_float), ("eps_T", c_float), ("alpha_min", c_float),
                ("alpha_max", c_float), ("dilation", c_float), ("bg", c_float * 3), ("cull_occluded", c_int),
                ("group_binning", c_int)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", c_size_t), ("max_slots", c_int), ("lanes", c_int), ("plain", c_int),
                ("max_width", c_int), ("max_height", c_int), ("max_queue", c_int), ("inst_per_pixel", c_float),
                ("group_per_splat", c_float), ("group_min_instances", c_float), ("batch_max_pixels", c_int64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("failed", c_int64), ("cancelled", c_int64),
                ("batches", c_int64), ("requeued", c_int64), ("instance_capacity", c_int64),
                ("mean_batch", ctypes.c_double)]


_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_2406_11836_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    L.rgs_last_error.restype = ctypes.c_char_p
    L.rgs_last_required_workspace.restype = c_size_t
    L.rgs_position_lr.restype = c_float
    L.rgs_position_lr.argtypes = [c_int64, c_int64, c_float, c_float]
    L.rgs_kd_partition.argtypes = [POINTER(Gaussians), c_int, c_float, POINTER(c_void_p), c_void_p]
    L.rgs_kd_info.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int64)]
    L.rgs_kd_from_splits.argtypes = [POINTER(Gaussians), c_int, c_void_p, c_void_p, c_float, POINTER(c_void_p),
                                     c_void_p]
    L.rgs_kd_splits.argtypes = [c_void_p, c_void_p, c_void_p]
    L.rgs_kd_subsets.argtypes = [c_void_p, c_void_p, c_void_p]
    L.rgs_kd_destroy.argtypes = [c_void_p]
    L.rgs_view_order.argtypes = [c_void_p, POINTER(CameraC), c_void_p]
    L.rgs_render_workspace_size.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts),
                                            c_int64, POINTER(c_size_t)]
    L.rgs_render_fwd.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts), c_void_p,
                                 c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]
    L.rgs_render_fwd_foot.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts), c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, POINTER(ctypes.c_uint64),
                                      c_void_p]
    L.rgs_render_bwd_foot.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts), c_void_p,
                                      c_void_p, POINTER(GaussianGrads), c_void_p, c_size_t, POINTER(ctypes.c_uint64),
                                      c_void_p]
    L.rgs_render_bwd.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts), c_void_p,
                                 c_void_p, c_void_p, c_void_p, POINTER(GaussianGrads), c_void_p, c_size_t, c_void_p]
    L.rgs_render_bwd_flat.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), POINTER(RenderOpts), c_void_p,
                                      c_void_p, c_void_p, POINTER(GaussianGrads), c_void_p, c_size_t, c_void_p]
    L.rgs_render_batch_fwd.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), c_int, POINTER(RenderOpts),
                                       c_void_p, c_void_p, c_size_t, c_void_p]
    L.rgs_render_batch_bwd.argtypes = [c_void_p, POINTER(Gaussians), POINTER(CameraC), c_int, POINTER(RenderOpts),
                                       c_void_p, c_void_p, POINTER(GaussianGrads), c_void_p, c_size_t, c_void_p]
    L.rgs_merge_partials.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p,
                                     c_void_p]
    L.rgs_merge_partials_bwd.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p,
                                         c_void_p, c_void_p, c_void_p, c_void_p]
    L.rgs_adam_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int, c_float,
                                c_float, c_float, c_int, c_int, c_void_p]
    L.rgs_adam_step_periodic.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_int,
                                         c_int, c_int64, c_int64, c_float, c_float, c_float, c_float, c_int, c_int,
                                         c_void_p]
    L.rgs_default_opts.argtypes = [POINTER(RenderOpts)]
    L.rgs_profile_enable.argtypes = [c_int]
    L.rgs_profile_stage_name.restype = ctypes.c_char_p
    L.rgs_profile_stage_name.argtypes = [c_int]
    L.rgs_profile_read.argtypes = [c_void_p, c_void_p, c_void_p, c_int]
    L.rgs_serve_default_config.argtypes = [POINTER(ServeConfig)]
    L.rgs_serve_default_config.restype = None
    L.rgs_serve_create_ex.argtypes = [c_void_p, POINTER(Gaussians), POINTER(RenderOpts), POINTER(ServeConfig),
                                      POINTER(c_void_p)]
    L.rgs_serve_submit.argtypes = [c_void_p, POINTER(CameraC), c_void_p, POINTER(ctypes.c_uint64)]
    L.rgs_serve_poll.argtypes = [c_void_p, ctypes.c_uint64, POINTER(c_int), POINTER(ctypes.c_double)]
    L.rgs_serve_stats_read.argtypes = [c_void_p, POINTER(ServeStats)]
    L.rgs_serve_lane_bytes.argtypes = [c_void_p, POINTER(Gaussians), POINTER(ServeConfig), c_int64, POINTER(c_size_t)]
    L.rgs_serve_destroy.argtypes = [c_void_p]
    L.rgs_serve_hold.argtypes = [c_void_p, c_int]
    L.rgs_sort_temp_bytes.restype = c_size_t
    L.rgs_sort_temp_bytes.argtypes = [c_int64]
    L.rgs_sort_pairs.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_int, c_void_p, c_size_t, c_void_p,
                                 POINTER(c_int)]
    _lib = L
    return L


def _check(rc):
    if rc != RGS_OK:
        raise RGSError(rc, lib().rgs_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def _ptr(t):
    return c_void_p(t.data_ptr()) if t is not None else c_void_p(0)


# --------------------------------------------------------------------------- conversions
def default_opts(**kw) -> RenderOpts:
    o = RenderOpts()
    lib().rgs_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                o.bg[i] = float(v[i])
        else:
            setattr(o, k, v)
    return o


def camera_c(cam) -> CameraC:
    c = CameraC()
    vm = np.asarray(cam.viewmat, np.float32).reshape(16)
    for i in range(16):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(cam.near_z)
    return c


def gaussians_c(means, log_scales, quats, opacity_logits, sh, sh_degree) -> Gaussians:
    for t in (means, log_scales, quats, opacity_logits, sh):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("splat parameters must be contiguous float32 CUDA tensors")
    return Gaussians(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                     int(means.shape[0]), int(sh_degree))


def scene_c(scene) -> Gaussians:
    return gaussians_c(scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh, scene.sh_degree)


# --------------------------------------------------------------------------- KD partition
class KD:
    """Owner of an ``rgs_kd`` handle (KD tree, leaf boxes and CSR subset lists)."""

    def __init__(self, handle: c_void_p):
        self.handle = handle
        L, K, M = c_int(), c_int(), c_int64()
        _check(lib().rgs_kd_info(handle, ctypes.byref(L), ctypes.byref(K), ctypes.byref(M)))
        self.L, self.K, self.M = L.value, K.value, M.value

    def splits(self):
        n = max(self.K - 1, 1)
        axis = np.zeros(n, np.int32)
        split = np.zeros(n, np.float32)
        _check(lib().rgs_kd_splits(self.handle, c_void_p(axis.ctypes.data), c_void_p(split.ctypes.data)))
        return axis[:self.K - 1], split[:self.K - 1]

    def subsets(self, device="cuda"):
        offsets = np.zeros(self.K + 1, np.int64)
        idx = torch.empty(max(self.M, 1), dtype=torch.int32, device=device)
        torch.cuda.synchronize()
        _check(lib().rgs_kd_subsets(self.handle, c_void_p(offsets.ctypes.data), _ptr(idx)))
        return offsets, idx[:self.M]

    def view_order(self, cam) -> np.ndarray:
        order = np.zeros(self.K, np.int32)
        c = camera_c(cam)
        _check(lib().rgs_view_order(self.handle, ctypes.byref(c), c_void_p(order.ctypes.data)))
        return order

    def __del__(self):
        try:
            if self.handle:
                lib().rgs_kd_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def kd_partition(scene, depth_L: int, trunc_mult: float = 3.0, stream=None) -> KD:
    g = scene if isinstance(scene, Gaussians) else scene_c(scene)
    h = c_void_p()
    _check(lib().rgs_kd_partition(ctypes.byref(g), int(depth_L), float(trunc_mult), ctypes.byref(h), _stream(stream)))
    return KD(h)


def kd_from_splits(scene, depth_L: int, axis, split, trunc_mult: float = 3.0, stream=None) -> KD:
    """Partition with the given planes (heap order), subsets by the D_i rule."""
    g = scene if isinstance(scene, Gaussians) else scene_c(scene)
    ax = np.ascontiguousarray(np.asarray(axis, np.int32).reshape(-1))
    sp = np.ascontiguousarray(np.asarray(split, np.float32).reshape(-1))
    if ax.size == 0:
        ax, sp = np.zeros(1, np.int32), np.zeros(1, np.float32)
    h = c_void_p()
    _check(lib().rgs_kd_from_splits(ctypes.byref(g), int(depth_L), c_void_p(ax.ctypes.data), c_void_p(sp.ctypes.data),
                                    float(trunc_mult), ctypes.byref(h), _stream(stream)))
    return KD(h)


# --------------------------------------------------------------------------- render
class Workspace:
    """Caller-owned render workspace (a CUDA byte tensor) that grows on demand."""

    def __init__(self, device="cuda", nbytes: int = 0):
        self.device = device
        self.buf = None
        if nbytes:
            self.ensure(nbytes)

    def ensure(self, nbytes: int):
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = None
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.buf

    @property
    def nbytes(self):
        return 0 if self.buf is None else self.buf.numel()

    def ptr(self):
        return c_void_p(0) if self.buf is None else c_void_p(self.buf.data_ptr())


def _retry(call, ws: Workspace):
    for _ in range(4):
        rc = call()
        if rc == RGS_EOVERFLOW:
            need = lib().rgs_last_required_workspace()
            if need and need > ws.nbytes:
                ws.ensure(int(need * 1.15) + (1 << 20))
                continue
        _check(rc)
        return
    _check(rc)


def render_fwd(kd: KD, g: Gaussians, cam, opts: RenderOpts, ws: Workspace, image=True, stream=None, out=None,
               partials=True):
    """Partial maps [K,3,H,W] / [K,H,W] and, if image, the merged image [3,H,W] and T_final.
    partials=False renders the image only (its backward: render_bwd_flat)."""
    H, W = int(cam.height), int(cam.width)
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        tiles = ((H + 15) // 16) * ((W + 15) // 16)
        out = {"tile_depth": torch.empty(tiles, kd.K, device=dev)}
        if partials:
            out["partial_C"] = torch.empty(kd.K, 3, H, W, device=dev)
            out["partial_T"] = torch.empty(kd.K, H, W, device=dev)
        if image or not partials:
            out["image"] = torch.empty(3, H, W, device=dev)
            out["T_final"] = torch.empty(H, W, device=dev)
    c = camera_c(cam)
    s = _stream(stream)
    _retry(lambda: lib().rgs_render_fwd(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                        _ptr(out.get("partial_C")), _ptr(out.get("partial_T")), _ptr(out.get("image")),
                                        _ptr(out.get("T_final")), _ptr(out.get("tile_depth")), ws.ptr(), ws.nbytes,
                                        s), ws)
    return out


def render_fwd_foot(kd: KD, g: Gaussians, cam, opts: RenderOpts, ws: Workspace, partials=True, stream=None,
                    out=None):
    """Forward render under the perpendicular-foot reading of x_i (Sec. 3.2; comparison
    mode): like render_fwd, plus "overflow", the number of contributors the per-pixel order
    buffer had to blend early (0: the per-pixel order is exact).  Its backward is
    render_bwd_foot."""
    H, W = int(cam.height), int(cam.width)
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = {"image": torch.empty(3, H, W, device=dev), "T_final": torch.empty(H, W, device=dev)}
        if partials:
            out["partial_C"] = torch.empty(kd.K, 3, H, W, device=dev)
            out["partial_T"] = torch.empty(kd.K, H, W, device=dev)
    c = camera_c(cam)
    s = _stream(stream)
    over = ctypes.c_uint64(0)
    _retry(lambda: lib().rgs_render_fwd_foot(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                             _ptr(out.get("partial_C")), _ptr(out.get("partial_T")),
                                             _ptr(out.get("image")), _ptr(out.get("T_final")), ws.ptr(), ws.nbytes,
                                             ctypes.byref(over), s), ws)
    out["overflow"] = int(over.value)
    return out


def render_bwd(kd: KD, g: Gaussians, cam, opts: RenderOpts, partial_C, partial_T, dL_dimage, grads, ws: Workspace,
               stream=None, tile_depth=None):
    """Accumulate dL/d(params) into grads = (means, log_scales, quats, opacity_logits, sh) tensors.
    `tile_depth` is the forward's per-(tile, subset) saturation depth (optional)."""
    gg = GaussianGrads(*(_ptr(t) for t in grads))
    c = camera_c(cam)
    s = _stream(stream)
    dL = dL_dimage.contiguous()
    _retry(lambda: lib().rgs_render_bwd(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                        _ptr(partial_C), _ptr(partial_T), _ptr(dL), _ptr(tile_depth), ctypes.byref(gg),
                                        ws.ptr(), ws.nbytes, s), ws)


def merge_partials(partial_C, partial_T, order, bg=(0.0, 0.0, 0.0), stream=None):
    K, _, H, W = partial_C.shape
    order_d = torch.as_tensor(np.asarray(order, np.int32), device=partial_C.device)
    image = torch.empty(3, H, W, device=partial_C.device)
    T = torch.empty(H, W, device=partial_C.device)
    bgv = (c_float * 3)(*bg)
    _check(lib().rgs_merge_partials(_ptr(partial_C), _ptr(partial_T), _ptr(order_d), K, H, W, ctypes.cast(bgv, c_void_p),
                                    _ptr(image), _ptr(T), _stream(stream)))
    torch.cuda.current_stream().synchronize()
    return image, T


def merge_partials_bwd(partial_C, partial_T, order, dL_dimage, dL_dT=None, bg=(0.0, 0.0, 0.0), stream=None):
    K, _, H, W = partial_C.shape
    order_d = torch.as_tensor(np.asarray(order, np.int32), device=partial_C.device)
    dC = torch.empty_like(partial_C)
    dT = torch.empty_like(partial_T)
    bgv = (c_float * 3)(*bg)
    _check(lib().rgs_merge_partials_bwd(_ptr(partial_C), _ptr(partial_T), _ptr(order_d), K, H, W,
                                        ctypes.cast(bgv, c_void_p), _ptr(dL_dimage.contiguous()),
                                        _ptr(dL_dT.contiguous() if dL_dT is not None else None), _ptr(dC), _ptr(dT),
                                        _stream(stream)))
    torch.cuda.current_stream().synchronize()
    return dC, dT


def sort_pairs(keys, vals, end_bit, stream=None):
    """Stable radix sort of int32 device tensors (uint32 bit patterns) whose keys are all
    below 2**end_bit; returns the sorted (keys, vals) (new tensors)."""
    n = int(keys.numel())
    if int(vals.numel()) != n:
        raise ValueError("sort_pairs: keys and values differ in length")
    ka, va = keys.contiguous().clone(), vals.contiguous().clone()
    kb, vb = torch.empty_like(ka), torch.empty_like(va)
    temp = torch.empty(int(lib().rgs_sort_temp_bytes(n)), dtype=torch.uint8, device=keys.device)
    alt = ctypes.c_int(0)
    _check(lib().rgs_sort_pairs(_ptr(ka), _ptr(va), _ptr(kb), _ptr(vb), n, int(end_bit), _ptr(temp), temp.numel(),
                                _stream(stream), ctypes.byref(alt)))
    torch.cuda.current_stream().synchronize()
    return (kb, vb) if alt.value else (ka, va)


def adam_step(param, grad, m, v, seg_offsets, seg_lr, step, beta1=0.9, beta2=0.999, eps=1e-15, zero_grad=True,
              stream=None, periodic=None):
    """One Adam step over flat buffers split into segments with their own rates.
    periodic = (segment, period, head, head_lr): inside that segment, elements whose offset
    from its start is below `head` modulo `period` take head_lr."""
    offs = np.asarray(seg_offsets, np.int64)
    lrs = np.asarray(seg_lr, np.float32)
    pseg, period, head, head_lr = periodic if periodic is not None else (-1, 1, 0, 0.0)
    _check(lib().rgs_adam_step_periodic(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(param.numel()),
                                        c_void_p(offs.ctypes.data), c_void_p(lrs.ctypes.data), len(lrs), int(pseg),
                                        int(period), int(head), float(head_lr), float(beta1), float(beta2),
                                        float(eps), int(step), 1 if zero_grad else 0, _stream(stream)))


def position_lr(step, max_steps, lr_init=1.6e-4, lr_final=1.6e-6) -> float:
    return float(lib().rgs_position_lr(int(step), int(max_steps), float(lr_init), float(lr_final)))


def render_bwd_flat(kd: KD, g: Gaussians, cam, opts: RenderOpts, image, dL_dimage, grads, ws: Workspace,
                    stream=None, tile_depth=None):
    """Flat-form backward (one front-to-back replay per pixel over the concatenated subset
    lists, from the forward's image; no partial maps).  Accumulates into grads like
    render_bwd."""
    gg = GaussianGrads(*(_ptr(t) for t in grads))
    c = camera_c(cam)
    s = _stream(stream)
    dL = dL_dimage.contiguous()
    _retry(lambda: lib().rgs_render_bwd_flat(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                             _ptr(image), _ptr(dL), _ptr(tile_depth), ctypes.byref(gg), ws.ptr(),
                                             ws.nbytes, s), ws)


def render_bwd_foot(kd: KD, g: Gaussians, cam, opts: RenderOpts, image, dL_dimage, grads, ws: Workspace,
                    stream=None):
    """Backward of render_fwd_foot (flat form, the foot reading's per-pixel order), from the
    forward's image (rendered without partial maps).  Accumulates into grads like
    render_bwd; returns the order buffer's overflow count."""
    gg = GaussianGrads(*(_ptr(t) for t in grads))
    c = camera_c(cam)
    s = _stream(stream)
    dL = dL_dimage.contiguous()
    over = ctypes.c_uint64(0)
    _retry(lambda: lib().rgs_render_bwd_foot(kd.handle, ctypes.byref(g), ctypes.byref(c), ctypes.byref(opts),
                                             _ptr(image), _ptr(dL), ctypes.byref(gg), ws.ptr(), ws.nbytes,
                                             ctypes.byref(over), s), ws)
    return int(over.value)


def _cams_c(cams):
    arr = (CameraC * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_c(c)
    return arr


def _ptrs(tensors):
    arr = (c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = t.data_ptr()
    return arr


def render_batch_fwd(kd: KD, g: Gaussians, cams, opts: RenderOpts, ws: Workspace, stream=None, images=None):
    """Images [3,H,W] of several views of one scene through one launch sequence (the
    batched training forward); the lists stay in `ws` for render_batch_bwd."""
    dev = torch.device("cuda", torch.cuda.current_device())
    if images is None:
        images = [torch.empty(3, int(c.height), int(c.width), device=dev) for c in cams]
    cc, ip = _cams_c(cams), _ptrs(images)
    s = _stream(stream)
    _retry(lambda: lib().rgs_render_batch_fwd(kd.handle, ctypes.byref(g), cc, len(cams), ctypes.byref(opts),
                                              ctypes.cast(ip, c_void_p), ws.ptr(), ws.nbytes, s), ws)
    return images


def render_batch_bwd(kd: KD, g: Gaussians, cams, opts: RenderOpts, images, dL_dimages, grads, ws: Workspace,
                     stream=None):
    """Flat backward of every view of render_batch_fwd in one launch sequence; accumulates
    into grads = (means, log_scales, quats, opacity_logits, sh)."""
    gg = GaussianGrads(*(_ptr(t) for t in grads))
    dls = [d.contiguous() for d in dL_dimages]
    cc, ip, dp = _cams_c(cams), _ptrs(images), _ptrs(dls)
    s = _stream(stream)
    _retry(lambda: lib().rgs_render_batch_bwd(kd.handle, ctypes.byref(g), cc, len(cams), ctypes.byref(opts),
                                              ctypes.cast(ip, c_void_p), ctypes.cast(dp, c_void_p), ctypes.byref(gg),
                                              ws.ptr(), ws.nbytes, s), ws)


# --------------------------------------------------------------------------- tracing
def profile_enable(timing: bool = True, counters: bool = False):
    """Per-pass CUDA-event timing (cheap) and/or pair counters (counting kernel variants)."""
    _check(lib().rgs_profile_enable((1 if timing else 0) | (2 if counters else 0)))


PAIR_COUNTERS = ("fwd_pairs", "fwd_contrib", "bwd_pairs", "bwd_contrib", "instances", "visible", "kernel_launches",
                 "fwd_fail_d2", "fwd_fail_ball", "fwd_fail_subset", "fwd_pairs_straddling", "fwd_instances_staged",
                 "fwd_instances_used", "fwd_warp_iterations", "fwd_pairs_behind_front", "bwd_warp_iterations")


def profile_read(reset: bool = True) -> dict:
    """Per-stage milliseconds and pass counts since the last reset, plus the pair/instance
    counters: {"stages": {name: (ms, launches)}, "counters": {...}}."""
    L = lib()
    n = L.rgs_profile_num_stages()
    ms = np.zeros(n, np.float64)
    launches = np.zeros(n, np.int64)
    counters = np.zeros(len(PAIR_COUNTERS), np.int64)
    _check(L.rgs_profile_read(c_void_p(ms.ctypes.data), c_void_p(launches.ctypes.data),
                              c_void_p(counters.ctypes.data), 1 if reset else 0))
    stages = {L.rgs_profile_stage_name(i).decode(): (float(ms[i]), int(launches[i])) for i in range(n)}
    return {"stages": stages, "counters": dict(zip(PAIR_COUNTERS, (int(c) for c in counters)))}


# --------------------------------------------------------------------------- serving
def serve_config(mem_budget_bytes=8 << 30, max_slots=8, lanes=2, plain=False, max_width=4096, max_height=4096,
                 max_queue=65536, inst_per_pixel=16.0, group_per_splat=12.0,
                 group_min_instances=float(1 << 24), batch_max_pixels=1 << 21) -> ServeConfig:
    cfg = ServeConfig()
    lib().rgs_serve_default_config(ctypes.byref(cfg))
    cfg.mem_budget_bytes = int(mem_budget_bytes)
    cfg.max_slots, cfg.lanes, cfg.plain = int(max_slots), int(lanes), 1 if plain else 0
    cfg.max_width, cfg.max_height, cfg.max_queue = int(max_width), int(max_height), int(max_queue)
    cfg.inst_per_pixel = float(inst_per_pixel)
    cfg.group_per_splat = float(group_per_splat)
    cfg.group_min_instances = float(group_min_instances)
    cfg.batch_max_pixels = int(batch_max_pixels)
    return cfg


def serve_lane_bytes(kd: KD, g: Gaussians, instance_capacity: int, **cfg_kw) -> int:
    """Device bytes of one batched lane holding `instance_capacity` tile instances."""
    cfg = serve_config(**cfg_kw)
    n = c_size_t()
    _check(lib().rgs_serve_lane_bytes(kd.handle, ctypes.byref(g), ctypes.byref(cfg), int(instance_capacity),
                                      ctypes.byref(n)))
    return int(n.value)


class Server:
    """Render server over a resident scene (rgs_serve_*).  The scene tensors behind `g` and
    the KD must stay alive while the server does; output images are caller-owned."""

    def __init__(self, kd: KD, g: Gaussians, opts: RenderOpts, mem_budget_bytes: int, max_slots: int = 8,
                 lanes: int = 2, plain: bool = False, max_width: int = 4096, max_height: int = 4096,
                 max_queue: int = 65536, inst_per_pixel: float = 16.0, group_per_splat: float = 12.0,
                 group_min_instances: float = float(1 << 24), batch_max_pixels: int = 1 << 21, keepalive=None):
        L = lib()
        cfg = serve_config(mem_budget_bytes, max_slots, lanes, plain, max_width, max_height, max_queue, inst_per_pixel,
                           group_per_splat, group_min_instances, batch_max_pixels)
        self._keep = (kd, g, opts, keepalive)
        self._g, self._opts = g, opts
        h = c_void_p()
        _check(L.rgs_serve_create_ex(kd.handle, ctypes.byref(g), ctypes.byref(opts), ctypes.byref(cfg),
                                     ctypes.byref(h)))
        self.handle = h
        self.outputs = {}

    def submit(self, cam, out) -> int:
        """Queue a render of cam into out ([3,H,W] float32 cuda tensor); returns the ticket."""
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert tuple(out.shape) == (3, int(cam.height), int(cam.width))
        c = camera_c(cam)
        t = ctypes.c_uint64()
        _check(lib().rgs_serve_submit(self.handle, ctypes.byref(c), _ptr(out), ctypes.byref(t)))
        self.outputs[t.value] = out
        return t.value

    def poll(self, ticket):
        """(done, latency_ms); raises RGSError if the request failed."""
        done = c_int(0)
        lat = ctypes.c_double(0.0)
        rc = lib().rgs_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(done), ctypes.byref(lat))
        if done.value:
            self.outputs.pop(ticket, None)
        _check(rc)
        return bool(done.value), float(lat.value)

    def wait(self, ticket, timeout_s: float = 60.0):
        """Poll until done (bounded); returns the latency in ms."""
        import time
        t0 = time.monotonic()
        while True:
            done, lat = self.poll(ticket)
            if done:
                return lat
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not done after {timeout_s} s")
            time.sleep(0.0002)

    def hold(self, on: bool = True):
        """Pause (True) or resume (False) the start of new batches."""
        _check(lib().rgs_serve_hold(self.handle, 1 if on else 0))

    def stats(self) -> dict:
        st = ServeStats()
        _check(lib().rgs_serve_stats_read(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            h, self.handle = self.handle, None
            _check(lib().rgs_serve_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


ABI_SYMBOLS = ("rgs_last_error", "rgs_last_required_workspace", "rgs_version", "rgs_default_opts", "rgs_kd_partition",
               "rgs_kd_info", "rgs_kd_from_splits", "rgs_kd_splits", "rgs_kd_subsets", "rgs_kd_destroy", "rgs_view_order",
               "rgs_render_workspace_size", "rgs_render_fwd", "rgs_render_fwd_foot", "rgs_merge_partials", "rgs_merge_partials_bwd",
               "rgs_render_bwd", "rgs_render_bwd_flat", "rgs_render_bwd_foot", "rgs_render_batch_fwd", "rgs_render_batch_bwd", "rgs_adam_step", "rgs_adam_step_periodic", "rgs_position_lr", "rgs_profile_enable",
               "rgs_profile_num_stages", "rgs_profile_stage_name", "rgs_profile_read", "rgs_render_fwd_noalloc",
               "rgs_serve_default_config", "rgs_serve_create", "rgs_serve_create_ex", "rgs_serve_submit",
               "rgs_serve_poll", "rgs_serve_stats_read", "rgs_serve_destroy", "rgs_serve_lane_bytes",
               "rgs_serve_hold", "rgs_sort_temp_bytes", "rgs_sort_pairs")
