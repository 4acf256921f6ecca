"""GB300-native hot path of On-the-Fly GS (arxiv 2503.13086): Python binding of the C ABI.

Argument marshalling only: every step of the rasterizer, loss, backward and optimizer runs in
the CUDA library ``_build/libgs_gb300.so`` (sources in ``csrc/``, ABI in ``include/gs.h``).
PyTorch supplies device memory and streams.  There is no CPU fallback: importing works without
a GPU, but every call needs the compiled library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["GSError", "load", "build", "Camera", "Raster", "Field", "FieldConfig", "Tiling", "adam_step", "NPARAM",
           "SYMBOLS", "library_path", "tiling_candidates"]

NPARAM = 59
MAX_TILINGS = 16
_lock = threading.Lock()
_lib = None


class GSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gs status {status}: {msg}")
        self.status = status


def build(force=False, verbose=False):
    return _build.build(force=force, verbose=verbose)


def library_path():
    return _build.LIB


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]

    @classmethod
    def of(cls, d):
        if isinstance(d, Camera):
            return d
        c = cls()
        R = np.asarray(d["R"], np.float32).reshape(9)
        t = np.asarray(d["t"], np.float32).reshape(3)
        for k in range(9):
            c.R[k] = float(R[k])
        for k in range(3):
            c.t[k] = float(t[k])
        c.fx, c.fy, c.cx, c.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
        c.width, c.height = int(d["width"]), int(d["height"])
        return c


class Tiling(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("batch", ctypes.c_int32)]

    def astuple(self):
        return (self.tile_w, self.tile_h, self.batch)


class LossWeights(ctypes.Structure):
    _fields_ = [("lambda_l1", ctypes.c_float), ("lambda_ssim", ctypes.c_float), ("lambda_load", ctypes.c_float)]


class AutotuneResult(ctypes.Structure):
    _fields_ = [("chosen", Tiling), ("n_candidates", ctypes.c_int32), ("candidates", Tiling * MAX_TILINGS),
                ("ms", ctypes.c_float * MAX_TILINGS)]


class FieldConfig(ctypes.Structure):
    _fields_ = [("T_I", ctypes.c_int32), ("N_m", ctypes.c_int32), ("T_a", ctypes.c_int32),
                ("batch_views", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("async_steps", ctypes.c_int32),
                ("eta0", ctypes.c_float), ("etaf", ctypes.c_float), ("lambda_ssim", ctypes.c_float),
                ("lr_scale", ctypes.c_float), ("lr_rot", ctypes.c_float), ("lr_opacity", ctypes.c_float),
                ("lr_sh_dc", ctypes.c_float), ("lr_sh_rest", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("adam_eps", ctypes.c_float),
                ("add_dist_thresh", ctypes.c_float), ("scene_extent", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("seed", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_uint64), ("initial_capacity", ctypes.c_int64),
                ("tiling", Tiling), ("batch_scaling", ctypes.c_int32), ("lambda_l1", ctypes.c_float),
                ("lambda_load", ctypes.c_float), ("densify_stats", ctypes.c_int32),
                ("sparse_adam", ctypes.c_int32), ("debug_canaries", ctypes.c_int32)]


class DensifyParams(ctypes.Structure):
    _fields_ = [("grad_thresh", ctypes.c_float), ("percent_dense", ctypes.c_float), ("min_opacity", ctypes.c_float),
                ("max_scale", ctypes.c_float)]


class DensifyResult(ctypes.Structure):
    _fields_ = [("n_before", ctypes.c_int64), ("n_after", ctypes.c_int64), ("cloned", ctypes.c_int64),
                ("split", ctypes.c_int64), ("pruned", ctypes.c_int64)]


class IntegrateStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("steps", ctypes.c_int32), ("key_images", ctypes.c_int32),
                ("new_gaussians", ctypes.c_int32), ("mean_loss", ctypes.c_double), ("pairs", ctypes.c_uint64)]


class FieldInfo(ctypes.Structure):
    _fields_ = [("n_gaussians", ctypes.c_int64), ("capacity", ctypes.c_int64), ("n_images", ctypes.c_int64),
                ("adam_step", ctypes.c_int64), ("bytes_in_use", ctypes.c_uint64), ("last_pairs", ctypes.c_uint64),
                ("last_blended", ctypes.c_uint64), ("last_instances", ctypes.c_int64), ("last_kernels", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("last_loss", ctypes.c_double), ("last_load_std", ctypes.c_double),
                ("last_tiling", Tiling), ("pad2", ctypes.c_int32), ("last_run_ms", ctypes.c_double),
                ("last_run_steps", ctypes.c_int64), ("last_h2d_bytes", ctypes.c_uint64),
                ("last_d2h_bytes", ctypes.c_uint64)]


P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
F32 = ctypes.c_float

# Every entry point of include/gs.h with its argument types.
SYMBOLS = {
    "gs_last_error": ([], ctypes.c_char_p),
    "gs_version": ([], ctypes.c_char_p),
    "gs_raster_create": ([P], I32),
    "gs_raster_destroy": ([P], I32),
    "gs_raster_forward": ([P, P, P, I64, I64, P, ctypes.c_int, P, P, P, P, P, P], I32),
    "gs_raster_loss": ([P, P, P, P, P, P, P], I32),
    "gs_raster_backward": ([P, P, P, P, P, P, P, P], I32),
    "gs_adam_step": ([P, P, P, P, P, I64, I64, P, F32, F32, F32, I64], I32),
    "gs_raster_read": ([P, ctypes.c_int, P, ctypes.c_size_t, P], I32),
    "gs_raster_set_timing": ([P, ctypes.c_int], I32),
    "gs_raster_kernel_times": ([P, P], I32),
    "gs_tiling_candidates": ([P, I32, P], I32),
    "gs_raster_set_tiling": ([P, P], I32),
    "gs_field_config_default": ([P], None),
    "gs_field_init": ([P, P, P], I32),
    "gs_field_destroy": ([P], I32),
    "gs_field_set_gaussians": ([P, P, I64, I64], I32),
    "gs_field_get_gaussians": ([P, P, P, P, I64, P], I32),
    "gs_add_image": ([P, P, P, ctypes.c_int, P, P, I32, P, P], I32),
    "gs_add_image_chw": ([P, P, P, ctypes.c_int, P, P, I32, P, P], I32),
    "gs_set_image": ([P, I32, P, P, ctypes.c_int], I32),
    "gs_set_image_chw": ([P, I32, P, P, ctypes.c_int], I32),
    "gs_select_neighbors": ([P, I32, I32, P, P, P], I32),
    "gs_optimize_step": ([P, P, I32, P], I32),
    "gs_integrate": ([P, I32, P], I32),
    "gs_initial_training": ([P, I32, I32, P], I32),
    "gs_render": ([P, P, P, P], I32),
    "gs_field_stats": ([P, P, P], I32),
    "gs_field_info_get": ([P, P], I32),
    "gs_image_info": ([P, I32, P, P, I32], I32),
    "gs_image_lr": ([P, I32, P], I32),
    "gs_field_snapshot": ([P], I32),
    "gs_field_restore": ([P], I32),
    "gs_field_set_timing": ([P, ctypes.c_int], I32),
    "gs_field_kernel_times": ([P, P, P], I32),
    "gs_field_autotune": ([P, P, I32, I32, P], I32),
    "gs_autotune_clear": ([], I32),
    "gs_field_save": ([P, ctypes.c_char_p], I32),
    "gs_field_load": ([ctypes.c_char_p, P, P], I32),
    "gs_scan_noalloc": ([P, P, I64, P, P], I32),
    "gs_field_densify": ([P, P, P], I32),
    "gs_field_densify_stats": ([P, P, P], I32),
    "gs_wait_probe": ([ctypes.c_uint32, P, P], I32),
    "gs_loss_wait_probe": ([ctypes.c_uint32, P, P], I32),
    "gs_field_corrupt_guard": ([P, I32, P, I32], I32),
    "gs_schedule_plan": ([P, P, P, I32, I32, P, P, P, P, P, P], I32),
}

KERNEL_NAMES = ["K1 project", "K2 scan", "K3 emit", "K4 sort", "K5 ranges", "K6 blend fwd", "K7 loss",
                "K8 blend bwd", "K9+K10 project bwd/adam"]


def load(build_if_missing=True):
    """Load the CUDA library (building it in-tree if needed).  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path}")
            path = _build.build()
        lib = ctypes.CDLL(path)
        for name, (args, res) in SYMBOLS.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status):
    if status != 0:
        raise GSError(status, load().gs_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required (the library has no CPU path)")
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _cams(cams):
    arr = (Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = Camera.of(c)
    return arr


def _sizes(cams):
    return [(int(Camera.of(c).width), int(Camera.of(c).height)) for c in cams]


def _check_params(params):
    torch = _torch()
    if not (params.is_cuda and params.dtype == torch.float32 and params.dim() == 2 and params.shape[0] == NPARAM
            and params.is_contiguous()):
        raise ValueError("params must be a contiguous float32 CUDA tensor of shape (59, stride)")
    if params.shape[1] % 32:
        raise ValueError("stride must be a multiple of 32")


class Raster:
    """Stateless rasterizer calls (K1-K9) on torch tensors.  See gs.h for the semantics."""

    def __init__(self):
        self._lib = load()
        h = ctypes.c_void_p()
        _check(self._lib.gs_raster_create(ctypes.byref(h)))
        self._h = h
        self._sizes = None
        self.generation = 0  # bumped by every forward (the workspace keeps only the latest one)

    def close(self):
        if self._h:
            self._lib.gs_raster_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, params, n, cams, bg=(0.0, 0.0, 0.0), want_T=True, want_gp=True, stream=None):
        torch = _torch()
        _check_params(params)
        sizes = _sizes(cams)
        npix = sum(w * h for w, h in sizes)
        dev = params.device
        image = torch.empty(3 * npix, device=dev, dtype=torch.float32)
        T = torch.empty(npix, device=dev, dtype=torch.float32) if want_T else None
        last = torch.empty(npix, device=dev, dtype=torch.int32)
        gp = torch.empty(npix, device=dev, dtype=torch.int32) if want_gp else None
        pairs = ctypes.c_uint64()
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        _check(self._lib.gs_raster_forward(self._h, _stream(stream), _ptr(params), int(n), params.shape[1],
                                           _cams(cams), len(cams), bgv, _ptr(image), _ptr(T), _ptr(last), _ptr(gp),
                                           ctypes.byref(pairs)))
        self._sizes = sizes
        self.generation += 1
        return dict(image=image, T=T, last=last, gp=gp, pairs=int(pairs.value), sizes=sizes)

    def loss(self, image, target, lambda_ssim=0.2, want_grad=True, stream=None, lambda_l1=None, lambda_load=0.0):
        """Eq. 10 on the last forward's views; lambda_l1 defaults to 1 - lambda_ssim."""
        torch = _torch()
        dimage = torch.empty_like(image) if want_grad else None
        out = ctypes.c_double()
        w = LossWeights(1.0 - lambda_ssim if lambda_l1 is None else lambda_l1, lambda_ssim, lambda_load)
        _check(self._lib.gs_raster_loss(self._h, _stream(stream), _ptr(image), _ptr(target.contiguous()),
                                        ctypes.byref(w), _ptr(dimage), ctypes.byref(out)))
        return float(out.value), dimage

    def backward(self, params, image, last, dimage, want_grad2d=False, stream=None):
        torch = _torch()
        grads = torch.zeros_like(params)
        grad2d = None
        if want_grad2d:
            grad2d = torch.zeros(len(self._sizes) * params.shape[1] * 9, device=params.device, dtype=torch.float32)
        _check(self._lib.gs_raster_backward(self._h, _stream(stream), _ptr(params), _ptr(image), _ptr(last),
                                            _ptr(dimage.contiguous()), _ptr(grads), _ptr(grad2d)))
        return grads, grad2d

    def read(self, which, dtype):
        nbytes = ctypes.c_size_t()
        _check(self._lib.gs_raster_read(self._h, int(which), None, 0, ctypes.byref(nbytes)))
        buf = np.empty(nbytes.value // np.dtype(dtype).itemsize, dtype=dtype)
        _check(self._lib.gs_raster_read(self._h, int(which), buf.ctypes.data_as(ctypes.c_void_p), buf.nbytes,
                                        ctypes.byref(nbytes)))
        return buf

    def set_tiling(self, tile_w, tile_h, batch):
        t = Tiling(int(tile_w), int(tile_h), int(batch))
        _check(self._lib.gs_raster_set_tiling(self._h, ctypes.byref(t)))

    def set_timing(self, on=True):
        _check(self._lib.gs_raster_set_timing(self._h, 1 if on else 0))

    def kernel_times(self):
        out = (ctypes.c_float * 9)()
        _check(self._lib.gs_raster_kernel_times(self._h, out))
        return list(out)


def adam_step(params, grads, m, v, n, lrs, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    lib = load()
    lr = (ctypes.c_float * 6)(*[float(x) for x in lrs])
    _check(lib.gs_adam_step(_stream(stream), _ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(n), params.shape[1], lr,
                            float(beta1), float(beta2), float(eps), int(step)))


def tiling_candidates():
    """The compiled (tile_w, tile_h, batch) combinations; the first is the default."""
    lib = load()
    arr = (Tiling * MAX_TILINGS)()
    n = ctypes.c_int32()
    _check(lib.gs_tiling_candidates(arr, MAX_TILINGS, ctypes.byref(n)))
    return [arr[k].astuple() for k in range(min(n.value, MAX_TILINGS))]


def autotune_clear():
    """Forget every autotuned view-set class (the cache is shared by all sessions)."""
    _check(load().gs_autotune_clear())


def wait_probe(spin_limit=0):
    """Run the scan's and the sort pass's look-back wait once each with a predecessor that never
    starts (spin_limit rounds, 0 = the steps' own limit).  Returns ((scan_error_bits, sort_error_bits),
    (scan_ms, sort_ms)); bit 0 set = the wait gave up."""
    _torch()
    err = (ctypes.c_uint32 * 2)()
    ms = (ctypes.c_float * 2)()
    _check(load().gs_wait_probe(int(spin_limit), err, ms))
    return (int(err[0]), int(err[1])), (float(ms[0]), float(ms[1]))


def loss_wait_probe(spin_limit=0):
    """Run the loss forward's two waits of a step (tile flags, blend-forward warp count) once with
    nothing that ever ends them (spin_limit polls each, 0 = the steps' own limit).  Returns
    (error_bits, ms); bit 0 set = a wait gave up."""
    _torch()
    err = ctypes.c_uint32()
    ms = ctypes.c_float()
    _check(load().gs_loss_wait_probe(int(spin_limit), ctypes.byref(err), ctypes.byref(ms)))
    return int(err.value), float(ms.value)


def schedule_plan(M, T, new_id, **config):
    """The schedule of one arrival computed on the host (no GPU): returns dict(slots, keys, w, lr) for
    overlap matrix M (n x n), iteration counts T (n) and the arriving image new_id; config fields of
    gs_field_config (T_I, N_m, seed, eta0, etaf, T_a) as keywords."""
    lib = load()
    cfg = default_config(**config)
    M = np.ascontiguousarray(M, np.float32)
    T = np.ascontiguousarray(T, np.int32)
    n = int(M.shape[0])
    slots = np.zeros(max(cfg.T_I, 1), np.int32)
    keys = np.zeros(max(cfg.N_m, 1), np.int32)
    w = np.zeros(n, np.float32)
    lr = np.zeros(n, np.float32)
    ns, nk = ctypes.c_int32(), ctypes.c_int32()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    _check(lib.gs_schedule_plan(ctypes.byref(cfg), vp(M), vp(T), n, int(new_id), vp(slots), ctypes.byref(ns),
                                vp(keys), ctypes.byref(nk), vp(w), vp(lr)))
    return dict(slots=slots[:ns.value].tolist(), keys=keys[:nk.value].tolist(), w=w, lr=lr)


def default_config(**kw):
    """Library defaults, overridden by keyword (bg=(r, g, b); tiling=(tile_w, tile_h, batch) or None
    for the autotuner)."""
    lib = load()
    cfg = FieldConfig()
    lib.gs_field_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                cfg.bg[i] = float(v[i])
        elif k == "tiling":
            t = (0, 0, 0) if v is None else tuple(int(x) for x in v)
            cfg.tiling = Tiling(*t)
        else:
            setattr(cfg, k, v)
    return cfg


class Field:
    """A session: field, Adam state and registered images resident on the device."""

    def __init__(self, config=None, stream=None, **kw):
        self._lib = load()
        _torch()
        cfg = config if config is not None else default_config(**kw)
        h = ctypes.c_void_p()
        self._stream_obj = stream
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(self._lib.gs_field_init(ctypes.byref(cfg), sp, ctypes.byref(h)))
        self._h = h
        self.config = cfg

    def close(self):
        if self._h:
            self._lib.gs_field_destroy(self._h)
            self._h = None

    def save(self, path):
        """Checkpoint the whole session to a file (see gs_field_save)."""
        _check(self._lib.gs_field_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path, stream=None):
        """A new session resumed from a file written by save()."""
        self = cls.__new__(cls)
        self._lib = load()
        _torch()
        h = ctypes.c_void_p()
        self._stream_obj = stream
        sp = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(self._lib.gs_field_load(os.fsencode(path), sp, ctypes.byref(h)))
        self._h = h
        self.config = None
        return self

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_gaussians(self, params_np, n=None):
        a = np.ascontiguousarray(params_np, np.float32)
        n = a.shape[1] if n is None else n
        _check(self._lib.gs_field_set_gaussians(self._h, a.ctypes.data_as(ctypes.c_void_p), int(n), a.shape[1]))

    def get_gaussians(self, with_adam=False):
        nn = ctypes.c_int64()
        _check(self._lib.gs_field_get_gaussians(self._h, None, None, None, 0, ctypes.byref(nn)))
        n = nn.value
        stride = max(1, n)
        p = np.zeros((NPARAM, stride), np.float32)
        m = np.zeros_like(p) if with_adam else None
        v = np.zeros_like(p) if with_adam else None
        _check(self._lib.gs_field_get_gaussians(self._h, p.ctypes.data_as(ctypes.c_void_p),
                                                m.ctypes.data_as(ctypes.c_void_p) if with_adam else None,
                                                v.ctypes.data_as(ctypes.c_void_p) if with_adam else None, stride,
                                                ctypes.byref(nn)))
        p = p[:, :n]
        if with_adam:
            return p, m[:, :n], v[:, :n]
        return p

    @staticmethod
    def _image_arg(rgb, width, height):
        """(pointer, on_device, interleaved, keep-alive) of a target image: (H, W, 3) is interleaved
        (gs_add_image / gs_set_image), (3, H, W) or flat planar (the _chw entry points)."""
        if hasattr(rgb, "data_ptr"):
            keep = rgb.contiguous()
            ptr = ctypes.c_void_p(keep.data_ptr())
            on_dev = 1 if keep.is_cuda else 0
        else:
            keep = np.ascontiguousarray(rgb, np.float32)
            ptr = keep.ctypes.data_as(ctypes.c_void_p)
            on_dev = 0
        shape = tuple(keep.shape)
        if width is None:  # size unknown here (a field loaded from a file): the shape decides
            hwc = len(shape) == 3 and shape[2] == 3 and shape[0] != 3
        elif shape == (height, width, 3):
            hwc = True
        elif shape == (3, height, width) or shape == (3 * height * width,):
            hwc = False
        else:
            raise ValueError(f"image of shape {shape} is neither ({height}, {width}, 3) nor (3, {height}, {width})")
        return ptr, on_dev, hwc, keep

    def add_image(self, cam, rgb, pts_xyz=None, pts_rgb=None, tracks=None):
        """rgb: (H, W, 3) interleaved or (3, H, W) planar float32, numpy (host) or a torch tensor."""
        cam_c = Camera.of(cam)
        ptr, on_dev, hwc, keep = self._image_arg(rgb, cam_c.width, cam_c.height)
        n_pts = 0 if pts_xyz is None else len(pts_xyz)
        xyz = np.ascontiguousarray(pts_xyz, np.float32) if n_pts else None
        prgb = np.ascontiguousarray(pts_rgb, np.float32) if n_pts else None
        tr = np.ascontiguousarray(tracks, np.int32) if (n_pts and tracks is not None) else None
        out = ctypes.c_int32()
        fn = self._lib.gs_add_image if hwc else self._lib.gs_add_image_chw
        _check(fn(self._h, ctypes.byref(cam_c), ptr, on_dev,
                  xyz.ctypes.data_as(ctypes.c_void_p) if xyz is not None else None,
                  prgb.ctypes.data_as(ctypes.c_void_p) if prgb is not None else None, n_pts,
                  tr.ctypes.data_as(ctypes.c_void_p) if tr is not None else None, ctypes.byref(out)))
        del keep
        if not hasattr(self, "_sizes"):
            self._sizes = {}
        self._sizes[out.value] = (cam_c.width, cam_c.height)
        return out.value

    def set_image(self, image_id, rgb=None, cam=None):
        """Replace a registered image's target ((H, W, 3) or (3, H, W)) and/or pose.  A pinned host
        tensor is read asynchronously (keep it unchanged until the next step returns)."""
        cam_c = Camera.of(cam) if cam is not None else None
        ptr, on_dev, hwc, keep = None, 0, False, None
        if rgb is not None:
            if cam_c is not None:
                W, H = cam_c.width, cam_c.height
            else:
                W, H = getattr(self, "_sizes", {}).get(int(image_id), (None, None))
            ptr, on_dev, hwc, keep = self._image_arg(rgb, W, H)
        self._keep_image = keep  # the asynchronous copy reads it after this call returns
        fn = self._lib.gs_set_image if hwc else self._lib.gs_set_image_chw
        _check(fn(self._h, int(image_id), ctypes.byref(cam_c) if cam_c is not None else None, ptr, on_dev))

    def select_neighbors(self, image_id, k):
        ids = (ctypes.c_int32 * (k + 1))()
        w = (ctypes.c_float * (k + 1))()
        n = ctypes.c_int32()
        _check(self._lib.gs_select_neighbors(self._h, int(image_id), int(k), ids, w, ctypes.byref(n)))
        return list(ids[:n.value]), list(w[:n.value])

    def optimize_step(self, view_ids):
        arr = (ctypes.c_int32 * len(view_ids))(*[int(v) for v in view_ids])
        loss = ctypes.c_float()
        _check(self._lib.gs_optimize_step(self._h, arr, len(view_ids), ctypes.byref(loss)))
        return float(loss.value)

    def integrate(self, image_id):
        st = IntegrateStats()
        _check(self._lib.gs_integrate(self._h, int(image_id), ctypes.byref(st)))
        return dict(iterations=st.iterations, steps=st.steps, key_images=st.key_images, mean_loss=st.mean_loss,
                    pairs=int(st.pairs))

    def initial_training(self, iterations, max_steps=30000):
        """Phase 1: iterations over the registered images with 3DGS's position-rate schedule."""
        st = IntegrateStats()
        _check(self._lib.gs_initial_training(self._h, int(iterations), int(max_steps), ctypes.byref(st)))
        return dict(iterations=st.iterations, steps=st.steps, mean_loss=st.mean_loss, pairs=int(st.pairs))

    def densify(self, grad_thresh=2e-4, percent_dense=0.01, min_opacity=0.005, max_scale=0.1):
        """3DGS's clone / split / prune on the accumulated statistics (needs densify_stats=1)."""
        prm = DensifyParams(grad_thresh, percent_dense, min_opacity, max_scale)
        res = DensifyResult()
        _check(self._lib.gs_field_densify(self._h, ctypes.byref(prm), ctypes.byref(res)))
        return {k: getattr(res, k) for k, _ in DensifyResult._fields_}

    def densify_stats(self):
        """(norm sums, counts) accumulated since the last densification, numpy (n,) each."""
        n = self.stats()["n_gaussians"]
        a = np.zeros(max(n, 1), np.float32)
        c = np.zeros(max(n, 1), np.float32)
        _check(self._lib.gs_field_densify_stats(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                c.ctypes.data_as(ctypes.c_void_p)))
        return a[:n], c[:n]

    def corrupt_guard(self, index):
        """Overwrite one guard word behind the index-th allocated device buffer of the session (host-side
        fault injection for the debug_canaries check); returns the buffer's name."""
        name = ctypes.create_string_buffer(64)
        _check(self._lib.gs_field_corrupt_guard(self._h, int(index), name, 64))
        return name.value.decode()

    def render(self, cam, want_T=False):
        torch = _torch()
        c = Camera.of(cam)
        img = torch.empty((3, c.height, c.width), device="cuda", dtype=torch.float32)
        T = torch.empty((c.height, c.width), device="cuda", dtype=torch.float32) if want_T else None
        s = torch.cuda.current_stream()
        s.synchronize()
        _check(self._lib.gs_render(self._h, ctypes.byref(c), _ptr(img), _ptr(T)))
        return (img, T) if want_T else img

    def stats(self):
        """gs_field_info_get as a dict (size, memory, and the last step's and run's bookkeeping)."""
        st = FieldInfo()
        _check(self._lib.gs_field_info_get(self._h, ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in FieldInfo._fields_}
        out["last_tiling"] = st.last_tiling.astuple()
        return out

    def footprint(self):
        """(Gaussians, device bytes in use) by gs_field_stats."""
        n, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.gs_field_stats(self._h, ctypes.byref(n), ctypes.byref(b)))
        return int(n.value), int(b.value)

    def autotune(self, view_ids, reps=3):
        """Time every compiled tiling on these views; returns the choice and ms per candidate."""
        arr = (ctypes.c_int32 * len(view_ids))(*[int(v) for v in view_ids])
        res = AutotuneResult()
        _check(self._lib.gs_field_autotune(self._h, arr, len(view_ids), int(reps), ctypes.byref(res)))
        n = min(res.n_candidates, MAX_TILINGS)
        return dict(chosen=res.chosen.astuple(),
                    candidates=[(res.candidates[k].astuple(), float(res.ms[k])) for k in range(n)])

    def image_info(self, image_id, n_images):
        T = ctypes.c_int32()
        row = (ctypes.c_float * max(1, n_images))()
        _check(self._lib.gs_image_info(self._h, int(image_id), ctypes.byref(T), row, n_images))
        return T.value, list(row[:n_images])

    def image_lr(self, image_id):
        out = ctypes.c_float()
        _check(self._lib.gs_image_lr(self._h, int(image_id), ctypes.byref(out)))
        return float(out.value)

    def snapshot(self):
        _check(self._lib.gs_field_snapshot(self._h))

    def restore(self):
        _check(self._lib.gs_field_restore(self._h))

    def set_timing(self, on=True):
        _check(self._lib.gs_field_set_timing(self._h, 1 if on else 0))

    def kernel_times(self):
        out = (ctypes.c_float * 9)()
        steps = ctypes.c_int64()
        _check(self._lib.gs_field_kernel_times(self._h, out, ctypes.byref(steps)))
        return list(out), steps.value
