"""Python binding of libfdgs.so: argument marshalling only.

Every step of the rendering path runs in the library's CUDA kernels; this module passes
device pointers (from CUDA torch tensors), camera structs and the current torch stream.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfdgs.so")

FDGS_OK = 0
_STATUS = {0: "OK", -1: "INVALID", -2: "CUDA", -3: "OOM", -4: "CAPACITY", -5: "TIMEOUT",
           -6: "STATE"}


class FdgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fdgs error {code} ({_STATUS.get(code, '?')}): {msg}")
        self.code = code


class fdgs_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int),
                ("mean4", ctypes.c_void_p), ("logscale4", ctypes.c_void_p),
                ("q_left", ctypes.c_void_p), ("q_right", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class fdgs_camera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("znear", ctypes.c_float)]


class fdgs_adam_opts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 7), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class fdgs_render_opts(ctypes.Structure):
    _fields_ = [("use_mask", ctypes.c_int), ("bg", ctypes.c_float * 3), ("tile_sets", ctypes.c_int),
                ("no_temporal_cull", ctypes.c_int)]


class fdgs_frame_stats(ctypes.Structure):
    _fields_ = [("n_active", ctypes.c_int64), ("n_visible", ctypes.c_int64),
                ("n_keys", ctypes.c_int64), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("tiles_x", ctypes.c_int), ("tiles_y", ctypes.c_int), ("key_l", ctypes.c_int),
                ("key_r", ctypes.c_int), ("key_bytes", ctypes.c_int),
                ("list_builder", ctypes.c_int)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "fdgs_create_scene": [ctypes.POINTER(fdgs_scene_desc), ctypes.POINTER(_P)],
    "fdgs_destroy_scene": [_P],
    "fdgs_update_scene": [_P, ctypes.POINTER(fdgs_scene_desc)],
    "fdgs_set_active_mask": [_P, _P, ctypes.POINTER(ctypes.c_float), ctypes.c_int, _P],
    "fdgs_render": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_float,
                    ctypes.POINTER(fdgs_render_opts), _P, ctypes.POINTER(_P), _P],
    "fdgs_render_async": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_float,
                          ctypes.POINTER(fdgs_render_opts), _P, _P],
    "fdgs_reserve_render_lists": [_P, ctypes.c_uint64],
    "fdgs_render_backward": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "fdgs_frame_release": [_P],
    "fdgs_frame_get_stats": [_P, ctypes.POINTER(fdgs_frame_stats)],
    "fdgs_frame_export": [_P, _P, _P, _P, _P, _P, _P, _P],
    "fdgs_render_batch": [_P, ctypes.POINTER(fdgs_camera), ctypes.POINTER(ctypes.c_float),
                          ctypes.c_int, ctypes.POINTER(fdgs_render_opts),
                          ctypes.POINTER(_P), _P],
    "fdgs_variation_score": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_int,
                             ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int, _P, _P],
    "fdgs_variation_score_variant": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _P, _P],
    "fdgs_variation_score_add": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, _P, _P],
    "fdgs_select_keep": [_P, _P, ctypes.c_int64, ctypes.c_float, _P, _P],
    "fdgs_select_keep_noalloc": [_P, ctypes.c_int64, ctypes.c_float, _P, _P],
    "fdgs_status_sync": [_P],
    "fdgs_profile_enable": [_P, ctypes.c_int],
    "fdgs_set_blend_shape": [ctypes.c_int],
    "fdgs_set_list_builder": [ctypes.c_int],
    "fdgs_batch_autotune": [_P, ctypes.POINTER(fdgs_camera), ctypes.POINTER(ctypes.c_float),
                            ctypes.c_int, ctypes.POINTER(fdgs_render_opts), ctypes.POINTER(_P),
                            _P],
    "fdgs_batch_info": [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int,
                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                        ctypes.POINTER(ctypes.c_float)],
    "fdgs_profile_read": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint64)],
    "fdgs_batch_counts": [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                          ctypes.POINTER(ctypes.c_uint64)],
    "fdgs_set_batch_list_capacity": [_P, ctypes.c_uint64],
    "fdgs_batch_tile_lists": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32),
                              ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint64,
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
    "fdgs_set_sh_codebook": [_P, _P, ctypes.c_int, _P],
    "fdgs_build_keyframe_masks": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_float), ctypes.c_int, _P, _P],
    "fdgs_debug_inject": [ctypes.c_int, ctypes.c_int64],
    "fdgs_set_batch_staging": [ctypes.c_int],
    "fdgs_set_batch_shape": [_P, ctypes.c_int, ctypes.c_int],
    "fdgs_finetune_step": [_P, ctypes.POINTER(fdgs_camera), ctypes.c_float,
                           ctypes.POINTER(fdgs_render_opts), _P, ctypes.POINTER(fdgs_adam_opts),
                           _P, _P],
    "fdgs_finetune_reset": [_P],
    "fdgs_measure_fp32_peak": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P],
}
# score variants of fdgs_variation_score_variant (Table 4 of the paper: f, b, c, d, e)
SCORE_VARIANTS = {"full": 0, "spatial": 1, "temporal": 2, "first_derivative": 3, "sigma_t": 4}
# fdgs_debug_inject kinds
INJECT_NONE, INJECT_SPIN_LIMIT, INJECT_WITHHOLD_PUBLISH, INJECT_FAIL_ALLOCS = 0, 1, 2, 3
INJECT_TMA_MISSING_ARRIVAL = 4
PROFILE_STAGES = ("preprocess", "depth_sort", "gather_scan", "host_sync", "tile_scan", "emit",
                  "tile_sort", "blend", "backward_blend", "backward_gauss")
BATCH_STAGES = ("preprocess", "depth_sort", "gather", "tile_scan", "lists", "queue_sort",
                "blend")

_lib = None


def lib():
    """Load libfdgs.so (built by ``paper_2503_16422_gb300.build``); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2503_16422_gb300.build.build()"
                               " (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.fdgs_last_error.restype = ctypes.c_char_p
        L.fdgs_last_error.argtypes = []
        L.fdgs_version.restype = ctypes.c_char_p
        L.fdgs_version.argtypes = []
        _lib = L
    return _lib


def check(rc):
    if rc != FDGS_OK:
        raise FdgsError(rc, lib().fdgs_last_error().decode())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_camera(cam) -> fdgs_camera:
    """fdgs_camera from an object with viewmat (4x4), fx, fy, cx, cy, width, height, znear."""
    c = fdgs_camera()
    vm = np.asarray(cam.viewmat, np.float32).reshape(16)
    for k in range(16):
        c.viewmat[k] = float(vm[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.znear = int(cam.width), int(cam.height), float(cam.znear)
    return c


# numpy image of fdgs_camera (same fields, same 4-byte packing), for marshalling many
# cameras without building one ctypes structure each
_CAM_DTYPE = np.dtype([("viewmat", np.float32, (16,)), ("fx", np.float32), ("fy", np.float32),
                       ("cx", np.float32), ("cy", np.float32), ("width", np.int32),
                       ("height", np.int32), ("znear", np.float32)])
assert _CAM_DTYPE.itemsize == ctypes.sizeof(fdgs_camera)


def make_cameras(cams):
    """Array of fdgs_camera for a list of cameras, as (numpy record array, ctypes pointer);
    keep the array alive while the pointer is in use."""
    n = len(cams)
    arr = np.zeros(max(n, 1), dtype=_CAM_DTYPE)
    if n:
        arr["viewmat"][:n] = np.asarray([c.viewmat for c in cams], np.float32).reshape(n, 16)
        for f in ("fx", "fy", "cx", "cy", "znear"):
            arr[f][:n] = [getattr(c, f) for c in cams]
        arr["width"][:n] = [c.width for c in cams]
        arr["height"][:n] = [c.height for c in cams]
    return arr, arr.ctypes.data_as(ctypes.POINTER(fdgs_camera))


def _times(ts):
    a = np.ascontiguousarray(np.asarray(ts, np.float32).reshape(-1))
    if a.size == 0:
        a = np.zeros(1, np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _opts(use_mask, bg, tight=False, temporal_cull=True):
    o = fdgs_render_opts()
    o.use_mask = int(bool(use_mask))
    for k in range(3):
        o.bg[k] = float(bg[k])
    o.tile_sets = int(bool(tight))
    o.no_temporal_cull = int(not temporal_cull)
    return o


def _check_param(t, shape_tail, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if shape_tail is not None and tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}")


@dataclass
class SceneTensors:
    mean4: torch.Tensor
    logscale4: torch.Tensor
    q_left: torch.Tensor
    q_right: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @staticmethod
    def from_host(scene, device="cuda"):
        def t(a):
            return torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        return SceneTensors(t(scene.mean4), t(scene.logscale4), t(scene.q_left),
                            t(scene.q_right), t(scene.opacity_logit), t(scene.sh),
                            int(scene.sh_degree))

    def list(self):
        return [self.mean4, self.logscale4, self.q_left, self.q_right, self.opacity_logit,
                self.sh]


class Frame:
    """Per-render state kept for the backward (fdgs_frame)."""

    def __init__(self, scene, handle):
        self.scene = scene
        self.handle = handle

    def stats(self):
        st = fdgs_frame_stats()
        check(lib().fdgs_frame_get_stats(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def export(self, stream=None):
        s = self.stats()
        dev = self.scene.device
        tiles = s["tiles_x"] * s["tiles_y"]
        n = self.scene.n
        out = dict(
            tile_ranges=torch.empty((tiles, 2), dtype=torch.int32, device=dev),
            tile_ids=torch.empty((max(s["n_keys"], 1),), dtype=torch.int32, device=dev),
            T_final=torch.empty((s["height"], s["width"]), dtype=torch.float32, device=dev),
            n_contrib=torch.empty((s["height"], s["width"]), dtype=torch.int32, device=dev),
            flags=torch.empty((max(n, 1),), dtype=torch.uint8, device=dev),
            records=torch.full((max(n, 1), 12), float("nan"), dtype=torch.float32, device=dev))
        check(lib().fdgs_frame_export(self.handle, _ptr(out["tile_ranges"]),
                                      _ptr(out["tile_ids"]), _ptr(out["T_final"]),
                                      _ptr(out["n_contrib"]), _ptr(out["flags"]),
                                      _ptr(out["records"]), _stream(stream)))
        out["tile_ids"] = out["tile_ids"][: s["n_keys"]]
        out["flags"] = out["flags"][:n]
        out["records"] = out["records"][:n]
        out["stats"] = s
        return out

    def release(self):
        if self.handle is not None:
            check(lib().fdgs_frame_release(self.handle))
            self.handle = None

    def __del__(self):
        try:
            if self.handle is not None and self.scene.handle is not None:
                lib().fdgs_frame_release(self.handle)
        except Exception:
            pass


class Scene:
    """A 4D Gaussian scene on the GPU (fdgs_scene). Borrows the parameter tensors."""

    def __init__(self, params: SceneTensors):
        self.params = params
        self.n = int(params.mean4.shape[0])
        self.device = params.mean4.device
        self._desc = self._make_desc(params)
        h = ctypes.c_void_p()
        check(lib().fdgs_create_scene(ctypes.byref(self._desc), ctypes.byref(h)))
        self.handle = h
        self._mask_hold = None

    @staticmethod
    def _make_desc(p: SceneTensors):
        n = int(p.mean4.shape[0])
        for name, t, tail in (("mean4", p.mean4, (4,)), ("logscale4", p.logscale4, (4,)),
                              ("q_left", p.q_left, (4,)), ("q_right", p.q_right, (4,)),
                              ("opacity_logit", p.opacity_logit, ())):
            _check_param(t, tail, name)
            if t.shape[0] != n:
                raise ValueError(f"{name} has {t.shape[0]} rows, expected {n}")
        k = (p.sh_degree + 1) ** 2
        _check_param(p.sh, None, "sh")
        if tuple(p.sh.shape) != (k, 3, n):
            raise ValueError(f"sh must be [{k},3,{n}], got {tuple(p.sh.shape)}")
        d = fdgs_scene_desc()
        d.n, d.sh_degree = n, int(p.sh_degree)
        d.mean4, d.logscale4 = p.mean4.data_ptr(), p.logscale4.data_ptr()
        d.q_left, d.q_right = p.q_left.data_ptr(), p.q_right.data_ptr()
        d.opacity_logit, d.sh = p.opacity_logit.data_ptr(), p.sh.data_ptr()
        return d

    @staticmethod
    def from_host(scene, device="cuda"):
        return Scene(SceneTensors.from_host(scene, device))

    def update(self, params: SceneTensors):
        self._desc = self._make_desc(params)
        check(lib().fdgs_update_scene(self.handle, ctypes.byref(self._desc)))
        self.params = params
        self.n = int(params.mean4.shape[0])

    def set_active_mask(self, bits, key_times, stream=None):
        """bits: uint8 CUDA tensor [n_key, ceil(n/8)] (LSB-first); key_times ascending."""
        kt = np.ascontiguousarray(np.asarray(key_times, np.float32))
        n_key = int(kt.shape[0])
        if n_key == 0:
            check(lib().fdgs_set_active_mask(self.handle, None, None, 0, _stream(stream)))
            return
        if not (bits.is_cuda and bits.dtype == torch.uint8 and bits.is_contiguous()
                and bits.shape == (n_key, (self.n + 7) // 8)):
            raise ValueError("bits must be a contiguous uint8 CUDA tensor [n_key, ceil(n/8)]")
        self._mask_hold = bits
        check(lib().fdgs_set_active_mask(
            self.handle, _ptr(bits), kt.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n_key,
            _stream(stream)))

    def render(self, cam, t, use_mask=True, bg=(0.0, 0.0, 0.0), keep_frame=False, out=None,
               stream=None, tight=False, temporal_cull=True):
        """Render [3,H,W] float32. With keep_frame=True also returns the Frame. tight: build
        the alpha-tight tile sets instead of the 3-sigma squares (same image).
        temporal_cull=False: keep the Gaussians with sigmoid(o) p(t) < 1/255 in the lists
        (same image, longer lists)."""
        c = make_camera(cam)
        if out is None:
            out = torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.device)
        o = _opts(use_mask, bg, tight, temporal_cull)
        fh = ctypes.c_void_p()
        check(lib().fdgs_render(self.handle, ctypes.byref(c), float(t), ctypes.byref(o),
                                _ptr(out), ctypes.byref(fh) if keep_frame else None,
                                _stream(stream)))
        if keep_frame:
            return out, Frame(self, fh)
        return out

    def render_async(self, cam, t, use_mask=True, bg=(0.0, 0.0, 0.0), out=None, stream=None,
                     tight=False):
        """Render [3,H,W] float32 without any host synchronisation (fdgs_render_async): the
        call only enqueues work on the stream, so it can be captured in a CUDA graph after a
        first, sizing call. A list-capacity overflow leaves the image at the background and
        is reported by the next status_sync(), which grows the capacity. tight: the
        alpha-tight tile sets (same image, shorter lists)."""
        c = make_camera(cam)
        if out is None:
            out = torch.empty((3, c.height, c.width), dtype=torch.float32, device=self.device)
        o = _opts(use_mask, bg, tight)
        check(lib().fdgs_render_async(self.handle, ctypes.byref(c), float(t), ctypes.byref(o),
                                      _ptr(out), _stream(stream)))
        return out

    def reserve_render_lists(self, entries):
        """List capacity of render_async in tile-list entries (0: size it at the next call)."""
        check(lib().fdgs_reserve_render_lists(self.handle, int(entries)))

    def finetune_step(self, cam, t, target, lr, betas=(0.9, 0.999), eps=1e-15, use_mask=True,
                      tight=True, loss_accum=None, stream=None):
        """One fine-tuning iteration in libfdgs (fdgs_finetune_step): render, L1 loss against
        ``target`` [3,H,W], reverse replay and an Adam step on the scene's own attribute
        tensors in place. ``lr``: the seven rates (mean4, logscale4, q_left, q_right,
        opacity_logit, SH DC, higher SH bands). The loss is added to ``loss_accum`` (a device
        float tensor) when given."""
        c = make_camera(cam)
        o = _opts(use_mask, (0.0, 0.0, 0.0), tight)
        a = fdgs_adam_opts()
        for i, v in enumerate(lr):
            a.lr[i] = float(v)
        a.beta1, a.beta2, a.eps = float(betas[0]), float(betas[1]), float(eps)
        tgt = target.contiguous()
        check(lib().fdgs_finetune_step(self.handle, ctypes.byref(c), float(t), ctypes.byref(o),
                                       _ptr(tgt), ctypes.byref(a),
                                       _ptr(loss_accum) if loss_accum is not None else None,
                                       _stream(stream)))

    def set_batch_shape(self, footprint, ctas_per_sm=0):
        """Launch shape of this scene's batched blend (fdgs_set_batch_shape)."""
        check(lib().fdgs_set_batch_shape(self.handle, int(footprint), int(ctas_per_sm)))

    def finetune_reset(self):
        """Clears the Adam moments and step count of fdgs_finetune_step."""
        check(lib().fdgs_finetune_reset(self.handle))

    def render_backward(self, frame: Frame, dL_drgb, grads=None, stream=None):
        """Adds the gradients of L (given dL/drgb [3,H,W]) into ``grads`` (a SceneTensors of
        zero-initialised buffers, created if None) and returns it."""
        if grads is None:
            grads = SceneTensors(*[torch.zeros_like(x) for x in self.params.list()],
                                 self.params.sh_degree)
        dL = dL_drgb.contiguous()
        check(lib().fdgs_render_backward(self.handle, frame.handle, _ptr(dL),
                                         *[_ptr(g) for g in grads.list()], _stream(stream)))
        return grads

    def render_batch(self, cams, ts, use_mask=True, bg=(0.0, 0.0, 0.0), outs=None, stream=None):
        n = len(cams)
        _ca, carr = make_cameras(cams)
        _ta, tarr = _times(ts)
        if outs is None:
            outs = [torch.empty((3, int(c.height), int(c.width)), dtype=torch.float32,
                                device=self.device) for c in cams]
        _pa = np.asarray([o.data_ptr() for o in outs] or [0], dtype=np.uint64)
        parr = _pa.ctypes.data_as(ctypes.POINTER(_P))
        o = _opts(use_mask, bg)
        check(lib().fdgs_render_batch(self.handle, carr, tarr, n, ctypes.byref(o), parr,
                                      _stream(stream)))
        return outs

    def batch_autotune(self, cams, ts, use_mask=True, bg=(0.0, 0.0, 0.0), outs=None,
                       stream=None, cache=None):
        """fdgs_batch_autotune. With ``cache`` (a JSON file path) the launch shape is looked up
        under the batch's key (autotune_key) first: on a hit it is set without a search and
        the batch rendered once; on a miss the search runs and its pick is stored.
        ``self.autotune_from_cache`` tells which happened."""
        self.autotune_from_cache = False
        key = None
        if cache is not None:
            key = autotune_key(cams, self.n, use_mask, bg, _device_name(self.device))
            hit = read_autotune_cache(cache).get(key)
            if hit is not None:
                self.set_batch_shape(hit["footprint"], hit["ctas_per_sm"])
                self.autotune_from_cache = True
                return self.render_batch(cams, ts, use_mask, bg, outs, stream)
        outs = self._batch_autotune(cams, ts, use_mask, bg, outs, stream)
        if key is not None:
            info = self.batch_info(0)
            write_autotune_cache(cache, key, info["footprint"], info["ctas_per_sm"])
        return outs

    def _batch_autotune(self, cams, ts, use_mask, bg, outs, stream):
        n = len(cams)
        _ca, carr = make_cameras(cams)
        _ta, tarr = _times(ts)
        if outs is None:
            outs = [torch.empty((3, int(c.height), int(c.width)), dtype=torch.float32,
                                device=self.device) for c in cams]
        _pa = np.asarray([o.data_ptr() for o in outs] or [0], dtype=np.uint64)
        parr = _pa.ctypes.data_as(ctypes.POINTER(_P))
        o = _opts(use_mask, bg)
        check(lib().fdgs_batch_autotune(self.handle, carr, tarr, n, ctypes.byref(o), parr,
                                        _stream(stream)))
        return outs

    def batch_info(self, n):
        lat = (ctypes.c_float * max(n, 1))()
        st = (ctypes.c_float * len(BATCH_STAGES))()
        fp, ctas = ctypes.c_int(), ctypes.c_int()
        check(lib().fdgs_batch_info(self.handle, lat, n, ctypes.byref(fp), ctypes.byref(ctas),
                                    st))
        return dict(latency_ms=list(lat)[:n], footprint=fp.value, ctas_per_sm=ctas.value,
                    stage_ms=dict(zip(BATCH_STAGES, list(st))))

    def set_sh_codebook(self, codebook, codes):
        """Vector-quantised SH: codebook float CUDA tensor [n_code, K-1, 3], codes int16/uint16
        CUDA tensor [n] (the bit pattern is read as uint16). None clears. The tensors are
        borrowed (kept referenced here)."""
        if codebook is None:
            check(lib().fdgs_set_sh_codebook(self.handle, None, 0, None))
            self._cb_hold = None
            return
        k = (self.params.sh_degree + 1) ** 2
        if not (codebook.is_cuda and codebook.dtype == torch.float32 and codebook.is_contiguous()
                and codebook.dim() == 3 and tuple(codebook.shape[1:]) == (k - 1, 3)):
            raise ValueError(f"codebook must be a contiguous float32 CUDA tensor [n_code,{k - 1},3]")
        if not (codes.is_cuda and codes.dtype in (torch.int16, torch.uint16)
                and codes.is_contiguous() and tuple(codes.shape) == (self.n,)):
            raise ValueError(f"codes must be a contiguous 16-bit CUDA tensor [{self.n}]")
        self._cb_hold = (codebook, codes)
        check(lib().fdgs_set_sh_codebook(self.handle, _ptr(codebook), int(codebook.shape[0]),
                                         _ptr(codes)))

    @property
    def active_mask(self):
        """The mask bits last given to ``set_active_mask`` (None if cleared)."""
        return self._mask_hold

    def build_keyframe_masks(self, cams, key_times, out=None, stream=None):
        """Key-frame masks from the training views ``cams`` at ``key_times``: uint8
        [n_key][ceil(n/8)] on the device, in the layout ``set_active_mask`` takes."""
        _ca, carr = make_cameras(cams)
        tarr = (ctypes.c_float * max(len(key_times), 1))(*[float(t) for t in key_times])
        if out is None:
            out = torch.empty((len(key_times), (self.n + 7) // 8), dtype=torch.uint8,
                              device=self.device)
        check(lib().fdgs_build_keyframe_masks(self.handle, carr, len(cams), tarr,
                                              len(key_times), _ptr(out), _stream(stream)))
        return out

    def batch_counts(self):
        """Visible Gaussians, tile-list entries and block-list entries of the last batch,
        over all requests."""
        nv, nk, nb = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().fdgs_batch_counts(self.handle, ctypes.byref(nv), ctypes.byref(nk),
                                      ctypes.byref(nb)))
        return dict(n_visible=nv.value, n_keys=nk.value, n_block_entries=nb.value)

    def set_batch_list_capacity(self, entries):
        """Block-list capacity batches start with (0: default); see the C header."""
        check(lib().fdgs_set_batch_list_capacity(self.handle, int(entries)))

    def batch_tile_lists(self, req):
        """Tile lists of request ``req`` of the last batch, as numpy arrays in the layout of
        Frame.export: ranges [tiles, 2] (start, end) and Gaussian ids (uint32)."""
        import numpy as np
        nt, n = ctypes.c_uint64(), ctypes.c_uint64()
        check(lib().fdgs_batch_tile_lists(self.handle, int(req), None, None, 0,
                                          ctypes.byref(nt), ctypes.byref(n)))
        ranges = np.zeros((nt.value, 2), dtype=np.uint32)
        ids = np.zeros((max(n.value, 1),), dtype=np.uint32)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        check(lib().fdgs_batch_tile_lists(self.handle, int(req), ranges.ctypes.data_as(u32p),
                                          ids.ctypes.data_as(u32p), ids.size,
                                          ctypes.byref(nt), ctypes.byref(n)))
        return ranges, ids[: n.value]

    def variation_score(self, cams, ts, batch=8, out=None, stream=None, variant="full",
                        accumulate=False):
        """Spatial-temporal variation score [n] over the (t, camera) renders; ``variant``
        selects a score of the paper's ablation (SCORE_VARIANTS; "full" is the paper's).
        accumulate=True adds the pass's scores into ``out`` (fdgs_variation_score_add), for a
        pass split into parts."""
        _ca, carr = make_cameras(cams)
        tarr = (ctypes.c_float * max(len(ts), 1))(*[float(t) for t in ts])
        if accumulate:
            if out is None:
                raise ValueError("accumulate=True adds into out, which must be given")
            check(lib().fdgs_variation_score_add(
                self.handle, carr, len(cams), tarr, len(ts), int(batch), SCORE_VARIANTS[variant],
                _ptr(out), _stream(stream)))
            return out
        if out is None:
            out = torch.empty((self.n,), dtype=torch.float32, device=self.device)
        if variant == "full":
            check(lib().fdgs_variation_score(self.handle, carr, len(cams), tarr, len(ts),
                                             int(batch), _ptr(out), _stream(stream)))
        else:
            check(lib().fdgs_variation_score_variant(
                self.handle, carr, len(cams), tarr, len(ts), int(batch), SCORE_VARIANTS[variant],
                _ptr(out), _stream(stream)))
        return out

    def select_keep(self, scores, prune_ratio=0.8, stream=None):
        keep = torch.empty((scores.shape[0],), dtype=torch.uint8, device=self.device)
        s = scores.contiguous()
        check(lib().fdgs_select_keep(self.handle, _ptr(s), int(s.shape[0]), float(prune_ratio),
                                     _ptr(keep), _stream(stream)))
        return keep

    def profile(self, flags):
        """flags bit0: per-stage CUDA events; bit1: count blend evaluations; 0: off."""
        check(lib().fdgs_profile_enable(self.handle, int(flags)))

    def profile_read(self):
        ms = (ctypes.c_float * len(PROFILE_STAGES))()
        ev = (ctypes.c_uint64 * 3)()
        check(lib().fdgs_profile_read(self.handle, ms, ev))
        return dict(zip(PROFILE_STAGES, list(ms))), int(ev[0]), int(ev[1])

    def blend_counts(self):
        """Counters of the last counted render or batch: evaluations executed, culling tests
        executed, evaluations with alpha >= 1/255 at a pixel still compositing."""
        ev = (ctypes.c_uint64 * 3)()
        check(lib().fdgs_profile_read(self.handle, None, ev))
        return int(ev[0]), int(ev[1]), int(ev[2])

    def status_sync(self):
        check(lib().fdgs_status_sync(self.handle))

    def close(self):
        if self.handle is not None:
            lib().fdgs_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _RenderFn(torch.autograd.Function):
    """Differentiable render: forward = fdgs_render (keeping the frame), backward =
    fdgs_render_backward (hand-written reverse kernels)."""

    @staticmethod
    def forward(ctx, scene, cam, t, use_mask, bg, tight, mean4, logscale4, q_left, q_right,
                opacity_logit, sh):
        img, frame = scene.render(cam, t, use_mask=use_mask, bg=bg, keep_frame=True,
                                  tight=tight)
        ctx.scene = scene
        ctx.frame = frame
        return img

    @staticmethod
    def backward(ctx, dL):
        scene, frame = ctx.scene, ctx.frame
        grads = scene.render_backward(frame, dL)
        frame.release()
        return (None, None, None, None, None, None, *grads.list())


def render(scene: Scene, cam, t, use_mask=True, bg=(0.0, 0.0, 0.0), tight=False):
    """Differentiable render of ``scene`` (its parameter tensors may require grad). tight:
    alpha-tight tile sets (same image and gradients, shorter lists)."""
    p = scene.params
    return _RenderFn.apply(scene, cam, float(t), use_mask, tuple(bg), bool(tight), p.mean4,
                           p.logscale4, p.q_left, p.q_right, p.opacity_logit, p.sh)


def _device_name(device):
    d = torch.device(device)
    if d.type != "cuda":
        return d.type
    p = torch.cuda.get_device_properties(d)
    return f"{p.name}/{p.multi_processor_count}sm"


def autotune_key(cams, n_gauss, use_mask, bg, device_name) -> str:
    """Key of a batch launch shape in the autotune cache: the GPU (name and SM count), the
    request count, the multiset of tile-grid sizes of the requests (16x16 tiles, so images of
    nearby sizes share an entry), the scene size rounded up to a power of two, the key-frame
    filter and whether the background is black (the blend variant depends on it)."""
    grids = sorted(((int(c.width) + 15) // 16, (int(c.height) + 15) // 16) for c in cams)
    runs, prev, cnt = [], None, 0
    for g in grids + [None]:
        if g == prev:
            cnt += 1
            continue
        if prev is not None:
            runs.append(f"{prev[0]}x{prev[1]}*{cnt}")
        prev, cnt = g, 1
    n_pow2 = 1 << max(int(n_gauss) - 1, 0).bit_length()
    black = all(float(v) == 0.0 for v in bg)
    return "|".join([device_name, f"n_req={len(cams)}", "tiles=" + ",".join(runs),
                     f"gauss<={n_pow2}", f"mask={int(bool(use_mask))}", f"black={int(black)}"])


def read_autotune_cache(path) -> dict:
    """The entries of an autotune cache file ({} if it does not exist or is unreadable)."""
    import json
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    return d if isinstance(d, dict) else {}


def write_autotune_cache(path, key, footprint, ctas_per_sm) -> None:
    """Adds (or replaces) one entry; the file is rewritten atomically."""
    import json
    d = read_autotune_cache(path)
    d[key] = {"footprint": int(footprint), "ctas_per_sm": int(ctas_per_sm)}
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def version():
    return lib().fdgs_version().decode()


def measure_fp32_peak(paired=False, stream=None):
    """Measured FP32 fma throughput of the current device in TFLOP/s (fdgs_measure_fp32_peak):
    scalar fma.rn.f32, or fma.rn.f32x2 on pairs when ``paired``."""
    v = ctypes.c_double()
    check(lib().fdgs_measure_fp32_peak(1 if paired else 0, ctypes.byref(v), _stream(stream)))
    return v.value


def set_list_builder(mode):
    """Tile-list builder (0: auto, 1: emit + radix sort, 2: coverage bitmasks), process-wide."""
    check(lib().fdgs_set_list_builder(int(mode)))


STAGING_CP_ASYNC, STAGING_TMA = 0, 1
DEFAULT_BATCH_STAGING = STAGING_CP_ASYNC    # the library's default (fdgs_set_batch_staging)


def set_batch_staging(mode):
    """Record staging of the batched blend, process-wide (0: per-thread cp.async, 1: TMA
    tile::gather4); results do not depend on it."""
    check(lib().fdgs_set_batch_staging(int(mode)))


# launch shapes when none is set: the blend that writes transmittance (8x8 warp footprint,
# two pixels a lane) and the forward-only blend (8x16, four pixels a lane)
DEFAULT_BLEND_SHAPE = 3
DEFAULT_BLEND_SHAPE_FWD = 5


def set_blend_shape(footprint):
    """Forward-blend launch shape, process-wide: the warp footprint and pixels per lane (0:
    16x2, 1: 8x4, 2: 4x8 with one pixel a lane; 3: 8x8 with two; 4: 16x8, 5: 8x16 with
    four; 6: 16x16 with eight, one warp per tile), for both the blend that writes
    transmittance and the forward-only one; None restores the defaults of each. Results do
    not depend on it."""
    check(lib().fdgs_set_blend_shape(-1 if footprint is None else int(footprint)))


def debug_inject(kind, value=0):
    """Failure injection for tests of the error paths (see fdgs_debug_inject in the header):
    INJECT_SPIN_LIMIT, INJECT_WITHHOLD_PUBLISH, INJECT_FAIL_ALLOCS, or INJECT_NONE to clear."""
    check(lib().fdgs_debug_inject(int(kind), int(value)))
