"""Thin ctypes binding of libstf.so (include/stf.h): argument marshalling only.

Every step of the render path runs in the library's CUDA kernels. torch is used for device
memory and streams. If the library cannot be loaded the calls raise; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_DEVICE_ASSERT = range(7)
FILTER_BILINEAR, FILTER_BSPLINE3, FILTER_PER_VIEW = 0, 1, -1
MODE_FULL, MODE_ONE_TAP, MODE_QUAD2, MODE_WAVE2, MODE_WAVE3, MODE_WAVE4, MODE_SPARSE9 = range(7)
MODE_FLAG_EXACT = 16  # exact filtering (bilinear), OR'd into a sharing mode
MODE_FLAG_BLUE_NOISE = 32  # blue-noise selection uniforms (stf_set_blue_noise)
# alternative estimators (evaluation modes): mode | (EST_* << MODE_EST_SHIFT) [| MODE_FLAG_CLAMP]
MODE_EST_SHIFT, MODE_FLAG_CLAMP = 8, 2048
EST_WIS, EST_IS, EST_MIS, EST_PAIRWISE_MIS, EST_REGRESSION = range(5)
FMT_FP32, FMT_FP16, FMT_BF16, FMT_E4M3, FMT_UNORM8, FMT_NEURAL = range(6)
MODE_NAMES = {"full": 0, "one_tap": 1, "quad2": 2, "wave2": 3, "wave3": 4, "wave4": 5, "sparse9": 6}


class StfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("stf status %d: %s" % (status, msg))
        self.status = status


class Plane(C.Structure):
    _fields_ = [("fmt", C.c_int), ("channels", C.c_int), ("data", C.c_void_p), ("data_on_device", C.c_int)]


class TextureDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("num_planes", C.c_int), ("planes", Plane * 4),
                ("tile_scales", C.c_void_p), ("scale_tile", C.c_int), ("scales_on_device", C.c_int),
                ("decoder", C.c_void_p)]


class View(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("H", C.c_float * 9), ("cam_pos", C.c_float * 3),
                ("plane_to_world", C.c_float * 6), ("light_dir", C.c_float * 3), ("shading", C.c_int),
                ("ch_albedo", C.c_int), ("ch_normal", C.c_int), ("ch_rough", C.c_int), ("ch_ao", C.c_int),
                ("roughness", C.c_float), ("filter", C.c_int), ("tile_w", C.c_int), ("tile_h", C.c_int),
                ("frame", C.c_int), ("view_id", C.c_int), ("tex", C.c_void_p), ("out_rgba", C.c_void_p),
                ("out_pitch_floats", C.c_longlong), ("debug_indices", C.c_void_p),
                ("debug_channels", C.c_void_p)]


_lock = threading.Lock()
_lib = None
EXPORTS = ("stf_create_texture", "stf_render_views", "stf_destroy", "stf_set_stream", "stf_sync",
           "stf_last_error", "stf_version", "stf_decoder_create", "stf_decoder_train", "stf_decoder_gradients",
           "stf_decoder_get_params", "stf_decoder_set_params", "stf_decoder_decode", "stf_decoder_info",
           "stf_decoder_save", "stf_decoder_load", "stf_decoder_destroy", "stf_set_option", "stf_get_stat",
           "stf_autotune", "stf_view_config", "stf_autotune_save", "stf_autotune_load", "stf_autotune_clear",
           "stf_render_views_noalloc", "stf_sparse_footprints", "stf_set_sparse_footprints",
           "stf_blue_noise_masks", "stf_set_blue_noise", "stf_update_texture", "stf_decoder_set_inference")
NOALLOC_MAX_VIEWS, NOALLOC_MAX_ITEMS = 224, 262144
OPT_BATCH_GRAPHS, OPT_PIPELINE_BLOCKS, OPT_TEST_DECODE_STALL, OPT_PAIRED_PIXELS, OPT_TMA_STAGE = 1, 2, 3, 4, 5
STAT_GRAPH_BUILDS, STAT_GRAPH_REPLAYS = 1, 2


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libstf.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            L.stf_create_texture.argtypes = [C.POINTER(TextureDesc), C.POINTER(C.c_void_p)]
            L.stf_render_views.argtypes = [C.POINTER(View), C.c_int, C.c_int, C.c_int, C.c_ulonglong]
            L.stf_destroy.argtypes = [C.c_void_p]
            L.stf_set_stream.argtypes = [C.c_void_p]
            L.stf_sync.argtypes = []
            L.stf_last_error.restype = C.c_char_p
            L.stf_version.restype = C.c_int
            for name in ("stf_create_texture", "stf_render_views", "stf_destroy", "stf_set_stream", "stf_sync"):
                getattr(L, name).restype = C.c_int
            _bind_extra(L)
            _lib = L
    return _lib


def _bind_extra(L):
    from . import neural
    neural._bind(L)
    L.stf_set_option.argtypes = [C.c_int, C.c_longlong]
    L.stf_get_stat.argtypes = [C.c_int, C.POINTER(C.c_longlong)]
    L.stf_autotune.argtypes = [C.POINTER(View), C.c_int, C.c_int, C.c_int, C.c_ulonglong]
    L.stf_view_config.argtypes = [C.POINTER(View), C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]
    L.stf_autotune_save.argtypes = [C.c_char_p]
    L.stf_autotune_load.argtypes = [C.c_char_p]
    L.stf_autotune_clear.argtypes = []
    L.stf_render_views_noalloc.argtypes = [C.POINTER(View), C.c_int, C.c_int, C.c_int, C.c_ulonglong]
    L.stf_set_sparse_footprints.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.stf_blue_noise_masks.argtypes = [C.c_int, C.c_double, C.c_int, C.c_ulonglong, C.c_void_p]
    L.stf_set_blue_noise.argtypes = [C.c_void_p, C.c_int]
    L.stf_update_texture.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.stf_sparse_footprints.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                        C.c_ulonglong, C.c_int, C.c_void_p, C.c_void_p]
    for n in ("stf_set_option", "stf_get_stat", "stf_autotune", "stf_view_config", "stf_autotune_save",
              "stf_autotune_load", "stf_autotune_clear", "stf_render_views_noalloc"):
        getattr(L, n).restype = C.c_int


def _check(status):
    if status != OK:
        raise StfError(status, load().stf_last_error().decode())


def last_error() -> str:
    return load().stf_last_error().decode()


def version() -> int:
    return load().stf_version()


def set_stream(stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None for the default stream."""
    ptr = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(load().stf_set_stream(ptr))


def sync():
    _check(load().stf_sync())


# ----------------------------------------------------------------------------- textures

class Texture:
    """A library-owned texture built from a material description:
    dict(width, height, planes=[(fmt, channels, array)], scales=array|None, scale_tile=int).
    Arrays are host numpy arrays or CUDA torch tensors."""

    def __init__(self, material=None, decoder=None):
        d = TextureDesc()
        keep = []
        if decoder is not None:
            d.width, d.height = decoder.width, decoder.height
            d.num_planes = 0
            d.decoder = decoder.handle
            self.channels = 8
        else:
            d.width, d.height = int(material["width"]), int(material["height"])
            planes = material["planes"]
            d.num_planes = len(planes)
            self.channels = 0
            for i, (fmt, ch, arr) in enumerate(planes):
                ptr, dev, k = _ptr(arr)
                keep.append(k)
                d.planes[i].fmt, d.planes[i].channels = int(fmt), int(ch)
                d.planes[i].data, d.planes[i].data_on_device = ptr, dev
                self.channels += int(ch)
            sc = material.get("scales")
            if sc is not None:
                ptr, dev, k = _ptr(sc if not isinstance(sc, np.ndarray) else np.ascontiguousarray(sc, np.float32))
                keep.append(k)
                d.tile_scales, d.scales_on_device = ptr, dev
                d.scale_tile = int(material["scale_tile"])
        h = C.c_void_p()
        _check(load().stf_create_texture(C.byref(d), C.byref(h)))
        self.handle = h.value
        self.width, self.height = d.width, d.height
        del keep

    def update(self, data, on_device=False):
        """Replaces the texels with plane 0 bytes laid out as at creation: a CUDA tensor
        (on_device) or a host buffer (numpy array or CPU tensor; pin it for an asynchronous copy).
        The caller keeps `data` alive until the library stream has run the copy."""
        ptr = data.data_ptr() if hasattr(data, "data_ptr") else data.ctypes.data
        _check(load().stf_update_texture(self.handle, ptr, 1 if on_device else 0))

    def close(self):
        if getattr(self, "handle", None):
            load().stf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(arr):
    """(pointer, on_device, keep-alive) for a numpy array or a torch tensor."""
    if isinstance(arr, np.ndarray):
        a = np.ascontiguousarray(arr)
        return a.ctypes.data, 0, a
    import torch
    if isinstance(arr, torch.Tensor):
        t = arr.contiguous()
        return t.data_ptr(), int(t.is_cuda), t
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(arr))


# ----------------------------------------------------------------------------- views

def make_view(view: dict, tex: Texture, out, debug_indices=None, debug_channels=None) -> View:
    """Fill the C struct from a view dict (see workloads) and torch CUDA tensors:
    out float32 [h, w, 4] (or a row-pitched view), optional debug tensors."""
    v = View()
    v.width, v.height = int(view["width"]), int(view["height"])
    for i in range(9):
        v.H[i] = float(view["H"][i])
    for i in range(3):
        v.cam_pos[i] = float(view.get("cam_pos", (0.0, 1.0, 0.0))[i])
        v.light_dir[i] = float(view.get("light_dir", (0.0, 1.0, 0.0))[i])
    for i in range(6):
        v.plane_to_world[i] = float(view.get("plane_to_world", (1, 0, 0, 0, 1, 0))[i])
    v.shading = int(view.get("shading", 0))
    v.ch_albedo = int(view.get("ch_albedo", -1))
    v.ch_normal = int(view.get("ch_normal", -1))
    v.ch_rough = int(view.get("ch_rough", -1))
    v.ch_ao = int(view.get("ch_ao", -1))
    v.roughness = float(view.get("roughness", 0.3))
    v.filter = int(view.get("filter", 0))
    v.tile_w, v.tile_h = view.get("tile", (0, 0))
    v.frame = int(view.get("frame", 0))
    v.view_id = int(view.get("view_id", 0))
    v.tex = tex.handle
    v._keep = (tex, out, debug_indices, debug_channels)  # the view holds what its pointers name
    v.out_rgba = out.data_ptr()
    v.out_pitch_floats = int(out.stride(0)) if out.dim() == 3 else 0
    v.debug_indices = debug_indices.data_ptr() if debug_indices is not None else None
    v.debug_channels = debug_channels.data_ptr() if debug_channels is not None else None
    return v


def render_views(views, filter=FILTER_PER_VIEW, mode=MODE_WAVE3, seed=0):
    """views: a sequence of View structs (make_view). Enqueues the work on the library stream."""
    arr = (View * len(views))(*views)
    _check(load().stf_render_views(arr, len(views), int(filter), int(mode), int(seed) & (2 ** 64 - 1)))


def render_views_noalloc(views, filter=FILTER_PER_VIEW, mode=MODE_WAVE3, seed=0):
    """Same as render_views, through the allocation-free entry point (fixed scratch inside the
    library, at most NOALLOC_MAX_VIEWS views)."""
    arr = (View * len(views))(*views)
    _check(load().stf_render_views_noalloc(arr, len(views), int(filter), int(mode), int(seed) & (2 ** 64 - 1)))


def render(tex: Texture, view: dict, mode, seed=0, debug=False, out=None, filter=FILTER_PER_VIEW):
    """Render one view into new (or given) CUDA tensors. Returns (rgba, idx|None, channels|None)."""
    import torch
    h, w = int(view["height"]), int(view["width"])
    if out is None:
        out = torch.empty((h, w, 4), dtype=torch.float32, device="cuda")
    idx = torch.zeros((h, w), dtype=torch.int32, device="cuda") if debug else None
    ch = torch.zeros((h, w, 8), dtype=torch.float32, device="cuda") if debug else None
    render_views([make_view(view, tex, out, idx, ch)], filter, mode, seed)
    return out, idx, ch


# ----------------------------------------------------------------------------- scheduling

def set_option(option, value):
    _check(load().stf_set_option(int(option), int(value)))


def get_stat(stat):
    v = C.c_longlong()
    _check(load().stf_get_stat(int(stat), C.byref(v)))
    return v.value


def autotune(views, filter=FILTER_PER_VIEW, mode=MODE_WAVE3, seed=0):
    arr = (View * len(views))(*views)
    _check(load().stf_autotune(arr, len(views), int(filter), int(mode), int(seed) & (2 ** 64 - 1)))


def view_config(view, filter=FILTER_PER_VIEW, mode=MODE_WAVE3):
    tw, th, sc = C.c_int(), C.c_int(), C.c_int()
    _check(load().stf_view_config(C.byref(view), int(filter), int(mode), C.byref(tw), C.byref(th), C.byref(sc)))
    return tw.value, th.value, sc.value


def autotune_save(path):
    _check(load().stf_autotune_save(str(path).encode()))


def autotune_load(path):
    _check(load().stf_autotune_load(str(path).encode()))


def autotune_clear():
    _check(load().stf_autotune_clear())


# ----------------------------------------------------------------------------- sparse footprints

def sparse_footprints(tile=(8, 4), count=9, sigma=1.4, candidates=32, picks=10000, restarts=30, seed=0, patterns=1):
    """Pseudorandom sparse sharing footprints: int8 [patterns, 32, count] lane indices (own lane
    first) and the per-pattern usage standard deviation (host code; no GPU needed)."""
    import numpy as np
    tab = np.zeros((patterns, 32, count), np.int8)
    sc = np.zeros(patterns, np.float64)
    _check(load().stf_sparse_footprints(int(tile[0]), int(tile[1]), int(count), float(sigma), int(candidates),
                                        int(picks), int(restarts), int(seed) & (2 ** 64 - 1), int(patterns),
                                        tab.ctypes.data, sc.ctypes.data))
    return tab, sc


def set_sparse_footprints(table, tile=(8, 4)):
    """Uploads footprint patterns int8 [patterns, 32, 9] for MODE_SPARSE9 (pattern = frame % patterns)."""
    import numpy as np
    t = np.ascontiguousarray(table, np.int8)
    assert t.ndim == 3 and t.shape[1:] == (32, 9)
    _check(load().stf_set_sparse_footprints(t.ctypes.data, int(t.shape[0]), int(tile[0]), int(tile[1])))


# ----------------------------------------------------------------------------- blue noise

def blue_noise_masks(size=64, sigma=1.5, quad_energy=True, seed=0):
    """Two void-and-cluster blue-noise masks: uint16 ranks [2, size, size] (host code)."""
    import numpy as np
    r = np.zeros((2, size, size), np.uint16)
    _check(load().stf_blue_noise_masks(int(size), float(sigma), 1 if quad_energy else 0, int(seed) & (2 ** 64 - 1),
                                       r.ctypes.data))
    return r


def set_blue_noise(ranks):
    """Uploads masks uint16 [2, n, n] for MODE_FLAG_BLUE_NOISE."""
    import numpy as np
    r = np.ascontiguousarray(ranks, np.uint16)
    assert r.ndim == 3 and r.shape[0] == 2 and r.shape[1] == r.shape[2]
    _check(load().stf_set_blue_noise(r.ctypes.data, int(r.shape[1])))
