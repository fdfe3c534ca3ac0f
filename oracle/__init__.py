"""CPU oracle for stochastic texture filtering with sample reuse (ctypes wrapper).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this module; the GPU library never does. The C source in this
directory (``stf_oracle.c``) is the oracle proper: plain C99 compiled with
``-ffp-contract=off`` so that every float operation is rounded once, in the written order.

The wrapper only marshals numpy arrays into the C structs; every step of the method runs
in the C code. Material descriptions are plain dicts (see ``Material``) so that this module
imports nothing from the GPU package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "stf_oracle.c")
HDR = os.path.join(HERE, "stf_oracle.h")
LIB = os.path.join(HERE, "_build", "liboracle.so")

BILINEAR, BSPLINE3 = 0, 1
FULL, ONE_TAP, QUAD2, WAVE2, WAVE3, WAVE4, SPARSE9 = 0, 1, 2, 3, 4, 5, 6
FLAG_EXACT = 16  # exact filtering (bilinear), OR'd into a sharing mode
FLAG_BLUE = 32  # blue-noise uniforms from the view's masks
EST_SHIFT, FLAG_CLAMP = 8, 2048  # alternative estimators: mode | (est << EST_SHIFT) [| FLAG_CLAMP]
EST_WIS, EST_IS, EST_MIS, EST_PMIS, EST_REG = range(5)


def est_mode(mode, est, clamp=False):
    return mode | (est << EST_SHIFT) | (FLAG_CLAMP if clamp else 0)
FP32, FP16, BF16, E4M3, UNORM8 = 0, 1, 2, 3, 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (one translation unit, a second or two)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    srcs = [SRC, HDR, os.path.join(HERE, "stf_oracle_neural.c")]
    if not force and os.path.exists(LIB):
        if all(os.path.getmtime(LIB) >= os.path.getmtime(s) for s in srcs if os.path.exists(s)):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, SRC]
    if os.path.exists(srcs[2]):
        cmd.append(srcs[2])
    cmd.append("-lm")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class RefMaterial(C.Structure):
    _fields_ = [
        ("width", C.c_int), ("height", C.c_int), ("num_planes", C.c_int),
        ("plane_fmt", C.c_int * 4), ("plane_ch", C.c_int * 4),
        ("plane_data", C.c_void_p * 4),
        ("scales", C.c_void_p), ("scale_tile", C.c_int),
        ("nn_lat16", C.c_void_p), ("nn_gw", C.c_int), ("nn_gh", C.c_int), ("nn_r", C.c_int),
        ("nn_w16", C.c_void_p), ("nn_b32", C.c_void_p),
    ]


class RefView(C.Structure):
    _fields_ = [
        ("width", C.c_int), ("height", C.c_int), ("H", C.c_float * 9),
        ("cam_pos", C.c_float * 3), ("plane_to_world", C.c_float * 6), ("light_dir", C.c_float * 3),
        ("shading", C.c_int), ("ch_albedo", C.c_int), ("ch_normal", C.c_int), ("ch_rough", C.c_int),
        ("ch_ao", C.c_int), ("roughness", C.c_float), ("filter", C.c_int),
        ("tile_w", C.c_int), ("tile_h", C.c_int), ("frame", C.c_int), ("view_id", C.c_int),
        ("fp_table", C.c_void_p), ("fp_patterns", C.c_int),
        ("blue", C.c_void_p), ("blue_size", C.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            L.stf_ref_pcg4d.argtypes = [C.POINTER(C.c_uint32)]
            L.stf_ref_uniforms.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64,
                                           C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.stf_ref_weight.argtypes = [C.c_int, C.c_float]
            L.stf_ref_weight.restype = C.c_float
            L.stf_ref_weight_f64.argtypes = [C.c_int, C.c_double]
            L.stf_ref_weight_f64.restype = C.c_double
            L.stf_ref_select_axis.argtypes = [C.c_int, C.c_float, C.c_float, C.POINTER(C.c_int),
                                              C.POINTER(C.c_float)]
            L.stf_ref_decode.argtypes = [C.c_int, C.c_uint32]
            L.stf_ref_decode.restype = C.c_float
            L.stf_ref_footprint.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
            L.stf_ref_footprint.restype = C.c_int
            L.stf_ref_texel_coords.argtypes = [C.POINTER(RefView), C.c_int, C.c_int, C.c_int, C.c_int,
                                               C.POINTER(C.c_float), C.POINTER(C.c_float)]
            L.stf_ref_shade.argtypes = [C.POINTER(RefView), C.POINTER(C.c_float), C.c_float, C.c_float,
                                        C.POINTER(C.c_float)]
            L.stf_ref_shade_f64.argtypes = [C.POINTER(RefView), C.POINTER(C.c_double), C.c_double,
                                            C.c_double, C.POINTER(C.c_double)]
            L.stf_ref_render.argtypes = [C.POINTER(RefMaterial), C.POINTER(RefView), C.c_int, C.c_uint64,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
            L.stf_ref_render.restype = C.c_int
            L.stf_ref_render_exact_f64.argtypes = [C.POINTER(RefMaterial), C.POINTER(RefView), C.c_void_p,
                                                   C.c_void_p, C.c_int]
            L.stf_ref_render_exact_f64.restype = C.c_int
            L.stf_ref_shade_sensitivity.argtypes = [C.POINTER(RefView), C.c_int, C.c_void_p, C.c_void_p, C.c_int]
            L.stf_ref_shade_sensitivity.restype = C.c_int
            L.stf_ref_fetch_texel.argtypes = [C.POINTER(RefMaterial), C.c_int, C.c_int, C.POINTER(C.c_float)]
            _bind_neural(L)
            _lib = L
    return _lib


def _bind_neural(L):
    dp, ci = C.c_void_p, C.c_int
    L.stf_ref_neural_features.argtypes = [dp, ci, ci, ci, ci, dp]
    L.stf_ref_neural_features.restype = ci
    L.stf_ref_mlp_forward.argtypes = [dp, dp, ci, dp, dp]
    L.stf_ref_mlp_forward.restype = ci
    L.stf_ref_neural_decode.argtypes = [dp, ci, ci, ci, dp, ci, dp, dp, ci, dp]
    L.stf_ref_neural_decode.restype = ci
    L.stf_ref_neural_decode_f64.argtypes = [dp, ci, ci, ci, dp, dp, ci, dp]
    L.stf_ref_neural_decode_f64.restype = ci
    L.stf_ref_neural_loss_grad.argtypes = [dp, ci, ci, ci, dp, ci, dp, ci, dp, ci, dp, dp, dp]
    L.stf_ref_neural_loss_grad.restype = C.c_double
    L.stf_ref_f16_round.argtypes = [C.c_float]
    L.stf_ref_f16_round.restype = C.c_float
    L.stf_ref_f32_to_f16.argtypes = [C.c_float]
    L.stf_ref_f32_to_f16.restype = C.c_uint16
    L.stf_ref_f64_to_e4m3.argtypes = [C.c_double]
    L.stf_ref_f64_to_e4m3.restype = C.c_uint8
    L.stf_ref_e4m3_to_f64.argtypes = [C.c_uint8]
    L.stf_ref_e4m3_to_f64.restype = C.c_double
    L.stf_ref_neural_e4m3_scales.argtypes = [dp, ci, ci, dp, dp]
    L.stf_ref_neural_e4m3_scales.restype = ci
    L.stf_ref_neural_decode_e4m3.argtypes = [dp, ci, ci, ci, dp, dp, ci, dp, dp]
    L.stf_ref_neural_decode_e4m3.restype = ci


NN_IN, NN_H, NN_OUT, NN_LAT = 24, 64, 8, 16
NN_PARAMS = NN_H * NN_IN + NN_H + NN_H * NN_H + NN_H + NN_OUT * NN_H + NN_OUT


def _p(a):
    return a.ctypes.data


def nn_split(P):
    """Views (W1, b1, W2, b2, W3, b3) of a flat parameter vector."""
    sizes = [NN_H * NN_IN, NN_H, NN_H * NN_H, NN_H, NN_OUT * NN_H, NN_OUT]
    out, o = [], 0
    for s in sizes:
        out.append(P[o:o + s])
        o += s
    return out


def nn_features(lat, R, ix, iy):
    lat = np.ascontiguousarray(lat, np.float64)
    gh, gw = lat.shape[:2]
    x = np.zeros(NN_IN)
    lib().stf_ref_neural_features(_p(lat), gw, gh, R, int(ix) | (int(iy) << 16), _p(x))
    return x


def nn_forward_f64(P, x):
    P = np.ascontiguousarray(P, np.float64)
    x = np.ascontiguousarray(x, np.float64).reshape(-1, NN_IN)
    y = np.zeros((x.shape[0], NN_OUT))
    lib().stf_ref_mlp_forward(_p(P), _p(x), x.shape[0], _p(y), None)
    return y


def nn_loss_grad(lat, R, P, target, idx):
    """FP64 loss and gradients (dP, dlat) over texel indices idx (packed ix | iy << 16)."""
    lat = np.ascontiguousarray(lat, np.float64)
    gh, gw = lat.shape[:2]
    P = np.ascontiguousarray(P, np.float64)
    t = np.ascontiguousarray(target, np.float32)
    idx = np.ascontiguousarray(idx, np.int32)
    dP = np.zeros(NN_PARAMS)
    dl = np.zeros_like(lat)
    loss = lib().stf_ref_neural_loss_grad(_p(lat), gw, gh, R, _p(P), NN_PARAMS, _p(t), t.shape[1], _p(idx),
                                          idx.size, _p(dP), _p(dl), None)
    return loss, dP, dl


def nn_decode_f64(lat, R, P, idx):
    lat = np.ascontiguousarray(lat, np.float64)
    gh, gw = lat.shape[:2]
    P = np.ascontiguousarray(P, np.float64)
    idx = np.ascontiguousarray(idx, np.int32)
    out = np.zeros((idx.size, NN_OUT))
    lib().stf_ref_neural_decode_f64(_p(lat), gw, gh, R, _p(P), _p(idx), idx.size, _p(out))
    return out


def nn_pack_inference(lat, P):
    """FP16 codes of the latent grid and of W1, W2, W3 (round to nearest even, numpy) and the
    FP32 biases: the inference parameters both paths consume."""
    W1, b1, W2, b2, W3, b3 = nn_split(np.asarray(P, np.float64))
    lat16 = np.ascontiguousarray(np.asarray(lat, np.float32).astype(np.float16)).view(np.uint16)
    w16 = np.concatenate([W1, W2, W3]).astype(np.float32).astype(np.float16).view(np.uint16)
    b32 = np.concatenate([b1, b2, b3]).astype(np.float32)
    return lat16, np.ascontiguousarray(w16), np.ascontiguousarray(b32)


def nn_decode_f32(lat16, R, w16, b32, idx):
    """Emulation of the GPU inference precision (FP16 storage and latent interpolation, FP32
    accumulation)."""
    lat16 = np.ascontiguousarray(lat16, np.uint16)
    gh, gw = lat16.shape[:2]
    idx = np.ascontiguousarray(idx, np.int32)
    out = np.zeros((idx.size, NN_OUT), np.float32)
    lib().stf_ref_neural_decode(_p(lat16), gw, gh, R, _p(w16), w16.size, _p(b32), _p(idx), idx.size, _p(out))
    return out


def e4m3_encode(x):
    """OCP E4M3 code of x: nearest, ties to the even code, saturating at +-448."""
    return int(lib().stf_ref_f64_to_e4m3(float(x)))


def e4m3_value(code):
    return float(lib().stf_ref_e4m3_to_f64(int(code)))


def nn_e4m3_scales(lat16, P):
    """Exponents (log2 s1, log2 s2, log2 s3, log2 of the output scale) of the E4M3 variant."""
    lat16 = np.ascontiguousarray(lat16, np.uint16)
    gh, gw = lat16.shape[:2]
    P32 = np.ascontiguousarray(P, np.float32)
    e = np.zeros(4, np.int32)
    lib().stf_ref_neural_e4m3_scales(_p(lat16), gw, gh, _p(P32), _p(e))
    return [int(v) for v in e]


def nn_decode_e4m3(lat16, R, P, idx):
    """Emulation of the E4M3 inference variant (FP16 layer 1, E4M3 hidden layers and weights of
    layers 2 and 3, FP32 accumulation) from the FP16 latent grid and the FP32 parameters."""
    lat16 = np.ascontiguousarray(lat16, np.uint16)
    gh, gw = lat16.shape[:2]
    P32 = np.ascontiguousarray(P, np.float32)
    idx = np.ascontiguousarray(idx, np.int32)
    out = np.zeros((idx.size, NN_OUT), np.float32)
    lib().stf_ref_neural_decode_e4m3(_p(lat16), gw, gh, R, _p(P32), _p(idx), idx.size, _p(out), None)
    return out


def neural_material(width, height, lat16, R, w16, b32):
    """Material dict for a neural texture (the oracle decodes with the FP32 emulation)."""
    return {"width": width, "height": height, "planes": [], "scales": None, "scale_tile": 0,
            "neural": (np.ascontiguousarray(lat16, np.uint16), R, np.ascontiguousarray(w16, np.uint16),
                       np.ascontiguousarray(b32, np.float32))}


# ----------------------------------------------------------------------------- helpers

def pcg4d(v):
    a = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in v])
    lib().stf_ref_pcg4d(a)
    return [int(x) for x in a]


def uniforms(x, y, frame, view_id, seed):
    ux, uy = C.c_float(), C.c_float()
    lib().stf_ref_uniforms(x, y, frame, view_id, seed, C.byref(ux), C.byref(uy))
    return ux.value, uy.value


def weight(filt, d):
    return lib().stf_ref_weight(filt, d)


def weight_f64(filt, d):
    return lib().stf_ref_weight_f64(filt, d)


def select_axis(filt, c, u):
    n, w = C.c_int(), C.c_float()
    lib().stf_ref_select_axis(filt, c, u, C.byref(n), C.byref(w))
    return n.value, w.value


def decode(fmt, code):
    return lib().stf_ref_decode(fmt, code)


def footprint(mode, tw, th, lane):
    lst = (C.c_int * 16)()
    n = lib().stf_ref_footprint(mode, tw, th, lane, lst)
    return [lst[i] for i in range(n)]


def _material_struct(mat):
    """mat: dict(width, height, planes=[(fmt, channels, ndarray)], scales=ndarray|None, scale_tile)."""
    m = RefMaterial()
    m.width, m.height = mat["width"], mat["height"]
    planes = mat["planes"]
    m.num_planes = len(planes)
    keep = []
    for i, (fmt, ch, arr) in enumerate(planes):
        a = np.ascontiguousarray(arr)
        keep.append(a)
        m.plane_fmt[i] = fmt
        m.plane_ch[i] = ch
        m.plane_data[i] = a.ctypes.data
    sc = mat.get("scales")
    if sc is not None:
        sc = np.ascontiguousarray(sc, dtype=np.float32)
        keep.append(sc)
        m.scales = sc.ctypes.data
        m.scale_tile = int(mat["scale_tile"])
    else:
        m.scales = None
        m.scale_tile = 0
    nn = mat.get("neural")
    if nn is not None:
        lat16, R, w16, b32 = nn
        keep.extend([lat16, w16, b32])
        m.nn_lat16, m.nn_gh, m.nn_gw, m.nn_r = lat16.ctypes.data, lat16.shape[0], lat16.shape[1], int(R)
        m.nn_w16, m.nn_b32 = w16.ctypes.data, b32.ctypes.data
    return m, keep


def _view_struct(view):
    v = RefView()
    v.width, v.height = view["width"], view["height"]
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
    v.filter = int(view["filter"])
    v.tile_w, v.tile_h = view.get("tile", (8, 4))
    v.frame = int(view.get("frame", 0))
    v.view_id = int(view.get("view_id", 0))
    fp = view.get("footprints")  # int8 [patterns, 32, 9] for SPARSE9
    if fp is not None:
        fp = np.ascontiguousarray(fp, np.int8)
        v._fp = fp  # kept alive with the struct
        v.fp_table = fp.ctypes.data
        v.fp_patterns = fp.shape[0]
    blue = view.get("blue")  # uint16 ranks [2, n, n] for FLAG_BLUE
    if blue is not None:
        blue = np.ascontiguousarray(blue, np.uint16)
        v._blue = blue
        v.blue = blue.ctypes.data
        v.blue_size = blue.shape[1]
    return v


def fetch_texel(mat, x, y):
    m, keep = _material_struct(mat)
    out = (C.c_float * 8)()
    lib().stf_ref_fetch_texel(C.byref(m), x, y, out)
    del keep
    return np.array(list(out), np.float32)


def texel_coords(view, tex_w, tex_h, x, y):
    v = _view_struct(view)
    cx, cy = C.c_float(), C.c_float()
    lib().stf_ref_texel_coords(C.byref(v), tex_w, tex_h, x, y, C.byref(cx), C.byref(cy))
    return cx.value, cy.value


def shade(view, ch, u, v_):
    v = _view_struct(view)
    a = (C.c_float * 8)(*[float(x) for x in list(ch) + [0.0] * (8 - len(ch))])
    out = (C.c_float * 4)()
    lib().stf_ref_shade(C.byref(v), a, u, v_, out)
    return np.array(list(out), dtype=np.float32)


def shade_f64(view, ch, u, v_):
    v = _view_struct(view)
    a = (C.c_double * 8)(*[float(x) for x in list(ch) + [0.0] * (8 - len(ch))])
    out = (C.c_double * 4)()
    lib().stf_ref_shade_f64(C.byref(v), a, u, v_, out)
    return np.array(list(out), dtype=np.float64)


def render(mat, view, mode, seed=0, nthreads=None, want_channels=False):
    """FP32 oracle render. Returns (rgba float32 [h,w,4], idx uint32 [h,w], channels|None)."""
    m, keep = _material_struct(mat)
    v = _view_struct(view)
    h, w = view["height"], view["width"]
    out = np.zeros((h, w, 4), np.float32)
    idx = np.zeros((h, w), np.uint32)
    ch = np.zeros((h, w, 8), np.float32) if want_channels else None
    nt = nthreads or os.cpu_count() or 1
    rc = lib().stf_ref_render(C.byref(m), C.byref(v), mode, seed & (2**64 - 1), out.ctypes.data,
                              idx.ctypes.data, ch.ctypes.data if ch is not None else None, nt)
    if rc != 0:
        raise ValueError("oracle render rejected its arguments (rc=%d)" % rc)
    del keep
    return out, idx, ch


def render_exact_f64(mat, view, nthreads=None, want_channels=False):
    """FP64 deterministic filter + FP64 shading (the ground truth)."""
    m, keep = _material_struct(mat)
    v = _view_struct(view)
    h, w = view["height"], view["width"]
    out = np.zeros((h, w, 4), np.float64)
    ch = np.zeros((h, w, 8), np.float64) if want_channels else None
    nt = nthreads or os.cpu_count() or 1
    rc = lib().stf_ref_render_exact_f64(C.byref(m), C.byref(v), out.ctypes.data,
                                        ch.ctypes.data if ch is not None else None, nt)
    if rc != 0:
        raise ValueError("oracle exact render rejected its arguments (rc=%d)" % rc)
    del keep
    return out, ch


def shade_sensitivity(view, channels, nchannels):
    """sum_k |d rgb / d ch_k| * max(|ch_k|, 1) per pixel, float64 [h, w, 3]."""
    v = _view_struct(view)
    ch = np.ascontiguousarray(channels, np.float32)
    h, w = ch.shape[:2]
    out = np.zeros((h, w, 3), np.float64)
    lib().stf_ref_shade_sensitivity(C.byref(v), nchannels, ch.ctypes.data, out.ctypes.data, h * w)
    return out


def unpack_idx(idx):
    """Packed (ix & 0xffff) | (iy << 16) -> signed int arrays (ix, iy)."""
    ix = (idx & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.int32)
    iy = (idx >> 16).astype(np.uint16).view(np.int16).astype(np.int32)
    return ix, iy


def psnr(a, ref):
    """Linear-RGB PSNR with peak 1.0 over the RGB channels (Section 5.1 computes PSNR in linear RGB)."""
    a = np.asarray(a, np.float64)[..., :3]
    r = np.asarray(ref, np.float64)[..., :3]
    mse = float(np.mean((a - r) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)
