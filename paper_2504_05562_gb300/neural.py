"""ctypes binding of the neural texel decoder entry points of libstf.so (stf_decoder_*).

Argument marshalling only: training, gradients and decoding run in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import stf

NN_PARAMS = 6280
NN_LAT = 16


class DecoderConfig(C.Structure):
    _fields_ = [("tex_w", C.c_int), ("tex_h", C.c_int), ("latent_w", C.c_int), ("latent_h", C.c_int),
                ("batch", C.c_int), ("lr_latent", C.c_float), ("lr_mlp", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_ulonglong)]


def _bind(L):
    vp, ip = C.c_void_p, C.c_int
    L.stf_decoder_create.argtypes = [C.POINTER(DecoderConfig), C.POINTER(C.c_void_p)]
    L.stf_decoder_train.argtypes = [vp, vp, ip, vp]
    L.stf_decoder_gradients.argtypes = [vp, vp, vp, ip, vp, vp, vp]
    L.stf_decoder_get_params.argtypes = [vp, vp, vp]
    L.stf_decoder_set_params.argtypes = [vp, vp, vp]
    L.stf_decoder_decode.argtypes = [vp, vp, ip, vp]
    L.stf_decoder_info.argtypes = [vp, C.POINTER(DecoderConfig), C.POINTER(C.c_longlong)]
    L.stf_decoder_save.argtypes = [vp, C.c_char_p]
    L.stf_decoder_load.argtypes = [C.c_char_p, C.POINTER(C.c_void_p)]
    L.stf_decoder_destroy.argtypes = [vp]
    L.stf_decoder_set_inference.argtypes = [vp, ip, vp]
    for n in ("stf_decoder_create", "stf_decoder_train", "stf_decoder_gradients", "stf_decoder_get_params",
              "stf_decoder_set_params", "stf_decoder_decode", "stf_decoder_info", "stf_decoder_save",
              "stf_decoder_load", "stf_decoder_destroy", "stf_decoder_set_inference"):
        getattr(L, n).restype = C.c_int


def _np_ptr(a):
    return a.ctypes.data


INFER_FP16, INFER_E4M3 = 0, 1


class Decoder:
    """Latent grid + MLP decoder of a tex_w x tex_h, 8-channel material (library-owned)."""

    def __init__(self, tex_w=None, tex_h=None, latent_w=None, latent_h=None, batch=65536, lr_latent=1e-2,
                 lr_mlp=5e-3, beta1=0.9, beta2=0.99, eps=1e-10, seed=0, handle=None):
        L = stf.load()
        if handle is None:
            cfg = DecoderConfig(tex_w, tex_h, latent_w, latent_h, batch, lr_latent, lr_mlp, beta1, beta2, eps, seed)
            h = C.c_void_p()
            stf._check(L.stf_decoder_create(C.byref(cfg), C.byref(h)))
            handle = h.value
        self.handle = handle
        cfg, _ = self.info()
        self.width, self.height = cfg.tex_w, cfg.tex_h
        self.latent_w, self.latent_h = cfg.latent_w, cfg.latent_h
        self.R = cfg.tex_w // cfg.latent_w

    def info(self):
        cfg = DecoderConfig()
        step = C.c_longlong()
        stf._check(stf.load().stf_decoder_info(self.handle, C.byref(cfg), C.byref(step)))
        return cfg, step.value

    @property
    def step(self):
        return self.info()[1]

    def train(self, target: "stf.Texture", steps: int) -> np.ndarray:
        losses = np.zeros(max(steps, 1), np.float32)
        stf._check(stf.load().stf_decoder_train(self.handle, target.handle, int(steps), _np_ptr(losses)))
        return losses[:steps]

    def gradients(self, target, texels):
        idx = np.ascontiguousarray(texels, np.int32)
        dP = np.zeros(NN_PARAMS, np.float32)
        dl = np.zeros((self.latent_h, self.latent_w, NN_LAT), np.float32)
        loss = np.zeros(1, np.float32)
        stf._check(stf.load().stf_decoder_gradients(self.handle, target.handle, _np_ptr(idx), idx.size,
                                                    _np_ptr(dP), _np_ptr(dl), _np_ptr(loss)))
        return float(loss[0]), dP, dl

    def get_params(self):
        lat = np.zeros((self.latent_h, self.latent_w, NN_LAT), np.float32)
        P = np.zeros(NN_PARAMS, np.float32)
        stf._check(stf.load().stf_decoder_get_params(self.handle, _np_ptr(lat), _np_ptr(P)))
        return lat, P

    def set_params(self, lat, P):
        lat = np.ascontiguousarray(lat, np.float32)
        P = np.ascontiguousarray(P, np.float32)
        assert lat.size == self.latent_w * self.latent_h * NN_LAT and P.size == NN_PARAMS
        stf._check(stf.load().stf_decoder_set_params(self.handle, _np_ptr(lat), _np_ptr(P)))

    def set_inference(self, fmt):
        """Inference precision: "fp16" (default) or "e4m3" (FP8 products for layers 2 and 3).
        Returns the exponents (log2 s1, log2 s2, log2 s3, log2 output scale) of the E4M3 scalings."""
        import numpy as np
        code = {"fp16": INFER_FP16, "e4m3": INFER_E4M3}[fmt]
        e = np.zeros(4, np.int32)
        stf._check(stf.load().stf_decoder_set_inference(self.handle, code, _np_ptr(e)))
        return [int(v) for v in e]

    def decode(self, texels):
        """texels: CUDA int32 tensor of packed ix | iy << 16 -> CUDA float32 tensor [n, 8]."""
        import torch
        n = int(texels.numel())
        out = torch.empty((n, 8), dtype=torch.float32, device=texels.device)
        stf._check(stf.load().stf_decoder_decode(self.handle, texels.data_ptr(), n, out.data_ptr()))
        return out

    def save(self, path):
        stf._check(stf.load().stf_decoder_save(self.handle, str(path).encode()))

    @classmethod
    def load(cls, path):
        h = C.c_void_p()
        stf._check(stf.load().stf_decoder_load(str(path).encode(), C.byref(h)))
        return cls(handle=h.value)

    def texture(self) -> "stf.Texture":
        return stf.Texture(decoder=self)

    def close(self):
        if getattr(self, "handle", None):
            stf.load().stf_decoder_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
