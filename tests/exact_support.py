"""Which pixels exact filtering applies to, found from the sampled texel indices and footprints.

Exact filtering (Section "Exact Filtering"), bilinear: a pixel qualifies when every texel of
positive weight in its own filter is among its footprint lanes' samples. Written here from that
definition, independently of the oracle's and the GPU's branch.
"""
import numpy as np

import oracle as O


def _signed16(a):
    a = a.astype(np.int64)
    return np.where(a >= 0x8000, a - 0x10000, a)


def qualifying(view, tex_w, tex_h, idx, mode):
    """Boolean [h, w]: pixels whose bilinear support is covered by their footprint's samples.
    idx: the sampled lattice indices (x | y << 16) of every pixel; whole tiles only."""
    tw, th = view["tile"]
    h, w = view["height"], view["width"]
    assert w % tw == 0 and h % th == 0
    ix, iy = _signed16(idx & 0xFFFF), _signed16(idx >> 16)
    ok = np.zeros((h, w), bool)
    for ty in range(0, h, th):
        for tx in range(0, w, tw):
            for lane in range(32):
                x, y = tx + lane % tw, ty + lane // tw
                cx, cy = O.texel_coords(view, tex_w, tex_h, x, y)
                samples = {(ix[ty + j // tw, tx + j % tw], iy[ty + j // tw, tx + j % tw])
                           for j in O.footprint(mode, tw, th, lane)}
                cx32, cy32 = np.float32(cx), np.float32(cy)
                x0, y0 = int(np.floor(cx32)), int(np.floor(cy32))
                need = []
                for ny in (y0, y0 + 1):
                    for nx in (x0, x0 + 1):
                        wx = O.weight(O.BILINEAR, float(cx32 - np.float32(nx)))  # FP32 differences
                        wy = O.weight(O.BILINEAR, float(cy32 - np.float32(ny)))
                        if np.float32(wx) * np.float32(wy) > 0:
                            need.append((nx, ny))
                ok[y, x] = all(t in samples for t in need)
    return ok
