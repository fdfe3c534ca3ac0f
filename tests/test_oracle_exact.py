"""Exact filtering (Section "Exact Filtering") in the CPU oracle.

With the bilinear filter, a pixel whose footprint samples include every texel its own filter
weighs (positive weight) returns the deterministic filter over those texels; every other pixel
returns the weighted-importance estimate. The pixels that qualify are found here independently
of the oracle's branch, from its sampled texel indices and footprints.
"""
import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W


def _qualifying(view, mat, idx, mode):
    """Pixels whose bilinear support (positive-weight taps) is covered by the footprint's samples."""
    tw, th = view["tile"]
    h, w = view["height"], view["width"]
    ok = np.zeros((h, w), bool)
    ix = (idx & 0xFFFF).astype(np.int64)
    ix = np.where(ix >= 0x8000, ix - 0x10000, ix)
    iy = (idx >> 16).astype(np.int64)
    iy = np.where(iy >= 0x8000, iy - 0x10000, iy)
    for ty in range(0, h, th):
        for tx in range(0, w, tw):
            for lane in range(32):
                x, y = tx + lane % tw, ty + lane // tw
                if x >= w or y >= h:
                    continue
                cx, cy = O.texel_coords(view, mat["width"], mat["height"], x, y)
                samples = set()
                for j in O.footprint(mode, tw, th, lane):
                    sx, sy = tx + j % tw, ty + j // tw
                    assert sx < w and sy < h  # whole tiles: every footprint lane is on screen
                    samples.add((ix[sy, sx], iy[sy, sx]))
                need = []
                cx32, cy32 = np.float32(cx), np.float32(cy)
                x0, y0 = int(np.floor(cx32)), int(np.floor(cy32))
                for ny in (y0, y0 + 1):
                    for nx in (x0, x0 + 1):
                        wx = O.weight(O.BILINEAR, float(cx32 - np.float32(nx)))  # FP32 differences, as the method
                        wy = O.weight(O.BILINEAR, float(cy32 - np.float32(ny)))
                        if np.float32(wx) * np.float32(wy) > 0:
                            need.append((nx, ny))
                ok[y, x] = all(t in samples for t in need)
    return ok


@pytest.mark.parametrize("mode", [O.QUAD2, O.WAVE2, O.WAVE3, O.WAVE4])
def test_exact_pixels_equal_full_filter_bitwise_others_the_estimate(mode):
    mat = W.material_c1()
    view = dict(W.config1_view(), width=96, height=40)
    full, _, _ = O.render(mat, view, O.FULL, seed=3)
    wis, idx, _ = O.render(mat, view, mode, seed=3)
    ex, idx2, _ = O.render(mat, view, mode | O.FLAG_EXACT, seed=3)
    assert np.array_equal(idx, idx2)  # the same selections
    q = _qualifying(view, mat, idx, mode)
    assert q.any() and not q.all()
    assert np.array_equal(ex[q], full[q])
    assert np.array_equal(ex[~q], wis[~q])


def test_exact_filtering_lowers_the_error_and_larger_footprints_qualify_more():
    mat = W.material_c1()
    view = dict(W.config1_view(), width=128, height=64)
    ref = O.render_exact_f64(mat, view)[0][..., :3]
    frac = {}
    for mode in (O.QUAD2, O.WAVE3, O.WAVE4):
        e_wis = e_ex = 0.0
        for seed in range(6):
            wis, idx, _ = O.render(mat, view, mode, seed=seed)
            ex, _, _ = O.render(mat, view, mode | O.FLAG_EXACT, seed=seed)
            e_wis += np.mean((wis[..., :3] - ref) ** 2)
            e_ex += np.mean((ex[..., :3] - ref) ** 2)
        assert e_ex < e_wis
        full, _, _ = O.render(mat, view, O.FULL, seed=0)
        ex, _, _ = O.render(mat, view, mode | O.FLAG_EXACT, seed=0)
        frac[mode] = float(np.mean(np.all(ex == full, axis=-1)))
    assert frac[O.QUAD2] < frac[O.WAVE3] < frac[O.WAVE4]


def test_exact_flag_rejected_without_sharing():
    mat = W.material_c1()
    view = dict(W.config1_view(), width=32, height=8)
    for mode in (O.FULL, O.ONE_TAP):
        with pytest.raises(ValueError):
            O.render(mat, view, mode | O.FLAG_EXACT)
