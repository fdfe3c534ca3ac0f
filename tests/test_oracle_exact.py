"""Exact filtering (Section "Exact Filtering") in the CPU oracle.

With the bilinear filter, a pixel whose footprint samples include every texel its own filter
weighs (positive weight) returns the deterministic filter over those texels; every other pixel
returns the weighted-importance estimate. The pixels that qualify are found independently of the
oracle's branch (exact_support.py), from its sampled texel indices and footprints.
"""
import numpy as np
import pytest

import oracle as O
from exact_support import qualifying
from paper_2504_05562_gb300 import workloads as W


@pytest.mark.parametrize("mode", [O.QUAD2, O.WAVE2, O.WAVE3, O.WAVE4])
def test_exact_pixels_equal_full_filter_bitwise_others_the_estimate(mode):
    mat = W.material_c1()
    view = dict(W.config1_view(), width=96, height=40)
    full, _, _ = O.render(mat, view, O.FULL, seed=3)
    wis, idx, _ = O.render(mat, view, mode, seed=3)
    ex, idx2, _ = O.render(mat, view, mode | O.FLAG_EXACT, seed=3)
    assert np.array_equal(idx, idx2)  # the same selections
    q = qualifying(view, mat["width"], mat["height"], idx, mode)
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
