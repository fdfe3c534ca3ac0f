"""Blue-noise selection uniforms (Section "Blue Noise Mask Improvements"): the void-and-cluster
masks against the properties blue noise has (a permutation of the ranks, little low-frequency
power, the quad modification spreading values inside 2x2 quads), the oracle's uniforms against
their formula, and the paper's finding that blue noise lowers the error of sample sharing,
the quad-energy masks most for quad sharing. No GPU (the masks are host code)."""
import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import stf
from paper_2504_05562_gb300 import workloads as W


def _lowfreq_power(v):
    n = v.shape[0]
    F = np.abs(np.fft.fft2(v - v.mean())) ** 2
    fy, fx = np.meshgrid(np.fft.fftfreq(n), np.fft.fftfreq(n), indexing="ij")
    rad = np.hypot(fx, fy)
    return F[(rad > 0) & (rad < 0.15)].mean()


def _quad_spread(v):
    n = v.shape[0]
    q = v.reshape(n // 2, 2, n // 2, 2).transpose(0, 2, 1, 3).reshape(-1, 4)
    return np.mean([np.abs(q[:, i] - q[:, j]).mean() for i in range(4) for j in range(i + 1, 4)])


def test_masks_are_blue_noise_permutations():
    r = stf.blue_noise_masks(64, seed=3)
    assert r.shape == (2, 64, 64)
    for c in range(2):
        assert np.array_equal(np.sort(r[c].ravel()), np.arange(4096))
    assert not np.array_equal(r[0], r[1])
    assert np.array_equal(r, stf.blue_noise_masks(64, seed=3))
    white = np.random.default_rng(0).permutation(4096).reshape(64, 64) / 4096.0
    for c in range(2):
        assert _lowfreq_power((r[c] + 0.5) / 4096.0) < 0.01 * _lowfreq_power(white)


def test_quad_energy_spreads_values_inside_quads():
    q = stf.blue_noise_masks(64, quad_energy=True, seed=5)
    p = stf.blue_noise_masks(64, quad_energy=False, seed=5)
    white = np.random.default_rng(1).permutation(4096).reshape(64, 64) / 4096.0
    sq = np.mean([_quad_spread((q[c] + 0.5) / 4096.0) for c in range(2)])
    sp = np.mean([_quad_spread((p[c] + 0.5) / 4096.0) for c in range(2)])
    assert sq > sp > _quad_spread(white)


def test_oracle_blue_uniforms_follow_their_formula():
    """One-tap selections with blue noise are the selections of the uniforms
    u = ((r + 1/2) / n^2 + frame * step + seed) mod 1 in 24-bit fixed point."""
    mat = W.material_c1()
    ranks = stf.blue_noise_masks(16, seed=2)
    view = W.screen_aligned_view(40, 24, 64, 64, 3.3, 0, origin=(1.7, 2.2))
    for frame, seed in ((0, 0), (5, 123456789), (77, 2 ** 40 + 7)):
        v = dict(view, frame=frame, blue=ranks)
        _, idx, _ = O.render(mat, v, O.ONE_TAP | O.FLAG_BLUE, seed=seed)
        fold = (seed & 0xFFFFFFFF) ^ (seed >> 32)
        off = (frame * 10368890 + (fold & 0xFFFFFF)) & 0xFFFFFF
        S = (1 << 24) // 256
        for y in range(24):
            for x in range(40):
                ux = ((int(ranks[0, y % 16, x % 16]) * S + S // 2 + off) & 0xFFFFFF) / 2.0 ** 24
                uy = ((int(ranks[1, y % 16, x % 16]) * S + S // 2 + off) & 0xFFFFFF) / 2.0 ** 24
                cx, cy = O.texel_coords(view, 64, 64, x, y)
                nx, _ = O.select_axis(O.BILINEAR, cx, ux)
                ny, _ = O.select_axis(O.BILINEAR, cy, uy)
                assert idx[y, x] == ((nx & 0xFFFF) | ((ny & 0xFFFF) << 16))


def test_blue_noise_lowers_the_sharing_error():
    """Section 5 (blue-noise evaluation): with blue-noise uniforms the sharing modes' error falls
    against the white-noise hash; the quad-energy masks help quad sharing most."""
    mat = W.material_c1()
    view = W.screen_aligned_view(128, 128, 64, 64, 4.0, 0, origin=(3.3, 7.6))
    ref = O.render_exact_f64(mat, view)[0][..., :3]
    bq = stf.blue_noise_masks(64, quad_energy=True, seed=1)
    bp = stf.blue_noise_masks(64, quad_energy=False, seed=1)

    def psnr(mode, blue=None):
        e = 0.0
        for f in range(4):
            v = dict(view, frame=f)
            m = mode
            if blue is not None:
                v["blue"], m = blue, mode | O.FLAG_BLUE
            e += np.mean((O.render(mat, v, m, seed=0)[0][..., :3] - ref) ** 2)
        return -10 * np.log10(e / 4)

    for mode in (O.QUAD2, O.WAVE3):
        assert psnr(mode, bq) > psnr(mode) + 1.0
    assert psnr(O.QUAD2, bq) > psnr(O.QUAD2, bp)


def test_blue_noise_argument_checks():
    with pytest.raises(stf.StfError):
        stf.blue_noise_masks(7)  # odd sizes have no 2x2 quads
    with pytest.raises(stf.StfError, match="power of two"):
        stf.set_blue_noise(stf.blue_noise_masks(12))  # masks are addressed modulo a power of two
    bad = stf.blue_noise_masks(8)
    bad[1, 0, 0] = bad[1, 0, 1]
    with pytest.raises(stf.StfError, match="permutation"):
        stf.set_blue_noise(bad)
    mat = W.material_c1()
    with pytest.raises(ValueError):
        O.render(mat, W.screen_aligned_view(8, 4, 64, 64, 2.0, 0), O.ONE_TAP | O.FLAG_BLUE)  # no masks


def test_temporal_average_converges_faster_than_white_noise():
    """The masks' time axis (a golden-ratio rotation of each pixel's uniforms per frame, the
    reading this build takes of the paper's spatiotemporal masks): averaging one-tap frames over
    time (as temporal accumulation does) converges faster than with the white-noise hash, whose
    per-pixel variance only falls as 1/N. Measured on the oracle: 16 frames, white 45.9 dB, blue
    53.7 dB; from 4 to 16 frames the blue average's MSE falls by more than the 4x of white noise."""
    mat = W.material_c1()
    view = W.screen_aligned_view(128, 128, 64, 64, 4.0, 0, origin=(3.3, 7.6))
    ref = O.render_exact_f64(mat, view)[0][..., :3]
    masks = stf.blue_noise_masks(64, quad_energy=True, seed=1)

    def mse(n, blue):
        acc = np.zeros_like(ref)
        for f in range(n):
            v = dict(view, frame=f)
            if blue:
                acc += O.render(mat, dict(v, blue=masks), O.ONE_TAP | O.FLAG_BLUE, seed=0)[0][..., :3]
            else:
                acc += O.render(mat, v, O.ONE_TAP, seed=0)[0][..., :3]
        return np.mean((acc / n - ref) ** 2)

    white4, white16 = mse(4, False), mse(16, False)
    blue4, blue16 = mse(4, True), mse(16, True)
    assert 10 * np.log10(white16 / blue16) > 3.0
    assert blue4 / blue16 > 1.5 * white4 / white16
