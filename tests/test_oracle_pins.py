"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed forms, library
routines (scipy's B-spline basis, numpy/torch float conversions), exact enumeration on tiny
inputs, and statistical laws the method obeys.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ULP1 = 2.0 ** -23


def _read_table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


# ----------------------------------------------------------------------------- filters

def test_bspline_golden_values():
    for d, num, den in _read_table("bspline_weights.txt"):
        exact = num / den
        assert O.weight_f64(O.BSPLINE3, d) == pytest.approx(exact, abs=1e-16)
        assert abs(O.weight(O.BSPLINE3, d) - exact) <= 2 * ULP1 * max(exact, 2 ** -10)


def test_bilinear_pmf_golden_values():
    for dx, dy, pmf in _read_table("bilinear_pmf.txt"):
        assert O.weight(O.BILINEAR, dx) * O.weight(O.BILINEAR, dy) == pmf


def test_bspline_matches_scipy_basis():
    from scipy.interpolate import BSpline
    b = BSpline.basis_element([-2.0, -1.0, 0.0, 1.0, 2.0], extrapolate=False)
    rng = np.random.default_rng(1)
    for d in rng.uniform(-1.999, 1.999, 2000):
        assert O.weight_f64(O.BSPLINE3, float(d)) == pytest.approx(float(b(d)), abs=1e-14)
        assert abs(O.weight(O.BSPLINE3, float(np.float32(d))) - float(b(np.float32(d)))) < 4e-7
    for d in (2.0, 2.5, -2.0, -3.75, 100.0):
        assert O.weight(O.BSPLINE3, d) == 0.0
        assert O.weight_f64(O.BSPLINE3, d) == 0.0


def test_partition_of_unity_and_symmetry():
    rng = np.random.default_rng(2)
    for f in rng.uniform(0.0, 1.0, 3000):
        f32 = float(np.float32(f))
        s64 = sum(O.weight_f64(O.BSPLINE3, f - k) for k in (-1, 0, 1, 2))
        assert abs(s64 - 1.0) <= 1e-15
        s32 = sum(O.weight(O.BSPLINE3, float(np.float32(f32 - k))) for k in (-1, 0, 1, 2))
        assert abs(s32 - 1.0) <= 4 * ULP1
        for filt in (O.BILINEAR, O.BSPLINE3):
            assert O.weight(filt, f32) == O.weight(filt, -f32) >= 0.0
    for k in range(1024):  # dyadic offsets: the bilinear pair sums to exactly 1
        f = k / 1024.0
        assert O.weight(O.BILINEAR, f) + O.weight(O.BILINEAR, f - 1.0) == 1.0


# ----------------------------------------------------------------------------- selection

def _exact_axis_weights(filt, c):
    i0 = math.floor(c)
    taps = [i0, i0 + 1] if filt == O.BILINEAR else [i0 - 1, i0, i0 + 1, i0 + 2]
    return taps, [O.weight_f64(filt, c - n) for n in taps]


def test_selection_frequencies_over_the_uniform_grid():
    """Over all 2^24 representable uniforms, each tap is picked a fraction of times equal to its
    filter weight (boundaries found by bisection; selection is monotone in u)."""
    rng = np.random.default_rng(3)
    N = 1 << 24
    for filt in (O.BILINEAR, O.BSPLINE3):
        for c in list(rng.uniform(-3.0, 70.0, 60)) + [5.0, 0.0, -0.5, 7.75]:
            c = float(np.float32(c))
            taps, wex = _exact_axis_weights(filt, c)

            def pick(j):
                return O.select_axis(filt, c, j / N)[0] - taps[0]

            bounds = [0]
            for k in range(1, len(taps)):
                lo, hi = 0, N
                while lo < hi:
                    mid = (lo + hi) // 2
                    if pick(mid) >= k:
                        hi = mid
                    else:
                        lo = mid + 1
                bounds.append(lo)
            bounds.append(N)
            counts = np.diff(bounds)
            assert counts.sum() == N
            for cnt, w in zip(counts, wex):
                assert abs(cnt / N - w) <= 4e-7
                if w == 0.0:
                    assert cnt == 0
            # the returned weight is the selected tap's weight
            n, w = O.select_axis(filt, c, 0.5)
            assert w == pytest.approx(wex[taps.index(n)], abs=3e-7) and w > 0.0


def _constant_uv_view(u0, v0, filt, size=256, frame=0):
    v = W._base_view(size, size, [[0, 0, u0], [0, 0, v0], [0, 0, 1]], filt, frame=frame)
    return v


@pytest.mark.parametrize("filt", [0, 1])
def test_selection_histogram_chi2(filt):
    """65,536 pixels that all filter the same point: the selected texels follow the 2D PMF."""
    from scipy.stats import chi2
    mat = W.material_c1()
    u0, v0 = 0.3712, 0.6283
    view = _constant_uv_view(u0, v0, filt)
    _, idx, _ = O.render(mat, view, O.ONE_TAP, seed=11)
    ix, iy = O.unpack_idx(idx)
    cx, cy = O.texel_coords(view, 64, 64, 0, 0)
    tx, wx = _exact_axis_weights(filt, cx)
    ty, wy = _exact_axis_weights(filt, cy)
    obs = np.zeros((len(ty), len(tx)))
    for a, b in zip(ix.ravel(), iy.ravel()):
        obs[ty.index(b), tx.index(a)] += 1
    exp = np.outer(wy, wx) * ix.size
    m = exp > 0
    assert obs[~m].sum() == 0
    stat = ((obs[m] - exp[m]) ** 2 / exp[m]).sum()
    assert chi2.sf(stat, m.sum() - 1) > 1e-4


# ----------------------------------------------------------------------------- RNG

def test_rng_uniformity_and_streams():
    from scipy.stats import chi2
    us = np.array([O.uniforms(x, y, 0, 0, 0) for y in range(64) for x in range(64)])
    for col in range(2):
        h, _ = np.histogram(us[:, col], bins=32, range=(0, 1))
        e = len(us) / 32
        assert chi2.sf(((h - e) ** 2 / e).sum(), 31) > 1e-4
        assert np.all((us[:, col] >= 0) & (us[:, col] < 1))
        assert np.all(us[:, col] * 2 ** 24 == np.floor(us[:, col] * 2 ** 24))
    assert abs(np.corrcoef(us[:, 0], us[:, 1])[0, 1]) < 0.05
    assert abs(np.corrcoef(us[:-1, 0], us[1:, 0])[0, 1]) < 0.05
    a = O.uniforms(5, 7, 0, 0, 0)
    assert a != O.uniforms(5, 7, 1, 0, 0) and a != O.uniforms(5, 7, 0, 1, 0)
    assert a != O.uniforms(5, 7, 0, 0, 1) and a != O.uniforms(5, 7, 0, 0, 1 << 40)
    assert a == O.uniforms(5, 7, 0, 0, 0)


def _pcg4d_inverse(v):
    """The inverse of the published pcg4d (Jarzynski and Olano 2020), undone step by step: each
    cross-lane multiply-add round is undone in reverse lane order, the xor-shift by 16 is its own
    inverse on 32 bits, and the LCG step is undone with the modular inverse of its odd multiplier."""
    M = 0xFFFFFFFF
    x, y, z, w = v

    def undo_round(x, y, z, w):
        w = (w - y * z) & M
        z = (z - x * y) & M
        y = (y - z * x) & M
        x = (x - y * w) & M
        return x, y, z, w

    x, y, z, w = undo_round(x, y, z, w)
    x, y, z, w = (t ^ (t >> 16) for t in (x, y, z, w))
    x, y, z, w = undo_round(x, y, z, w)
    inv = pow(1664525, -1, 1 << 32)
    return [((t - 1013904223) * inv) & M for t in (x, y, z, w)]


def test_pcg4d_is_the_published_bijection():
    """pcg4d maps (Z / 2^32)^4 onto itself one to one. The oracle's output, run backwards through
    the inverse of the published steps, must give back the input: a wrong constant, shift, lane
    index or a dropped step breaks this for almost every input."""
    rng = np.random.default_rng(11)
    cases = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [5, 7, 0, 0]]
    cases += [list(map(int, r)) for r in rng.integers(0, 1 << 32, (2000, 4), dtype=np.uint64)]
    for v in cases:
        out = O.pcg4d(v)
        assert _pcg4d_inverse(out) == v
    # and the inverse is not the identity: outputs differ from inputs
    assert O.pcg4d([1, 2, 3, 4]) != [1, 2, 3, 4]


def test_pcg4d_avalanche():
    """Flipping one input bit changes about half of the bits of every output lane (both rounds of
    cross-lane products present), and the two uniforms a pixel draws use different lanes."""
    rng = np.random.default_rng(12)
    flips = np.zeros((4, 4))
    n = 0
    for r in rng.integers(0, 1 << 32, (64, 4), dtype=np.uint64):
        v = list(map(int, r))
        base = O.pcg4d(v)
        for lane in range(4):
            for bit in (0, 7, 16, 31):
                u = list(v)
                u[lane] ^= 1 << bit
                out = O.pcg4d(u)
                for j in range(4):
                    flips[lane, j] += bin(out[j] ^ base[j]).count("1")
        n += 4
    mean = flips / (n * 32)
    # lane 3 of the input (the seed) feeds every output lane through the cross products
    assert np.all(mean > 0.40) and np.all(mean < 0.60), mean


# ----------------------------------------------------------------------------- decoders

def test_decoders_exhaustive():
    import torch
    codes = np.arange(65536, dtype=np.uint16)
    ref16 = codes.view(np.float16).astype(np.float32)
    refb = torch.from_numpy(codes.astype(np.int16)).view(torch.bfloat16).float().numpy()
    for c in range(0, 65536, 1):
        a = O.decode(O.FP16, c)
        b = ref16[c]
        assert (a == b) or (math.isnan(a) and math.isnan(b))
        a = O.decode(O.BF16, c)
        b = refb[c]
        assert (a == b) or (math.isnan(a) and math.isnan(b))
    ref8 = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    for c in range(256):
        a, b = O.decode(O.E4M3, c), ref8[c]
        assert (a == b) or (math.isnan(a) and math.isnan(b))
        assert O.decode(O.UNORM8, c) == np.float32(c) / np.float32(255.0)
    assert O.decode(O.E4M3, 0x7E) == 448.0 and O.decode(O.E4M3, 0x01) == 2.0 ** -9


@pytest.mark.parametrize("fmt", [0, 1, 2, 3])
def test_material_fetch_matches_library_decode(fmt):
    mat = W.material_c3(fmt, size=256)
    ref = W.decoded_reference(mat)
    rng = np.random.default_rng(4)
    for _ in range(300):
        x, y = (int(v) for v in rng.integers(-3, 259, 2))
        got = O.fetch_texel(mat, x, y)
        cx, cy = min(max(x, 0), 255), min(max(y, 0), 255)
        assert np.array_equal(got[:8], ref[cy, cx].astype(np.float32))


def test_two_plane_material_fetch():
    mat = W.material_c2(size=128)
    ref = W.decoded_reference(mat)
    for x, y in [(0, 0), (5, 100), (127, 127), (64, 3)]:
        got = O.fetch_texel(mat, x, y)
        assert np.array_equal(got[:6], ref[y, x].astype(np.float32))
        assert np.all(got[6:] == 0)


def test_e4m3_per_tile_scale_error_bound():
    """E4M3 keeps 3 fraction bits: relative error of the scaled decode <= 2^-4 (normal range)."""
    src = W.brick_material(256).astype(np.float32)
    dec = W.decoded_reference(W.material_c3(W.E4M3, size=256))
    big = np.abs(src) > 0.02
    assert np.all(np.abs(dec[big] - src[big]) <= 2.0 ** -4 * np.abs(src[big]) + 1e-7)


# ----------------------------------------------------------------------------- footprints

def test_footprints_shapes():
    sizes = {(8, 4): {O.QUAD2: 4, O.WAVE2: 4, O.WAVE3: 9, O.WAVE4: 16},
             (4, 8): {O.QUAD2: 4, O.WAVE2: 4, O.WAVE3: 9, O.WAVE4: 16},
             (16, 2): {O.QUAD2: 4, O.WAVE2: 4, O.WAVE3: 10, O.WAVE4: 16}}
    for (tw, th), per_mode in sizes.items():
        for mode, n in per_mode.items():
            for lane in range(32):
                fp = O.footprint(mode, tw, th, lane)
                assert len(fp) == n and lane in fp and len(set(fp)) == n
                xs = sorted({j % tw for j in fp})
                ys = sorted({j // tw for j in fp})
                assert len(xs) * len(ys) == n  # a full rectangle of lanes
                assert xs == list(range(xs[0], xs[0] + len(xs)))
                assert ys == list(range(ys[0], ys[0] + len(ys)))
                assert fp == sorted(fp)  # row-major order
        for lane in range(32):
            assert O.footprint(O.ONE_TAP, tw, th, lane) == [lane]


def test_quad_footprints_are_shared_and_wave_footprints_vary():
    """Section 4.3.1: with quads, the four lanes of a quad read the same lanes; wave footprints
    can be placed per lane and give more distinct sets."""
    quads = {tuple(O.footprint(O.QUAD2, 8, 4, lane)) for lane in range(32)}
    assert len(quads) == 8
    for lane in range(32):
        fp = O.footprint(O.QUAD2, 8, 4, lane)
        for j in fp:
            assert O.footprint(O.QUAD2, 8, 4, j) == fp
    waves = {tuple(O.footprint(O.WAVE2, 8, 4, lane)) for lane in range(32)}
    assert len(waves) > len(quads)


def test_wave3_usage_histogram_favours_centre():
    """Section 4.3.2: the 3x3 square under-uses corner lanes and over-uses central ones."""
    use = np.zeros(32, int)
    for lane in range(32):
        for j in O.footprint(O.WAVE3, 8, 4, lane):
            use[j] += 1
    assert use.sum() == 32 * 9
    assert use[0] < use[9] and use[31] < use[22]


# ----------------------------------------------------------------------------- coordinates

def test_texel_coords_dyadic_case():
    v = W.config1_view()
    for x, y in [(0, 0), (1, 2), (255, 255), (17, 200)]:
        cx, cy = O.texel_coords(v, 64, 64, x, y)
        assert cx == (x + 0.5) / 4.0 - 0.5 and cy == (y + 0.5) / 4.0 - 0.5


def test_texel_coords_clamp_and_nan():
    v = W._base_view(4, 4, [[0, 0, 1e9], [0, 0, -1e9], [0, 0, 1]], 0)
    cx, cy = O.texel_coords(v, 64, 64, 0, 0)
    assert cx == 32000.0 and cy == -16384.0
    v = W._base_view(4, 4, [[0, 0, 0], [0, 0, 0], [0, 0, 0]], 0)  # 0/0 -> NaN -> low clamp
    assert O.texel_coords(v, 64, 64, 1, 1) == (-16384.0, -16384.0)


# ----------------------------------------------------------------------------- exact filter

def _ramp_material(fn, size=16):
    y, x = np.mgrid[0:size, 0:size].astype(np.float64)
    t = np.stack([fn(x, y)] * 4, -1).astype(np.float32)
    assert np.array_equal(t.astype(np.float64), fn(x, y)[..., None].repeat(4, -1))
    return W.make_material(t, W.FP32)


def _interior_pixels(view, tex, margin):
    H = np.array(view["H"], np.float64).reshape(3, 3)
    ys, xs = np.mgrid[0:view["height"], 0:view["width"]]
    p = H @ np.stack([xs.ravel() + 0.5, ys.ravel() + 0.5, np.ones(xs.size)])
    cx = (p[0] / p[2] * tex - 0.5).reshape(xs.shape)
    cy = (p[1] / p[2] * tex - 0.5).reshape(xs.shape)
    ok = (cx > margin) & (cx < tex - 1 - margin) & (cy > margin) & (cy < tex - 1 - margin)
    return cx, cy, ok


@pytest.mark.parametrize("filt", [0, 1])
def test_exact_filter_reproduces_linear_and_quadratic(filt):
    """Bilinear and the cubic B-spline reproduce linear functions; on x^2 the discrete second
    moments are f(1-f) (tent) and exactly 1/3 (cubic B-spline)."""
    view = W.screen_aligned_view(40, 40, 16, 16, 3.0, filt, origin=(1.3, 1.7))
    lin = _ramp_material(lambda x, y: 0.25 + 0.5 * x - 0.125 * y)
    out, ch = O.render_exact_f64(lin, view, want_channels=True)
    cx, cy, ok = _interior_pixels(view, 16, 2.0)
    np.testing.assert_allclose(ch[..., 0][ok], (0.25 + 0.5 * cx - 0.125 * cy)[ok], rtol=0, atol=1e-12)
    sq = _ramp_material(lambda x, y: x * x)
    _, ch = O.render_exact_f64(sq, view, want_channels=True)
    f = cx - np.floor(cx)
    extra = f * (1.0 - f) if filt == O.BILINEAR else 1.0 / 3.0
    np.testing.assert_allclose(ch[..., 0][ok], (cx * cx + extra)[ok], rtol=0, atol=1e-10)


def test_fp32_full_filter_close_to_fp64():
    mat = W.material_c1()
    for filt in (0, 1):
        v = W.config1_view(filt)
        out, _, _ = O.render(mat, v, O.FULL)
        ex, _ = O.render_exact_f64(mat, v)
        assert np.max(np.abs(out - ex)) < 2e-6


# ----------------------------------------------------------------------------- estimators

def _tex_decoded(mat):
    return W.decoded_reference(mat)


def _exact_moments_one_tap(mat, view):
    """Exact mean and variance of one-tap STF per pixel from the filter weights (FP64)."""
    T = _tex_decoded(mat)
    h, w = view["height"], view["width"]
    mu = np.zeros((h, w, T.shape[-1]))
    m2 = np.zeros_like(mu)
    for y in range(h):
        for x in range(w):
            cx, cy = O.texel_coords(view, mat["width"], mat["height"], x, y)
            tx, wx = _exact_axis_weights(view["filter"], cx)
            ty, wy = _exact_axis_weights(view["filter"], cy)
            for b, wb in zip(ty, wy):
                for a, wa in zip(tx, wx):
                    t = T[min(max(b, 0), mat["height"] - 1), min(max(a, 0), mat["width"] - 1)]
                    mu[y, x] += wa * wb * t
                    m2[y, x] += wa * wb * t * t
    return mu, m2 - mu * mu


@pytest.mark.parametrize("filt", [0, 1])
def test_one_tap_is_unbiased(filt):
    """Eq. mc-estimator / Section S1: the mean of one-tap STF over 4096 seeds lies within 5 sigma
    of the exact filter, sigma from the exact per-pixel variance."""
    mat = W.material_c1()
    view = W.screen_aligned_view(16, 16, 64, 64, 3.3, filt, origin=(10.2, 20.7))
    mu, var = _exact_moments_one_tap(mat, view)
    N = 4096
    acc = np.zeros(mu.shape)
    for s in range(N):
        out, _, ch = O.render(mat, view, O.ONE_TAP, seed=s * 7919 + 1, nthreads=1, want_channels=True)
        acc += ch[..., :4]
    mean = acc / N
    sig = np.sqrt(np.maximum(var, 0) / N)
    z = np.abs(mean - mu) / np.maximum(sig, 1e-12)
    assert np.all((z < 5.0) | (np.abs(mean - mu) < 1e-6))


@pytest.mark.parametrize("filt", [0, 1])
def test_shading_after_one_tap_is_biased_by_the_filter_variance(filt):
    """Section S2 (filtering before vs after shading): with a nonlinear shading f(x) = x^2
    applied to the one-tap estimate X, E[f(X)] - f(E[X]) = Var(X) exactly. The Monte Carlo mean
    of X^2 over 2048 seeds lies within 5 sigma of mu^2 + Var(X), with mu, Var(X) and the
    variance of X^2 from the exact filter weights, and differs from the filtered-then-shaded
    mu^2 where the filter variance is large."""
    rng = np.random.default_rng(17 + filt)
    tex = rng.integers(0, 2, (64, 64, 4)).astype(np.float32) * 0.75 + 0.125  # high contrast
    mat = W.make_material(tex, W.FP32)
    view = W.screen_aligned_view(16, 16, 64, 64, 2.1, filt, origin=(4.6, 30.3))
    T = _tex_decoded(mat)
    h, w = view["height"], view["width"]
    mu = np.zeros((h, w, 4))
    m2 = np.zeros_like(mu)
    m4 = np.zeros_like(mu)
    for y in range(h):
        for x in range(w):
            cx, cy = O.texel_coords(view, mat["width"], mat["height"], x, y)
            tx, wx = _exact_axis_weights(filt, cx)
            ty, wy = _exact_axis_weights(filt, cy)
            for b, wb in zip(ty, wy):
                for a, wa in zip(tx, wx):
                    t = T[min(max(b, 0), 63), min(max(a, 0), 63)].astype(np.float64)
                    mu[y, x] += wa * wb * t
                    m2[y, x] += wa * wb * t ** 2
                    m4[y, x] += wa * wb * t ** 4
    var = m2 - mu ** 2
    N = 2048
    acc = np.zeros(mu.shape)
    for s in range(N):
        _, _, ch = O.render(mat, view, O.ONE_TAP, seed=s * 104729 + 5, nthreads=1, want_channels=True)
        acc += ch[..., :4].astype(np.float64) ** 2
    mean_f = acc / N
    sig = np.sqrt(np.maximum(m4 - m2 ** 2, 0) / N)
    assert np.all(np.abs(mean_f - (mu ** 2 + var)) <= 5 * sig + 1e-9)
    big = var > 6 * np.maximum(sig, 1e-12)
    assert big.sum() > 50
    assert np.all(mean_f[big] - mu[big] ** 2 > 0)


def _tiny_case(filt):
    rng = np.random.default_rng(5 + filt)
    tex = rng.uniform(0, 1, (4, 4, 4)).astype(np.float32)
    tex[..., 3] = 0.5  # a constant channel: zero error for every estimator (Section 3 goal 1)
    mat = W.make_material(tex, W.FP32)
    view = W.screen_aligned_view(8, 4, 4, 4, 2.3 if filt == 0 else 3.1, filt, origin=(0.4, 0.7))
    return mat, view


def _enumerate_reuse(mat, view, mode, lane):
    """Exact distribution of the WIS estimate of one lane: enumerate every joint selection of
    the lanes in its footprint (Eq. estimator-convex with w_i = f_c(x_i) / f_i(x_i))."""
    import itertools
    T = _tex_decoded(mat)
    tw, th = view["tile"]
    filt = view["filter"]
    fp = O.footprint(mode, tw, th, lane)
    coords = [O.texel_coords(view, 4, 4, j % tw, j // tw) for j in range(32)]

    def choices(j):
        cx, cy = coords[j]
        tx, wx = _exact_axis_weights(filt, cx)
        ty, wy = _exact_axis_weights(filt, cy)
        return [((a, b), pa * pb) for b, pb in zip(ty, wy) for a, pa in zip(tx, wx) if pa * pb > 0]

    opts = [choices(j) for j in fp]
    cx, cy = coords[lane]
    vals, probs = [], []
    for combo in itertools.product(*opts):
        p = 1.0
        num = np.zeros(4)
        den = 0.0
        for (a, b), pj in combo:
            p *= pj
            wc = O.weight_f64(filt, cx - a) * O.weight_f64(filt, cy - b)
            wgt = wc / pj
            num += wgt * T[min(max(b, 0), 3), min(max(a, 0), 3)]
            den += wgt
        vals.append(num / den)
        probs.append(p)
    vals, probs = np.array(vals), np.array(probs)
    assert abs(probs.sum() - 1.0) < 1e-12
    mean = (probs[:, None] * vals).sum(0)
    return vals, probs, mean


@pytest.mark.parametrize("filt,mode", [(0, 2), (0, 4), (1, 2)])
def test_reuse_estimator_by_enumeration(filt, mode):
    """Monte Carlo of the oracle's reuse estimate agrees with the exact enumeration; every
    outcome stays within the own filter's texel range (Eq. stf_error); the expected squared error
    against the exact filter does not exceed one-tap's variance on this case."""
    mat, view = _tiny_case(filt)
    T = _tex_decoded(mat)
    N = 6000
    lanes = [9, 10, 21]
    runs = np.array([O.render(mat, view, mode, seed=s, nthreads=1, want_channels=True)[2][..., :4]
                     for s in range(N)])
    mu_exact, var_one = _exact_moments_one_tap(mat, view)
    for lane in lanes:
        x, y = lane % 8, lane // 8
        vals, probs, mean = _enumerate_reuse(mat, view, mode, lane)
        var = (probs[:, None] * (vals - mean) ** 2).sum(0)
        mc = runs[:, y, x].mean(0)
        assert np.all(np.abs(mc - mean) <= 5 * np.sqrt(var / N) + 1e-7)
        # bounded error: inside the range of the texels under the own filter
        cx, cy = O.texel_coords(view, 4, 4, x, y)
        tx, wx = _exact_axis_weights(filt, cx)
        ty, wy = _exact_axis_weights(filt, cy)
        own = np.array([T[min(max(b, 0), 3), min(max(a, 0), 3)] for b, pb in zip(ty, wy)
                        for a, pa in zip(tx, wx) if pa * pb > 0])
        assert np.all(vals >= own.min(0) - 1e-12) and np.all(vals <= own.max(0) + 1e-12)
        assert np.all(np.abs(vals[:, 3] - 0.5) < 1e-12)
        mse_reuse = (probs[:, None] * (vals - mu_exact[y, x]) ** 2).sum(0)[:3].sum()
        assert mse_reuse <= var_one[y, x, :3].sum() + 1e-12


@pytest.mark.parametrize("filt,mag", [(0, 0.45), (1, 0.24)])
def test_reuse_equals_one_tap_when_nothing_is_shared(filt, mag):
    """Section 4.5: the own lane has weight exactly 1 and texels outside the own filter weight 0,
    so under minification every sharing mode returns one-tap STF bit for bit."""
    mat = W.material_c1()
    view = W.screen_aligned_view(24, 16, 64, 64, mag, filt, origin=(3.3, 2.1))
    base = O.render(mat, view, O.ONE_TAP, seed=3, want_channels=True)
    for mode in (O.QUAD2, O.WAVE2, O.WAVE3, O.WAVE4):
        got = O.render(mat, view, mode, seed=3, want_channels=True)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])


def test_one_tap_returns_the_selected_texel():
    mat = W.material_c1()
    view = W.config1_view(1)
    _, idx, ch = O.render(mat, view, O.ONE_TAP, seed=9, want_channels=True)
    ix, iy = O.unpack_idx(idx)
    T = _tex_decoded(mat).astype(np.float32)
    got = T[np.clip(iy, 0, 63), np.clip(ix, 0, 63)]
    assert np.array_equal(ch[..., :4], got)


def test_constant_texture_is_reproduced_exactly():
    tex = np.full((32, 32, 4), 0.3137, np.float32)
    mat = W.make_material(tex, W.FP32)
    for filt in (0, 1):
        view = W.screen_aligned_view(64, 32, 32, 32, 3.7, filt, origin=(2.2, 5.1))
        # exact in real arithmetic (Eq. estimator-convex: the weights are normalised); in FP32 the
        # n-term sums may each add one rounding, so allow one ulp per summed term
        ulp = 2.0 ** -25  # spacing of floats in [0.25, 0.5)
        for mode, n in ((O.ONE_TAP, 0), (O.QUAD2, 4), (O.WAVE3, 9), (O.WAVE4, 16), (O.FULL, 16)):
            out, _, _ = O.render(mat, view, mode, seed=1)
            assert np.all(np.abs(out - np.float32(0.3137)) <= n * ulp)


@pytest.mark.parametrize("filt", [0, 1])
def test_reuse_stays_in_own_texel_range(filt):
    mat = W.material_c1()
    view = W.screen_aligned_view(64, 64, 64, 64, 5.0, filt, origin=(8.0, 9.0))
    T = _tex_decoded(mat)
    for mode in (O.QUAD2, O.WAVE3, O.WAVE4):
        _, _, ch = O.render(mat, view, mode, seed=2, want_channels=True)
        for y in range(0, 64, 3):
            for x in range(0, 64, 3):
                cx, cy = O.texel_coords(view, 64, 64, x, y)
                tx, wx = _exact_axis_weights(filt, cx)
                ty, wy = _exact_axis_weights(filt, cy)
                own = np.array([T[min(max(b, 0), 63), min(max(a, 0), 63)] for b, pb in zip(ty, wy)
                                for a, pa in zip(tx, wx) if pa * pb > 0])
                lo, hi = own.min(0), own.max(0)
                v = ch[y, x, :4]
                assert np.all(v >= lo - 3e-7 * np.abs(lo)) and np.all(v <= hi + 3e-7 * np.abs(hi))


def test_config1_reuse_beats_one_tap_and_orders_by_footprint():
    """Table 1 trend (Section 5.2): larger footprints give lower error; every variant beats one-tap."""
    mat = W.material_c1()
    view = W.config1_view(0)
    ex, _ = O.render_exact_f64(mat, view)
    ps = {}
    for mode in (O.ONE_TAP, O.QUAD2, O.WAVE3, O.WAVE4):
        mses = [np.mean((O.render(mat, view, mode, seed=s)[0][..., :3] - ex[..., :3]) ** 2) for s in range(4)]
        ps[mode] = 10 * np.log10(1.0 / np.mean(mses))
    assert ps[O.ONE_TAP] < ps[O.QUAD2] < ps[O.WAVE3] < ps[O.WAVE4]


def test_config2_reduced_reuse_beats_one_tap():
    mat = W.material_c2(size=256)
    view = W.config2_view(width=320, height=180, tex=256)
    ex, _ = O.render_exact_f64(mat, view)
    res = {}
    for mode in (O.ONE_TAP, O.WAVE3):
        res[mode] = np.mean([np.mean((O.render(mat, view, mode, seed=s)[0][..., :3] - ex[..., :3]) ** 2)
                             for s in range(3)])
    assert res[O.WAVE3] < res[O.ONE_TAP]


# ----------------------------------------------------------------------------- shading

def _shade_view(**kw):
    v = W._base_view(4, 4, np.eye(3), 0)
    v.update(shading=1, ch_albedo=0, ch_normal=3, ch_rough=5, ch_ao=6, light_dir=(0.0, 1.0, 0.0),
             cam_pos=(0.0, 2.0, 0.0), plane_to_world=(1.0, 0.0, -0.5, 0.0, 1.0, -0.5))
    v.update(kw)
    return v


def test_shading_closed_form_head_on():
    """N = V = L = +y: D = 1/(pi a^2), Vis = 1/4, F = F0 = 0.04, so rgb = ao (albedo + 0.01 / a^2)
    with a = roughness^2."""
    v = _shade_view()
    for r in (0.2, 0.3, 0.5, 1.0):
        ch = [0.2, 0.5, 0.7, 0.0, 0.0, r, 0.8, 0.0]
        want = 0.8 * (np.array([0.2, 0.5, 0.7]) + 0.01 / r ** 4)
        np.testing.assert_allclose(O.shade_f64(v, ch, 0.5, 0.5)[:3], want, rtol=1e-13)
        np.testing.assert_allclose(O.shade(v, ch, 0.5, 0.5)[:3], want, rtol=3e-6)


def _ggx_textbook(N, V, L, alb, r, ao):
    Hh = (V + L) / np.linalg.norm(V + L)
    nl, nv, nh, vh = N @ L, max(N @ V, 1e-4), max(N @ Hh, 0), max(V @ Hh, 0)
    a2 = (r * r) ** 2
    D = a2 / (np.pi * (nh * nh * (a2 - 1) + 1) ** 2)
    lam_v = nl * np.sqrt(nv * nv * (1 - a2) + a2)
    lam_l = nv * np.sqrt(nl * nl * (1 - a2) + a2)
    F = 0.04 + 0.96 * (1 - vh) ** 5
    return ao * nl * (alb + np.pi * D * 0.5 / (lam_v + lam_l) * F) if nl > 0 else 0 * alb


def test_shading_matches_textbook_ggx_and_fp32_is_close():
    rng = np.random.default_rng(7)
    for _ in range(400):
        X, Y = rng.uniform(-0.6, 0.6, 2)
        r = rng.uniform(0.2, 0.8)
        alb = rng.uniform(0, 1, 3)
        # the view struct carries FP32 camera and light vectors: round them here too
        cam = tuple(float(np.float32(c)) for c in (rng.uniform(-1, 1), rng.uniform(0.5, 3), rng.uniform(-1, 1)))
        L = np.array(W.LIGHT_DIR, np.float32).astype(np.float64)
        v = _shade_view(light_dir=tuple(L), cam_pos=cam)
        u, vv = rng.uniform(0, 1, 2)
        ch = [*alb, X, Y, r, 0.9, 0.0]
        got = O.shade_f64(v, ch, u, vv)
        n = np.array([X, np.sqrt(max(0, 1 - X * X - Y * Y)), Y])
        n /= np.linalg.norm(n)
        P = np.array([u - 0.5, 0.0, vv - 0.5])
        V = np.array(cam) - P
        V /= np.linalg.norm(V)
        want = _ggx_textbook(n, V, L, alb, max(r, 0.02), 0.9)
        np.testing.assert_allclose(got[:3], want, rtol=1e-9, atol=1e-12)
        f32 = O.shade(v, [float(np.float32(c)) for c in ch], float(np.float32(u)), float(np.float32(vv)))
        assert np.all(np.abs(f32[:3] - got[:3]) <= 1e-5 * np.maximum(np.abs(got[:3]), 1e-3))


def test_reuse_error_falls_with_magnification():
    """Section 5.1 (error against zoom factor): near a 1:1 texel-to-pixel mapping neighbouring
    filters barely overlap and the weighted estimator stays close to one-tap STF; as the
    magnification grows, neighbouring pixels draw from nearly the same distributions and the
    shared estimate's error falls, while one-tap's stays put."""
    mat = W.material_c1()
    gains, reuse = [], []
    for mag in (1.0, 2.0, 4.0, 8.0):
        view = W.screen_aligned_view(64, 64, 64, 64, mag, 0, origin=(7.3, 9.1))
        ex, _ = O.render_exact_f64(mat, view)
        ps = {}
        for mode in (O.ONE_TAP, O.WAVE3):
            mses = [np.mean((O.render(mat, view, mode, seed=s)[0][..., :3] - ex[..., :3]) ** 2) for s in range(6)]
            ps[mode] = 10 * np.log10(1.0 / np.mean(mses))
        gains.append(ps[O.WAVE3] - ps[O.ONE_TAP])
        reuse.append(ps[O.WAVE3])
    assert all(b > a for a, b in zip(reuse, reuse[1:])), reuse
    assert all(b > a for a, b in zip(gains, gains[1:])), gains
    assert gains[0] > 0.0 and gains[-1] > 3 * gains[0]
