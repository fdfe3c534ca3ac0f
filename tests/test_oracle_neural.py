"""Pins of the oracle's neural texel decoder (no GPU): features, forward pass against numpy's
matrix products, gradients against central finite differences, FP16 rounding against numpy,
and the FP32 inference emulation against the FP64 decoder within FP16 error bounds."""
import math

import numpy as np
import pytest

import oracle as O


def _rand_params(rng, scale=0.3):
    return rng.normal(0, scale, O.NN_PARAMS)


def _rand_lat(rng, gh, gw, scale=0.5):
    return rng.normal(0, scale, (gh, gw, O.NN_LAT))


def test_phase_features_closed_form():
    s = math.sqrt(0.5)
    lat = np.zeros((4, 4, 16))
    want = {0: [s, s, 1, 0], 1: [s, -s, -1, 0], 2: [-s, -s, 1, 0], 3: [-s, s, -1, 0]}
    for ix in range(8):
        for iy in range(8):
            x = O.nn_features(lat, 4, ix, iy)
            np.testing.assert_allclose(x[16:20], want[ix % 4], atol=1e-15)
            np.testing.assert_allclose(x[20:24], want[iy % 4], atol=1e-15)
            assert np.all(x[:16] == 0)


def test_latent_bilinear_reproduces_linear_grid():
    """A latent grid linear in the cell index is reproduced exactly at the texel's latent
    position (i + 0.5) / R - 0.5 away from the clamped border."""
    gh, gw, R = 8, 8, 4
    yy, xx = np.mgrid[0:gh, 0:gw].astype(np.float64)
    lat = np.zeros((gh, gw, 16))
    for c in range(16):
        lat[..., c] = 0.25 * c + 0.5 * xx - 0.75 * yy
    for ix in range(2, 4 * gw - 3):
        for iy in range(2, 4 * gh - 3):
            lx, ly = (ix + 0.5) / R - 0.5, (iy + 0.5) / R - 0.5
            x = O.nn_features(lat, R, ix, iy)
            np.testing.assert_allclose(x[:16], 0.25 * np.arange(16) + 0.5 * lx - 0.75 * ly, atol=1e-12)
    x = O.nn_features(lat, R, 0, 0)  # clamped corner: all four taps on cell (0, 0)
    np.testing.assert_allclose(x[:16], 0.25 * np.arange(16), atol=1e-12)


def test_forward_matches_numpy_matmul():
    rng = np.random.default_rng(10)
    P = _rand_params(rng)
    W1, b1, W2, b2, W3, b3 = O.nn_split(P)
    X = rng.normal(0, 1, (50, O.NN_IN))
    h1 = np.maximum(X @ W1.reshape(64, 24).T + b1, 0)
    h2 = np.maximum(h1 @ W2.reshape(64, 64).T + b2, 0)
    y = h2 @ W3.reshape(8, 64).T + b3
    np.testing.assert_allclose(O.nn_forward_f64(P, X), y, rtol=1e-12, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(11)
    gh, gw, R = 4, 4, 4
    lat = _rand_lat(rng, gh, gw)
    P = _rand_params(rng)
    tgt = rng.uniform(0, 1, (gh * R, gw * R, 8)).astype(np.float32)
    idx = np.array([(int(x) | (int(y) << 16)) for x, y in rng.integers(0, gw * R, (64, 2))], np.int32)
    loss, dP, dl = O.nn_loss_grad(lat, R, P, tgt, idx)
    h = 1e-6
    for k in rng.choice(O.NN_PARAMS, 40, replace=False):
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (O.nn_loss_grad(lat, R, Pp, tgt, idx)[0] - O.nn_loss_grad(lat, R, Pm, tgt, idx)[0]) / (2 * h)
        assert abs(fd - dP[k]) <= 1e-6 * max(1.0, abs(dP[k])) + 1e-9
    flat = lat.reshape(-1)
    for k in rng.choice(flat.size, 40, replace=False):
        lp, lm = flat.copy(), flat.copy()
        lp[k] += h
        lm[k] -= h
        fd = (O.nn_loss_grad(lp.reshape(lat.shape), R, P, tgt, idx)[0] -
              O.nn_loss_grad(lm.reshape(lat.shape), R, P, tgt, idx)[0]) / (2 * h)
        assert abs(fd - dl.reshape(-1)[k]) <= 1e-6 * max(1.0, abs(dl.reshape(-1)[k])) + 1e-9
    assert loss > 0


def test_f16_rounding_matches_numpy():
    L = O.lib()
    rng = np.random.default_rng(12)
    vals = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-5, 5000), rng.normal(0, 3e4, 2000),
                           [0.0, -0.0, 65504.0, 65519.0, 65520.0, 1e-8, 2 ** -24, 3 * 2 ** -25, 2 ** -25]])
    for v in vals.astype(np.float32):
        with np.errstate(over="ignore"):
            want = np.float32(v).astype(np.float16).view(np.uint16)
        assert L.stf_ref_f32_to_f16(float(v)) == int(want), v
    # exact midpoints between representable halves round to even
    for code in range(0, 0x7bff, 97):
        a = np.uint16(code).view(np.float16).astype(np.float32)
        b = np.uint16(code + 1).view(np.float16).astype(np.float32)
        mid = np.float32((np.float64(a) + np.float64(b)) / 2)
        want = np.float32(mid).astype(np.float16).view(np.uint16)
        assert L.stf_ref_f32_to_f16(float(mid)) == int(want)


def test_fp32_emulation_close_to_fp64():
    """Decoding with FP16 storage and FP32 accumulation stays within the FP16 error budget of
    the FP64 decode of the same (rounded) parameters."""
    rng = np.random.default_rng(13)
    gh, gw, R = 8, 8, 4
    lat = _rand_lat(rng, gh, gw).astype(np.float16).astype(np.float64)
    P = _rand_params(rng, 0.2)
    W1, b1, W2, b2, W3, b3 = O.nn_split(P.copy())
    for w in (W1, W2, W3):
        w[:] = w.astype(np.float16).astype(np.float64)
    for b in (b1, b2, b3):
        b[:] = b.astype(np.float32).astype(np.float64)
    Pr = np.concatenate([W1, b1, W2, b2, W3, b3])
    lat16, w16, b32 = O.nn_pack_inference(lat, Pr)
    idx = np.array([(x | (y << 16)) for y in range(4 * gh) for x in range(4 * gw)], np.int32)
    y32 = O.nn_decode_f32(lat16, R, w16, b32, idx)
    y64 = O.nn_decode_f64(lat, R, Pr, idx)
    # inputs and two hidden layers rounded to FP16 (relative 2^-11 each), amplified by |W| sums
    scale = 1.0 + np.abs(y64)
    assert np.max(np.abs(y32 - y64) / scale) < 2e-2
    assert np.mean(np.abs(y32 - y64)) < 3e-3


def _rn_f16(q):
    """Round a Fraction to the nearest IEEE binary16 value (ties to even), as a Fraction."""
    from fractions import Fraction
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (max(e, -14) - 10)  # 11 significant bits; subnormals below 2^-14
    m = a / ulp
    f = math.floor(m)
    r = m - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return (f * ulp) if q > 0 else -(f * ulp)


def test_fp16_interpolation_is_correctly_rounded():
    """The emulated decoder interpolates the latents in binary16 arithmetic: corner weights
    rounded to FP16, then w00 L00, + w10 L10, + w01 L01, + w11 L11, each multiply and each fused
    multiply-add rounded once (ties to even). A decoder whose MLP passes 8 of the 16 inputs
    through exactly (y_j = relu(x_j) - relu(-x_j) with unit weights) exposes the inputs, which
    are checked against exact rational arithmetic rounded by an independent binary16 rounding,
    over every texel of a 16 x 16 material (clamped border cells included)."""
    from fractions import Fraction
    rng = np.random.default_rng(21)
    gh = gw = 4
    R = 4
    lat = (rng.normal(0, 1, (gh, gw, 16)) * np.exp2(rng.integers(-6, 4, (gh, gw, 16)))).astype(np.float16)
    idx = np.array([(x | (y << 16)) for y in range(R * gh) for x in range(R * gw)], np.int32)
    for half in (0, 1):
        W1 = np.zeros((64, 24))
        W2 = np.zeros((64, 64))
        W3 = np.zeros((8, 64))
        for j in range(8):
            W1[j, 8 * half + j] = 1.0
            W1[8 + j, 8 * half + j] = -1.0
            W2[j, j] = 1.0
            W2[8 + j, 8 + j] = 1.0
            W3[j, j] = 1.0
            W3[j, 8 + j] = -1.0
        P = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3.ravel(), np.zeros(8)])
        lat16, w16, b32 = O.nn_pack_inference(lat.astype(np.float32), P)
        got = O.nn_decode_f32(lat16, R, w16, b32, idx)
        for b, t in enumerate(idx):
            ix, iy = int(t) & 0xffff, int(t) >> 16
            axes = []
            for i, g in ((ix, gw), (iy, gh)):
                pos = Fraction(2 * i + 1, 2 * R) - Fraction(1, 2)
                c0 = math.floor(pos)
                axes.append((min(max(c0, 0), g - 1), min(max(c0 + 1, 0), g - 1), pos - c0))
            (x0, x1, fx), (y0, y1, fy) = axes
            w = [_rn_f16((1 - fx) * (1 - fy)), _rn_f16(fx * (1 - fy)), _rn_f16((1 - fx) * fy), _rn_f16(fx * fy)]
            cells = [(y0, x0), (y0, x1), (y1, x0), (y1, x1)]
            for j in range(8):
                ch = 8 * half + j
                L = [Fraction(float(lat[cy, cx, ch])) for cy, cx in cells]
                s = _rn_f16(w[0] * L[0])
                for k in (1, 2, 3):
                    s = _rn_f16(w[k] * L[k] + s)
                assert Fraction(float(got[b, j])) == s, (ix, iy, ch)
