"""Pins of the oracle's neural texel decoder (no GPU): features, forward pass against numpy's
matrix products, gradients against central finite differences, FP16 rounding against numpy,
and the FP32 inference emulation against the FP64 decoder within FP16 error bounds."""
import math

import numpy as np
import pytest

import oracle as O
from nn_bounds import e4m3_first_order_bound as _e4m3_first_order_bound


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


# ----------------------------------------------------------------------------- E4M3 variant

def test_e4m3_encoder_matches_torch_cast():
    """The oracle's E4M3 rounding (nearest, ties to even) against torch's float8_e4m3fn cast on
    random values, every exact midpoint between neighbouring codes, and the subnormal range."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    rng = np.random.default_rng(21)
    vals = [O.e4m3_value(c) for c in range(0x7f)]
    mids = [(a + b) / 2 for a, b in zip(vals[:-1], vals[1:])]
    xs = np.concatenate([rng.uniform(-448, 448, 4000), rng.uniform(-0.03, 0.03, 4000),
                         np.array(mids), -np.array(mids), np.array(vals), [0.0, -0.0]]).astype(np.float32)
    want = torch.from_numpy(xs).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([O.e4m3_encode(float(x)) for x in xs], np.uint8)
    np.testing.assert_array_equal(got, want)
    # decode of every finite code against torch
    codes = np.arange(256, dtype=np.uint8)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy()
    for c in range(256):
        if c & 0x7f == 0x7f:
            assert math.isnan(O.e4m3_value(c))
        else:
            assert O.e4m3_value(c) == ref[c]


def test_e4m3_saturates_and_keeps_nan():
    assert O.e4m3_encode(448.0) == 0x7e and O.e4m3_value(0x7e) == 448.0
    assert O.e4m3_encode(463.9) == 0x7e and O.e4m3_encode(1e30) == 0x7e and O.e4m3_encode(-1e30) == 0xfe
    assert O.e4m3_encode(float("nan")) & 0x7f == 0x7f
    assert O.e4m3_encode(2.0 ** -10) == 0 and O.e4m3_encode(2.0 ** -10 * 1.0001) == 1  # tie to even, then up


@pytest.mark.parametrize("wscale,lscale", [(0.2, 0.5), (0.6, 3.0), (0.05, 0.1)])
def test_e4m3_emulation_within_first_order_bound_of_fp64(wscale, lscale):
    """The E4M3 emulation stays within the first-order rounding bound of the FP64 decode of the
    same parameters (FP16-rounded latents), for small and large activations (the power-of-two
    scales keep them in range); and its error is well above the FP16 emulation's, so the E4M3
    roundings do take place."""
    rng = np.random.default_rng(int(wscale * 100 + lscale * 10))
    gh, gw, R = 8, 8, 4
    lat = _rand_lat(rng, gh, gw, lscale).astype(np.float16).astype(np.float64)
    P = _rand_params(rng, wscale).astype(np.float32).astype(np.float64)
    lat16, w16, b32 = O.nn_pack_inference(lat, P)
    idx = np.array([(x | (y << 16)) for y in range(4 * gh) for x in range(4 * gw)], np.int32)
    e = O.nn_e4m3_scales(lat16, P)
    assert e[3] == -(e[0] + e[1] + e[2]) and e[0] <= 8
    y8 = O.nn_decode_e4m3(lat16, R, P, idx).astype(np.float64)
    y64 = O.nn_decode_f64(lat, R, P, idx)
    y16 = O.nn_decode_f32(lat16, R, w16, b32, idx).astype(np.float64)
    bound = _e4m3_first_order_bound(lat, R, P, idx, e)
    err = np.abs(y8 - y64)
    assert np.all(err <= 1.5 * bound + 1e-6), float(np.max(err / (bound + 1e-12)))
    assert np.mean(err) > 4 * np.mean(np.abs(y16 - y64))


def test_e4m3_scales_follow_the_activation_bound():
    """Scaling the first layer's weights by 2^k moves log2 s1 by -k (the activation bound scales
    with them) and leaves the decoded values unchanged up to the same output scale, since a
    power-of-two scaling commutes with E4M3 rounding in the normal range."""
    rng = np.random.default_rng(31)
    gh, gw, R = 8, 8, 4
    lat = _rand_lat(rng, gh, gw).astype(np.float16).astype(np.float64)
    P = _rand_params(rng, 0.2).astype(np.float32).astype(np.float64)
    lat16, _, _ = O.nn_pack_inference(lat, P)
    e = O.nn_e4m3_scales(lat16, P)
    Q = P.copy()
    W1, b1, W2, b2, W3, b3 = O.nn_split(Q)
    W1 *= 4.0
    b1 *= 4.0
    f = O.nn_e4m3_scales(lat16, Q)
    assert f[0] == e[0] - 2
    idx = np.array([(x | (y << 16)) for y in range(0, 4 * gh, 3) for x in range(0, 4 * gw, 3)], np.int32)
    ya = O.nn_decode_e4m3(lat16, R, P, idx).astype(np.float64)
    yb = O.nn_decode_e4m3(lat16, R, Q, idx).astype(np.float64)
    # h1 doubles twice and W2 is unchanged, so layer 2 sees 4x inputs: s2 absorbs them only if its
    # range limit binds; either way the decode of the scaled network is 4x in the hidden layers
    y64a = O.nn_decode_f64(lat, R, P, idx)
    y64b = O.nn_decode_f64(lat, R, Q, idx)
    assert np.all(np.isfinite(ya)) and np.all(np.isfinite(yb))
    assert np.mean(np.abs(yb - y64b)) < 0.2 * np.mean(np.abs(y64b - y64b.mean())) + 1e-3
    assert np.mean(np.abs(ya - y64a)) < 0.2 * np.mean(np.abs(y64a - y64a.mean())) + 1e-3


def test_e4m3_decode_of_a_sparse_network_in_closed_form():
    """A network with one path per output (W1 reads latent 0 only, W2 and W3 diagonal) over a
    constant latent grid: each output is then a short chain of roundings that can be written out
    with torch's float8_e4m3fn cast (nearest even) as the E4M3 rounding: h1 = E4M3(relu(
    fp16(s1 a) L + s1 b1)), h2 = E4M3(relu(E4M3(s2 c) h1 + parts(s1 s2 b2))), y = (E4M3(s3 d) h2
    + parts(s1 s2 s3 b3)) / (s1 s2 s3), with FP32 sums in that order; the scale exponents are the
    closed form of the rule for this network."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")

    def q8(v):
        return float(torch.tensor([v], dtype=torch.float64).to(torch.float32).to(torch.float8_e4m3fn).to(torch.float64)[0])

    def parts(v):
        p0 = q8(v)
        p1 = q8(v - p0)
        return p0, p1, q8(v - p0 - p1)

    rng = np.random.default_rng(41)
    gh, gw, R, L = 4, 4, 4, 0.75
    lat = np.full((gh, gw, O.NN_LAT), L)
    P = np.zeros(O.NN_PARAMS)
    W1, b1, W2, b2, W3, b3 = O.nn_split(P)
    a = rng.uniform(-3, 3, 64).astype(np.float16).astype(np.float64)
    W1.reshape(64, 24)[:, 0] = a
    b1[:] = rng.uniform(-1, 1, 64).astype(np.float32)
    c = rng.uniform(-2, 2, 64).astype(np.float32)
    W2.reshape(64, 64)[np.arange(64), np.arange(64)] = c
    b2[:] = rng.uniform(-1, 1, 64).astype(np.float32)
    d = rng.uniform(-2, 2, 8).astype(np.float32)
    W3.reshape(8, 64)[np.arange(8), np.arange(8)] = d
    b3[:] = rng.uniform(-1, 1, 8).astype(np.float32)
    P = P.astype(np.float32).astype(np.float64)
    W1, b1, W2, b2, W3, b3 = O.nn_split(P)
    lat16, _, _ = O.nn_pack_inference(lat, P)
    e = O.nn_e4m3_scales(lat16, P)
    # the rule in closed form: B1_j = m |a_j| L + |b1_j|; B2_i = m^2 |c_i| B1_i + |b2_i|
    m = 1.0625
    B1 = m * np.abs(a) * L + np.abs(b1)
    B2 = m * m * np.abs(c) * B1 + np.abs(b2)
    fl = lambda v: int(np.floor(np.log2(v)))  # v is never an exact power of two here
    e1 = min(8, fl(448 / B1.max()))
    e2 = fl(min(448 / (2.0 ** e1 * B2.max()), 448 / np.abs(c).max()))
    e3 = fl(min(448 / np.abs(d).max(), 448 / (2.0 ** (e1 + e2) * np.abs(b3).max())))
    assert e == [e1, e2, e3, -(e1 + e2 + e3)]
    s1, s2, s3 = 2.0 ** e1, 2.0 ** e2, 2.0 ** e3
    f32 = np.float32
    want = np.zeros(8)
    for o in range(8):
        z1 = f32(f32(np.float16(s1 * a[o])) * f32(L)) + f32(s1 * b1[o])
        h1 = q8(max(float(z1), 0.0))
        t = f32(f32(q8(s2 * c[o])) * f32(h1))
        for p in parts(s2 * s1 * b2[o]):
            t = f32(t + f32(p))
        h2 = q8(max(float(t), 0.0))
        y = f32(f32(q8(s3 * d[o])) * f32(h2))
        for p in parts(s3 * s2 * s1 * b3[o]):
            y = f32(y + f32(p))
        want[o] = float(f32(y * f32(2.0 ** -(e1 + e2 + e3))))
    idx = np.array([(x | (y << 16)) for y in range(0, 16, 5) for x in range(0, 16, 3)], np.int32)
    got = O.nn_decode_e4m3(lat16, R, P, idx).astype(np.float64)
    for row in got:
        np.testing.assert_array_equal(row, want)
