"""The alternative estimators of Section 4.1 in the CPU oracle (IS, MIS balance heuristic,
pairwise MIS, regression; each optionally clamped), pinned against an FP64 enumeration of every
joint texel selection written here from the estimators' definitions, against the unbiasedness
the MIS estimators have by construction, and against the ordering of the paper's estimator
comparison (Section 5.1: the weighted estimator has the lowest error, clamping lowers the error of
the others, plain importance sampling is worst).
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import workloads as W

ESTS = [O.EST_IS, O.EST_MIS, O.EST_PMIS, O.EST_REG]


def _axis(filt, c):
    i0 = math.floor(c)
    taps = [i0, i0 + 1] if filt == O.BILINEAR else [i0 - 1, i0, i0 + 1, i0 + 2]
    return taps, [O.weight_f64(filt, c - n) for n in taps]


def _pmf(filt, c, a, b):
    return O.weight_f64(filt, c[0] - a) * O.weight_f64(filt, c[1] - b)


def _estimate(est, clamp, filt, coords, fp, ic, combo, T):
    """FP64 value of estimator `est` for the pixel of footprint position ic, given the selections."""
    n = len(fp)
    c = coords[fp[ic]]
    xs = [t for t, _ in combo]
    ps = [p for _, p in combo]
    Ts = np.array([T[min(max(b, 0), 3), min(max(a, 0), 3)] for a, b in xs])
    pc = np.array([_pmf(filt, c, a, b) for a, b in xs])
    if est == O.EST_IS:
        F = sum(pc[i] / ps[i] * Ts[i] for i in range(n)) / n
    elif est == O.EST_MIS:
        F = sum(pc[i] * Ts[i] / sum(_pmf(filt, coords[fp[k]], *xs[i]) for k in range(n)) for i in range(n))
    elif est == O.EST_PMIS:
        xc = xs[ic]
        mc = sum(pc[ic] / (pc[ic] + (n - 1) * _pmf(filt, coords[fp[j]], *xc)) for j in range(n) if j != ic) / (n - 1)
        F = mc * Ts[ic] + sum(pc[i] * Ts[i] / (pc[i] + (n - 1) * ps[i]) for i in range(n) if i != ic)
    else:
        h = pc / np.array(ps)
        y = h[:, None] * Ts
        hb = h.mean()
        shh = ((h - hb) ** 2).sum()
        beta = ((h - hb)[:, None] * y).sum(0) / shh if shh > 0 else np.zeros(Ts.shape[1])
        F = y.mean(0) - beta * (hb - 1.0)
    if clamp:
        used = Ts[pc > 0]
        F = np.clip(F, used.min(0), used.max(0))
    return F


def _enumerate(est, clamp, mat, view, mode, lane):
    T = W.decoded_reference(mat)
    tw, th = view["tile"]
    filt = view["filter"]
    fp = O.footprint(mode, tw, th, lane)
    coords = {j: O.texel_coords(view, 4, 4, j % tw, j // tw) for j in fp}

    def choices(j):
        cx, cy = coords[j]
        tx, wx = _axis(filt, cx)
        ty, wy = _axis(filt, cy)
        return [((a, b), pa * pb) for b, pb in zip(ty, wy) for a, pa in zip(tx, wx) if pa * pb > 0]

    ic = fp.index(lane)
    vals, probs = [], []
    for combo in itertools.product(*[choices(j) for j in fp]):
        vals.append(_estimate(est, clamp, filt, coords, fp, ic, combo, T))
        probs.append(np.prod([p for _, p in combo]))
    vals, probs = np.array(vals), np.array(probs)
    assert abs(probs.sum() - 1.0) < 1e-12
    return vals, probs, (probs[:, None] * vals).sum(0), coords[lane]


def _tiny_case(filt):
    rng = np.random.default_rng(11 + filt)
    tex = rng.uniform(0, 1, (4, 4, 4)).astype(np.float32)
    mat = W.make_material(tex, W.FP32)
    view = W.screen_aligned_view(8, 4, 4, 4, 2.3 if filt == 0 else 3.1, filt, origin=(0.4, 0.7))
    return mat, view


def _exact_filter(mat, filt, c):
    T = W.decoded_reference(mat)
    tx, wx = _axis(filt, c[0])
    ty, wy = _axis(filt, c[1])
    return sum(pa * pb * T[min(max(b, 0), 3), min(max(a, 0), 3)] for b, pb in zip(ty, wy) for a, pa in zip(tx, wx))


@pytest.mark.parametrize("filt,mode", [(0, O.QUAD2), (0, O.WAVE2)])
def test_estimators_by_enumeration(filt, mode):
    """The oracle's Monte Carlo mean of each estimator agrees with its exact expectation; MIS and
    pairwise MIS are unbiased (the expectation is the deterministic filter); every clamped outcome
    lies in the range of the texels its own filter weighs."""
    mat, view = _tiny_case(filt)
    N = 3000
    lanes = [9, 10, 20]
    for est in ESTS:
        for clamp in (False, True):
            m = O.est_mode(mode, est, clamp)
            runs = np.array([O.render(mat, view, m, seed=s, nthreads=1, want_channels=True)[2][..., :4]
                             for s in range(N)])
            for lane in lanes:
                x, y = lane % 8, lane // 8
                vals, probs, mean, c = _enumerate(est, clamp, mat, view, mode, lane)
                var = (probs[:, None] * (vals - mean) ** 2).sum(0)
                mc = runs[:, y, x].mean(0)
                assert np.all(np.abs(mc - mean) <= 5 * np.sqrt(var / N) + 1e-6), (est, clamp, lane)
                if est in (O.EST_MIS, O.EST_PMIS) and not clamp:
                    assert np.allclose(mean, _exact_filter(mat, filt, c), atol=1e-12)


def test_estimator_ordering_on_the_magnified_scene():
    """Section 5.1 (bilinear, 3x3 footprints, magnified): the weighted estimator has the lowest
    error, clamped regression is close behind, clamping helps IS / MIS / pairwise MIS, and plain IS
    is the worst."""
    mat = W.material_c1()
    view = W.screen_aligned_view(96, 96, 64, 64, 4.0, 0, origin=(3.3, 7.6))
    ref = O.render_exact_f64(mat, view)[0][..., :3]

    def psnr(mode):
        e = np.mean([np.mean((O.render(mat, view, mode, seed=s)[0][..., :3] - ref) ** 2) for s in range(4)])
        return -10 * np.log10(e)

    wis = psnr(O.WAVE3)
    one = psnr(O.ONE_TAP)
    plain = {e: psnr(O.est_mode(O.WAVE3, e)) for e in ESTS}
    clamped = {e: psnr(O.est_mode(O.WAVE3, e, True)) for e in ESTS}
    for e in ESTS:
        assert wis > plain[e] and wis > clamped[e]
        assert clamped[e] >= plain[e] - 0.05
    assert plain[O.EST_IS] == min(plain.values())
    assert clamped[O.EST_REG] == max(clamped.values())
    assert wis - clamped[O.EST_REG] < 1.5
    assert wis > one and clamped[O.EST_REG] > one


def test_estimator_mode_validation():
    mat = W.material_c1()
    view = W.screen_aligned_view(16, 8, 64, 64, 4.0, 0)
    with pytest.raises(ValueError):
        O.render(mat, view, O.est_mode(O.ONE_TAP, O.EST_IS))  # needs sharing
    with pytest.raises(ValueError):
        O.render(mat, view, O.WAVE3 | O.FLAG_CLAMP)  # the weighted estimator needs no clamp
    with pytest.raises(ValueError):
        O.render(mat, view, O.est_mode(O.WAVE3, O.EST_MIS) | O.FLAG_EXACT)
