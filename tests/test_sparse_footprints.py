"""Pseudorandom sparse sharing footprints (Section "Sharing Footprints Within Waves", Appendix
"Pseudorandom Sparse Footprint Generation Algorithm"): the host generator's output against the
properties the paper asks of it, and the oracle's table-driven sharing against its square
footprints. No GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2504_05562_gb300 import stf
from paper_2504_05562_gb300 import workloads as W


def _usage_std(table, tw, th):
    use = np.zeros(32)
    for lane in range(32):
        for j in table[lane]:
            use[j] += 1
    return use.std()


def _square_table(mode, tw, th):
    return np.array([O.footprint(mode, tw, th, lane) for lane in range(32)], np.int8)


@pytest.mark.parametrize("tile", [(8, 4), (4, 8), (16, 2)])
def test_generated_footprints_are_valid_uniform_and_local(tile):
    tw, th = tile
    tab, sc = stf.sparse_footprints(tile=tile, patterns=3, seed=7, picks=2000, restarts=6)
    assert tab.shape == (3, 32, 9)
    for p in range(3):
        for lane in range(32):
            row = list(tab[p, lane])
            assert row[0] == lane and len(set(row)) == 9 and min(row) >= 0 and max(row) < 32
        # the score is the usage standard deviation, and it beats the 3x3 footprints' by far
        assert sc[p] == pytest.approx(_usage_std(tab[p], tw, th), abs=1e-12)
        assert sc[p] < 0.5 * _usage_std(_square_table(O.WAVE3, tw, th), tw, th)
        # locality: elements stay near the lane (sigma 1.4 lanes per axis)
        d = [np.hypot(j % tw - lane % tw, j // tw - lane // tw) for lane in range(32) for j in tab[p, lane][1:]]
        assert np.mean(d) < 2.6
    # patterns differ (cycled over frames to break up structure); deterministic for a seed
    assert not np.array_equal(tab[0], tab[1])
    tab2, _ = stf.sparse_footprints(tile=tile, patterns=3, seed=7, picks=2000, restarts=6)
    assert np.array_equal(tab, tab2)


def test_larger_sigma_spreads_the_footprints():
    """Appendix figure: a larger sigma gives farther lanes and a usage histogram at least as flat."""
    def stats(sigma):
        tab, sc = stf.sparse_footprints(sigma=sigma, patterns=4, seed=3, picks=2000, restarts=6)
        d = np.mean([np.hypot(j % 8 - l % 8, j // 8 - l // 8) for p in range(4) for l in range(32) for j in tab[p, l][1:]])
        return d, sc.mean()
    d_small, s_small = stats(0.8)
    d_large, s_large = stats(2.5)
    assert d_large > d_small + 0.3
    assert s_large <= s_small + 1e-9


def test_oracle_table_sharing_equals_square_footprints():
    """The table-driven footprint path with the 3x3 footprints as its table gives the WAVE3
    estimate bit for bit (the same samples summed in the same order)."""
    mat = W.material_c1()
    view = dict(W.config1_view(), width=64, height=32)
    ref, ridx, _ = O.render(mat, view, O.WAVE3, seed=4)
    sq = np.array([O.footprint(O.WAVE3, 8, 4, lane) for lane in range(32)], np.int8)[None]
    got, gidx, _ = O.render(mat, dict(view, footprints=sq), O.SPARSE9, seed=4)
    assert np.array_equal(gidx, ridx) and np.array_equal(got, ref)


def test_sparse_estimate_stays_in_the_own_filter_range():
    """Eq. estimator-convex: every estimate lies within the range of the texels its own filter
    weighs, whatever lanes the footprint names."""
    mat = W.material_c1()
    view = W.screen_aligned_view(64, 32, 64, 64, 4.0, 0, origin=(2.3, 4.6))
    rng = np.random.default_rng(2)
    tab = np.zeros((2, 32, 9), np.int8)
    for p in range(2):
        for lane in range(32):
            others = rng.permutation([j for j in range(32) if j != lane])[:8]
            tab[p, lane] = [lane] + list(others)
    T = W.decoded_reference(mat)
    for frame in (0, 1):
        _, _, ch = O.render(mat, dict(view, footprints=tab, frame=frame), O.SPARSE9, seed=1, want_channels=True)
        for y in range(32):
            for x in range(64):
                cx, cy = O.texel_coords(view, 64, 64, x, y)
                x0, y0 = int(np.floor(cx)), int(np.floor(cy))
                own = T[np.clip([y0, y0, y0 + 1, y0 + 1], 0, 63), np.clip([x0, x0 + 1, x0, x0 + 1], 0, 63)]
                assert np.all(ch[y, x, :4] >= own.min(0) - 1e-6) and np.all(ch[y, x, :4] <= own.max(0) + 1e-6)


def test_malformed_patterns_rejected_on_host():
    bad = np.tile(np.arange(9, dtype=np.int8), (1, 32, 1))  # lane l's row does not start with l
    with pytest.raises(stf.StfError, match="own lane"):
        stf.set_sparse_footprints(bad)
    ok = np.array([[[l] + [(l + k) % 32 for k in range(1, 9)] for l in range(32)]], np.int8)
    rep = ok.copy()
    rep[0, 5, 3] = rep[0, 5, 2]
    with pytest.raises(stf.StfError, match="repeated"):
        stf.set_sparse_footprints(rep)


def _bank_replays(tab):
    """Shared-memory replays of reading the tables step by step: a quarter-warp's 8 lanes are served
    together and lane r's 48-byte record sits in bank groups (3 r + k) mod 8, so different records
    with equal r mod 8 in one quarter are served one after another."""
    total = 0
    for p in range(tab.shape[0]):
        for s in range(tab.shape[2]):
            for q in range(4):
                rec = [int(r) for r in tab[p, 8 * q:8 * q + 8, s]]
                total += max(len({r for r in rec if r % 8 == g}) for g in range(8)) - 1
    return total


@pytest.mark.parametrize("tile", [(8, 4), (4, 8), (16, 2)])
def test_generated_order_avoids_bank_conflicts(tile):
    """The generator orders each lane's set so that a reading step's records fall in distinct bank
    groups per quarter-warp: far fewer replays than the same sets in a random order."""
    tab, _ = stf.sparse_footprints(tile=tile, patterns=4, seed=3)
    rng = np.random.default_rng(0)
    shuffled = tab.copy()
    for p in range(tab.shape[0]):
        for lane in range(32):
            rest = shuffled[p, lane, 1:].copy()
            rng.shuffle(rest)
            shuffled[p, lane, 1:] = rest
    assert _bank_replays(tab) <= 0.2 * _bank_replays(shuffled)
    assert all(tab[p, lane, 0] == lane for p in range(4) for lane in range(32))
