// Pseudorandom sparse sharing footprints (Section "Sharing Footprints Within Waves", Appendix
// "Pseudorandom Sparse Footprint Generation Algorithm"): for every lane of a TW x TH warp tile, a
// set of `count` lanes (the lane itself and count - 1 others) whose samples it shares, chosen so
// that every lane is used about equally often, while staying near the lane.
//
// Three stages, repeated from scratch `restarts` times (the best result kept):
//   1. per lane, `candidates` candidate sets: the lane itself, then lanes at normally distributed
//      offsets (standard deviation sigma per axis, rounded to the nearest lane) inside the tile,
//      repeats discarded; a lane near the tile's border, whose draws keep falling outside, draws
//      with sigma grown by 10 % every 64 misses (up to twice the tile's longer side);
//   2. `picks` random choices of one candidate per lane; score = the standard deviation of how
//      often each lane appears in the chosen sets; keep the best;
//   3. coordinate descent: for each lane in turn, switch to whichever of its candidates lowers the
//      score; sweep until no switch helps.
// Host code; the tables go to the device with stf_set_sparse_footprints. Random numbers come from
// splitmix64 (Steele, Lea and Flood 2014), normal variates from the Box-Muller transform.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "stf.h"
#include "stf_internal.h"

namespace {

struct SplitMix64 {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
    double normal()
    {
        double u1 = uniform();
        while (u1 <= 0.0) u1 = uniform();
        const double u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

constexpr int kLanes = 32;

// Standard deviation of the lanes' usage counts of a choice of one candidate set per lane.
double score(const std::vector<std::vector<std::vector<int>>>& cand, const std::vector<int>& pick)
{
    int use[kLanes] = {0};
    for (int l = 0; l < kLanes; ++l)
        for (int j : cand[l][pick[l]]) ++use[j];
    double mean = 0.0;
    for (int l = 0; l < kLanes; ++l) mean += use[l];
    mean /= kLanes;
    double var = 0.0;
    for (int l = 0; l < kLanes; ++l) var += (use[l] - mean) * (use[l] - mean);
    return std::sqrt(var / kLanes);
}

}  // namespace

extern "C" stf_status stf_sparse_footprints(int tile_w, int tile_h, int count, double sigma, int candidates, int picks,
                                            int restarts, unsigned long long seed, int patterns, signed char* table,
                                            double* scores)
{
    if (tile_w < 1 || tile_h < 1 || tile_w * tile_h != kLanes)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_sparse_footprints: tile %dx%d is not 32 lanes", tile_w, tile_h);
    if (count < 1 || count > STF_SPARSE_MAX_COUNT || !(sigma > 0.0) || candidates < 1 || picks < 1 || restarts < 1 ||
        patterns < 1 || !table)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_sparse_footprints: bad arguments");
    SplitMix64 rng{seed};
    for (int pat = 0; pat < patterns; ++pat) {
        double best_score = INFINITY;
        std::vector<std::vector<int>> best(kLanes);
        for (int rs = 0; rs < restarts; ++rs) {
            // stage 1: candidate sets
            std::vector<std::vector<std::vector<int>>> cand(kLanes, std::vector<std::vector<int>>(candidates));
            for (int l = 0; l < kLanes; ++l) {
                const int lx = l % tile_w, ly = l / tile_w;
                for (int c = 0; c < candidates; ++c) {
                    std::vector<int>& set = cand[l][c];
                    set.push_back(l);
                    double s = sigma;
                    // wider than the tile, the draws are all but uniform over it: stop growing
                    const double smax = std::fmax(sigma, 2.0 * (tile_w > tile_h ? tile_w : tile_h));
                    int misses = 0;
                    while ((int)set.size() < count) {
                        const int x = lx + (int)std::lround(rng.normal() * s);
                        const int y = ly + (int)std::lround(rng.normal() * s);
                        const int j = y * tile_w + x;
                        bool ok = x >= 0 && x < tile_w && y >= 0 && y < tile_h;
                        for (int e : set) ok = ok && e != j;
                        if (ok) {
                            set.push_back(j);
                        } else if (++misses % 64 == 0) {
                            s = std::fmin(s * 1.1, smax);  // relax near the borders and corners
                        }
                    }
                }
            }
            // stage 2: best of `picks` random choices
            std::vector<int> pick(kLanes), trial(kLanes);
            double sc = INFINITY;
            for (int t = 0; t < picks; ++t) {
                for (int l = 0; l < kLanes; ++l) trial[l] = (int)(rng.next() % (uint64_t)candidates);
                const double s2 = score(cand, trial);
                if (s2 < sc) { sc = s2; pick = trial; }
            }
            // stage 3: coordinate descent
            for (bool improved = true; improved;) {
                improved = false;
                for (int l = 0; l < kLanes; ++l) {
                    for (int c = 0; c < candidates; ++c) {
                        if (c == pick[l]) continue;
                        const int keep = pick[l];
                        pick[l] = c;
                        const double s2 = score(cand, pick);
                        if (s2 < sc - 1e-12) { sc = s2; improved = true; }
                        else pick[l] = keep;
                    }
                }
            }
            if (sc < best_score) {
                best_score = sc;
                for (int l = 0; l < kLanes; ++l) best[l] = cand[l][pick[l]];
            }
        }
        for (int l = 0; l < kLanes; ++l)
            for (int i = 0; i < count; ++i) table[((size_t)pat * kLanes + l) * count + i] = (signed char)best[l][i];
        if (scores) scores[pat] = best_score;
    }
    return STF_OK;
}
