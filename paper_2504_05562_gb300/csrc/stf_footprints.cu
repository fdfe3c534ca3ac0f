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
// A last pass orders each lane's set for the device's shared-memory banks (order_for_banks); it
// changes no set. Host code; the tables go to the device with stf_set_sparse_footprints. Random
// numbers come from splitmix64 (Steele, Lea and Flood 2014), normal variates from the Box-Muller
// transform.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
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

// Shared-memory replays of one reading step: each lane reads the 48-byte record of the lane it
// names, as three 16-byte pieces; a quarter-warp's 8 lanes are served together, and record r's
// piece k sits in bank group (3 r + k) mod 8, so lanes of a quarter that read different records
// with the same r mod 8 are served one after another (the same record is broadcast).
int step_replays(const int (&rec)[kLanes])
{
    int replays = 0;
    for (int q = 0; q < 4; ++q) {
        int worst = 1;
        for (int g = 0; g < 8; ++g) {
            int distinct[8], n = 0;
            for (int l = 8 * q; l < 8 * q + 8; ++l) {
                if ((rec[l] & 7) != g) continue;
                bool seen = false;
                for (int i = 0; i < n; ++i) seen = seen || distinct[i] == rec[l];
                if (!seen) distinct[n++] = rec[l];
            }
            worst = n > worst ? n : worst;
        }
        replays += worst - 1;
    }
    return replays;
}

// Orders every lane's shared lanes (its own lane stays first) so that, step by step, the lanes of
// each quarter-warp read records in distinct bank groups: per step, a maximum matching of the
// quarter's lanes to bank groups among their remaining entries (augmenting paths, lanes and
// entries tried in a random order), the unmatched lanes taking the entry that adds the fewest
// replays; the best of `tries` randomised schedules per quarter is kept. Only the reading order
// changes: every lane keeps its set, so the estimate is the same sum taken in another order.
void order_for_banks(std::vector<std::vector<int>>& rows, SplitMix64& rng, int tries)
{
    const int n = (int)rows[0].size();
    for (int q = 0; q < 4; ++q) {
        std::vector<std::vector<int>> best;
        int best_cost = 1 << 30;
        for (int t = 0; t < tries && best_cost > 0; ++t) {
            std::vector<std::vector<int>> left(8), out(8);
            for (int i = 0; i < 8; ++i) {
                left[i].assign(rows[8 * q + i].begin() + 1, rows[8 * q + i].end());
                out[i].push_back(rows[8 * q + i][0]);
                for (int k = (int)left[i].size() - 1; k > 0; --k)  // random order of the entries
                    std::swap(left[i][k], left[i][(int)(rng.next() % (uint64_t)(k + 1))]);
            }
            int cost = 0;
            for (int s = 1; s < n; ++s) {
                // lanes -> bank groups (match_g[g] = lane, choice[lane] = entry index)
                int match_g[8], choice[8];
                for (int g = 0; g < 8; ++g) match_g[g] = -1;
                for (int i = 0; i < 8; ++i) choice[i] = -1;
                int order[8];
                for (int i = 0; i < 8; ++i) order[i] = i;
                for (int k = 7; k > 0; --k) std::swap(order[k], order[(int)(rng.next() % (uint64_t)(k + 1))]);
                for (int oi = 0; oi < 8; ++oi) {
                    bool visited[8] = {false};
                    // augmenting path from lane order[oi] (depth-first, explicit recursion)
                    struct Aug {
                        std::vector<std::vector<int>>& left; int* match_g; int* choice; bool* visited;
                        bool run(int lane)
                        {
                            for (int e = 0; e < (int)left[lane].size(); ++e) {
                                const int g = left[lane][e] & 7;
                                if (visited[g]) continue;
                                visited[g] = true;
                                if (match_g[g] < 0 || run(match_g[g])) {
                                    match_g[g] = lane;
                                    choice[lane] = e;
                                    return true;
                                }
                            }
                            return false;
                        }
                    } aug{left, match_g, choice, visited};
                    aug.run(order[oi]);
                }
                int rec[kLanes];
                for (int l = 0; l < kLanes; ++l) rec[l] = l;  // other quarters: conflict-free stand-ins
                for (int i = 0; i < 8; ++i)
                    if (choice[i] >= 0) rec[8 * q + i] = left[i][choice[i]];
                for (int i = 0; i < 8; ++i) {
                    if (choice[i] >= 0) continue;
                    int pick = 0, pick_cost = 1 << 30;
                    for (int e = 0; e < (int)left[i].size(); ++e) {
                        rec[8 * q + i] = left[i][e];
                        const int c = step_replays(rec);
                        if (c < pick_cost) { pick_cost = c; pick = e; }
                    }
                    choice[i] = pick;
                    rec[8 * q + i] = left[i][pick];
                }
                cost += step_replays(rec);
                for (int i = 0; i < 8; ++i) {
                    out[i].push_back(left[i][choice[i]]);
                    left[i].erase(left[i].begin() + choice[i]);
                }
            }
            if (cost < best_cost) { best_cost = cost; best = out; }
        }
        for (int i = 0; i < 8; ++i) rows[8 * q + i] = best[i];
    }
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
        order_for_banks(best, rng, 64);
        for (int l = 0; l < kLanes; ++l)
            for (int i = 0; i < count; ++i) table[((size_t)pat * kLanes + l) * count + i] = (signed char)best[l][i];
        if (scores) scores[pat] = best_score;
    }
    return STF_OK;
}
