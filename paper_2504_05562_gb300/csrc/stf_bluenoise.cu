// Blue-noise masks for the texel-selection uniforms (Section "Blue Noise Mask Improvements").
//
// Scalar masks made with the void-and-cluster method (Ulichney 1993) on a size x size torus: the
// energy of a pixel is the sum over the set pixels q of exp(-d(p, q)^2 / (2 sigma^2)), d the
// toroidal distance. The paper's modification splats twice as much energy onto the other pixels of
// the same aligned 2x2 quad (quad sharing reuses exactly those neighbours, so their values should
// differ most). Two independent realizations give the two uniforms of a pixel (the paper's
// replacement for a Vec2 mask). The result is a rank per pixel, 0 .. size^2 - 1 (each once).
//
// Steps (Ulichney): an initial binary pattern of size^2 / 10 random ones is relaxed by moving the
// one in the tightest cluster (highest energy) to the largest void (lowest energy) until that
// move would undo itself; phase 1 ranks the initial ones by removing tightest clusters (ranks
// counting down); phase 2 fills largest voids up to half the pixels; phase 3 keeps filling the
// largest void (the tightest cluster of zeros) until every pixel is ranked. Host code, splitmix64
// for the initial pattern.
#include <cmath>
#include <cstdint>
#include <vector>

#include "stf.h"
#include "stf_internal.h"

namespace {

struct Mask {
    int n;
    double sigma;
    bool quad;
    std::vector<double> kern;  // energy of an offset (dx, dy) on the torus, quad rule applied per pair
    std::vector<double> e;     // energy per pixel
    std::vector<uint8_t> on;

    Mask(int n_, double s, bool q) : n(n_), sigma(s), quad(q), kern((size_t)n_ * n_), e((size_t)n_ * n_, 0.0), on((size_t)n_ * n_, 0)
    {
        for (int dy = 0; dy < n; ++dy)
            for (int dx = 0; dx < n; ++dx) {
                const int ax = dx < n - dx ? dx : n - dx, ay = dy < n - dy ? dy : n - dy;
                kern[(size_t)dy * n + dx] = std::exp(-(double)(ax * ax + ay * ay) / (2.0 * sigma * sigma));
            }
    }
    double k(int p, int q) const
    {
        const int px = p % n, py = p / n, qx = q % n, qy = q / n;
        const int dx = (px - qx + n) % n, dy = (py - qy + n) % n;
        double v = kern[(size_t)dy * n + dx];
        if (quad && p != q && (px >> 1) == (qx >> 1) && (py >> 1) == (qy >> 1)) v *= 2.0;
        return v;
    }
    void set(int q, bool v)
    {
        on[q] = v;
        const double sgn = v ? 1.0 : -1.0;
        for (int p = 0; p < n * n; ++p) e[p] += sgn * k(p, q);
    }
    int tightest() const  // highest energy among ones
    {
        int best = -1;
        for (int p = 0; p < n * n; ++p)
            if (on[p] && (best < 0 || e[p] > e[best])) best = p;
        return best;
    }
    int largest_void() const  // lowest energy among zeros
    {
        int best = -1;
        for (int p = 0; p < n * n; ++p)
            if (!on[p] && (best < 0 || e[p] < e[best])) best = p;
        return best;
    }
};

uint64_t splitmix(uint64_t& s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

void void_and_cluster(int n, double sigma, bool quad, uint64_t seed, uint16_t* rank)
{
    const int N = n * n;
    Mask m(n, sigma, quad);
    uint64_t s = seed;
    const int ones = N / 10 > 0 ? N / 10 : 1;
    for (int placed = 0; placed < ones;) {
        const int q = (int)(splitmix(s) % (uint64_t)N);
        if (!m.on[q]) { m.set(q, true); ++placed; }
    }
    for (int it = 0; it < 16 * N; ++it) {  // relaxation (converges in far fewer moves)
        const int c = m.tightest();
        m.set(c, false);
        const int v = m.largest_void();
        if (v == c) { m.set(c, true); break; }
        m.set(v, true);
    }
    const std::vector<uint8_t> initial = m.on;
    const std::vector<double> e0 = m.e;
    for (int r = ones - 1; r >= 0; --r) {  // phase 1
        const int c = m.tightest();
        m.set(c, false);
        rank[c] = (uint16_t)r;
    }
    m.on = initial;
    m.e = e0;
    for (int r = ones; r < N; ++r) {  // phases 2 and 3
        const int v = m.largest_void();
        m.set(v, true);
        rank[v] = (uint16_t)r;
    }
}

}  // namespace

extern "C" stf_status stf_blue_noise_masks(int size, double sigma, int quad_energy, unsigned long long seed,
                                           uint16_t* ranks)
{
    if (size < 4 || size > 256 || (size & 1) || !(sigma > 0.0) || !ranks)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_blue_noise_masks: bad arguments");
    for (int c = 0; c < 2; ++c)
        void_and_cluster(size, sigma, quad_energy != 0, seed * 2 + (unsigned long long)c + 1, ranks + (size_t)c * size * size);
    return STF_OK;
}
