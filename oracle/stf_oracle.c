/*
 * CPU oracle for magnified stochastic texture filtering (STF) with sample reuse.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's CPU
 * baseline. The GPU library never links or calls it, and it shares no code with it.
 *
 * Plain, slow and written to be checked against the paper by eye:
 *   - texture filtering as a weighted sum over texels (Eq. texture-continuous-sum, Section 2.1);
 *   - one-tap STF: pick one texel with probability equal to its filter weight (Eq. mc-estimator,
 *     Section 2.2 and the derivation in Section S1);
 *   - texel float coordinates uv * size - 0.5 and the bilinear filter PMF (Section 4.5 listing,
 *     Section S6);
 *   - the uniform cubic B-spline filter (Section 5.4 names it; the kernel is the textbook one);
 *   - sample sharing inside a 32-lane warp tile and the bounded weighted importance sampling
 *     combine w_i = f_c(x_i) / f_i(x_i), result = sum w_i T_i / sum w_j (Eqs. bart-weighted-
 *     estimator, estimator-for-stf, estimator-convex; Section 4.2 and Section 4.5);
 *   - square sharing footprints in the wave (Section 4.3.1).
 *
 * Compile with -ffp-contract=off: each float operation below is rounded once, in the order
 * written. Selection decisions (which texel) depend only on this op sequence.
 *
 * pcg4d (the sample source) is pinned without published test vectors: its output, run back
 * through the inverse of the published steps, gives the input back (a wrong constant, shift,
 * lane index or dropped step fails this), and its avalanche and the uniforms' statistics
 * (uniformity, independence, distinct streams) are checked; the GPU implements the same
 * definition.
 */
#include "stf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI_F 3.14159265f
#define ORACLE_PI_D 3.14159265358979323846
#define C_LO (-16384.0f)
#define C_HI (32000.0f)

/* ------------------------------------------------------------------ RNG */

/* pcg4d from Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 9(3), 2020:
 * an LCG step on all four lanes, a round of cross-lane multiply-adds, a xor-shift by 16,
 * and a second round of cross-lane multiply-adds. All arithmetic is modulo 2^32. */
void stf_ref_pcg4d(uint32_t v[4])
{
    for (int i = 0; i < 4; ++i) v[i] = v[i] * 1664525u + 1013904223u;
    v[0] += v[1] * v[3];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
    v[3] += v[1] * v[2];
    for (int i = 0; i < 4; ++i) v[i] ^= v[i] >> 16;
    v[0] += v[1] * v[3];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
    v[3] += v[1] * v[2];
}

void stf_ref_uniforms(int x, int y, int frame, int view_id, uint64_t seed, float* ux, float* uy)
{
    uint32_t v[4];
    v[0] = (uint32_t)x;
    v[1] = (uint32_t)y;
    v[2] = (uint32_t)frame | ((uint32_t)view_id << 16);
    v[3] = (uint32_t)seed ^ (uint32_t)(seed >> 32);
    stf_ref_pcg4d(v);
    /* the top 24 bits as an exact dyadic float in [0, 1) */
    *ux = (float)(v[0] >> 8) * (1.0f / 16777216.0f);
    *uy = (float)(v[1] >> 8) * (1.0f / 16777216.0f);
}

/* -------------------------------------------------------------- filters */

/* Bilinear (tent) weight per axis: clamp(1 - |d|, 0, 1) (Section S6). */
static float w_bilinear(float d)
{
    float t = 1.0f - fabsf(d);
    if (t < 0.0f) t = 0.0f;
    if (t > 1.0f) t = 1.0f;
    return t;
}

/* Uniform cubic B-spline per axis, a = |d|:
 *   a < 1 : (3a^3 - 6a^2 + 4) / 6, evaluated as ((3a - 6) a) a + 4, times 1/6
 *   a < 2 : (2 - a)^3 / 6
 *   else  : 0 */
static float w_bspline(float d)
{
    float a = fabsf(d);
    if (a < 1.0f) {
        float t = 3.0f * a;
        t = t - 6.0f;
        t = t * a;
        t = t * a;
        t = t + 4.0f;
        return t * (1.0f / 6.0f);
    }
    if (a < 2.0f) {
        float s = 2.0f - a;
        float t = s * s;
        t = t * s;
        return t * (1.0f / 6.0f);
    }
    return 0.0f;
}

float stf_ref_weight(int filter, float d)
{
    return filter == REF_BILINEAR ? w_bilinear(d) : w_bspline(d);
}

double stf_ref_weight_f64(int filter, double d)
{
    double a = fabs(d);
    if (filter == REF_BILINEAR) return a < 1.0 ? 1.0 - a : 0.0;
    if (a < 1.0) return (3.0 * a * a * a - 6.0 * a * a + 4.0) / 6.0;
    if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
    return 0.0;
}

/* First lattice tap offset relative to floor(c), and the tap count. */
static int tap_first(int filter) { return filter == REF_BILINEAR ? 0 : -1; }
static int tap_count(int filter) { return filter == REF_BILINEAR ? 2 : 4; }

/* One-tap selection along one axis: the taps in increasing lattice order, their weights, the
 * running FP32 sum as a CDF; the first tap with u < CDF is chosen. If rounding leaves u above
 * the last CDF value, the last tap with positive weight is chosen. */
void stf_ref_select_axis(int filter, float c, float u, int* n, float* w)
{
    int i0 = (int)floorf(c);
    int k0 = tap_first(filter), nt = tap_count(filter);
    float wt[4];
    for (int t = 0; t < nt; ++t) wt[t] = stf_ref_weight(filter, c - (float)(i0 + k0 + t));
    float cdf = 0.0f;
    int pick = -1;
    for (int t = 0; t < nt; ++t) {
        cdf = cdf + wt[t];
        if (u < cdf) { pick = t; break; }
    }
    if (pick < 0) {
        for (int t = nt - 1; t >= 0; --t)
            if (wt[t] > 0.0f) { pick = t; break; }
    }
    *n = i0 + k0 + pick;
    *w = wt[pick];
}

/* -------------------------------------------------------------- decoders */

/* IEEE-754 binary16: 1 sign, 5 exponent (bias 15), 10 fraction bits. */
static float dec_fp16(uint32_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
    float r;
    if (e == 0) r = ldexpf((float)f, -24);
    else if (e == 31) r = f ? NAN : INFINITY;
    else r = ldexpf((float)(1024 + f), e - 25);
    return s ? -r : r;
}

/* bfloat16: the upper 16 bits of a binary32. */
static float dec_bf16(uint32_t b)
{
    uint32_t u = (b & 0xffffu) << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

/* OCP 8-bit float E4M3 (the "FN" variant): 1 sign, 4 exponent (bias 7), 3 fraction bits;
 * no infinities, S.1111.111 is NaN, exponent 0 is subnormal. */
static float dec_e4m3(uint32_t q)
{
    int s = (q >> 7) & 1, e = (q >> 3) & 15, f = q & 7;
    float r;
    if (e == 0) r = ldexpf((float)f, -9);
    else if (e == 15 && f == 7) r = NAN;
    else r = ldexpf((float)(8 + f), e - 10);
    return s ? -r : r;
}

float stf_ref_decode(int fmt, uint32_t code)
{
    switch (fmt) {
    case REF_FP32: { float r; memcpy(&r, &code, 4); return r; }
    case REF_FP16: return dec_fp16(code);
    case REF_BF16: return dec_bf16(code);
    case REF_E4M3: return dec_e4m3(code);
    case REF_UNORM8: return (float)(code & 255u) / 255.0f;
    }
    return NAN;
}

static int fmt_bytes(int fmt)
{
    switch (fmt) {
    case REF_FP32: return 4;
    case REF_FP16: case REF_BF16: return 2;
    default: return 1;
    }
}

static int material_channels(const ref_material* m)
{
    if (m->nn_lat16) return 8;
    int c = 0;
    for (int p = 0; p < m->num_planes; ++p) c += m->plane_ch[p];
    return c;
}

/* Decoded channels of texel (x, y) with clamp-to-edge addressing (reading: the paper does not
 * state an addressing mode). Channels beyond the material's count are 0. */
static void fetch_texel(const ref_material* m, int x, int y, float* out)
{
    if (x < 0) x = 0;
    if (x > m->width - 1) x = m->width - 1;
    if (y < 0) y = 0;
    if (y > m->height - 1) y = m->height - 1;
    if (m->nn_lat16) {
        int packed = x | (y << 16);
        stf_ref_neural_decode(m->nn_lat16, m->nn_gw, m->nn_gh, m->nn_r, m->nn_w16, 0, m->nn_b32, &packed, 1, out);
        return;
    }
    int C = material_channels(m);
    int ch = 0;
    for (int p = 0; p < m->num_planes; ++p) {
        int nb = fmt_bytes(m->plane_fmt[p]);
        const uint8_t* base = (const uint8_t*)m->plane_data[p];
        size_t off = ((size_t)y * m->width + x) * m->plane_ch[p] * nb;
        for (int c = 0; c < m->plane_ch[p]; ++c, ++ch) {
            uint32_t code = 0;
            memcpy(&code, base + off + (size_t)c * nb, nb); /* little-endian hosts */
            out[ch] = stf_ref_decode(m->plane_fmt[p], code);
        }
    }
    if (m->scales) {
        int st = m->scale_tile;
        int ntx = (m->width + st - 1) / st;
        const float* s = m->scales + ((size_t)(y / st) * ntx + (x / st)) * C;
        for (int c = 0; c < C; ++c) out[c] = out[c] * s[c];
    }
    for (int c = C; c < REF_MAX_CH; ++c) out[c] = 0.0f;
}

void stf_ref_fetch_texel(const ref_material* m, int x, int y, float* out) { fetch_texel(m, x, y, out); }

/* ------------------------------------------------------------ footprints */

/* Lanes a lane reads from, row-major inside its block (Section 4.3.1). Lane = ly * tw + lx.
 *   QUAD2: the aligned 2x2 quad holding the lane;
 *   WAVEk: a kx-by-ky block, ky = min(k, th), kx = min(tw, round(k*k / ky)), placed at the
 *          lane's position minus (k-1)/2 and shifted to lie inside the tile (reading: the
 *          paper's footprint figures are not in the text). */
int stf_ref_footprint(int mode, int tw, int th, int lane, int* list)
{
    int lx = lane % tw, ly = lane / tw;
    int ox, oy, kx, ky;
    if (mode == REF_ONE_TAP || mode == REF_FULL) { list[0] = lane; return 1; }
    if (mode == REF_QUAD2) {
        ox = lx - (lx % 2); oy = ly - (ly % 2); kx = 2; ky = 2;
    } else {
        int k = mode == REF_WAVE2 ? 2 : (mode == REF_WAVE3 ? 3 : 4);
        ky = k < th ? k : th;
        kx = (k * k + ky / 2) / ky;
        if (kx > tw) kx = tw;
        ox = lx - (kx - 1) / 2;
        if (ox < 0) ox = 0;
        if (ox > tw - kx) ox = tw - kx;
        oy = ly - (ky - 1) / 2;
        if (oy < 0) oy = 0;
        if (oy > th - ky) oy = th - ky;
    }
    int n = 0;
    for (int r = 0; r < ky; ++r)
        for (int c = 0; c < kx; ++c) list[n++] = (oy + r) * tw + (ox + c);
    return n;
}

/* ---------------------------------------------------------- coordinates */

/* Pixel centre through the view's homography to uv, then uv * size - 0.5 (Section 4.5
 * listing). Each product and sum is rounded separately, left to right. The result is clamped
 * to [-16384, 32000] (NaN goes to -16384) so that lattice indices stay in 16-bit range. */
void stf_ref_texel_coords(const ref_view* v, int tex_w, int tex_h, int x, int y, float* cx, float* cy)
{
    const float* H = v->H;
    float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float hx = H[0] * px + H[1] * py + H[2];
    float hy = H[3] * px + H[4] * py + H[5];
    float hw = H[6] * px + H[7] * py + H[8];
    float u = hx / hw, w = hy / hw;
    float a = u * (float)tex_w - 0.5f;
    float b = w * (float)tex_h - 0.5f;
    *cx = fminf(fmaxf(a, C_LO), C_HI);
    *cy = fminf(fmaxf(b, C_LO), C_HI);
}

static void uv_of_pixel(const ref_view* v, int x, int y, float* u, float* w)
{
    const float* H = v->H;
    float px = (float)x + 0.5f, py = (float)y + 0.5f;
    float hx = H[0] * px + H[1] * py + H[2];
    float hy = H[3] * px + H[4] * py + H[5];
    float hw = H[6] * px + H[7] * py + H[8];
    *u = hx / hw;
    *w = hy / hw;
}

/* -------------------------------------------------------------- shading */

/* Shading after filtering (filtering before shading is the ground truth, Section 1 and
 * Section S2). Tangent frame of the ground plane: T = +x, B = +z, N = +y. Lambert plus GGX with
 * the height-correlated Smith visibility and Schlick Fresnel (F0 = 0.04); irradiance pi so that
 * the diffuse term is albedo * (N.L). The GGX denominator (N.H)^2 (a^2 - 1) + 1 is written as
 * a^2 (N.H)^2 + |N x H|^2, which is the same quantity for unit vectors. */
void stf_ref_shade(const ref_view* v, const float* ch, float u, float vv, float* rgba)
{
    float alb[3] = {1.0f, 1.0f, 1.0f};
    if (v->ch_albedo >= 0) { alb[0] = ch[v->ch_albedo]; alb[1] = ch[v->ch_albedo + 1]; alb[2] = ch[v->ch_albedo + 2]; }
    float X = 0.0f, Y = 0.0f;
    if (v->ch_normal >= 0) { X = ch[v->ch_normal]; Y = ch[v->ch_normal + 1]; }
    float z2 = 1.0f - X * X - Y * Y;
    float Z = sqrtf(fmaxf(z2, 0.0f));
    float nl = sqrtf(X * X + Z * Z + Y * Y);
    float N[3] = {X / nl, Z / nl, Y / nl};
    float r = v->ch_rough >= 0 ? ch[v->ch_rough] : v->roughness;
    r = fmaxf(r, 0.02f);
    float ao = v->ch_ao >= 0 ? ch[v->ch_ao] : 1.0f;
    const float* m = v->plane_to_world;
    float P[3] = {m[0] * u + m[1] * vv + m[2], 0.0f, m[3] * u + m[4] * vv + m[5]};
    float V[3] = {v->cam_pos[0] - P[0], v->cam_pos[1] - P[1], v->cam_pos[2] - P[2]};
    float vl = sqrtf(V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
    V[0] = V[0] / vl; V[1] = V[1] / vl; V[2] = V[2] / vl;
    const float* L = v->light_dir;
    float NL = N[0] * L[0] + N[1] * L[1] + N[2] * L[2];
    rgba[3] = 1.0f;
    if (!(NL > 0.0f)) { rgba[0] = rgba[1] = rgba[2] = 0.0f; return; }
    float NV = fmaxf(N[0] * V[0] + N[1] * V[1] + N[2] * V[2], 1e-4f);
    float Hv[3] = {L[0] + V[0], L[1] + V[1], L[2] + V[2]};
    float hl = sqrtf(Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2]);
    Hv[0] = Hv[0] / hl; Hv[1] = Hv[1] / hl; Hv[2] = Hv[2] / hl;
    float NH = fmaxf(N[0] * Hv[0] + N[1] * Hv[1] + N[2] * Hv[2], 0.0f);
    float VH = fmaxf(V[0] * Hv[0] + V[1] * Hv[1] + V[2] * Hv[2], 0.0f);
    float c0 = N[1] * Hv[2] - N[2] * Hv[1];
    float c1 = N[2] * Hv[0] - N[0] * Hv[2];
    float c2 = N[0] * Hv[1] - N[1] * Hv[0];
    float s2 = c0 * c0 + c1 * c1 + c2 * c2;
    float alpha = r * r;
    float a2 = alpha * alpha;
    float t = a2 * NH * NH + s2;
    float D = a2 / (ORACLE_PI_F * t * t);
    float gv = NL * sqrtf(NV * NV * (1.0f - a2) + a2);
    float gl = NV * sqrtf(NL * NL * (1.0f - a2) + a2);
    float Vis = 0.5f / (gv + gl);
    float q = 1.0f - VH;
    float q2 = q * q;
    float q5 = q2 * q2 * q;
    float F = 0.04f + 0.96f * q5;
    float spec = D * Vis * F;
    float ps = ORACLE_PI_F * spec;
    for (int c = 0; c < 3; ++c) rgba[c] = ao * NL * (alb[c] + ps);
}

void stf_ref_shade_f64(const ref_view* v, const double* ch, double u, double vv, double* rgba)
{
    double alb[3] = {1.0, 1.0, 1.0};
    if (v->ch_albedo >= 0) { alb[0] = ch[v->ch_albedo]; alb[1] = ch[v->ch_albedo + 1]; alb[2] = ch[v->ch_albedo + 2]; }
    double X = 0.0, Y = 0.0;
    if (v->ch_normal >= 0) { X = ch[v->ch_normal]; Y = ch[v->ch_normal + 1]; }
    double z2 = 1.0 - X * X - Y * Y;
    double Z = sqrt(z2 > 0.0 ? z2 : 0.0);
    double nl = sqrt(X * X + Z * Z + Y * Y);
    double N[3] = {X / nl, Z / nl, Y / nl};
    double r = v->ch_rough >= 0 ? ch[v->ch_rough] : (double)v->roughness;
    if (r < 0.02) r = 0.02;
    double ao = v->ch_ao >= 0 ? ch[v->ch_ao] : 1.0;
    const float* m = v->plane_to_world;
    double P[3] = {(double)m[0] * u + (double)m[1] * vv + (double)m[2], 0.0,
                   (double)m[3] * u + (double)m[4] * vv + (double)m[5]};
    double V[3] = {v->cam_pos[0] - P[0], v->cam_pos[1] - P[1], v->cam_pos[2] - P[2]};
    double vl = sqrt(V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
    V[0] /= vl; V[1] /= vl; V[2] /= vl;
    double L[3] = {v->light_dir[0], v->light_dir[1], v->light_dir[2]};
    double NL = N[0] * L[0] + N[1] * L[1] + N[2] * L[2];
    rgba[3] = 1.0;
    if (!(NL > 0.0)) { rgba[0] = rgba[1] = rgba[2] = 0.0; return; }
    double NV = N[0] * V[0] + N[1] * V[1] + N[2] * V[2];
    if (NV < 1e-4) NV = 1e-4;
    double Hv[3] = {L[0] + V[0], L[1] + V[1], L[2] + V[2]};
    double hl = sqrt(Hv[0] * Hv[0] + Hv[1] * Hv[1] + Hv[2] * Hv[2]);
    Hv[0] /= hl; Hv[1] /= hl; Hv[2] /= hl;
    double NH = N[0] * Hv[0] + N[1] * Hv[1] + N[2] * Hv[2];
    if (NH < 0.0) NH = 0.0;
    double VH = V[0] * Hv[0] + V[1] * Hv[1] + V[2] * Hv[2];
    if (VH < 0.0) VH = 0.0;
    double c0 = N[1] * Hv[2] - N[2] * Hv[1];
    double c1 = N[2] * Hv[0] - N[0] * Hv[2];
    double c2 = N[0] * Hv[1] - N[1] * Hv[0];
    double s2 = c0 * c0 + c1 * c1 + c2 * c2;
    double alpha = r * r, a2 = alpha * alpha;
    double t = a2 * NH * NH + s2;
    double D = a2 / (ORACLE_PI_D * t * t);
    double gv = NL * sqrt(NV * NV * (1.0 - a2) + a2);
    double gl = NV * sqrt(NL * NL * (1.0 - a2) + a2);
    double Vis = 0.5 / (gv + gl);
    double q = 1.0 - VH;
    double F = 0.04 + 0.96 * q * q * q * q * q;
    double spec = D * Vis * F;
    for (int c = 0; c < 3; ++c) rgba[c] = ao * NL * (alb[c] + ORACLE_PI_D * spec);
}

/* Condition of shading with respect to the filtered channels: for each pixel and colour
 * channel, sum_k |d colour / d ch_k| * max(|ch_k|, 1) by central differences in FP64. Used by
 * the tests to bound how far a few-ulp change of the filtered channels can move the shaded
 * colour (the shading is ill-conditioned near the terminator and at grazing normals). */
int stf_ref_shade_sensitivity(const ref_view* v, int C, const float* ch, double* sens, int npix)
{
    const float* H = v->H;
    for (int i = 0; i < npix; ++i) {
        int x = i % v->width, y = i / v->width;
        float u, w;
        {
            float px = (float)x + 0.5f, py = (float)y + 0.5f;
            float hx = H[0] * px + H[1] * py + H[2];
            float hy = H[3] * px + H[4] * py + H[5];
            float hw = H[6] * px + H[7] * py + H[8];
            u = hx / hw;
            w = hy / hw;
        }
        double base[REF_MAX_CH], a[4], b[4];
        for (int c = 0; c < REF_MAX_CH; ++c) base[c] = ch[(size_t)i * REF_MAX_CH + c];
        double acc[3] = {0, 0, 0};
        for (int k = 0; k < C; ++k) {
            double sc = fabs(base[k]) > 1.0 ? fabs(base[k]) : 1.0;
            double h = 1e-7 * sc;
            double save = base[k];
            base[k] = save + h;
            stf_ref_shade_f64(v, base, u, w, a);
            base[k] = save - h;
            stf_ref_shade_f64(v, base, u, w, b);
            base[k] = save;
            for (int c = 0; c < 3; ++c) acc[c] += fabs(a[c] - b[c]) / (2.0 * h) * sc;
        }
        for (int c = 0; c < 3; ++c) sens[(size_t)i * 3 + c] = acc[c];
    }
    return 0;
}

/* ---------------------------------------------------------- FP32 render */

typedef struct {
    const ref_material* m;
    const ref_view* v;
    int mode;                /* sharing mode without flags */
    int exact;               /* REF_FLAG_EXACT given */
    int est, clamp;          /* REF_EST_*, REF_FLAG_CLAMP given */
    int blue;                /* REF_FLAG_BLUE given */
    uint64_t seed;
    float* out_rgba;
    uint32_t* out_idx;
    float* out_ch;
    double* out_rgba64;
    double* out_ch64;
    int tid, nthreads;
} job_t;

static void final_rgba(const ref_view* v, int C, const float* f, float u, float w, float* rgba)
{
    if (v->shading) { stf_ref_shade(v, f, u, w, rgba); return; }
    for (int k = 0; k < 4; ++k) rgba[k] = k < C ? f[k] : (k == 3 ? 1.0f : 0.0f);
}

/* The deterministic filter at (cx, cy): sum over the lattice taps of W(dx) W(dy) T, y outer,
 * x inner, into res. With samples (n > 0: lattice indices six/siy of the lanes in list), every
 * tap of positive weight must be one of the samples and takes that sample's texel; if one is
 * missing, res is left unchanged and 0 is returned. */
static int full_filter(const ref_material* m, int f, int C, float cx, float cy, const int* six, const int* siy,
                       const int* list, int n, float* res)
{
    int i0x = (int)floorf(cx), i0y = (int)floorf(cy);
    int k0 = tap_first(f), nt = tap_count(f);
    float acc[REF_MAX_CH] = {0};
    float Tt[REF_MAX_CH];
    for (int s = 0; s < nt; ++s) {
        int ny = i0y + k0 + s;
        float wy = stf_ref_weight(f, cy - (float)ny);
        for (int t = 0; t < nt; ++t) {
            int nx = i0x + k0 + t;
            float wx = stf_ref_weight(f, cx - (float)nx);
            float w = wx * wy;
            if (n > 0 && w > 0.0f) {
                int found = 0;
                for (int i = 0; i < n && !found; ++i) found = six[list[i]] == nx && siy[list[i]] == ny;
                if (!found) return 0;
            }
            /* a sampled texel is the fetch at its lattice index, so fetching here is the same */
            fetch_texel(m, nx, ny, Tt);
            for (int c = 0; c < C; ++c) acc[c] = acc[c] + w * Tt[c];
        }
    }
    for (int c = 0; c < C; ++c) res[c] = acc[c];
    return 1;
}

/* Blue-noise uniforms of pixel (x, y) (REF_FLAG_BLUE in the header). */
static void blue_uniforms(const ref_view* v, int x, int y, uint64_t seed, float* ux, float* uy)
{
    const uint32_t n = (uint32_t)v->blue_size, N = n * n;
    const uint32_t S = (1u << 24) / N; /* 2^24 / n^2, n a power of two */
    const uint32_t fold = ((uint32_t)seed ^ (uint32_t)(seed >> 32)) & 0xffffffu;
    const uint32_t off = ((uint32_t)v->frame * 10368890u + fold) & 0xffffffu;
    const uint32_t k = ((uint32_t)y % n) * n + (uint32_t)x % n;
    const uint32_t a = ((uint32_t)v->blue[k] * S + S / 2 + off) & 0xffffffu;
    const uint32_t b = ((uint32_t)v->blue[N + k] * S + S / 2 + off) & 0xffffffu;
    *ux = (float)a * (1.0f / 16777216.0f);
    *uy = (float)b * (1.0f / 16777216.0f);
}

/* The footprint of a lane: the square footprints of the sharing modes, or the lane's row of the
 * view's sparse pattern for this frame. */
static int lane_footprint(const job_t* J, int lane, int* list)
{
    const ref_view* v = J->v;
    if (J->mode == REF_SPARSE9) {
        const signed char* row = v->fp_table + ((size_t)(v->frame % v->fp_patterns) * 32 + lane) * 9;
        for (int i = 0; i < 9; ++i) list[i] = row[i];
        return 9;
    }
    return stf_ref_footprint(J->mode, v->tile_w, v->tile_h, lane, list);
}

/* Lane j's filter weight (its PMF) at texel (nx, ny). */
static float pmf_at(int f, const float* cx, const float* cy, int j, int nx, int ny)
{
    return stf_ref_weight(f, cx[j] - (float)nx) * stf_ref_weight(f, cy[j] - (float)ny);
}

/* The alternative estimators of the pixel of lane c over its footprint samples list[0..n)
 * (see REF_EST_* in the header), each sum in list order. */
static void alt_estimate(int est, int clamp, int f, int C, int c, const float* cx, const float* cy, const int* ix,
                         const int* iy, const float* p, const float (*T)[REF_MAX_CH], const int* list, int n,
                         float* res)
{
    float acc[REF_MAX_CH] = {0};
    const float nf = (float)n;
    if (est == REF_EST_IS) {
        for (int i = 0; i < n; ++i) {
            int j = list[i];
            float r = pmf_at(f, cx, cy, c, ix[j], iy[j]) / p[j];
            for (int k = 0; k < C; ++k) acc[k] = acc[k] + r * T[j][k];
        }
        for (int k = 0; k < C; ++k) res[k] = acc[k] / nf;
    } else if (est == REF_EST_MIS) {
        for (int i = 0; i < n; ++i) {
            int j = list[i];
            float den = 0.0f;
            for (int q = 0; q < n; ++q) den = den + pmf_at(f, cx, cy, list[q], ix[j], iy[j]);
            float r = pmf_at(f, cx, cy, c, ix[j], iy[j]) / den;
            for (int k = 0; k < C; ++k) acc[k] = acc[k] + r * T[j][k];
        }
        for (int k = 0; k < C; ++k) res[k] = acc[k];
    } else if (est == REF_EST_PMIS) {
        const float m1 = nf - 1.0f;
        for (int i = 0; i < n; ++i) {
            int j = list[i];
            float pc = pmf_at(f, cx, cy, c, ix[j], iy[j]);
            float r;
            if (j == c) {
                /* canonical: m_c(x_c) f(x_c)/p_c(x_c) = m_c(x_c) T_c */
                float mc = 0.0f;
                for (int q = 0; q < n; ++q) {
                    if (list[q] == c) continue;
                    float pj = pmf_at(f, cx, cy, list[q], ix[j], iy[j]);
                    mc = mc + pc / (pc + m1 * pj);
                }
                r = mc / m1;
            } else {
                /* m_i(x_i) f(x_i)/p_i(x_i) = p_c(x_i) T_i / (p_c(x_i) + (n-1) p_i(x_i)) */
                r = pc / (pc + m1 * p[j]);
            }
            for (int k = 0; k < C; ++k) acc[k] = acc[k] + r * T[j][k];
        }
        for (int k = 0; k < C; ++k) res[k] = acc[k];
    } else { /* REF_EST_REG */
        float h[16], hbar = 0.0f;
        for (int i = 0; i < n; ++i) {
            int j = list[i];
            h[i] = pmf_at(f, cx, cy, c, ix[j], iy[j]) / p[j];
            hbar = hbar + h[i];
        }
        hbar = hbar / nf;
        float shh = 0.0f;
        for (int i = 0; i < n; ++i) {
            float d = h[i] - hbar;
            shh = shh + d * d;
        }
        for (int k = 0; k < C; ++k) {
            float sy = 0.0f, shy = 0.0f;
            for (int i = 0; i < n; ++i) {
                float y = h[i] * T[list[i]][k];
                sy = sy + y;
                shy = shy + (h[i] - hbar) * y;
            }
            float beta = shh > 0.0f ? shy / shh : 0.0f;
            res[k] = sy / nf - beta * (hbar - 1.0f);
        }
    }
    if (clamp) {
        for (int k = 0; k < C; ++k) {
            float lo = INFINITY, hi = -INFINITY;
            for (int i = 0; i < n; ++i) {
                int j = list[i];
                if (pmf_at(f, cx, cy, c, ix[j], iy[j]) > 0.0f) {
                    lo = fminf(lo, T[j][k]);
                    hi = fmaxf(hi, T[j][k]);
                }
            }
            res[k] = fminf(fmaxf(res[k], lo), hi);
        }
    }
}

static void render_tile(const job_t* J, int tx, int ty)
{
    const ref_material* m = J->m;
    const ref_view* v = J->v;
    const int tw = v->tile_w, th = v->tile_h, f = v->filter;
    const int C = material_channels(m);
    float cx[32], cy[32], p[32], T[32][REF_MAX_CH];
    int ix[32], iy[32], px[32], py[32];

    /* every lane samples its one texel (one-tap STF) before any sharing */
    for (int lane = 0; lane < 32; ++lane) {
        px[lane] = tx * tw + lane % tw;
        py[lane] = ty * th + lane / tw;
        stf_ref_texel_coords(v, m->width, m->height, px[lane], py[lane], &cx[lane], &cy[lane]);
        if (J->mode == REF_FULL) continue;
        float ux, uy, wx, wy;
        if (J->blue) blue_uniforms(v, px[lane], py[lane], J->seed, &ux, &uy);
        else stf_ref_uniforms(px[lane], py[lane], v->frame, v->view_id, J->seed, &ux, &uy);
        stf_ref_select_axis(f, cx[lane], ux, &ix[lane], &wx);
        stf_ref_select_axis(f, cy[lane], uy, &iy[lane], &wy);
        /* the PMF of the chosen texel is its 2D filter weight */
        p[lane] = stf_ref_weight(f, cx[lane] - (float)ix[lane]) * stf_ref_weight(f, cy[lane] - (float)iy[lane]);
        fetch_texel(m, ix[lane], iy[lane], T[lane]);
    }

    for (int lane = 0; lane < 32; ++lane) {
        int x = px[lane], y = py[lane];
        if (x >= v->width || y >= v->height) continue; /* off-screen lanes still shared above */
        float res[REF_MAX_CH] = {0};
        if (J->mode == REF_FULL) {
            /* deterministic filter: sum over the lattice taps of W(dx) W(dy) T, y outer */
            full_filter(m, f, C, cx[lane], cy[lane], NULL, NULL, NULL, 0, res);
        } else if (J->est != REF_EST_WIS) {
            int list[16];
            int n = lane_footprint(J, lane, list);
            alt_estimate(J->est, J->clamp, f, C, lane, cx, cy, ix, iy, p, (const float(*)[REF_MAX_CH])T, list, n, res);
        } else {
            /* weighted importance sampling over the footprint (Section 4.5):
             * w_j = p_c(x_j) / p_j(x_j), result = sum w_j T_j / sum w_j */
            int list[16];
            int n = lane_footprint(J, lane, list);
            float acc[REF_MAX_CH] = {0};
            float wsum = 0.0f;
            for (int i = 0; i < n; ++i) {
                int j = list[i];
                float pc = stf_ref_weight(f, cx[lane] - (float)ix[j]) * stf_ref_weight(f, cy[lane] - (float)iy[j]);
                float w = pc / p[j];
                for (int c = 0; c < C; ++c) acc[c] = acc[c] + w * T[j][c];
                wsum = wsum + w;
            }
            for (int c = 0; c < C; ++c) res[c] = acc[c] / wsum;
            /* exact filtering: every texel the pixel's own bilinear filter weighs is among the
             * footprint's samples -> the deterministic filter over those samples */
            if (J->exact && f == REF_BILINEAR)
                full_filter(m, f, C, cx[lane], cy[lane], ix, iy, list, n, res);
        }
        size_t pix = (size_t)y * v->width + x;
        if (J->out_ch) for (int c = 0; c < REF_MAX_CH; ++c) J->out_ch[pix * REF_MAX_CH + c] = res[c];
        if (J->out_idx)
            J->out_idx[pix] = J->mode == REF_FULL ? 0u
                            : ((uint32_t)(ix[lane] & 0xffff) | ((uint32_t)(iy[lane] & 0xffff) << 16));
        float u, w, rgba[4];
        uv_of_pixel(v, x, y, &u, &w);
        final_rgba(v, C, res, u, w, rgba);
        for (int k = 0; k < 4; ++k) J->out_rgba[pix * 4 + k] = rgba[k];
    }
}

static void* render_worker(void* arg)
{
    const job_t* J = (const job_t*)arg;
    const ref_view* v = J->v;
    int tiles_x = (v->width + v->tile_w - 1) / v->tile_w;
    int tiles_y = (v->height + v->tile_h - 1) / v->tile_h;
    for (int ty = J->tid; ty < tiles_y; ty += J->nthreads)
        for (int tx = 0; tx < tiles_x; ++tx) render_tile(J, tx, ty);
    return NULL;
}

static int check_args(const ref_material* m, const ref_view* v)
{
    if (!m || !v) return 1;
    if (m->width < 1 || m->height < 1 || m->width > 16384 || m->height > 16384) return 1;
    if (m->nn_lat16) {
        if (m->num_planes != 0 || m->nn_r < 1 || m->nn_gw < 1 || m->nn_gh < 1) return 1;
    } else if (m->num_planes < 1 || m->num_planes > REF_MAX_PLANES) {
        return 1;
    }
    int C = material_channels(m);
    if (C < 1 || C > REF_MAX_CH) return 1;
    if (m->scales && m->scale_tile < 1) return 1;
    if (v->width < 1 || v->height < 1) return 1;
    if (v->tile_w * v->tile_h != 32 || v->tile_w < 1) return 1;
    if (v->filter != REF_BILINEAR && v->filter != REF_BSPLINE3) return 1;
    if (v->shading) {
        if (v->ch_albedo >= 0 && v->ch_albedo + 2 >= C) return 1;
        if (v->ch_normal >= 0 && v->ch_normal + 1 >= C) return 1;
        if (v->ch_rough >= C || v->ch_ao >= C) return 1;
    }
    return 0;
}

static int run_jobs(job_t* proto, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job_t jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; ++i) {
        jobs[i] = *proto;
        jobs[i].tid = i;
        jobs[i].nthreads = nthreads;
    }
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, render_worker, &jobs[i]) != 0) return 3;
    render_worker(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

int stf_ref_render(const ref_material* m, const ref_view* v, int mode, uint64_t seed,
                   float* out_rgba, uint32_t* out_idx, float* out_ch, int nthreads)
{
    if (check_args(m, v) || !out_rgba) return 1;
    const int exact = (mode & REF_FLAG_EXACT) != 0;
    const int est = (mode >> REF_EST_SHIFT) & 7;
    const int clamp = (mode & REF_FLAG_CLAMP) != 0;
    const int blue = (mode & REF_FLAG_BLUE) != 0;
    mode &= 15;
    if (blue) {
        if (mode == REF_FULL || !v->blue || v->blue_size < 4 || v->blue_size > 256 ||
            (v->blue_size & (v->blue_size - 1)))
            return 1;
    }
    if (mode < REF_FULL || mode > REF_SPARSE9) return 1;
    if (mode == REF_SPARSE9) {
        if (!v->fp_table || v->fp_patterns < 1) return 1;
        for (long i = 0; i < (long)v->fp_patterns * 32 * 9; ++i)
            if (v->fp_table[i] < 0 || v->fp_table[i] > 31) return 1;
    }
    if (exact && mode < REF_QUAD2) return 1; /* exact filtering needs shared samples */
    if ((est != REF_EST_WIS || clamp) && mode < REF_QUAD2) return 1;
    if (est > REF_EST_REG || (clamp && est == REF_EST_WIS) || (exact && est != REF_EST_WIS)) return 1;
    if (mode == REF_QUAD2 && (v->tile_w % 2 || v->tile_h % 2)) return 1;
    job_t J;
    memset(&J, 0, sizeof J);
    J.m = m; J.v = v; J.mode = mode; J.exact = exact; J.est = est; J.clamp = clamp; J.blue = blue; J.seed = seed;
    J.out_rgba = out_rgba; J.out_idx = out_idx; J.out_ch = out_ch;
    return run_jobs(&J, nthreads);
}

/* ----------------------------------------------------- FP64 exact filter */

static void* exact_worker(void* arg)
{
    const job_t* J = (const job_t*)arg;
    const ref_material* m = J->m;
    const ref_view* v = J->v;
    const int f = v->filter, C = material_channels(m);
    const int k0 = tap_first(f), nt = tap_count(f);
    for (int y = J->tid; y < v->height; y += J->nthreads) {
        for (int x = 0; x < v->width; ++x) {
            const float* H = v->H;
            double px = x + 0.5, py = y + 0.5;
            double hx = (double)H[0] * px + (double)H[1] * py + (double)H[2];
            double hy = (double)H[3] * px + (double)H[4] * py + (double)H[5];
            double hw = (double)H[6] * px + (double)H[7] * py + (double)H[8];
            double u = hx / hw, w = hy / hw;
            double cx = u * m->width - 0.5, cy = w * m->height - 0.5;
            if (!(cx >= C_LO)) cx = C_LO;
            if (cx > C_HI) cx = C_HI;
            if (!(cy >= C_LO)) cy = C_LO;
            if (cy > C_HI) cy = C_HI;
            int i0x = (int)floor(cx), i0y = (int)floor(cy);
            double res[REF_MAX_CH] = {0};
            float Tt[REF_MAX_CH];
            for (int s = 0; s < nt; ++s) {
                int ny = i0y + k0 + s;
                double wy = stf_ref_weight_f64(f, cy - ny);
                for (int t = 0; t < nt; ++t) {
                    int nx = i0x + k0 + t;
                    double wx = stf_ref_weight_f64(f, cx - nx);
                    fetch_texel(m, nx, ny, Tt);
                    for (int c = 0; c < C; ++c) res[c] += wx * wy * (double)Tt[c];
                }
            }
            size_t pix = (size_t)y * v->width + x;
            if (J->out_ch64) for (int c = 0; c < REF_MAX_CH; ++c) J->out_ch64[pix * REF_MAX_CH + c] = res[c];
            double rgba[4];
            if (v->shading) stf_ref_shade_f64(v, res, u, w, rgba);
            else for (int k = 0; k < 4; ++k) rgba[k] = k < C ? res[k] : (k == 3 ? 1.0 : 0.0);
            for (int k = 0; k < 4; ++k) J->out_rgba64[pix * 4 + k] = rgba[k];
        }
    }
    return NULL;
}

int stf_ref_render_exact_f64(const ref_material* m, const ref_view* v, double* out_rgba,
                             double* out_ch, int nthreads)
{
    if (check_args(m, v) || !out_rgba) return 1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    job_t jobs[256];
    pthread_t th[256];
    for (int i = 0; i < nthreads; ++i) {
        memset(&jobs[i], 0, sizeof(job_t));
        jobs[i].m = m; jobs[i].v = v;
        jobs[i].out_rgba64 = out_rgba; jobs[i].out_ch64 = out_ch;
        jobs[i].tid = i; jobs[i].nthreads = nthreads;
    }
    for (int i = 1; i < nthreads; ++i)
        if (pthread_create(&th[i], NULL, exact_worker, &jobs[i]) != 0) return 3;
    exact_worker(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}
