/*
 * CPU oracle for the neural texel decoder (latent grid + MLP) that stands in for the costly
 * per-texel decode STF amortises (neural texture compression, Sections 1 and 5.6).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark CPU leg); shares no code with the GPU.
 *
 * The decoder of texel (ix, iy) of a W x H material with an R-times coarser latent grid
 * (R = W / GW, 16 channels per latent cell):
 *   latent position  l = (i + 0.5) / R - 0.5 per axis; bilinear over the grid, clamp-to-edge;
 *   position phase   phi = ((i mod R) + 0.5) / R per axis; features sin/cos(2 pi phi),
 *                    sin/cos(4 pi phi) for x then y;
 *   input            x = (16 interpolated latents, 4 x-features, 4 y-features) (24 values);
 *   MLP              h1 = relu(W1 x + b1) (64), h2 = relu(W2 h1 + b2) (64), y = W3 h2 + b3 (8).
 * Parameter vector (FP32/FP64, this order): W1[64][24], b1[64], W2[64][64], b2[64], W3[8][64],
 * b3[8] (6280 values). The loss of a batch is mean over texels and channels of (y - t)^2.
 *
 * Two evaluation paths:
 *   FP64           forward and backward in double (gradient checks, ground truth);
 *   FP32 emulation the GPU's inference precision: latents and weights stored in FP16, the 16
 *                  interpolated latents computed in FP16 arithmetic, the 8 position features and
 *                  both hidden layers rounded to FP16, products accumulated in FP32, biases and
 *                  output in FP32.
 *   E4M3 emulation the FP8 inference variant: layer 1 as above with its weights and bias scaled
 *                  by a power of two s1; both hidden layers, W2 and W3 rounded to OCP E4M3 after
 *                  power-of-two scalings (s2, s3) chosen from a first-order bound of the
 *                  activations so that nothing saturates; each bias of layers 2 and 3 split into
 *                  three E4M3 parts; products accumulated in FP32; the output scaled back.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define NN_IN 24
#define NN_H 64
#define NN_OUT 8
#define NN_LAT 16
#define NN_PARAMS (NN_H * NN_IN + NN_H + NN_H * NN_H + NN_H + NN_OUT * NN_H + NN_OUT)

static const double PI_D = 3.14159265358979323846;

/* binary16 -> float (exact) and float -> binary16 round-to-nearest-even, from the IEEE 754
 * definition (1 sign, 5 exponent bits biased by 15, 10 fraction bits). */
static float h2f(uint16_t h)
{
    int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
    float r;
    if (e == 0) r = ldexpf((float)f, -24);
    else if (e == 31) r = f ? NAN : INFINITY;
    else r = ldexpf((float)(1024 + f), e - 25);
    return s ? -r : r;
}

static uint16_t d2h(double x)
{
    uint16_t sign = (uint16_t)(signbit(x) ? 0x8000u : 0u);
    double a = fabs(x);
    if (isnan(x)) return (uint16_t)(sign | 0x7e00u);
    if (a >= 65520.0) return (uint16_t)(sign | 0x7c00u); /* rounds to infinity */
    if (a < ldexp(1.0, -14)) {
        /* subnormal: multiple of 2^-24, round to nearest even */
        double q = (double)a * 16777216.0;
        double fl = floor(q);
        double r = q - fl;
        uint32_t m = (uint32_t)fl;
        if (r > 0.5 || (r == 0.5 && (m & 1u))) m++;
        return (uint16_t)(sign | m); /* m == 1024 becomes the smallest normal, as it should */
    }
    int e;
    double fr = frexp(a, &e);         /* a = fr * 2^e, fr in [0.5, 1) */
    double q = fr * 2048.0;           /* 11 significant bits */
    double fl = floor(q);
    double r = q - fl;
    uint32_t m = (uint32_t)fl;
    if (r > 0.5 || (r == 0.5 && (m & 1u))) m++;
    if (m == 2048) { m = 1024; e++; }
    int E = e - 1 + 15;
    if (E >= 31) return (uint16_t)(sign | 0x7c00u);
    return (uint16_t)(sign | (uint16_t)(E << 10) | (uint16_t)(m - 1024));
}

static uint16_t f2h(float x) { return d2h((double)x); }
static float round_h(float x) { return h2f(f2h(x)); }

/* binary16 arithmetic (IEEE 754: the exact result rounded once to binary16, nearest even). The
 * product of two binary16 values is exact in double; adding a third is exact in double unless
 * the operands lie more than 31 binades apart, and then the far smaller one cannot move the
 * result across a binary16 rounding boundary, so one rounding of the double result is exact. */
static float mul_h(float a, float b) { return h2f(d2h((double)a * (double)b)); }
static float fma_h(float a, float b, float c) { return h2f(d2h((double)a * (double)b + (double)c)); }

float stf_ref_f16_round(float x) { return round_h(x); }
uint16_t stf_ref_f32_to_f16(float x) { return f2h(x); }

/* Bilinear position of texel i on the latent axis: lower cell and its fraction (exact dyadic for
 * power-of-two R). */
static void latent_axis(int i, int R, int G, int* c0, int* c1, double* f)
{
    double l = (i + 0.5) / R - 0.5;
    double fl = floor(l);
    *f = l - fl;
    int a = (int)fl, b = a + 1;
    if (a < 0) a = 0;
    if (a > G - 1) a = G - 1;
    if (b < 0) b = 0;
    if (b > G - 1) b = G - 1;
    *c0 = a;
    *c1 = b;
}

static void phase_features(int i, int R, double* out4)
{
    double phi = ((i % R) + 0.5) / R;
    out4[0] = sin(2.0 * PI_D * phi);
    out4[1] = cos(2.0 * PI_D * phi);
    out4[2] = sin(4.0 * PI_D * phi);
    out4[3] = cos(4.0 * PI_D * phi);
}

/* The 24 inputs in FP64 from an FP64 latent grid [GH][GW][16]. */
static void features_f64(const double* lat, int GW, int GH, int R, int ix, int iy, double* x)
{
    int x0, x1, y0, y1;
    double fx, fy;
    latent_axis(ix, R, GW, &x0, &x1, &fx);
    latent_axis(iy, R, GH, &y0, &y1, &fy);
    const double w[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
    const double* c[4] = {lat + ((size_t)y0 * GW + x0) * NN_LAT, lat + ((size_t)y0 * GW + x1) * NN_LAT,
                          lat + ((size_t)y1 * GW + x0) * NN_LAT, lat + ((size_t)y1 * GW + x1) * NN_LAT};
    for (int k = 0; k < NN_LAT; ++k) x[k] = w[0] * c[0][k] + w[1] * c[1][k] + w[2] * c[2][k] + w[3] * c[3][k];
    phase_features(ix, R, x + 16);
    phase_features(iy, R, x + 20);
}

/* Exported: FP64 inputs of texel (ix, iy) (test helper). Returns 0. */
int stf_ref_neural_features(const double* lat, int GW, int GH, int R, int ix_iy, double* x)
{
    features_f64(lat, GW, GH, R, ix_iy & 0xffff, ix_iy >> 16, x);
    return 0;
}

/* FP64 MLP forward of one input; keeps pre-activations for the backward pass. */
static void mlp_f64(const double* P, const double* x, double* a1, double* a2, double* y)
{
    const double* W1 = P;
    const double* b1 = W1 + NN_H * NN_IN;
    const double* W2 = b1 + NN_H;
    const double* b2 = W2 + NN_H * NN_H;
    const double* W3 = b2 + NN_H;
    const double* b3 = W3 + NN_OUT * NN_H;
    double h1[NN_H], h2[NN_H];
    for (int o = 0; o < NN_H; ++o) {
        double s = b1[o];
        for (int i = 0; i < NN_IN; ++i) s += W1[o * NN_IN + i] * x[i];
        a1[o] = s;
        h1[o] = s > 0 ? s : 0;
    }
    for (int o = 0; o < NN_H; ++o) {
        double s = b2[o];
        for (int i = 0; i < NN_H; ++i) s += W2[o * NN_H + i] * h1[i];
        a2[o] = s;
        h2[o] = s > 0 ? s : 0;
    }
    for (int o = 0; o < NN_OUT; ++o) {
        double s = b3[o];
        for (int i = 0; i < NN_H; ++i) s += W3[o * NN_H + i] * h2[i];
        y[o] = s;
    }
}

/* Exported: FP64 forward of n inputs x[n][24] with parameters P -> y[n][8]. */
int stf_ref_mlp_forward(const double* P, const double* x, int n, double* y, double* unused)
{
    (void)unused;
    double a1[NN_H], a2[NN_H];
    for (int b = 0; b < n; ++b) mlp_f64(P, x + (size_t)b * NN_IN, a1, a2, y + (size_t)b * NN_OUT);
    return 0;
}

/* FP64 loss and gradients over a batch of texels idx[n] (packed ix | iy << 16) of a target
 * material tgt[H][W][8]: loss = mean over texels and channels of (y - t)^2. Writes dP[6280] and
 * dlat[GH][GW][16] (both overwritten). Returns the loss. */
double stf_ref_neural_loss_grad(const double* lat, int GW, int GH, int R, const double* P, int nparams,
                                const float* tgt, int W, const int* idx, int n, double* dP, double* dlat,
                                double* unused)
{
    (void)nparams;
    (void)unused;
    memset(dP, 0, sizeof(double) * NN_PARAMS);
    memset(dlat, 0, sizeof(double) * (size_t)GW * GH * NN_LAT);
    const double* W1 = P;
    const double* W2 = W1 + NN_H * NN_IN + NN_H;
    const double* W3 = W2 + NN_H * NN_H + NN_H;
    double* dW1 = dP;
    double* db1 = dW1 + NN_H * NN_IN;
    double* dW2 = db1 + NN_H;
    double* db2 = dW2 + NN_H * NN_H;
    double* dW3 = db2 + NN_H;
    double* db3 = dW3 + NN_OUT * NN_H;
    double loss = 0.0;
    const double scale = 1.0 / ((double)n * NN_OUT);
    for (int b = 0; b < n; ++b) {
        int ix = idx[b] & 0xffff, iy = idx[b] >> 16;
        double x[NN_IN], a1[NN_H], a2[NN_H], y[NN_OUT], h1[NN_H], h2[NN_H];
        features_f64(lat, GW, GH, R, ix, iy, x);
        mlp_f64(P, x, a1, a2, y);
        for (int o = 0; o < NN_H; ++o) { h1[o] = a1[o] > 0 ? a1[o] : 0; h2[o] = a2[o] > 0 ? a2[o] : 0; }
        double g3[NN_OUT], g2[NN_H], g1[NN_H], gx[NN_IN];
        const float* t = tgt + ((size_t)iy * W + ix) * NN_OUT;
        for (int o = 0; o < NN_OUT; ++o) {
            double d = y[o] - (double)t[o];
            loss += d * d * scale;
            g3[o] = 2.0 * d * scale;
        }
        for (int i = 0; i < NN_H; ++i) {
            double s = 0;
            for (int o = 0; o < NN_OUT; ++o) s += W3[o * NN_H + i] * g3[o];
            g2[i] = a2[i] > 0 ? s : 0;
        }
        for (int i = 0; i < NN_H; ++i) {
            double s = 0;
            for (int o = 0; o < NN_H; ++o) s += W2[o * NN_H + i] * g2[o];
            g1[i] = a1[i] > 0 ? s : 0;
        }
        for (int i = 0; i < NN_IN; ++i) {
            double s = 0;
            for (int o = 0; o < NN_H; ++o) s += W1[o * NN_IN + i] * g1[o];
            gx[i] = s;
        }
        for (int o = 0; o < NN_OUT; ++o) {
            db3[o] += g3[o];
            for (int i = 0; i < NN_H; ++i) dW3[o * NN_H + i] += g3[o] * h2[i];
        }
        for (int o = 0; o < NN_H; ++o) {
            db2[o] += g2[o];
            for (int i = 0; i < NN_H; ++i) dW2[o * NN_H + i] += g2[o] * h1[i];
            db1[o] += g1[o];
            for (int i = 0; i < NN_IN; ++i) dW1[o * NN_IN + i] += g1[o] * x[i];
        }
        /* latent gradient: the bilinear weights route gx[0..15] to the four corners */
        int x0, x1, y0, y1;
        double fx, fy;
        latent_axis(ix, R, GW, &x0, &x1, &fx);
        latent_axis(iy, R, GH, &y0, &y1, &fy);
        const double w[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
        const int cx[4] = {x0, x1, x0, x1}, cy[4] = {y0, y0, y1, y1};
        for (int k = 0; k < 4; ++k)
            for (int c = 0; c < NN_LAT; ++c) dlat[((size_t)cy[k] * GW + cx[k]) * NN_LAT + c] += w[k] * gx[c];
    }
    return loss;
}

/* FP32 emulation of the GPU inference precision. lat16 [GH][GW][16] binary16 codes; w16 the
 * FP16 codes of W1, W2, W3 (in the parameter order, biases skipped); b32 the FP32 biases
 * b1, b2, b3. Decodes n texels idx[n] -> out[n][8]. */
int stf_ref_neural_decode(const uint16_t* lat16, int GW, int GH, int R, const uint16_t* w16, int nw,
                          const float* b32, const int* idx, int n, float* out)
{
    (void)nw;
    const uint16_t* W1 = w16;
    const uint16_t* W2 = W1 + NN_H * NN_IN;
    const uint16_t* W3 = W2 + NN_H * NN_H;
    const float* b1 = b32;
    const float* b2 = b1 + NN_H;
    const float* b3 = b2 + NN_H;
    for (int b = 0; b < n; ++b) {
        int ix = idx[b] & 0xffff, iy = idx[b] >> 16;
        int x0, x1, y0, y1;
        double fxd, fyd;
        latent_axis(ix, R, GW, &x0, &x1, &fxd);
        latent_axis(iy, R, GH, &y0, &y1, &fyd);
        const float fx = (float)fxd, fy = (float)fyd;
        /* corner weights in FP32, then rounded to FP16; the interpolation in FP16 arithmetic, one
         * rounding per multiply and per fused multiply-add, in this order */
        const float w00 = round_h((1.0f - fx) * (1.0f - fy)), w10 = round_h(fx * (1.0f - fy));
        const float w01 = round_h((1.0f - fx) * fy), w11 = round_h(fx * fy);
        const uint16_t* c00 = lat16 + ((size_t)y0 * GW + x0) * NN_LAT;
        const uint16_t* c10 = lat16 + ((size_t)y0 * GW + x1) * NN_LAT;
        const uint16_t* c01 = lat16 + ((size_t)y1 * GW + x0) * NN_LAT;
        const uint16_t* c11 = lat16 + ((size_t)y1 * GW + x1) * NN_LAT;
        float x[NN_IN];
        for (int k = 0; k < NN_LAT; ++k) {
            float s = mul_h(w00, h2f(c00[k]));
            s = fma_h(w10, h2f(c10[k]), s);
            s = fma_h(w01, h2f(c01[k]), s);
            s = fma_h(w11, h2f(c11[k]), s);
            x[k] = s;
        }
        double ph[8];
        phase_features(ix, R, ph);
        phase_features(iy, R, ph + 4);
        for (int k = 0; k < 8; ++k) x[16 + k] = round_h((float)ph[k]);
        float h1[NN_H], h2[NN_H];
        for (int o = 0; o < NN_H; ++o) {
            float s = 0.0f;
            for (int i = 0; i < NN_IN; ++i) s = s + h2f(W1[o * NN_IN + i]) * x[i];
            s = s + b1[o];
            h1[o] = round_h(s > 0.0f ? s : 0.0f);
        }
        for (int o = 0; o < NN_H; ++o) {
            float s = 0.0f;
            for (int i = 0; i < NN_H; ++i) s = s + h2f(W2[o * NN_H + i]) * h1[i];
            s = s + b2[o];
            h2[o] = round_h(s > 0.0f ? s : 0.0f);
        }
        for (int o = 0; o < NN_OUT; ++o) {
            float s = 0.0f;
            for (int i = 0; i < NN_H; ++i) s = s + h2f(W3[o * NN_H + i]) * h2[i];
            out[(size_t)b * NN_OUT + o] = s + b3[o];
        }
    }
    return 0;
}

/* FP64 decode of n texels from an FP64 latent grid and parameters (no storage rounding). */
int stf_ref_neural_decode_f64(const double* lat, int GW, int GH, int R, const double* P, const int* idx, int n,
                              double* out)
{
    double x[NN_IN], a1[NN_H], a2[NN_H];
    for (int b = 0; b < n; ++b) {
        features_f64(lat, GW, GH, R, idx[b] & 0xffff, idx[b] >> 16, x);
        mlp_f64(P, x, a1, a2, out + (size_t)b * NN_OUT);
    }
    return 0;
}

/* ------------------------------------------------------------------------------ E4M3 variant */

/* OCP 8-bit E4M3 ("FN"): 1 sign, 4 exponent bits biased by 7, 3 fraction bits, no infinities,
 * largest finite 448 (code 0x7e), 0x7f / 0xff NaN; exponent field 0 holds the subnormals
 * m * 2^-9. */
static double e4m3_value(int code)
{
    int s = (code >> 7) & 1, e = (code >> 3) & 15, f = code & 7;
    double r;
    if (e == 15 && f == 7) return NAN;
    if (e == 0) r = ldexp((double)f, -9);
    else r = ldexp((double)(8 + f), e - 10);
    return s ? -r : r;
}

/* Round to nearest E4M3, ties to the even code, saturating to +-448 (the rounding of the GPU's
 * satfinite conversion); NaN gives 0x7f. Plain search over the 127 finite magnitudes. */
static uint8_t e4m3_encode(double x)
{
    if (isnan(x)) return 0x7f;
    const int neg = signbit(x) ? 1 : 0;
    const double a = fabs(x);
    int best = 0;
    double berr = INFINITY;
    for (int c = 0; c <= 0x7e; ++c) {
        const double err = fabs(e4m3_value(c) - a);
        if (err < berr || (err == berr && (c & 1) == 0)) { best = c; berr = err; }
    }
    return (uint8_t)(best | (neg << 7));
}

static double e4m3_round(double x) { return e4m3_value(e4m3_encode(x)); }

uint8_t stf_ref_f64_to_e4m3(double x) { return e4m3_encode(x); }
double stf_ref_e4m3_to_f64(uint8_t c) { return e4m3_value(c); }

/* floor(log2(v)) for v > 0, exactly (frexp: v = f 2^e, f in [0.5, 1)). */
static int floor_log2(double v)
{
    int e;
    (void)frexp(v, &e);
    return e - 1;
}

/* The power-of-two exponents of the E4M3 variant (e[0] = log2 s1, e[1] = log2 s2, e[2] = log2 s3,
 * e[3] = -(e[0] + e[1] + e[2]), the output scale), from the FP16 latent grid and the FP32
 * parameters; every sum in FP64, terms in index order. With m = 1.0625 (one E4M3 rounding; it
 * also covers the FP16 roundings of layer 1):
 *   xmax_k   max over the grid of |latent k| for k < 16, 1 for the 8 position features;
 *   B1_j     m (sum_k |W1_jk| xmax_k) + |b1_j|              bounds |h1_j|;
 *   B2_i     m^2 (sum_j |W2_ij| B1_j) + |b2_i|              bounds |h2_i|;
 *   s1       2^floor(log2(448 / max_j B1_j)), at most 2^8;
 *   s2       2^floor(log2(min(448 / (s1 max B2), 448 / max |W2|))), so that s1 s2 h2 and s2 W2
 *            stay in range (the biases of layer 2 are covered by B2);
 *   s3       2^floor(log2(min(448 / max |W3|, 448 / (s1 s2 max |b3|)))).
 * Returns 0. */
int stf_ref_neural_e4m3_scales(const uint16_t* lat16, int GW, int GH, const float* P32, int* e)
{
    const float* W1 = P32;
    const float* b1 = W1 + NN_H * NN_IN;
    const float* W2 = b1 + NN_H;
    const float* b2 = W2 + NN_H * NN_H;
    const float* W3 = b2 + NN_H;
    const float* b3 = W3 + NN_OUT * NN_H;
    const double m = 1.0625;
    double xmax[NN_IN];
    for (int k = 0; k < NN_IN; ++k) xmax[k] = k < NN_LAT ? 0.0 : 1.0;
    for (long long c = 0; c < (long long)GW * GH; ++c)
        for (int k = 0; k < NN_LAT; ++k) {
            const double v = fabs((double)h2f(lat16[c * NN_LAT + k]));
            if (v > xmax[k]) xmax[k] = v;
        }
    double B1[NN_H], maxB1 = 0.0, maxB2 = 0.0, maxW2 = 0.0, maxW3 = 0.0, maxb3 = 0.0;
    for (int j = 0; j < NN_H; ++j) {
        double t = 0.0;
        for (int k = 0; k < NN_IN; ++k) t += fabs((double)W1[j * NN_IN + k]) * xmax[k];
        B1[j] = m * t + fabs((double)b1[j]);
        if (B1[j] > maxB1) maxB1 = B1[j];
    }
    for (int i = 0; i < NN_H; ++i) {
        double t = 0.0;
        for (int j = 0; j < NN_H; ++j) {
            t += fabs((double)W2[i * NN_H + j]) * B1[j];
            if (fabs((double)W2[i * NN_H + j]) > maxW2) maxW2 = fabs((double)W2[i * NN_H + j]);
        }
        const double b2i = m * m * t + fabs((double)b2[i]);
        if (b2i > maxB2) maxB2 = b2i;
    }
    for (int k = 0; k < NN_OUT * NN_H; ++k)
        if (fabs((double)W3[k]) > maxW3) maxW3 = fabs((double)W3[k]);
    for (int o = 0; o < NN_OUT; ++o)
        if (fabs((double)b3[o]) > maxb3) maxb3 = fabs((double)b3[o]);
    int e1 = maxB1 > 0.0 ? floor_log2(448.0 / maxB1) : 8;
    if (e1 > 8) e1 = 8;
    double lim2 = maxW2 > 0.0 ? 448.0 / maxW2 : INFINITY;
    if (maxB2 > 0.0 && 448.0 / (ldexp(1.0, e1) * maxB2) < lim2) lim2 = 448.0 / (ldexp(1.0, e1) * maxB2);
    int e2 = isinf(lim2) ? 0 : floor_log2(lim2);
    double lim3 = maxW3 > 0.0 ? 448.0 / maxW3 : INFINITY;
    if (maxb3 > 0.0 && 448.0 / (ldexp(1.0, e1 + e2) * maxb3) < lim3) lim3 = 448.0 / (ldexp(1.0, e1 + e2) * maxb3);
    int e3 = isinf(lim3) ? 0 : floor_log2(lim3);
    e[0] = e1;
    e[1] = e2;
    e[2] = e3;
    e[3] = -(e1 + e2 + e3);
    return 0;
}

/* Three E4M3 parts of v: p0 = E4M3(v), p1 = E4M3(v - p0), p2 = E4M3(v - p0 - p1) (each
 * difference exact in double). */
static void e4m3_parts(double v, double* p)
{
    p[0] = e4m3_round(v);
    p[1] = e4m3_round(v - p[0]);
    p[2] = e4m3_round(v - p[0] - p[1]);
}

/* FP32 emulation of the E4M3 variant. lat16 [GH][GW][16] binary16 codes, P32 the FP32
 * parameters (the variant's weights and scales are derived from them as the GPU does); decodes
 * n texels idx[n] -> out[n][8]. e (optional) receives the four exponents. */
int stf_ref_neural_decode_e4m3(const uint16_t* lat16, int GW, int GH, int R, const float* P32, const int* idx,
                               int n, float* out, int* e_out)
{
    int e[4];
    stf_ref_neural_e4m3_scales(lat16, GW, GH, P32, e);
    if (e_out) memcpy(e_out, e, sizeof e);
    const double s1 = ldexp(1.0, e[0]), s2 = ldexp(1.0, e[1]), s3 = ldexp(1.0, e[2]);
    const float os = (float)ldexp(1.0, e[3]);
    const float* W1 = P32;
    const float* b1 = W1 + NN_H * NN_IN;
    const float* W2 = b1 + NN_H;
    const float* b2 = W2 + NN_H * NN_H;
    const float* W3 = b2 + NN_H;
    const float* b3 = W3 + NN_OUT * NN_H;
    float w1[NN_H * NN_IN], w2[NN_H * NN_H], w3[NN_OUT * NN_H], c1[NN_H], c2[NN_H][3], c3[NN_OUT][3];
    /* layer 1: binary16 of s1 W1, the FP32 bias s1 b1 */
    for (int k = 0; k < NN_H * NN_IN; ++k) w1[k] = round_h((float)(s1 * (double)W1[k]));
    for (int j = 0; j < NN_H; ++j) c1[j] = (float)(s1 * (double)b1[j]);
    /* layers 2, 3: E4M3 of s2 W2 and s3 W3; bias parts of s2 s1 b2 and s3 s2 s1 b3 */
    for (int k = 0; k < NN_H * NN_H; ++k) w2[k] = (float)e4m3_round(s2 * (double)W2[k]);
    for (int k = 0; k < NN_OUT * NN_H; ++k) w3[k] = (float)e4m3_round(s3 * (double)W3[k]);
    for (int i = 0; i < NN_H; ++i) {
        double p[3];
        e4m3_parts(s2 * s1 * (double)b2[i], p);
        for (int q = 0; q < 3; ++q) c2[i][q] = (float)p[q];
    }
    for (int o = 0; o < NN_OUT; ++o) {
        double p[3];
        e4m3_parts(s3 * s2 * s1 * (double)b3[o], p);
        for (int q = 0; q < 3; ++q) c3[o][q] = (float)p[q];
    }
    for (int b = 0; b < n; ++b) {
        const int ix = idx[b] & 0xffff, iy = idx[b] >> 16;
        int x0, x1, y0, y1;
        double fxd, fyd;
        latent_axis(ix, R, GW, &x0, &x1, &fxd);
        latent_axis(iy, R, GH, &y0, &y1, &fyd);
        const float fx = (float)fxd, fy = (float)fyd;
        const float w00 = round_h((1.0f - fx) * (1.0f - fy)), w10 = round_h(fx * (1.0f - fy));
        const float w01 = round_h((1.0f - fx) * fy), w11 = round_h(fx * fy);
        const uint16_t* c00 = lat16 + ((size_t)y0 * GW + x0) * NN_LAT;
        const uint16_t* c10 = lat16 + ((size_t)y0 * GW + x1) * NN_LAT;
        const uint16_t* c01 = lat16 + ((size_t)y1 * GW + x0) * NN_LAT;
        const uint16_t* c11 = lat16 + ((size_t)y1 * GW + x1) * NN_LAT;
        float x[NN_IN];
        for (int k = 0; k < NN_LAT; ++k) {
            float t = mul_h(w00, h2f(c00[k]));
            t = fma_h(w10, h2f(c10[k]), t);
            t = fma_h(w01, h2f(c01[k]), t);
            t = fma_h(w11, h2f(c11[k]), t);
            x[k] = t;
        }
        double ph[8];
        phase_features(ix, R, ph);
        phase_features(iy, R, ph + 4);
        for (int k = 0; k < 8; ++k) x[16 + k] = round_h((float)ph[k]);
        float h1[NN_H], h2[NN_H];
        for (int j = 0; j < NN_H; ++j) {
            float t = 0.0f;
            for (int k = 0; k < NN_IN; ++k) t = t + w1[j * NN_IN + k] * x[k];
            t = t + c1[j];
            h1[j] = (float)e4m3_round(t > 0.0f ? t : 0.0f);
        }
        for (int i = 0; i < NN_H; ++i) {
            float t = 0.0f;
            for (int j = 0; j < NN_H; ++j) t = t + w2[i * NN_H + j] * h1[j];
            t = t + c2[i][0] + c2[i][1] + c2[i][2];
            h2[i] = (float)e4m3_round(t > 0.0f ? t : 0.0f);
        }
        for (int o = 0; o < NN_OUT; ++o) {
            float t = 0.0f;
            for (int i = 0; i < NN_H; ++i) t = t + w3[o * NN_H + i] * h2[i];
            t = t + c3[o][0] + c3[o][1] + c3[o][2];
            out[(size_t)b * NN_OUT + o] = t * os;
        }
    }
    return 0;
}
