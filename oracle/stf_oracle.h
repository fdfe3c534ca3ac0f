/*
 * CPU oracle for magnified stochastic texture filtering (STF) with sample reuse,
 * "Improved Stochastic Texture Filtering Through Sample Reuse" (Wronski, Pharr,
 * Akenine-Moller 2025).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the GPU library includes, links or calls
 * this code; only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg use it. It shares no source with the CUDA path: every definition here is
 * written out again from the paper (and, where the paper is silent, from a stated
 * reading: the cubic B-spline kernel, the pcg4d hash, clamp-to-edge addressing, the
 * footprint placement and the shading model, each described where it is defined).
 *
 * Build: plain C99, -O2 -ffp-contract=off, so that every float expression is
 * evaluated as written (one IEEE rounding per operation, left to right).
 */
#ifndef STF_ORACLE_H
#define STF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Filters (Section 2.1; bilinear per Section S6, cubic B-spline per Section 5.4). */
enum { REF_BILINEAR = 0, REF_BSPLINE3 = 1 };

/* Sharing modes (Sections 4.3.1, 4.5; Table 1). FULL is the deterministic filter. */
enum { REF_FULL = 0, REF_ONE_TAP = 1, REF_QUAD2 = 2, REF_WAVE2 = 3, REF_WAVE3 = 4, REF_WAVE4 = 5,
       REF_SPARSE9 = 6 /* the view's footprint table, pattern frame % patterns (Section
                        * "Sharing Footprints Within Waves") */ };

/* Exact filtering (Section "Exact Filtering"), OR'd into a sharing mode: with the bilinear filter,
 * a pixel whose footprint samples include every texel of positive weight in its own filter
 * returns the deterministic filter over those texels instead of the estimate. */
#define REF_FLAG_EXACT 16

/* Blue-noise uniforms (Section "Blue Noise Mask Improvements"), OR'd into a mode: the pixel's
 * uniforms are its ranks r in the view's two masks at (x mod n, y mod n), u = (r + 1/2) / n^2 +
 * frame * (sqrt(5) - 1) / 2 + (seed's folded low 24 bits) / 2^24 modulo 1, in 24-bit fixed point
 * (the golden-ratio step rounded to 10368890 / 2^24). */
#define REF_FLAG_BLUE 32

/* The estimator of a sharing mode, (mode >> REF_EST_SHIFT) & 7 (Section 4.1 and Section 4.2),
 * over the footprint's samples x_i drawn from the PMFs p_i (lane i's filter weights), with
 * f(x) = w_c(x) T(x) for the pixel's own filter w_c:
 *   WIS   sum_i (w_c(x_i)/p_i(x_i)) T_i / sum_i w_c(x_i)/p_i(x_i)   (the paper's estimator; default)
 *   IS    (1/n) sum_i f(x_i)/p_i(x_i)                                 (Eq. eq_basic_mc)
 *   MIS   sum_i f(x_i) / sum_k p_k(x_i)                               (balance heuristic)
 *   PMIS  pairwise MIS with the pixel's own sample as the canonical technique (Bitterli 2022):
 *         m_c(x) = 1/(n-1) sum_{j!=c} p_c(x)/(p_c(x) + (n-1) p_j(x)),
 *         m_i(x) = p_i(x)/(p_c(x) + (n-1) p_i(x)) (i != c), F = sum_i m_i(x_i) f(x_i)/p_i(x_i)
 *   REG   regression (control variate h = w_c/p with mean 1; Owen 2013, Eq. 9.11):
 *         y_i = f(x_i)/p_i(x_i), h_i = w_c(x_i)/p_i(x_i), beta = sum (h_i - hbar) y_i / sum (h_i - hbar)^2
 *         (0 if the denominator is 0), F = ybar - beta (hbar - 1)      (Eq. eq_mc_regression)
 * REF_FLAG_CLAMP clamps each channel of a non-WIS estimate to the range of the texels with
 * w_c > 0 among the samples (Section 4.1). */
#define REF_EST_SHIFT 8
enum { REF_EST_WIS = 0, REF_EST_IS = 1, REF_EST_MIS = 2, REF_EST_PMIS = 3, REF_EST_REG = 4 };
#define REF_FLAG_CLAMP 2048

/* Stored texel formats. */
enum { REF_FP32 = 0, REF_FP16 = 1, REF_BF16 = 2, REF_E4M3 = 3, REF_UNORM8 = 4 };

#define REF_MAX_CH 8
#define REF_MAX_PLANES 4

typedef struct {
    int width, height;             /* texels */
    int num_planes;
    int plane_fmt[REF_MAX_PLANES];
    int plane_ch[REF_MAX_PLANES];  /* channels per plane; total <= 8 */
    const void* plane_data[REF_MAX_PLANES]; /* row-major, channels interleaved */
    const float* scales;           /* NULL, or [tiles_y][tiles_x][total channels] */
    int scale_tile;                /* tile edge in texels when scales != NULL */
    /* Neural material (num_planes == 0): latent grid [nn_gh][nn_gw][16] binary16 codes, the
     * binary16 codes of W1, W2, W3 and the FP32 biases b1, b2, b3 (see stf_oracle_neural.c);
     * texels are decoded by the FP32 emulation of the GPU's inference precision. */
    const uint16_t* nn_lat16;
    int nn_gw, nn_gh, nn_r;
    const uint16_t* nn_w16;
    const float* nn_b32;
} ref_material;

/* Neural decoder (stf_oracle_neural.c). */
int stf_ref_neural_e4m3_scales(const uint16_t* lat16, int GW, int GH, const float* P32, int* e);
int stf_ref_neural_decode_e4m3(const uint16_t* lat16, int GW, int GH, int R, const float* P32, const int* idx,
                               int n, float* out, int* e_out);
int stf_ref_neural_decode(const uint16_t* lat16, int GW, int GH, int R, const uint16_t* w16, int nw,
                          const float* b32, const int* idx, int n, float* out);

typedef struct {
    int width, height;             /* pixels */
    float H[9];                    /* (x+.5, y+.5, 1) -> (u, v, w) projective, row-major */
    float cam_pos[3];
    float plane_to_world[6];       /* world x = m0 u + m1 v + m2, world z = m3 u + m4 v + m5, y = 0 */
    float light_dir[3];            /* unit vector towards the light */
    int shading;                   /* 0: output filtered channels 0..3; 1: Lambert + GGX */
    int ch_albedo, ch_normal, ch_rough, ch_ao;  /* channel indices, -1 = constant */
    float roughness;               /* used when ch_rough < 0 */
    int filter;
    int tile_w, tile_h;            /* warp pixel tile, tile_w * tile_h == 32 */
    int frame, view_id;
    /* REF_SPARSE9: fp_table[fp_patterns][32][9] lane indices (own lane first), else NULL */
    const signed char* fp_table;
    int fp_patterns;
    /* blue-noise uniforms (REF_FLAG_BLUE): ranks [2][blue_size][blue_size], else NULL */
    const uint16_t* blue;
    int blue_size;
} ref_view;

/* Counter-based hash (pcg4d, Jarzynski and Olano 2020), in place. */
void stf_ref_pcg4d(uint32_t v[4]);
/* The two per-pixel uniforms in [0,1) with 24-bit resolution. */
void stf_ref_uniforms(int x, int y, int frame, int view_id, uint64_t seed, float* ux, float* uy);
/* 1D filter weight W(d), float and double. */
float stf_ref_weight(int filter, float d);
double stf_ref_weight_f64(int filter, double d);
/* Per-axis selection: lattice index and its weight (= its 1D PMF). */
void stf_ref_select_axis(int filter, float c, float u, int* n, float* w);
/* Texel decode of one stored value. */
float stf_ref_decode(int fmt, uint32_t code);
/* Decoded channels (8 slots, unused = 0) of texel (x, y), clamp-to-edge. */
void stf_ref_fetch_texel(const ref_material* m, int x, int y, float* out);
/* Sharing footprint of a lane: returns its size, fills list (<= 16 entries). */
int stf_ref_footprint(int mode, int tile_w, int tile_h, int lane, int* list);
/* Screen -> texel float coordinates of pixel (x, y) (Section 4.5 listing, first statement). */
void stf_ref_texel_coords(const ref_view* v, int tex_w, int tex_h, int x, int y, float* cx, float* cy);
/* Shading of filtered channels (float and double), writes rgba. */
void stf_ref_shade(const ref_view* v, const float* ch, float u, float vv, float* rgba);
void stf_ref_shade_f64(const ref_view* v, const double* ch, double u, double vv, double* rgba);

/* Per pixel and colour channel: sum_k |d colour / d ch_k| * max(|ch_k|, 1) (FP64 central
 * differences) at the given filtered channels ch [npix][8]; sens [npix][3]. */
int stf_ref_shade_sensitivity(const ref_view* v, int C, const float* ch, double* sens, int npix);

/* FP32 render of one view: out_rgba [h][w][4]; out_idx [h][w] packed (ix & 0xffff) | (iy << 16)
 * of the selected texel (one-tap and sharing modes), may be NULL; out_ch [h][w][8] filtered
 * channels before shading, may be NULL. Returns 0 on success. */
int stf_ref_render(const ref_material* m, const ref_view* v, int mode, uint64_t seed,
                   float* out_rgba, uint32_t* out_idx, float* out_ch, int nthreads);

/* FP64 exact filter (Eq. texture-continuous-sum) followed by FP64 shading: the ground truth. */
int stf_ref_render_exact_f64(const ref_material* m, const ref_view* v, double* out_rgba,
                             double* out_ch, int nthreads);

#ifdef __cplusplus
}
#endif
#endif
