/*
 * stf.h - C interface of the GB300 library for magnified stochastic texture filtering (STF)
 * with sample reuse ("Improved Stochastic Texture Filtering Through Sample Reuse",
 * Wronski, Pharr, Akenine-Moller, 2025).
 *
 * The problem (Section 2.1, Eq. texture-continuous-sum): for each pixel, estimate the filtered
 * texture value sum_i f_r(u - u_i, v - v_i) T_i at the pixel's texture coordinate, then shade.
 * The library estimates it the paper's way: each pixel draws ONE texel with probability equal
 * to its filter weight (one-tap STF, Eq. mc-estimator and Section S1), the pixels of a 32-lane
 * warp tile share their texels through per-warp shared-memory records, the CUDA counterpart of
 * the paper's wave intrinsics (Section 4.3, Section 4.5), and each pixel
 * combines the shared texels with the bounded weighted importance sampling estimator
 * w_i = f_c(x_i) / f_i(x_i), result = sum_i w_i T_i / sum_j w_j (Eqs. bart-weighted-estimator,
 * estimator-for-stf and estimator-convex, Section 4.2).
 *
 * Conventions for every entry point:
 *   - Functions return stf_status; no C++ exception crosses the interface.
 *   - On a non-OK status, stf_last_error() returns a message for the calling thread.
 *   - Work is enqueued asynchronously on the stream set with stf_set_stream (default: the
 *     legacy default stream). Device-side error flags are reported by stf_sync() and by the
 *     next stf_render_views() call.
 *   - Pointers documented as "device" must be CUDA device (or managed) memory of the current
 *     device; "host" pointers are ordinary CPU memory.
 *   - Not thread-safe: callers serialise calls that share a stream or a texture.
 */
#ifndef STF_H
#define STF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    STF_OK = 0,
    STF_ERR_INVALID_ARG = 1,   /* rejected on the host, nothing enqueued */
    STF_ERR_UNSUPPORTED = 2,   /* a valid request this build does not implement */
    STF_ERR_OUT_OF_MEMORY = 3, /* a device allocation failed */
    STF_ERR_CUDA = 4,          /* a CUDA runtime call failed; the message names it */
    STF_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (persistent scheduler) */
    STF_ERR_DEVICE_ASSERT = 6  /* a device-side check recorded an out-of-range index */
} stf_status;

/* Reconstruction filters: bilinear (tent) per Section S6; uniform cubic B-spline per Section
 * 5.4. STF_FILTER_PER_VIEW takes stf_view.filter for each view. */
typedef enum { STF_FILTER_BILINEAR = 0, STF_FILTER_BSPLINE3 = 1, STF_FILTER_PER_VIEW = -1 } stf_filter;

/* Estimators:
 *   FULL     deterministic filter, every texel under the filter fetched and weighted (the
 *            comparator of Section 5.6);
 *   ONE_TAP  one-tap STF, the texel drawn by the pixel itself (Section 2.2);
 *   QUAD2    sharing inside aligned 2x2 pixel quads (Table 1 "2x2q");
 *   WAVE2/3/4 square k x k sharing footprints placed per lane inside the warp tile (Section
 *            4.3.1; Table 1 "2x2w", "3x3", "4x4"). On a 16x2 tile the k x k block becomes
 *            min(k,2) rows by round(k*k/2) columns. */
typedef enum {
    STF_MODE_FULL = 0, STF_MODE_ONE_TAP = 1, STF_MODE_QUAD2 = 2,
    STF_MODE_WAVE2 = 3, STF_MODE_WAVE3 = 4, STF_MODE_WAVE4 = 5,
    STF_MODE_SPARSE9 = 6  /* pseudorandom sparse 9-lane footprints, the patterns set by
                           * stf_set_sparse_footprints, pattern frame % patterns (Section
                           * "Sharing Footprints Within Waves"); views take the patterns' tile */
} stf_reuse_mode;

/* Exact filtering (Section "Exact Filtering"), OR'd into a sharing mode (QUAD2 .. WAVE4): with
 * the bilinear filter, a pixel whose footprint samples include every texel of positive weight in
 * its own filter returns the deterministic filter over those samples (bit-identical to
 * STF_MODE_FULL at that pixel) instead of the estimate. B-spline views ignore the flag (16 taps
 * are rarely all drawn, Section "Exact Filtering"). With FULL or ONE_TAP: STF_ERR_INVALID_ARG. */
#define STF_MODE_FLAG_EXACT 16

/* Blue-noise selection uniforms (Section "Blue Noise Mask Improvements"), OR'd into any mode but
 * FULL: a pixel's two uniforms are its ranks r in the two masks set by stf_set_blue_noise, at
 * (x mod n, y mod n), as (r + 1/2) / n^2 plus the frame's offset frame * (sqrt(5) - 1) / 2 + the
 * seed's low 24 bits / 2^24, modulo 1 (all in 24-bit fixed point) instead of the pcg4d hash. */
#define STF_MODE_FLAG_BLUE_NOISE 32

/* The estimator of a sharing mode, reuse_mode | (estimator << STF_MODE_EST_SHIFT), over the
 * footprint's samples x_i (drawn from the PMFs p_i = lane i's filter weights), with
 * f(x) = w_c(x) T(x) for the pixel's own filter w_c (Section 4.1 and Section 4.2):
 *   STF_EST_WIS           the paper's weighted estimator (default)
 *   STF_EST_IS            importance sampling, (1/n) sum f(x_i)/p_i(x_i)  (Eq. eq_basic_mc)
 *   STF_EST_MIS           balance heuristic, sum f(x_i) / sum_k p_k(x_i)
 *   STF_EST_PAIRWISE_MIS  pairwise MIS with the pixel's own sample as the canonical technique
 *   STF_EST_REGRESSION    control variate h = w_c/p (mean 1), y = f/p, beta from the samples
 *                         (Eq. eq_mc_regression)
 * STF_MODE_FLAG_CLAMP clamps a non-weighted estimate per channel to the range of the sampled
 * texels its own filter weighs. These are evaluation modes for the estimator comparison: one
 * view per call, stored material kinds, 8x4 tiles, no exact filtering; anything else
 * STF_ERR_INVALID_ARG. */
#define STF_MODE_EST_SHIFT 8
typedef enum {
    STF_EST_WIS = 0, STF_EST_IS = 1, STF_EST_MIS = 2, STF_EST_PAIRWISE_MIS = 3, STF_EST_REGRESSION = 4
} stf_estimator;
#define STF_MODE_FLAG_CLAMP 2048

/* Stored texel formats. FP16 = IEEE binary16, BF16 = bfloat16, E4M3 = OCP FP8 E4M3 ("FN"),
 * UNORM8 = q / 255. NEURAL = texels decoded by a small MLP from a latent grid (see
 * stf_decoder_*). */
typedef enum {
    STF_FMT_FP32 = 0, STF_FMT_FP16 = 1, STF_FMT_BF16 = 2, STF_FMT_E4M3 = 3, STF_FMT_UNORM8 = 4,
    STF_FMT_NEURAL = 5
} stf_format;

typedef struct stf_texture stf_texture; /* opaque, library-owned */
typedef struct stf_decoder stf_decoder; /* opaque, library-owned */

/* One plane of a material: `channels` values of format `fmt` per texel, texels row-major,
 * channels interleaved. `data` is host memory unless data_on_device != 0. */
typedef struct {
    int fmt;
    int channels;
    const void* data;
    int data_on_device;
} stf_plane;

/* A material: 1..4 planes sharing one width x height (max 16384 x 16384), 1..8 channels in
 * total, numbered across planes in order. Optional per-(tile, channel) FP32 scales multiply
 * the decoded value: tile_scales[(ty * tiles_x + tx) * channels + c] with tiles of scale_tile x
 * scale_tile texels (tiles_x = ceil(width / scale_tile)); pass NULL for none. For a NEURAL
 * material set num_planes = 0 and `decoder`. */
typedef struct {
    int width, height;
    int num_planes;
    stf_plane planes[4];
    const float* tile_scales;
    int scale_tile;
    int scales_on_device;
    const stf_decoder* decoder;
} stf_texture_desc;

/* One view (one output image). The pixel centre (x + 0.5, y + 0.5, 1) is mapped by the
 * row-major projective matrix H to (hu, hv, hw); uv = (hu / hw, hv / hw) in [0, 1]^2 spans the
 * texture (an analytic stand-in for the paper's G-buffer UVs, Section 5). Texel float
 * coordinates are uv * size - 0.5 (Section 4.5 listing). Addressing is clamp-to-edge.
 *
 * Shading (shading = 1) runs after the estimate, on the filtered channels: Lambert plus GGX
 * (Smith height-correlated visibility, Schlick Fresnel with F0 = 0.04) lit by one directional
 * light of irradiance pi from light_dir (unit, towards the light). The ground plane is y = 0 with
 * tangent frame T = +x, B = +z, N = +y; a pixel's world point is (m0 u + m1 v + m2, 0,
 * m3 u + m4 v + m5) with m = plane_to_world. Channel map: ch_albedo (3 channels), ch_normal
 * (tangent-space X, Y; Z reconstructed), ch_rough (else `roughness`), ch_ao (else 1); -1 means
 * absent. shading = 0 writes the filtered channels 0..3 (missing ones 0, alpha 1).
 *
 * tile_w x tile_h is the warp's pixel tile: 8x4, 4x8 or 16x2, or 0x0 to let the library pick.
 * Outputs: out_rgba (device, float4 per pixel, row pitch out_pitch_floats floats, 0 = 4 *
 * width) is written for every on-screen pixel. debug_indices (device, optional, width * height
 * uint32) receives the selected texel as (ix & 0xffff) | (iy << 16) (unclamped lattice
 * coordinates; 0 in FULL mode). debug_channels (device, optional, width * height * 8 floats)
 * receives the filtered channels before shading. The random stream of a pixel is keyed by
 * (x, y, frame | view_id << 16, seed); frame and view_id must be below 65536. */
typedef struct {
    int width, height;
    float H[9];
    float cam_pos[3];
    float plane_to_world[6];
    float light_dir[3];
    int shading;
    int ch_albedo, ch_normal, ch_rough, ch_ao;
    float roughness;
    int filter;
    int tile_w, tile_h;
    int frame;
    int view_id;
    const stf_texture* tex;
    float* out_rgba;
    long long out_pitch_floats;
    uint32_t* debug_indices;
    float* debug_channels;
} stf_view;

/* Creates a texture from a material description (Section 2.1, Eq. texture-definition: a texel
 * lattice). The library copies the texels into its own device memory, interleaving all planes
 * of a texel into one record of 4, 8, 16 or 32 bytes; stf_destroy frees it. Formats are kept
 * as stored (FP16 stays FP16 in device memory) where a dedicated kernel exists; any other
 * combination is widened to FP32 at creation, which is exact because every decode is.
 * Errors: STF_ERR_INVALID_ARG for a bad description (the message says which field),
 * STF_ERR_OUT_OF_MEMORY, STF_ERR_CUDA. *out is set only on success. Synchronous. */
stf_status stf_create_texture(const stf_texture_desc* desc, stf_texture** out);

/* Renders n views (host array `views`, n >= 1) with one estimator for all of them: for every
 * pixel, the filtered texture value of Eq. texture-continuous-sum (Section 2.1) at the pixel's
 * texture coordinate, estimated by one-tap STF (Section 2.2, Section S1) and, in the sharing
 * modes, by the weighted combination of the warp tile's samples (Section 4.2, the loop of
 * Section 4.5), then shaded. `filter` is STF_FILTER_BILINEAR / STF_FILTER_BSPLINE3 for every view, or STF_FILTER_PER_VIEW.
 * `reuse_mode` is an stf_reuse_mode, optionally | STF_MODE_FLAG_EXACT or an estimator
 * (STF_MODE_EST_SHIFT, STF_MODE_FLAG_CLAMP). `seed` keys the
 * counter-based random stream (pcg4d of
 * Jarzynski and Olano 2020) together with each pixel's (x, y, frame, view_id).
 * Each view's texture must outlive the enqueued work. Every view is validated before anything
 * is enqueued; on STF_ERR_INVALID_ARG no output is touched. Several views are rendered by one
 * persistent launch that pulls (view, tile range) items from a device queue.
 * Asynchronous on the library stream. */
stf_status stf_render_views(const stf_view* views, int n, int filter, int reuse_mode,
                            unsigned long long seed);

/* Multi-view scheduling (used when stf_render_views gets n > 1 views). Views are grouped by
 * material kind and cut into work items of 8 x schedule tiles; one persistent kernel per kind
 * pulls items from a device counter, costliest views first. The view constants and item list go
 * to the device in one copy from a pinned staging buffer; copy, counter reset and kernels are
 * captured once into a CUDA graph and replayed while the batch keeps its shape (same views per
 * kind, same item count). */
enum { STF_OPT_BATCH_GRAPHS = 1,   /* 1 (default): replay CUDA graphs */
       STF_OPT_PIPELINE_BLOCKS = 2, /* > 0: at most this many persistent blocks for a neural-material
                                     * view (each then runs more decode rounds); 0 (default): fill the
                                     * SMs */
       STF_OPT_TEST_DECODE_STALL = 3, /* testing aid for failure detection: 1 makes the next
                                      * stf_decoder_decode pipeline (the render kernels ignore the
                                      * switch) withhold its first layer-1 products, so its
                                      * bounded waits run out (2^20 polls) and every wait of the
                                      * launch then returns at once; outputs of that launch are
                                      * garbage and stf_sync reports STF_ERR_TIMEOUT, which also
                                      * clears the switch. No device fault is involved. */
       STF_OPT_PAIRED_PIXELS = 4,    /* 1 (default): single-view renders of the stored kinds with the
                                      * bilinear filter (no exact filtering, estimator or blue noise)
                                      * run two vertically adjacent pixels per thread wherever the
                                      * pair shares one sharing footprint (same estimates, fewer
                                      * shared-memory reads and packed arithmetic); 0: one pixel per
                                      * thread everywhere */
       STF_OPT_TMA_STAGE = 5         /* 1: the paired single-view kernels first stage each block's texel
                                      * footprint in shared memory with the tensor memory accelerator
                                      * (cp.async.bulk.tensor), then fetch from there; 0 (default):
                                      * fetch through the read-only global path. Same pixels. */ };
enum { STF_STAT_GRAPH_BUILDS = 1, STF_STAT_GRAPH_REPLAYS = 2 };
stf_status stf_set_option(int option, long long value);
stf_status stf_get_stat(int stat, long long* value);

/* Autotuner. A view class is (material kind, filter, estimator, magnification bucket at the view
 * centre: <2, <8, <32, >=32 pixels per texel, resolution bucket: <0.5, <3, >=3 Mpixel). For
 * every class present in `views`, stf_autotune renders the class's largest view with each warp
 * tile (8x4, 4x8, 16x2; sharing modes only) and schedule (1, 2, 4, 8 tiles per warp per work
 * item), times them with CUDA events on the library stream, and keeps the fastest. Views with
 * tile 0x0 then use their class's tile; the schedule applies to multi-view batches. The tile
 * shape changes the sharing footprints, so it changes the estimate (not its validity).
 * Autotuning renders into the given views' outputs. Synchronous. */
stf_status stf_autotune(const stf_view* views, int n, int filter, int reuse_mode, unsigned long long seed);
/* Tile shape and schedule `view` would be rendered with. */
stf_status stf_view_config(const stf_view* view, int filter, int reuse_mode, int* tile_w, int* tile_h,
                           int* schedule);
/* Text table of tuned classes (one "class tile_w tile_h schedule ms" line each, under a header
 * naming the GPU); load merges entries into the current table. */
stf_status stf_autotune_save(const char* path);
stf_status stf_autotune_load(const char* path);
stf_status stf_autotune_clear(void);

/* Allocation-free multi-view rendering (this entry point has no counterpart in the paper).
 * For callers that cannot let a library allocate device memory: a render thread working inside a
 * fixed, pre-reserved device-memory budget, or a frame loop that must not stall, since
 * cudaMalloc / cudaFree can synchronise the device and can fail mid-frame. Renders the batch
 * exactly as stf_render_views does (same kernels, same pixels) but calls no cudaMalloc, cudaFree
 * or other allocating routine: its scratch (view constants, work items, work-queue counters) is a
 * fixed __device__ array of about 4.2 MB inside the library, held by every GPU that loads it
 * until the process exits. Inputs (textures, created beforehand) and outputs stay the caller's.
 * Limits: at most STF_NOALLOC_MAX_VIEWS views per call (more -> STF_ERR_INVALID_ARG, nothing
 * enqueued); work items are coarsened to fit STF_NOALLOC_MAX_ITEMS, which changes no pixel;
 * neural-texture views of one call must share one decoder (else STF_ERR_INVALID_ARG).
 * The first call on a device looks up the array's device address and uploads a 1 KB table with
 * a blocking copy: make it before any stream capture. The per-device error flags the kernels
 * report through are set up by stf_create_texture; on a device where no texture was created the
 * call returns STF_ERR_UNSUPPORTED instead of allocating them. All calls share the array (the
 * counters are cleared on each call): calls that overlap on the GPU race. The host-side staging
 * is static as well; a lock serialises calls made from several host threads. Asynchronous on the
 * library stream otherwise. */
#define STF_NOALLOC_MAX_VIEWS 224
#define STF_NOALLOC_MAX_ITEMS 262144
stf_status stf_render_views_noalloc(const stf_view* views, int n, int filter, int reuse_mode,
                                    unsigned long long seed);

/* Pseudorandom sparse sharing footprints (Section "Sharing Footprints Within Waves"; Appendix
 * "Pseudorandom Sparse Footprint Generation Algorithm"): for each of `patterns` patterns and each
 * lane of a tile_w x tile_h tile (32 lanes), `count` lane indices (the lane first, then count - 1
 * distinct others) into table[pattern][lane][count] (host). Three stages per restart: per lane
 * `candidates` candidate sets drawn at normally distributed offsets (standard deviation `sigma`
 * lanes per axis, relaxed near the tile's border), the best of `picks` random choices by the
 * standard deviation of the lanes' usage counts, then coordinate descent over the candidates;
 * the best of `restarts` restarts is kept, its score in scores[pattern] (host, may be NULL).
 * Deterministic for a seed. The paper's setting: count 9, sigma 1.4, 16-32 candidates, 10,000
 * picks, 30 restarts. Host only, synchronous. Errors: STF_ERR_INVALID_ARG. */
#define STF_SPARSE_MAX_COUNT 16
stf_status stf_sparse_footprints(int tile_w, int tile_h, int count, double sigma, int candidates, int picks,
                                 int restarts, unsigned long long seed, int patterns, signed char* table,
                                 double* scores);

/* Sets the current device's footprint patterns for STF_MODE_SPARSE9: table[patterns][32][9]
 * (host) of lane indices for a tile_w x tile_h tile, own lane first, distinct, 0..31 (as
 * stf_sparse_footprints makes with count 9). Frame f uses pattern f % patterns. Waits for the
 * device (the old patterns may be in use), may allocate device memory. Errors:
 * STF_ERR_INVALID_ARG for a malformed table (nothing changes). */
#define STF_SPARSE_MAX_PATTERNS 256
stf_status stf_set_sparse_footprints(const signed char* table, int patterns, int tile_w, int tile_h);

/* Blue-noise masks (Section "Blue Noise Mask Improvements"): two independent scalar masks of
 * size x size (a power of two, 4..256) made with the void-and-cluster method on the torus
 * (Gaussian energy of standard deviation `sigma` pixels); with quad_energy != 0 the energy a pixel
 * splats onto the other pixels of its aligned 2x2 quad is doubled (the paper's modification for
 * quad sharing). ranks[2][size][size] (host) receives each pixel's rank 0 .. size^2 - 1.
 * Deterministic for a seed. Host only, synchronous. */
stf_status stf_blue_noise_masks(int size, double sigma, int quad_energy, unsigned long long seed, uint16_t* ranks);
/* Sets the current device's masks for STF_MODE_FLAG_BLUE_NOISE: ranks[2][size][size] (host),
 * each mask a permutation of 0 .. size^2 - 1. Waits for the device, may allocate device memory.
 * Errors: STF_ERR_INVALID_ARG (nothing changes). */
stf_status stf_set_blue_noise(const uint16_t* ranks, int size);

/* Replaces a texture's texels (no allocation): `data` holds plane 0 exactly as at creation
 * (width * height records of the plane's format and channels), host or device memory
 * (data_on_device). For textures kept in their plane's own layout (one plane: FP32 x 4 or 8,
 * FP16 x 4 or 8, BF16 x 8, E4M3 x 8 whose scales stay); others STF_ERR_UNSUPPORTED. One
 * cudaMemcpyAsync on the library stream, ordered with renders there: host data must stay valid
 * until the stream reaches the copy, and must be pinned for the copy to be asynchronous. This
 * is how a frame loop streams new texel data (e.g. a video or procedural texture) each frame. */
stf_status stf_update_texture(stf_texture* tex, const void* data, int data_on_device);

/* Frees a texture (NULL is a no-op). The caller ensures no enqueued work still reads it. */
stf_status stf_destroy(stf_texture* tex);

/* Sets the CUDA stream (a cudaStream_t passed as void*) for all later work; NULL = legacy
 * default stream. */
stf_status stf_set_stream(void* cuda_stream);

/* Waits for the library stream and reports device-side error flags (STF_ERR_TIMEOUT,
 * STF_ERR_DEVICE_ASSERT), clearing them. */
stf_status stf_sync(void);

/* Message for the last non-OK status on the calling thread ("" if none). */
const char* stf_last_error(void);

/* ------------------------------------------------------------------------------------------
 * Neural texel decoder (the costly per-texel decode that stochastic filtering amortises,
 * Sections 1 and 5.6: neural texture compression). Not a model from the paper, whose
 * compressed-material format is not given; the library's small stand-in:
 *   latents: a latent_w x latent_h grid of 16 channels, R = tex_w / latent_w texels per cell
 *            (a power of two <= 16, the same on both axes);
 *   inputs:  the grid bilinearly interpolated at (i + 0.5) / R - 0.5 per axis (clamp-to-edge),
 *            plus sin/cos(2 pi phi), sin/cos(4 pi phi) of phi = ((i mod R) + 0.5) / R per axis;
 *   MLP:     24 -> 64 -> 64 -> 8 with ReLU; parameters W1[64][24], b1, W2[64][64], b2, W3[8][64],
 *            b3 (6280 values, in this order).
 * Training: Adam on the mean squared error over the 8 channels of an FP32 target texture,
 * `batch` texels per step drawn by a counter hash of (step, seed); FP32 on the CUDA cores,
 * bit-reproducible. Inference (render path, stf_decoder_decode): FP16 latents and weights, the
 * latent interpolation in FP16 arithmetic (corner weights rounded to FP16, w00 L00 + w10 L10 +
 * w01 L01 + w11 L11 with one rounding per multiply and per fused multiply-add), FP16 inputs and
 * hidden activations, FP32 accumulation on the tensor cores.
 * ------------------------------------------------------------------------------------------ */
typedef struct {
    int tex_w, tex_h;
    int latent_w, latent_h;
    int batch;                     /* texels per step, a multiple of 256 */
    float lr_latent, lr_mlp, beta1, beta2, eps;
    unsigned long long seed;       /* initialisation and batch sampling */
} stf_decoder_config;

/* Creates a decoder with seeded random initialisation (device memory, library-owned). */
stf_status stf_decoder_create(const stf_decoder_config* cfg, stf_decoder** out);
/* Runs `steps` Adam steps against `target` (an 8-channel FP32 texture of the decoder's size);
 * losses (host, may be NULL) receives each step's batch loss. Synchronous. */
stf_status stf_decoder_train(stf_decoder* d, const stf_texture* target, int steps, float* losses);
/* Loss and gradients over the given texels (host array of packed ix | iy << 16) without updating:
 * grad_params (host, 6280), grad_latent (host, latent_w * latent_h * 16), loss (host). Synchronous. */
stf_status stf_decoder_gradients(stf_decoder* d, const stf_texture* target, const int32_t* texels, int n,
                                 float* grad_params, float* grad_latent, float* loss);
/* Copies the FP32 parameters out (host) / in (host; the inference copy is refreshed). */
stf_status stf_decoder_get_params(const stf_decoder* d, float* latent, float* params);
stf_status stf_decoder_set_params(stf_decoder* d, const float* latent, const float* params);
/* Decodes n texels (device array of packed ix | iy << 16) into out (device, n * 8 floats,
 * 16-byte aligned) with the inference kernel. Asynchronous on the library stream. */
stf_status stf_decoder_decode(const stf_decoder* d, const int32_t* texels, int n, float* out);
/* Inference precision of a decoder (Section 5.6 names neural texture decompression as the costly
 * decode that stochastic filtering amortises; the FP8 option is this library's, as the compressed
 * format is not given):
 *   STF_NN_FP16 (the default) as described above;
 *   STF_NN_E4M3 layers 2 and 3 as OCP E4M3 tensor-core products (kind::f8f6f4, FP32 accumulation):
 *               W2, W3 and both hidden activations rounded to E4M3 (nearest even, saturating,
 *               ReLU before the rounding), each bias of those layers as three E4M3 parts; layer 1
 *               stays FP16. Power-of-two scalings s1 (layer-1 weights and bias), s2 (W2), s3 (W3),
 *               chosen from a first-order bound of the activations (max |latent| per channel, the
 *               parameters' absolute row sums) so that no weight or activation exceeds 448, keep
 *               the values in range; outputs are multiplied by 1 / (s1 s2 s3).
 * The choice holds for stf_decoder_decode and for every texture made from the decoder, and is
 * kept across training and stf_decoder_set_params (the scalings are recomputed whenever the
 * inference copy is refreshed); a loaded checkpoint starts in FP16. exponents (host, may be
 * NULL) receives log2 s1, log2 s2, log2 s3 and log2 of the output scale (zeros for FP16).
 * Synchronous (it reads the latent grid back to find the bound). Must not overlap a render or
 * decode that uses the decoder. STF_ERR_INVALID_ARG for another format. */
enum { STF_NN_FP16 = 0, STF_NN_E4M3 = 1 };
stf_status stf_decoder_set_inference(stf_decoder* d, int format, int* exponents);
/* Configuration and number of completed training steps. */
stf_status stf_decoder_info(const stf_decoder* d, stf_decoder_config* cfg, long long* step);
/* Checkpoints: parameters, Adam moments, step, configuration and a CRC-32 of the file. load
 * rejects a wrong magic, an inconsistent header or a checksum mismatch with
 * STF_ERR_INVALID_ARG before touching the GPU. */
stf_status stf_decoder_save(const stf_decoder* d, const char* path);
stf_status stf_decoder_load(const char* path, stf_decoder** out);
/* Frees a decoder; textures created from it must be destroyed first. */
stf_status stf_decoder_destroy(stf_decoder* d);

/* Library version as major * 10000 + minor * 100 + patch. */
int stf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* STF_H */
