// Host-side internals shared by the library's translation units (not part of the C interface).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdarg>

#include "stf.h"
#include "stf_device.cuh"

struct stf_texture {
    int width, height, channels;
    int kind;                       // stf::MatKind
    void* texels;                   // device records
    float* scales;                  // device, E4M3 kind only
    int scale_shift, scale_tiles_x;
    const stf_decoder* decoder;     // NEURAL kind
    const void* decoder_params;     // device parameter block of the decoder (NEURAL kind)
    bool widened = false;           // texels converted at creation (no plane-byte updates)
    // tensor map over the texel records for the TMA-staged render variant, made on first use
    // (tmap_state 1) or found impossible (-1: a row pitch that is not a multiple of 16 bytes)
    mutable CUtensorMap tmap;
    mutable int tmap_state = 0;
};

// The texture's tensor map (made on first use), or null if its layout has none.
const CUtensorMap* stf_texture_tmap(const stf_texture* t);
// STF_OPT_TMA_STAGE (0, default: the read-only global path).
extern int g_tma_stage;

stf_status stf_fail(stf_status s, const char* fmt, ...);
stf_status stf_cuda_fail(cudaError_t e, const char* what);
cudaStream_t stf_stream();
stf_status stf_device_state(int** flags, const float** lut);
stf_status stf_device_state_ready(int** flags);  // no set-up, no allocation
stf_status stf_validate_view(const stf_view& v, int i, int filter, int mode);
void stf_fill_devview(const stf_view& v, int filter, int mode, unsigned long long seed, const float* lut,
                      stf::DevView& d);
cudaError_t stf_launch_single(const stf::DevView& d, int kind, int mode, cudaStream_t s);

// multi-view scheduler (stf_sched.cu)
stf_status stf_render_batch(const stf_view* views, int n, int filter, int mode, unsigned long long seed);

// tile shape and schedule of a view, as the multi-view scheduler resolves them (no heap use)
void stf_resolve_view_config_nohalloc(const stf_view& v, int filter, int mode, int* tw, int* th, int* sched);

// STF_OK for a valid reuse mode (optionally with STF_MODE_FLAG_EXACT), else sets the error.
stf_status stf_check_mode(int mode);

// The current device's sparse footprint patterns (stf_set_sparse_footprints); false if none.
bool stf_sparse_state(const uint8_t** table, int* patterns, int* tile_w, int* tile_h);

// The current device's blue-noise masks (stf_set_blue_noise); false if none.
bool stf_blue_state(const uint16_t** ranks, int* shift);

// STF_OPT_PIPELINE_BLOCKS (0: fill the SMs).
extern int g_pipeline_blocks;
// STF_OPT_PAIRED_PIXELS (1, default: two pixels per thread where the paired path exists).
extern int g_paired_pixels;

// resident blocks per SM, counted from the kernel's resources (stf_api.cu)
cudaError_t stf_resident_blocks(const void* kernel, int threads, int dyn_bytes, int* n);

// neural decoder (stf_neural.cu)
stf_status stf_create_neural_texture(const stf_texture_desc* d, stf_texture** out);
cudaError_t stf_launch_neural_view(const stf::DevView& d, int mode, cudaStream_t s);
