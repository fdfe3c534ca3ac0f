// Per-material-kind launcher: maps (filter, mode, tile shape) to the template instance.
// Each stf_kind_*.cu translation unit instantiates it for one kind, so the kinds compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include "stf_kernels.cuh"
#include "stf_nn_render.cuh"
#include "stf_pair.cuh"
#include "stf_internal.h"

namespace stf {

// Opts a kernel into its dynamic shared memory (once: `cached` is the caller's per-instance
// static) and returns its resident blocks per SM for `threads`-thread blocks.
template <class K>
static cudaError_t prepare_dynamic(K kernel, int dyn_bytes, int threads, int& cached, int* per_sm)
{
    if (!cached) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_bytes);
        // the largest shared-memory carve-out, so that every block the registers allow fits
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
        e = stf_resident_blocks(reinterpret_cast<const void*>(kernel), threads, dyn_bytes, &cached);
        if (e != cudaSuccess) return e;
        if (cached < 1) cached = 1;
    }
    *per_sm = cached;
    return cudaSuccess;
}

static int device_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <int KIND, int F, int MODE, int TW, int TH, bool EX, bool ALT, bool BLUE>
static cudaError_t launch_one(const DevView& v, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.tiles_x + kViewWarps - 1) / kViewWarps), (unsigned)v.tiles_y);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    if constexpr (KIND == K_NEURAL) {  // persistent decode-pipeline blocks over the 8-tile groups
        static int cached = 0;
        int per_sm = 1;
        constexpr int dyn = (int)sizeof(NnPipeSmem);
        cudaError_t e = prepare_dynamic(k_render_neural<F, MODE, TW, TH, EX, BLUE>, dyn, kNnPipeThreads, cached, &per_sm);
        if (e != cudaSuccess) return e;
        const long long groups = (long long)((v.tiles_x + kNnClientWarps - 1) / kNnClientWarps) * v.tiles_y;
        long long cap = (long long)per_sm * device_sms();
        if (g_pipeline_blocks > 0 && g_pipeline_blocks < cap) cap = g_pipeline_blocks;
        const unsigned blocks = (unsigned)(groups < cap ? groups : cap);
        k_render_neural<F, MODE, TW, TH, EX, BLUE><<<blocks, kNnPipeThreads, dyn, s>>>(v);
    } else {
        if constexpr (pair_path<KIND, F, MODE, TW, TH, EX, ALT, BLUE>()) {
            if (g_paired_pixels) {
                const dim3 g2((unsigned)((v.tiles_x + 2 * kPairWarps - 1) / (2 * kPairWarps)), (unsigned)v.tiles_y);
                if constexpr (!BLUE && !EX) {
                    if (v.tmap_host) {
                        k_render_pair_tma<KIND, F, MODE, TW, TH><<<g2, 32 * kPairWarps, 0, s>>>(
                            *reinterpret_cast<const CUtensorMap*>(v.tmap_host), v);
                        return cudaGetLastError();
                    }
                }
                k_render_pair<KIND, F, MODE, TW, TH, BLUE, EX><<<g2, 32 * kPairWarps, 0, s>>>(v);
                return cudaGetLastError();
            }
        }
        k_render_view<KIND, F, MODE, TW, TH, EX, ALT, BLUE><<<grid, 32 * kViewWarps, 0, s>>>(v);
    }
    return cudaGetLastError();
}

template <int KIND, int F, int MODE, bool EX, bool BLUE>
static cudaError_t launch_tiles(const DevView& v, cudaStream_t s)
{
    if (v.tile_w == 8 && v.tile_h == 4) return launch_one<KIND, F, MODE, 8, 4, EX, false, BLUE>(v, s);
    if (v.tile_w == 4 && v.tile_h == 8) return launch_one<KIND, F, MODE, 4, 8, EX, false, BLUE>(v, s);
    if (v.tile_w == 16 && v.tile_h == 2) return launch_one<KIND, F, MODE, 16, 2, EX, false, BLUE>(v, s);
    return cudaErrorInvalidValue;
}

// Sharing modes; exact filtering exists for the bilinear filter (the B-spline ignores the flag);
// the alternative estimators (v.estimator != 0) for stored kinds on 8x4 tiles.
template <int KIND, int F, int MODE, bool BLUE>
static cudaError_t launch_sharing(const DevView& v, bool ex, cudaStream_t s)
{
    if constexpr (KIND != K_NEURAL && MODE != kModeSparse9)
        if (v.estimator != 0) {
            if (v.tile_w != 8 || v.tile_h != 4) return cudaErrorInvalidValue;
            return launch_one<KIND, F, MODE, 8, 4, false, true, BLUE>(v, s);
        }
    if constexpr (F == 0)
        if (ex) return launch_tiles<KIND, F, MODE, true, BLUE>(v, s);
    return launch_tiles<KIND, F, MODE, false, BLUE>(v, s);
}

template <int KIND, int F, bool BLUE>
static cudaError_t launch_modes(const DevView& v, int mode, cudaStream_t s)
{
    const bool ex = (mode & kModeFlagExact) != 0;
    switch (mode & kModeBase) {
    case 0: return launch_one<KIND, F, 0, 8, 4, false, false, false>(v, s);  // no sharing: tile shape irrelevant
    case 1: return launch_one<KIND, F, 1, 8, 4, false, false, BLUE>(v, s);
    case 2: return launch_sharing<KIND, F, 2, BLUE>(v, ex, s);
    case 3: return launch_sharing<KIND, F, 3, BLUE>(v, ex, s);
    case 4: return launch_sharing<KIND, F, 4, BLUE>(v, ex, s);
    case 5: return launch_sharing<KIND, F, 5, BLUE>(v, ex, s);
    case 6: return launch_sharing<KIND, F, 6, BLUE>(v, ex, s);
    }
    return cudaErrorInvalidValue;
}

// mode: the C interface's reuse mode, with STF_MODE_FLAG_EXACT (kModeFlagExact) allowed.
template <int KIND, bool BLUE>
cudaError_t launch_view_kind(const DevView& v, int mode, cudaStream_t s)
{
    return v.filter == 0 ? launch_modes<KIND, 0, BLUE>(v, mode, s) : launch_modes<KIND, 1, BLUE>(v, mode, s);
}

// ------------------------------------------------------------------------------ multi-view

// The view constants of a batch, one copy per material-kind module (each stf_kind_*.cu includes
// this header once): reads with a block-uniform view index are served by the constant cache like
// kernel parameters, at no issue cost.
static __constant__ DevView c_batch_views[kBatchMaxViews];

// Persistent multi-view kernel for one (filter, tile shape) variant: each warp pulls work items
// (a run of tiles of one view) from a device counter until the list is exhausted. Nothing waits
// on another warp or block, so no wait can stall. One kernel per variant keeps the code of a
// launch as small as a single-view kernel's.
template <int KIND, int MODE, int F, int TW, int TH, bool EX, bool BLUE>
__global__ void __launch_bounds__(256, kMinBlocks)
    k_render_batch(const WorkItem* __restrict__ items, int n_items, int* counter)
{
    __shared__ float4 recs[kWarpsPerBlock * 32 * kRecPerLane];
    __shared__ float wtabs[kWarpsPerBlock * 32 * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* rec = recs + warp * 32 * kRecPerLane;
    float* wtab = wtabs + warp * 32 * 8;
    for (;;) {  // every warp pulls its own items
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;  // warp-uniform
        const WorkItem w = items[it];
        const DevView& v = c_batch_views[w.view];
        for (int k = 0; k < w.ntiles; ++k) {
            const int t = w.tile0 + k;
            const int ty = t / v.tiles_x;
            render_tile<KIND, F, MODE, TW, TH, EX, false, BLUE>(v, t - ty * v.tiles_x, ty, lane, rec, wtab);
        }
    }
}

// The multi-view kernel on the paired path (pair_path variants): every warp pulls work items on
// its own (no block barrier, so no warp waits for another's tiles) and renders two tiles of its
// item at a time, one per half-warp; a half-warp without a tile of its own renders the item's
// first tile as a stand-in, storing nothing, so that both halves reach the warp's barriers. Three
// resident 8-warp blocks per SM leave the paired path its registers.
constexpr int kPairBatchMinBlocks = 3;
template <int KIND, int MODE, int F, int TW, int TH, bool BLUE, bool EX>
__global__ void __launch_bounds__(256, kPairBatchMinBlocks)
    k_render_batch_pair(const WorkItem* __restrict__ items, int n_items, int* counter)
{
    __shared__ float4 recs[kWarpsPerBlock * 2 * 32 * kRecPerLane];
    __shared__ float wtabs[F == 1 ? kWarpsPerBlock * 2 * 32 * 8 : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4;
    const int tile = warp * 2 + half;
    float4* rec = recs + tile * 32 * kRecPerLane;
    float* wtab = wtabs + (F == 1 ? tile * 32 * 8 : 0);
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(kFull, it, 0);
        if (it >= n_items) break;  // warp-uniform
        const WorkItem w = items[it];
        const DevView& v = c_batch_views[w.view];
        for (int k = 0; k < w.ntiles; k += 2) {  // warp-uniform
            const bool live = k + half < w.ntiles;
            const int t = w.tile0 + (live ? k + half : 0);
            const int ty = t / v.tiles_x;
            render_pair<KIND, F, MODE, TW, TH, BLUE, EX>(v, t - ty * v.tiles_x, ty, lane & 15, rec, wtab, live, GlobalFetch<KIND>{v});
        }
    }
}

struct NnConstViews {
    __device__ __forceinline__ const DevView& operator()(int i) const { return c_batch_views[i]; }
};

// The neural kind's multi-view kernel: the same work items, rendered by the client warps of the
// decode pipeline (all of a batch's neural views share one decoder; view 0 names it). The client
// warps pull items together (named barrier 1), so every client takes the same rounds.
template <int MODE, int F, int TW, int TH, bool EX, bool BLUE>
__global__ void __launch_bounds__(kNnPipeThreads, 2)
    k_render_neural_batch(const WorkItem* __restrict__ items, int n_items, int* counter)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ float wtabs[kNnWtabFloats];
    __shared__ WorkItem sw;
    NnPipeSmem& sm = *reinterpret_cast<NnPipeSmem*>(dyn);
    nn_pipe_setup(sm, reinterpret_cast<const NeuralDev*>(c_batch_views[0].neural));
    if (threadIdx.x >= kNnClients) {
        nn_decode_role(sm, c_batch_views[0].flags);
    } else {
        const int warp = threadIdx.x >> 5;
        NnRenderClient<F, MODE, TW, TH, EX, BLUE, NnConstViews> cl(sm, wtabs + warp * 256, NnConstViews{}, c_batch_views[0].flags);
#pragma unroll 1
        for (;;) {
            if (threadIdx.x == 0) {
                const int it = atomicAdd(counter, 1);
                sw = it < n_items ? items[it] : WorkItem{-1, 0, 0, 0};
            }
            asm volatile("bar.sync 1, %0;" :: "n"(kNnClients) : "memory");
            const WorkItem w = sw;
            asm volatile("bar.sync 1, %0;" :: "n"(kNnClients) : "memory");  // sw is rewritten by the next pull
            if (w.view < 0) break;
            const DevView& v = c_batch_views[w.view];
            const int groups = (w.ntiles + kNnClientWarps - 1) / kNnClientWarps;
#pragma unroll 1
            for (int k = 0; k < groups; ++k) {
                const int j = k * kNnClientWarps + warp;
                const bool active = j < w.ntiles;
                const int t = w.tile0 + (active ? j : 0);
                const int ty = t / v.tiles_x;
                cl.group(w.view, active, t - ty * v.tiles_x, ty);
            }
        }
        cl.finish();
    }
    nn_pipe_teardown(sm);
}

// grid > 0 launches; grid == 0 only reports the instance's resident blocks per SM in *per_sm.
template <int KIND, int MODE, int F, int TW, int TH, bool EX, bool BLUE>
static cudaError_t launch_batch_v(const WorkItem* items, int n_items, int* counter, int grid, int* per_sm, cudaStream_t s)
{
    if constexpr (KIND == K_NEURAL) {
        static int cached = 0;
        constexpr int dyn = (int)sizeof(NnPipeSmem);
        int n = 0;
        cudaError_t e = prepare_dynamic(k_render_neural_batch<MODE, F, TW, TH, EX, BLUE>, dyn, kNnPipeThreads, cached, &n);
        if (e != cudaSuccess || grid == 0) {
            *per_sm = n;
            return e;
        }
        k_render_neural_batch<MODE, F, TW, TH, EX, BLUE><<<grid, kNnPipeThreads, dyn, s>>>(items, n_items, counter);
    } else {
        if constexpr (pair_path<KIND, F, MODE, TW, TH, EX, false, BLUE>()) {
            if (g_paired_pixels) {
                if (grid == 0)
                    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_render_batch_pair<KIND, MODE, F, TW, TH, BLUE, EX>, 256, 0);
                k_render_batch_pair<KIND, MODE, F, TW, TH, BLUE, EX><<<grid, 256, 0, s>>>(items, n_items, counter);
                return cudaGetLastError();
            }
        }
        if (grid == 0)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_render_batch<KIND, MODE, F, TW, TH, EX, BLUE>, 256, 0);
        k_render_batch<KIND, MODE, F, TW, TH, EX, BLUE><<<grid, 256, 0, s>>>(items, n_items, counter);
    }
    return cudaGetLastError();
}

// variant = filter * 3 + tile shape (0: 8x4, 1: 4x8, 2: 16x2), + 6 for bilinear with exact
// filtering; without sharing only 8x4 exists.
template <int KIND, int MODE, bool BLUE>
static cudaError_t launch_batch_mode(const WorkItem* items, int n_items, int* counter, int grid, int variant, int* per_sm,
                                     cudaStream_t s)
{
    if constexpr (MODE <= 1) {
        if (variant == 0) return launch_batch_v<KIND, MODE, 0, 8, 4, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        if (variant == 3) return launch_batch_v<KIND, MODE, 1, 8, 4, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        return cudaErrorInvalidValue;
    } else {
        switch (variant) {
        case 0: return launch_batch_v<KIND, MODE, 0, 8, 4, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 1: return launch_batch_v<KIND, MODE, 0, 4, 8, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 2: return launch_batch_v<KIND, MODE, 0, 16, 2, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 3: return launch_batch_v<KIND, MODE, 1, 8, 4, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 4: return launch_batch_v<KIND, MODE, 1, 4, 8, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 5: return launch_batch_v<KIND, MODE, 1, 16, 2, false, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 6: return launch_batch_v<KIND, MODE, 0, 8, 4, true, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 7: return launch_batch_v<KIND, MODE, 0, 4, 8, true, BLUE>(items, n_items, counter, grid, per_sm, s);
        case 8: return launch_batch_v<KIND, MODE, 0, 16, 2, true, BLUE>(items, n_items, counter, grid, per_sm, s);
        }
        return cudaErrorInvalidValue;
    }
}

template <int KIND, bool BLUE>
cudaError_t launch_batch_kind(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant,
                              int* per_sm, cudaStream_t s)
{
    switch (mode & kModeBase) {  // the exact flag is in the variant
    case 0: return launch_batch_mode<KIND, 0, BLUE && 0 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 1: return launch_batch_mode<KIND, 1, BLUE && 1 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 2: return launch_batch_mode<KIND, 2, BLUE && 2 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 3: return launch_batch_mode<KIND, 3, BLUE && 3 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 4: return launch_batch_mode<KIND, 4, BLUE && 4 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 5: return launch_batch_mode<KIND, 5, BLUE && 5 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    case 6: return launch_batch_mode<KIND, 6, BLUE && 6 != 0>(items, n_items, counter, grid, variant, per_sm, s);
    }
    return cudaErrorInvalidValue;
}

// Copies a batch's view constants (device memory, at most kBatchMaxViews) into this module's
// constant bank on stream s.
static cudaError_t set_batch_views(const DevView* views, int n_views, cudaStream_t s)
{
    if (n_views < 1 || n_views > kBatchMaxViews) return cudaErrorInvalidValue;
    return cudaMemcpyToSymbolAsync(c_batch_views, views, (size_t)n_views * sizeof(DevView), 0, cudaMemcpyDeviceToDevice, s);
}

}  // namespace stf

// A kind's entry points: NAME renders one view, NAME##_batch runs a batch variant, and
// NAME##_batch_views fills this module's view constants. Blue-noise modes run kernels compiled in
// the kind's second translation unit (STF_INSTANTIATE_KIND_BLUE, the same entry points with the
// suffix _b and its own constant bank), so that the plain kernels carry no trace of them.
#define STF_INSTANTIATE_KIND(KIND, NAME)                                                        \
    namespace stf {                                                                             \
    cudaError_t NAME##_b(const DevView& v, int mode, cudaStream_t s);                           \
    cudaError_t NAME##_b_batch(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant, \
                               int* per_sm, cudaStream_t s);                                    \
    cudaError_t NAME##_b_batch_views(const DevView* views, int n_views, cudaStream_t s);        \
    cudaError_t NAME(const DevView& v, int mode, cudaStream_t s)                                \
    {                                                                                           \
        if (mode & kModeFlagBlue) return NAME##_b(v, mode, s);                                  \
        return launch_view_kind<KIND, false>(v, mode, s);                                       \
    }                                                                                           \
    cudaError_t NAME##_batch(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant, \
                             int* per_sm, cudaStream_t s)                                       \
    {                                                                                           \
        if (mode & kModeFlagBlue) return NAME##_b_batch(items, n_items, counter, grid, mode, variant, per_sm, s); \
        return launch_batch_kind<KIND, false>(items, n_items, counter, grid, mode, variant, per_sm, s); \
    }                                                                                           \
    cudaError_t NAME##_batch_views(const DevView* views, int n_views, int mode, cudaStream_t s) \
    {                                                                                           \
        if (mode & kModeFlagBlue) return NAME##_b_batch_views(views, n_views, s);               \
        return set_batch_views(views, n_views, s);                                              \
    }                                                                                           \
    }

#define STF_INSTANTIATE_KIND_BLUE(KIND, NAME)                                                   \
    namespace stf {                                                                             \
    cudaError_t NAME##_b(const DevView& v, int mode, cudaStream_t s) { return launch_view_kind<KIND, true>(v, mode, s); } \
    cudaError_t NAME##_b_batch(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant, \
                               int* per_sm, cudaStream_t s)                                     \
    {                                                                                           \
        return launch_batch_kind<KIND, true>(items, n_items, counter, grid, mode, variant, per_sm, s); \
    }                                                                                           \
    cudaError_t NAME##_b_batch_views(const DevView* views, int n_views, cudaStream_t s)         \
    {                                                                                           \
        return set_batch_views(views, n_views, s);                                              \
    }                                                                                           \
    }
