// Per-material-kind launcher: maps (filter, mode, tile shape) to the template instance.
// Each stf_kind_*.cu translation unit instantiates it for one kind, so the kinds compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include "stf_kernels.cuh"

namespace stf {

template <int KIND, int F, int MODE, int TW, int TH>
static cudaError_t launch_one(const DevView& v, cudaStream_t s)
{
    const dim3 grid((unsigned)((v.tiles_x + kWarpsPerBlock - 1) / kWarpsPerBlock), (unsigned)v.tiles_y);
    if (grid.x == 0 || grid.y == 0) return cudaSuccess;
    k_render_view<KIND, F, MODE, TW, TH><<<grid, 32 * kWarpsPerBlock, 0, s>>>(v);
    return cudaGetLastError();
}

template <int KIND, int F, int MODE>
static cudaError_t launch_tiles(const DevView& v, cudaStream_t s)
{
    if (v.tile_w == 8 && v.tile_h == 4) return launch_one<KIND, F, MODE, 8, 4>(v, s);
    if (v.tile_w == 4 && v.tile_h == 8) return launch_one<KIND, F, MODE, 4, 8>(v, s);
    if (v.tile_w == 16 && v.tile_h == 2) return launch_one<KIND, F, MODE, 16, 2>(v, s);
    return cudaErrorInvalidValue;
}

template <int KIND, int F>
static cudaError_t launch_modes(const DevView& v, int mode, cudaStream_t s)
{
    switch (mode) {
    case 0: return launch_one<KIND, F, 0, 8, 4>(v, s);  // no sharing: tile shape irrelevant
    case 1: return launch_one<KIND, F, 1, 8, 4>(v, s);
    case 2: return launch_tiles<KIND, F, 2>(v, s);
    case 3: return launch_tiles<KIND, F, 3>(v, s);
    case 4: return launch_tiles<KIND, F, 4>(v, s);
    case 5: return launch_tiles<KIND, F, 5>(v, s);
    }
    return cudaErrorInvalidValue;
}

template <int KIND>
cudaError_t launch_view_kind(const DevView& v, int mode, cudaStream_t s)
{
    return v.filter == 0 ? launch_modes<KIND, 0>(v, mode, s) : launch_modes<KIND, 1>(v, mode, s);
}

// ------------------------------------------------------------------------------ multi-view

// One tile of any view of a batch: the view's filter and tile shape select the instance.
template <int KIND, int MODE>
__device__ __forceinline__ void render_tile_any(const DevView& v, int variant, int tx, int ty, int lane, float4* rec,
                                                float* wtab, unsigned char* scratch)
{
    if constexpr (MODE <= 1) {
        if (variant < 3) render_tile<KIND, 0, MODE, 8, 4>(v, tx, ty, lane, rec, wtab, scratch);
        else render_tile<KIND, 1, MODE, 8, 4>(v, tx, ty, lane, rec, wtab, scratch);
    } else {
        switch (variant) {
        case 0: render_tile<KIND, 0, MODE, 8, 4>(v, tx, ty, lane, rec, wtab, scratch); break;
        case 1: render_tile<KIND, 0, MODE, 4, 8>(v, tx, ty, lane, rec, wtab, scratch); break;
        case 2: render_tile<KIND, 0, MODE, 16, 2>(v, tx, ty, lane, rec, wtab, scratch); break;
        case 3: render_tile<KIND, 1, MODE, 8, 4>(v, tx, ty, lane, rec, wtab, scratch); break;
        case 4: render_tile<KIND, 1, MODE, 4, 8>(v, tx, ty, lane, rec, wtab, scratch); break;
        default: render_tile<KIND, 1, MODE, 16, 2>(v, tx, ty, lane, rec, wtab, scratch); break;
        }
    }
}

// Persistent multi-view kernel: each block pulls work items (a run of tiles of one view) from a
// device counter until the list is exhausted; the view's constants are staged in shared memory.
// Nothing waits on another block, so no wait can stall.
template <int KIND, int MODE>
__global__ void __launch_bounds__(256, MinBlocks<KIND>::n)
    k_render_batch(const DevView* __restrict__ views, const WorkItem* __restrict__ items, int n_items, int* counter)
{
    __shared__ float4 recs[kWarpsPerBlock * 32 * kRecPerLane];
    __shared__ float wtabs[kWarpsPerBlock * 32 * 8];
    __shared__ __align__(16) unsigned char scratch[kWarpsPerBlock * DecodeScratch<KIND>::bytes];
    __shared__ DevView sv;
    __shared__ WorkItem sw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            const int it = atomicAdd(counter, 1);
            sw = it < n_items ? items[it] : WorkItem{-1, 0, 0, 0};
        }
        __syncthreads();
        const WorkItem w = sw;
        if (w.view < 0) break;
        {
            const int* src = reinterpret_cast<const int*>(views + w.view);
            int* dst = reinterpret_cast<int*>(&sv);
            for (int i = threadIdx.x; i < (int)(sizeof(DevView) / 4); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        for (int t = w.tile0 + warp; t < w.tile0 + w.ntiles; t += kWarpsPerBlock) {
            const int ty = t / sv.tiles_x;
            render_tile_any<KIND, MODE>(sv, w.variant, t - ty * sv.tiles_x, ty, lane, recs + warp * 32 * kRecPerLane,
                                        wtabs + warp * 32 * 8, scratch + warp * DecodeScratch<KIND>::bytes);
        }
        __syncthreads();  // sv and sw are rewritten for the next item
    }
}

// grid > 0 launches; grid == 0 only reports the instance's resident blocks per SM in *per_sm.
template <int KIND, int MODE>
static cudaError_t launch_batch_mode(const DevView* views, const WorkItem* items, int n_items, int* counter, int grid,
                                     int* per_sm, cudaStream_t s)
{
    if (grid == 0) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_render_batch<KIND, MODE>, 256, 0);
    k_render_batch<KIND, MODE><<<grid, 256, 0, s>>>(views, items, n_items, counter);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_batch_kind(const DevView* views, const WorkItem* items, int n_items, int* counter, int grid, int mode,
                              int* per_sm, cudaStream_t s)
{
    switch (mode) {
    case 0: return launch_batch_mode<KIND, 0>(views, items, n_items, counter, grid, per_sm, s);
    case 1: return launch_batch_mode<KIND, 1>(views, items, n_items, counter, grid, per_sm, s);
    case 2: return launch_batch_mode<KIND, 2>(views, items, n_items, counter, grid, per_sm, s);
    case 3: return launch_batch_mode<KIND, 3>(views, items, n_items, counter, grid, per_sm, s);
    case 4: return launch_batch_mode<KIND, 4>(views, items, n_items, counter, grid, per_sm, s);
    case 5: return launch_batch_mode<KIND, 5>(views, items, n_items, counter, grid, per_sm, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace stf

#define STF_INSTANTIATE_KIND(KIND, NAME)                                                        \
    namespace stf {                                                                             \
    cudaError_t NAME(const DevView& v, int mode, cudaStream_t s) { return launch_view_kind<KIND>(v, mode, s); } \
    cudaError_t NAME##_batch(const DevView* views, const WorkItem* items, int n_items, int* counter, int grid, \
                             int mode, int* per_sm, cudaStream_t s)                             \
    {                                                                                           \
        return launch_batch_kind<KIND>(views, items, n_items, counter, grid, mode, per_sm, s); \
    }                                                                                           \
    }
