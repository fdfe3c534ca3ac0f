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

}  // namespace stf

#define STF_INSTANTIATE_KIND(KIND, NAME)                                                        \
    namespace stf {                                                                             \
    cudaError_t NAME(const DevView& v, int mode, cudaStream_t s) { return launch_view_kind<KIND>(v, mode, s); } \
    }
