// Multi-view rendering without any allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: a render thread that owns a fixed device
// memory budget carved out up front, or a frame loop that must not stall, since cudaMalloc and
// cudaFree may synchronise the whole device and can fail under fragmentation mid-frame. For them,
// stf_render_views_noalloc renders a batch with the same persistent kernel as stf_render_views,
// but its scratch (the view constants, the work items, the work-queue counters and the UNORM8
// table) lives in one file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits. It allocates no host heap memory either: the host-side
// lists are built in a static buffer.
//
// In host code the array's name only stands in for the device symbol; its device address is
// looked up once per device with cudaGetSymbolAddress (the first call on a device does this
// set-up and a blocking copy of the UNORM8 table, so make that first call before any stream
// capture). All calls share the array and it keeps the last call's contents: the counters are
// cleared on every call, and calls that overlap on the GPU (different streams, or the same
// stream from different threads) race on it. The library's per-device error flags, which the
// kernels report bounded-wait timeouts through, are set up by stf_create_texture; a call on a
// device where no texture was created is refused rather than allocating them. The host-side
// staging is static too: a lock (no allocation) serialises calls from several host threads over
// its fill, upload and launches, so one call's item list is never paired with another's views.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <mutex>

#include "stf.h"
#include "stf_internal.h"

using namespace stf;

namespace stf {
#define STF_DECLARE_BATCH_NA(NAME)                                                                           \
    cudaError_t NAME##_batch(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant, \
                             int* per_sm, cudaStream_t s);                                                     \
    cudaError_t NAME##_batch_views(const DevView* views, int n_views, int mode, cudaStream_t s);
STF_DECLARE_BATCH_NA(launch_view_F32x4)
STF_DECLARE_BATCH_NA(launch_view_F32x8)
STF_DECLARE_BATCH_NA(launch_view_F16x4)
STF_DECLARE_BATCH_NA(launch_view_F16x8)
STF_DECLARE_BATCH_NA(launch_view_BF16x8)
STF_DECLARE_BATCH_NA(launch_view_E4M3x8)
STF_DECLARE_BATCH_NA(launch_view_U8x4_F16x2)
STF_DECLARE_BATCH_NA(launch_view_NEURAL)
}  // namespace stf

namespace {

constexpr int kVariants = 9;  // filter * 3 + tile, 6 + tile for bilinear with exact filtering

struct NoallocScratch {
    DevView views[STF_NOALLOC_MAX_VIEWS];
    WorkItem items[STF_NOALLOC_MAX_ITEMS];
    float unorm_lut[256];
    int counters[K_COUNT * kVariants];
};
static_assert(STF_NOALLOC_MAX_VIEWS <= kBatchMaxViews, "one persistent launch per material kind");

// The scratch, one copy per device that loads the library.
__device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoallocScratch)];

constexpr int kMaxDevices = 64;
NoallocScratch* g_dev_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device
NoallocScratch g_stage;                  // host-side lists (static: no heap use)
int g_order[STF_NOALLOC_MAX_VIEWS];
std::mutex g_stage_lock;                 // guards g_stage, g_order and g_dev_ptr

#define STF_KIND_SWITCH_NA(CALL)                                   \
    switch (kind) {                                                \
    case K_F32x4: return launch_view_F32x4_##CALL;                 \
    case K_F32x8: return launch_view_F32x8_##CALL;                 \
    case K_F16x4: return launch_view_F16x4_##CALL;                 \
    case K_F16x8: return launch_view_F16x8_##CALL;                 \
    case K_BF16x8: return launch_view_BF16x8_##CALL;               \
    case K_E4M3x8: return launch_view_E4M3x8_##CALL;               \
    case K_U8x4_F16x2: return launch_view_U8x4_F16x2_##CALL;       \
    case K_NEURAL: return launch_view_NEURAL_##CALL;               \
    }                                                              \
    return cudaErrorInvalidValue;

cudaError_t launch_batch_na(int kind, const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant,
                            int* per_sm, cudaStream_t s)
{
    STF_KIND_SWITCH_NA(batch(items, n_items, counter, grid, mode, variant, per_sm, s))
}

cudaError_t set_views_na(int kind, const DevView* views, int n_views, int mode, cudaStream_t s)
{
    STF_KIND_SWITCH_NA(batch_views(views, n_views, mode, s))
}

// Once per device, with that device current: the scratch's device address and its UNORM8 table.
// Also returns the device's error flags, which must exist already (nothing is allocated here).
stf_status setup(NoallocScratch** out, int** flags)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return stf_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return stf_fail(STF_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    stf_status st = stf_device_state_ready(flags);
    if (st != STF_OK) return st;
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return stf_cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        for (int q = 0; q < 256; ++q) g_stage.unorm_lut[q] = (float)q / 255.0f;
        NoallocScratch* d = static_cast<NoallocScratch*>(p);
        e = cudaMemcpy(d->unorm_lut, g_stage.unorm_lut, sizeof g_stage.unorm_lut, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return stf_cuda_fail(e, "no-alloc scratch set-up");
        g_dev_ptr[dev] = d;
    }
    *out = g_dev_ptr[dev];
    return STF_OK;
}

int sm_count_na()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

extern "C" stf_status stf_render_views_noalloc(const stf_view* views, int n, int filter, int reuse_mode,
                                               unsigned long long seed)
{
    if (!views || n < 1) return stf_fail(STF_ERR_INVALID_ARG, "stf_render_views_noalloc: need n >= 1 views");
    if (n > STF_NOALLOC_MAX_VIEWS)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_render_views_noalloc: %d views exceed the fixed scratch limit of %d",
                        n, STF_NOALLOC_MAX_VIEWS);
    if (filter != STF_FILTER_BILINEAR && filter != STF_FILTER_BSPLINE3 && filter != STF_FILTER_PER_VIEW)
        return stf_fail(STF_ERR_INVALID_ARG, "filter %d", filter);
    if (stf_check_mode(reuse_mode) != STF_OK) return STF_ERR_INVALID_ARG;
    if ((reuse_mode >> STF_MODE_EST_SHIFT) & 7)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_render_views_noalloc: the weighted estimator only");
    for (int i = 0; i < n; ++i) {
        stf_status s = stf_validate_view(views[i], i, filter, reuse_mode);
        if (s != STF_OK) return s;
    }
    // one persistent launch per material kind: neural views must share a decoder (its weights are
    // staged once per block)
    const void* decoder = nullptr;
    for (int i = 0; i < n; ++i) {
        if (views[i].tex->kind != K_NEURAL) continue;
        if (decoder && views[i].tex->decoder != decoder)
            return stf_fail(STF_ERR_INVALID_ARG, "stf_render_views_noalloc: view %d uses a second neural decoder", i);
        decoder = views[i].tex->decoder;
    }
    std::lock_guard<std::mutex> hold(g_stage_lock);
    NoallocScratch* dev = nullptr;
    int* flags = nullptr;
    stf_status st = setup(&dev, &flags);
    if (st != STF_OK) return st;
    const float* lut = dev->unorm_lut;

    // views grouped by material kind, each group costliest first (the order stf_render_views uses)
    int group_start[K_COUNT + 1], total_tiles[STF_NOALLOC_MAX_VIEWS];
    int tw[STF_NOALLOC_MAX_VIEWS], th[STF_NOALLOC_MAX_VIEWS], sc[STF_NOALLOC_MAX_VIEWS];
    double cost[STF_NOALLOC_MAX_VIEWS];
    for (int i = 0; i < n; ++i) {
        stf_resolve_view_config_nohalloc(views[i], filter, reuse_mode, &tw[i], &th[i], &sc[i]);
        total_tiles[i] = ((views[i].width + tw[i] - 1) / tw[i]) * ((views[i].height + th[i] - 1) / th[i]);
        const int f = filter == STF_FILTER_PER_VIEW ? views[i].filter : filter;
        cost[i] = (double)views[i].width * views[i].height * (f == STF_FILTER_BSPLINE3 ? 1.5 : 1.0);
    }
    // work items hold whole runs of 8 * schedule tiles; coarsen them evenly if the list would not
    // fit (the split does not change any pixel)
    long long coarsen = 1;
    for (;;) {
        long long items = 0;
        for (int i = 0; i < n; ++i) {
            const long long per = (long long)kWarpsPerBlock * sc[i] * coarsen;
            items += (total_tiles[i] + per - 1) / per;
        }
        if (items <= STF_NOALLOC_MAX_ITEMS) break;
        coarsen *= 2;
    }
    int nv = 0, ni = 0;
    int var_of[STF_NOALLOC_MAX_VIEWS];
    int sub_start[K_COUNT][kVariants + 1];
    group_start[0] = 0;
    for (int k = 0; k < K_COUNT; ++k) {
        const int v0 = nv;
        for (int i = 0; i < n; ++i)
            if (views[i].tex->kind == k) g_order[nv++] = i;
        for (int a = v0 + 1; a < nv; ++a) {  // stable insertion sort by decreasing cost
            const int x = g_order[a];
            int b = a - 1;
            while (b >= v0 && cost[g_order[b]] < cost[x]) { g_order[b + 1] = g_order[b]; --b; }
            g_order[b + 1] = x;
        }
        for (int j = v0; j < nv; ++j) {
            const int i = g_order[j];
            DevView& d = g_stage.views[j];
            stf_fill_devview(views[i], filter, reuse_mode, seed, lut, d);
            d.flags = flags;
            d.tile_w = tw[i];
            d.tile_h = th[i];
            d.tiles_x = (d.width + tw[i] - 1) / tw[i];
            d.tiles_y = (d.height + th[i] - 1) / th[i];
            const int f = filter == STF_FILTER_PER_VIEW ? views[i].filter : filter;
            const int tc = tw[i] == 8 ? 0 : (tw[i] == 4 ? 1 : 2);
            var_of[j] = (reuse_mode & STF_MODE_FLAG_EXACT) && f == STF_FILTER_BILINEAR ? 6 + tc : f * 3 + tc;
        }
        // items of the group, contiguous per variant (one persistent kernel per variant)
        for (int var = 0; var < kVariants; ++var) {
            sub_start[k][var] = ni;
            for (int j = v0; j < nv; ++j) {
                if (var_of[j] != var) continue;
                const int i = g_order[j];
                const int per = (int)((long long)kWarpsPerBlock * sc[i] * coarsen);
                for (int t0 = 0; t0 < total_tiles[i]; t0 += per)
                    g_stage.items[ni++] = WorkItem{j - v0, t0, total_tiles[i] - t0 < per ? total_tiles[i] - t0 : per, var};
            }
        }
        sub_start[k][kVariants] = ni;
        group_start[k + 1] = nv;
    }

    cudaStream_t s = stf_stream();
    cudaError_t e = cudaMemcpyAsync(dev->views, g_stage.views, (size_t)n * sizeof(DevView), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev->items, g_stage.items, (size_t)ni * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev->counters, 0, sizeof dev->counters, s);
    if (e != cudaSuccess) return stf_cuda_fail(e, "no-alloc batch upload");
    for (int k = 0; k < K_COUNT; ++k) {
        const int nvk = group_start[k + 1] - group_start[k];
        if (nvk == 0) continue;
        e = set_views_na(k, dev->views + group_start[k], nvk, reuse_mode, s);
        if (e != cudaSuccess) return stf_cuda_fail(e, "no-alloc view upload");
        for (int var = 0; var < kVariants; ++var) {
            const int nitems = sub_start[k][var + 1] - sub_start[k][var];
            if (nitems == 0) continue;
            int per_sm = 0;
            e = launch_batch_na(k, nullptr, 0, nullptr, 0, reuse_mode, var, &per_sm, s);
            if (e != cudaSuccess) return stf_cuda_fail(e, "occupancy query");
            int grid = (per_sm < 1 ? 1 : (per_sm > 8 ? 8 : per_sm)) * sm_count_na();
            if (grid > nitems) grid = nitems;
            e = launch_batch_na(k, dev->items + sub_start[k][var], nitems, dev->counters + k * kVariants + var, grid,
                                reuse_mode, var, &per_sm, s);
            if (e != cudaSuccess) return stf_cuda_fail(e, "no-alloc batch launch");
        }
    }
    return STF_OK;
}
