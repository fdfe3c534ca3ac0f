// Multi-view scheduler: work lists for the persistent kernel, CUDA-graph replay, autotuner.
//
// A batch of views is cut into work items (a run of 8 * schedule tiles of one view); items of
// the costliest views come first and every block of the persistent kernel pulls the next item
// from a device counter, so uneven views balance across the SMs. The view constants and the
// item list travel in one host-to-device copy from a pinned staging buffer; copy, counter reset
// and the kernels are captured once into a CUDA graph and replayed while the batch keeps its
// shape (its views may change: the copy reads the staging buffer at replay time).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <string_view>
#include <vector>

#include "stf.h"
#include "stf_internal.h"

using namespace stf;

namespace stf {
#define STF_DECLARE_BATCH(NAME)                                                                              \
    cudaError_t NAME##_batch(const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant, \
                             int* per_sm, cudaStream_t s);                                                     \
    cudaError_t NAME##_batch_views(const DevView* views, int n_views, int mode, cudaStream_t s);
STF_DECLARE_BATCH(launch_view_F32x4)
STF_DECLARE_BATCH(launch_view_F32x8)
STF_DECLARE_BATCH(launch_view_F16x4)
STF_DECLARE_BATCH(launch_view_F16x8)
STF_DECLARE_BATCH(launch_view_BF16x8)
STF_DECLARE_BATCH(launch_view_E4M3x8)
STF_DECLARE_BATCH(launch_view_U8x4_F16x2)
STF_DECLARE_BATCH(launch_view_NEURAL)
}  // namespace stf

namespace {

#define STF_KIND_SWITCH(CALL)                                      \
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

cudaError_t launch_batch(int kind, const WorkItem* items, int n_items, int* counter, int grid, int mode, int variant,
                         int* per_sm, cudaStream_t s)
{
    STF_KIND_SWITCH(batch(items, n_items, counter, grid, mode, variant, per_sm, s))
}

// The batch's view constants into the constant bank of the module whose kernels will run (mode
// selects the kind's blue-noise module or the plain one).
cudaError_t set_views(int kind, const DevView* views, int n_views, int mode, cudaStream_t s)
{
    STF_KIND_SWITCH(batch_views(views, n_views, mode, s))
}

// ------------------------------------------------------------------------------ view classes

constexpr int kDefaultSchedule = 2;  // tiles per warp per work item when untuned
const int kSchedules[4] = {1, 2, 4, 8};
const int kTiles[3][2] = {{8, 4}, {4, 8}, {16, 2}};

struct TuneEntry {
    int tile_w, tile_h, schedule;
    float ms;
};
std::map<std::string, TuneEntry, std::less<>> g_tune;  // transparent: lookups by string_view

// Area magnification at the view centre: pixels per texel, 1 / sqrt(|det d(texel) / d(pixel)|).
double view_magnification(const stf_view& v, const stf_texture* t)
{
    auto texel = [&](double x, double y, double* cx, double* cy) {
        const double hx = v.H[0] * x + v.H[1] * y + v.H[2];
        const double hy = v.H[3] * x + v.H[4] * y + v.H[5];
        const double hw = v.H[6] * x + v.H[7] * y + v.H[8];
        *cx = hx / hw * t->width;
        *cy = hy / hw * t->height;
    };
    const double x = v.width * 0.5, y = v.height * 0.5;
    double a0, b0, a1, b1, a2, b2;
    texel(x, y, &a0, &b0);
    texel(x + 1.0, y, &a1, &b1);
    texel(x, y + 1.0, &a2, &b2);
    const double det = std::fabs((a1 - a0) * (b2 - b0) - (a2 - a0) * (b1 - b0));
    return det > 0.0 && std::isfinite(det) ? 1.0 / std::sqrt(det) : 1.0;
}

std::string class_key(const stf_view& v, int filter, int mode)
{
    const double m = view_magnification(v, v.tex);
    const int mb = m < 2.0 ? 0 : (m < 8.0 ? 1 : (m < 32.0 ? 2 : 3));
    const long long px = (long long)v.width * v.height;
    const int rb = px < 500000 ? 0 : (px < 3000000 ? 1 : 2);
    char buf[96];
    snprintf(buf, sizeof buf, "kind%d/filter%d/mode%d/mag%d/res%d", v.tex->kind, filter, mode, mb, rb);
    return buf;
}

int view_filter(const stf_view& v, int filter) { return filter == STF_FILTER_PER_VIEW ? v.filter : filter; }

// Tile shape and schedule a view is rendered with: its own tile if given, else the tuned one of
// its class, else 8x4; the schedule is the tuned one, else the default.
void resolve(const stf_view& v, int filter, int mode, int* tw, int* th, int* sched)
{
    const auto it = g_tune.find(class_key(v, view_filter(v, filter), mode));
    *sched = it != g_tune.end() ? it->second.schedule : kDefaultSchedule;
    if (v.tile_w) { *tw = v.tile_w; *th = v.tile_h; }
    else if (it != g_tune.end()) { *tw = it->second.tile_w; *th = it->second.tile_h; }
    else { *tw = 8; *th = 4; }
    if ((mode & kModeBase) <= STF_MODE_ONE_TAP || ((mode >> STF_MODE_EST_SHIFT) & 7)) { *tw = 8; *th = 4; }
    if ((mode & kModeBase) == STF_MODE_SPARSE9) stf_sparse_state(nullptr, nullptr, tw, th);
}

int tile_code(int tw, int th) { return tw == 8 ? 0 : (tw == 4 ? 1 : 2); }

// ------------------------------------------------------------------------------ batches

struct Sub {  // the items of one (filter, tile shape) variant within a group
    int variant;
    std::vector<WorkItem> items;
    size_t items_off;
    int grid, counter;
};

struct Group {  // views of one material kind, at most kBatchMaxViews, costliest first
    int kind;
    std::vector<int> views;
    std::vector<Sub> subs;
    size_t views_off;
};

constexpr int kBranches = 6;  // concurrent variant kernels of a group

struct BatchState {
    int device = -1;
    cudaStream_t cap = nullptr;
    cudaStream_t branch[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    unsigned char* host[2] = {nullptr, nullptr};  // pinned staging
    unsigned char* dev[2] = {nullptr, nullptr};
    int* counters[2] = {nullptr, nullptr};
    size_t cap_bytes = 0;
    int cap_counters = 0;
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::string shape[2];
    int next = 0;
    long long graph_builds = 0, graph_replays = 0;
};
BatchState g_batch;

int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

stf_status ensure_buffers(size_t bytes, int counters)
{
    BatchState& b = g_batch;
    int dev = 0;
    cudaGetDevice(&dev);
    if (b.device != dev && b.device >= 0) return stf_fail(STF_ERR_UNSUPPORTED, "multi-view batches on a second device");
    b.device = dev;
    cudaError_t e;
    if (!b.cap && (e = cudaStreamCreateWithFlags(&b.cap, cudaStreamNonBlocking)) != cudaSuccess)
        return stf_cuda_fail(e, "capture stream");
    for (int i = 0; i < kBranches; ++i) {
        if (!b.branch[i] && (e = cudaStreamCreateWithFlags(&b.branch[i], cudaStreamNonBlocking)) != cudaSuccess)
            return stf_cuda_fail(e, "branch stream");
        if (!b.join[i] && (e = cudaEventCreateWithFlags(&b.join[i], cudaEventDisableTiming)) != cudaSuccess)
            return stf_cuda_fail(e, "event");
    }
    if (!b.fork && (e = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming)) != cudaSuccess)
        return stf_cuda_fail(e, "event");
    for (int k = 0; k < 2; ++k)
        if (!b.done[k] && (e = cudaEventCreateWithFlags(&b.done[k], cudaEventDisableTiming)) != cudaSuccess)
            return stf_cuda_fail(e, "event");
    if (bytes <= b.cap_bytes && counters <= b.cap_counters) return STF_OK;
    for (int k = 0; k < 2; ++k) {
        if (b.used[k]) cudaEventSynchronize(b.done[k]);
        if (b.host[k]) cudaFreeHost(b.host[k]);
        if (b.dev[k]) cudaFree(b.dev[k]);
        if (b.counters[k]) cudaFree(b.counters[k]);
        if (b.exec[k]) cudaGraphExecDestroy(b.exec[k]);
        b.host[k] = nullptr; b.dev[k] = nullptr; b.counters[k] = nullptr; b.exec[k] = nullptr;
        b.shape[k].clear();
        b.used[k] = false;
    }
    b.cap_bytes = 0;
    const size_t nb = std::max(bytes * 2, (size_t)65536);
    const int nc = std::max(counters * 2, 64);
    for (int k = 0; k < 2; ++k) {
        if ((e = cudaMallocHost(&b.host[k], nb)) != cudaSuccess || (e = cudaMalloc(&b.dev[k], nb)) != cudaSuccess ||
            (e = cudaMalloc(&b.counters[k], nc * sizeof(int))) != cudaSuccess)
            return stf_cuda_fail(e, "batch buffers");
    }
    b.cap_bytes = nb;
    b.cap_counters = nc;
    return STF_OK;
}

// Views grouped by material kind (at most kBatchMaxViews per group), costliest first; items cut
// per view and collected per variant.
void build_groups(const stf_view* views, int n, int filter, int mode, std::vector<Group>& groups)
{
    // one group per material kind and, for neural textures, per decoder: a neural group's kernels
    // stage one decoder's weights in shared memory
    std::map<std::pair<int, const void*>, int> gi;
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) {
        const int f = view_filter(views[i], filter);
        cost[i] = (double)views[i].width * views[i].height * (f == STF_FILTER_BSPLINE3 ? 1.5 : 1.0);
        const int k = views[i].tex->kind;
        const std::pair<int, const void*> key{k, k == K_NEURAL ? (const void*)views[i].tex->decoder : nullptr};
        auto it = gi.find(key);
        if (it == gi.end() || (int)groups[it->second].views.size() == kBatchMaxViews) {
            gi[key] = (int)groups.size();
            groups.push_back(Group{k, {}, {}, 0});
        }
        groups[gi[key]].views.push_back(i);
    }
    for (Group& g : groups) {
        std::stable_sort(g.views.begin(), g.views.end(), [&](int a, int b) { return cost[a] > cost[b]; });
        for (int local = 0; local < (int)g.views.size(); ++local) {
            const stf_view& v = views[g.views[local]];
            int tw, th, sc;
            resolve(v, filter, mode, &tw, &th, &sc);
            const int tiles = ((v.width + tw - 1) / tw) * ((v.height + th - 1) / th);
            const int per = kWarpsPerBlock * sc;
            const int f = view_filter(v, filter);
            const bool ex = (mode & STF_MODE_FLAG_EXACT) && f == STF_FILTER_BILINEAR;
            const int variant = ex ? 6 + tile_code(tw, th) : f * 3 + tile_code(tw, th);
            Sub* sub = nullptr;
            for (Sub& x : g.subs)
                if (x.variant == variant) sub = &x;
            if (!sub) {
                g.subs.push_back(Sub{variant, {}, 0, 0, 0});
                sub = &g.subs.back();
            }
            for (int t0 = 0; t0 < tiles; t0 += per) sub->items.push_back(WorkItem{local, t0, std::min(per, tiles - t0), variant});
        }
    }
}

stf_status render_batch_impl(const stf_view* views, int n, int filter, int mode, unsigned long long seed, bool use_graph)
{
    const float* lut = nullptr;
    stf_status st = stf_device_state(nullptr, &lut);
    if (st != STF_OK) return st;
    std::vector<Group> groups;
    build_groups(views, n, filter, mode, groups);
    // staging layout: per group [DevView x views] then [WorkItem x items] per variant, 256-byte aligned
    size_t off = 0;
    int ncounters = 0;
    std::string shape = "m" + std::to_string(mode);
    for (Group& g : groups) {
        g.views_off = off;
        off += ((g.views.size() * sizeof(DevView) + 255) / 256) * 256;
        shape += "|k" + std::to_string(g.kind) + "v" + std::to_string(g.views.size());
        for (Sub& sub : g.subs) {
            sub.items_off = off;
            off += ((sub.items.size() * sizeof(WorkItem) + 255) / 256) * 256;
            int per_sm = 0;
            cudaError_t e = launch_batch(g.kind, nullptr, 0, nullptr, 0, mode, sub.variant, &per_sm, nullptr);
            if (e != cudaSuccess) return stf_cuda_fail(e, "occupancy query");
            sub.grid = (int)std::min<long long>((long long)std::max(1, std::min(per_sm, 8)) * sm_count(),
                                                (long long)sub.items.size());
            sub.counter = ncounters++;
            shape += "/x" + std::to_string(sub.variant) + "i" + std::to_string(sub.items.size()) + "g" +
                     std::to_string(sub.grid);
        }
    }
    if ((st = ensure_buffers(off, ncounters)) != STF_OK) return st;
    BatchState& b = g_batch;
    const int k = b.next;
    b.next ^= 1;
    if (b.used[k]) {
        cudaError_t e = cudaEventSynchronize(b.done[k]);  // the copy that last read this staging buffer
        if (e != cudaSuccess) return stf_cuda_fail(e, "staging reuse");
    }
    for (const Group& g : groups) {
        DevView* dv = reinterpret_cast<DevView*>(b.host[k] + g.views_off);
        for (size_t i = 0; i < g.views.size(); ++i) {
            const stf_view& v = views[g.views[i]];
            stf_fill_devview(v, filter, mode, seed, lut, dv[i]);
            int tw, th, sc;
            resolve(v, filter, mode, &tw, &th, &sc);  // the tile shape the items were cut for
            dv[i].tile_w = tw;
            dv[i].tile_h = th;
            dv[i].tiles_x = (dv[i].width + tw - 1) / tw;
            dv[i].tiles_y = (dv[i].height + th - 1) / th;
        }
        for (const Sub& sub : g.subs)
            memcpy(b.host[k] + sub.items_off, sub.items.data(), sub.items.size() * sizeof(WorkItem));
    }
    cudaStream_t user = stf_stream();
    cudaError_t e;
    // copy, counter reset, then per group: its views into the kind's constant bank and its variant
    // kernels as concurrent branches (a variant's tail overlaps the next one's start)
    auto enqueue = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(b.dev[k], b.host[k], off, cudaMemcpyHostToDevice, s);
        if (r == cudaSuccess) r = cudaMemsetAsync(b.counters[k], 0, ncounters * sizeof(int), s);
        for (size_t gi = 0; gi < groups.size() && r == cudaSuccess; ++gi) {
            const Group& g = groups[gi];
            r = set_views(g.kind, reinterpret_cast<const DevView*>(b.dev[k] + g.views_off), (int)g.views.size(), mode, s);
            if (r == cudaSuccess) r = cudaEventRecord(b.fork, s);
            for (size_t j = 0; j < g.subs.size() && r == cudaSuccess; ++j) {
                const Sub& sub = g.subs[j];
                cudaStream_t bs = b.branch[j % kBranches];
                int unused = 0;
                r = cudaStreamWaitEvent(bs, b.fork, 0);
                if (r == cudaSuccess)
                    r = launch_batch(g.kind, reinterpret_cast<const WorkItem*>(b.dev[k] + sub.items_off), (int)sub.items.size(),
                                     b.counters[k] + sub.counter, sub.grid, mode, sub.variant, &unused, bs);
                if (r == cudaSuccess) r = cudaEventRecord(b.join[j % kBranches], bs);
                if (r == cudaSuccess) r = cudaStreamWaitEvent(s, b.join[j % kBranches], 0);
            }
        }
        return r;
    };
    if (!use_graph) {
        if ((e = enqueue(user)) != cudaSuccess) return stf_cuda_fail(e, "batch launch");
    } else {
        if (b.shape[k] != shape || !b.exec[k]) {
            if (b.exec[k]) { cudaGraphExecDestroy(b.exec[k]); b.exec[k] = nullptr; }
            cudaGraph_t graph = nullptr;
            if ((e = cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return stf_cuda_fail(e, "begin capture");
            const cudaError_t r = enqueue(b.cap);
            e = cudaStreamEndCapture(b.cap, &graph);
            if (r != cudaSuccess) { if (graph) cudaGraphDestroy(graph); return stf_cuda_fail(r, "capture"); }
            if (e != cudaSuccess) return stf_cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&b.exec[k], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) { b.exec[k] = nullptr; return stf_cuda_fail(e, "graph instantiate"); }
            b.shape[k] = shape;
            ++b.graph_builds;
        } else {
            ++b.graph_replays;
        }
        if ((e = cudaGraphLaunch(b.exec[k], user)) != cudaSuccess) return stf_cuda_fail(e, "graph launch");
    }
    if ((e = cudaEventRecord(b.done[k], user)) != cudaSuccess) return stf_cuda_fail(e, "event record");
    b.used[k] = true;
    return STF_OK;
}

int g_use_graphs = 1;

}  // namespace

int g_pipeline_blocks = 0;  // STF_OPT_PIPELINE_BLOCKS
int g_paired_pixels = 1;    // STF_OPT_PAIRED_PIXELS
int g_tma_stage = 0;        // STF_OPT_TMA_STAGE

// The same resolution as `resolve`, with the class key built in a stack buffer (no heap use).
void stf_resolve_view_config_nohalloc(const stf_view& v, int filter, int mode, int* tw, int* th, int* sched)
{
    const int f = view_filter(v, filter);
    const double m = view_magnification(v, v.tex);
    const int mb = m < 2.0 ? 0 : (m < 8.0 ? 1 : (m < 32.0 ? 2 : 3));
    const long long px = (long long)v.width * v.height;
    const int rb = px < 500000 ? 0 : (px < 3000000 ? 1 : 2);
    char buf[96];
    const int len = snprintf(buf, sizeof buf, "kind%d/filter%d/mode%d/mag%d/res%d", v.tex->kind, f, mode, mb, rb);
    const auto it = g_tune.find(std::string_view(buf, (size_t)len));
    *sched = it != g_tune.end() ? it->second.schedule : kDefaultSchedule;
    if (v.tile_w) { *tw = v.tile_w; *th = v.tile_h; }
    else if (it != g_tune.end()) { *tw = it->second.tile_w; *th = it->second.tile_h; }
    else { *tw = 8; *th = 4; }
    if ((mode & kModeBase) <= STF_MODE_ONE_TAP || ((mode >> STF_MODE_EST_SHIFT) & 7)) { *tw = 8; *th = 4; }
    if ((mode & kModeBase) == STF_MODE_SPARSE9) stf_sparse_state(nullptr, nullptr, tw, th);
}

stf_status stf_render_batch(const stf_view* views, int n, int filter, int mode, unsigned long long seed)
{
    return render_batch_impl(views, n, filter, mode, seed, g_use_graphs != 0);
}

extern "C" stf_status stf_set_option(int option, long long value)
{
    switch (option) {
    case STF_OPT_BATCH_GRAPHS: g_use_graphs = value != 0; return STF_OK;
    case STF_OPT_PAIRED_PIXELS: g_paired_pixels = value != 0; return STF_OK;
    case STF_OPT_TMA_STAGE: g_tma_stage = value != 0; return STF_OK;
    case STF_OPT_PIPELINE_BLOCKS:
        if (value < 0 || value > (1 << 20)) return stf_fail(STF_ERR_INVALID_ARG, "pipeline blocks %lld", value);
        g_pipeline_blocks = (int)value;
        return STF_OK;
    case STF_OPT_TEST_DECODE_STALL: {
        // flags[2] is read by the MMA warp of each decode pipeline; stf_sync clears all flags
        int* flags = nullptr;
        stf_status st = stf_device_state(&flags, nullptr);
        if (st != STF_OK) return st;
        const int v = value != 0;
        cudaError_t e = cudaMemcpy(flags + 2, &v, sizeof v, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "test stall switch");
    }
    }
    return stf_fail(STF_ERR_INVALID_ARG, "unknown option %d", option);
}

extern "C" stf_status stf_get_stat(int stat, long long* value)
{
    if (!value) return stf_fail(STF_ERR_INVALID_ARG, "null value");
    switch (stat) {
    case STF_STAT_GRAPH_BUILDS: *value = g_batch.graph_builds; return STF_OK;
    case STF_STAT_GRAPH_REPLAYS: *value = g_batch.graph_replays; return STF_OK;
    }
    return stf_fail(STF_ERR_INVALID_ARG, "unknown statistic %d", stat);
}

// ------------------------------------------------------------------------------ autotuner

extern "C" stf_status stf_view_config(const stf_view* view, int filter, int reuse_mode, int* tile_w, int* tile_h,
                                      int* schedule)
{
    if (!view || !view->tex) return stf_fail(STF_ERR_INVALID_ARG, "stf_view_config: null view or texture");
    int tw, th, sc;
    resolve(*view, filter, reuse_mode, &tw, &th, &sc);
    if (tile_w) *tile_w = tw;
    if (tile_h) *tile_h = th;
    if (schedule) *schedule = sc;
    return STF_OK;
}

extern "C" stf_status stf_autotune(const stf_view* views, int n, int filter, int reuse_mode, unsigned long long seed)
{
    if (!views || n < 1) return stf_fail(STF_ERR_INVALID_ARG, "stf_autotune: need n >= 1 views");
    if (stf_check_mode(reuse_mode) != STF_OK) return STF_ERR_INVALID_ARG;
    if ((reuse_mode >> STF_MODE_EST_SHIFT) & 7)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_autotune: the weighted estimator only");
    for (int i = 0; i < n; ++i) {
        stf_status s = stf_validate_view(views[i], i, filter, reuse_mode);
        if (s != STF_OK) return s;
    }
    // one representative (the largest view) per class
    std::map<std::string, int> rep;
    for (int i = 0; i < n; ++i) {
        const std::string key = class_key(views[i], view_filter(views[i], filter), reuse_mode);
        const auto it = rep.find(key);
        if (it == rep.end() || (long long)views[i].width * views[i].height >
                                   (long long)views[it->second].width * views[it->second].height)
            rep[key] = i;
    }
    cudaStream_t s = stf_stream();
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool shares = (reuse_mode & kModeBase) >= STF_MODE_QUAD2;
    stf_status st = STF_OK;
    for (const auto& kv : rep) {
        TuneEntry best{8, 4, kDefaultSchedule, 1e30f};
        for (int ti = 0; ti < (shares ? 3 : 1) && st == STF_OK; ++ti) {
            for (int si = 0; si < 4 && st == STF_OK; ++si) {
                g_tune[kv.first] = TuneEntry{kTiles[ti][0], kTiles[ti][1], kSchedules[si], 0.0f};
                stf_view v = views[kv.second];
                v.tile_w = 0;
                v.tile_h = 0;
                float ms_best = 1e30f;
                for (int rep_i = 0; rep_i < 4 && st == STF_OK; ++rep_i) {
                    cudaEventRecord(e0, s);
                    st = render_batch_impl(&v, 1, filter, reuse_mode, seed, false);
                    cudaEventRecord(e1, s);
                    cudaError_t e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) st = stf_cuda_fail(e, "autotune timing");
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep_i > 0) ms_best = std::min(ms_best, ms);  // the first run warms up
                }
                if (ms_best < best.ms) best = TuneEntry{kTiles[ti][0], kTiles[ti][1], kSchedules[si], ms_best};
            }
        }
        g_tune[kv.first] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STF_OK) {
        for (const auto& kv : rep) g_tune.erase(kv.first);
        return st;
    }
    return STF_OK;
}

extern "C" stf_status stf_autotune_save(const char* path)
{
    if (!path) return stf_fail(STF_ERR_INVALID_ARG, "null path");
    FILE* f = fopen(path, "w");
    if (!f) return stf_fail(STF_ERR_INVALID_ARG, "cannot open %s", path);
    cudaDeviceProp p;
    int dev = 0;
    cudaGetDevice(&dev);
    const bool have = cudaGetDeviceProperties(&p, dev) == cudaSuccess;
    fprintf(f, "# stf autotune v1 gpu=%s\n", have ? p.name : "unknown");
    for (const auto& kv : g_tune)
        fprintf(f, "%s %d %d %d %.6f\n", kv.first.c_str(), kv.second.tile_w, kv.second.tile_h, kv.second.schedule, kv.second.ms);
    fclose(f);
    return STF_OK;
}

extern "C" stf_status stf_autotune_load(const char* path)
{
    if (!path) return stf_fail(STF_ERR_INVALID_ARG, "null path");
    FILE* f = fopen(path, "r");
    if (!f) return stf_fail(STF_ERR_INVALID_ARG, "cannot open %s", path);
    char line[256];
    std::map<std::string, TuneEntry> tab;
    bool header = false;
    while (fgets(line, sizeof line, f)) {
        if (line[0] == '#') { header = header || strstr(line, "stf autotune v1") != nullptr; continue; }
        char key[128];
        TuneEntry t;
        if (sscanf(line, "%127s %d %d %d %f", key, &t.tile_w, &t.tile_h, &t.schedule, &t.ms) != 5) continue;
        const bool tile_ok = (t.tile_w == 8 && t.tile_h == 4) || (t.tile_w == 4 && t.tile_h == 8) || (t.tile_w == 16 && t.tile_h == 2);
        if (!tile_ok || t.schedule < 1 || t.schedule > 64) { fclose(f); return stf_fail(STF_ERR_INVALID_ARG, "bad entry in %s", path); }
        tab[key] = t;
    }
    fclose(f);
    if (!header) return stf_fail(STF_ERR_INVALID_ARG, "%s is not an autotune table", path);
    for (const auto& kv : tab) g_tune[kv.first] = kv.second;
    return STF_OK;
}

extern "C" stf_status stf_autotune_clear(void)
{
    g_tune.clear();
    return STF_OK;
}
