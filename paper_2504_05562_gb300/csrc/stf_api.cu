// C interface of the STF library: argument validation, texture creation and relayout, and
// dispatch of the render kernels. Declarations and the contract are in include/stf.h.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "stf.h"
#include "stf_device.cuh"
#include "stf_internal.h"

using namespace stf;

// ------------------------------------------------------------------------------ errors

static thread_local std::string g_err;
static cudaStream_t g_stream = nullptr;

stf_status stf_fail(stf_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

stf_status stf_cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return stf_fail(STF_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    return stf_fail(STF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaStream_t stf_stream() { return g_stream; }

extern "C" const char* stf_last_error(void) { return g_err.c_str(); }
extern "C" int stf_version(void) { return 10000; }

extern "C" stf_status stf_set_stream(void* s)
{
    g_stream = (cudaStream_t)s;
    return STF_OK;
}

// ------------------------------------------------------------------------------ occupancy

// Resident blocks per SM of a kernel, counted from its registers, shared memory and threads (and
// at most four, the blocks whose 128 tensor-memory columns fit in an SM's 512). The runtime's
// occupancy query reports one block for kernels that allocate tensor memory, which would leave
// the persistent decode-pipeline grids at half the SMs' capacity.
cudaError_t stf_resident_blocks(const void* kernel, int threads, int dyn_bytes, int* n)
{
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, reserved = 0;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, kernel)) != cudaSuccess || (e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess)
        return e;
    const int warps = (threads + 31) / 32;
    const int regs_block = warps * ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in 256s
    const int smem_block = (int)fa.sharedSizeBytes + dyn_bytes + reserved;
    int b = regs_block > 0 ? regs_sm / regs_block : 1;
    b = std::min(b, smem_sm / std::max(smem_block, 1));
    b = std::min(b, thr_sm / std::max(threads, 1));
    *n = std::max(1, std::min(b, 4));
    return cudaSuccess;
}

// ------------------------------------------------------------------------------ per-device state

static bool tile_ok(int tw, int th);

struct DeviceState {
    bool ready = false;
    float* unorm_lut = nullptr;  // q / 255 for q = 0..255, computed on the host in IEEE FP32
    int* flags = nullptr;        // [0] timeout, [1] device assert
    uint8_t* fp = nullptr;       // sparse footprint patterns [fp_patterns][32][16] (STF_MODE_SPARSE9)
    int fp_patterns = 0, fp_capacity = 0, fp_tw = 0, fp_th = 0;
    uint16_t* blue = nullptr;    // blue-noise ranks [2][n][n] (STF_MODE_FLAG_BLUE_NOISE)
    int blue_shift = 0, blue_capacity = 0;
};
static DeviceState g_dev[64];

static DeviceState* current_state()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &g_dev[dev];
}

// The current device's sparse footprints: false if none were set.
bool stf_sparse_state(const uint8_t** table, int* patterns, int* tile_w, int* tile_h)
{
    const DeviceState* d = current_state();
    if (!d || !d->fp || d->fp_patterns < 1) return false;
    if (table) *table = d->fp;
    if (patterns) *patterns = d->fp_patterns;
    if (tile_w) *tile_w = d->fp_tw;
    if (tile_h) *tile_h = d->fp_th;
    return true;
}

// The current device's blue-noise masks: false if none were set.
bool stf_blue_state(const uint16_t** ranks, int* shift)
{
    const DeviceState* d = current_state();
    if (!d || !d->blue) return false;
    if (ranks) *ranks = d->blue;
    if (shift) *shift = d->blue_shift;
    return true;
}

extern "C" stf_status stf_set_blue_noise(const uint16_t* ranks, int size)
{
    int shift = 0;
    while ((1 << shift) < size) ++shift;
    if (!ranks || size < 4 || size > 256 || (1 << shift) != size)
        return stf_fail(STF_ERR_INVALID_ARG, "stf_set_blue_noise: size %d (a power of two, 4..256)", size);
    const int N = size * size;
    for (int c = 0; c < 2; ++c) {  // each mask a permutation of the ranks 0 .. size^2 - 1
        std::vector<uint8_t> seen((size_t)N, 0);
        for (int i = 0; i < N; ++i) {
            const int r = ranks[(size_t)c * N + i];
            if (r >= N || seen[r]) return stf_fail(STF_ERR_INVALID_ARG, "stf_set_blue_noise: mask %d is not a permutation", c);
            seen[r] = 1;
        }
    }
    stf_status st = stf_device_state(nullptr, nullptr);
    if (st != STF_OK) return st;
    DeviceState& d = *current_state();
    cudaError_t e;
    if (2 * N > d.blue_capacity) {
        if (d.blue && (e = cudaFree(d.blue)) != cudaSuccess) return stf_cuda_fail(e, "cudaFree(blue noise)");
        d.blue = nullptr;
        d.blue_capacity = 0;
        if ((e = cudaMalloc(&d.blue, (size_t)2 * N * sizeof(uint16_t))) != cudaSuccess) return stf_cuda_fail(e, "cudaMalloc(blue noise)");
        d.blue_capacity = 2 * N;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return stf_cuda_fail(e, "synchronize");
    if ((e = cudaMemcpy(d.blue, ranks, (size_t)2 * N * sizeof(uint16_t), cudaMemcpyHostToDevice)) != cudaSuccess)
        return stf_cuda_fail(e, "cudaMemcpy(blue noise)");
    d.blue_shift = shift;
    return STF_OK;
}

extern "C" stf_status stf_set_sparse_footprints(const signed char* table, int patterns, int tile_w, int tile_h)
{
    if (!table || patterns < 1 || patterns > STF_SPARSE_MAX_PATTERNS || !tile_ok(tile_w, tile_h))
        return stf_fail(STF_ERR_INVALID_ARG, "stf_set_sparse_footprints: bad arguments");
    std::vector<uint8_t> h((size_t)patterns * 32 * 16, 0);
    for (int p = 0; p < patterns; ++p)
        for (int l = 0; l < 32; ++l) {
            const signed char* row = table + ((size_t)p * 32 + l) * 9;
            if (row[0] != l) return stf_fail(STF_ERR_INVALID_ARG, "pattern %d lane %d: the own lane must come first", p, l);
            for (int i = 0; i < 9; ++i) {
                if (row[i] < 0 || row[i] > 31) return stf_fail(STF_ERR_INVALID_ARG, "pattern %d lane %d: lane index %d", p, l, row[i]);
                for (int k = 0; k < i; ++k)
                    if (row[k] == row[i]) return stf_fail(STF_ERR_INVALID_ARG, "pattern %d lane %d: repeated lane %d", p, l, row[i]);
                h[((size_t)p * 32 + l) * 16 + i] = (uint8_t)row[i];
            }
        }
    stf_status st = stf_device_state(nullptr, nullptr);
    if (st != STF_OK) return st;
    DeviceState& d = *current_state();
    cudaError_t e;
    if (patterns > d.fp_capacity) {
        if (d.fp && (e = cudaFree(d.fp)) != cudaSuccess) return stf_cuda_fail(e, "cudaFree(footprints)");
        d.fp = nullptr;
        d.fp_patterns = d.fp_capacity = 0;
        if ((e = cudaMalloc(&d.fp, h.size())) != cudaSuccess) return stf_cuda_fail(e, "cudaMalloc(footprints)");
        d.fp_capacity = patterns;
    }
    // synchronous: the previous patterns may still be read by enqueued work
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return stf_cuda_fail(e, "synchronize");
    if ((e = cudaMemcpy(d.fp, h.data(), h.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return stf_cuda_fail(e, "cudaMemcpy(footprints)");
    d.fp_patterns = patterns;
    d.fp_tw = tile_w;
    d.fp_th = tile_h;
    return STF_OK;
}

stf_status stf_device_state(int** flags, const float** lut)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return stf_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return stf_fail(STF_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    DeviceState& d = g_dev[dev];
    if (!d.ready) {
        float h[256];
        for (int q = 0; q < 256; ++q) h[q] = (float)q / 255.0f;
        if ((e = cudaMalloc(&d.unorm_lut, sizeof h)) != cudaSuccess) return stf_cuda_fail(e, "cudaMalloc(lut)");
        if ((e = cudaMemcpy(d.unorm_lut, h, sizeof h, cudaMemcpyHostToDevice)) != cudaSuccess)
            return stf_cuda_fail(e, "cudaMemcpy(lut)");
        if ((e = cudaMalloc(&d.flags, 4 * sizeof(int))) != cudaSuccess) return stf_cuda_fail(e, "cudaMalloc(flags)");
        if ((e = cudaMemset(d.flags, 0, 4 * sizeof(int))) != cudaSuccess) return stf_cuda_fail(e, "cudaMemset(flags)");
        d.ready = true;
    }
    if (flags) *flags = d.flags;
    if (lut) *lut = d.unorm_lut;
    return STF_OK;
}

// The current device's error flags if its per-device state exists, without setting it up (so
// without allocating); STF_ERR_UNSUPPORTED otherwise. stf_create_texture sets the state up.
stf_status stf_device_state_ready(int** flags)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return stf_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return stf_fail(STF_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    if (!g_dev[dev].ready)
        return stf_fail(STF_ERR_UNSUPPORTED, "no texture was created on device %d (stf_create_texture sets up the "
                                             "per-device state)", dev);
    if (flags) *flags = g_dev[dev].flags;
    return STF_OK;
}

extern "C" stf_status stf_sync(void)
{
    cudaError_t e = cudaStreamSynchronize(g_stream);
    if (e != cudaSuccess) return stf_cuda_fail(e, "cudaStreamSynchronize");
    int* flags = nullptr;
    stf_status s = stf_device_state(&flags, nullptr);
    if (s != STF_OK) return s;
    int h[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpy(h, flags, sizeof h, cudaMemcpyDeviceToHost)) != cudaSuccess) return stf_cuda_fail(e, "read flags");
    if (h[0] || h[1]) {
        cudaMemset(flags, 0, sizeof h);
        if (h[0]) return stf_fail(STF_ERR_TIMEOUT, "a persistent-scheduler wait gave up (%d times)", h[0]);
        return stf_fail(STF_ERR_DEVICE_ASSERT, "a device-side index check failed (%d times)", h[1]);
    }
    return STF_OK;
}

// ------------------------------------------------------------------------------ textures

static int fmt_bytes(int fmt)
{
    switch (fmt) {
    case STF_FMT_FP32: return 4;
    case STF_FMT_FP16: case STF_FMT_BF16: return 2;
    case STF_FMT_E4M3: case STF_FMT_UNORM8: return 1;
    }
    return 0;
}

// Widening decode of any plane combination into FP32 records of `out_ch` floats (4 or 8);
// value = decode(code) * scale, each step exact or rounded once like the oracle.
struct PlaneDesc {
    const unsigned char* data[4];
    int fmt[4], ch[4], num;
};

__global__ void k_widen(PlaneDesc pd, int w, int h, const float* scales, int st, int stx, int C, int out_ch, float* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)w * h) return;
    const int x = (int)(i % w), y = (int)(i / w);
    float* o = out + i * out_ch;
    int c = 0;
    for (int p = 0; p < pd.num; ++p) {
        const int nb = pd.fmt[p] == STF_FMT_FP32 ? 4 : (pd.fmt[p] == STF_FMT_FP16 || pd.fmt[p] == STF_FMT_BF16 ? 2 : 1);
        const unsigned char* b = pd.data[p] + (size_t)i * pd.ch[p] * nb;
        for (int k = 0; k < pd.ch[p]; ++k, ++c) {
            float v;
            switch (pd.fmt[p]) {
            case STF_FMT_FP32: v = reinterpret_cast<const float*>(b)[k]; break;
            case STF_FMT_FP16: v = __half2float(__ushort_as_half(reinterpret_cast<const unsigned short*>(b)[k])); break;
            case STF_FMT_BF16: v = __uint_as_float((uint32_t)reinterpret_cast<const unsigned short*>(b)[k] << 16); break;
            case STF_FMT_E4M3: {
                const __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b[k], __NV_E4M3);
                v = __half2float(__half(hr));
                break;
            }
            default: v = __fdiv_rn((float)b[k], 255.0f); break;
            }
            if (scales) v = __fmul_rn(v, scales[((size_t)(y / st) * stx + (x / st)) * C + c]);
            o[c] = v;
        }
    }
    for (; c < out_ch; ++c) o[c] = 0.0f;
}

// RGBA8 plane + RG16F plane -> 8-byte records.
__global__ void k_interleave_u8_f16(const uint32_t* rgba, const uint32_t* rg, long long n, uint2* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_uint2(rgba[i], rg[i]);
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    void* release() { void* r = p; p = nullptr; return r; }
};

static stf_status to_device(const void* src, size_t bytes, int on_device, DevBuf& keep, const void** out)
{
    if (on_device) { *out = src; return STF_OK; }
    cudaError_t e = cudaMalloc(&keep.p, bytes);
    if (e != cudaSuccess) return stf_cuda_fail(e, "cudaMalloc(texture staging)");
    if ((e = cudaMemcpy(keep.p, src, bytes, cudaMemcpyHostToDevice)) != cudaSuccess) return stf_cuda_fail(e, "cudaMemcpy(texture)");
    *out = keep.p;
    return STF_OK;
}

extern "C" stf_status stf_update_texture(stf_texture* t, const void* data, int data_on_device)
{
    if (!t || !data) return stf_fail(STF_ERR_INVALID_ARG, "stf_update_texture: null argument");
    size_t rec = 0;
    switch (t->kind) {
    case K_F32x4: rec = 16; break;
    case K_F32x8: rec = 32; break;
    case K_F16x4: rec = 8; break;
    case K_F16x8: case K_BF16x8: rec = 16; break;
    case K_E4M3x8: rec = 8; break;
    default:
        return stf_fail(STF_ERR_UNSUPPORTED, "stf_update_texture: the texture's texels are not its plane's bytes "
                                             "(interleaved, widened or neural): create a new texture");
    }
    if (t->widened) return stf_fail(STF_ERR_UNSUPPORTED, "stf_update_texture: the texture was widened at creation");
    const size_t bytes = (size_t)t->width * t->height * rec;
    const cudaError_t e = cudaMemcpyAsync(t->texels, data, bytes, data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                          stf_stream());
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "stf_update_texture copy");
}

extern "C" stf_status stf_create_texture(const stf_texture_desc* d, stf_texture** out)
{
    if (!d || !out) return stf_fail(STF_ERR_INVALID_ARG, "stf_create_texture: null argument");
    if (d->width < 1 || d->height < 1 || d->width > 16384 || d->height > 16384)
        return stf_fail(STF_ERR_INVALID_ARG, "texture size %dx%d outside 1..16384", d->width, d->height);
    // the per-device state (error flags, UNORM8 table) is set up with every texture, before its
    // first allocation, so that rendering (the allocation-free entry point included) never
    // allocates it later
    if (d->num_planes == 0 && d->decoder) {
        stf_status ds = stf_device_state(nullptr, nullptr);
        if (ds != STF_OK) return ds;
        return stf_create_neural_texture(d, out);
    }
    if (d->num_planes < 1 || d->num_planes > 4) return stf_fail(STF_ERR_INVALID_ARG, "num_planes %d outside 1..4", d->num_planes);
    int C = 0;
    for (int p = 0; p < d->num_planes; ++p) {
        const stf_plane& pl = d->planes[p];
        if (fmt_bytes(pl.fmt) == 0) return stf_fail(STF_ERR_INVALID_ARG, "plane %d: unknown format %d", p, pl.fmt);
        if (pl.channels < 1) return stf_fail(STF_ERR_INVALID_ARG, "plane %d: channels %d < 1", p, pl.channels);
        if (!pl.data) return stf_fail(STF_ERR_INVALID_ARG, "plane %d: null data", p);
        C += pl.channels;
    }
    if (C > kMaxCh) return stf_fail(STF_ERR_INVALID_ARG, "%d channels in total, at most 8", C);
    if (d->tile_scales && d->scale_tile < 1) return stf_fail(STF_ERR_INVALID_ARG, "scale_tile %d < 1", d->scale_tile);

    const int W = d->width, H = d->height;
    const long long n = (long long)W * H;
    const int stx = d->tile_scales ? (W + d->scale_tile - 1) / d->scale_tile : 0;
    const int sty = d->tile_scales ? (H + d->scale_tile - 1) / d->scale_tile : 0;
    const size_t scale_bytes = (size_t)stx * sty * C * sizeof(float);
    const bool pow2_tile = d->tile_scales && (d->scale_tile & (d->scale_tile - 1)) == 0;
    const stf_plane& p0 = d->planes[0];

    int kind = -1;
    if (d->num_planes == 1) {
        if (!d->tile_scales && p0.fmt == STF_FMT_FP32 && p0.channels == 4) kind = K_F32x4;
        else if (!d->tile_scales && p0.fmt == STF_FMT_FP32 && p0.channels == 8) kind = K_F32x8;
        else if (!d->tile_scales && p0.fmt == STF_FMT_FP16 && p0.channels == 4) kind = K_F16x4;
        else if (!d->tile_scales && p0.fmt == STF_FMT_FP16 && p0.channels == 8) kind = K_F16x8;
        else if (!d->tile_scales && p0.fmt == STF_FMT_BF16 && p0.channels == 8) kind = K_BF16x8;
        else if (p0.fmt == STF_FMT_E4M3 && p0.channels == 8 && (!d->tile_scales || pow2_tile)) kind = K_E4M3x8;
    } else if (d->num_planes == 2 && !d->tile_scales && p0.fmt == STF_FMT_UNORM8 && p0.channels == 4 &&
               d->planes[1].fmt == STF_FMT_FP16 && d->planes[1].channels == 2) {
        kind = K_U8x4_F16x2;
    }

    stf_status ds = stf_device_state(nullptr, nullptr);
    if (ds != STF_OK) return ds;
    stf_texture* t = new (std::nothrow) stf_texture();
    if (!t) return stf_fail(STF_ERR_OUT_OF_MEMORY, "host allocation");
    t->width = W; t->height = H; t->channels = C; t->decoder = nullptr;
    cudaError_t e;
    DevBuf texels, scales;
    stf_status st = STF_OK;

    auto fail = [&](stf_status s) { delete t; return s; };

    if (kind == K_F32x4 || kind == K_F32x8 || kind == K_F16x4 || kind == K_F16x8 || kind == K_BF16x8 || kind == K_E4M3x8) {
        const size_t bytes = (size_t)n * p0.channels * fmt_bytes(p0.fmt);
        if ((e = cudaMalloc(&texels.p, bytes)) != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMalloc(texels)"));
        e = cudaMemcpy(texels.p, p0.data, bytes, p0.data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMemcpy(texels)"));
        t->scale_shift = 14;
        t->scale_tiles_x = 1;
        if (kind == K_E4M3x8) {
            if (d->tile_scales) {
                if ((e = cudaMalloc(&scales.p, scale_bytes)) != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMalloc(scales)"));
                e = cudaMemcpy(scales.p, d->tile_scales, scale_bytes, d->scales_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
                if (e != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMemcpy(scales)"));
                int sh = 0;
                while ((1 << sh) < d->scale_tile) ++sh;
                t->scale_shift = sh;
                t->scale_tiles_x = stx;
            } else {  // one tile of unit scales covering the whole texture
                const float ones[8] = {1, 1, 1, 1, 1, 1, 1, 1};
                if ((e = cudaMalloc(&scales.p, sizeof ones)) != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMalloc(scales)"));
                if ((e = cudaMemcpy(scales.p, ones, sizeof ones, cudaMemcpyHostToDevice)) != cudaSuccess)
                    return fail(stf_cuda_fail(e, "cudaMemcpy(scales)"));
            }
        }
    } else if (kind == K_U8x4_F16x2) {
        DevBuf s0, s1;
        const void *a = nullptr, *b = nullptr;
        if ((st = to_device(p0.data, n * 4, p0.data_on_device, s0, &a)) != STF_OK) return fail(st);
        if ((st = to_device(d->planes[1].data, n * 4, d->planes[1].data_on_device, s1, &b)) != STF_OK) return fail(st);
        if ((e = cudaMalloc(&texels.p, n * 8)) != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMalloc(texels)"));
        k_interleave_u8_f16<<<(unsigned)((n + 255) / 256), 256>>>((const uint32_t*)a, (const uint32_t*)b, n, (uint2*)texels.p);
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(stf_cuda_fail(e, "interleave kernel"));
        t->scale_shift = 14;
        t->scale_tiles_x = 1;
    } else {
        // widen to FP32 records of 4 or 8 channels
        kind = C <= 4 ? K_F32x4 : K_F32x8;
        t->widened = true;
        const int oc = C <= 4 ? 4 : 8;
        DevBuf stage[4], sdev;
        PlaneDesc pd;
        memset(&pd, 0, sizeof pd);
        pd.num = d->num_planes;
        for (int p = 0; p < d->num_planes; ++p) {
            const void* dp = nullptr;
            const size_t bytes = (size_t)n * d->planes[p].channels * fmt_bytes(d->planes[p].fmt);
            if ((st = to_device(d->planes[p].data, bytes, d->planes[p].data_on_device, stage[p], &dp)) != STF_OK) return fail(st);
            pd.data[p] = (const unsigned char*)dp;
            pd.fmt[p] = d->planes[p].fmt;
            pd.ch[p] = d->planes[p].channels;
        }
        const void* sc = nullptr;
        if (d->tile_scales && (st = to_device(d->tile_scales, scale_bytes, d->scales_on_device, sdev, &sc)) != STF_OK) return fail(st);
        if ((e = cudaMalloc(&texels.p, (size_t)n * oc * sizeof(float))) != cudaSuccess) return fail(stf_cuda_fail(e, "cudaMalloc(texels)"));
        k_widen<<<(unsigned)((n + 255) / 256), 256>>>(pd, W, H, (const float*)sc, d->scale_tile, stx, C, oc, (float*)texels.p);
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(stf_cuda_fail(e, "widen kernel"));
        t->scale_shift = 14;
        t->scale_tiles_x = 1;
    }
    t->kind = kind;
    t->texels = texels.release();
    t->scales = (float*)scales.release();
    *out = t;
    return STF_OK;
}

// Tensor map over a stored texture's records as a [height][width * R / 4] array of 32-bit
// words, box 16 texels x 4 rows (the TMA-staged render variant's tile). The encode entry point is
// taken from the driver through the runtime, so the library links no driver library.
const CUtensorMap* stf_texture_tmap(const stf_texture* t)
{
    if (t->tmap_state) return t->tmap_state > 0 ? &t->tmap : nullptr;
    t->tmap_state = -1;
    int rec = 0;
    switch (t->kind) {
    case K_F32x4: case K_F16x8: case K_BF16x8: rec = 16; break;
    case K_F32x8: rec = 32; break;
    case K_F16x4: case K_E4M3x8: case K_U8x4_F16x2: rec = 8; break;
    default: return nullptr;
    }
    if (((size_t)t->width * rec) % 16 != 0) return nullptr;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)t->width * rec / 4, (cuuint64_t)t->height};
    const cuuint64_t strides[1] = {(cuuint64_t)t->width * rec};
    const cuuint32_t box[2] = {(cuuint32_t)(16 * rec / 4), 4};
    const cuuint32_t estr[2] = {1, 1};
    if (encode(&t->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, t->texels, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return nullptr;
    t->tmap_state = 1;
    return &t->tmap;
}

extern "C" stf_status stf_destroy(stf_texture* t)
{
    if (!t) return STF_OK;
    if (t->texels) cudaFree(t->texels);
    if (t->scales) cudaFree(t->scales);
    delete t;
    return STF_OK;
}

// ------------------------------------------------------------------------------ views

static bool tile_ok(int tw, int th)
{
    return (tw == 8 && th == 4) || (tw == 4 && th == 8) || (tw == 16 && th == 2);
}

stf_status stf_validate_view(const stf_view& v, int i, int filter, int mode)
{
    if (!v.tex) return stf_fail(STF_ERR_INVALID_ARG, "view %d: null texture", i);
    if (v.width < 1 || v.height < 1 || v.width > 32768 || v.height > 32768)
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: size %dx%d outside 1..32768", i, v.width, v.height);
    if (!v.out_rgba) return stf_fail(STF_ERR_INVALID_ARG, "view %d: null out_rgba", i);
    if (v.out_pitch_floats != 0 && v.out_pitch_floats < 4LL * v.width)
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: out_pitch_floats %lld < 4 * width", i, v.out_pitch_floats);
    if ((v.out_pitch_floats & 3) != 0) return stf_fail(STF_ERR_INVALID_ARG, "view %d: out_pitch_floats not a multiple of 4", i);
    if (((uintptr_t)v.out_rgba & 15) != 0) return stf_fail(STF_ERR_INVALID_ARG, "view %d: out_rgba not 16-byte aligned", i);
    if (v.debug_channels && ((uintptr_t)v.debug_channels & 15) != 0)
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: debug_channels not 16-byte aligned", i);
    const int f = filter == STF_FILTER_PER_VIEW ? v.filter : filter;
    if (f != STF_FILTER_BILINEAR && f != STF_FILTER_BSPLINE3) return stf_fail(STF_ERR_INVALID_ARG, "view %d: filter %d", i, f);
    if (!(v.tile_w == 0 && v.tile_h == 0) && !tile_ok(v.tile_w, v.tile_h))
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: tile %dx%d (8x4, 4x8, 16x2 or 0x0)", i, v.tile_w, v.tile_h);
    if (v.frame < 0 || v.frame > 65535 || v.view_id < 0 || v.view_id > 65535)
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: frame and view_id must be in 0..65535", i);
    const int C = v.tex->channels;
    if (v.shading) {
        if (v.shading != 1) return stf_fail(STF_ERR_INVALID_ARG, "view %d: shading %d", i, v.shading);
        if (v.ch_albedo < -1 || v.ch_albedo + 2 >= C + (v.ch_albedo < 0 ? 3 : 0))
            return stf_fail(STF_ERR_INVALID_ARG, "view %d: ch_albedo %d", i, v.ch_albedo);
        if (v.ch_normal < -1 || v.ch_normal + 1 >= C + (v.ch_normal < 0 ? 2 : 0))
            return stf_fail(STF_ERR_INVALID_ARG, "view %d: ch_normal %d", i, v.ch_normal);
        if (v.ch_rough < -1 || v.ch_rough >= C) return stf_fail(STF_ERR_INVALID_ARG, "view %d: ch_rough %d", i, v.ch_rough);
        if (v.ch_ao < -1 || v.ch_ao >= C) return stf_fail(STF_ERR_INVALID_ARG, "view %d: ch_ao %d", i, v.ch_ao);
    }
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(v.H[k])) return stf_fail(STF_ERR_INVALID_ARG, "view %d: H[%d] not finite", i, k);
    if ((mode & STF_MODE_FLAG_BLUE_NOISE) && !stf_blue_state(nullptr, nullptr))
        return stf_fail(STF_ERR_INVALID_ARG, "view %d: STF_MODE_FLAG_BLUE_NOISE without stf_set_blue_noise", i);
    if ((mode & kModeBase) == STF_MODE_SPARSE9) {
        int tw = 0, th = 0;
        if (!stf_sparse_state(nullptr, nullptr, &tw, &th))
            return stf_fail(STF_ERR_INVALID_ARG, "view %d: STF_MODE_SPARSE9 without stf_set_sparse_footprints", i);
        if (v.tile_w != 0 && (v.tile_w != tw || v.tile_h != th))
            return stf_fail(STF_ERR_INVALID_ARG, "view %d: tile %dx%d differs from the sparse footprints' %dx%d", i,
                            v.tile_w, v.tile_h, tw, th);
    }
    return STF_OK;
}

void stf_fill_devview(const stf_view& v, int filter, int mode, unsigned long long seed, const float* lut, DevView& d)
{
    memset(&d, 0, sizeof d);
    for (int k = 0; k < 9; ++k) d.H[k] = v.H[k];
    for (int k = 0; k < 3; ++k) { d.cam[k] = v.cam_pos[k]; d.light[k] = v.light_dir[k]; }
    for (int k = 0; k < 6; ++k) d.p2w[k] = v.plane_to_world[k];
    d.rough_const = v.roughness;
    d.width = v.width;
    d.height = v.height;
    d.filter = filter == STF_FILTER_PER_VIEW ? v.filter : filter;
    int tw = v.tile_w, th = v.tile_h;
    if (tw == 0 || (mode & kModeBase) <= STF_MODE_ONE_TAP) { tw = 8; th = 4; }
    if ((mode & kModeBase) == STF_MODE_SPARSE9) {  // the frame's pattern, on the patterns' tile
        const uint8_t* fp = nullptr;
        int np = 1;
        stf_sparse_state(&fp, &np, &tw, &th);
        d.fp = fp ? fp + (size_t)(v.frame % np) * 32 * 16 : nullptr;
    }
    d.tile_w = tw;
    d.tile_h = th;
    d.tiles_x = (v.width + tw - 1) / tw;
    d.tiles_y = (v.height + th - 1) / th;
    const stf_texture* t = v.tex;
    d.tex_w = t->width;
    d.tex_h = t->height;
    d.tex_wf = (float)t->width;
    d.tex_hf = (float)t->height;
    d.texels = t->texels;
    d.scales = t->scales;
    d.unorm_lut = lut;
    d.scale_shift = t->scale_shift;
    d.scale_tiles_x = t->scale_tiles_x;
    d.out = v.out_rgba;
    d.pitch = v.out_pitch_floats ? v.out_pitch_floats : 4LL * v.width;
    d.dbg_idx = v.debug_indices;
    d.dbg_ch = v.debug_channels;
    d.rng_z = (uint32_t)v.frame | ((uint32_t)v.view_id << 16);
    d.rng_w = (uint32_t)seed ^ (uint32_t)(seed >> 32);
    d.ch_albedo = v.ch_albedo;
    d.ch_normal = v.ch_normal;
    d.ch_rough = v.ch_rough;
    d.ch_ao = v.ch_ao;
    d.c_true = t->channels;
    d.neural = t->decoder_params;
    stf_device_state(&d.flags, nullptr);
    d.affine = (v.H[6] == 0.0f && v.H[7] == 0.0f && v.H[8] == 1.0f) ? 1 : 0;
    d.estimator = ((mode >> STF_MODE_EST_SHIFT) & 7) | ((mode & STF_MODE_FLAG_CLAMP) ? 8 : 0);
    d.tmap_host = g_tma_stage ? stf_texture_tmap(t) : nullptr;
    const uint16_t* r = nullptr;
    int sh = 0;
    if ((mode & STF_MODE_FLAG_BLUE_NOISE) && stf_blue_state(&r, &sh)) {
        d.blue = r;
        d.blue_shift = sh;
        d.blue_offset = ((uint32_t)v.frame * kBlueFrameStep + (d.rng_w & 0xffffffu)) & 0xffffffu;
    }
    if (!v.shading) d.shade_layout = 0;
    else if (v.ch_albedo == 0 && v.ch_normal == 3 && v.ch_rough == 5 && v.ch_ao == 6) d.shade_layout = 1;
    else if (v.ch_albedo == 0 && v.ch_normal == 4 && v.ch_rough == -1 && v.ch_ao == -1) d.shade_layout = 2;
    else d.shade_layout = 3;
}

namespace stf {
cudaError_t launch_view_F32x4(const DevView&, int, cudaStream_t);
cudaError_t launch_view_F32x8(const DevView&, int, cudaStream_t);
cudaError_t launch_view_F16x4(const DevView&, int, cudaStream_t);
cudaError_t launch_view_F16x8(const DevView&, int, cudaStream_t);
cudaError_t launch_view_BF16x8(const DevView&, int, cudaStream_t);
cudaError_t launch_view_E4M3x8(const DevView&, int, cudaStream_t);
cudaError_t launch_view_U8x4_F16x2(const DevView&, int, cudaStream_t);
}  // namespace stf

cudaError_t stf_launch_single(const DevView& d, int kind, int mode, cudaStream_t s)
{
    switch (kind) {
    case K_F32x4: return launch_view_F32x4(d, mode, s);
    case K_F32x8: return launch_view_F32x8(d, mode, s);
    case K_F16x4: return launch_view_F16x4(d, mode, s);
    case K_F16x8: return launch_view_F16x8(d, mode, s);
    case K_BF16x8: return launch_view_BF16x8(d, mode, s);
    case K_E4M3x8: return launch_view_E4M3x8(d, mode, s);
    case K_U8x4_F16x2: return launch_view_U8x4_F16x2(d, mode, s);
    case K_NEURAL: return stf_launch_neural_view(d, mode, s);
    }
    return cudaErrorInvalidValue;
}

// A reuse mode of the C interface: an stf_reuse_mode, optionally | STF_MODE_FLAG_EXACT with a
// sharing mode.
stf_status stf_check_mode(int mode)
{
    const int base = mode & kModeBase;
    const int est = (mode >> STF_MODE_EST_SHIFT) & 7;
    const int known = kModeBase | STF_MODE_FLAG_EXACT | STF_MODE_FLAG_BLUE_NOISE | (7 << STF_MODE_EST_SHIFT) | STF_MODE_FLAG_CLAMP;
    if (base > STF_MODE_SPARSE9 || (mode & ~known) || est > STF_EST_REGRESSION)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d", mode);
    if ((mode & STF_MODE_FLAG_EXACT) && base < STF_MODE_QUAD2)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d: exact filtering needs a sharing mode", mode);
    if ((mode & STF_MODE_FLAG_BLUE_NOISE) && base == STF_MODE_FULL)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d: the full filter draws no random numbers", mode);
    if ((est || (mode & STF_MODE_FLAG_CLAMP)) && base < STF_MODE_QUAD2)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d: an estimator needs a sharing mode", mode);
    if ((mode & STF_MODE_FLAG_CLAMP) && est == STF_EST_WIS)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d: the weighted estimator is bounded already (no clamp)", mode);
    if ((mode & STF_MODE_FLAG_EXACT) && est != STF_EST_WIS)
        return stf_fail(STF_ERR_INVALID_ARG, "reuse_mode %d: exact filtering goes with the weighted estimator", mode);
    return STF_OK;
}

// Alternative estimators are evaluation modes: one view of a stored material kind, 8x4 tiles.
static stf_status check_alt(const stf_view* views, int n, int mode)
{
    if (((mode >> STF_MODE_EST_SHIFT) & 7) == STF_EST_WIS) return STF_OK;
    if (n != 1) return stf_fail(STF_ERR_INVALID_ARG, "alternative estimators render one view per call");
    if ((mode & kModeBase) == STF_MODE_SPARSE9)
        return stf_fail(STF_ERR_INVALID_ARG, "alternative estimators: square footprints only");
    if (views[0].tex->kind == K_NEURAL)
        return stf_fail(STF_ERR_INVALID_ARG, "alternative estimators: stored material kinds only");
    if (views[0].tile_w != 0 && (views[0].tile_w != 8 || views[0].tile_h != 4))
        return stf_fail(STF_ERR_INVALID_ARG, "alternative estimators: 8x4 tiles only");
    return STF_OK;
}

extern "C" stf_status stf_render_views(const stf_view* views, int n, int filter, int reuse_mode, unsigned long long seed)
{
    if (!views || n < 1) return stf_fail(STF_ERR_INVALID_ARG, "stf_render_views: need n >= 1 views");
    if (filter != STF_FILTER_BILINEAR && filter != STF_FILTER_BSPLINE3 && filter != STF_FILTER_PER_VIEW)
        return stf_fail(STF_ERR_INVALID_ARG, "filter %d", filter);
    if (stf_check_mode(reuse_mode) != STF_OK) return STF_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        stf_status s = stf_validate_view(views[i], i, filter, reuse_mode);
        if (s != STF_OK) return s;
    }
    if (check_alt(views, n, reuse_mode) != STF_OK) return STF_ERR_INVALID_ARG;
    const float* lut = nullptr;
    stf_status s = stf_device_state(nullptr, &lut);
    if (s != STF_OK) return s;
    if (n > 1) return stf_render_batch(views, n, filter, reuse_mode, seed);
    DevView d;
    stf_fill_devview(views[0], filter, reuse_mode, seed, lut, d);
    int tw, th, sched;  // a 0x0 tile takes the autotuned shape of the view's class
    stf_resolve_view_config_nohalloc(views[0], filter, reuse_mode, &tw, &th, &sched);
    d.tile_w = tw;
    d.tile_h = th;
    d.tiles_x = (d.width + tw - 1) / tw;
    d.tiles_y = (d.height + th - 1) / th;
    cudaError_t e = stf_launch_single(d, views[0].tex->kind, reuse_mode, g_stream);
    if (e != cudaSuccess) return stf_cuda_fail(e, "render launch");
    return STF_OK;
}
