// Device side of the STF render path: per-view constants, texel formats, the per-axis
// selection, the warp-tile sharing loop with the weighted importance sampling combine, and
// shading. Everything a render kernel needs is a __forceinline__ function of this header;
// the kernels themselves are instantiated in stf_kernels.cuh.
//
// Bit-exactness contract with the CPU oracle: the choice of texel (the screen -> texel
// coordinates, the 1D filter weights, the running CDF and the comparison with the uniform)
// is computed with explicitly rounded intrinsics (__fmul_rn / __fadd_rn / __fdiv_rn), which
// the compiler never contracts into FMAs, in the same order as the oracle. The colour path
// (weights w_i, sums, shading) may use FMAs and fast reciprocals.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace stf {

constexpr float kCoordLo = -16384.0f;  // texel coordinates are clamped to [lo, hi] (NaN -> lo)
constexpr float kCoordHi = 32000.0f;
constexpr float kPi = 3.14159265f;
constexpr int kMaxCh = 8;
constexpr int kWarpsPerBlock = 8;  // warps (pixel tiles in flight) per render block
constexpr int kModeFlagExact = 16;  // STF_MODE_FLAG_EXACT of the C interface
constexpr int kModeEstShift = 8;     // STF_MODE_EST_SHIFT: (mode >> 8) & 7 = the estimator
constexpr int kModeFlagClamp = 2048; // STF_MODE_FLAG_CLAMP
constexpr int kModeBase = 15;        // the stf_reuse_mode bits
constexpr int kModeSparse9 = 6;      // STF_MODE_SPARSE9: 9-element pseudorandom sparse footprints
constexpr int kModeFlagBlue = 32;    // STF_MODE_FLAG_BLUE_NOISE
constexpr uint32_t kBlueFrameStep = 10368890u;  // round(2^24 (sqrt(5) - 1) / 2): the golden-ratio step
constexpr int kBatchMaxViews = 224; // views per persistent launch (their constants sit in a constant bank)

// Material kinds with a dedicated kernel. Anything else is widened to FP32 at creation.
enum MatKind : int {
    K_F32x4 = 0,      // RGBA FP32, 16-byte records
    K_F32x8 = 1,      // 8 x FP32, 32-byte records
    K_F16x4 = 2,      // 4 x FP16, 8-byte records
    K_F16x8 = 3,      // 8 x FP16, 16-byte records
    K_BF16x8 = 4,     // 8 x BF16, 16-byte records
    K_E4M3x8 = 5,     // 8 x E4M3 with per-(tile, channel) FP32 scales, 8-byte records
    K_U8x4_F16x2 = 6, // RGBA UNORM8 + XY FP16, 8-byte records
    K_NEURAL = 7,     // latent grid + MLP decoder
    K_COUNT = 8
};

// Per-view constants, passed by value (kernel parameter space) or read from a device array
// by the multi-view scheduler.
struct DevView {
    float H[9];
    float cam[3];
    float p2w[6];
    float light[3];
    float rough_const;
    int width, height;
    int tiles_x, tiles_y;
    int tex_w, tex_h;
    float tex_wf, tex_hf;
    const void* texels;
    const float* scales;
    const float* unorm_lut;   // 256 entries q / 255 (IEEE), for UNORM8 planes
    int scale_shift, scale_tiles_x;
    float* out;
    long long pitch;          // floats per output row
    uint32_t* dbg_idx;
    float* dbg_ch;
    uint32_t rng_z, rng_w;    // frame | view_id << 16, and the folded 64-bit seed
    int shade_layout;         // 0 none, 1 = (albedo 0, normal 3, rough 5, ao 6), 2 = (albedo 0, normal 4), 3 generic
    int ch_albedo, ch_normal, ch_rough, ch_ao;
    int c_true;               // channels of the material (alpha default when < 4)
    int filter, tile_w, tile_h;
    int affine;               // H[6] == H[7] == 0 and H[8] == 1: hw == 1 exactly, no division needed
    const void* neural;       // decoder parameters for K_NEURAL
    int* flags;               // device error counters: [0] timed-out waits
    const uint8_t* fp;        // STF_MODE_SPARSE9: the frame's pattern, [32 lanes][16] lane indices
    const uint16_t* blue;     // STF_MODE_FLAG_BLUE_NOISE: ranks [2][n][n] (n = 1 << blue_shift)
    int blue_shift;
    uint32_t blue_offset;     // 24-bit offset of the frame: frame * golden-ratio step + seed (mod 2^24)
    int estimator;            // alternative estimator (kernels compiled with ALT): 1 IS, 2 MIS,
                              // 3 pairwise MIS, 4 regression; + 8: clamp to the texels' range
    const void* tmap_host;    // host address of the texture's tensor map when the TMA-staged render
                              // variant is selected (read by the host launcher only), else null
};

// A run of tiles of one view for the persistent multi-view kernel. variant = filter * 3 + tile
// shape (0: 8x4, 1: 4x8, 2: 16x2).
struct WorkItem {
    int view, tile0, ntiles, variant;
};

// Single-instruction approximations for the colour path (never for the texel choice).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// The .ftz forms: the shading inputs are never subnormal (unit vectors, squared lengths of sums
// of unit vectors, a^2 >= 1.6e-7), so flushing changes no result and saves the subnormal fixups.
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Shared-memory address of a generic pointer to shared memory (for PTX operands).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ------------------------------------------------------------------------------ RNG

// pcg4d (Jarzynski and Olano, "Hash Functions for GPU Rendering", JCGT 2020): LCG step on the
// four words, cross multiply-add round, xor-shift by 16, second cross multiply-add round.
__device__ __forceinline__ void pcg4d(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d)
{
    a = a * 1664525u + 1013904223u;
    b = b * 1664525u + 1013904223u;
    c = c * 1664525u + 1013904223u;
    d = d * 1664525u + 1013904223u;
    a += b * d; b += c * a; c += a * b; d += b * c;
    a ^= a >> 16; b ^= b >> 16; c ^= c >> 16; d ^= d >> 16;
    a += b * d; b += c * a; c += a * b; d += b * c;
}

// ------------------------------------------------------------------------------ filters

template <int F> struct Taps;
template <> struct Taps<0> { static constexpr int N = 2, K0 = 0; };   // bilinear: floor(c) + {0, 1}
template <> struct Taps<1> { static constexpr int N = 4, K0 = -1; };  // cubic B-spline: floor(c) + {-1..2}

// Bilinear tent per axis, clamp(1 - |d|, 0, 1) (Section S6). 1 - |d| never exceeds 1, so the
// clamp is the subtraction's saturation (one instruction; NaN and negative results give +0,
// as max(., 0) would).
__device__ __forceinline__ float w_bilinear(float d)
{
    return __saturatef(__fsub_rn(1.0f, fabsf(d)));
}

// B-spline branches of W with a = |d|: r1 for a < 1, r2 for 1 <= a < 2 (each step rounded once).
__device__ __forceinline__ float bspline_r1(float a)
{
    float t = __fmul_rn(3.0f, a);
    t = __fsub_rn(t, 6.0f);
    t = __fmul_rn(t, a);
    t = __fmul_rn(t, a);
    t = __fadd_rn(t, 4.0f);
    return __fmul_rn(t, 1.0f / 6.0f);
}
__device__ __forceinline__ float bspline_r2(float a)
{
    const float s = __fsub_rn(2.0f, a);
    float q = __fmul_rn(s, s);
    q = __fmul_rn(q, s);
    return __fmul_rn(q, 1.0f / 6.0f);
}

// Weight of tap t (lattice point floor(c) + K0 + t, given as the exact float nf) of coordinate c.
// For the B-spline the branch of W is known per tap: d = c - n lies in [1, 2] for t = 0, [0, 1]
// for t = 1, [-1, 0] for t = 2 and [-2, -1] for t = 3 (c - floor(c) is in [0, 1] after
// rounding). Where |d| lands exactly on 1 or 2 both candidate branches give the same float
// (r1(1) = r2(1) = 1/6 in FP32, r2(2) = 0), so this equals W(c - n) bit for bit.
template <int F> __device__ __forceinline__ float tap_weight(float c, float nf, int t)
{
    const float d = __fsub_rn(c, nf);
    if constexpr (F == 0) return w_bilinear(d);
    const float a = fabsf(d);
    return (t == 1 || t == 2) ? bspline_r1(a) : bspline_r2(a);
}

// One axis of a lane: its lattice base, the weights of its taps, and its one-tap selection.
template <int F> struct Axis {
    int base;                  // floor(c) + K0: lattice index of tap 0
    float basef;               // the same as a float (exact)
    float w[Taps<F>::N];       // W(c - (base + t))
    int n;                     // selected lattice index
    float nf;                  // the same as a float
    float p;                   // its weight (the 1D PMF value)
};

// Tap weights only (for the deterministic filter). Bilinear: c - floor(c) lies in [0, 1] and
// c - (floor(c) + 1) in [-1, 0], so 1 - |d| is never negative and the clamp of W is dropped
// (the same floats as w_bilinear).
template <int F> __device__ __forceinline__ void axis_weights(float c, Axis<F>& A)
{
    const float i0f = floorf(c);
    A.base = __float2int_rn(i0f) + Taps<F>::K0;
    A.basef = __fadd_rn(i0f, (float)Taps<F>::K0);
#pragma unroll
    for (int t = 0; t < Taps<F>::N; ++t) {
        const float nf = __fadd_rn(A.basef, (float)t);
        if constexpr (F == 0) A.w[t] = __fsub_rn(1.0f, fabsf(__fsub_rn(c, nf)));
        else A.w[t] = tap_weight<F>(c, nf, t);
    }
}

// Taps in increasing lattice order; running FP32 CDF; first tap with u < CDF, else the last
// tap with positive weight; both filters in closed form. Bilinear: CDF_0 = w0 and CDF_1 = w0 + w1
// >= w0, so u >= w0 picks tap 1 whenever w1 > 0 (through the CDF or as the last positive tap)
// and tap 0 otherwise (w0 > 0 then, the weights summing to about 1). Cubic B-spline: the running
// CDF never decreases, so the first tap with u < CDF_t is the number k of CDF_0 .. CDF_2 at or
// below u whenever u < CDF_3; otherwise (rounding left u above the total) the last positive tap
// is 3, or 2 when w3 = 0 (the middle taps always weigh at least 1/6).
template <int F> __device__ __forceinline__ void axis_select(float c, float u, Axis<F>& A)
{
    axis_weights<F>(c, A);
    if constexpr (F == 0) {
        const bool one = !(u < A.w[0]) && A.w[1] > 0.0f;
        A.n = A.base + (one ? 1 : 0);
        A.nf = one ? __fadd_rn(A.basef, 1.0f) : A.basef;
        A.p = one ? A.w[1] : A.w[0];
    } else {
        const float c0 = A.w[0], c1 = __fadd_rn(c0, A.w[1]), c2 = __fadd_rn(c1, A.w[2]);
        const float c3 = __fadd_rn(c2, A.w[3]);
        const int k = (u < c0 ? 0 : 1) + (u < c1 ? 0 : 1) + (u < c2 ? 0 : 1);
        const int pick = k - ((!(u < c3) && !(A.w[3] > 0.0f)) ? 1 : 0);
        A.n = A.base + pick;
        A.nf = __fadd_rn(A.basef, __int2float_rn(pick));
        A.p = pick == 0 ? A.w[0] : (pick == 1 ? A.w[1] : (pick == 2 ? A.w[2] : A.w[3]));
    }
}

// The pixel's two selection uniforms as exact 24-bit dyadic floats: the counter hash pcg4d of
// (x, y, frame | view << 16, seed), or (BLUE) the ranks r of (x mod n, y mod n) in two
// independent blue-noise masks as (r + 1/2) / n^2 shifted by the frame's offset modulo 1 (a
// golden-ratio step per frame, Cranley-Patterson rotation). BLUE is a kernel variant: a runtime
// choice here costs the render kernels registers, and spills, in their sharing loops.
template <bool BLUE>
__device__ __forceinline__ void pixel_uniforms(const DevView& v, int x, int y, float& ux, float& uy)
{
    uint32_t a, b;
    if constexpr (BLUE) {
        const int sh = v.blue_shift, m = (1 << sh) - 1;
        const int k = ((y & m) << sh) | (x & m);
        const uint32_t step = 24 - 2 * sh;  // 2^24 / n^2 = 1 << step
        const uint32_t half = (1u << step) >> 1;
        a = (((uint32_t)__ldg(v.blue + k) << step) + half + v.blue_offset) & 0xffffffu;
        b = (((uint32_t)__ldg(v.blue + ((m + 1) << sh) + k) << step) + half + v.blue_offset) & 0xffffffu;
    } else {
        uint32_t ra = (uint32_t)x, rb = (uint32_t)y, rc = v.rng_z, rd = v.rng_w;
        pcg4d(ra, rb, rc, rd);
        a = ra >> 8;
        b = rb >> 8;
    }
    ux = __uint2float_rn(a) * (1.0f / 16777216.0f);
    uy = __uint2float_rn(b) * (1.0f / 16777216.0f);
}

// ------------------------------------------------------------------------------ coordinates

// Pixel centre -> uv through the view homography, rounded step by step like the oracle.
__device__ __forceinline__ void pixel_uv(const DevView& v, int x, int y, float& u, float& w)
{
    const float px = __fadd_rn(__int2float_rn(x), 0.5f);
    const float py = __fadd_rn(__int2float_rn(y), 0.5f);
    const float hx = __fadd_rn(__fadd_rn(__fmul_rn(v.H[0], px), __fmul_rn(v.H[1], py)), v.H[2]);
    const float hy = __fadd_rn(__fadd_rn(__fmul_rn(v.H[3], px), __fmul_rn(v.H[4], py)), v.H[5]);
    if (v.affine) {  // hw = 0 * px + 0 * py + 1 = 1 exactly, and x / 1 = x
        u = hx;
        w = hy;
        return;
    }
    const float hw = __fadd_rn(__fadd_rn(__fmul_rn(v.H[6], px), __fmul_rn(v.H[7], py)), v.H[8]);
    u = __fdiv_rn(hx, hw);
    w = __fdiv_rn(hy, hw);
}

// uv * size - 0.5 (Section 4.5 listing), clamped so lattice indices fit 16 bits.
__device__ __forceinline__ float texel_coord(float uv, float size)
{
    const float c = __fsub_rn(__fmul_rn(uv, size), 0.5f);
    return fminf(fmaxf(c, kCoordLo), kCoordHi);
}

__device__ __forceinline__ uint32_t pack_idx(int ix, int iy)
{
    return (uint32_t)(ix & 0xffff) | ((uint32_t)(iy & 0xffff) << 16);
}
__device__ __forceinline__ int unpack_x(uint32_t p) { return (int)(int16_t)(p & 0xffffu); }
__device__ __forceinline__ int unpack_y(uint32_t p) { return ((int)p) >> 16; }

// ------------------------------------------------------------------------------ texel formats

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return min(max(a, lo), hi); }

__device__ __forceinline__ float h2f(uint32_t bits16) { return __half2float(__ushort_as_half((unsigned short)bits16)); }
__device__ __forceinline__ float bf2f(uint32_t bits16) { return __uint_as_float(bits16 << 16); }

template <int KIND> struct Mat;

// A texel record as R / 4 32-bit words, read from global memory (read-only path) or from a
// shared-memory copy (the staged footprint box of the TMA render variant).
template <int R> struct Raw { uint32_t w[R / 4]; };
template <int R> __device__ __forceinline__ Raw<R> ld_record(const void* base, size_t i)
{
    Raw<R> r;
    if constexpr (R == 8) {
        const uint2 a = __ldg(reinterpret_cast<const uint2*>(base) + i);
        r.w[0] = a.x; r.w[1] = a.y;
    } else {
#pragma unroll
        for (int k = 0; k < R / 16; ++k) {
            const uint4 a = __ldg(reinterpret_cast<const uint4*>(base) + (R / 16) * i + k);
            r.w[4 * k] = a.x; r.w[4 * k + 1] = a.y; r.w[4 * k + 2] = a.z; r.w[4 * k + 3] = a.w;
        }
    }
    return r;
}
template <int R> __device__ __forceinline__ Raw<R> ld_record_shared(uint32_t addr)
{
    Raw<R> r;
    if constexpr (R == 8) {
        asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(r.w[0]), "=r"(r.w[1]) : "r"(addr));
    } else {
#pragma unroll
        for (int k = 0; k < R / 16; ++k)
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r.w[4 * k]), "=r"(r.w[4 * k + 1]), "=r"(r.w[4 * k + 2]), "=r"(r.w[4 * k + 3])
                         : "r"(addr + 16 * k));
    }
    return r;
}

// Every kind: C channels from an R-byte record; decode(record, texel) and fetch = decode(load).
template <> struct Mat<K_F32x4> {
    static constexpr int C = 4, R = 16;
    __device__ static __forceinline__ void decode(const DevView&, const Raw<R>& r, int, int, float (&t)[C])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = __uint_as_float(r.w[i]);
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_F32x8> {
    static constexpr int C = 8, R = 32;
    __device__ static __forceinline__ void decode(const DevView&, const Raw<R>& r, int, int, float (&t)[C])
    {
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = __uint_as_float(r.w[i]);
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_F16x4> {
    static constexpr int C = 4, R = 8;
    __device__ static __forceinline__ void decode(const DevView&, const Raw<R>& r, int, int, float (&t)[C])
    {
        t[0] = h2f(r.w[0] & 0xffffu); t[1] = h2f(r.w[0] >> 16); t[2] = h2f(r.w[1] & 0xffffu); t[3] = h2f(r.w[1] >> 16);
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_F16x8> {
    static constexpr int C = 8, R = 16;
    __device__ static __forceinline__ void decode(const DevView&, const Raw<R>& r, int, int, float (&t)[C])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) { t[2 * i] = h2f(r.w[i] & 0xffffu); t[2 * i + 1] = h2f(r.w[i] >> 16); }
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_BF16x8> {
    static constexpr int C = 8, R = 16;
    __device__ static __forceinline__ void decode(const DevView&, const Raw<R>& r, int, int, float (&t)[C])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) { t[2 * i] = bf2f(r.w[i] & 0xffffu); t[2 * i + 1] = __uint_as_float(r.w[i] & 0xffff0000u); }
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_E4M3x8> {
    static constexpr int C = 8, R = 8;
    __device__ static __forceinline__ void decode(const DevView& v, const Raw<R>& r, int x, int y, float (&t)[C])
    {
        const float4* sp = reinterpret_cast<const float4*>(
            v.scales + ((size_t)(y >> v.scale_shift) * v.scale_tiles_x + (x >> v.scale_shift)) * 8);
        const float4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
        const float s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const __half2_raw h2 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(r.w[i] >> (16 * j)), __NV_E4M3);
                const float lo = __half2float(__half(__half_raw{h2.x}));
                const float hi = __half2float(__half(__half_raw{h2.y}));
                t[4 * i + 2 * j] = __fmul_rn(lo, s[4 * i + 2 * j]);
                t[4 * i + 2 * j + 1] = __fmul_rn(hi, s[4 * i + 2 * j + 1]);
            }
        }
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

template <> struct Mat<K_U8x4_F16x2> {
    static constexpr int C = 8, R = 8;  // 6 used; channels 6 and 7 read as 0
    __device__ static __forceinline__ void decode(const DevView& v, const Raw<R>& r, int, int, float (&t)[C])
    {
#pragma unroll
        for (int i = 0; i < 4; ++i) t[i] = __ldg(v.unorm_lut + ((r.w[0] >> (8 * i)) & 255u));
        t[4] = h2f(r.w[1] & 0xffffu);
        t[5] = h2f(r.w[1] >> 16);
        t[6] = 0.0f;
        t[7] = 0.0f;
    }
    __device__ static __forceinline__ void fetch(const DevView& v, int x, int y, float (&t)[C])
    {
        decode(v, ld_record<R>(v.texels, (size_t)y * v.tex_w + x), x, y, t);
    }
};

// ------------------------------------------------------------------------------ shading

// Lambert + GGX after filtering; see the interface header for the conventions. The GGX
// denominator uses a^2 (N.H)^2 + |N x H|^2 (equal to (N.H)^2 (a^2 - 1) + 1 for unit vectors),
// which keeps the specular peak well conditioned in FP32. With irradiance pi the specular term
// pi * D * Vis * F simplifies to a^2 F / (2 t^2 (g_v + g_l)), t = the GGX denominator.
// Every step is an explicitly rounded operation (a multiply, an add or a fused multiply-add) so
// that the compiler contracts nothing: the two-pixel packed version (shade2, one f32x2
// instruction per step) gives the same bits.
__device__ __forceinline__ float4 shade(const DevView& v, float r0, float r1, float r2, float nx, float ny,
                                        float rough, float ao, float u, float w)
{
    // tangent-space normal (X, Y, sqrt(1 - X^2 - Y^2)) has unit length unless |XY| > 1
    const float xy2 = fmaf(nx, nx, __fmul_rn(ny, ny));
    const float nz = sqrt_approx(fmaxf(__fadd_rn(1.0f, -xy2), 0.0f));
    const float inl = rsqrt_approx(fmaxf(xy2, 1.0f));
    const float N0 = __fmul_rn(nx, inl), N1 = __fmul_rn(nz, inl), N2 = __fmul_rn(ny, inl);  // world (x, y, z) = (T, N, B)
    const float P0 = fmaf(v.p2w[0], u, fmaf(v.p2w[1], w, v.p2w[2]));
    const float P2 = fmaf(v.p2w[3], u, fmaf(v.p2w[4], w, v.p2w[5]));
    float V0 = __fadd_rn(v.cam[0], -P0), V2 = __fadd_rn(v.cam[2], -P2);
    const float ivl = rsqrt_approx(fmaf(V0, V0, fmaf(v.cam[1], v.cam[1], __fmul_rn(V2, V2))));
    V0 = __fmul_rn(V0, ivl);
    const float V1 = __fmul_rn(v.cam[1], ivl);
    V2 = __fmul_rn(V2, ivl);
    const float L0 = v.light[0], L1 = v.light[1], L2 = v.light[2];
    const float NL = fmaf(N0, L0, fmaf(N1, L1, __fmul_rn(N2, L2)));
    const float NV = fmaxf(fmaf(N0, V0, fmaf(N1, V1, __fmul_rn(N2, V2))), 1e-4f);
    float H0 = __fadd_rn(L0, V0), H1 = __fadd_rn(L1, V1), H2 = __fadd_rn(L2, V2);
    const float ihl = rsqrt_approx(fmaf(H0, H0, fmaf(H1, H1, __fmul_rn(H2, H2))));
    H0 = __fmul_rn(H0, ihl); H1 = __fmul_rn(H1, ihl); H2 = __fmul_rn(H2, ihl);
    const float NH = fmaxf(fmaf(N0, H0, fmaf(N1, H1, __fmul_rn(N2, H2))), 0.0f);
    const float VH = fmaxf(fmaf(V0, H0, fmaf(V1, H1, __fmul_rn(V2, H2))), 0.0f);
    const float c0 = fmaf(N1, H2, -__fmul_rn(N2, H1)), c1 = fmaf(N2, H0, -__fmul_rn(N0, H2));
    const float c2 = fmaf(N0, H1, -__fmul_rn(N1, H0));
    const float s2 = fmaf(c0, c0, fmaf(c1, c1, __fmul_rn(c2, c2)));
    rough = fmaxf(rough, 0.02f);
    const float al = __fmul_rn(rough, rough);
    const float a2 = __fmul_rn(al, al);
    const float t = fmaf(__fmul_rn(a2, NH), NH, s2);
    const float ia2 = __fadd_rn(1.0f, -a2);
    const float NLp = fmaxf(NL, 0.0f);  // keeps g_v + g_l > 0 (and ps finite) when the pixel is unlit
    const float gv = __fmul_rn(NLp, sqrt_approx(fmaf(__fmul_rn(NV, NV), ia2, a2)));
    const float gl = __fmul_rn(NV, sqrt_approx(fmaf(__fmul_rn(NLp, NLp), ia2, a2)));
    const float q = __fadd_rn(1.0f, -VH);
    const float q2 = __fmul_rn(q, q);
    const float F = fmaf(0.96f, __fmul_rn(__fmul_rn(q2, q2), q), 0.04f);
    const float ps = __fdividef(__fmul_rn(__fmul_rn(0.5f, a2), F), __fmul_rn(__fmul_rn(t, t), __fadd_rn(gv, gl)));
    const float ka = __fmul_rn(ao, NL);
    const float k = NL > 0.0f ? ka : 0.0f;
    const float kp = __fmul_rn(k, ps);
    return make_float4(fmaf(k, r0, kp), fmaf(k, r1, kp), fmaf(k, r2, kp), 1.0f);
}

template <int C> __device__ __forceinline__ float pick_ch(const float (&f)[C], int idx)
{
    float r = 0.0f;
#pragma unroll
    for (int c = 0; c < C; ++c) r = (idx == c) ? f[c] : r;
    return r;
}

template <int C> __device__ __forceinline__ float4 finish_pixel(const DevView& v, const float (&f)[C], float u, float w)
{
    if (v.shade_layout == 0) {
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = (k < C && k < v.c_true) ? f[k < C ? k : 0] : (k == 3 ? 1.0f : 0.0f);
        return make_float4(o[0], o[1], o[2], o[3]);
    }
    if constexpr (C >= 7) {
        if (v.shade_layout == 1) return shade(v, f[0], f[1], f[2], f[3], f[4], f[5], f[6], u, w);
        if (v.shade_layout == 2) return shade(v, f[0], f[1], f[2], f[4], f[5], v.rough_const, 1.0f, u, w);
    }
    // generic channel map (uniform per view)
    const float r0 = v.ch_albedo >= 0 ? pick_ch(f, v.ch_albedo) : 1.0f;
    const float r1 = v.ch_albedo >= 0 ? pick_ch(f, v.ch_albedo + 1) : 1.0f;
    const float r2 = v.ch_albedo >= 0 ? pick_ch(f, v.ch_albedo + 2) : 1.0f;
    const float nx = v.ch_normal >= 0 ? pick_ch(f, v.ch_normal) : 0.0f;
    const float ny = v.ch_normal >= 0 ? pick_ch(f, v.ch_normal + 1) : 0.0f;
    const float ro = v.ch_rough >= 0 ? pick_ch(f, v.ch_rough) : v.rough_const;
    const float ao = v.ch_ao >= 0 ? pick_ch(f, v.ch_ao) : 1.0f;
    return shade(v, r0, r1, r2, nx, ny, ro, ao, u, w);
}

// ------------------------------------------------------------------------------ footprints

// Source-lane block of the sharing footprint (row-major kx x ky block at (ox, oy)); the same
// placement rule as the oracle: QUAD2 = aligned 2x2; WAVEk = ky = min(k, TH) rows,
// kx = min(TW, round(k^2 / ky)) columns, centred on the lane and shifted inside the tile.
template <int MODE, int TW, int TH> struct Footprint;
// Pseudorandom sparse footprints: 9 lanes per lane from a table (the shape constants are nominal).
template <int TW, int TH> struct Footprint<6, TW, TH> {
    static constexpr int KX = 9, KY = 1, N = 9;
    __device__ static __forceinline__ int base(int, int) { return 0; }
};
template <int MODE, int TW, int TH> struct Footprint {
    static constexpr int k = MODE == 3 ? 2 : (MODE == 4 ? 3 : (MODE == 5 ? 4 : 2));
    static constexpr int KY = MODE == 2 ? 2 : (k < TH ? k : TH);
    static constexpr int KXr = MODE == 2 ? 2 : (k * k + KY / 2) / KY;
    static constexpr int KX = KXr < TW ? KXr : TW;
    static constexpr int N = KX * KY;
    __device__ static __forceinline__ int base(int lx, int ly)
    {
        int ox, oy;
        if (MODE == 2) { ox = lx & ~1; oy = ly & ~1; }
        else {
            ox = min(max(lx - (KX - 1) / 2, 0), TW - KX);
            oy = min(max(ly - (KY - 1) / 2, 0), TH - KY);
        }
        return oy * TW + ox;
    }
};

}  // namespace stf
