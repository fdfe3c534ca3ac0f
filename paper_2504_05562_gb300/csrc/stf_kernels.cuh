// Render kernels of the stored material kinds. One warp renders one TW x TH pixel tile
// (lane = ly * TW + lx), which is the paper's wave-to-pixel mapping with linear row lane order
// (Section 2.3, Figure "wave"); texels are exchanged through per-warp shared-memory records, the
// CUDA counterpart of WaveReadLaneAt (Section 4.5). The neural kind has its own kernels
// (stf_nn_render.cuh).
#pragma once

#include <float.h>

#include "stf_device.cuh"

namespace stf {

constexpr unsigned kFull = 0xffffffffu;

template <int KIND> struct Channels { static constexpr int C = Mat<KIND>::C; };

// Fetch one texel of lattice point (x, y) with clamp-to-edge addressing.
template <int KIND>
__device__ __forceinline__ void fetch_texel(const DevView& v, int x, int y, float (&t)[Channels<KIND>::C])
{
    x = clampi(x, 0, v.tex_w - 1);
    y = clampi(y, 0, v.tex_h - 1);
    Mat<KIND>::fetch(v, x, y, t);
}

// Exact filtering (Section "Exact Filtering"), bilinear: `srcs` holds, per bilinear tap
// k = 2 ky + kx, 1 + the footprint lane whose sample is that tap's texel (0: none). If every tap of
// positive weight has one, the deterministic filter over those samples replaces the estimate,
// summed exactly as the full-filter mode sums (y outer, FMA per channel), so such a pixel equals
// the full filter bit for bit. REC(j, T) reads lane j's decoded channels.
template <int C, class REC>
__device__ __forceinline__ void exact_bilinear(const Axis<0>& ax, const Axis<0>& ay, uint32_t srcs, float (&res)[C], REC rec)
{
    bool all = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) all = all && (((srcs >> (8 * k)) & 0xffu) != 0u || __fmul_rn(ax.w[k & 1], ay.w[k >> 1]) == 0.0f);
    if (!all) return;
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float wt = __fmul_rn(ax.w[k & 1], ay.w[k >> 1]);
        const uint32_t j = (srcs >> (8 * k)) & 0xffu;
        float T[C];
        if (j) rec((int)j - 1, T);
        else
#pragma unroll
            for (int c = 0; c < C; ++c) T[c] = 0.0f;  // a zero-weight tap nobody drew
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(wt, T[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) res[c] = acc[c];
}

// W(d) for any lattice offset (the same value tap_weight gives for its own taps).
template <int F> __device__ __forceinline__ float w_any(float d)
{
    if constexpr (F == 0) return w_bilinear(d);
    const float a = fabsf(d);
    return a < 1.0f ? bspline_r1(a) : (a < 2.0f ? bspline_r2(a) : 0.0f);
}

// The alternative estimators (Section 4.1; an evaluation mode beside the weighted estimator) of
// lane `lane` over its footprint's records, each sum in footprint order with the operations
// rounded one by one: est & 7 = 1 importance sampling (1/n) sum f/p, 2 MIS balance heuristic
// sum f(x_i) / sum_k p_k(x_i), 3 pairwise MIS with the own sample canonical, 4 regression with
// the control variate h = w_c / p (mean 1); est & 8 clamps each channel to the range of the
// sampled texels the own filter weighs. Record 3 of a lane holds its (cx, cy, p).
template <int C, int F, class FP, int TW, int RPL>
__device__ __forceinline__ void alt_combine(int est, int lane, float cx, float cy, int b0, const float4* rec, float (&res)[C])
{
    constexpr int N = FP::N;
    const float nf = (float)N;
    int src[N];
    float pc[N], T[N][C];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        src[i] = b0 + (i / FP::KX) * TW + (i % FP::KX);
        const float4 m = rec[RPL * src[i]];
        pc[i] = __fmul_rn(w_any<F>(__fsub_rn(cx, m.x)), w_any<F>(__fsub_rn(cy, m.y)));
        const float4 t0 = rec[RPL * src[i] + 1];
        const float4 t1 = C > 4 ? rec[RPL * src[i] + 2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        const float tt[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int c = 0; c < C; ++c) T[i][c] = tt[c];
    }
    // lane j's PMF at sample i's texel
    auto pmf = [&](int j, int i) {
        const float4 q = rec[RPL * j + 3];
        const float4 m = rec[RPL * src[i]];
        return __fmul_rn(w_any<F>(__fsub_rn(q.x, m.x)), w_any<F>(__fsub_rn(q.y, m.y)));
    };
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.0f;
    const int kind = est & 7;
    if (kind == 1 || kind == 2 || kind == 3) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float pi = rec[RPL * src[i] + 3].z;
            float r;
            if (kind == 1) {
                r = __fdiv_rn(pc[i], pi);
            } else if (kind == 2) {
                float den = 0.0f;
#pragma unroll
                for (int k = 0; k < N; ++k) den = __fadd_rn(den, pmf(src[k], i));
                r = __fdiv_rn(pc[i], den);
            } else {
                const float m1 = nf - 1.0f;
                if (src[i] == lane) {
                    float mc = 0.0f;
#pragma unroll
                    for (int k = 0; k < N; ++k)
                        if (src[k] != lane) mc = __fadd_rn(mc, __fdiv_rn(pc[i], __fadd_rn(pc[i], __fmul_rn(m1, pmf(src[k], i)))));
                    r = __fdiv_rn(mc, m1);
                } else {
                    r = __fdiv_rn(pc[i], __fadd_rn(pc[i], __fmul_rn(m1, pi)));
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = __fadd_rn(acc[c], __fmul_rn(r, T[i][c]));
        }
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] = kind == 1 ? __fdiv_rn(acc[c], nf) : acc[c];
    } else {
        float h[N], hbar = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            h[i] = __fdiv_rn(pc[i], rec[RPL * src[i] + 3].z);
            hbar = __fadd_rn(hbar, h[i]);
        }
        hbar = __fdiv_rn(hbar, nf);
        float shh = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const float d = __fsub_rn(h[i], hbar);
            shh = __fadd_rn(shh, __fmul_rn(d, d));
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float sy = 0.0f, shy = 0.0f;
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const float y = __fmul_rn(h[i], T[i][c]);
                sy = __fadd_rn(sy, y);
                shy = __fadd_rn(shy, __fmul_rn(__fsub_rn(h[i], hbar), y));
            }
            const float beta = shh > 0.0f ? __fdiv_rn(shy, shh) : 0.0f;
            res[c] = __fsub_rn(__fdiv_rn(sy, nf), __fmul_rn(beta, __fsub_rn(hbar, 1.0f)));
        }
    }
    if (est & 8) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float lo = INFINITY, hi = -INFINITY;
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (pc[i] > 0.0f) { lo = fminf(lo, T[i][c]); hi = fmaxf(hi, T[i][c]); }
            res[c] = fminf(fmaxf(res[c], lo), hi);
        }
    }
}

// One warp tile of one view. MODE: 0 full filter, 1 one-tap, 2 quad 2x2, 3..5 wave k x k; EX:
// exact filtering (bilinear sharing modes only); ALT: the alternative estimators instead of the
// weighted one (v.estimator).
// All 32 lanes execute every shuffle (off-screen lanes of a partial tile compute with
// extrapolated coordinates and only skip the store).
template <int KIND, int F, int MODE, int TW, int TH, bool EX = false, bool ALT = false, bool BLUE = false>
__device__ __forceinline__ void render_tile(const DevView& v, int tx, int ty, int lane, float4* rec, float* wtab)
{
    constexpr int C = Channels<KIND>::C;
    constexpr int RPL = ALT ? 4 : 3;  // records per lane (ALT adds the lane's coordinates and p)
    const int lx = lane % TW, ly = lane / TW;
    const int x = tx * TW + lx, y = ty * TH + ly;
    float u, w;
    pixel_uv(v, x, y, u, w);
    const float cx = texel_coord(u, v.tex_wf);
    const float cy = texel_coord(w, v.tex_hf);
    float res[C];
    uint32_t pk = 0;

    if constexpr (MODE == 0) {
        // deterministic filter: sum over taps of W(dx) W(dy) T, y outer (Eq. texture-continuous-sum)
        Axis<F> ax, ay;
        axis_weights<F>(cx, ax);
        axis_weights<F>(cy, ay);
#pragma unroll
        for (int c = 0; c < C; ++c) res[c] = 0.0f;
#pragma unroll
        for (int s = 0; s < Taps<F>::N; ++s) {
#pragma unroll
            for (int t = 0; t < Taps<F>::N; ++t) {
                const float wt = __fmul_rn(ax.w[t], ay.w[s]);
                float T[C];
                fetch_texel<KIND>(v, ax.base + t, ay.base + s, T);
#pragma unroll
                for (int c = 0; c < C; ++c) res[c] = fmaf(wt, T[c], res[c]);
            }
        }
    } else {
        // one-tap STF: one texel drawn from the lane's own filter PMF (Section 2.2, Section S1)
        float ux, uy;
        pixel_uniforms<BLUE>(v, x, y, ux, uy);
        Axis<F> ax, ay;
        axis_select<F>(cx, ux, ax);
        axis_select<F>(cy, uy, ay);
        const float p = __fmul_rn(ax.p, ay.p);
        float T[C];
        fetch_texel<KIND>(v, ax.n, ay.n, T);
        pk = pack_idx(ax.n, ay.n);
        if constexpr (MODE == 1) {
#pragma unroll
            for (int c = 0; c < C; ++c) res[c] = T[c];
        } else {
            // sharing over the lane's footprint with w_j = f_c(x_j) / f_j(x_j) (Eq. estimator-
            // for-stf, Section 4.5 listing); the own lane's weight is exactly 1, texels outside
            // the own filter weigh 0. Each lane publishes (texel coordinates, 1 / p, decoded texel)
            // in its warp's shared-memory records; the footprint lanes' records are then read with
            // 128-bit loads, the shared-memory form of WaveReadLaneAt.
            using FP = Footprint<MODE, TW, TH>;
            static_assert(C % 2 == 0 && C <= 8, "channels are accumulated in pairs, at most 8");
            // 1 / p_j once per owner; rcp.approx of a denormal p flushes to +inf, clamped so that a
            // zero p_c still gives a zero weight
            const float rinv = fminf(rcp_approx(p), FLT_MAX);
            rec[RPL * lane] = make_float4(ax.nf, ay.nf, rinv, __uint_as_float(pk));
            if constexpr (ALT) rec[RPL * lane + 3] = make_float4(cx, cy, p, 0.0f);
            rec[RPL * lane + 1] = make_float4(T[0], T[1], C > 2 ? T[2 % C] : 0.0f, C > 3 ? T[3 % C] : 0.0f);
            if constexpr (C > 4) rec[RPL * lane + 2] = make_float4(T[4 % C], T[5 % C], T[6 % C], T[7 % C]);
            if constexpr (F == 1) {
                // this lane's tap weights, one column per lane (conflict-free indexed reads)
#pragma unroll
                for (int t = 0; t < 4; ++t) { wtab[t * 32 + lane] = ax.w[t]; wtab[(4 + t) * 32 + lane] = ay.w[t]; }
            }
            __syncwarp();
            const int b0 = FP::base(lx, ly);
            if constexpr (ALT) {
                alt_combine<C, F, FP, TW, RPL>(v.estimator, lane, cx, cy, b0, rec, res);
            } else {
                float2 acc[C / 2];
#pragma unroll
                for (int c = 0; c < C / 2; ++c) acc[c] = make_float2(0.0f, 0.0f);
                float wsum = 0.0f;
                uint32_t srcs = 0;  // exact filtering: per bilinear tap, 1 + a lane holding its texel
                // one footprint element: lane src's record
                auto visit = [&](int src) {
                    const float4 m = rec[RPL * src];
                    float wx, wy;
                    if constexpr (F == 0) {  // W(c - n) evaluated as the oracle does
                        wx = w_bilinear(__fsub_rn(cx, m.x));
                        wy = w_bilinear(__fsub_rn(cy, m.y));
                        if constexpr (EX) {
                            const uint32_t pj = __float_as_uint(m.w);
                            const int kx = unpack_x(pj) - ax.base, ky = unpack_y(pj) - ay.base;
                            if (((kx | ky) & ~1) == 0) {
                                const int sh = 8 * (2 * ky + kx);
                                srcs = (srcs & ~(0xffu << sh)) | ((uint32_t)(src + 1) << sh);
                            }
                        }
                    } else {
                        // the same values read from this lane's taps: lattice points outside the
                        // taps have zero weight
                        const uint32_t pj = __float_as_uint(m.w);
                        const int kx = unpack_x(pj) - ax.base, ky = unpack_y(pj) - ay.base;
                        const bool in = ((kx | ky) & ~3) == 0;
                        wx = in ? wtab[kx * 32 + lane] : 0.0f;
                        wy = in ? wtab[(4 + ky) * 32 + lane] : 0.0f;
                    }
                    const float wt = (src == lane) ? 1.0f : (wx * wy) * m.z;
                    const float2 w2 = make_float2(wt, wt);
                    const float4 t0 = rec[RPL * src + 1];
                    acc[0] = __ffma2_rn(w2, make_float2(t0.x, t0.y), acc[0]);
                    if constexpr (C > 2) acc[1 % (C / 2)] = __ffma2_rn(w2, make_float2(t0.z, t0.w), acc[1 % (C / 2)]);
                    if constexpr (C > 4) {
                        const float4 t1 = rec[RPL * src + 2];
                        acc[2 % (C / 2)] = __ffma2_rn(w2, make_float2(t1.x, t1.y), acc[2 % (C / 2)]);
                        acc[3 % (C / 2)] = __ffma2_rn(w2, make_float2(t1.z, t1.w), acc[3 % (C / 2)]);
                    }
                    wsum += wt;
                };
                if constexpr (MODE == kModeSparse9) {
                    // the lane's row of the frame's sparse footprint pattern (own lane first)
                    const uint4 row = __ldg(reinterpret_cast<const uint4*>(v.fp) + lane);
                    const uint32_t w4[4] = {row.x, row.y, row.z, row.w};
#pragma unroll
                    for (int i = 0; i < 9; ++i) visit((int)((w4[i >> 2] >> (8 * (i & 3))) & 0x1fu));
                } else {
#pragma unroll
                    for (int r = 0; r < FP::KY; ++r)
#pragma unroll
                        for (int q = 0; q < FP::KX; ++q) visit(b0 + r * TW + q);
                }
                const float inv = rcp_approx(wsum);
#pragma unroll
                for (int c = 0; c < C / 2; ++c) { res[2 * c] = acc[c].x * inv; res[2 * c + 1] = acc[c].y * inv; }
                if constexpr (EX && F == 0)
                    exact_bilinear<C>(ax, ay, srcs, res, [&](int j, float (&T)[C]) {
                        const float4 t0 = rec[RPL * j + 1];
                        const float4 t1 = C > 4 ? rec[RPL * j + 2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        const float tt[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                        for (int c = 0; c < C; ++c) T[c] = tt[c];
                    });
            }
            __syncwarp();  // records are rewritten by the warp's next tile
        }
    }

    if (x < v.width && y < v.height) {
        const float4 o = finish_pixel<C>(v, res, u, w);
        __stcs(reinterpret_cast<float4*>(v.out + (size_t)y * v.pitch + 4 * (size_t)x), o);
        const size_t pix = (size_t)y * v.width + x;
        if (v.dbg_idx) v.dbg_idx[pix] = pk;
        if (v.dbg_ch) {
            float4* d = reinterpret_cast<float4*>(v.dbg_ch + pix * 8);
            float z[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) z[c] = (c < C && c < v.c_true) ? res[c < C ? c : 0] : 0.0f;
            d[0] = make_float4(z[0], z[1], z[2], z[3]);
            d[1] = make_float4(z[4], z[5], z[6], z[7]);
        }
    }
}


// Shared-memory sample records: 3 x 16 bytes per lane (texel coordinates and 1/p, then up to 8
// decoded channels); the 48-byte stride keeps 128-bit reads of neighbouring lanes conflict-free.
constexpr int kRecPerLane = 3;

// Blocks resident per SM the multi-view kernel (8-warp blocks) is compiled for (caps registers
// per thread at 65536 / (256 n)): five blocks (<= 51 registers) keep the issue-bound texture
// kinds at 40 warps per SM.
constexpr int kMinBlocks = 5;

// The single-view kernel runs 4-warp blocks, ten resident per SM (<= 51 registers): the same 40
// warps per SM as 8-warp blocks, but a block's slot frees sooner when its warps finish unevenly
// (measured 3-5 % faster on the 4K frame).
constexpr int kViewWarps = 4;
constexpr int kViewMinBlocks = 10;

// One view: block (bx, by) holds kViewWarps warps on tile row by, tiles bx * kViewWarps + warp.
template <int KIND, int F, int MODE, int TW, int TH, bool EX = false, bool ALT = false, bool BLUE = false>
__global__ void __launch_bounds__(32 * kViewWarps, kViewMinBlocks) k_render_view(const DevView v)
{
    constexpr int RPL = ALT ? 4 : kRecPerLane;
    __shared__ float4 recs[kViewWarps * 32 * RPL];
    __shared__ float wtabs[kViewWarps * 32 * 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = blockIdx.x * kViewWarps + warp;
    if (tx >= v.tiles_x) return;  // warp-uniform
    render_tile<KIND, F, MODE, TW, TH, EX, ALT, BLUE>(v, tx, blockIdx.y, lane, recs + warp * 32 * RPL, wtabs + warp * 32 * 8);
}

}  // namespace stf
