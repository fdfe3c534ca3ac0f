// Paired-pixel render path of the stored material kinds: each thread renders the two vertically
// adjacent pixels (lx, 2r) and (lx, 2r + 1) of a TW x TH warp tile, and a warp renders two tiles
// (one per half-warp). The method is unchanged: the tile is still the paper's 32-lane wave
// (Section 2.3, Section 4.3), every pixel draws its own texel, and each pixel's estimate reads
// the records of its own sharing footprint. Two things get cheaper:
//   - where the two pixels of a pair have the same footprint window (every vertical pair of
//     one-tap, full filtering, QUAD2, and of WAVEk when k covers the tile's height or the
//     window's clamping lines up, as for WAVE3 in 8 x 4 tiles), each footprint record is read
//     from shared memory once for both pixels: half the shared-memory wavefronts of the
//     one-pixel-per-thread path, which the sharing step saturates;
//   - the two pixels' colour work runs as packed f32x2 instructions (FADD2, FMUL2, FFMA2):
//     shading, and the neighbour weights and channel sums of the sharing loop.
// The texel choice keeps the oracle's operation order exactly: coordinates and the per-axis
// selection run per pixel with the scalar, explicitly rounded helpers (a chained packed
// homography was seen to differ from the scalar chain, so the bit-exact path does not use it).
// Variants: hash or blue-noise uniforms (BLUE), and exact filtering of the bilinear filter (EX).
#pragma once

#include <cuda.h>

#include "stf_kernels.cuh"

namespace stf {

// Packed f32x2 arithmetic, each element rounded once to nearest. The operations are written in
// PTX with the explicit .rn modifier, which the compiler never contracts: a multiply followed by
// an add stays two roundings, exactly as the oracle and the scalar __fmul_rn / __fadd_rn steps.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ unsigned long long pk2(float2 a) { return *reinterpret_cast<const unsigned long long*>(&a); }
__device__ __forceinline__ float2 up2(unsigned long long a) { return *reinterpret_cast<const float2*>(&a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
    return up2(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
    return up2(d);
}
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// Whether the pixels of every vertical pair (rows 2r and 2r + 1) of a TW x TH tile share one
// footprint window in sharing mode MODE (always without sharing).
template <int MODE, int TW, int TH> __host__ __device__ constexpr bool pair_rows_share()
{
    if (MODE <= 2) return TH % 2 == 0;
    if (MODE == kModeSparse9 || MODE > 5 || TH % 2 != 0) return false;
    using FP = Footprint<MODE, TW, TH>;
    for (int ly = 0; ly < TH; ly += 2) {
        int o0 = ly - (FP::KY - 1) / 2, o1 = ly + 1 - (FP::KY - 1) / 2;
        o0 = o0 < 0 ? 0 : (o0 > TH - FP::KY ? TH - FP::KY : o0);
        o1 = o1 < 0 ? 0 : (o1 > TH - FP::KY ? TH - FP::KY : o1);
        if (o0 != o1) return false;
    }
    return true;
}

// The paired path covers the stored kinds with the weighted estimator, with hash or blue-noise
// uniforms, with or without exact filtering of the bilinear filter; everything else (the
// alternative estimators, the neural material) renders one pixel per thread.
template <int KIND, int F, int MODE, int TW, int TH, bool EX, bool ALT, bool BLUE>
__host__ __device__ constexpr bool pair_path()
{
    return KIND != K_NEURAL && (!EX || F == 0) && !ALT && pair_rows_share<MODE, TW, TH>();
}

// pixel_uv / texel_coord for the pixels (x, y) and (x, y + 1), the same rounded steps per element.
__device__ __forceinline__ void pixel_uv2(const DevView& v, int x, int y, float2& u, float2& w)
{
    const float px = __fadd_rn(__int2float_rn(x), 0.5f);
    const float2 py = make_float2(__fadd_rn(__int2float_rn(y), 0.5f), __fadd_rn(__int2float_rn(y + 1), 0.5f));
    const float2 hx = add2(add2(f2(__fmul_rn(v.H[0], px)), mul2(f2(v.H[1]), py)), f2(v.H[2]));
    const float2 hy = add2(add2(f2(__fmul_rn(v.H[3], px)), mul2(f2(v.H[4]), py)), f2(v.H[5]));
    if (v.affine) {
        u = hx;
        w = hy;
        return;
    }
    const float2 hw = add2(add2(f2(__fmul_rn(v.H[6], px)), mul2(f2(v.H[7]), py)), f2(v.H[8]));
    u = make_float2(__fdiv_rn(hx.x, hw.x), __fdiv_rn(hx.y, hw.y));
    w = make_float2(__fdiv_rn(hy.x, hw.x), __fdiv_rn(hy.y, hw.y));
}

__device__ __forceinline__ float2 texel_coord2(float2 uv, float size)
{
    const float2 c = add2(mul2(uv, f2(size)), f2(-0.5f));  // x - 0.5 == x + (-0.5) in IEEE arithmetic
    return make_float2(fminf(fmaxf(c.x, kCoordLo), kCoordHi), fminf(fmaxf(c.y, kCoordLo), kCoordHi));
}

// shade() for two pixels, packed: the same formula and operation order per element.
__device__ __forceinline__ void shade2(const DevView& v, float2 r0, float2 r1, float2 r2, float2 nx, float2 ny,
                                       float2 rough, float2 ao, float2 u, float2 w, float4& o0, float4& o1)
{
    const float2 xy2 = fma2(nx, nx, mul2(ny, ny));
    const float2 omx = add2(f2(1.0f), neg2(xy2));
    const float2 nz = make_float2(sqrt_approx(fmaxf(omx.x, 0.0f)), sqrt_approx(fmaxf(omx.y, 0.0f)));
    const float2 inl = make_float2(rsqrt_approx(fmaxf(xy2.x, 1.0f)), rsqrt_approx(fmaxf(xy2.y, 1.0f)));
    const float2 N0 = mul2(nx, inl), N1 = mul2(nz, inl), N2 = mul2(ny, inl);
    const float2 P0 = fma2(f2(v.p2w[0]), u, fma2(f2(v.p2w[1]), w, f2(v.p2w[2])));
    const float2 P2 = fma2(f2(v.p2w[3]), u, fma2(f2(v.p2w[4]), w, f2(v.p2w[5])));
    float2 V0 = add2(f2(v.cam[0]), neg2(P0)), V2 = add2(f2(v.cam[2]), neg2(P2));
    const float2 V1c = f2(v.cam[1]);
    const float2 vl = fma2(V0, V0, fma2(V1c, V1c, mul2(V2, V2)));
    const float2 ivl = make_float2(rsqrt_approx(vl.x), rsqrt_approx(vl.y));
    V0 = mul2(V0, ivl);
    const float2 V1 = mul2(V1c, ivl);
    V2 = mul2(V2, ivl);
    const float2 L0 = f2(v.light[0]), L1 = f2(v.light[1]), L2 = f2(v.light[2]);
    const float2 NL = fma2(N0, L0, fma2(N1, L1, mul2(N2, L2)));
    const float2 nv = fma2(N0, V0, fma2(N1, V1, mul2(N2, V2)));
    const float2 NV = make_float2(fmaxf(nv.x, 1e-4f), fmaxf(nv.y, 1e-4f));
    float2 H0 = add2(L0, V0), H1 = add2(L1, V1), H2 = add2(L2, V2);
    const float2 hl = fma2(H0, H0, fma2(H1, H1, mul2(H2, H2)));
    const float2 ihl = make_float2(rsqrt_approx(hl.x), rsqrt_approx(hl.y));
    H0 = mul2(H0, ihl); H1 = mul2(H1, ihl); H2 = mul2(H2, ihl);
    const float2 nh = fma2(N0, H0, fma2(N1, H1, mul2(N2, H2)));
    const float2 vh = fma2(V0, H0, fma2(V1, H1, mul2(V2, H2)));
    const float2 NH = make_float2(fmaxf(nh.x, 0.0f), fmaxf(nh.y, 0.0f));
    const float2 VH = make_float2(fmaxf(vh.x, 0.0f), fmaxf(vh.y, 0.0f));
    const float2 c0 = fma2(N1, H2, neg2(mul2(N2, H1)));
    const float2 c1 = fma2(N2, H0, neg2(mul2(N0, H2)));
    const float2 c2 = fma2(N0, H1, neg2(mul2(N1, H0)));
    const float2 s2 = fma2(c0, c0, fma2(c1, c1, mul2(c2, c2)));
    rough = make_float2(fmaxf(rough.x, 0.02f), fmaxf(rough.y, 0.02f));
    const float2 al = mul2(rough, rough);
    const float2 a2 = mul2(al, al);
    const float2 t = fma2(mul2(a2, NH), NH, s2);
    const float2 ia2 = add2(f2(1.0f), neg2(a2));
    const float2 NLp = make_float2(fmaxf(NL.x, 0.0f), fmaxf(NL.y, 0.0f));
    const float2 qv = fma2(mul2(NV, NV), ia2, a2), ql = fma2(mul2(NLp, NLp), ia2, a2);
    const float2 gv = mul2(NLp, make_float2(sqrt_approx(qv.x), sqrt_approx(qv.y)));
    const float2 gl = mul2(NV, make_float2(sqrt_approx(ql.x), sqrt_approx(ql.y)));
    const float2 q = add2(f2(1.0f), neg2(VH));
    const float2 q2 = mul2(q, q);
    const float2 Fr = fma2(f2(0.96f), mul2(mul2(q2, q2), q), f2(0.04f));
    const float2 num = mul2(mul2(f2(0.5f), a2), Fr);
    const float2 den = mul2(mul2(t, t), add2(gv, gl));
    const float2 ps = make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    const float2 ka = mul2(ao, NL);
    const float2 k = make_float2(NL.x > 0.0f ? ka.x : 0.0f, NL.y > 0.0f ? ka.y : 0.0f);
    const float2 kp = mul2(k, ps);
    const float2 R = fma2(k, r0, kp), G = fma2(k, r1, kp), B = fma2(k, r2, kp);
    o0 = make_float4(R.x, G.x, B.x, 1.0f);
    o1 = make_float4(R.y, G.y, B.y, 1.0f);
}

// finish_pixel() for two pixels: unshaded channels 0..3, or the view's shading channel map.
template <int C>
__device__ __forceinline__ void finish_pair(const DevView& v, const float (&a)[C], const float (&b)[C], float2 u,
                                            float2 w, float4& o0, float4& o1)
{
    if (v.shade_layout == 0) {
        o0 = finish_pixel<C>(v, a, u.x, w.x);
        o1 = finish_pixel<C>(v, b, u.y, w.y);
        return;
    }
    auto P = [&](int c) { return make_float2(pick_ch(a, c), pick_ch(b, c)); };
    if constexpr (C >= 7) {
        if (v.shade_layout == 1) {
            shade2(v, make_float2(a[0], b[0]), make_float2(a[1], b[1]), make_float2(a[2], b[2]), make_float2(a[3], b[3]),
                   make_float2(a[4], b[4]), make_float2(a[5], b[5]), make_float2(a[6], b[6]), u, w, o0, o1);
            return;
        }
        if (v.shade_layout == 2) {
            shade2(v, make_float2(a[0], b[0]), make_float2(a[1], b[1]), make_float2(a[2], b[2]), make_float2(a[4], b[4]),
                   make_float2(a[5], b[5]), f2(v.rough_const), f2(1.0f), u, w, o0, o1);
            return;
        }
    }
    const float2 r0 = v.ch_albedo >= 0 ? P(v.ch_albedo) : f2(1.0f);
    const float2 r1 = v.ch_albedo >= 0 ? P(v.ch_albedo + 1) : f2(1.0f);
    const float2 r2 = v.ch_albedo >= 0 ? P(v.ch_albedo + 2) : f2(1.0f);
    const float2 nx = v.ch_normal >= 0 ? P(v.ch_normal) : f2(0.0f);
    const float2 ny = v.ch_normal >= 0 ? P(v.ch_normal + 1) : f2(0.0f);
    const float2 ro = v.ch_rough >= 0 ? P(v.ch_rough) : f2(v.rough_const);
    const float2 ao = v.ch_ao >= 0 ? P(v.ch_ao) : f2(1.0f);
    shade2(v, r0, r1, r2, nx, ny, ro, ao, u, w, o0, o1);
}

// Output and debug stores of one pixel (skipped off screen).
template <int C>
__device__ __forceinline__ void store_pixel(const DevView& v, int x, int y, float4 o, uint32_t pk, const float (&res)[C])
{
    if (x >= v.width || y >= v.height) return;
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

// Texel fetch with clamp-to-edge addressing from global memory (the read-only path).
template <int KIND> struct GlobalFetch {
    const DevView& v;
    __device__ __forceinline__ void operator()(int x, int y, float (&t)[Channels<KIND>::C]) const { fetch_texel<KIND>(v, x, y, t); }
};

// One pair of pixels of one warp tile: hl in [0, 16) picks column hl % TW and rows 2 (hl / TW)
// and 2 (hl / TW) + 1; rec holds the tile's 32 lane records (3 x 16 bytes each), wtab (B-spline)
// its lanes' tap weights, fetch reads a texel (clamp-to-edge). All 16 threads of the half-warp
// (and of the whole warp) execute every shared-memory step. BLUE: the selection uniforms come
// from the blue-noise masks; EX: a pixel whose window holds all four of its bilinear taps
// returns the full filter over those records (Section 4.2's exact filtering).
template <int KIND, int F, int MODE, int TW, int TH, bool BLUE = false, bool EX = false, class FETCH = GlobalFetch<KIND>>
__device__ __forceinline__ void render_pair(const DevView& v, int tx, int ty, int hl, float4* rec, float* wtab,
                                            bool live, const FETCH& fetch)
{
    constexpr int C = Channels<KIND>::C;
    const int lx = hl % TW, ly = 2 * (hl / TW);
    const int x = tx * TW + lx, y = ty * TH + ly;
    float2 u, w;
    pixel_uv(v, x, y, u.x, w.x);
    pixel_uv(v, x, y + 1, u.y, w.y);
    const float2 cx = make_float2(texel_coord(u.x, v.tex_wf), texel_coord(u.y, v.tex_wf));
    const float2 cy = make_float2(texel_coord(w.x, v.tex_hf), texel_coord(w.y, v.tex_hf));
    float ra[C], rb[C];
    uint32_t pka = 0, pkb = 0;

    if constexpr (MODE == 0) {
        // deterministic filter of both pixels: y outer, x inner, one FMA per channel and tap
        Axis<F> xa, ya, xb, yb;
        axis_weights<F>(cx.x, xa);
        axis_weights<F>(cy.x, ya);
        axis_weights<F>(cx.y, xb);
        axis_weights<F>(cy.y, yb);
#pragma unroll
        for (int c = 0; c < C; ++c) { ra[c] = 0.0f; rb[c] = 0.0f; }
#pragma unroll
        for (int s = 0; s < Taps<F>::N; ++s) {
#pragma unroll
            for (int t = 0; t < Taps<F>::N; ++t) {
                const float2 wt = mul2(make_float2(xa.w[t], xb.w[t]), make_float2(ya.w[s], yb.w[s]));
                float Ta[C], Tb[C];
                fetch(xa.base + t, ya.base + s, Ta);
                fetch(xb.base + t, yb.base + s, Tb);
#pragma unroll
                for (int c = 0; c < C; c += 2) {
                    const float2 pa = fma2(f2(wt.x), make_float2(Ta[c], Ta[c + 1]), make_float2(ra[c], ra[c + 1]));
                    const float2 pb = fma2(f2(wt.y), make_float2(Tb[c], Tb[c + 1]), make_float2(rb[c], rb[c + 1]));
                    ra[c] = pa.x; ra[c + 1] = pa.y; rb[c] = pb.x; rb[c + 1] = pb.y;
                }
            }
        }
    } else {
        // one-tap STF per pixel (Section 2.2, Section S1)
        float uxa, uya, uxb, uyb;
        pixel_uniforms<BLUE>(v, x, y, uxa, uya);
        pixel_uniforms<BLUE>(v, x, y + 1, uxb, uyb);
        Axis<F> xa, ya, xb, yb;
        axis_select<F>(cx.x, uxa, xa);
        axis_select<F>(cy.x, uya, ya);
        axis_select<F>(cx.y, uxb, xb);
        axis_select<F>(cy.y, uyb, yb);
        const float2 p = mul2(make_float2(xa.p, xb.p), make_float2(ya.p, yb.p));
        float Ta[C], Tb[C];
        fetch(xa.n, ya.n, Ta);
        fetch(xb.n, yb.n, Tb);
        pka = pack_idx(xa.n, ya.n);
        pkb = pack_idx(xb.n, yb.n);
        if constexpr (MODE == 1) {
#pragma unroll
            for (int c = 0; c < C; ++c) { ra[c] = Ta[c]; rb[c] = Tb[c]; }
        } else {
            // sharing over the pair's common footprint window with w_j = f_c(x_j) / f_j(x_j)
            // (Eq. estimator-for-stf, Section 4.5 loop): both pixels publish (texel coordinates,
            // 1 / p, decoded texel) records, then every window record is read once and weighed
            // for both pixels; a pixel's own record weighs exactly 1
            using FP = Footprint<MODE, TW, TH>;
            static_assert(C % 2 == 0 && C <= 8, "channels are accumulated in pairs, at most 8");
            const int la = ly * TW + lx, lb = la + TW;
            const float2 rinv = make_float2(fminf(rcp_approx(p.x), FLT_MAX), fminf(rcp_approx(p.y), FLT_MAX));
            rec[kRecPerLane * la] = make_float4(xa.nf, ya.nf, rinv.x, __uint_as_float(pka));
            rec[kRecPerLane * lb] = make_float4(xb.nf, yb.nf, rinv.y, __uint_as_float(pkb));
            rec[kRecPerLane * la + 1] = make_float4(Ta[0], Ta[1], C > 2 ? Ta[2 % C] : 0.0f, C > 3 ? Ta[3 % C] : 0.0f);
            rec[kRecPerLane * lb + 1] = make_float4(Tb[0], Tb[1], C > 2 ? Tb[2 % C] : 0.0f, C > 3 ? Tb[3 % C] : 0.0f);
            if constexpr (C > 4) {
                rec[kRecPerLane * la + 2] = make_float4(Ta[4 % C], Ta[5 % C], Ta[6 % C], Ta[7 % C]);
                rec[kRecPerLane * lb + 2] = make_float4(Tb[4 % C], Tb[5 % C], Tb[6 % C], Tb[7 % C]);
            }
            if constexpr (F == 1) {
                // both pixels' tap weights, one column per lane (conflict-free indexed reads)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    wtab[t * 32 + la] = xa.w[t]; wtab[(4 + t) * 32 + la] = ya.w[t];
                    wtab[t * 32 + lb] = xb.w[t]; wtab[(4 + t) * 32 + lb] = yb.w[t];
                }
            }
            __syncwarp();
            const int b0 = FP::base(lx, ly);  // the same window for rows ly and ly + 1
            float2 acca[C / 2], accb[C / 2];
#pragma unroll
            for (int c = 0; c < C / 2; ++c) { acca[c] = f2(0.0f); accb[c] = f2(0.0f); }
            float2 wsum = f2(0.0f);
            uint32_t srcsa = 0, srcsb = 0;  // exact filtering: per bilinear tap, 1 + a lane holding its texel
#pragma unroll
            for (int r = 0; r < FP::KY; ++r) {
#pragma unroll
                for (int q = 0; q < FP::KX; ++q) {
                    const int src = b0 + r * TW + q;
                    const float4 m = rec[kRecPerLane * src];
                    float2 wx, wy;
                    if constexpr (F == 0) {  // W(c - n) evaluated as the oracle does
                        const float2 dx = add2(cx, f2(-m.x)), dy = add2(cy, f2(-m.y));
                        wx = make_float2(w_bilinear(dx.x), w_bilinear(dx.y));
                        wy = make_float2(w_bilinear(dy.x), w_bilinear(dy.y));
                        if constexpr (EX) {
                            const uint32_t pj = __float_as_uint(m.w);
                            const int kxa = unpack_x(pj) - xa.base, kya = unpack_y(pj) - ya.base;
                            const int kxb = unpack_x(pj) - xb.base, kyb = unpack_y(pj) - yb.base;
                            if (((kxa | kya) & ~1) == 0) {
                                const int sh = 8 * (2 * kya + kxa);
                                srcsa = (srcsa & ~(0xffu << sh)) | ((uint32_t)(src + 1) << sh);
                            }
                            if (((kxb | kyb) & ~1) == 0) {
                                const int sh = 8 * (2 * kyb + kxb);
                                srcsb = (srcsb & ~(0xffu << sh)) | ((uint32_t)(src + 1) << sh);
                            }
                        }
                    } else {
                        // the same values read from each pixel's taps: lattice points outside the
                        // taps have zero weight
                        const uint32_t pj = __float_as_uint(m.w);
                        const int kxa = unpack_x(pj) - xa.base, kya = unpack_y(pj) - ya.base;
                        const int kxb = unpack_x(pj) - xb.base, kyb = unpack_y(pj) - yb.base;
                        const bool ina = ((kxa | kya) & ~3) == 0, inb = ((kxb | kyb) & ~3) == 0;
                        wx = make_float2(ina ? wtab[kxa * 32 + la] : 0.0f, inb ? wtab[kxb * 32 + lb] : 0.0f);
                        wy = make_float2(ina ? wtab[(4 + kya) * 32 + la] : 0.0f, inb ? wtab[(4 + kyb) * 32 + lb] : 0.0f);
                    }
                    float2 wt = mul2(mul2(wx, wy), f2(m.z));
                    wt.x = src == la ? 1.0f : wt.x;
                    wt.y = src == lb ? 1.0f : wt.y;
                    wsum = add2(wsum, wt);
                    const float4 t0 = rec[kRecPerLane * src + 1];
                    acca[0] = fma2(f2(wt.x), make_float2(t0.x, t0.y), acca[0]);
                    accb[0] = fma2(f2(wt.y), make_float2(t0.x, t0.y), accb[0]);
                    if constexpr (C > 2) {
                        acca[1 % (C / 2)] = fma2(f2(wt.x), make_float2(t0.z, t0.w), acca[1 % (C / 2)]);
                        accb[1 % (C / 2)] = fma2(f2(wt.y), make_float2(t0.z, t0.w), accb[1 % (C / 2)]);
                    }
                    if constexpr (C > 4) {
                        const float4 t1 = rec[kRecPerLane * src + 2];
                        acca[2 % (C / 2)] = fma2(f2(wt.x), make_float2(t1.x, t1.y), acca[2 % (C / 2)]);
                        accb[2 % (C / 2)] = fma2(f2(wt.y), make_float2(t1.x, t1.y), accb[2 % (C / 2)]);
                        acca[3 % (C / 2)] = fma2(f2(wt.x), make_float2(t1.z, t1.w), acca[3 % (C / 2)]);
                        accb[3 % (C / 2)] = fma2(f2(wt.y), make_float2(t1.z, t1.w), accb[3 % (C / 2)]);
                    }
                }
            }
            const float ia = rcp_approx(wsum.x), ib = rcp_approx(wsum.y);
#pragma unroll
            for (int c = 0; c < C / 2; ++c) {
                const float2 qa = mul2(acca[c], f2(ia)), qb = mul2(accb[c], f2(ib));
                ra[2 * c] = qa.x; ra[2 * c + 1] = qa.y;
                rb[2 * c] = qb.x; rb[2 * c + 1] = qb.y;
            }
            if constexpr (EX && F == 0) {
                // exact filtering (Section 4.2): a pixel whose four bilinear taps were all drawn in
                // its window gets the full filter from those records instead of the estimate
                auto rec_texel = [&](int j, float (&T)[C]) {
                    const float4 t0 = rec[kRecPerLane * j + 1];
                    const float4 t1 = C > 4 ? rec[kRecPerLane * j + 2] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    const float tt[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
                    for (int c = 0; c < C; ++c) T[c] = tt[c];
                };
                exact_bilinear<C>(xa, ya, srcsa, ra, rec_texel);
                exact_bilinear<C>(xb, yb, srcsb, rb, rec_texel);
            }
            __syncwarp();  // records are rewritten by the warp's next tiles
        }
    }
    if (!live) return;  // a stand-in tile that only keeps its half-warp in step
    float4 oa, ob;
    finish_pair<C>(v, ra, rb, u, w, oa, ob);
    store_pixel<C>(v, x, y, oa, pka, ra);
    store_pixel<C>(v, x, y + 1, ob, pkb, rb);
}

// Warps per block of the paired single-view kernel (each warp renders two tiles) and the blocks
// it is compiled to keep resident per SM (caps registers at 65536 / (128 n) per thread): eight
// for one-tap (64 registers, no spills; measured 0.0577 against 0.0598 ms at six on the 4K
// frame), six for the sharing modes and the full filter (more blocks gained nothing there).
constexpr int kPairWarps = 4;
template <int MODE> constexpr int pair_min_blocks() { return MODE == 1 ? 8 : 6; }

// One view, paired path: block (bx, by) renders tiles 2 (bx kPairWarps + warp) + half of tile row
// by. BLUE: blue-noise selection uniforms; EX: exact filtering (bilinear). A tile past the row's end (right edge of the grid) is rendered with every store skipped,
// so that both half-warps reach the warp's barriers.
template <int KIND, int F, int MODE, int TW, int TH, bool BLUE = false, bool EX = false>
__global__ void __launch_bounds__(32 * kPairWarps, pair_min_blocks<MODE>()) k_render_pair(const DevView v)
{
    __shared__ float4 recs[kPairWarps * 2 * 32 * kRecPerLane];
    __shared__ float wtabs[F == 1 ? kPairWarps * 2 * 32 * 8 : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = (blockIdx.x * kPairWarps + warp) * 2;
    if (t0 >= v.tiles_x) return;  // warp-uniform
    const int half = lane >> 4, tile = warp * 2 + half;
    render_pair<KIND, F, MODE, TW, TH, BLUE, EX>(v, t0 + half, blockIdx.y, lane & 15, recs + tile * 32 * kRecPerLane,
                                       wtabs + (F == 1 ? tile * 32 * 8 : 0), true, GlobalFetch<KIND>{v});
}

// ------------------------------------------------------------------------------ TMA-staged variant
//
// The same paired kernel with the block's texel footprint staged in shared memory by the tensor
// memory accelerator before any pixel is computed: one thread bounds the texels the block's
// 2 kPairWarps tiles can touch (the filter taps of its four corner pixels, which bound those of
// every pixel in between for an affine view, plus one texel of margin on every side, clamped to
// the texture), and loads that box with cp.async.bulk.tensor (a tensor map over this GPU's own
// texture; no multicast) as kTmaBoxW x kTmaBoxH texel tiles completing on one mbarrier. Fetches
// inside the box read shared memory, the rest (a projective view's far texels, extrapolated
// pixels of a partial tile) the read-only global path, so the result never depends on the box.
// A footprint of more than kTmaStageBytes (minification) is not staged at all.

constexpr int kTmaBoxW = 16, kTmaBoxH = 4;  // texels per TMA tile (the tensor map's box)
constexpr int kTmaStageBytes = 16384;      // staged texels per block: 16 tiles of 16-byte texels
constexpr unsigned kTmaWaitLimit = 1u << 20;

template <int KIND> struct StagedFetch {
    static constexpr int R = Mat<KIND>::R;
    const DevView& v;
    uint32_t smem;           // shared address of the staged box (grid of kTmaBoxW x kTmaBoxH tiles)
    int x0, y0, bw, bh;      // texel box; bw = 0: nothing staged
    __device__ __forceinline__ void operator()(int x, int y, float (&t)[Channels<KIND>::C]) const
    {
        x = clampi(x, 0, v.tex_w - 1);
        y = clampi(y, 0, v.tex_h - 1);
        const int dx = x - x0, dy = y - y0;
        if ((unsigned)dx < (unsigned)bw && (unsigned)dy < (unsigned)bh) {
            const int tile = (dy / kTmaBoxH) * (bw / kTmaBoxW) + dx / kTmaBoxW;
            const uint32_t a = smem + (uint32_t)(((tile * kTmaBoxH + dy % kTmaBoxH) * kTmaBoxW + dx % kTmaBoxW) * R);
            Mat<KIND>::decode(v, ld_record_shared<R>(a), x, y, t);
        } else {
            Mat<KIND>::fetch(v, x, y, t);
        }
    }
};

__device__ __forceinline__ bool tma_wait(uint32_t bar, uint32_t parity)
{
    for (unsigned it = 0; it < kTmaWaitLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

template <int KIND, int F, int MODE, int TW, int TH>
__global__ void __launch_bounds__(32 * kPairWarps, pair_min_blocks<MODE>())
    k_render_pair_tma(const __grid_constant__ CUtensorMap tmap, const DevView v)
{
    constexpr int R = Mat<KIND>::R;
    __shared__ float4 recs[kPairWarps * 2 * 32 * kRecPerLane];
    __shared__ float wtabs[F == 1 ? kPairWarps * 2 * 32 * 8 : 1];
    constexpr int kMaxBoxes = kTmaStageBytes / (kTmaBoxW * kTmaBoxH * R);
    __shared__ alignas(128) unsigned char box[kTmaStageBytes];
    __shared__ alignas(8) unsigned long long bar;
    __shared__ int4 geo;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tb = blockIdx.x * kPairWarps * 2;  // the block's first tile
    const uint32_t sbar = smem_u32(&bar);
    if (threadIdx.x == 0) {
        int4 g = make_int4(0, 0, 0, 0);
        const int x_lo = tb * TW, x_hi = min((tb + 2 * kPairWarps) * TW, v.width) - 1;
        const int y_lo = blockIdx.y * TH, y_hi = min(y_lo + TH, v.height) - 1;
        float lo_x = INFINITY, hi_x = -INFINITY, lo_y = INFINITY, hi_y = -INFINITY;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float u, w;
            pixel_uv(v, (k & 1) ? x_hi : x_lo, (k & 2) ? y_hi : y_lo, u, w);
            const float cx = texel_coord(u, v.tex_wf), cy = texel_coord(w, v.tex_hf);
            lo_x = fminf(lo_x, cx); hi_x = fmaxf(hi_x, cx); lo_y = fminf(lo_y, cy); hi_y = fmaxf(hi_y, cy);
        }
        // taps floor(c) + K0 .. floor(c) + K0 + N - 1, one texel of margin, clamped to the texture;
        // x starts on a 16-byte boundary of the row (TMA)
        int x0 = clampi((int)floorf(lo_x) + Taps<F>::K0 - 1, 0, v.tex_w - 1);
        const int x1 = clampi((int)floorf(hi_x) + Taps<F>::K0 + Taps<F>::N, 0, v.tex_w - 1);
        const int y0 = clampi((int)floorf(lo_y) + Taps<F>::K0 - 1, 0, v.tex_h - 1);
        const int y1 = clampi((int)floorf(hi_y) + Taps<F>::K0 + Taps<F>::N, 0, v.tex_h - 1);
        if (R < 16) x0 &= ~(16 / R - 1);
        const int nbx = (x1 - x0) / kTmaBoxW + 1, nby = (y1 - y0) / kTmaBoxH + 1;
        if (nbx * nby <= kMaxBoxes) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(sbar) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t bytes = (uint32_t)(nbx * nby * kTmaBoxW * kTmaBoxH * R);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(sbar), "r"(bytes) : "memory");
            const uint64_t map = reinterpret_cast<uint64_t>(&tmap);
            for (int j = 0; j < nby; ++j)
                for (int i = 0; i < nbx; ++i) {
                    const uint32_t dst = smem_u32(box) + (uint32_t)((j * nbx + i) * kTmaBoxW * kTmaBoxH * R);
                    const int cx = (x0 + i * kTmaBoxW) * (R / 4), cy = y0 + j * kTmaBoxH;  // uint32 elements, rows
                    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                 " [%0], [%1, {%2, %3}], [%4];"
                                 :: "r"(dst), "l"(map), "r"(cx), "r"(cy), "r"(sbar) : "memory");
                }
            g = make_int4(x0, y0, nbx * kTmaBoxW, nby * kTmaBoxH);
        }
        geo = g;
    }
    __syncthreads();
    int4 g = geo;
    if (g.z && !tma_wait(sbar, 0)) {
        // bounded: record the give-up, wait (bounded) for the copies still in flight, then read
        // every texel from global memory
        if (threadIdx.x == 0) atomicAdd(v.flags, 1);
        tma_wait(sbar, 0);
        g.z = 0;
    }
    const int t0 = tb + warp * 2;
    if (t0 >= v.tiles_x) return;  // warp-uniform, after the block-wide barrier
    const int half = lane >> 4, tile = warp * 2 + half;
    render_pair<KIND, F, MODE, TW, TH, false, false>(v, t0 + half, blockIdx.y, lane & 15, recs + tile * 32 * kRecPerLane,
                                       wtabs + (F == 1 ? tile * 32 * 8 : 0), true,
                                       StagedFetch<KIND>{v, smem_u32(box), g.x, g.y, g.z, g.w});
}

}  // namespace stf
