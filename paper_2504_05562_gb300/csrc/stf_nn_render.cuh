// Rendering a neural material: the per-pixel steps of the texture kinds (pixel -> uv, random
// numbers, one-tap texel choice, sharing with the bounded weighted-importance combine, shading)
// run on the client warps of the decode pipeline, split around the decode:
//   produce: the pixel's chosen texel (or, for the full filter, one tap per round) -> its sample
//            record and its 24 decoder inputs as a row of the round;
//   consume: after the decoder has finished the round, the decoded texels of the warp's
//            rows -> the estimate of Eq. estimator-for-stf (or the running filter sum) -> shaded
//            output.
// Round r is produced before round r - 1 is consumed, so the clients' arithmetic overlaps the
// tensor-core work. The selection, combine and shading arithmetic is the texture kinds' (the same
// helpers and operation order), so a neural render differs from them only in how a texel's
// channels are obtained.
#pragma once

#include <float.h>

#include "stf_device.cuh"
#include "stf_kernels.cuh"
#include "stf_neural.cuh"

namespace stf {

// Per-warp B-spline tap-weight table of the sharing loop: 8 columns of 32 lanes.
constexpr int kNnWtabFloats = kNnClientWarps * 32 * 8;

// The client side of one block. VIEWS maps a view index to its constants (a kernel parameter or
// the batch's constant bank). Every client thread calls round() for the same rounds. EX: exact
// filtering (bilinear sharing modes).
template <int F, int MODE, int TW, int TH, bool EX, bool BLUE, class VIEWS>
struct NnRenderClient {
    static constexpr int NT = MODE == 0 ? Taps<F>::N * Taps<F>::N : 1;  // rounds per tile group
    NnPipeSmem& sm;
    float* wtab;  // this warp's columns
    VIEWS views;
    NnWaiter w;
    int warp, lane;
    uint32_t r = 0;  // rounds published
    bool pend = false;
    int pview = 0, ptx = 0, pty = 0, pt = 0;
    bool pact = false;
    float acc[8];  // full filter: the pixel's running sum over taps

    __device__ NnRenderClient(NnPipeSmem& s, float* wt, VIEWS v, int* flags)
        : sm(s), wtab(wt), views(v), w{flags, 0}, warp((int)threadIdx.x >> 5), lane((int)threadIdx.x & 31)
    {
    }

    __device__ __forceinline__ void produce(int view, bool active, int tx, int ty, int t, int slot)
    {
        const int row = warp * 32 + lane;
        // the slot's previous round (r - 2) may still be read by other lanes of this warp, whose
        // sharing loops read every lane's record and decoded texel: wait for all of them
        __syncwarp();
        if (active) {
            const DevView& v = views(view);
            const int x = tx * TW + lane % TW, y = ty * TH + lane / TW;
            float u, wv;
            pixel_uv(v, x, y, u, wv);
            const float cx = texel_coord(u, v.tex_wf), cy = texel_coord(wv, v.tex_hf);
            int nx, ny;
            float4 rec;
            if constexpr (MODE == 0) {
                // tap t of the deterministic filter, y outer (Eq. texture-continuous-sum)
                const int q = t % Taps<F>::N, s = t / Taps<F>::N;
                const float ix = floorf(cx), iy = floorf(cy);
                const float bx = __fadd_rn(ix, (float)Taps<F>::K0), by = __fadd_rn(iy, (float)Taps<F>::K0);
                const float wx = tap_weight<F>(cx, __fadd_rn(bx, (float)q), q);
                const float wy = tap_weight<F>(cy, __fadd_rn(by, (float)s), s);
                nx = __float2int_rn(ix) + Taps<F>::K0 + q;
                ny = __float2int_rn(iy) + Taps<F>::K0 + s;
                rec = make_float4(__fmul_rn(wx, wy), 0.0f, 0.0f, 0.0f);
            } else {
                // one texel drawn from the pixel's filter PMF (Section 2.2, Section S1)
                float ux, uy;
                pixel_uniforms<BLUE>(v, x, y, ux, uy);
                Axis<F> ax, ay;
                axis_select<F>(cx, ux, ax);
                axis_select<F>(cy, uy, ay);
                const float p = __fmul_rn(ax.p, ay.p);
                nx = ax.n;
                ny = ay.n;
                rec = make_float4(ax.nf, ay.nf, fminf(rcp_approx(p), FLT_MAX), __uint_as_float(pack_idx(ax.n, ay.n)));
            }
            sm.rec[slot][row] = rec;
            sm.geo[slot][row] = make_float4(u, wv, cx, cy);  // read back by this thread's consume
            uint32_t in[12];
            nn_inputs(*reinterpret_cast<const NeuralDev*>(v.neural), clampi(nx, 0, v.tex_w - 1), clampi(ny, 0, v.tex_h - 1), in);
            nn_put_inputs(sm, slot, row, in);
        }
        nn_publish(sm, slot, 1);
    }

    __device__ __forceinline__ void consume(int view, bool active, int tx, int ty, int t, uint32_t rr)
    {
        const int slot = rr & 1;
        // every client waits, active or not: the slot is rewritten two rounds later
        w.wait(sm.out_full[slot], (rr >> 1) & 1u);
        if (!active) return;
        const DevView& v = views(view);
        const int lx = lane % TW, ly = lane / TW;
        const int x = tx * TW + lx, y = ty * TH + ly;
        const int row0 = warp * 32;
        float res[8];
        uint32_t pk = 0;
        if constexpr (MODE == 0) {
            float T[8];
            nn_get_outputs(sm, slot, row0 + lane, T);
            const float wt = sm.rec[slot][row0 + lane].x;
            if (t == 0)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[c] = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = fmaf(wt, T[c], acc[c]);
            if (t != NT - 1) return;
#pragma unroll
            for (int c = 0; c < 8; ++c) res[c] = acc[c];
        } else if constexpr (MODE == 1) {
            nn_get_outputs(sm, slot, row0 + lane, res);
            pk = __float_as_uint(sm.rec[slot][row0 + lane].w);
        } else {
            // the estimate of Eq. estimator-for-stf over the lane's footprint, w_j = f_c(x_j) / f_j(x_j),
            // the own weight exactly 1 (the texture kinds' combine, records read from the round)
            using FP = Footprint<MODE, TW, TH>;
            const float4 g = sm.geo[slot][row0 + lane];
            const float cx = g.z, cy = g.w;
            Axis<F> ax, ay;
            if constexpr (F == 0 && EX) {
                axis_weights<F>(cx, ax);
                axis_weights<F>(cy, ay);
            }
            if constexpr (F == 1) {
                axis_weights<F>(cx, ax);
                axis_weights<F>(cy, ay);
#pragma unroll
                for (int k = 0; k < 4; ++k) { wtab[k * 32 + lane] = ax.w[k]; wtab[(4 + k) * 32 + lane] = ay.w[k]; }
                __syncwarp();
            }
            pk = __float_as_uint(sm.rec[slot][row0 + lane].w);
            const int b0 = FP::base(lx, ly);
            float2 a2[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) a2[c] = make_float2(0.0f, 0.0f);
            float wsum = 0.0f;
            uint32_t srcs = 0;  // exact filtering: per bilinear tap, 1 + a lane holding its texel
            auto visit = [&](int src) {
                const float4 m = sm.rec[slot][row0 + src];
                float wx, wy;
                if constexpr (F == 0) {
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
                    const uint32_t pj = __float_as_uint(m.w);
                    const int kx = unpack_x(pj) - ax.base, ky = unpack_y(pj) - ay.base;
                    const bool in = ((kx | ky) & ~3) == 0;
                    wx = in ? wtab[kx * 32 + lane] : 0.0f;
                    wy = in ? wtab[(4 + ky) * 32 + lane] : 0.0f;
                }
                const float wt = (src == lane) ? 1.0f : (wx * wy) * m.z;
                const float2 w2 = make_float2(wt, wt);
                const float4 t0 = sm.out[slot][0][row0 + src];
                const float4 t1 = sm.out[slot][1][row0 + src];
                a2[0] = __ffma2_rn(w2, make_float2(t0.x, t0.y), a2[0]);
                a2[1] = __ffma2_rn(w2, make_float2(t0.z, t0.w), a2[1]);
                a2[2] = __ffma2_rn(w2, make_float2(t1.x, t1.y), a2[2]);
                a2[3] = __ffma2_rn(w2, make_float2(t1.z, t1.w), a2[3]);
                wsum += wt;
            };
            if constexpr (MODE == kModeSparse9) {
                const uint4 fr = __ldg(reinterpret_cast<const uint4*>(v.fp) + lane);
                const uint32_t w4[4] = {fr.x, fr.y, fr.z, fr.w};
#pragma unroll
                for (int i = 0; i < 9; ++i) visit((int)((w4[i >> 2] >> (8 * (i & 3))) & 0x1fu));
            } else {
#pragma unroll
                for (int rr2 = 0; rr2 < FP::KY; ++rr2)
#pragma unroll
                    for (int q = 0; q < FP::KX; ++q) visit(b0 + rr2 * TW + q);
            }
            if constexpr (F == 1) __syncwarp();  // the table is rewritten by the warp's next round
            const float inv = rcp_approx(wsum);
#pragma unroll
            for (int c = 0; c < 4; ++c) { res[2 * c] = a2[c].x * inv; res[2 * c + 1] = a2[c].y * inv; }
            if constexpr (EX && F == 0)
                exact_bilinear<8>(ax, ay, srcs, res, [&](int j, float (&T)[8]) { nn_get_outputs(sm, slot, row0 + j, T); });
        }
        if (x < v.width && y < v.height) {
            const float4 g = sm.geo[slot][row0 + lane];  // (u, v) of the pixel, from its produce
            const float4 o = finish_pixel<8>(v, res, g.x, g.y);
            __stcs(reinterpret_cast<float4*>(v.out + (size_t)y * v.pitch + 4 * (size_t)x), o);
            const size_t pix = (size_t)y * v.width + x;
            if (v.dbg_idx) v.dbg_idx[pix] = pk;
            if (v.dbg_ch) {
                float4* d = reinterpret_cast<float4*>(v.dbg_ch + pix * 8);
                float z[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) z[c] = c < v.c_true ? res[c] : 0.0f;
                d[0] = make_float4(z[0], z[1], z[2], z[3]);
                d[1] = make_float4(z[4], z[5], z[6], z[7]);
            }
        }
    }

    // One tile per warp (tile (tx, ty) of view `view`; inactive warps only keep the rounds in step).
    __device__ __forceinline__ void group(int view, bool active, int tx, int ty)
    {
#pragma unroll 1
        for (int t = 0; t < NT; ++t) {
            produce(view, active, tx, ty, t, r & 1);
            if (pend) consume(pview, pact, ptx, pty, pt, r - 1);
            pend = true;
            pview = view;
            pact = active;
            ptx = tx;
            pty = ty;
            pt = t;
            ++r;
        }
    }

    // Ends the clients' stream: a round without rows, then the last pending round.
    __device__ __forceinline__ void finish()
    {
        nn_publish(sm, r & 1, 0);
        if (pend) consume(pview, pact, ptx, pty, pt, r - 1);
    }
};

struct NnParamView {
    const DevView* v;
    __device__ __forceinline__ const DevView& operator()(int) const { return *v; }
};

// One view: persistent blocks walk the view's tile groups (kNnClientWarps tiles of one tile row).
template <int F, int MODE, int TW, int TH, bool EX = false, bool BLUE = false>
__global__ void __launch_bounds__(kNnPipeThreads, 2) k_render_neural(const __grid_constant__ DevView v)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    __shared__ float wtabs[kNnWtabFloats];
    NnPipeSmem& sm = *reinterpret_cast<NnPipeSmem*>(dyn);
    nn_pipe_setup(sm, reinterpret_cast<const NeuralDev*>(v.neural));
    if (threadIdx.x >= kNnClients) {
        nn_decode_role(sm, v.flags);
    } else {
        const int warp = threadIdx.x >> 5;
        NnRenderClient<F, MODE, TW, TH, EX, BLUE, NnParamView> cl(sm, wtabs + warp * 256, NnParamView{&v}, v.flags);
        const int gx = (v.tiles_x + kNnClientWarps - 1) / kNnClientWarps;
        const int groups = gx * v.tiles_y;
#pragma unroll 1
        for (int g = blockIdx.x; g < groups; g += gridDim.x) {
            const int by = g / gx;
            const int tx = (g - by * gx) * kNnClientWarps + warp;
            cl.group(0, tx < v.tiles_x, tx, by);
        }
        cl.finish();
    }
    nn_pipe_teardown(sm);
}

}  // namespace stf
