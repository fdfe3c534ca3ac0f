// Neural texel decoder on the GPU: inference with tensor cores.
//
// The decoder of texel (ix, iy) of a material with an R-times coarser latent grid (16 channels
// per latent cell): bilinear interpolation of the latent grid at (i + 0.5) / R - 0.5 per axis
// (clamp-to-edge), 8 position features sin/cos(2 pi phi), sin/cos(4 pi phi) of the phase
// phi = ((i mod R) + 0.5) / R per axis, then an MLP 24 -> 64 -> 64 -> 8 with ReLU. This is the
// costly per-texel decode that stochastic filtering amortises (Sections 1 and 5.7).
//
// Inference precision: latents and weights FP16, the 24 inputs and both hidden layers rounded to
// FP16, products accumulated in FP32 by the tensor cores, biases and outputs FP32.
//
// A warp decodes the 32 texels its lanes hold at once: the 32 input rows form the A operand of
// m16n8k16 tensor-core products (two 16-row tiles), the weights are pre-arranged B fragments,
// and each layer's FP32 accumulators are converted in registers into the next layer's FP16 A
// fragments (no shared-memory round trip between layers).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "stf_device.cuh"

namespace stf {

constexpr int kNnIn = 24, kNnH = 64, kNnOut = 8, kNnLat = 16;
constexpr int kNnParams = kNnH * kNnIn + kNnH + kNnH * kNnH + kNnH + kNnOut * kNnH + kNnOut;  // 6280
constexpr int kNnFrags = 16 + 32 + 4;       // B fragments of layers 1, 2, 3
constexpr int kNnRowBytes = 80;             // A-tile row stride (32 halves + pad, conflict-free ldmatrix)
constexpr int kNnWarpSmem = 32 * kNnRowBytes;  // 2560 bytes of shared scratch per warp

// Device parameter block of a decoder's inference copy.
struct NeuralDev {
    const uint4* lat16;   // [gh][gw][2]: 16 FP16 latents per cell
    const uint2* wfrag;   // [kNnFrags][32 lanes]: B fragments (W1 k-tile 0..1 x n-tile 0..7,
                          // W2 k-tile 0..3 x n-tile 0..7, W3 k-tile 0..3)
    const float* bias;    // b1[64], b2[64], b3[8]
    int gw, gh, rshift;   // R = 1 << rshift
    float inv_r;          // 1 / R (exact)
    uint2 feat[16];       // phase p: (sin, cos)(2 pi phi) and (sin, cos)(4 pi phi) as half2 pairs
};

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float2 unpack_h2(uint32_t w)
{
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint2 b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr));
}

// Bilinear position along one latent axis: lower cell, upper cell (both clamped) and fraction.
__device__ __forceinline__ void nn_axis(int i, const NeuralDev& nd, int G, int& c0, int& c1, float& f)
{
    const float l = __fsub_rn(__fmul_rn(__fadd_rn(__int2float_rn(i), 0.5f), nd.inv_r), 0.5f);
    const float fl = floorf(l);
    f = __fsub_rn(l, fl);
    const int a = __float2int_rn(fl);
    c0 = clampi(a, 0, G - 1);
    c1 = clampi(a + 1, 0, G - 1);
}

// The 24 FP16 inputs of texel (x, y) as 12 packed words (interpolation rounded per operation in
// the order (w00 L00 + w10 L10) + w01 L01, + w11 L11).
__device__ __forceinline__ void nn_inputs(const NeuralDev& nd, int x, int y, uint32_t (&row)[12])
{
    int x0, x1, y0, y1;
    float fx, fy;
    nn_axis(x, nd, nd.gw, x0, x1, fx);
    nn_axis(y, nd, nd.gh, y0, y1, fy);
    const float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
    const float w00 = __fmul_rn(gx, gy), w10 = __fmul_rn(fx, gy), w01 = __fmul_rn(gx, fy), w11 = __fmul_rn(fx, fy);
    const uint4* c00 = nd.lat16 + 2 * ((size_t)y0 * nd.gw + x0);
    const uint4* c10 = nd.lat16 + 2 * ((size_t)y0 * nd.gw + x1);
    const uint4* c01 = nd.lat16 + 2 * ((size_t)y1 * nd.gw + x0);
    const uint4* c11 = nd.lat16 + 2 * ((size_t)y1 * nd.gw + x1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 a = __ldg(c00 + h), b = __ldg(c10 + h), c = __ldg(c01 + h), d = __ldg(c11 + h);
        const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
        const uint32_t cw[4] = {c.x, c.y, c.z, c.w}, dw[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 A = unpack_h2(aw[k]), B = unpack_h2(bw[k]), Cc = unpack_h2(cw[k]), D = unpack_h2(dw[k]);
            float s0 = __fmul_rn(w00, A.x), s1 = __fmul_rn(w00, A.y);
            s0 = __fadd_rn(s0, __fmul_rn(w10, B.x));
            s1 = __fadd_rn(s1, __fmul_rn(w10, B.y));
            s0 = __fadd_rn(s0, __fmul_rn(w01, Cc.x));
            s1 = __fadd_rn(s1, __fmul_rn(w01, Cc.y));
            s0 = __fadd_rn(s0, __fmul_rn(w11, D.x));
            s1 = __fadd_rn(s1, __fmul_rn(w11, D.y));
            row[4 * h + k] = pack_h2(s0, s1);
        }
    }
    const int mask = (1 << nd.rshift) - 1;
    const uint2 fxw = nd.feat[x & mask], fyw = nd.feat[y & mask];
    row[8] = fxw.x;
    row[9] = fxw.y;
    row[10] = fyw.x;
    row[11] = fyw.y;
}

// Bias-initialised accumulator of an n-tile: columns nt * 8 + 2 (lane % 4) + {0, 1}.
__device__ __forceinline__ void nn_bias(float (&c)[4], const float* b, int nt, int lane)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(b + nt * 8 + 2 * (lane & 3)));
    c[0] = v.x; c[1] = v.y; c[2] = v.x; c[3] = v.y;
}

// ReLU of two n-tiles' accumulators -> the FP16 A fragment of one 16-wide k-tile.
__device__ __forceinline__ void nn_relu_pack(const float (&lo)[4], const float (&hi)[4], uint32_t (&a)[4])
{
    a[0] = pack_h2(fmaxf(lo[0], 0.0f), fmaxf(lo[1], 0.0f));
    a[1] = pack_h2(fmaxf(lo[2], 0.0f), fmaxf(lo[3], 0.0f));
    a[2] = pack_h2(fmaxf(hi[0], 0.0f), fmaxf(hi[1], 0.0f));
    a[3] = pack_h2(fmaxf(hi[2], 0.0f), fmaxf(hi[3], 0.0f));
}

// Decodes the texel (x, y) of every lane (all 32 lanes call together). `smem` is this warp's
// kNnWarpSmem bytes of 16-byte-aligned shared scratch.
__device__ __forceinline__ void nn_decode_warp(const NeuralDev* ndp, int x, int y, float (&t)[8], unsigned char* smem)
{
    const NeuralDev& nd = *ndp;
    const int lane = threadIdx.x & 31;
    uint32_t row[12];
    nn_inputs(nd, x, y, row);
    uint4* my = reinterpret_cast<uint4*>(smem + lane * kNnRowBytes);
    my[0] = make_uint4(row[0], row[1], row[2], row[3]);
    my[1] = make_uint4(row[4], row[5], row[6], row[7]);
    my[2] = make_uint4(row[8], row[9], row[10], row[11]);
    my[3] = make_uint4(0u, 0u, 0u, 0u);  // inputs 24..31 are zero padding
    __syncwarp();
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    float out[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        // layer 1: [16 x 32] x [32 x 64]
        uint32_t a1[2][4];
#pragma unroll
        for (int kt = 0; kt < 2; ++kt) {
            const int r = mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
            const int c = kt * 16 + (lane >> 4) * 8;
            ldmatrix_x4(a1[kt], sbase + r * kNnRowBytes + c * 2);
        }
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            nn_bias(acc[nt], nd.bias, nt, lane);
#pragma unroll
            for (int kt = 0; kt < 2; ++kt) mma_16816(acc[nt], a1[kt], __ldg(nd.wfrag + (kt * 8 + nt) * 32 + lane));
        }
        // layer 2: [16 x 64] x [64 x 64]
        uint32_t a2[4][4];
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) nn_relu_pack(acc[2 * kt], acc[2 * kt + 1], a2[kt]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            nn_bias(acc[nt], nd.bias + kNnH, nt, lane);
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) mma_16816(acc[nt], a2[kt], __ldg(nd.wfrag + (16 + kt * 8 + nt) * 32 + lane));
        }
        // layer 3: [16 x 64] x [64 x 8]
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) nn_relu_pack(acc[2 * kt], acc[2 * kt + 1], a2[kt]);
        nn_bias(out[mt], nd.bias + 2 * kNnH, 0, lane);
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) mma_16816(out[mt], a2[kt], __ldg(nd.wfrag + (48 + kt) * 32 + lane));
    }
    __syncwarp();  // every lane has read the A tile
    // rows mt * 16 + lane / 4 (+ 8), columns 2 (lane % 4) + {0, 1} -> 48-byte rows
    float* ob = reinterpret_cast<float*>(smem);
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int r = mt * 16 + (lane >> 2);
        const int c = 2 * (lane & 3);
        *reinterpret_cast<float2*>(ob + r * 12 + c) = make_float2(out[mt][0], out[mt][1]);
        *reinterpret_cast<float2*>(ob + (r + 8) * 12 + c) = make_float2(out[mt][2], out[mt][3]);
    }
    __syncwarp();
    const float4 o0 = *reinterpret_cast<const float4*>(ob + lane * 12);
    const float4 o1 = *reinterpret_cast<const float4*>(ob + lane * 12 + 4);
    t[0] = o0.x; t[1] = o0.y; t[2] = o0.z; t[3] = o0.w;
    t[4] = o1.x; t[5] = o1.y; t[6] = o1.z; t[7] = o1.w;
    __syncwarp();  // the scratch may be rewritten by the next decode
}

}  // namespace stf
