// Neural texel decoder on the GPU: inference with tensor cores.
//
// The decoder of texel (ix, iy) of a material with an R-times coarser latent grid (16 channels
// per latent cell): bilinear interpolation of the latent grid at (i + 0.5) / R - 0.5 per axis
// (clamp-to-edge), 8 position features sin/cos(2 pi phi), sin/cos(4 pi phi) of the phase
// phi = ((i mod R) + 0.5) / R per axis, then an MLP 24 -> 64 -> 64 -> 8 with ReLU. This is the
// costly per-texel decode that stochastic filtering amortises (Sections 1 and 5.6).
//
// Inference precision: latents and weights FP16, the 24 inputs and both hidden layers rounded to
// FP16, products and biases accumulated in FP32 by the tensor cores, outputs FP32.
//
// Decoding runs as a pipeline inside each block: client warps prepare the inputs of 256 texels,
// a decode warpgroup evaluates the MLP with tcgen05 tensor-core products (see the decode pipeline
// section below).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "stf_device.cuh"

namespace stf {

constexpr int kNnIn = 24, kNnH = 64, kNnOut = 8, kNnLat = 16;
constexpr int kNnParams = kNnH * kNnIn + kNnH + kNnH * kNnH + kNnH + kNnOut * kNnH + kNnOut;  // 6280

// tcgen05 operand images (FP16, K-major, no swizzle: element (r, k) of an R x K matrix at byte
// (r / 8) * (K / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, i.e. 8 x 8 core matrices
// of 128 bytes, K-adjacent ones 128 bytes apart, row groups (K / 8) * 128 bytes apart). Each
// layer's bias rides in two extra K columns: the weight image holds its FP16 high part hi(b) and
// the FP16 rounding of b - hi(b), the activation operand holds 1 in both, so the FP32
// accumulation adds b to within 2^-22 |b| and the epilogue is a plain ReLU.
constexpr int kNnK1 = 32;                   // layer 1: 24 inputs, bias columns 24 / 25, zeros
constexpr int kNnK2 = 80;                   // layers 2, 3: 64 hidden, bias columns 64 / 65, zeros
constexpr int kNnB1Bytes = 64 * kNnK1 * 2;  // W1: N = 64 x K = 32
constexpr int kNnB2Bytes = 64 * kNnK2 * 2;  // W2: N = 64 x K = 80
constexpr int kNnB3Bytes = 16 * kNnK2 * 2;  // W3: N = 16 (8 outputs + zero rows) x K = 80
constexpr int kNnImgBytes = kNnB1Bytes + kNnB2Bytes + kNnB3Bytes;  // 16896

// E4M3 variant of the image (the FP8 inference precision the c4 workload allows): layer 1 stays
// FP16 with its weights and bias scaled by s1; layers 2 and 3 are OCP E4M3 kind::f8f6f4
// products, W2 and W3 scaled by s2 and s3, each bias split into three E4M3 parts (K 64 .. 66)
// against activation columns of 1, so a row is K = 96 bytes (three K steps of 32). The hidden
// activations are rounded to E4M3 (ReLU, satfinite) in the epilogue; the outputs are scaled back
// by 1 / (s1 s2 s3). s1, s2, s3 are powers of two from a first-order bound of the activations
// (stf_decoder_set_inference), so that neither weights nor activations saturate.
constexpr int kNnK8 = 96;
constexpr int kNnB2Bytes8 = 64 * kNnK8, kNnB3Bytes8 = 16 * kNnK8;
static_assert(kNnB1Bytes + kNnB2Bytes8 + kNnB3Bytes8 <= kNnImgBytes, "the E4M3 image fits the FP16 one's space");

// Device parameter block of a decoder's inference copy.
struct NeuralDev {
    const uint4* lat16;   // [gh][gw][2]: 16 FP16 latents per cell
    int gw, gh, rshift;   // R = 1 << rshift
    float inv_r;          // 1 / R (exact)
    uint2 feat[16];       // phase p: (sin, cos)(2 pi phi) and (sin, cos)(4 pi phi) as half2 pairs
    const uint4* wimg;    // the three layers (weights and biases) as tensor-core B operands
    int fp8;              // 1: the E4M3 variant (layers 2 and 3 as FP8 products, see below)
    float out_scale;      // E4M3 variant: 1 / (s1 s2 s3), exact; 1 otherwise
};

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

// The four latent cells texel (x, y) interpolates (c[0..3] = (x0, y0), (x1, y0), (x0, y1),
// (x1, y1), 2 x 16 bytes each) and their bilinear weights.
__device__ __forceinline__ void nn_cells(const NeuralDev& nd, int x, int y, const uint4* (&c)[4], float (&w)[4])
{
    int x0, x1, y0, y1;
    float fx, fy;
    nn_axis(x, nd, nd.gw, x0, x1, fx);
    nn_axis(y, nd, nd.gh, y0, y1, fy);
    const float gx = __fsub_rn(1.0f, fx), gy = __fsub_rn(1.0f, fy);
    w[0] = __fmul_rn(gx, gy);
    w[1] = __fmul_rn(fx, gy);
    w[2] = __fmul_rn(gx, fy);
    w[3] = __fmul_rn(fx, fy);
    c[0] = nd.lat16 + 2 * ((size_t)y0 * nd.gw + x0);
    c[1] = nd.lat16 + 2 * ((size_t)y0 * nd.gw + x1);
    c[2] = nd.lat16 + 2 * ((size_t)y1 * nd.gw + x0);
    c[3] = nd.lat16 + 2 * ((size_t)y1 * nd.gw + x1);
}

// The 16 interpolated latents as 8 packed FP16 words from the cells' 8 chunks L[2 q + h] (cell q,
// half h) in FP16 arithmetic, the precision of the decoder's inputs: the four corner weights
// rounded to FP16, then w00 L00, + w10 L10, + w01 L01, + w11 L11 with one rounding per multiply
// and per fused multiply-add (two channels per half2 operation).
__device__ __forceinline__ void nn_interp(const uint4 (&L)[8], const float (&w)[4], uint32_t (&row)[12])
{
    const __half2 w0 = __float2half2_rn(w[0]), w1 = __float2half2_rn(w[1]);
    const __half2 w2 = __float2half2_rn(w[2]), w3 = __float2half2_rn(w[3]);
    auto h2 = [](uint32_t v) { return *reinterpret_cast<const __half2*>(&v); };
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 a = L[h], b = L[2 + h], c = L[4 + h], d = L[6 + h];
        const uint32_t aw[4] = {a.x, a.y, a.z, a.w}, bw[4] = {b.x, b.y, b.z, b.w};
        const uint32_t cw[4] = {c.x, c.y, c.z, c.w}, dw[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __half2 s2 = __hmul2_rn(w0, h2(aw[k]));
            s2 = __hfma2(w1, h2(bw[k]), s2);
            s2 = __hfma2(w2, h2(cw[k]), s2);
            s2 = __hfma2(w3, h2(dw[k]), s2);
            row[4 * h + k] = *reinterpret_cast<const uint32_t*>(&s2);
        }
    }
}

// The position features of texel (x, y) as packed FP16 words 8 .. 11.
__device__ __forceinline__ void nn_features(const NeuralDev& nd, int x, int y, uint32_t (&row)[12])
{
    const int mask = (1 << nd.rshift) - 1;
    const uint2 fxw = nd.feat[x & mask], fyw = nd.feat[y & mask];
    row[8] = fxw.x;
    row[9] = fxw.y;
    row[10] = fyw.x;
    row[11] = fyw.y;
}

// The 24 FP16 inputs of texel (x, y) as 12 packed words.
__device__ __forceinline__ void nn_inputs(const NeuralDev& nd, int x, int y, uint32_t (&row)[12])
{
    const uint4* c[4];
    float w[4];
    nn_cells(nd, x, y, c, w);
    uint4 L[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) { L[2 * q] = __ldg(c[q]); L[2 * q + 1] = __ldg(c[q] + 1); }
    nn_interp(L, w, row);
    nn_features(nd, x, y, row);
}

// ------------------------------------------------------------------------------ tcgen05 primitives


// Shared-memory matrix descriptor, K-major without swizzle: start address, leading (K) byte
// offset between core matrices, stride (M/N) byte offset between 8-row groups, version 1.
__device__ __forceinline__ uint64_t nn_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, N, M = 128.
__host__ __device__ constexpr uint32_t nn_idesc(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void nn_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

// The same product with A read from tensor memory (row m = lane m, K packed two per column).
__device__ __forceinline__ void nn_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
        :: "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum));
}

// The same with kind::f8f6f4 (A and B E4M3: the type fields of the instruction descriptor are 0).
__device__ __forceinline__ void nn_mma_ts_f8(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n"
        :: "r"(d_tmem), "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void nn_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ uint32_t nn_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n" : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    return done;
}

__device__ __forceinline__ void nn_arrive(uint32_t mbar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// ReLU, then round to FP16 (negative values become +0 or -0, equal as a next-layer input).
__device__ __forceinline__ uint32_t relu_pack_h2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// ReLU, then round four values to E4M3 (nearest even, saturating), packed low to high.
__device__ __forceinline__ uint32_t relu_pack_e4m3x4(float a, float b, float c, float d)
{
    uint32_t r;
    asm("{\n\t.reg .b16 lo, hi;\n\t"
        "cvt.rn.satfinite.relu.e4m3x2.f32 lo, %2, %1;\n\t"
        "cvt.rn.satfinite.relu.e4m3x2.f32 hi, %4, %3;\n\t"
        "mov.b32 %0, {lo, hi};\n}\n"
        : "=r"(r) : "f"(a), "f"(b), "f"(c), "f"(d));
    return r;
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" :: "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// Byte offset of the 16-byte chunk j (elements 8j .. 8j + 7) of row m in a K-wide operand image.
__device__ __forceinline__ uint32_t nn_chunk(int m, int j, int K) { return (m >> 3) * (K / 8) * 128 + j * 128 + (m & 7) * 16; }

// ------------------------------------------------------------------------------ decode pipeline
//
// A block of 416 threads: 8 client warps (one decode row per thread and round), one MMA warp
// (warp 8) and four epilogue warps (9 .. 12; warp w reaches TMEM lanes 32 (w mod 4) .. + 31, so
// together they cover all 128). A round decodes the clients' 256 texels as two M = 128 tiles:
//   1. each client thread writes its texel's 24 FP16 inputs (plus the two bias columns) as row
//      `row` of the round's layer-1 operand and arrives on in_full[slot];
//   2. the MMA warp issues the three layers' tcgen05 products of both tiles (FP32 accumulators in
//      TMEM); between layers the epilogue warpgroup turns a tile's accumulators into FP16
//      activations (ReLU) in TMEM, the A operand of the next layer, and arrives on epi[tile]; the
//      tiles alternate, so one tile's products overlap the other's epilogue;
//   3. the epilogue warpgroup writes the 8 FP32 outputs of each row into the slot's output planes
//      and arrives on out_full[slot]; the client threads read their rows back (and, when sharing,
//      their warp's other rows).
// Two slots let the clients prepare round r + 1 while round r is decoded. Every wait is bounded:
// one that gives up counts itself in flags[0], and all later waits of the launch return at once
// (the outputs are then garbage, and the library reports the timeout).

constexpr int kNnClientWarps = 8;
constexpr int kNnClients = kNnClientWarps * 32;    // 256 texels per round
constexpr int kNnMmaWarp = 8;
constexpr int kNnRows = 256;                       // operand rows per round (two M = 128 tiles)
constexpr int kNnPipeThreads = 416;
constexpr int kNnIoBytes = kNnRows * kNnK1 * 2;    // 16384: the layer-1 operand of a round
// TMEM columns of a block: layer-1/2 FP32 accumulators of the two tiles at 0 and 64 (64 columns
// each), the tiles' FP16 hidden activations (the A operand of layers 2 and 3, two K elements per
// 32-bit column, K = 80 -> 40 columns) at 128 and 168, layer-3 accumulators at 224 and 240.
constexpr int kNnTmemCols = 256;
constexpr int kNnHidCol = 128, kNnHidCols = kNnK2 / 2;
// layer-3 accumulators (N = 16) of tile mt at columns kNnOutCol + 16 mt, apart from the layer-1/2
// accumulators, so the next round's layer 1 can run while the epilogue reads this round's outputs
constexpr int kNnOutCol = 224;
constexpr unsigned kNnWaitLimit = 1u << 20;        // mbarrier polls before a wait gives up

struct NnPipeSmem {
    alignas(128) unsigned char b[kNnImgBytes];
    alignas(128) unsigned char io[2][kNnIoBytes];
    float4 rec[2][kNnRows];  // per-row sample records of the clients (see the render kernels)
    float4 geo[2][kNnRows];  // per-row pixel geometry (u, v, cx, cy) of the render clients
    // decoded channels 0-3 and 4-7 of each row, per slot: a plane per half keeps a warp's 128-bit
    // reads of its rows conflict-free and their addresses linear in the row
    float4 out[2][2][kNnRows];
    // mma: layer-1/2 commits, mma_out: layer-3 commits, epi: activations stored (one per tile)
    unsigned long long in_full[2], out_full[2], mma[2], mma_out[2], epi[2];
    uint32_t tmem;
    int more[2];             // 1: the round in this slot carries rows, 0: the clients are done
    int fp8;                 // the decoder's E4M3 variant (NeuralDev::fp8)
    float out_scale;         // and its output scale
};

// Bounded mbarrier waits of one thread.
struct NnWaiter {
    int* flags;
    uint32_t dead;
    __device__ __forceinline__ bool wait(const unsigned long long& bar, uint32_t parity)
    {
        if (dead) return false;
        const uint32_t a = smem_u32(&bar);
        for (unsigned it = 0;; ++it) {
            if (nn_try_wait(a, parity)) return true;
            if ((it & 1023u) == 1023u && *reinterpret_cast<volatile int*>(flags) != 0) break;
            if (it >= kNnWaitLimit) {
                atomicAdd(flags, 1);
                break;
            }
        }
        dead = 1;
        return false;
    }
};

// Prologue (all threads): weight images into shared memory, barriers, the TMEM columns
// (allocated by warp 8, which also frees them).
__device__ __forceinline__ void nn_pipe_setup(NnPipeSmem& sm, const NeuralDev* nd)
{
    const uint4* src = nd->wimg;
    uint4* dst = reinterpret_cast<uint4*>(sm.b);
    for (int i = threadIdx.x; i < kNnImgBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    if (threadIdx.x == 0) {
        sm.fp8 = nd->fp8;
        sm.out_scale = nd->out_scale;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.in_full[0])), "r"(kNnClients) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.in_full[1])), "r"(kNnClients) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.epi[0])), "r"(128) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.epi[1])), "r"(128) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.out_full[0])), "r"(128) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.out_full[1])), "r"(128) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.mma[0])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.mma[1])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.mma_out[0])), "r"(1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(&sm.mma_out[1])), "r"(1) : "memory");
    }
    if ((threadIdx.x >> 5) == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&sm.tmem)), "r"(kNnTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void nn_pipe_teardown(NnPipeSmem& sm)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 8)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(sm.tmem), "r"(kNnTmemCols) : "memory");
}

// ---- client side

// Row `row` of the round's layer-1 operand: chunks 0..2 = the 24 inputs, chunk 3 = (1, 1, 0 ...)
// (the columns that carry the bias, split into FP16 high and low parts, in the weight image).
__device__ __forceinline__ void nn_put_inputs(NnPipeSmem& sm, int slot, int row, const uint32_t (&in)[12])
{
    const uint32_t base = smem_u32(sm.io[slot]);
#pragma unroll
    for (int j = 0; j < 3; ++j) sts128(base + nn_chunk(row, j, kNnK1), in[4 * j], in[4 * j + 1], in[4 * j + 2], in[4 * j + 3]);
    sts128(base + nn_chunk(row, 3, kNnK1), 0x3c003c00u, 0u, 0u, 0u);
}

// Hands the slot's rows to the decoder (every client thread calls it once per round; thread 0
// also says whether the round carries rows).
__device__ __forceinline__ void nn_publish(NnPipeSmem& sm, int slot, int more)
{
    if (threadIdx.x == 0) sm.more[slot] = more;
    fence_async_smem();
    nn_arrive(smem_u32(&sm.in_full[slot]));
}

// The 8 decoded FP32 channels of row `row` (valid after out_full of its round).
__device__ __forceinline__ void nn_get_outputs(const NnPipeSmem& sm, int slot, int row, float (&t)[8])
{
    const float4 a = sm.out[slot][0][row];
    const float4 b = sm.out[slot][1][row];
    t[0] = a.x; t[1] = a.y; t[2] = a.z; t[3] = a.w;
    t[4] = b.x; t[5] = b.y; t[6] = b.z; t[7] = b.w;
}

// ---- decode warpgroup

// 64 consecutive FP32 columns of this thread's TMEM lane (two loads in flight, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64])
{
    uint32_t r[64];
#define STF_LD32(OFF, R)                                                                                        \
    asm volatile(                                                                                               \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"         \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"                           \
        : "=r"(R[0]), "=r"(R[1]), "=r"(R[2]), "=r"(R[3]), "=r"(R[4]), "=r"(R[5]), "=r"(R[6]), "=r"(R[7]),       \
          "=r"(R[8]), "=r"(R[9]), "=r"(R[10]), "=r"(R[11]), "=r"(R[12]), "=r"(R[13]), "=r"(R[14]), "=r"(R[15]), \
          "=r"(R[16]), "=r"(R[17]), "=r"(R[18]), "=r"(R[19]), "=r"(R[20]), "=r"(R[21]), "=r"(R[22]),            \
          "=r"(R[23]), "=r"(R[24]), "=r"(R[25]), "=r"(R[26]), "=r"(R[27]), "=r"(R[28]), "=r"(R[29]),            \
          "=r"(R[30]), "=r"(R[31])                                                                              \
        : "r"(taddr + (OFF)))
    STF_LD32(0, r);
    STF_LD32(32, (r + 32));
#undef STF_LD32
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive 32-bit columns of this thread's TMEM lane from registers.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n"
        :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
           "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
           "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
           "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
        :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
           "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                 :: "r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Hidden-layer epilogue of one tile: this thread's TMEM lane (64 FP32 accumulator columns at
// t_acc), ReLU, FP16, into the first 32 columns of the tile's hidden operand at t_hid.
__device__ __forceinline__ void nn_hidden_epilogue(uint32_t t_acc, uint32_t t_hid)
{
    float v[64];
    tmem_ld64(t_acc, v);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t h[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) h[j] = relu_pack_h2(v[32 * q + 2 * j], v[32 * q + 2 * j + 1]);
        tmem_st16(t_hid + 16 * q, h);
    }
    tmem_wait_st();
}

// E4M3 variant: the 64 activations as 16 columns of four E4M3 each (K order low to high bytes).
__device__ __forceinline__ void nn_hidden_epilogue_e4m3(uint32_t t_acc, uint32_t t_hid)
{
    float v[64];
    tmem_ld64(t_acc, v);
    uint32_t h[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) h[j] = relu_pack_e4m3x4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    tmem_st16(t_hid, h);
    tmem_wait_st();
}

// One layer's three E4M3 products of one tile (K = 96: A from TMEM, 8 columns per K step of 32;
// B advanced by two 128-byte core matrices).
__device__ __forceinline__ void nn_issue_tile_f8(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, uint32_t mbar)
{
#pragma unroll
    for (int s = 0; s < kNnK8 / 32; ++s) nn_mma_ts_f8(d_tmem, a_tmem + 8 * s, b_desc + 16 * s, idesc, s > 0 ? 1u : 0u);
    nn_commit(mbar);
}

// One layer's K / 16 products of one tile, issued by one thread and committed to the tile's
// barrier. A from shared memory: a_desc / b_desc describe the first K step and a step advances
// both by 256 bytes (16 in the descriptors' address field).
template <int K>
__device__ __forceinline__ void nn_issue_tile(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc, uint32_t mbar)
{
#pragma unroll
    for (int s = 0; s < K / 16; ++s) nn_mma(d_tmem, a_desc + 16 * s, b_desc + 16 * s, idesc, s > 0 ? 1u : 0u);
    nn_commit(mbar);
}

// A from tensor memory: a K step advances A by 8 columns.
template <int K>
__device__ __forceinline__ void nn_issue_tile_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc, uint32_t mbar)
{
#pragma unroll
    for (int s = 0; s < K / 16; ++s) nn_mma_ts(d_tmem, a_tmem + 8 * s, b_desc + 16 * s, idesc, s > 0 ? 1u : 0u);
    nn_commit(mbar);
}

// The MMA warp (lane 0 issues): per round, wait for the clients' rows, issue layer 1 of both
// tiles, then each later layer of a tile as soon as the epilogue warpgroup has stored that tile's
// activations. Layer 1 of round r + 1 overwrites a tile's layer-1/2 accumulators, which the
// epilogue has read before its arrival that released layer 3 of round r; layer 3 accumulates
// elsewhere (kNnOutCol), so the next round starts without waiting for round r's outputs.
// Commits: mma[mt] completes twice per round (layers 1, 2), mma_out[mt] once (layer 3); neither
// runs more than one phase ahead of the epilogue, which consumes them in issue order.
template <bool TEST, bool F8>
__device__ __forceinline__ void nn_mma_role(NnPipeSmem& sm, int* flags)
{
    const uint32_t tmem = sm.tmem, b = smem_u32(sm.b);
    const uint32_t bar[2] = {smem_u32(&sm.mma[0]), smem_u32(&sm.mma[1])};
    const uint32_t bar_out[2] = {smem_u32(&sm.mma_out[0]), smem_u32(&sm.mma_out[1])};
    constexpr uint32_t sbo1 = kNnK1 / 8 * 128, sbo2 = kNnK2 / 8 * 128;
    constexpr bool f8 = F8;
    constexpr uint32_t sbo8 = kNnK8 / 16 * 128;
    const uint64_t b1 = nn_sdesc(b, 128, sbo1);
    const uint64_t b2 = f8 ? nn_sdesc(b + kNnB1Bytes, 128, sbo8) : nn_sdesc(b + kNnB1Bytes, 128, sbo2);
    const uint64_t b3 = f8 ? nn_sdesc(b + kNnB1Bytes + kNnB2Bytes8, 128, sbo8) : nn_sdesc(b + kNnB1Bytes + kNnB2Bytes, 128, sbo2);
    const bool leader = (threadIdx.x & 31) == 0;
    NnWaiter w{flags, 0};
    uint32_t eph[2] = {0u, 0u}, c12 = 0, c3 = 0;  // commits per tile on mma[] and on mma_out[]
    // failure-detection test switch (flags[2], decode-list kernel only): withhold round 0's
    // layer-1 products, so the epilogue's bounded wait for them runs out
    bool stall = false;
    if constexpr (TEST) stall = *reinterpret_cast<volatile int*>(flags + 2) != 0;
#pragma unroll 1
    for (uint32_t r = 0;; ++r) {
        const int slot = r & 1;
        w.wait(sm.in_full[slot], (r >> 1) & 1u);
        if (__shfl_sync(0xffffffffu, sm.more[slot], 0) == 0 || __any_sync(0xffffffffu, w.dead)) break;
        tc_fence_after();
        const uint32_t io = smem_u32(sm.io[slot]);
        const bool withhold = stall && r == 0;
        if (leader && !withhold)
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                nn_issue_tile<kNnK1>(tmem + mt * 64, nn_sdesc(io + mt * (kNnRows / 2 / 8) * sbo1, 128, sbo1), b1,
                                     nn_idesc(64), bar[mt]);
        c12 += withhold ? 1 : 2;
        c3 += 1;
#pragma unroll
        for (int layer = 2; layer <= 3; ++layer) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                w.wait(sm.epi[mt], eph[mt]);
                eph[mt] ^= 1u;
                tc_fence_after();
                if (leader) {
                    const uint32_t a = tmem + kNnHidCol + mt * kNnHidCols;
                    if constexpr (F8) {
                        if (layer == 2) nn_issue_tile_f8(tmem + mt * 64, a, b2, nn_idesc(64), bar[mt]);
                        else nn_issue_tile_f8(tmem + kNnOutCol + mt * 16, a, b3, nn_idesc(16), bar_out[mt]);
                    } else {
                        if (layer == 2) nn_issue_tile_ts<kNnK2>(tmem + mt * 64, a, b2, nn_idesc(64), bar[mt]);
                        else nn_issue_tile_ts<kNnK2>(tmem + kNnOutCol + mt * 16, a, b3, nn_idesc(16), bar_out[mt]);
                    }
                }
                __syncwarp();
            }
        }
    }
    // after a timeout, products may still be in flight: wait (bounded) for each barrier's last
    // commit before the teardown frees TMEM
    if (leader && c12 > 0 && w.dead)
        for (int mt = 0; mt < 2; ++mt) {
            for (unsigned it = 0; it < kNnWaitLimit && !nn_try_wait(bar[mt], (c12 - 1) & 1u); ++it) {}
            for (unsigned it = 0; it < kNnWaitLimit && !nn_try_wait(bar_out[mt], (c3 - 1) & 1u); ++it) {}
        }
}

// The epilogue warpgroup: per round and tile, turn layer 1 and 2 accumulators into the next
// layer's FP16 activations (in TMEM), then write the layer-3 outputs to shared memory.
template <bool TEST, bool F8>
__device__ __forceinline__ void nn_epilogue_role(NnPipeSmem& sm, int* flags)
{
    // row within a tile = TMEM lane: a warp reaches the 32 lanes of quarter (warp id mod 4)
    const int m = (((int)threadIdx.x >> 5) & 3) * 32 + ((int)threadIdx.x & 31);
    const uint32_t t_lane = sm.tmem + ((uint32_t)(m & ~31) << 16);
    // the constant bias columns of the hidden operands: K 64, 65 = 1, K 66 .. 79 = 0 (FP16, from
    // column 32); E4M3 variant: K 64 .. 66 = 1, K 67 .. 95 = 0 (from column 16)
    constexpr bool f8 = F8;
    {
        const uint32_t c[8] = {f8 ? 0x00383838u : 0x3c003c00u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        const uint32_t at = f8 ? 16u : 32u;
        tmem_st8(t_lane + kNnHidCol + at, c);
        tmem_st8(t_lane + kNnHidCol + kNnHidCols + at, c);
        tmem_wait_st();
    }
    NnWaiter w{flags, 0};
    uint32_t ph[2] = {0u, 0u}, po[2] = {0u, 0u};
    // under the failure-detection test switch (flags[2], decode-list kernel only) the warp stops
    // touching TMEM once a wait has timed out (products may still be running)
    bool guard = false;
    if constexpr (TEST) guard = *reinterpret_cast<volatile int*>(flags + 2) != 0;
    auto tile_wait = [&](int mt) {
        w.wait(sm.mma[mt], ph[mt]);
        ph[mt] ^= 1u;
        tc_fence_after();
    };
#pragma unroll 1
    for (uint32_t r = 0;; ++r) {
        const int slot = r & 1;
        w.wait(sm.in_full[slot], (r >> 1) & 1u);
        // leave together per warp (the TMEM accesses below are warp-collective)
        if (__shfl_sync(0xffffffffu, sm.more[slot], 0) == 0 || __any_sync(0xffffffffu, w.dead)) break;
#pragma unroll
        for (int layer = 2; layer <= 3; ++layer) {
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                tile_wait(mt);
                // after a timeout (test switch) no TMEM access, but the arrivals go on so the other
                // roles drain
                if (!(TEST && guard && __any_sync(0xffffffffu, w.dead))) {
                    if constexpr (F8) nn_hidden_epilogue_e4m3(t_lane + mt * 64, t_lane + kNnHidCol + mt * kNnHidCols);
                    else nn_hidden_epilogue(t_lane + mt * 64, t_lane + kNnHidCol + mt * kNnHidCols);
                }
                tc_fence_before();
                nn_arrive(smem_u32(&sm.epi[mt]));
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            w.wait(sm.mma_out[mt], po[mt]);
            po[mt] ^= 1u;
            tc_fence_after();
            float o[8];
            if constexpr (TEST) {
                if (guard && __any_sync(0xffffffffu, w.dead))
#pragma unroll
                    for (int c = 0; c < 8; ++c) o[c] = 0.0f;
                else
                    tmem_ld8(t_lane + kNnOutCol + mt * 16, o);
            } else {
                tmem_ld8(t_lane + kNnOutCol + mt * 16, o);
            }
            if constexpr (F8) {
                const float os = sm.out_scale;
#pragma unroll
                for (int c = 0; c < 8; ++c) o[c] *= os;
            }
            sm.out[slot][0][mt * 128 + m] = make_float4(o[0], o[1], o[2], o[3]);
            sm.out[slot][1][mt * 128 + m] = make_float4(o[4], o[5], o[6], o[7]);
        }
        tc_fence_before();
        nn_arrive(smem_u32(&sm.out_full[slot]));
    }
}

// The decode side of a pipeline block (threads kNnClients .. kNnPipeThreads - 1).
// TEST: honour the failure-detection test switch (the decode-list kernel).
template <bool TEST = false>
__device__ __forceinline__ void nn_decode_role(NnPipeSmem& sm, int* flags)
{
    // the decoder's format is fixed for the launch: each role is compiled for both and chosen once
    if ((threadIdx.x >> 5) == kNnMmaWarp) {
        if (sm.fp8) nn_mma_role<TEST, true>(sm, flags);
        else nn_mma_role<TEST, false>(sm, flags);
    } else {
        if (sm.fp8) nn_epilogue_role<TEST, true>(sm, flags);
        else nn_epilogue_role<TEST, false>(sm, flags);
    }
}

}  // namespace stf
