// Neural texel decoder: parameters, training kernels (forward, backward, Adam), inference
// export, checkpoints, and the neural material kind's texture and render entry points.
//
// Training runs on the CUDA cores in FP32 and is deterministic: parameter gradients are reduced
// over fixed chunks of the batch in a fixed order, and latent gradients are accumulated as 64-bit
// fixed-point integers, whose atomic sums do not depend on the order of the additions.
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <vector>

#include "stf.h"
#include "stf_internal.h"
#include "stf_neural.cuh"

using namespace stf;

namespace {

constexpr float kFixScaleF = 17592186044416.0f;    // 2^44: latent-gradient fixed point
constexpr float kFixInvF = 1.0f / 17592186044416.0f;

// Offsets inside the flat parameter vector W1, b1, W2, b2, W3, b3.
constexpr int oW1 = 0, ob1 = oW1 + kNnH * kNnIn, oW2 = ob1 + kNnH, ob2 = oW2 + kNnH * kNnH, oW3 = ob2 + kNnH,
              ob3 = oW3 + kNnOut * kNnH;

__device__ __forceinline__ uint32_t hash_u32(uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    pcg4d(a, b, c, d);
    return a;
}

__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    return (float)(hash_u32(a, b, c, d) >> 8) * (1.0f / 16777216.0f);
}

// Initialisation: latents uniform in [-0.1, 0.1]; weights uniform in +-sqrt(6 / fan_in); biases 0.
__global__ void k_nn_init(float* P, float* lat, long long nlat, uint32_t s0, uint32_t s1)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNnParams) {
        float v = 0.0f;
        float fan = 0.0f;
        if (i < ob1) fan = kNnIn;
        else if (i >= oW2 && i < ob2) fan = kNnH;
        else if (i >= oW3 && i < ob3) fan = kNnH;
        if (fan > 0.0f) v = (2.0f * hash_unit((uint32_t)i, 0x9e3779b9u, s0, s1) - 1.0f) * sqrtf(6.0f / fan);
        P[i] = v;
    }
    if (i < nlat) lat[i] = (2.0f * hash_unit((uint32_t)i, (uint32_t)(i >> 32) + 0x85ebca6bu, s0, s1) - 1.0f) * 0.1f;
}

// Training batch: texel b of step t, uniform over the W x H texels.
__global__ void k_nn_batch(int* idx, int n, int W, int H, uint32_t step, uint32_t s0, uint32_t s1)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const uint32_t r = hash_u32((uint32_t)b, step, s0, s1 ^ 0x5bd1e995u);
    const uint32_t t = (uint32_t)(((unsigned long long)r * (unsigned long long)(W * H)) >> 32);
    idx[b] = (int)((t % W) | ((t / W) << 16));
}

struct TrainArgs {
    const float* P;
    const float* lat;
    int gw, gh, rshift;
    float inv_r;
    float feat[16][4];
    const float* target;  // [H][W][8]
    int W;
    const int* idx;
    int n;
    float inv_count;       // 1 / (n * 8)
    float* part;           // [blocks][kNnParams] block-local parameter gradients
    unsigned long long* lat_acc;
    float* loss_part;      // [blocks]
};

constexpr int kTB = 64;    // texels per training block (256 threads: 4 per texel)
constexpr int kLD = 65;    // padded row of the 64-wide activation matrices (conflict-free columns)
constexpr int kSmemFloats = kNnParams + kTB * 25 + 4 * kTB * kLD + kTB * 9 + kTB * 4 + 256;
constexpr int kTrainSmemBytes = kSmemFloats * 4 + kTB * 4 * 4;

// One training block: 64 texels. Forward (layer by layer, activations in shared memory),
// backward, the block's partial parameter gradients (fixed order over its texels), and the
// latent gradient scattered into fixed-point accumulators.
__global__ void __launch_bounds__(256) k_nn_train_block(const TrainArgs a)
{
    extern __shared__ float sm[];
    float* sP = sm;
    float* X = sP + kNnParams;        // [64][25]
    float* H1 = X + kTB * 25;         // [64][65]
    float* H2 = H1 + kTB * kLD;
    float* G2 = H2 + kTB * kLD;
    float* G1 = G2 + kTB * kLD;
    float* G3 = G1 + kTB * kLD;       // [64][9]
    float* WC = G3 + kTB * 9;         // [64][4] corner weights
    float* red = WC + kTB * 4;        // [256]
    int* CELL = reinterpret_cast<int*>(red + 256);  // [64][4] corner cell indices
    const int tid = threadIdx.x, b = tid & (kTB - 1), q = tid >> 6;  // texel, quarter
    const int gb = blockIdx.x * kTB + b;
    const bool valid = gb < a.n;
    for (int i = tid; i < kNnParams; i += 256) sP[i] = a.P[i];
    // inputs: quarter q interpolates latent channels 4q..4q+3; quarter 0 adds the phase features
    int ix = 0, iy = 0;
    if (valid) { ix = a.idx[gb] & 0xffff; iy = a.idx[gb] >> 16; }
    {
        const float lx = (ix + 0.5f) * a.inv_r - 0.5f, ly = (iy + 0.5f) * a.inv_r - 0.5f;
        const float flx = floorf(lx), fly = floorf(ly);
        const float fx = lx - flx, fy = ly - fly;
        const int x0 = clampi((int)flx, 0, a.gw - 1), x1 = clampi((int)flx + 1, 0, a.gw - 1);
        const int y0 = clampi((int)fly, 0, a.gh - 1), y1 = clampi((int)fly + 1, 0, a.gh - 1);
        const float w[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
        const int cell[4] = {y0 * a.gw + x0, y0 * a.gw + x1, y1 * a.gw + x0, y1 * a.gw + x1};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ch = 4 * q + k;
            float s = 0.0f;
#pragma unroll
            for (int c = 0; c < 4; ++c) s = fmaf(w[c], a.lat[(size_t)cell[c] * kNnLat + ch], s);
            X[b * 25 + ch] = valid ? s : 0.0f;
        }
        if (q == 0) {
            const int mask = (1 << a.rshift) - 1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                X[b * 25 + 16 + k] = a.feat[ix & mask][k];
                X[b * 25 + 20 + k] = a.feat[iy & mask][k];
                WC[b * 4 + k] = valid ? w[k] : 0.0f;
                CELL[b * 4 + k] = cell[k];
            }
        }
    }
    __syncthreads();
    // layer 1: thread (b, q) computes outputs 16q .. 16q + 15
    {
        float acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = sP[ob1 + 16 * q + j];
        for (int i = 0; i < kNnIn; ++i) {
            const float xi = X[b * 25 + i];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(sP[oW1 + (16 * q + j) * kNnIn + i], xi, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) H1[b * kLD + 16 * q + j] = fmaxf(acc[j], 0.0f);
    }
    __syncthreads();
    {
        float acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = sP[ob2 + 16 * q + j];
        for (int i = 0; i < kNnH; ++i) {
            const float hi = H1[b * kLD + i];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(sP[oW2 + (16 * q + j) * kNnH + i], hi, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) H2[b * kLD + 16 * q + j] = fmaxf(acc[j], 0.0f);
    }
    __syncthreads();
    // layer 3 and the loss: quarter q computes outputs 2q, 2q + 1
    float loss = 0.0f;
    {
        float acc[2] = {sP[ob3 + 2 * q], sP[ob3 + 2 * q + 1]};
        for (int i = 0; i < kNnH; ++i) {
            const float hi = H2[b * kLD + i];
            acc[0] = fmaf(sP[oW3 + (2 * q) * kNnH + i], hi, acc[0]);
            acc[1] = fmaf(sP[oW3 + (2 * q + 1) * kNnH + i], hi, acc[1]);
        }
        const float* t = a.target + ((size_t)iy * a.W + ix) * kNnOut;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const float d = valid ? acc[j] - t[2 * q + j] : 0.0f;
            loss = fmaf(d * d, a.inv_count, loss);
            G3[b * 9 + 2 * q + j] = 2.0f * d * a.inv_count;
        }
    }
    __syncthreads();
    // g2 = (W3^T g3) masked by h2 > 0
    {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = 16 * q + j;
            float s = 0.0f;
#pragma unroll
            for (int o = 0; o < kNnOut; ++o) s = fmaf(sP[oW3 + o * kNnH + i], G3[b * 9 + o], s);
            G2[b * kLD + i] = H2[b * kLD + i] > 0.0f ? s : 0.0f;
        }
    }
    __syncthreads();
    // g1 = (W2^T g2) masked by h1 > 0
    {
        float acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
        for (int o = 0; o < kNnH; ++o) {
            const float g = G2[b * kLD + o];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = fmaf(sP[oW2 + o * kNnH + 16 * q + j], g, acc[j]);
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) G1[b * kLD + 16 * q + j] = H1[b * kLD + 16 * q + j] > 0.0f ? acc[j] : 0.0f;
    }
    __syncthreads();
    // latent gradient: quarter q handles channels 4q .. 4q + 3
    if (valid) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int ch = 4 * q + k;
            float s = 0.0f;
            for (int o = 0; o < kNnH; ++o) s = fmaf(sP[oW1 + o * kNnIn + ch], G1[b * kLD + o], s);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const long long v = __float2ll_rn(WC[b * 4 + c] * s * kFixScaleF);
                atomicAdd(a.lat_acc + (size_t)CELL[b * 4 + c] * kNnLat + ch, (unsigned long long)v);
            }
        }
    }
    // block-local parameter gradients, summed over the block's texels in order
    float* part = a.part + (size_t)blockIdx.x * kNnParams;
    for (int p = tid; p < kNnParams; p += 256) {
        const float* gsrc;
        const float* asrc;
        int gs, as, go, ao;
        if (p < ob1) { gsrc = G1; gs = kLD; go = p / kNnIn; asrc = X; as = 25; ao = p % kNnIn; }
        else if (p < oW2) { gsrc = G1; gs = kLD; go = p - ob1; asrc = nullptr; as = 0; ao = 0; }
        else if (p < ob2) { gsrc = G2; gs = kLD; go = (p - oW2) / kNnH; asrc = H1; as = kLD; ao = (p - oW2) % kNnH; }
        else if (p < oW3) { gsrc = G2; gs = kLD; go = p - ob2; asrc = nullptr; as = 0; ao = 0; }
        else if (p < ob3) { gsrc = G3; gs = 9; go = (p - oW3) / kNnH; asrc = H2; as = kLD; ao = (p - oW3) % kNnH; }
        else { gsrc = G3; gs = 9; go = p - ob3; asrc = nullptr; as = 0; ao = 0; }
        float s = 0.0f;
        if (asrc) {
            for (int t = 0; t < kTB; ++t) s = fmaf(gsrc[t * gs + go], asrc[t * as + ao], s);
        } else {
            for (int t = 0; t < kTB; ++t) s += gsrc[t * gs + go];
        }
        part[p] = s;
    }
    red[tid] = loss;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0) a.loss_part[blockIdx.x] = red[0];
}

// Sums the partials in chunk order; either writes the gradient or applies Adam. Thread 0 also
// sums the loss partials.
__global__ void k_nn_param_update(float* P, float* m, float* v, const float* part, int nchunks, const float* loss_part,
                                  int nloss, float* loss_out, float* grad_out, int adam, float lr, float b1, float b2,
                                  float eps, float c1, float c2)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        float s = 0.0f;
        for (int i = 0; i < nloss; ++i) s += loss_part[i];
        *loss_out = s;
    }
    if (p >= kNnParams) return;
    float g = 0.0f;
    for (int c = 0; c < nchunks; ++c) g += part[(size_t)c * kNnParams + p];
    if (grad_out) grad_out[p] = g;
    if (!adam) return;
    const float mm = b1 * m[p] + (1.0f - b1) * g;
    const float vv = b2 * v[p] + (1.0f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    P[p] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Latent gradients from the fixed-point accumulators (which are cleared); Adam, or export.
__global__ void k_nn_latent_update(float* lat, float* m, float* v, unsigned long long* acc, long long nlat, float* grad_out,
                                   int adam, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nlat) return;
    const float g = (float)(long long)acc[i] * kFixInvF;
    acc[i] = 0ull;
    if (grad_out) grad_out[i] = g;
    if (!adam) return;
    const float mm = b1 * m[i] + (1.0f - b1) * g;
    const float vv = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mm;
    v[i] = vv;
    lat[i] -= lr * (mm * c1) / (sqrtf(vv * c2) + eps);
}

// Inference copy: FP16 latents and the three layers as tensor-core B operand images, each bias
// in two extra K columns (FP16 high part and the FP16 rounding of the remainder).
__global__ void k_nn_export(const float* P, const float* lat, long long nlat, __half* lat16, __half* wimg)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nlat) lat16[i] = __float2half_rn(lat[i]);
    constexpr int n1 = 64 * kNnK1, n2 = 64 * kNnK2, n3 = 16 * kNnK2;
    if (i < n1 + n2 + n3) {
        int j = (int)i, r, k, K, base, nin, rows;
        const float *Wm, *bv;
        if (j < n1) { K = kNnK1; base = 0; Wm = P + oW1; bv = P + ob1; nin = kNnIn; rows = kNnH; }
        else if (j < n1 + n2) { j -= n1; K = kNnK2; base = kNnB1Bytes; Wm = P + oW2; bv = P + ob2; nin = kNnH; rows = kNnH; }
        else { j -= n1 + n2; K = kNnK2; base = kNnB1Bytes + kNnB2Bytes; Wm = P + oW3; bv = P + ob3; nin = kNnH; rows = kNnOut; }
        r = j / K;
        k = j % K;
        __half val = __float2half_rn(0.0f);
        if (r < rows) {
            if (k < nin) val = __float2half_rn(Wm[r * nin + k]);
            else if (k == nin) val = __float2half_rn(bv[r]);
            else if (k == nin + 1) val = __float2half_rn(bv[r] - __half2float(__float2half_rn(bv[r])));
        }
        wimg[(base + (r / 8) * (K / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2) / 2] = val;
    }
}

// The E4M3 variant's image (see kNnK8): layer 1 as k_nn_export with W1 and b1 scaled by
// s1 = 2^e1, then W2 / W3 as E4M3 of s2 W2 / s3 W3 and the three E4M3 parts of s1 s2 b2 and
// s1 s2 s3 b3 in K 64 .. 66 (every scaling exact, every difference of the parts exact).
__device__ __forceinline__ unsigned char nn_e4m3(float v) { return (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); }
__device__ __forceinline__ float nn_e4m3_value(unsigned char c)
{
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3)));
}

__global__ void k_nn_export_e4m3(const float* P, unsigned char* img, int e1, int e2, int e3)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float s1 = ldexpf(1.0f, e1), s2 = ldexpf(1.0f, e2), s3 = ldexpf(1.0f, e3);
    constexpr int n1 = 64 * kNnK1, n2 = 64 * kNnK8, n3 = 16 * kNnK8;
    if (i < n1) {
        const int r = i / kNnK1, k = i % kNnK1;
        const float b = s1 * P[ob1 + r];
        __half val = __float2half_rn(0.0f);
        if (k < kNnIn) val = __float2half_rn(s1 * P[oW1 + r * kNnIn + k]);
        else if (k == kNnIn) val = __float2half_rn(b);
        else if (k == kNnIn + 1) val = __float2half_rn(b - __half2float(__float2half_rn(b)));
        *reinterpret_cast<__half*>(img + (r / 8) * (kNnK1 / 8) * 128 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2) = val;
    } else if (i < n1 + n2 + n3) {
        int j = i - n1, base = kNnB1Bytes, rows = kNnH;
        const float* Wm = P + oW2;
        const float* bv = P + ob2;
        float sw = s2, sb = s1 * s2;
        if (j >= n2) { j -= n2; base += kNnB2Bytes8; rows = kNnOut; Wm = P + oW3; bv = P + ob3; sw = s3; sb = s1 * s2 * s3; }
        const int r = j / kNnK8, k = j % kNnK8;
        unsigned char val = 0;
        if (r < rows) {
            if (k < kNnH) val = nn_e4m3(sw * Wm[r * kNnH + k]);
            else if (k < kNnH + 3) {
                float v = sb * bv[r];
                unsigned char q = nn_e4m3(v);
                for (int t = kNnH; t < k; ++t) {  // the part k - 64 of v: peel the earlier parts
                    v -= nn_e4m3_value(q);
                    q = nn_e4m3(v);
                }
                val = q;
            }
        }
        img[base + (r / 8) * (kNnK8 / 16) * 128 + (k / 16) * 128 + (r % 8) * 16 + (k % 16)] = val;
    }
}

// Decodes a list of texels (packed ix | iy << 16) through the decode pipeline: persistent blocks,
// kNnClients texels per round (a tail round decodes fewer rows).
__global__ void __launch_bounds__(kNnPipeThreads, 2) k_nn_decode_list(const NeuralDev* nd, const int* idx, int n, int W,
                                                                      int H, float* out, int* flags)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    NnPipeSmem& sm = *reinterpret_cast<NnPipeSmem*>(dyn);
    nn_pipe_setup(sm, nd);
    if (threadIdx.x >= kNnClients) {
        nn_decode_role<true>(sm, flags);
    } else {
        const int row = threadIdx.x;
        NnWaiter w{flags, 0};
        uint32_t r = 0;
        int prev = -1;
#pragma unroll 1
        for (int base = blockIdx.x * kNnClients;; base += gridDim.x * kNnClients) {
            const bool more = base < n;
            const int i = base + row;
            if (more && i < n) {
                uint32_t in[12];
                nn_inputs(*nd, clampi(idx[i] & 0xffff, 0, W - 1), clampi(idx[i] >> 16, 0, H - 1), in);
                nn_put_inputs(sm, r & 1, row, in);
            }
            nn_publish(sm, r & 1, more ? 1 : 0);
            if (prev >= 0) {
                const uint32_t q = r - 1;
                w.wait(sm.out_full[q & 1], (q >> 1) & 1u);
                if (prev + row < n) {
                    float t[8];
                    nn_get_outputs(sm, q & 1, row, t);
                    float4* o = reinterpret_cast<float4*>(out + (size_t)(prev + row) * 8);
                    o[0] = make_float4(t[0], t[1], t[2], t[3]);
                    o[1] = make_float4(t[4], t[5], t[6], t[7]);
                }
            }
            if (!more) break;
            prev = base;
            ++r;
        }
    }
    nn_pipe_teardown(sm);
}

uint32_t crc32(const unsigned char* p, size_t n, uint32_t crc = 0)
{
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) {
        crc ^= p[i];
        for (int k = 0; k < 8; ++k) crc = (crc >> 1) ^ (0xEDB88320u & (0u - (crc & 1u)));
    }
    return ~crc;
}

}  // namespace

struct stf_decoder {
    stf_decoder_config cfg;
    int R, rshift;
    long long nlat;
    long long step;
    float *P = nullptr, *Pm = nullptr, *Pv = nullptr;
    float *lat = nullptr, *latm = nullptr, *latv = nullptr;
    unsigned long long* lat_acc = nullptr;
    __half* lat16 = nullptr;
    __half* wimg = nullptr;
    NeuralDev* dev = nullptr;  // device copy of the inference parameter block
    int infer_fmt = 0;         // STF_NN_FP16 or STF_NN_E4M3
    int e8[4] = {0, 0, 0, 0};  // E4M3 variant: log2 s1, s2, s3 and of the output scale
    float feat[16][4];         // FP32 phase features (training)
    // per-batch scratch
    int cap = 0;
    int* idx = nullptr;
    float* part = nullptr;
    float* loss_part = nullptr;
    float* loss = nullptr;
};

namespace {

template <class T> cudaError_t dalloc(T** p, size_t count) { return cudaMalloc((void**)p, count * sizeof(T)); }

void dfree(stf_decoder* d)
{
    void* ps[] = {d->P, d->Pm, d->Pv, d->lat, d->latm, d->latv, d->lat_acc, d->lat16, d->wimg, d->dev,
                  d->idx, d->part, d->loss_part, d->loss};
    for (void* p : ps)
        if (p) cudaFree(p);
}

stf_status check_config(const stf_decoder_config* c, int* rshift)
{
    if (!c) return stf_fail(STF_ERR_INVALID_ARG, "null decoder config");
    if (c->tex_w < 1 || c->tex_h < 1 || c->tex_w > 16384 || c->tex_h > 16384)
        return stf_fail(STF_ERR_INVALID_ARG, "decoder texture size %dx%d", c->tex_w, c->tex_h);
    if (c->latent_w < 1 || c->latent_h < 1 || c->tex_w % c->latent_w || c->tex_h % c->latent_h)
        return stf_fail(STF_ERR_INVALID_ARG, "latent grid %dx%d must divide the texture", c->latent_w, c->latent_h);
    const int R = c->tex_w / c->latent_w;
    if (R != c->tex_h / c->latent_h || R > 16 || (R & (R - 1)))
        return stf_fail(STF_ERR_INVALID_ARG, "texels per latent cell must be the same power of two <= 16 on both axes");
    if (c->batch < 256 || c->batch % 256 || c->batch > (1 << 22))
        return stf_fail(STF_ERR_INVALID_ARG, "batch %d must be a multiple of 256 in [256, 4194304]", c->batch);
    int s = 0;
    while ((1 << s) < R) ++s;
    *rshift = s;
    return STF_OK;
}

stf_status alloc_decoder(stf_decoder* d)
{
    cudaError_t e;
    const long long nl = d->nlat;
    if ((e = dalloc(&d->P, kNnParams)) || (e = dalloc(&d->Pm, kNnParams)) || (e = dalloc(&d->Pv, kNnParams)) ||
        (e = dalloc(&d->lat, nl)) || (e = dalloc(&d->latm, nl)) || (e = dalloc(&d->latv, nl)) ||
        (e = dalloc(&d->lat_acc, nl)) || (e = dalloc(&d->lat16, nl)) || (e = dalloc(&d->wimg, kNnImgBytes / 2)) ||
        (e = dalloc(&d->dev, 1)) || (e = dalloc(&d->loss, 1)))
        return stf_cuda_fail(e, "decoder allocation");
    cudaMemset(d->Pm, 0, kNnParams * 4);
    cudaMemset(d->Pv, 0, kNnParams * 4);
    cudaMemset(d->latm, 0, nl * 4);
    cudaMemset(d->latv, 0, nl * 4);
    if ((e = cudaMemset(d->lat_acc, 0, nl * 8)) != cudaSuccess) return stf_cuda_fail(e, "cudaMemset");
    // phase features sin/cos(2 pi phi), sin/cos(4 pi phi), phi = (p + 0.5) / R, computed in FP64
    NeuralDev h;
    memset(&h, 0, sizeof h);
    for (int p = 0; p < 16; ++p) {
        const double phi = ((p % d->R) + 0.5) / d->R;
        const double v[4] = {sin(2.0 * M_PI * phi), cos(2.0 * M_PI * phi), sin(4.0 * M_PI * phi), cos(4.0 * M_PI * phi)};
        for (int k = 0; k < 4; ++k) d->feat[p][k] = (float)v[k];
        const __half2 a = __floats2half2_rn((float)v[0], (float)v[1]);
        const __half2 b = __floats2half2_rn((float)v[2], (float)v[3]);
        h.feat[p] = make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
    }
    h.lat16 = reinterpret_cast<const uint4*>(d->lat16);
    h.wimg = reinterpret_cast<const uint4*>(d->wimg);
    h.gw = d->cfg.latent_w;
    h.gh = d->cfg.latent_h;
    h.rshift = d->rshift;
    h.inv_r = 1.0f / (float)d->R;
    if ((e = cudaMemcpy(d->dev, &h, sizeof h, cudaMemcpyHostToDevice)) != cudaSuccess) return stf_cuda_fail(e, "cudaMemcpy");
    return STF_OK;
}

stf_status ensure_scratch(stf_decoder* d, int n)
{
    if (n <= d->cap) return STF_OK;
    for (void* p : {(void*)d->idx, (void*)d->part, (void*)d->loss_part})
        if (p) cudaFree(p);
    d->idx = nullptr; d->part = nullptr; d->loss_part = nullptr;
    const int nb = (n + kTB - 1) / kTB;
    cudaError_t e;
    if ((e = dalloc(&d->idx, n)) || (e = dalloc(&d->part, (size_t)nb * kNnParams)) || (e = dalloc(&d->loss_part, nb)))
        return stf_cuda_fail(e, "decoder scratch allocation");
    d->cap = n;
    return STF_OK;
}

// floor(log2(v)) of a positive v, exactly.
int floor_log2(double v)
{
    int e;
    (void)std::frexp(v, &e);
    return e - 1;
}

// The E4M3 variant's power-of-two exponents from the FP16 latent grid and the FP32 parameters,
// every sum in FP64 in index order (m = 1.0625, one E4M3 rounding):
//   xmax_k  max |latent k| over the grid (k < 16), 1 for the position features;
//   B1_j    m sum_k |W1_jk| xmax_k + |b1_j|  (bounds |h1_j|),  B2_i  m^2 sum_j |W2_ij| B1_j + |b2_i|;
//   e1      floor(log2(448 / max B1)), at most 8;
//   e2      floor(log2(min(448 / (2^e1 max B2), 448 / max |W2|)));
//   e3      floor(log2(min(448 / max |W3|, 448 / (2^(e1 + e2) max |b3|))));
// e[3] = -(e1 + e2 + e3), the output scale's exponent. No activation or weight then exceeds 448.
void e4m3_exponents(const std::vector<__half>& lat16, const std::vector<float>& P, int (&e)[4])
{
    const double m = 1.0625;
    double xmax[kNnIn];
    for (int k = 0; k < kNnIn; ++k) xmax[k] = k < kNnLat ? 0.0 : 1.0;
    for (size_t c = 0; c + kNnLat <= lat16.size(); c += kNnLat)
        for (int k = 0; k < kNnLat; ++k) xmax[k] = std::max(xmax[k], std::fabs((double)__half2float(lat16[c + k])));
    double B1[kNnH], maxB1 = 0.0, maxB2 = 0.0, maxW2 = 0.0, maxW3 = 0.0, maxb3 = 0.0;
    for (int j = 0; j < kNnH; ++j) {
        double t = 0.0;
        for (int k = 0; k < kNnIn; ++k) t += std::fabs((double)P[oW1 + j * kNnIn + k]) * xmax[k];
        B1[j] = m * t + std::fabs((double)P[ob1 + j]);
        maxB1 = std::max(maxB1, B1[j]);
    }
    for (int i = 0; i < kNnH; ++i) {
        double t = 0.0;
        for (int j = 0; j < kNnH; ++j) {
            const double w = std::fabs((double)P[oW2 + i * kNnH + j]);
            t += w * B1[j];
            maxW2 = std::max(maxW2, w);
        }
        maxB2 = std::max(maxB2, m * m * t + std::fabs((double)P[ob2 + i]));
    }
    for (int k = 0; k < kNnOut * kNnH; ++k) maxW3 = std::max(maxW3, std::fabs((double)P[oW3 + k]));
    for (int o = 0; o < kNnOut; ++o) maxb3 = std::max(maxb3, std::fabs((double)P[ob3 + o]));
    int e1 = maxB1 > 0.0 ? floor_log2(448.0 / maxB1) : 8;
    if (e1 > 8) e1 = 8;
    double lim2 = maxW2 > 0.0 ? 448.0 / maxW2 : INFINITY;
    if (maxB2 > 0.0) lim2 = std::min(lim2, 448.0 / (std::ldexp(1.0, e1) * maxB2));
    const int e2 = std::isinf(lim2) ? 0 : floor_log2(lim2);
    double lim3 = maxW3 > 0.0 ? 448.0 / maxW3 : INFINITY;
    if (maxb3 > 0.0) lim3 = std::min(lim3, 448.0 / (std::ldexp(1.0, e1 + e2) * maxb3));
    const int e3 = std::isinf(lim3) ? 0 : floor_log2(lim3);
    e[0] = e1;
    e[1] = e2;
    e[2] = e3;
    e[3] = -(e1 + e2 + e3);
}

// The inference copy of the parameters: FP16 latents, and the weight image of the decoder's
// inference format (for the E4M3 variant, its exponents from the exported latents and the
// current parameters), then the format fields of the device parameter block.
stf_status export_inference(stf_decoder* d, cudaStream_t s)
{
    const long long n = d->nlat > kNnImgBytes / 2 ? d->nlat : kNnImgBytes / 2;
    k_nn_export<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d->P, d->lat, d->nlat, d->lat16, d->wimg);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return stf_cuda_fail(e, "export kernel");
    int fp8 = 0;
    float os = 1.0f;
    if (d->infer_fmt == STF_NN_E4M3) {
        std::vector<__half> lat((size_t)d->nlat);
        std::vector<float> P(kNnParams);
        if ((e = cudaMemcpyAsync(lat.data(), d->lat16, lat.size() * sizeof(__half), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(P.data(), d->P, P.size() * sizeof(float), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return stf_cuda_fail(e, "reading the parameters for the E4M3 scales");
        e4m3_exponents(lat, P, d->e8);
        constexpr int nimg = 64 * kNnK1 + 64 * kNnK8 + 16 * kNnK8;
        k_nn_export_e4m3<<<(nimg + 255) / 256, 256, 0, s>>>(d->P, reinterpret_cast<unsigned char*>(d->wimg), d->e8[0],
                                                            d->e8[1], d->e8[2]);
        if ((e = cudaGetLastError()) != cudaSuccess) return stf_cuda_fail(e, "E4M3 export kernel");
        fp8 = 1;
        os = std::ldexp(1.0f, d->e8[3]);
    }
    struct { int fp8; float out_scale; } f{fp8, os};
    static_assert(offsetof(NeuralDev, out_scale) == offsetof(NeuralDev, fp8) + sizeof(int), "adjacent fields");
    if ((e = cudaMemcpyAsync(reinterpret_cast<char*>(d->dev) + offsetof(NeuralDev, fp8), &f, sizeof f, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return stf_cuda_fail(e, "inference format");
    return STF_OK;
}

stf_status target_args(const stf_decoder* d, const stf_texture* t)
{
    if (!t) return stf_fail(STF_ERR_INVALID_ARG, "null training target");
    if (t->kind != K_F32x8 || t->channels != 8)
        return stf_fail(STF_ERR_INVALID_ARG, "training target must be an 8-channel FP32 texture");
    if (t->width != d->cfg.tex_w || t->height != d->cfg.tex_h)
        return stf_fail(STF_ERR_INVALID_ARG, "training target %dx%d differs from the decoder's %dx%d", t->width, t->height,
                        d->cfg.tex_w, d->cfg.tex_h);
    return STF_OK;
}

// Forward + backward over idx[0..n) (already on the device), then the gradient reduction.
stf_status run_batch(stf_decoder* d, const stf_texture* target, int n, int adam, float* grad_p, float* grad_l, cudaStream_t s)
{
    TrainArgs a;
    a.P = d->P;
    a.lat = d->lat;
    a.gw = d->cfg.latent_w;
    a.gh = d->cfg.latent_h;
    a.rshift = d->rshift;
    a.inv_r = 1.0f / (float)d->R;
    memcpy(a.feat, d->feat, sizeof a.feat);
    a.target = (const float*)target->texels;
    a.W = d->cfg.tex_w;
    a.idx = d->idx;
    a.n = n;
    a.inv_count = (float)(1.0 / ((double)n * kNnOut));
    a.part = d->part;
    a.lat_acc = d->lat_acc;
    a.loss_part = d->loss_part;
    const int nb = (n + kTB - 1) / kTB;
    cudaError_t ea = cudaFuncSetAttribute(k_nn_train_block, cudaFuncAttributeMaxDynamicSharedMemorySize, kTrainSmemBytes);
    if (ea != cudaSuccess) return stf_cuda_fail(ea, "cudaFuncSetAttribute");
    k_nn_train_block<<<nb, 256, kTrainSmemBytes, s>>>(a);
    const int nch = nb;
    const double t = (double)(d->step + 1);
    const float c1 = adam ? (float)(1.0 / (1.0 - pow(d->cfg.beta1, t))) : 1.0f;
    const float c2 = adam ? (float)(1.0 / (1.0 - pow(d->cfg.beta2, t))) : 1.0f;
    k_nn_param_update<<<(kNnParams + 255) / 256, 256, 0, s>>>(d->P, d->Pm, d->Pv, d->part, nch, d->loss_part, nb, d->loss,
                                                               grad_p, adam, d->cfg.lr_mlp, d->cfg.beta1, d->cfg.beta2,
                                                               d->cfg.eps, c1, c2);
    k_nn_latent_update<<<(unsigned)((d->nlat + 255) / 256), 256, 0, s>>>(d->lat, d->latm, d->latv, d->lat_acc, d->nlat, grad_l,
                                                                         adam, d->cfg.lr_latent, d->cfg.beta1, d->cfg.beta2,
                                                                         d->cfg.eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "training kernels");
}

struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t tex_w, tex_h, latent_w, latent_h, batch;
    float lr_latent, lr_mlp, beta1, beta2, eps;
    uint64_t seed;
    int64_t step;
    int64_t nlat;
    int32_t nparams;
    int32_t pad;
};

}  // namespace

extern "C" stf_status stf_decoder_create(const stf_decoder_config* cfg, stf_decoder** out)
{
    if (!out) return stf_fail(STF_ERR_INVALID_ARG, "null output handle");
    int rs = 0;
    stf_status st = check_config(cfg, &rs);
    if (st != STF_OK) return st;
    stf_decoder* d = new (std::nothrow) stf_decoder();
    if (!d) return stf_fail(STF_ERR_OUT_OF_MEMORY, "host allocation");
    d->cfg = *cfg;
    d->rshift = rs;
    d->R = 1 << rs;
    d->nlat = (long long)cfg->latent_w * cfg->latent_h * kNnLat;
    d->step = 0;
    if ((st = alloc_decoder(d)) != STF_OK) { dfree(d); delete d; return st; }
    const long long n = d->nlat > kNnParams ? d->nlat : kNnParams;
    k_nn_init<<<(unsigned)((n + 255) / 256), 256>>>(d->P, d->lat, d->nlat, (uint32_t)cfg->seed, (uint32_t)(cfg->seed >> 32));
    if ((st = export_inference(d, 0)) != STF_OK) { dfree(d); delete d; return st; }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { dfree(d); delete d; return stf_cuda_fail(e, "decoder init"); }
    *out = d;
    return STF_OK;
}

extern "C" stf_status stf_decoder_destroy(stf_decoder* d)
{
    if (!d) return STF_OK;
    dfree(d);
    delete d;
    return STF_OK;
}

extern "C" stf_status stf_decoder_train(stf_decoder* d, const stf_texture* target, int steps, float* losses)
{
    if (!d) return stf_fail(STF_ERR_INVALID_ARG, "null decoder");
    if (steps < 0) return stf_fail(STF_ERR_INVALID_ARG, "steps %d < 0", steps);
    stf_status st = target_args(d, target);
    if (st != STF_OK) return st;
    if ((st = ensure_scratch(d, d->cfg.batch)) != STF_OK) return st;
    cudaStream_t s = stf_stream();
    const int n = d->cfg.batch;
    for (int i = 0; i < steps; ++i) {
        k_nn_batch<<<(n + 255) / 256, 256, 0, s>>>(d->idx, n, d->cfg.tex_w, d->cfg.tex_h, (uint32_t)d->step,
                                                   (uint32_t)d->cfg.seed, (uint32_t)(d->cfg.seed >> 32));
        if ((st = run_batch(d, target, n, 1, nullptr, nullptr, s)) != STF_OK) return st;
        if (losses) {
            cudaError_t e = cudaMemcpyAsync(losses + i, d->loss, 4, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) return stf_cuda_fail(e, "loss copy");
        }
        ++d->step;
    }
    if ((st = export_inference(d, s)) != STF_OK) return st;
    cudaError_t e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "training");
}

extern "C" stf_status stf_decoder_gradients(stf_decoder* d, const stf_texture* target, const int32_t* texels, int n,
                                            float* grad_params, float* grad_latent, float* loss)
{
    if (!d || !texels || n < 1) return stf_fail(STF_ERR_INVALID_ARG, "stf_decoder_gradients: bad arguments");
    stf_status st = target_args(d, target);
    if (st != STF_OK) return st;
    for (int i = 0; i < n; ++i) {
        const int x = texels[i] & 0xffff, y = texels[i] >> 16;
        if (x >= d->cfg.tex_w || y < 0 || y >= d->cfg.tex_h) return stf_fail(STF_ERR_INVALID_ARG, "texel %d out of range", i);
    }
    if ((st = ensure_scratch(d, n)) != STF_OK) return st;
    cudaStream_t s = stf_stream();
    float *gp = nullptr, *gl = nullptr;
    cudaError_t e;
    if ((e = dalloc(&gp, kNnParams)) || (e = dalloc(&gl, d->nlat))) {
        if (gp) cudaFree(gp);
        return stf_cuda_fail(e, "gradient buffers");
    }
    e = cudaMemcpyAsync(d->idx, texels, (size_t)n * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) st = run_batch(d, target, n, 0, gp, gl, s);
    if (e == cudaSuccess && st == STF_OK && grad_params) e = cudaMemcpyAsync(grad_params, gp, kNnParams * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && st == STF_OK && grad_latent) e = cudaMemcpyAsync(grad_latent, gl, d->nlat * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && st == STF_OK && loss) e = cudaMemcpyAsync(loss, d->loss, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(gp);
    cudaFree(gl);
    if (st != STF_OK) return st;
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "gradients");
}

extern "C" stf_status stf_decoder_get_params(const stf_decoder* d, float* latent, float* params)
{
    if (!d) return stf_fail(STF_ERR_INVALID_ARG, "null decoder");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && latent) e = cudaMemcpy(latent, d->lat, d->nlat * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && params) e = cudaMemcpy(params, d->P, kNnParams * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "get params");
}

extern "C" stf_status stf_decoder_set_params(stf_decoder* d, const float* latent, const float* params)
{
    if (!d) return stf_fail(STF_ERR_INVALID_ARG, "null decoder");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && latent) e = cudaMemcpy(d->lat, latent, d->nlat * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && params) e = cudaMemcpy(d->P, params, kNnParams * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return stf_cuda_fail(e, "set params");
    stf_status st = export_inference(d, 0);
    if (st != STF_OK) return st;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "set params");
}

extern "C" stf_status stf_decoder_decode(const stf_decoder* d, const int32_t* texels, int n, float* out)
{
    if (!d || !texels || !out || n < 0) return stf_fail(STF_ERR_INVALID_ARG, "stf_decoder_decode: bad arguments");
    if (((uintptr_t)out & 15) != 0) return stf_fail(STF_ERR_INVALID_ARG, "out must be 16-byte aligned");
    if (n == 0) return STF_OK;
    int* flags = nullptr;
    stf_status st = stf_device_state(&flags, nullptr);
    if (st != STF_OK) return st;
    static int per_sm = 0;
    cudaError_t e = cudaSuccess;
    if (!per_sm) {
        e = cudaFuncSetAttribute(k_nn_decode_list, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(NnPipeSmem));
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_nn_decode_list, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e == cudaSuccess) e = stf_resident_blocks(reinterpret_cast<const void*>(k_nn_decode_list), kNnPipeThreads, (int)sizeof(NnPipeSmem), &per_sm);
        if (e != cudaSuccess) return stf_cuda_fail(e, "decode kernel set-up");
        if (per_sm < 1) per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rounds = (n + kNnClients - 1) / kNnClients;
    const int blocks = rounds < per_sm * sms ? rounds : per_sm * sms;
    k_nn_decode_list<<<blocks, kNnPipeThreads, sizeof(NnPipeSmem), stf_stream()>>>(d->dev, texels, n, d->cfg.tex_w, d->cfg.tex_h, out, flags);
    e = cudaGetLastError();
    return e == cudaSuccess ? STF_OK : stf_cuda_fail(e, "decode kernel");
}

extern "C" stf_status stf_decoder_set_inference(stf_decoder* d, int format, int* exponents)
{
    if (!d) return stf_fail(STF_ERR_INVALID_ARG, "null decoder");
    if (format != STF_NN_FP16 && format != STF_NN_E4M3)
        return stf_fail(STF_ERR_INVALID_ARG, "inference format %d (STF_NN_FP16 or STF_NN_E4M3)", format);
    const int before = d->infer_fmt;
    d->infer_fmt = format;
    stf_status st = export_inference(d, stf_stream());
    if (st != STF_OK) {
        d->infer_fmt = before;  // the device copy may be half refreshed: the next refresh redoes it
        return st;
    }
    if (exponents)
        for (int k = 0; k < 4; ++k) exponents[k] = format == STF_NN_E4M3 ? d->e8[k] : 0;
    return STF_OK;
}

extern "C" stf_status stf_decoder_info(const stf_decoder* d, stf_decoder_config* cfg, long long* step)
{
    if (!d) return stf_fail(STF_ERR_INVALID_ARG, "null decoder");
    if (cfg) *cfg = d->cfg;
    if (step) *step = d->step;
    return STF_OK;
}

extern "C" stf_status stf_decoder_save(const stf_decoder* d, const char* path)
{
    if (!d || !path) return stf_fail(STF_ERR_INVALID_ARG, "stf_decoder_save: bad arguments");
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "STFDEC01", 8);
    h.version = 1;
    h.tex_w = d->cfg.tex_w; h.tex_h = d->cfg.tex_h; h.latent_w = d->cfg.latent_w; h.latent_h = d->cfg.latent_h;
    h.batch = d->cfg.batch;
    h.lr_latent = d->cfg.lr_latent; h.lr_mlp = d->cfg.lr_mlp; h.beta1 = d->cfg.beta1; h.beta2 = d->cfg.beta2; h.eps = d->cfg.eps;
    h.seed = d->cfg.seed;
    h.step = d->step;
    h.nlat = d->nlat;
    h.nparams = kNnParams;
    std::vector<float> buf(3 * (size_t)d->nlat + 3 * kNnParams);
    cudaError_t e = cudaDeviceSynchronize();
    const float* src[6] = {d->lat, d->latm, d->latv, d->P, d->Pm, d->Pv};
    size_t off = 0;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
        const size_t cnt = k < 3 ? (size_t)d->nlat : (size_t)kNnParams;
        e = cudaMemcpy(buf.data() + off, src[k], cnt * 4, cudaMemcpyDeviceToHost);
        off += cnt;
    }
    if (e != cudaSuccess) return stf_cuda_fail(e, "checkpoint read-back");
    uint32_t crc = crc32((const unsigned char*)&h, sizeof h);
    crc = crc32((const unsigned char*)buf.data(), buf.size() * 4, crc);
    FILE* f = fopen(path, "wb");
    if (!f) return stf_fail(STF_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(buf.data(), 4, buf.size(), f) == buf.size() &&
                    fwrite(&crc, 4, 1, f) == 1;
    fclose(f);
    return ok ? STF_OK : stf_fail(STF_ERR_INVALID_ARG, "short write to %s", path);
}

extern "C" stf_status stf_decoder_load(const char* path, stf_decoder** out)
{
    if (!path || !out) return stf_fail(STF_ERR_INVALID_ARG, "stf_decoder_load: bad arguments");
    FILE* f = fopen(path, "rb");
    if (!f) return stf_fail(STF_ERR_INVALID_ARG, "cannot open %s", path);
    CkptHeader h;
    if (fread(&h, sizeof h, 1, f) != 1 || memcmp(h.magic, "STFDEC01", 8) != 0 || h.version != 1 || h.nparams != kNnParams) {
        fclose(f);
        return stf_fail(STF_ERR_INVALID_ARG, "%s is not a decoder checkpoint", path);
    }
    stf_decoder_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.tex_w = h.tex_w; cfg.tex_h = h.tex_h; cfg.latent_w = h.latent_w; cfg.latent_h = h.latent_h; cfg.batch = h.batch;
    cfg.lr_latent = h.lr_latent; cfg.lr_mlp = h.lr_mlp; cfg.beta1 = h.beta1; cfg.beta2 = h.beta2; cfg.eps = h.eps;
    cfg.seed = h.seed;
    int rs = 0;
    stf_status st = check_config(&cfg, &rs);
    if (st != STF_OK || h.nlat != (int64_t)cfg.latent_w * cfg.latent_h * kNnLat) {
        fclose(f);
        return stf_fail(STF_ERR_INVALID_ARG, "%s: inconsistent checkpoint header", path);
    }
    std::vector<float> buf(3 * (size_t)h.nlat + 3 * kNnParams);
    uint32_t crc_file = 0;
    const bool ok = fread(buf.data(), 4, buf.size(), f) == buf.size() && fread(&crc_file, 4, 1, f) == 1 && fgetc(f) == EOF;
    fclose(f);
    if (!ok) return stf_fail(STF_ERR_INVALID_ARG, "%s: truncated or oversized checkpoint", path);
    uint32_t crc = crc32((const unsigned char*)&h, sizeof h);
    crc = crc32((const unsigned char*)buf.data(), buf.size() * 4, crc);
    if (crc != crc_file) return stf_fail(STF_ERR_INVALID_ARG, "%s: checksum mismatch (corrupted checkpoint)", path);
    stf_decoder* d = new (std::nothrow) stf_decoder();
    if (!d) return stf_fail(STF_ERR_OUT_OF_MEMORY, "host allocation");
    d->cfg = cfg;
    d->rshift = rs;
    d->R = 1 << rs;
    d->nlat = h.nlat;
    d->step = h.step;
    if ((st = alloc_decoder(d)) != STF_OK) { dfree(d); delete d; return st; }
    float* dst[6] = {d->lat, d->latm, d->latv, d->P, d->Pm, d->Pv};
    size_t off = 0;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
        const size_t cnt = k < 3 ? (size_t)d->nlat : (size_t)kNnParams;
        e = cudaMemcpy(dst[k], buf.data() + off, cnt * 4, cudaMemcpyHostToDevice);
        off += cnt;
    }
    if (e != cudaSuccess) { dfree(d); delete d; return stf_cuda_fail(e, "checkpoint upload"); }
    if ((st = export_inference(d, 0)) != STF_OK || (e = cudaDeviceSynchronize()) != cudaSuccess) {
        dfree(d);
        delete d;
        return st != STF_OK ? st : stf_cuda_fail(e, "checkpoint export");
    }
    *out = d;
    return STF_OK;
}

// ------------------------------------------------------------------------------ neural textures

stf_status stf_create_neural_texture(const stf_texture_desc* desc, stf_texture** out)
{
    const stf_decoder* d = desc->decoder;
    if (desc->width != d->cfg.tex_w || desc->height != d->cfg.tex_h)
        return stf_fail(STF_ERR_INVALID_ARG, "neural texture %dx%d differs from its decoder's %dx%d", desc->width,
                        desc->height, d->cfg.tex_w, d->cfg.tex_h);
    stf_texture* t = new (std::nothrow) stf_texture();
    if (!t) return stf_fail(STF_ERR_OUT_OF_MEMORY, "host allocation");
    t->width = desc->width;
    t->height = desc->height;
    t->channels = 8;
    t->kind = K_NEURAL;
    t->texels = nullptr;
    t->scales = nullptr;
    t->scale_shift = 14;
    t->scale_tiles_x = 1;
    t->decoder = d;
    t->decoder_params = d->dev;
    *out = t;
    return STF_OK;
}

namespace stf {
cudaError_t launch_view_NEURAL(const DevView&, int, cudaStream_t);
}

cudaError_t stf_launch_neural_view(const DevView& d, int mode, cudaStream_t s) { return launch_view_NEURAL(d, mode, s); }
