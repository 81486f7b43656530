// simt_mlp.cuh -- the density and colour MLPs (Sec. 6) in fp32 on the CUDA
// cores with the weights in shared memory; shared by the fp32 renderer and
// the training kernels.
#pragma once
#include "common.cuh"

namespace vrn {

// Shared-memory weight layout (SIMT-friendly, float4 rows):
// W1 [64][D], W2^T [64][16], W3 [64][32], W4 [64][64], W5^T [64][4]
template <int D>
struct SimtW {
    static constexpr int oW1 = 0;
    static constexpr int oW2T = oW1 + 64 * D;
    static constexpr int oW3 = oW2T + 64 * 16;
    static constexpr int oW4 = oW3 + 64 * 32;
    static constexpr int oW5T = oW4 + 64 * 64;
    static constexpr int size = oW5T + 64 * 4;
};

template <int D>
__device__ void load_weights_simt(const float *__restrict__ mlp, float *s) {
    using W = SimtW<D>;
    for (int i = threadIdx.x; i < 64 * D; i += blockDim.x) s[W::oW1 + i] = mlp[i];
    const float *W2 = mlp + 64 * D;
    for (int i = threadIdx.x; i < 64 * 16; i += blockDim.x) s[W::oW2T + i] = W2[(i & 15) * 64 + (i >> 4)];
    const float *W3 = W2 + 16 * 64;
    for (int i = threadIdx.x; i < 64 * 32; i += blockDim.x) s[W::oW3 + i] = W3[i];
    const float *W4 = W3 + 64 * 32;
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) s[W::oW4 + i] = W4[i];
    const float *W5 = W4 + 64 * 64;
    for (int i = threadIdx.x; i < 64 * 4; i += blockDim.x) {
        int j = i >> 2, c = i & 3;
        s[W::oW5T + i] = c < 3 ? W5[c * 64 + j] : 0.0f;
    }
}

// Density MLP (D -> 64 -> 16, ReLU), sigma = exp(o_0 + bias); colour MLP
// ([o, SH(d)] 32 -> 64 -> 64 -> 3, ReLU) and sigmoid to PQ colour.
template <int D>
__device__ __forceinline__ void mlp_simt(const float *__restrict__ s, const float feat[D],
                                         const float dir[3], float density_bias, float &sigma,
                                         float rgb[3], float o_out[16] = nullptr) {
    using W = SimtW<D>;
    float o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = 0.0f;
#pragma unroll 4
    for (int j = 0; j < 64; ++j) {
        const float4 *w = reinterpret_cast<const float4 *>(s + W::oW1 + j * D);
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < D / 4; ++k) {
            float4 q = w[k];
            a = fmaf(q.x, feat[4 * k], a);
            a = fmaf(q.y, feat[4 * k + 1], a);
            a = fmaf(q.z, feat[4 * k + 2], a);
            a = fmaf(q.w, feat[4 * k + 3], a);
        }
        a = fmaxf(a, 0.0f);
        const float4 *w2 = reinterpret_cast<const float4 *>(s + W::oW2T + j * 16);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float4 q = w2[k];
            o[4 * k] = fmaf(q.x, a, o[4 * k]);
            o[4 * k + 1] = fmaf(q.y, a, o[4 * k + 1]);
            o[4 * k + 2] = fmaf(q.z, a, o[4 * k + 2]);
            o[4 * k + 3] = fmaf(q.w, a, o[4 * k + 3]);
        }
    }
    sigma = expf(o[0] + density_bias);
    if (o_out) {
#pragma unroll
        for (int i = 0; i < 16; ++i) o_out[i] = o[i];
    }
    float x[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = o[i];
    sh16(dir[0], dir[1], dir[2], x + 16);
    float h1[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) {
        const float4 *w = reinterpret_cast<const float4 *>(s + W::oW3 + j * 32);
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float4 q = w[k];
            a = fmaf(q.x, x[4 * k], a);
            a = fmaf(q.y, x[4 * k + 1], a);
            a = fmaf(q.z, x[4 * k + 2], a);
            a = fmaf(q.w, x[4 * k + 3], a);
        }
        h1[j] = fmaxf(a, 0.0f);
    }
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;
#pragma unroll 2
    for (int j = 0; j < 64; ++j) {
        const float4 *w = reinterpret_cast<const float4 *>(s + W::oW4 + j * 64);
        float a = 0.0f;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            float4 q = w[k];
            a = fmaf(q.x, h1[4 * k], a);
            a = fmaf(q.y, h1[4 * k + 1], a);
            a = fmaf(q.z, h1[4 * k + 2], a);
            a = fmaf(q.w, h1[4 * k + 3], a);
        }
        a = fmaxf(a, 0.0f);
        float4 w5 = reinterpret_cast<const float4 *>(s + W::oW5T)[j];
        z0 = fmaf(w5.x, a, z0);
        z1 = fmaf(w5.y, a, z1);
        z2 = fmaf(w5.z, a, z2);
    }
    rgb[0] = 1.0f / (1.0f + expf(-z0));
    rgb[1] = 1.0f / (1.0f + expf(-z1));
    rgb[2] = 1.0f / (1.0f + expf(-z2));
}

}  // namespace vrn
