// train.cu -- the training step (Sec. 6; Sec. 4.1 and supplement "Loss
// Design"): L1 loss in PQ space, its gradient through compositing, the
// colour and density MLPs and the hash grid, and Adam.
//
// 1. forward: the fp32 renderer on the batch's rays gives each ray's
//    composited PQ colour C and the number n of composited samples;
// 2. loss: mean |C - PQ(target / 100)|, dL/dC = sign(C - target) / (3B);
// 3. backward: every ray is marched again and its samples recomputed in order
//    (nothing per sample is stored between the passes). With w_i = T_i a_i
//    and the suffix S_i = C - sum_{j<=i} w_j c_j:
//        dL/dc_i = w_i dL/dC,   dL/dsigma_i = delta_i (T_{i+1} c_i - S_i) . dL/dC,
//    then the colour and density MLPs are back-propagated per sample on the
//    CUDA cores; each warp stages its 32 samples' layer inputs and deltas in
//    shared memory and accumulates the weight gradients as 32-sample
//    mini-GEMMs into a per-CTA accumulator; feature gradients are scattered
//    into the hash grid with float2 atomics (weight w_l x trilinear weight).
// 4. Adam (beta = 0.9, 0.99, eps = 1e-15): fp32 master parameters, first and
//    second moments; an fp16 grid is rewritten from its master copy.
#include <cmath>
#include <cstring>

#include "field.h"

namespace vrn {

constexpr int kBwdThreads = 128;
constexpr int kStride = 68;  // padded row stride (floats) of the per-warp staging rows

template <int D>
struct GradSm {  // weight-gradient accumulator in shared memory, padded rows
    static constexpr int s1 = D + 1, g1 = 0;
    static constexpr int s2 = 65, g2 = g1 + 64 * s1;
    static constexpr int s3 = 33, g3 = g2 + 16 * s2;
    static constexpr int s4 = 65, g4 = g3 + 64 * s3;
    static constexpr int s5 = 65, g5 = g4 + 64 * s4;
    static constexpr int size = ((g5 + 3 * s5) + 3) & ~3;
};

__device__ __forceinline__ float dot_row(const float *__restrict__ w, const float *x, int K) {
    float a = 0.0f;
    for (int k = 0; k < K; k += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(w + k));
        a = fmaf(q.x, x[k], a);
        a = fmaf(q.y, x[k + 1], a);
        a = fmaf(q.z, x[k + 2], a);
        a = fmaf(q.w, x[k + 3], a);
    }
    return a;
}

// dW[n][k] += sum over the warp's 32 samples of sD[s][n] * sA[s][k]; this
// lane owns rows n = lane and lane + 32 (those below N).
template <int N, int K>
__device__ __forceinline__ void minigemm_rows(const float *sD, const float *sA, float *sG, int stride_g,
                                              int lane) {
#pragma unroll 1
    for (int rr = 0; rr < 2; ++rr) {
        const int n = lane + 32 * rr;
        if (n >= N) break;
        float acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0f;
#pragma unroll 4
        for (int s = 0; s < 32; ++s) {
            const float d = sD[s * kStride + n];
            const float4 *a = reinterpret_cast<const float4 *>(sA + s * kStride);
#pragma unroll
            for (int k4 = 0; k4 < K / 4; ++k4) {
                const float4 v = a[k4];
                acc[4 * k4] = fmaf(d, v.x, acc[4 * k4]);
                acc[4 * k4 + 1] = fmaf(d, v.y, acc[4 * k4 + 1]);
                acc[4 * k4 + 2] = fmaf(d, v.z, acc[4 * k4 + 2]);
                acc[4 * k4 + 3] = fmaf(d, v.w, acc[4 * k4 + 3]);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) atomicAdd(sG + n * stride_g + k, acc[k]);
    }
}

// Same, for few rows: this lane owns columns k = lane and lane + 32 of all N rows.
template <int N, int K>
__device__ __forceinline__ void minigemm_cols(const float *sD, const float *sA, float *sG, int stride_g,
                                              int lane) {
    float acc[N][2];
#pragma unroll
    for (int n = 0; n < N; ++n) acc[n][0] = acc[n][1] = 0.0f;
#pragma unroll 4
    for (int s = 0; s < 32; ++s) {
        const float a0 = sA[s * kStride + lane], a1 = K > 32 ? sA[s * kStride + lane + 32] : 0.0f;
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const float d = sD[s * kStride + n];
            acc[n][0] = fmaf(d, a0, acc[n][0]);
            acc[n][1] = fmaf(d, a1, acc[n][1]);
        }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) {
        atomicAdd(sG + n * stride_g + lane, acc[n][0]);
        if (K > 32) atomicAdd(sG + n * stride_g + lane + 32, acc[n][1]);
    }
}

template <int L>
__global__ void __launch_bounds__(kBwdThreads)
backward_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                const float *__restrict__ r_in, int B, const float *__restrict__ C_fin,
                const int *__restrict__ n_fin, const float *__restrict__ gC_in,
                float *__restrict__ grid_grad, float *__restrict__ mlp_grad,
                unsigned long long *__restrict__ counter) {
    constexpr int D = 2 * L;
    using G = GradSm<D>;
    extern __shared__ float4 smem4[];
    float *sG = reinterpret_cast<float *>(smem4);
    float *sT = sG + G::size;
    float *stage = sT + ((f.S + 1 + 3) & ~3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sA = stage + warp * 2 * 32 * kStride;
    float *sD = sA + 32 * kStride;
    for (int i = threadIdx.x; i < G::size; i += blockDim.x) sG[i] = 0.0f;
    for (int i = threadIdx.x; i <= f.S; i += blockDim.x) sT[i] = f.t_tab[i];
    __syncthreads();

    const float *W1 = f.mlp, *W2 = W1 + 64 * D, *W3 = W2 + 16 * 64, *W4 = W3 + 64 * 32, *W5 = W4 + 64 * 64;
    constexpr unsigned FULL = 0xffffffffu;
    long long ray = -1;
    bool exhausted = false;
    MarchRay mr;
    float r = 0.0f, T = 1.0f, Cpre[3] = {0, 0, 0}, Cf[3] = {0, 0, 0}, g[3] = {0, 0, 0};
    int k_done = 0, n_tot = 0;
    unsigned tested = 0;

    while (true) {
        bool have = false;
        float p[3] = {0, 0, 0};
        while (true) {
            const bool need = ray < 0 && !exhausted;
            const unsigned m = __ballot_sync(FULL, need);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
                if (need) {
                    const long long b = (long long)base + __popc(m & ((1u << lane) - 1u));
                    if (b >= B) {
                        exhausted = true;
                    } else if (n_fin[b] > 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            mr.o[c] = o_in[3 * b + c];
                            mr.d[c] = d_in[3 * b + c];
                            Cf[c] = C_fin[3 * b + c];
                            g[c] = gC_in[3 * b + c];
                            Cpre[c] = 0.0f;
                        }
                        r = r_in[b];
                        march_init(f, mr);
                        T = 1.0f;
                        k_done = 0;
                        n_tot = n_fin[b];
                        ray = b;
                    }
                }
            }
            if (ray >= 0 && !have) {
                const int mres = march_next(f, sT, mr, p, 8, tested);
                if (mres == MARCH_SAMPLE) have = true;
                else if (mres == MARCH_END) ray = -1;  // cannot happen before n_tot samples
            }
            if (__all_sync(FULL, have || exhausted)) break;
        }
        if (!__any_sync(FULL, have)) break;

        // ---- recompute the sample: features and forward MLPs ----
        float feat[D], dir[3] = {0.0f, 0.0f, 1.0f};
        float t = 0.0f, delta = 0.0f, rn = 0.0f;
        if (have) {
            t = sT[mr.step];
            delta = sT[mr.step + 1] - t;
            rn = footprint(f, t, r, p, nullptr, nullptr);  // explicit rays
            gather_features<L>(f, p, rn, feat);
            dir[0] = mr.d[0];
            dir[1] = mr.d[1];
            dir[2] = mr.d[2];
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) feat[k] = 0.0f;
        }
        float o[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) o[i] = 0.0f;
#pragma unroll 2
        for (int j = 0; j < 64; ++j) {
            const float h = fmaxf(dot_row(W1 + j * D, feat, D), 0.0f);
#pragma unroll
            for (int i = 0; i < 16; ++i) o[i] = fmaf(__ldg(W2 + i * 64 + j), h, o[i]);
        }
        const float sigma = expf(o[0] + f.density_bias);
        float h1[64];
        {
            float x[32];
#pragma unroll
            for (int i = 0; i < 16; ++i) x[i] = o[i];
            sh16(dir[0], dir[1], dir[2], x + 16);
#pragma unroll
            for (int j = 0; j < 64; ++j) h1[j] = fmaxf(dot_row(W3 + j * 32, x, 32), 0.0f);
        }
        float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;
#pragma unroll 2
        for (int j = 0; j < 64; ++j) {
            const float h2 = fmaxf(dot_row(W4 + j * 64, h1, 64), 0.0f);
            sA[lane * kStride + j] = h2;
            z0 = fmaf(__ldg(W5 + j), h2, z0);
            z1 = fmaf(__ldg(W5 + 64 + j), h2, z1);
            z2 = fmaf(__ldg(W5 + 128 + j), h2, z2);
        }
        const float c0 = 1.0f / (1.0f + expf(-z0)), c1 = 1.0f / (1.0f + expf(-z1)),
                    c2 = 1.0f / (1.0f + expf(-z2));

        // ---- compositing gradient ----
        const float sd = sigma * delta;
        const float alpha = -expm1f(-sd), Tn = T * expf(-sd), w = T * alpha;
        float dz[3] = {0, 0, 0}, dsig = 0.0f;
        if (have) {
            const float cc[3] = {c0, c1, c2};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float suffix = Cf[c] - (Cpre[c] + w * cc[c]);
                dsig += g[c] * delta * (Tn * cc[c] - suffix);
                dz[c] = w * g[c] * cc[c] * (1.0f - cc[c]);
            }
        }
        // ---- W5: dz x h2 ----
        sD[lane * kStride + 0] = dz[0];
        sD[lane * kStride + 1] = dz[1];
        sD[lane * kStride + 2] = dz[2];
        __syncwarp();
        minigemm_cols<3, 64>(sD, sA, sG + G::g5, G::s5, lane);
        // dh2 = mask(h2) W5^T dz, staged straight into sD (own row)
        __syncwarp();
        {
            float dh2v[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                const float h2 = sA[lane * kStride + j];
                const float a = __ldg(W5 + j) * dz[0] + __ldg(W5 + 64 + j) * dz[1] + __ldg(W5 + 128 + j) * dz[2];
                dh2v[j] = h2 > 0.0f ? a : 0.0f;
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 64; ++j) {
                sD[lane * kStride + j] = dh2v[j];
                sA[lane * kStride + j] = h1[j];
            }
        }
        __syncwarp();
        // ---- W4: dh2 x h1 ----
        minigemm_rows<64, 64>(sD, sA, sG + G::g4, G::s4, lane);
        float dh1[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) dh1[k] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            const float d = sD[lane * kStride + j];
            const float4 *wr = reinterpret_cast<const float4 *>(W4 + j * 64);
#pragma unroll
            for (int k4 = 0; k4 < 16; ++k4) {
                const float4 q = __ldg(wr + k4);
                dh1[4 * k4] = fmaf(q.x, d, dh1[4 * k4]);
                dh1[4 * k4 + 1] = fmaf(q.y, d, dh1[4 * k4 + 1]);
                dh1[4 * k4 + 2] = fmaf(q.z, d, dh1[4 * k4 + 2]);
                dh1[4 * k4 + 3] = fmaf(q.w, d, dh1[4 * k4 + 3]);
            }
        }
#pragma unroll
        for (int k = 0; k < 64; ++k) dh1[k] = sA[lane * kStride + k] > 0.0f ? dh1[k] : 0.0f;
        __syncwarp();
        // ---- W3: dh1 x x, x = [o, SH(d)] rebuilt ----
#pragma unroll
        for (int j = 0; j < 64; ++j) sD[lane * kStride + j] = dh1[j];
        {
            float shv[16];
            sh16(dir[0], dir[1], dir[2], shv);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                sA[lane * kStride + k] = o[k];
                sA[lane * kStride + 16 + k] = shv[k];
            }
        }
        __syncwarp();
        minigemm_rows<64, 32>(sD, sA, sG + G::g3, G::s3, lane);
        float dout[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) dout[i] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            const float d = sD[lane * kStride + j];
#pragma unroll
            for (int i = 0; i < 16; ++i) dout[i] = fmaf(__ldg(W3 + j * 32 + i), d, dout[i]);
        }
        dout[0] += dsig * sigma;
        __syncwarp();
        // ---- W2: dout x h (h recomputed) ----
        float h[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) h[j] = fmaxf(dot_row(W1 + j * D, feat, D), 0.0f);
#pragma unroll
        for (int i = 0; i < 16; ++i) sD[lane * kStride + i] = dout[i];
#pragma unroll
        for (int j = 0; j < 64; ++j) sA[lane * kStride + j] = h[j];
        __syncwarp();
        minigemm_cols<16, 64>(sD, sA, sG + G::g2, G::s2, lane);
        float dh[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            float a = 0.0f;
#pragma unroll
            for (int i = 0; i < 16; ++i) a = fmaf(__ldg(W2 + i * 64 + j), dout[i], a);
            dh[j] = h[j] > 0.0f ? a : 0.0f;
        }
        __syncwarp();
        // ---- W1: dh x feat ----
#pragma unroll
        for (int j = 0; j < 64; ++j) sD[lane * kStride + j] = dh[j];
#pragma unroll
        for (int k = 0; k < D; ++k) sA[lane * kStride + k] = feat[k];
        __syncwarp();
        minigemm_rows<64, D>(sD, sA, sG + G::g1, G::s1, lane);
        float dfeat[D];
#pragma unroll
        for (int k = 0; k < D; ++k) dfeat[k] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            const float d = dh[j];
#pragma unroll
            for (int k = 0; k < D; ++k) dfeat[k] = fmaf(__ldg(W1 + j * D + k), d, dfeat[k]);
        }
        __syncwarp();

        // ---- hash-grid scatter and compositing state ----
        if (have) {
            const float Ls = lod_star(f, rn);
            for (int l = 0; l < L; ++l) {
                const float wl = lod_weight(Ls, l);
                if (wl <= 0.0f) break;
                uint32_t idx[8];
                float fr[3];
                level_corners(f, l, p, idx, fr);
                float2 *base = reinterpret_cast<float2 *>(grid_grad) + (size_t)l * (f.T_mask + 1u);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const float cw = (b & 1 ? fr[0] : 1.0f - fr[0]) * (b & 2 ? fr[1] : 1.0f - fr[1]) *
                                     (b & 4 ? fr[2] : 1.0f - fr[2]) * wl;
                    atomicAdd(base + idx[b], make_float2(cw * dfeat[2 * l], cw * dfeat[2 * l + 1]));
                }
            }
            Cpre[0] += w * c0;
            Cpre[1] += w * c1;
            Cpre[2] += w * c2;
            T = Tn;
            ++mr.step;
            if (++k_done >= n_tot) ray = -1;
        }
    }
    __syncthreads();
    // per-CTA weight gradients -> global, in the [out][in] layout
    for (int e = threadIdx.x; e < 64 * D + 16 * 64 + 64 * 32 + 64 * 64 + 3 * 64; e += blockDim.x) {
        int q = e, v;
        if (q < 64 * D) v = G::g1 + (q / D) * G::s1 + q % D;
        else if ((q -= 64 * D) < 16 * 64) v = G::g2 + (q / 64) * G::s2 + q % 64;
        else if ((q -= 16 * 64) < 64 * 32) v = G::g3 + (q / 32) * G::s3 + q % 32;
        else if ((q -= 64 * 32) < 64 * 64) v = G::g4 + (q / 64) * G::s4 + q % 64;
        else v = G::g5 + ((q -= 64 * 64) / 64) * G::s5 + q % 64;
        const float val = sG[v];
        if (val != 0.0f) atomicAdd(mlp_grad + e, val);
    }
}

// loss = sum |C - PQ(target / 100)| (divided by 3B on the host); dL/dC.
__global__ void loss_kernel(const float *__restrict__ C, const float *__restrict__ target, int n3, float inv,
                            float *__restrict__ gC, float *__restrict__ loss_sum) {
    float s = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) {
        const float diff = C[i] - linear_to_pq(target[i]);
        gC[i] = diff > 0.0f ? inv : (diff < 0.0f ? -inv : 0.0f);
        s += fabsf(diff);
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, s);
}

__global__ void adam_kernel(float *__restrict__ p32, __half *__restrict__ p16, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, long long n, float lr, float b1,
                            float b2, float eps, float inv_bc1, float inv_bc2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p32[i] - lr * (mi * inv_bc1) / (sqrtf(vi * inv_bc2) + eps);
        p32[i] = pi;
        if (p16) p16[i] = __float2half_rn(pi);
    }
}

__global__ void half_to_float_kernel(const __half *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = __half2float(a[i]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct TrainScratch {
    float *C = nullptr, *gC = nullptr;
    int *n = nullptr;
    int cap = 0;
};
static int ensure_train(vrnerf_field *F, int B) {
    cudaError_t e = cudaSuccess;
    const uint64_t ng = grid_entries(F->desc);
    const size_t nm = (size_t)F->view.n_mlp;
    if (!F->grid_grad && (e = cudaMalloc(&F->grid_grad, ng * sizeof(float))) != cudaSuccess)
        return fail(VRNERF_ENOMEM, "grid gradient: %s", cudaGetErrorString(e));
    if (!F->mlp_grad && (e = cudaMalloc(&F->mlp_grad, nm * sizeof(float))) != cudaSuccess)
        return fail(VRNERF_ENOMEM, "mlp gradient: %s", cudaGetErrorString(e));
    if (!F->loss_acc && (e = cudaMalloc(&F->loss_acc, 64)) != cudaSuccess)
        return fail(VRNERF_ENOMEM, "loss: %s", cudaGetErrorString(e));
    if (!F->train_scratch) F->train_scratch = new TrainScratch();
    TrainScratch &S = *static_cast<TrainScratch *>(F->train_scratch);
    if (B > S.cap) {
        if (S.C) cudaFree(S.C);
        if (S.gC) cudaFree(S.gC);
        if (S.n) cudaFree(S.n);
        S.C = S.gC = nullptr;
        S.n = nullptr;
        S.cap = 0;
        if ((e = cudaMalloc(&S.C, sizeof(float) * 3 * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.gC, sizeof(float) * 3 * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.n, sizeof(int) * (size_t)B)) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "training scratch: %s", cudaGetErrorString(e));
        S.cap = B;
    }
    return VRNERF_OK;
}

void release_train_scratch(vrnerf_field *F) {
    if (!F->train_scratch) return;
    TrainScratch *S = static_cast<TrainScratch *>(F->train_scratch);
    if (S->C) cudaFree(S->C);
    if (S->gC) cudaFree(S->gC);
    if (S->n) cudaFree(S->n);
    delete S;
    F->train_scratch = nullptr;
}

template <int L>
static cudaError_t launch_backward_t(vrnerf_field *F, const float *o, const float *d, const float *r, int B,
                                     const float *C_fin, const int *n_fin, const float *gC, cudaStream_t st) {
    constexpr int D = 2 * L;
    const size_t smem = sizeof(float) * ((size_t)GradSm<D>::size + ((F->view.S + 1 + 3) & ~3) +
                                         (size_t)(kBwdThreads / 32) * 2 * 32 * kStride);
    auto kern = backward_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kBwdThreads, smem)) != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long grid = (long long)num_sms() * bps, want = (B + kBwdThreads - 1) / kBwdThreads;
    if (want < grid) grid = want;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(F->counter);
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
    kern<<<(unsigned)grid, kBwdThreads, smem, st>>>(F->view, o, d, r, B, C_fin, n_fin, gC, F->grid_grad, F->mlp_grad,
                                                   cnt);
    return cudaGetLastError();
}

}  // namespace vrn

using namespace vrn;

extern "C" {

int vrnerf_backward(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii,
                    const float *target_linear, int32_t B, float *loss_host, void *stream) {
    try {
        if (!F || !rays_o || !rays_d || !radii || !target_linear) return fail(VRNERF_EINVAL, "NULL argument");
        if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
        int rc = ensure_train(F, B);
        if (rc) return rc;
        TrainScratch &S = *static_cast<TrainScratch *>(F->train_scratch);
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaMemsetAsync(F->grid_grad, 0, grid_entries(F->desc) * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(F->mlp_grad, 0, sizeof(float) * F->view.n_mlp, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(F->loss_acc, 0, 64, st);
        // forward: composited PQ colour and sample count of every ray
        RaySource src;
        memset(&src, 0, sizeof src);
        src.o = rays_o;
        src.d = rays_d;
        src.r = radii;
        src.n_slots = B;
        // (the linear colour is not needed: it lands in gC, which the loss kernel fills next)
        RenderOut ro{S.gC, S.C, nullptr, S.n, nullptr, nullptr, F->hist};
        if (e == cudaSuccess) e = cudaMemsetAsync(F->counter, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess)
            e = launch_render_simt(F->view, src, ro, reinterpret_cast<unsigned long long *>(F->counter), st);
        if (e == cudaSuccess) {
            loss_kernel<<<num_sms() * 4, 256, 0, st>>>(S.C, target_linear, 3 * B, 1.0f / (3.0f * B), S.gC,
                                                        F->loss_acc);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = F->view.L == 8 ? launch_backward_t<8>(F, rays_o, rays_d, radii, B, S.C, S.n, S.gC, st)
                               : launch_backward_t<16>(F, rays_o, rays_d, radii, B, S.C, S.n, S.gC, st);
        if (e != cudaSuccess) return cuda_fail(e, "backward");
        if (loss_host) {
            float sum = 0.0f;
            e = cudaMemcpyAsync(&sum, F->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "backward: loss");
            *loss_host = sum / (3.0f * B);
        }
        return VRNERF_OK;
    } catch (...) {
        return fail(VRNERF_EINVAL, "backward: unexpected C++ exception");
    }
}

int vrnerf_backward_from_grad(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii,
                              int32_t B, const float *pq_fwd, const int32_t *n_fwd, const float *grad_pq,
                              void *stream) {
    try {
        if (!F || !rays_o || !rays_d || !radii || !pq_fwd || !n_fwd || !grad_pq)
            return fail(VRNERF_EINVAL, "NULL argument");
        if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
        int rc = ensure_train(F, 1);
        if (rc) return rc;
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaMemsetAsync(F->grid_grad, 0, grid_entries(F->desc) * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(F->mlp_grad, 0, sizeof(float) * F->view.n_mlp, st);
        if (e == cudaSuccess)
            e = F->view.L == 8 ? launch_backward_t<8>(F, rays_o, rays_d, radii, B, pq_fwd, n_fwd, grad_pq, st)
                               : launch_backward_t<16>(F, rays_o, rays_d, radii, B, pq_fwd, n_fwd, grad_pq, st);
        if (e != cudaSuccess) return cuda_fail(e, "backward_from_grad");
        return VRNERF_OK;
    } catch (...) {
        return fail(VRNERF_EINVAL, "backward_from_grad: unexpected C++ exception");
    }
}

int vrnerf_field_param_ptrs(vrnerf_field *F, void **grid, float **mlp, float **grid_grad, float **mlp_grad) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (grid_grad || mlp_grad) {
        int rc = ensure_train(F, 1);
        if (rc) return rc;
    }
    if (grid) *grid = F->grid;
    if (mlp) *mlp = F->mlp;
    if (grid_grad) *grid_grad = F->grid_grad;
    if (mlp_grad) *mlp_grad = F->mlp_grad;
    return VRNERF_OK;
}

int vrnerf_field_params_changed(vrnerf_field *F) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && F->grid_master && F->desc.feat_fp16) {
        const long long ng = (long long)grid_entries(F->desc);
        half_to_float_kernel<<<num_sms() * 8, 256>>>(static_cast<const __half *>(F->grid), F->grid_master, ng);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) return cuda_fail(e, "params_changed");
    ++F->mlp_version;
    return VRNERF_OK;
}

int vrnerf_field_get_grads(vrnerf_field *F, float *grid_grad_host, float *mlp_grad_host) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (!F->grid_grad || !F->mlp_grad) return fail(VRNERF_EINVAL, "no gradients yet: call vrnerf_backward");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess && grid_grad_host)
        e = cudaMemcpy(grid_grad_host, F->grid_grad, grid_entries(F->desc) * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mlp_grad_host)
        e = cudaMemcpy(mlp_grad_host, F->mlp_grad, sizeof(float) * F->view.n_mlp, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "get_grads");
    return VRNERF_OK;
}

int vrnerf_field_set_grads(vrnerf_field *F, const float *grid_grad_host, const float *mlp_grad_host) {
    if (!F || !grid_grad_host || !mlp_grad_host) return fail(VRNERF_EINVAL, "NULL argument");
    int rc = ensure_train(F, 1);
    if (rc) return rc;
    cudaError_t e =
        cudaMemcpy(F->grid_grad, grid_grad_host, grid_entries(F->desc) * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(F->mlp_grad, mlp_grad_host, sizeof(float) * F->view.n_mlp, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "set_grads");
    return VRNERF_OK;
}

int vrnerf_adam_step(vrnerf_field *F, float lr_grid, float lr_mlp, void *stream) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (!F->grid_grad || !F->mlp_grad) return fail(VRNERF_EINVAL, "no gradients yet: call vrnerf_backward");
    if (!(lr_grid >= 0.0f) || !(lr_mlp >= 0.0f)) return fail(VRNERF_EINVAL, "learning rates must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    const long long ng = (long long)grid_entries(F->desc);
    const long long nm = F->view.n_mlp;
    cudaError_t e = cudaSuccess;
    if (!F->m_grid) {
        if ((e = cudaMalloc(&F->m_grid, ng * 4)) != cudaSuccess || (e = cudaMalloc(&F->v_grid, ng * 4)) != cudaSuccess ||
            (e = cudaMalloc(&F->m_mlp, nm * 4)) != cudaSuccess || (e = cudaMalloc(&F->v_mlp, nm * 4)) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "Adam moments: %s", cudaGetErrorString(e));
        cudaMemsetAsync(F->m_grid, 0, ng * 4, st);
        cudaMemsetAsync(F->v_grid, 0, ng * 4, st);
        cudaMemsetAsync(F->m_mlp, 0, nm * 4, st);
        cudaMemsetAsync(F->v_mlp, 0, nm * 4, st);
        if (F->desc.feat_fp16) {
            if ((e = cudaMalloc(&F->grid_master, ng * 4)) != cudaSuccess)
                return fail(VRNERF_ENOMEM, "fp32 master grid: %s", cudaGetErrorString(e));
            half_to_float_kernel<<<num_sms() * 8, 256, 0, st>>>(static_cast<const __half *>(F->grid), F->grid_master, ng);
        }
    }
    ++F->adam_t;
    const double b1 = 0.9, b2 = 0.99, eps = 1e-15;
    const float inv_bc1 = (float)(1.0 / (1.0 - pow(b1, F->adam_t)));
    const float inv_bc2 = (float)(1.0 / (1.0 - pow(b2, F->adam_t)));
    float *g32 = F->desc.feat_fp16 ? F->grid_master : static_cast<float *>(F->grid);
    __half *g16 = F->desc.feat_fp16 ? static_cast<__half *>(F->grid) : nullptr;
    adam_kernel<<<num_sms() * 8, 256, 0, st>>>(g32, g16, F->grid_grad, F->m_grid, F->v_grid, ng, lr_grid, (float)b1,
                                               (float)b2, (float)eps, inv_bc1, inv_bc2);
    adam_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(F->mlp, nullptr, F->mlp_grad, F->m_mlp, F->v_mlp, nm,
                                                               lr_mlp, (float)b1, (float)b2, (float)eps, inv_bc1,
                                                               inv_bc2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "adam");
    ++F->mlp_version;  // tensor-core weight images are rebuilt on next use
    return VRNERF_OK;
}

int vrnerf_train_step(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii,
                      const float *target_linear, int32_t B, float lr_grid, float lr_mlp, float *loss_host,
                      void *stream) {
    int rc = vrnerf_backward(F, rays_o, rays_d, radii, target_linear, B, loss_host, stream);
    if (rc) return rc;
    return vrnerf_adam_step(F, lr_grid, lr_mlp, stream);
}

}  // extern "C"
