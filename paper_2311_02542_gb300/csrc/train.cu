// train.cu -- the training step (Sec. 6; Sec. 4.1 and supplement "Loss
// Design"): L1 loss in PQ space, its gradient through compositing, the
// colour and density MLPs and the hash grid, and Adam.
//
// The batch is processed sample-parallel, so that small batches (the paper's
// 12 800 rays) still fill the GPU:
// 1. count / emit: every ray is marched (occupancy rule of Sec. 4.3, no
//    early termination) and its evaluated samples are listed contiguously
//    as (ray, step) records, in ray order (offsets by a prefix sum);
// 2. sample forward: one thread per sample gathers the LOD-weighted features
//    and runs the fp32 MLPs: sigma and PQ colour per sample;
// 3. ray composite: each lane composites one ray at a time (and takes the
//    next ray when it is done) front to back
//    (stopping where transmittance drops below T_eps, or after the number of
//    samples a forward pass reported), forms dL/dC (L1: sign(C - target) /
//    3B, or a given upstream gradient) and walks its samples backwards: with
//    w_i = T_i a_i and the suffix S_i = C - sum_{j<=i} w_j c_j,
//        dL/dc_i = w_i dL/dC,   dL/dsigma_i = delta_i (T_{i+1} c_i - S_i) . dL/dC;
// 4. sample backward: one thread per sample recomputes its features and
//    activations (nothing but sigma, colour and these two gradients is kept
//    per sample) and back-propagates the MLPs; each warp stages its 32
//    samples' layer inputs and deltas in shared memory and accumulates the
//    weight gradients as 32-sample mini-GEMMs into a per-CTA accumulator;
//    feature gradients are scattered into the hash grid with float2 atomics
//    (weight w_l x trilinear weight).
// 5. Adam (beta = 0.9, 0.99, eps = 1e-15): fp32 master parameters, first and
//    second moments; an fp16 grid is rewritten from its master copy.
#include <cmath>
#include <cstring>

#include "field.h"
#include "simt_mlp.cuh"

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

// ---- 1. count / emit ----------------------------------------------------
// Rays differ widely in length (a few evaluated samples for most, hundreds
// for some), and with one ray per thread a warp runs as long as its longest
// ray while its other lanes idle. The per-ray kernels below (count, and the
// ray composite of step 3) keep every lane busy instead: a lane whose ray is
// done takes the next ray index from its warp's batch of 32, and the warp
// takes a new batch from a global counter (one atomic per batch) when the
// batch runs out. Which lane handles which ray does not change any result.
struct RayQueue {
    long long base;  // next ray index of the warp's batch
    int left;        // rays of the batch not handed out yet
    bool empty;      // every ray has been handed out
};

// Called by all 32 lanes of the warp together; each lane with want == true
// receives a ray index, or -1 once all B rays have been handed out.
__device__ __forceinline__ long long take_ray(RayQueue &q, bool want, unsigned long long *__restrict__ next,
                                              long long B) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    long long mine = -1;
    unsigned need = __ballot_sync(FULL, want);
    while (need && !q.empty) {
        if (q.left == 0) {
            unsigned long long g = 0;
            if (lane == 0) g = atomicAdd(next, 32ull);
            g = __shfl_sync(FULL, g, 0);
            if ((long long)g >= B) {
                q.empty = true;
                break;
            }
            q.base = (long long)g;
            q.left = (int)(B - q.base < 32 ? B - q.base : 32);
        }
        const int take = min(__popc(need), q.left);
        const int rank = __popc(need & ((1u << lane) - 1u));
        if (((need >> lane) & 1u) && rank < take) mine = q.base + rank;
        q.base += take;
        q.left -= take;
        need = __ballot_sync(FULL, want && mine < 0);
    }
    return mine;
}

#ifndef VRN_COUNT_CHUNK
#define VRN_COUNT_CHUNK 8
#endif
constexpr int kCountChunk = VRN_COUNT_CHUNK;  // march iterations of a lane between two refills

// A ray past this many evaluated samples goes to a warp of its own: a few
// rays hold hundreds of samples (a hundred times the median), and one lane
// walking them alone sets the time of the whole kernel at small batches.
constexpr int kLongRay = 32;
#ifndef VRN_LONG_COUNT
#define VRN_LONG_COUNT 32
#endif
constexpr int kLongCount = VRN_LONG_COUNT;  // samples after which count_kernel hands a ray on

// Evaluated samples of every ray (no early termination) -> cnt; with `mask`
// (mw words per ray, zeroed beforehand) the ray's evaluated step indices are
// also kept as bits, so that emit needs no second march. The records'
// offsets come from the scan kernels below. `next` and *n_long start at 0.
// A ray that reaches kLongCount samples stops here: its count so far goes
// to cnt and (ray, next step) to long_rays, for count_long_kernel.
__global__ void __launch_bounds__(128)
count_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in, int B,
             int *__restrict__ cnt, uint32_t *__restrict__ mask, int mw, unsigned long long *__restrict__ next,
             int2 *__restrict__ long_rays, unsigned int *__restrict__ n_long) {
    RayQueue q{0, 0, false};
    bool live = false, retired = false;
    long long b = -1;
    MarchRay m;
    int n = 0, wi = -1;
    uint32_t word = 0u, *mrow = nullptr;
    unsigned tested = 0;
    while (true) {
        const long long got = take_ray(q, !live && !retired, next, B);
        if (!live && !retired) {
            if (got < 0) {
                retired = true;
            } else {
                b = got;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    m.o[k] = o_in[3 * b + k];
                    m.d[k] = d_in[3 * b + k];
                }
                march_init(f, m);
                n = 0;
                wi = -1;
                word = 0u;
                mrow = mask ? mask + (size_t)b * mw : nullptr;
                live = true;
            }
        }
        if (__all_sync(0xffffffffu, retired)) break;
        if (!live) continue;
        float p[3];
        const int r = march_next(f, f.t_tab, m, p, kCountChunk, tested);
        if (r == MARCH_SAMPLE) {
            ++n;
            if (mrow) {
                const int w = m.step >> 5;
                if (w != wi) {
                    if (wi >= 0) mrow[wi] = word;
                    wi = w;
                    word = 0u;
                }
                word |= 1u << (m.step & 31);
            }
            ++m.step;
            if (n >= kLongCount && m.step < f.S) {  // the rest of the ray to a warp of its own
                if (mrow) mrow[wi] = word;
                cnt[b] = n;
                long_rays[atomicAdd(n_long, 1u)] = make_int2((int)b, m.step);
                live = false;
            }
        } else if (r == MARCH_END) {
            if (mrow && wi >= 0) mrow[wi] = word;
            cnt[b] = n;
            live = false;
        }
    }
}

// The rest of each long ray, from the step where count_kernel left it: the
// warp's 32 lanes march consecutive segments of the remaining steps. The
// march finds every step whose sample lies in an occupied voxel (the skip
// never passes one, and a bounded ray that has left the grid does not come
// back), so the segments together give the same steps as one march, and
// their counts add up. Mask words that two segments (or count_kernel) share
// are merged with atomicOr.
__global__ void __launch_bounds__(128)
count_long_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                  int *__restrict__ cnt, uint32_t *__restrict__ mask, int mw,
                  const int2 *__restrict__ long_rays, const unsigned int *__restrict__ n_long) {
    const int lane = threadIdx.x & 31;
    const unsigned total = *n_long;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    for (unsigned e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += warps) {
        const int2 lr = long_rays[e];
        const long long b = lr.x;
        const int len = (f.S - lr.y + 31) / 32;
        const int s0 = lr.y + lane * len, s1 = min(f.S, s0 + len);
        int n = 0;
        if (s0 < s1) {
            MarchRay m;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                m.o[k] = o_in[3 * b + k];
                m.d[k] = d_in[3 * b + k];
            }
            march_init(f, m);
            m.step = s0;
            uint32_t *mrow = mask ? mask + (size_t)b * mw : nullptr;
            uint32_t word = 0u;
            int wi = -1;
            unsigned tested = 0;
            float p[3];
            while (true) {
                const int r = march_next(f, f.t_tab, m, p, kCountChunk, tested);
                if (r == MARCH_END || m.step >= s1) break;
                if (r == MARCH_SAMPLE) {
                    ++n;
                    if (mrow) {
                        const int w = m.step >> 5;
                        if (w != wi) {
                            if (wi >= 0) atomicOr(mrow + wi, word);
                            wi = w;
                            word = 0u;
                        }
                        word |= 1u << (m.step & 31);
                    }
                    ++m.step;
                }
            }
            if (mrow && wi >= 0) atomicOr(mrow + wi, word);
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) n += __shfl_xor_sync(0xffffffffu, n, s);
        if (lane == 0) cnt[b] += n;
    }
}

// Exclusive prefix sums of cnt[0..B) -> off, and their total, in three
// launches: per-block sums of kScanPer counts, a scan of those sums by one
// block, then each block's own scan plus its block's offset.
constexpr int kScanThreads = 1024, kScanItems = 4, kScanPer = kScanThreads * kScanItems;

// inclusive scan over the block's threads (all threads call it); *total = the block's sum
__device__ __forceinline__ long long block_scan(long long v, long long *warp_sums, long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, s);
        if (lane >= s) v += u;
    }
    if (lane == 31) warp_sums[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, w, s);
            if (lane >= s) w += u;
        }
        warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const long long r = v + (warp > 0 ? warp_sums[warp - 1] : 0);
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();  // warp_sums may be reused after this
    return r;
}

// Small batches (up to kScanOneBlock x kScanPer rays): one block walks the
// counts in chunks of kScanPer with a running carry, in one launch.
constexpr int kScanOneBlock = 8;

__global__ void __launch_bounds__(kScanThreads)
scan_one_block_kernel(const int *__restrict__ cnt, int B, long long *__restrict__ off,
                      unsigned long long *__restrict__ total_out) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (long long c = 0; c < B; c += kScanPer) {  // uniform over the block
        const long long base = c + (long long)threadIdx.x * kScanItems;
        int v4[kScanItems];
        long long v = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v4[k] = base + k < B ? cnt[base + k] : 0;
            v += v4[k];
        }
        long long tot;
        long long x = block_scan(v, ws, &tot) - v + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < B) off[base + k] = x;
            x += v4[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_sums_kernel(const int *__restrict__ cnt, int B, long long *__restrict__ bsum) {
    __shared__ long long ws[32];
    const long long base = (long long)blockIdx.x * kScanPer + (long long)threadIdx.x * kScanItems;
    long long v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < B) v += cnt[base + k];
    long long total;
    block_scan(v, ws, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_blocks_kernel(long long *__restrict__ bsum, int nb, unsigned long long *__restrict__ total_out) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (int c = 0; c < nb; c += kScanThreads) {  // uniform over the block
        const int i = c + threadIdx.x;
        const long long v = i < nb ? bsum[i] : 0;
        long long tot;
        const long long incl = block_scan(v, ws, &tot);
        if (i < nb) bsum[i] = carry + incl - v;  // exclusive: offset of block i
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_offsets_kernel(const int *__restrict__ cnt, int B, const long long *__restrict__ boff,
                    long long *__restrict__ off) {
    __shared__ long long ws[32];
    const long long base = (long long)blockIdx.x * kScanPer + (long long)threadIdx.x * kScanItems;
    int c[kScanItems];
    long long v = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        c[k] = base + k < B ? cnt[base + k] : 0;
        v += c[k];
    }
    long long total;
    long long x = block_scan(v, ws, &total) - v + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < B) off[base + k] = x;
        x += c[k];
    }
}

__global__ void __launch_bounds__(128)
emit_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in, int B,
            const long long *__restrict__ off, const int *__restrict__ cnt, int2 *__restrict__ rec,
            const uint32_t *__restrict__ mask, int mw) {
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
        if (mask) {  // the steps count_kernel found, in order, from its bits
            const uint32_t *mrow = mask + (size_t)b * mw;
            long long q = off[b];
            const long long end = q + cnt[b];
            for (int w = 0; w < mw && q < end; ++w) {
                uint32_t x = __ldg(mrow + w);
                while (x) {
                    if (VRN_CHECKED && !vrn_check(f.check, q < end, kCheckRecord)) break;
                    rec[q++] = make_int2((int)b, 32 * w + __ffs(x) - 1);
                    x &= x - 1u;
                }
            }
            continue;
        }
        MarchRay m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            m.o[k] = o_in[3 * b + k];
            m.d[k] = d_in[3 * b + k];
        }
        march_init(f, m);
        unsigned tested = 0;
        float p[3];
        long long q = off[b];
        const long long end = q + cnt[b];
        while (march_next(f, f.t_tab, m, p, 1 << 30, tested) == MARCH_SAMPLE) {
            if (VRN_CHECKED && !vrn_check(f.check, q < end, kCheckRecord)) break;
            rec[q++] = make_int2((int)b, m.step);
            ++m.step;
        }
    }
}

// ---- 2. sample forward ------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(128)
sample_fwd_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                  const float *__restrict__ r_in, const int2 *__restrict__ rec, long long n,
                  float4 *__restrict__ sc, uint4 *__restrict__ feat_out) {
    constexpr int D = 2 * L;
    extern __shared__ float4 smem4[];
    float *sW = reinterpret_cast<float *>(smem4);
    load_weights_simt<D>(f.mlp, sW);
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int2 q = rec[i];
        const long long b = q.x;
        const float o[3] = {o_in[3 * b], o_in[3 * b + 1], o_in[3 * b + 2]};
        const float d[3] = {d_in[3 * b], d_in[3 * b + 1], d_in[3 * b + 2]};
        const float t = f.t_tab[q.y];
        float p[3];
        int vox;
        sample_voxel(f, o, d, t, p, vox);  // the march's fp32 position
        float feat[D], sigma, rgb[3];
        gather_features<L>(f, p, footprint(f, t, r_in[b], p, nullptr, nullptr), feat);
        mlp_simt<D>(sW, feat, d, f.density_bias, sigma, rgb);
        sc[i] = make_float4(sigma, rgb[0], rgb[1], rgb[2]);
        if (feat_out) {  // bf16 features for the tensor-core backward (D / 8 16-byte words)
#pragma unroll
            for (int k = 0; k < D / 8; ++k) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(feat[8 * k + 2 * j], feat[8 * k + 2 * j + 1]);
                    w[j] = *reinterpret_cast<const uint32_t *>(&h);
                }
                feat_out[i * (D / 8) + k] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// ---- 3. ray composite: C, dL/dC, per-sample gradients -----------------------
// n_given (nullable): composite exactly that many samples (a forward pass's
// count); else stop after the sample where T < T_eps. target (nullable): L1
// loss against PQ(target / 100), else gC_given is dL/dC. Overwrites sc with
// (dL/dsigma, dL/dz_0..2) of every composited sample (z: pre-sigmoid colour)
// and zeros for the rest. C_out (nullable): forward only, the composited PQ
// colour and sample count per ray.
// Each lane walks one ray at a time and takes the next ray when it is done
// (take_ray): per iteration a lane handles up to kCompSamples samples of its
// ray, in the composite (phase 0) or the gradient walk (phase 1), or up to 8
// records of the zero tail (phase 2). `next` starts at 0.
#ifndef VRN_COMP_SAMPLES
#define VRN_COMP_SAMPLES 4
#endif
constexpr int kCompSamples = VRN_COMP_SAMPLES;

__global__ void __launch_bounds__(128)
ray_comp_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in, int B,
                const int *__restrict__ cnt, const long long *__restrict__ off, const int2 *__restrict__ rec,
                const int *__restrict__ n_given, const float *__restrict__ target, const float *__restrict__ gC_given,
                float inv_n, float4 *__restrict__ sc, int *__restrict__ n_used, float *__restrict__ loss_sum,
                float *__restrict__ hist, float *__restrict__ C_out, unsigned long long *__restrict__ next,
                int *__restrict__ long_rays, unsigned int *__restrict__ n_long) {
    RayQueue q{0, 0, false};
    float loss = 0.0f;
    bool live = false, retired = false;
    long long b = -1, k0 = 0;
    int m = 0, lim = 0, n = 0, k = 0, phase = 0;
    float T = 1.0f, C[3] = {0, 0, 0}, g[3] = {0, 0, 0}, Cpre[3] = {0, 0, 0}, ro[3] = {0, 0, 0}, rd[3] = {0, 0, 1};
    while (true) {
        const long long got = take_ray(q, !live && !retired, next, B);
        if (!live && !retired) {
            if (got < 0) {
                retired = true;
            } else {
                b = got;
                k0 = off[b];
                m = cnt[b];
                if (m > kLongRay) {  // composited by ray_comp_long_kernel; this lane takes another ray
                    long_rays[atomicAdd(n_long, 1u)] = (int)b;
                } else {
                    lim = n_given ? min(n_given[b], m) : m;
                    n = 0;
                    phase = 0;
                    T = 1.0f;
                    C[0] = C[1] = C[2] = 0.0f;
                    if (hist) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            ro[c] = o_in[3 * b + c];
                            rd[c] = d_in[3 * b + c];
                        }
                    }
                    live = true;
                }
            }
        }
        if (__all_sync(0xffffffffu, retired)) break;
        if (!live) continue;
        if (phase == 0) {  // composite samples n, n + 1, ...
            bool done = n >= lim;
#pragma unroll 1
            for (int e = 0; e < kCompSamples && !done; ++e) {
                const float4 v = sc[k0 + n];
                const int step = rec[k0 + n].y;
                const float t = f.t_tab[step], sd = v.x * (f.t_tab[step + 1] - t);
                const float alpha = -expm1f(-sd), w = T * alpha;
                C[0] += w * v.y;
                C[1] += w * v.z;
                C[2] += w * v.w;
                if (hist) {
                    float p[3];
                    int vox;
                    sample_voxel(f, ro, rd, t, p, vox);
                    atomicMax(reinterpret_cast<int *>(hist) + vox, __float_as_int(alpha));
                }
                T *= expf(-sd);
                ++n;
                done = n >= lim || (!n_given && T < f.T_eps);
            }
            if (done) {
                if (C_out) {  // forward only: composited PQ colour and sample count
                    C_out[3 * b] = C[0];
                    C_out[3 * b + 1] = C[1];
                    C_out[3 * b + 2] = C[2];
                    n_used[b] = n;
                    live = false;
                    continue;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (target) {
                        const float diff = C[c] - linear_to_pq(target[3 * b + c]);
                        g[c] = diff > 0.0f ? inv_n : (diff < 0.0f ? -inv_n : 0.0f);
                        loss += fabsf(diff);
                    } else {
                        g[c] = gC_given[3 * b + c];
                    }
                    Cpre[c] = 0.0f;
                }
                T = 1.0f;
                k = 0;
                phase = n > 0 ? 1 : 2;
            }
        } else if (phase == 1) {  // gradients of samples k, k + 1, ...
#pragma unroll 1
            for (int e = 0; e < kCompSamples && k < n; ++e) {
                const float4 v = sc[k0 + k];
                const int step = rec[k0 + k].y;
                const float delta = f.t_tab[step + 1] - f.t_tab[step], sd = v.x * delta;
                const float alpha = -expm1f(-sd), Tn = T * expf(-sd), w = T * alpha;
                const float cc[3] = {v.y, v.z, v.w};
                float dsig = 0.0f, dz[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float suffix = C[c] - (Cpre[c] + w * cc[c]);
                    dsig += g[c] * delta * (Tn * cc[c] - suffix);
                    dz[c] = w * g[c] * cc[c] * (1.0f - cc[c]);
                    Cpre[c] += w * cc[c];
                }
                // dL/do_0 = dL/dsigma * sigma (sigma = exp(o_0 + bias)), with this pass's sigma
                sc[k0 + k] = make_float4(dsig * v.x, dz[0], dz[1], dz[2]);
                T = Tn;
                ++k;
            }
            if (k == n) phase = 2;
        } else {  // zeros for the samples after the last composited one
#pragma unroll 1
            for (int e = 0; e < 8 && k < m; ++e, ++k) sc[k0 + k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (k >= m) {
                n_used[b] = n;
                live = false;
            }
        }
    }
    if (loss_sum) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, s);
        if ((threadIdx.x & 31) == 0 && loss != 0.0f) atomicAdd(loss_sum, loss);
    }
}

// Warp inclusive scans over the 32 lanes.
__device__ __forceinline__ float warp_prod_scan(float x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x *= u;
    }
    return x;
}
__device__ __forceinline__ float warp_sum_scan(float x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x += u;
    }
    return x;
}

// The long rays of ray_comp_kernel (more than kLongRay samples), one warp
// each, 32 samples at a time: the transmittance before sample j is the carry
// times the product of exp(-sigma_i delta_i) over the chunk's earlier samples
// (a warp product scan), the composite stops after the first sample whose
// transmittance drops below T_eps, and the gradient walk takes the prefix of
// w_i c_i from a warp sum scan. The same quantities as ray_comp_kernel, with
// the fp32 products and sums in another order.
__global__ void __launch_bounds__(128)
ray_comp_long_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                     const int *__restrict__ cnt, const long long *__restrict__ off, const int2 *__restrict__ rec,
                     const int *__restrict__ n_given, const float *__restrict__ target,
                     const float *__restrict__ gC_given, float inv_n, float4 *__restrict__ sc,
                     int *__restrict__ n_used, float *__restrict__ loss_sum, float *__restrict__ hist,
                     float *__restrict__ C_out, const int *__restrict__ long_rays,
                     const unsigned int *__restrict__ n_long) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned total = *n_long;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    float loss = 0.0f;
    for (unsigned e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += warps) {
        const long long b = long_rays[e];
        const long long k0 = off[b];
        const int m = cnt[b];
        const int lim = n_given ? min(n_given[b], m) : m;
        float ro[3] = {0, 0, 0}, rd[3] = {0, 0, 1};
        if (hist) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ro[c] = o_in[3 * b + c];
                rd[c] = d_in[3 * b + c];
            }
        }
        // ---- composite ----
        float T = 1.0f, C[3] = {0, 0, 0};
        int n = 0;
        for (int c0 = 0; c0 < lim;) {  // uniform over the warp
            const int j = c0 + lane;
            const bool valid = j < lim;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float t = 0.0f, sd = 0.0f;
            if (valid) {
                v = sc[k0 + j];
                const int step = rec[k0 + j].y;
                t = f.t_tab[step];
                sd = v.x * (f.t_tab[step + 1] - t);
            }
            const float incl = warp_prod_scan(valid ? expf(-sd) : 1.0f);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 1.0f;
            const float Tj = T * excl, Ta = T * incl;
            const unsigned term = __ballot_sync(FULL, valid && !n_given && Ta < f.T_eps);
            const int last = term ? __ffs(term) - 1 : min(31, lim - 1 - c0);  // last composited lane
            const bool used = lane <= last;
            const float w = used ? Tj * (-expm1f(-sd)) : 0.0f;
            // the chunk's sum taken from the same scan the gradient walk uses, so
            // that its prefix at the last sample is C exactly (suffix 0 there)
            C[0] += __shfl_sync(FULL, warp_sum_scan(w * v.y), last);
            C[1] += __shfl_sync(FULL, warp_sum_scan(w * v.z), last);
            C[2] += __shfl_sync(FULL, warp_sum_scan(w * v.w), last);
            if (hist && used) {
                float p[3];
                int vox;
                sample_voxel(f, ro, rd, t, p, vox);
                atomicMax(reinterpret_cast<int *>(hist) + vox, __float_as_int(-expm1f(-sd)));
            }
            n += last + 1;
            T = __shfl_sync(FULL, Ta, last);
            if (term) break;
            c0 += 32;
        }
        if (C_out) {  // forward only
            if (lane == 0) {
                C_out[3 * b] = C[0];
                C_out[3 * b + 1] = C[1];
                C_out[3 * b + 2] = C[2];
                n_used[b] = n;
            }
            continue;
        }
        float g[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (target) {
                const float diff = C[c] - linear_to_pq(target[3 * b + c]);
                g[c] = diff > 0.0f ? inv_n : (diff < 0.0f ? -inv_n : 0.0f);
                if (lane == 0) loss += fabsf(diff);
            } else {
                g[c] = gC_given[3 * b + c];
            }
        }
        // ---- gradients of the composited samples ----
        T = 1.0f;
        float carry[3] = {0, 0, 0};
        for (int c0 = 0; c0 < n; c0 += 32) {  // uniform over the warp
            const int j = c0 + lane;
            const bool valid = j < n;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float delta = 0.0f, sd = 0.0f;
            if (valid) {
                v = sc[k0 + j];
                const int step = rec[k0 + j].y;
                delta = f.t_tab[step + 1] - f.t_tab[step];
                sd = v.x * delta;
            }
            const float incl = warp_prod_scan(valid ? expf(-sd) : 1.0f);
            float excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 1.0f;
            const float Tj = T * excl, Tn = T * incl;
            const float w = valid ? Tj * (-expm1f(-sd)) : 0.0f;
            const float cc[3] = {v.y, v.z, v.w};
            float dsig = 0.0f, dz[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float wc = w * cc[c];
                const float pre = warp_sum_scan(wc);  // inclusive prefix of w c in this chunk
                const float suffix = C[c] - (carry[c] + pre);
                dsig += g[c] * delta * (Tn * cc[c] - suffix);
                dz[c] = w * g[c] * cc[c] * (1.0f - cc[c]);
                carry[c] += __shfl_sync(FULL, pre, 31);
            }
            if (valid) sc[k0 + j] = make_float4(dsig * v.x, dz[0], dz[1], dz[2]);
            T = __shfl_sync(FULL, Tn, min(31, n - 1 - c0));
        }
        for (int j = n + lane; j < m; j += 32) sc[k0 + j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (lane == 0) n_used[b] = n;
    }
    if (loss_sum && lane == 0 && loss != 0.0f) atomicAdd(loss_sum, loss);
}

// ---- 4. sample backward -------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(kBwdThreads)
sample_bwd_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                  const float *__restrict__ r_in, const int2 *__restrict__ rec, const long long *__restrict__ off,
                  const int *__restrict__ n_used, long long n_samples, const float4 *__restrict__ grad_s,
                  float4 *__restrict__ dfeat_out, float *__restrict__ mlp_grad) {
    constexpr int D = 2 * L;
    using G = GradSm<D>;
    extern __shared__ float4 smem4[];
    float *sG = reinterpret_cast<float *>(smem4);
    float *stage = sG + G::size;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sA = stage + warp * 2 * 32 * kStride;
    float *sD = sA + 32 * kStride;
    for (int i = threadIdx.x; i < G::size; i += blockDim.x) sG[i] = 0.0f;
    __syncthreads();

    const float *W1 = f.mlp, *W2 = W1 + 64 * D, *W3 = W2 + 16 * 64, *W4 = W3 + 64 * 32, *W5 = W4 + 64 * 64;
    constexpr unsigned FULL = 0xffffffffu;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 32; base < n_samples;
         base += warps * 32) {
        const long long i = base + lane;
        bool have = false;
        float p[3] = {0, 0, 0}, dir[3] = {0.0f, 0.0f, 1.0f}, rn = 0.0f, dsig = 0.0f, dz[3] = {0, 0, 0};
        if (i < n_samples) {  // dsig: dL/do_0 (dL/dsigma * sigma)
            const int2 q = rec[i];
            const long long b = q.x;
            if (i - off[b] < n_used[b]) {
                have = true;
                const float o[3] = {o_in[3 * b], o_in[3 * b + 1], o_in[3 * b + 2]};
                dir[0] = d_in[3 * b];
                dir[1] = d_in[3 * b + 1];
                dir[2] = d_in[3 * b + 2];
                const float t = f.t_tab[q.y];
                int vox;
                sample_voxel(f, o, dir, t, p, vox);
                rn = footprint(f, t, r_in[b], p, nullptr, nullptr);
                const float4 gs = grad_s[i];
                dsig = gs.x;
                dz[0] = gs.y;
                dz[1] = gs.z;
                dz[2] = gs.w;
            }
        }
        if (!__any_sync(FULL, have)) continue;

        // ---- recompute the sample: features and forward MLPs ----
        float feat[D];
        if (have) {
            gather_features<L>(f, p, rn, feat);
        } else {
#pragma unroll
            for (int k = 0; k < D; ++k) feat[k] = 0.0f;
        }
        float o[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) o[k] = 0.0f;
#pragma unroll 2
        for (int j = 0; j < 64; ++j) {
            const float h = fmaxf(dot_row(W1 + j * D, feat, D), 0.0f);
#pragma unroll
            for (int k = 0; k < 16; ++k) o[k] = fmaf(__ldg(W2 + k * 64 + j), h, o[k]);
        }
        float h1[64];
        {
            float x[32];
#pragma unroll
            for (int k = 0; k < 16; ++k) x[k] = o[k];
            sh16(dir[0], dir[1], dir[2], x + 16);
#pragma unroll
            for (int j = 0; j < 64; ++j) h1[j] = fmaxf(dot_row(W3 + j * 32, x, 32), 0.0f);
        }
#pragma unroll 2
        for (int j = 0; j < 64; ++j) sA[lane * kStride + j] = fmaxf(dot_row(W4 + j * 64, h1, 64), 0.0f);

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
        for (int k = 0; k < 16; ++k) dout[k] = 0.0f;
#pragma unroll 4
        for (int j = 0; j < 64; ++j) {
            const float d = sD[lane * kStride + j];
#pragma unroll
            for (int k = 0; k < 16; ++k) dout[k] = fmaf(__ldg(W3 + j * 32 + k), d, dout[k]);
        }
        dout[0] += dsig;  // dL/do_0 from the ray pass (dL/dsigma * sigma)
        __syncwarp();
        // ---- W2: dout x h (h recomputed) ----
        float h[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) h[j] = fmaxf(dot_row(W1 + j * D, feat, D), 0.0f);
#pragma unroll
        for (int k = 0; k < 16; ++k) sD[lane * kStride + k] = dout[k];
#pragma unroll
        for (int j = 0; j < 64; ++j) sA[lane * kStride + j] = h[j];
        __syncwarp();
        minigemm_cols<16, 64>(sD, sA, sG + G::g2, G::s2, lane);
        float dh[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            float a = 0.0f;
#pragma unroll
            for (int k = 0; k < 16; ++k) a = fmaf(__ldg(W2 + k * 64 + j), dout[k], a);
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

        // ---- dL/dfeatures for the hash-grid scatter (a separate full-occupancy kernel) ----
        if (have) {
#pragma unroll
            for (int k = 0; k < D / 4; ++k)
                dfeat_out[i * (D / 4) + k] = make_float4(dfeat[4 * k], dfeat[4 * k + 1], dfeat[4 * k + 2], dfeat[4 * k + 3]);
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
// Samples one pass of the training pipeline holds at most unless the field
// sets its own budget (2^26 records: about 10 to 15 GB of per-sample buffers).
constexpr long long kDefaultSampleBudget = 1ll << 26;

struct TrainScratch {
    // per ray
    int *cnt = nullptr, *n_used = nullptr;
    long long *off = nullptr;
    int cap = 0;
    // per sample
    int2 *rec = nullptr;
    float4 *sc = nullptr;
    uint4 *feat = nullptr;    // bf16 features per sample (tensor-core backward only)
    float4 *dfeat = nullptr;  // dL/dfeatures per sample, fp32 (backward)
    long long scap = 0, fcap = 0, dcap = 0;
    unsigned long long *total = nullptr;   // device: [0] records, [1] [2] ray counters of count / ray composite,
                                           // [3] [4] long rays of ray composite / count (unsigned int each)
    long long *bsum = nullptr;             // per block of kScanPer rays: sum, then offset (count_pass)
    int2 *long_count = nullptr;            // per ray: (ray, step) handed from count_kernel to count_long_kernel
    int *long_comp = nullptr;              // per ray: rays handed from ray_comp_kernel to ray_comp_long_kernel
    unsigned long long *total_h = nullptr; // pinned host copy
    uint32_t *mask = nullptr;              // per ray: bits of its evaluated steps (count -> emit)
    long long mask_cap = 0;                // words allocated
    bool mask_valid = false;               // the last count pass wrote the bits
};

// The step bits of count_kernel cost S/8 bytes per ray; above this many bytes
// for a pass, emit marches the rays again instead.
constexpr long long kMaskBytesMax = 1ll << 30;

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
    if (!S.total) {
        if ((e = cudaMalloc(&S.total, 8 * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMallocHost(&S.total_h, sizeof(unsigned long long))) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "training scratch: %s", cudaGetErrorString(e));
    }
    if (B > S.cap) {
        cudaFree(S.cnt);
        cudaFree(S.n_used);
        cudaFree(S.off);
        cudaFree(S.bsum);
        cudaFree(S.long_count);
        cudaFree(S.long_comp);
        S.cnt = S.n_used = nullptr;
        S.off = S.bsum = nullptr;
        S.long_count = nullptr;
        S.long_comp = nullptr;
        S.cap = 0;
        if ((e = cudaMalloc(&S.cnt, sizeof(int) * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.n_used, sizeof(int) * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.off, sizeof(long long) * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.bsum, sizeof(long long) * (size_t)((B + kScanPer - 1) / kScanPer))) != cudaSuccess ||
            (e = cudaMalloc(&S.long_count, sizeof(int2) * (size_t)B)) != cudaSuccess ||
            (e = cudaMalloc(&S.long_comp, sizeof(int) * (size_t)B)) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "training scratch: %s", cudaGetErrorString(e));
        S.cap = B;
    }
    return VRNERF_OK;
}

static int ensure_samples(TrainScratch &S, long long n) {
    if (n <= S.scap) return VRNERF_OK;
    cudaFree(S.rec);
    cudaFree(S.sc);
    S.rec = nullptr;
    S.sc = nullptr;
    S.scap = 0;
    const long long want = n + n / 4 + 1024;
    cudaError_t e;
    if ((e = cudaMalloc(&S.rec, sizeof(int2) * (size_t)want)) != cudaSuccess ||
        (e = cudaMalloc(&S.sc, sizeof(float4) * (size_t)want)) != cudaSuccess) {
        cudaFree(S.rec);
        S.rec = nullptr;
        cudaGetLastError();  // a failed allocation leaves no error behind
        return fail(VRNERF_ENOMEM, "sample records (%lld): %s", want, cudaGetErrorString(e));
    }
    S.scap = want;
    return VRNERF_OK;
}

void release_train_scratch(vrnerf_field *F) {
    if (!F->train_scratch) return;
    TrainScratch *S = static_cast<TrainScratch *>(F->train_scratch);
    cudaFree(S->cnt);
    cudaFree(S->n_used);
    cudaFree(S->off);
    cudaFree(S->bsum);
    cudaFree(S->long_count);
    cudaFree(S->long_comp);
    cudaFree(S->rec);
    cudaFree(S->sc);
    cudaFree(S->feat);
    cudaFree(S->dfeat);
    cudaFree(S->mask);
    cudaFree(S->total);
    if (S->total_h) cudaFreeHost(S->total_h);
    delete S;
    F->train_scratch = nullptr;
}

template <typename K>
static cudaError_t grid_for(K kern, int threads, size_t smem, long long work, int &blocks) {
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    long long g = (long long)num_sms() * bps, want = (work + threads - 1) / threads;
    blocks = (int)(want < g ? (want < 1 ? 1 : want) : g);
    return cudaSuccess;
}

// CTAs (4 warps each) of the warp-per-ray kernels for the long rays of a
// pass of B rays: their number is known on the device only, so the grid is
// sized for the worst case up to 4 CTAs per SM and the warps loop.
static int long_ray_blocks(long long B) {
    const long long want = (B + 3) / 4, cap = (long long)num_sms() * 4;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

// Marches rays [0, B) of (o, d), counts their evaluated samples and reserves
// their records (S.cnt, S.off: contiguous per ray, in ray order); *n receives
// the total. One small read-back.
static int count_pass(vrnerf_field *F, TrainScratch &S, const float *o, const float *d, int B, cudaStream_t st,
                      long long *n) {
    int blocks = 0;
    cudaError_t e = cudaMemsetAsync(S.total, 0, 8 * sizeof(unsigned long long), st);
    // step bits for emit, when they fit (else emit marches again)
    const int mw = (F->view.S + 31) / 32;
    const long long words = (long long)B * mw;
    if (words * 4 <= kMaskBytesMax && words > S.mask_cap) {
        cudaFree(S.mask);
        S.mask = nullptr;
        S.mask_cap = 0;
        if (cudaMalloc(&S.mask, (size_t)words * 4) == cudaSuccess)
            S.mask_cap = words;
        else
            cudaGetLastError();  // no bits this time: emit marches again
    }
    uint32_t *mask = words <= S.mask_cap ? S.mask : nullptr;
    if (e == cudaSuccess && mask) e = cudaMemsetAsync(mask, 0, (size_t)words * 4, st);
    S.mask_valid = mask != nullptr;
    if (e == cudaSuccess) e = grid_for(count_kernel, 128, 0, B, blocks);
    if (e == cudaSuccess) {
        unsigned int *n_long = reinterpret_cast<unsigned int *>(S.total + 4);
        count_kernel<<<blocks, 128, 0, st>>>(F->view, o, d, B, S.cnt, mask, mw, S.total + 1, S.long_count, n_long);
        if ((e = cudaGetLastError()) == cudaSuccess)
            count_long_kernel<<<long_ray_blocks(B), 128, 0, st>>>(F->view, o, d, S.cnt, mask, mw, S.long_count,
                                                                  n_long);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && B > 0) {  // record offsets: exclusive prefix sums of the counts
        const int nb = (B + kScanPer - 1) / kScanPer;
        if (nb <= kScanOneBlock) {
            scan_one_block_kernel<<<1, kScanThreads, 0, st>>>(S.cnt, B, S.off, S.total);
        } else {
            scan_sums_kernel<<<nb, kScanThreads, 0, st>>>(S.cnt, B, S.bsum);
            scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(S.bsum, nb, S.total);
            scan_offsets_kernel<<<nb, kScanThreads, 0, st>>>(S.cnt, B, S.bsum, S.off);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(S.total_h, S.total, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "backward: count");
    *n = (long long)*S.total_h;
    return VRNERF_OK;
}

// The per-sample part of the pipeline for Bc rays whose samples count_pass
// has just counted (n records); pointers are already offset to the rays.
// inv3B is 1 / (3 B) of the whole batch. ENOMEM when the per-sample buffers
// cannot be allocated (nothing launched then).
template <int L>
static int samples_pass(vrnerf_field *F, TrainScratch &S, const float *o, const float *d, const float *r, int Bc,
                        long long n, float inv3B, const float *target, const float *gC, const int *n_given,
                        cudaStream_t st, float *C_out, int *n_out) {
    constexpr int D = 2 * L;
    const FieldView &f = F->view;
    cudaError_t e = cudaSuccess;
    int blocks = 0;
    int rc = ensure_samples(S, n);
    if (rc) return rc;
    const bool tc_bwd = !C_out && F->train_prec == VRNERF_BF16;
    if (tc_bwd && n > S.fcap) {
        cudaFree(S.feat);
        S.feat = nullptr;
        S.fcap = 0;
        const long long want = n + n / 4 + 1024;
        if ((e = cudaMalloc(&S.feat, sizeof(uint4) * (size_t)(D / 8) * (size_t)want)) != cudaSuccess)
            return cudaGetLastError(), fail(VRNERF_ENOMEM, "sample features (%lld): %s", want, cudaGetErrorString(e));
        S.fcap = want;
    }
    if (!C_out && n > S.dcap) {
        cudaFree(S.dfeat);
        S.dfeat = nullptr;
        S.dcap = 0;
        const long long want = n + n / 4 + 1024;
        if ((e = cudaMalloc(&S.dfeat, sizeof(float4) * (size_t)(D / 4) * (size_t)want)) != cudaSuccess)
            return cudaGetLastError(), fail(VRNERF_ENOMEM, "sample feature gradients (%lld): %s", want,
                                            cudaGetErrorString(e));
        S.dcap = want;
    }
    if (n > 0) {
        e = grid_for(emit_kernel, 128, 0, Bc, blocks);
        if (e == cudaSuccess) {
            emit_kernel<<<blocks, 128, 0, st>>>(f, o, d, Bc, S.off, S.cnt, S.rec, S.mask_valid ? S.mask : nullptr,
                                                (f.S + 31) / 32);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && tc_bwd) {
            // bf16 training: the MLPs of the forward on the tensor cores too
            e = launch_fwd_tc(F, o, d, r, S.rec, n, S.sc, S.feat, st);
        } else if (e == cudaSuccess) {
            const size_t smem_f = sizeof(float) * SimtW<D>::size;
            e = cudaFuncSetAttribute(sample_fwd_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_f);
            if (e == cudaSuccess) e = grid_for(sample_fwd_kernel<L>, 128, smem_f, n, blocks);
            if (e == cudaSuccess) {
                sample_fwd_kernel<L><<<blocks, 128, smem_f, st>>>(f, o, d, r, S.rec, n, S.sc, nullptr);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = grid_for(ray_comp_kernel, 128, 0, Bc, blocks);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.total + 2, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        unsigned int *n_long = reinterpret_cast<unsigned int *>(S.total + 3);
        ray_comp_kernel<<<blocks, 128, 0, st>>>(f, o, d, Bc, S.cnt, S.off, S.rec, n_given, target, gC, inv3B, S.sc,
                                                C_out ? n_out : S.n_used, target ? F->loss_acc : nullptr,
                                                C_out ? nullptr : F->hist, C_out, S.total + 2, S.long_comp, n_long);
        if ((e = cudaGetLastError()) == cudaSuccess)
            ray_comp_long_kernel<<<long_ray_blocks(Bc), 128, 0, st>>>(
                f, o, d, S.cnt, S.off, S.rec, n_given, target, gC, inv3B, S.sc, C_out ? n_out : S.n_used,
                target ? F->loss_acc : nullptr, C_out ? nullptr : F->hist, C_out, S.long_comp, n_long);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && n > 0 && tc_bwd) {
        e = launch_bwd_tc(F, o, d, r, S.rec, S.off, S.n_used, n, S.sc, S.feat, S.dfeat, st);
    } else if (e == cudaSuccess && n > 0 && !C_out) {
        const size_t smem_b = sizeof(float) * ((size_t)GradSm<D>::size + (size_t)(kBwdThreads / 32) * 2 * 32 * kStride);
        e = cudaFuncSetAttribute(sample_bwd_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
        if (e == cudaSuccess) e = grid_for(sample_bwd_kernel<L>, kBwdThreads, smem_b, n, blocks);
        if (e == cudaSuccess) {
            sample_bwd_kernel<L><<<blocks, kBwdThreads, smem_b, st>>>(f, o, d, r, S.rec, S.off, S.n_used, n, S.sc,
                                                                      S.dfeat, F->mlp_grad);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = launch_grid_scatter(F, o, d, r, S.rec, S.off, S.n_used, n, S.dfeat, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "backward");
    return VRNERF_OK;
}

// The sample-parallel backward (header comment): gradients into the field's
// buffers (zeroed here). target != nullptr: L1 loss, accumulated into
// F->loss_acc; else gC (dL/dC per ray) and n_given (composited samples).
//
// Per-step memory grows with the batch's samples (record, sigma/colour and
// their gradients, feature gradients: 152 B per sample, 216 B with bf16
// features). A batch whose samples exceed the field's sample budget, or whose
// buffers cannot be allocated, runs in ray ranges that fit, one after the
// other; gradients, loss and history accumulate over the ranges, so the
// result is the same as one pass (up to the order of float additions).
template <int L>
static int backward_t(vrnerf_field *F, const float *o, const float *d, const float *r, int B, const float *target,
                      const float *gC, const int *n_given, cudaStream_t st, float *C_out = nullptr,
                      int *n_out = nullptr) {
    TrainScratch &S = *static_cast<TrainScratch *>(F->train_scratch);
    const FieldView &f = F->view;
    cudaError_t e = cudaSuccess;
    if (!C_out) {
        e = cudaMemsetAsync(F->grid_grad, 0, grid_entries(F->desc) * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(F->mlp_grad, 0, sizeof(float) * f.n_mlp, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(F->loss_acc, 0, 64, st);
        if (e != cudaSuccess) return cuda_fail(e, "backward: zero gradients");
    }
    const float inv3B = 1.0f / (3.0f * B);
    // a single ray never needs more than max_steps records
    long long budget = F->sample_budget > 0 ? (long long)F->sample_budget : kDefaultSampleBudget;
    if (budget < f.S) budget = f.S;
    long long n = 0;
    int rc = count_pass(F, S, o, d, B, st, &n);
    if (rc) return rc;
    long long rays_per = n > budget ? (long long)((double)B * (double)budget / (double)n) : B;
    if (rays_per < 1) rays_per = 1;
    int b0 = 0;
    bool counted = rays_per >= B;  // S.cnt / S.off hold the counts of the next range
    while (b0 < B) {
        const int Bc = (int)(B - b0 < rays_per ? B - b0 : rays_per);
        if (!counted && (rc = count_pass(F, S, o + 3ll * b0, d + 3ll * b0, Bc, st, &n))) return rc;
        counted = false;
        if (n > budget && Bc > 1) {  // this range still holds too many samples: halve it
            rays_per = Bc / 2;
            continue;
        }
        rc = samples_pass<L>(F, S, o + 3ll * b0, d + 3ll * b0, r + b0, Bc, n, inv3B, target ? target + 3ll * b0 : nullptr,
                             gC ? gC + 3ll * b0 : nullptr, n_given ? n_given + b0 : nullptr, st,
                             C_out ? C_out + 3ll * b0 : nullptr, n_out ? n_out + b0 : nullptr);
        if (rc == VRNERF_ENOMEM && Bc > 1) {
            // not enough device memory for this range: clear the failed
            // allocation's error state and retry with half the rays
            cudaGetLastError();
            budget = n / 2 > f.S ? n / 2 : f.S;
            rays_per = Bc / 2;
            continue;
        }
        if (rc) return rc;
        b0 += Bc;
    }
    return VRNERF_OK;
}

}  // namespace vrn

using namespace vrn;

extern "C" {

int vrnerf_backward(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii,
                    const float *target_linear, int32_t B, float *loss_host, void *stream) {
    try {
        NvtxRange nvtx_range("vrnerf_backward");
        if (!F || !rays_o || !rays_d || !radii || !target_linear) return fail(VRNERF_EINVAL, "NULL argument");
        if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
        int rc = ensure_train(F, B);
        if (rc) return rc;
        cudaStream_t st = (cudaStream_t)stream;
        rc = F->view.L == 8 ? backward_t<8>(F, rays_o, rays_d, radii, B, target_linear, nullptr, nullptr, st)
                            : backward_t<16>(F, rays_o, rays_d, radii, B, target_linear, nullptr, nullptr, st);
        if (rc) return rc;
        if (loss_host) {
            float sum = 0.0f;
            cudaError_t e = cudaMemcpyAsync(&sum, F->loss_acc, sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "backward: loss");
            *loss_host = sum / (3.0f * B);
        }
        return VRNERF_OK;
    } catch (...) {
        return fail(VRNERF_EINVAL, "backward: unexpected C++ exception");
    }
}

int vrnerf_forward_rays(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii, int32_t B,
                        float *out_pq, int32_t *out_n, void *stream) {
    try {
        NvtxRange nvtx_range("vrnerf_forward_rays");
        if (!F || !rays_o || !rays_d || !radii || !out_pq || !out_n) return fail(VRNERF_EINVAL, "NULL argument");
        if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
        int rc = ensure_train(F, B);
        if (rc) return rc;
        cudaStream_t st = (cudaStream_t)stream;
        return F->view.L == 8
                   ? backward_t<8>(F, rays_o, rays_d, radii, B, nullptr, nullptr, nullptr, st, out_pq, out_n)
                   : backward_t<16>(F, rays_o, rays_d, radii, B, nullptr, nullptr, nullptr, st, out_pq, out_n);
    } catch (...) {
        return fail(VRNERF_EINVAL, "forward_rays: unexpected C++ exception");
    }
}

int vrnerf_backward_from_grad(vrnerf_field *F, const float *rays_o, const float *rays_d, const float *radii,
                              int32_t B, const int32_t *n_fwd, const float *grad_pq, void *stream) {
    try {
        NvtxRange nvtx_range("vrnerf_backward_from_grad");
        if (!F || !rays_o || !rays_d || !radii || !n_fwd || !grad_pq) return fail(VRNERF_EINVAL, "NULL argument");
        if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
        int rc = ensure_train(F, B);
        if (rc) return rc;
        cudaStream_t st = (cudaStream_t)stream;
        return F->view.L == 8 ? backward_t<8>(F, rays_o, rays_d, radii, B, nullptr, grad_pq, n_fwd, st)
                              : backward_t<16>(F, rays_o, rays_d, radii, B, nullptr, grad_pq, n_fwd, st);
    } catch (...) {
        return fail(VRNERF_EINVAL, "backward_from_grad: unexpected C++ exception");
    }
}

int vrnerf_field_set_sample_budget(vrnerf_field *F, uint64_t max_samples) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    F->sample_budget = max_samples;
    return VRNERF_OK;
}

int vrnerf_field_set_train_precision(vrnerf_field *F, int32_t precision) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (precision != VRNERF_FP32 && precision != VRNERF_BF16)
        return fail(VRNERF_EINVAL, "training precision must be VRNERF_FP32 or VRNERF_BF16");
    F->train_prec = precision;
    return VRNERF_OK;
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
    NvtxRange nvtx_range("vrnerf_adam_step");
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
