// render_simt.cu -- plain fp32 renderer: the whole per-ray path in one
// persistent kernel with the MLP on the CUDA cores (the fp32 baseline).
//
// Each thread owns one ray slot. A round has two phases:
//  1. march: every thread advances its ray through the exponential samples
//     (Sec. 6) until it reaches a sample in an occupied voxel (Sec. 4.3) or
//     the ray ends; finished slots take new rays from a global counter, one
//     atomic per warp;
//  2. evaluate: threads holding a sample gather the LOD-weighted hash-grid
//     features (Sec. 4.2.1, Eq. 3), run the density and colour MLPs (Sec. 6)
//     with weights in shared memory, and composite front to back, stopping
//     when transmittance drops below T_eps; the output is PQ-decoded
//     (Eq. 1-2).
// Phase 2 runs with the warp converged, so the MLP's FMAs are not serialised
// against the march.
#include <mutex>

#include "internal.h"
#include "simt_mlp.cuh"

namespace vrn {

constexpr int kSimtThreads = 128;
constexpr int kChunk = 32;  // march steps between refill points

// d o_0 / d feat = W1^T (relu'(W1 feat) * W2[0, :]) with the weights in
// shared memory (W2^T row j holds W2[:, j]).
template <int D>
__device__ __forceinline__ void density_feat_grad(const float *__restrict__ s, const float feat[D], float g[D]) {
    using W = SimtW<D>;
#pragma unroll
    for (int q = 0; q < D; ++q) g[q] = 0.0f;
    for (int j = 0; j < 64; ++j) {
        const float4 *w = reinterpret_cast<const float4 *>(s + W::oW1 + j * D);
        float a = 0.0f;
#pragma unroll
        for (int q = 0; q < D / 4; ++q) {
            const float4 v = w[q];
            a = fmaf(v.x, feat[4 * q], a);
            a = fmaf(v.y, feat[4 * q + 1], a);
            a = fmaf(v.z, feat[4 * q + 2], a);
            a = fmaf(v.w, feat[4 * q + 3], a);
        }
        if (a > 0.0f) {
            const float c = s[W::oW2T + j * 16];
#pragma unroll
            for (int q = 0; q < D / 4; ++q) {
                const float4 v = w[q];
                g[4 * q] = fmaf(c, v.x, g[4 * q]);
                g[4 * q + 1] = fmaf(c, v.y, g[4 * q + 1]);
                g[4 * q + 2] = fmaf(c, v.z, g[4 * q + 2]);
                g[4 * q + 3] = fmaf(c, v.w, g[4 * q + 3]);
            }
        }
    }
}

// v = sum_q g_q d feat_q / d p at a fixed footprint: per level, w_l N_l
// times the derivative of the trilinear interpolation along each axis (the
// corner weight's factor of that axis replaced by +-1) gives the gradient in
// grid coordinates, then the grid map's Jacobian (1 / extent, or the
// contraction's) takes it to world coordinates. The corners are fetched
// again (L2-resident) instead of kept from the gather.
template <int L>
__device__ __forceinline__ void feature_pos_grad(const FieldView &f, const float p[3], float r_norm,
                                                 const float g[2 * L], float v[3]) {
    float ph[3];
    grid_position(f, p, ph);
    const float Ls = lod_star(f, r_norm);
    v[0] = v[1] = v[2] = 0.0f;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const float wl = lod_weight(Ls, l);
        if (wl == 0.0f) continue;
        uint32_t idx[8];
        float fr[3];
        level_corners_ph(f, l, ph, idx, fr);
        float d0[3] = {0, 0, 0}, d1[3] = {0, 0, 0};
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float2 e = load_feat(f, l, idx[b]);
            const float wx = b & 1 ? fr[0] : 1.0f - fr[0], wy = b & 2 ? fr[1] : 1.0f - fr[1],
                        wz = b & 4 ? fr[2] : 1.0f - fr[2];
            const float dw[3] = {(b & 1 ? 1.0f : -1.0f) * wy * wz, (b & 2 ? 1.0f : -1.0f) * wx * wz,
                                 (b & 4 ? 1.0f : -1.0f) * wx * wy};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                d0[k] = fmaf(dw[k], e.x, d0[k]);
                d1[k] = fmaf(dw[k], e.y, d1[k]);
            }
        }
        const float sc = wl * (float)f.N[l];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = fmaf(sc, fmaf(g[2 * l], d0[k], g[2 * l + 1] * d1[k]), v[k]);
    }
    // v is the gradient with respect to the grid position ph; chain to p
    if (f.contract) {
        float x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = (p[k] - f.cen[k]) * f.inv_h;
        contract_jtv(x, v);
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] *= 0.25f * f.inv_h;
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] *= f.inv_ext;
    }
}

template <int L, bool NRM, bool CT>
__global__ void __launch_bounds__(kSimtThreads, 4)
render_simt_kernel(const FieldView f, const RaySource src, const RenderOut out,
                   unsigned long long *__restrict__ counter) {
    constexpr int D = 2 * L;
    extern __shared__ float4 smem4[];
    float *sW = reinterpret_cast<float *>(smem4);
    float *sT = sW + SimtW<D>::size;
    load_weights_simt<D>(f.mlp, sW);
    for (int i = threadIdx.x; i <= f.S; i += blockDim.x) sT[i] = f.t_tab[i];
    __syncthreads();

    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    long long ray = -1, pix = 0;
    bool exhausted = false;
    MarchRay mr;
    float r = 0.0f, T = 1.0f, C[3] = {0, 0, 0}, Dp = 0.0f;
    float Nm[3] = {0, 0, 0};
    float adj[CT ? 6 : 1];  // contracted scenes: offsets to the adjacent pixels' rays
    bool has_adj = false;
    int n_eval = 0;
    unsigned st_samples = 0, st_levels = 0, st_steps = 0, st_rays = 0;

    while (true) {
        bool have = false;
        float p[3];
        // ---- phase 1: march to the next occupied sample, refilling slots ----
        while (true) {
            const bool need = ray < 0 && !exhausted;
            const unsigned m = __ballot_sync(FULL, need);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
                if (need) {
                    long long slot = (long long)base + __popc(m & ((1u << lane) - 1u));
                    if (slot >= src.n_slots) {
                        exhausted = true;
                    } else if (slot_ray(src, f, slot, mr.o, mr.d, r, pix, CT ? adj : nullptr,
                                        CT ? &has_adj : nullptr)) {
                        march_init(f, mr);
                        ray = slot;
                        n_eval = 0;
                        T = 1.0f;
                        Dp = 0.0f;
                        C[0] = C[1] = C[2] = 0.0f;
                        Nm[0] = Nm[1] = Nm[2] = 0.0f;
                    }
                }
            }
            if (ray >= 0 && !have) {
                const int mres = march_next(f, sT, mr, p, kChunk, st_steps);
                if (mres == MARCH_SAMPLE) {
                    have = true;
                } else if (mres == MARCH_END) {
                    finish_outputs(out, pix, C, T, n_eval, Dp, NRM ? Nm : nullptr, f.check);
                    ray = -1;
                    ++st_rays;
                }
            }
            if (__all_sync(FULL, have || exhausted)) break;
        }
        if (!__any_sync(FULL, have)) break;
        // ---- phase 2: features, MLPs, compositing ----
        if (have) {
            const float t = sT[mr.step], delta = sT[mr.step + 1] - t;
            float r_norm;
            if constexpr (CT)
                r_norm = footprint(f, t, r, p, has_adj ? adj : nullptr, has_adj ? adj + 3 : nullptr);
            else
                r_norm = t * r * f.inv_ext;
            float feat[D];
            st_levels += gather_features<L>(f, p, r_norm, feat);
            ++st_samples;
            float sigma, rgb[3];
            mlp_simt<D>(sW, feat, mr.d, f.density_bias, sigma, rgb);
            const float sd = sigma * delta;
            const float w = T * (-expm1f(-sd));
            C[0] += w * rgb[0];
            C[1] += w * rgb[1];
            C[2] += w * rgb[2];
            Dp += w * t;
            if constexpr (NRM) {
                float g[D], v[3];
                density_feat_grad<D>(sW, feat, g);
                feature_pos_grad<L>(f, p, r_norm, g, v);
                const float len = sqrtf(fmaf(v[0], v[0], fmaf(v[1], v[1], v[2] * v[2])));
                if (len > 0.0f) {
                    const float s = -w / len;
                    Nm[0] = fmaf(s, v[0], Nm[0]);
                    Nm[1] = fmaf(s, v[1], Nm[1]);
                    Nm[2] = fmaf(s, v[2], Nm[2]);
                }
            }
            T *= expf(-sd);
            ++n_eval;
            ++mr.step;
            if (T < f.T_eps) {
                finish_outputs(out, pix, C, T, n_eval, Dp, NRM ? Nm : nullptr, f.check);
                ray = -1;
                ++st_rays;
            }
        }
    }
    add_stats(out.stats, st_samples, st_levels, st_steps, st_rays);
}

template <int L>
__global__ void __launch_bounds__(kSimtThreads)
query_simt_kernel(const FieldView f, const float *__restrict__ pos, const float *__restrict__ dir,
                  const float *__restrict__ radius, int n, float *__restrict__ sigma_out,
                  float *__restrict__ rgb_out, float *__restrict__ feat_out) {
    constexpr int D = 2 * L;
    extern __shared__ float4 smem4[];
    float *sW = reinterpret_cast<float *>(smem4);
    load_weights_simt<D>(f.mlp, sW);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    float dd[3] = {dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]};
    float feat[D];
    gather_features<L>(f, p, footprint(f, 1.0f, radius[i], p, nullptr, nullptr), feat);
    float sigma, rgb[3];
    mlp_simt<D>(sW, feat, dd, f.density_bias, sigma, rgb);
    sigma_out[i] = sigma;
    for (int c = 0; c < 3; ++c) rgb_out[3 * i + c] = rgb[c];
    if (feat_out)
        for (int k = 0; k < D; ++k) feat_out[(long long)i * D + k] = feat[k];
}

__global__ void tonemap_kernel(const float *__restrict__ pq, const float *__restrict__ T, long long n,
                               float exposure, unsigned int *__restrict__ rgba8) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float lin[3] = {pq_to_linear(__ldg(pq + 3 * i)), pq_to_linear(__ldg(pq + 3 * i + 1)),
                              pq_to_linear(__ldg(pq + 3 * i + 2))};
        rgba8[i] = tonemap_rgba8(lin, T ? __ldg(T + i) : 0.0f, exposure);
    }
}

cudaError_t launch_tonemap(const float *pq, const float *T, long long n, float exposure, unsigned int *rgba8,
                           cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    long long blocks = (n + 255) / 256, cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    tonemap_kernel<<<(unsigned)blocks, 256, 0, st>>>(pq, T, n, exposure, rgba8);
    return cudaGetLastError();
}

__global__ void debug_march_kernel(const FieldView f, const float *__restrict__ o_in,
                                   const float *__restrict__ d_in, int B, int cap,
                                   int *__restrict__ rec_i, int *__restrict__ rec_vox,
                                   int *__restrict__ count) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // the render kernels' march (with empty-space skipping when enabled)
    MarchRay m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m.o[k] = o_in[3 * b + k];
        m.d[k] = d_in[3 * b + k];
    }
    march_init(f, m);
    unsigned tested = 0;
    int n = 0;
    float p[3];
    while (march_next(f, f.t_tab, m, p, 1 << 30, tested) == MARCH_SAMPLE) {
        int vox;
        sample_voxel(f, m.o, m.d, f.t_tab[m.step], p, vox);
        if (n < cap) {
            rec_i[(long long)b * cap + n] = m.step;
            rec_vox[(long long)b * cap + n] = vox;
        }
        ++n;
        ++m.step;
    }
    count[b] = n;
}

__global__ void debug_corners_kernel(const FieldView f, const float *__restrict__ pos, int n,
                                     uint32_t *__restrict__ idx) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (long long)n * f.L) return;
    const int i = (int)(q / f.L), l = (int)(q % f.L);
    float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
    uint32_t id[8];
    float fr[3];
    level_corners(f, l, p, id, fr);
    for (int b = 0; b < 8; ++b) idx[q * 8 + b] = id[b];
}

// ---------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------
size_t simt_smem_bytes(const FieldView &f) {
    const int wsize = f.L == 8 ? SimtW<16>::size : SimtW<32>::size;
    return sizeof(float) * (size_t)(wsize + f.S + 1);
}

template <int L, bool NRM, bool CT>
static cudaError_t render_simt_t(const FieldView &f, const RaySource &src, const RenderOut &out,
                                 unsigned long long *counter, cudaStream_t st) {
    // launch shape cached per device: the shared-memory attribute is a
    // per-device setting, and host threads may render on different devices
    constexpr int kDevices = 64;
    static std::mutex mu;
    static size_t configured_smem[kDevices] = {};
    static int cached_blocks[kDevices] = {};
    const size_t smem = simt_smem_bytes(f);
    auto kern = render_simt_kernel<L, NRM, CT>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int blocks_per_sm = 0;
    if (dev >= 0 && dev < kDevices) {
        std::lock_guard<std::mutex> lock(mu);
        if (configured_smem[dev] != smem) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_blocks[dev], kern, kSimtThreads, smem);
            if (e != cudaSuccess) return e;
            configured_smem[dev] = smem;
        }
        blocks_per_sm = cached_blocks[dev];
    } else {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, kSimtThreads, smem);
        if (e != cudaSuccess) return e;
    }
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    long long want = (src.n_slots + kSimtThreads - 1) / kSimtThreads;
    long long grid = (long long)num_sms() * blocks_per_sm;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kSimtThreads, smem, st>>>(f, src, out, counter);
    return cudaGetLastError();
}

cudaError_t launch_render_simt(const FieldView &f, const RaySource &src, const RenderOut &out,
                               unsigned long long *counter, cudaStream_t st) {
    const bool nrm = out.normal != nullptr, ct = f.contract != 0;
    if (f.L == 8) {
        if (ct) return nrm ? render_simt_t<8, true, true>(f, src, out, counter, st)
                           : render_simt_t<8, false, true>(f, src, out, counter, st);
        return nrm ? render_simt_t<8, true, false>(f, src, out, counter, st)
                   : render_simt_t<8, false, false>(f, src, out, counter, st);
    }
    if (ct) return nrm ? render_simt_t<16, true, true>(f, src, out, counter, st)
                       : render_simt_t<16, false, true>(f, src, out, counter, st);
    return nrm ? render_simt_t<16, true, false>(f, src, out, counter, st)
               : render_simt_t<16, false, false>(f, src, out, counter, st);
}

template <int L>
static cudaError_t query_simt_t(const FieldView &f, const float *pos, const float *dir,
                                const float *radius, int n, float *sigma, float *rgb, float *feat,
                                cudaStream_t st) {
    const size_t smem = sizeof(float) * SimtW<2 * L>::size;
    auto kern = query_simt_kernel<L>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(n + kSimtThreads - 1) / kSimtThreads, kSimtThreads, smem, st>>>(f, pos, dir, radius, n,
                                                                             sigma, rgb, feat);
    return cudaGetLastError();
}

cudaError_t launch_query_simt(const FieldView &f, const float *pos, const float *dir,
                              const float *radius, int n, float *sigma, float *rgb, float *feat,
                              cudaStream_t st) {
    return f.L == 8 ? query_simt_t<8>(f, pos, dir, radius, n, sigma, rgb, feat, st)
                    : query_simt_t<16>(f, pos, dir, radius, n, sigma, rgb, feat, st);
}

cudaError_t launch_debug_march(const FieldView &f, const float *o, const float *d, int B, int cap,
                               int *rec_i, int *rec_vox, int *count, cudaStream_t st) {
    debug_march_kernel<<<(B + 127) / 128, 128, 0, st>>>(f, o, d, B, cap, rec_i, rec_vox, count);
    return cudaGetLastError();
}

cudaError_t launch_debug_corners(const FieldView &f, const float *pos, int n, uint32_t *idx,
                                 cudaStream_t st) {
    long long q = (long long)n * f.L;
    debug_corners_kernel<<<(unsigned)((q + 127) / 128), 128, 0, st>>>(f, pos, n, idx);
    return cudaGetLastError();
}

}  // namespace vrn
