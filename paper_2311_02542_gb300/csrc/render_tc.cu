// render_tc.cu -- the renderer with its MLPs on the tcgen05 tensor cores
// (the paper's in-register tensor-core MLP, Sec. 5, rebuilt for sm_103a).
//
// A CTA of 128 threads owns 128 ray slots; each round every slot marches to
// its next evaluated sample (Sec. 4.3), gathers its LOD-weighted hash-grid
// features (Sec. 4.2.1, Eq. 3) and writes them as one row of a 128-row
// operand tile in shared memory. The five layers of the density and colour
// MLPs (Sec. 6) then run as M=128 tcgen05 MMAs (fp16 or bf16 operands, fp32
// accumulation in TMEM): one thread issues each layer and commits it to an
// mbarrier; all four warps read their 32 TMEM lanes back (tcgen05.ld),
// apply ReLU / exp / sigmoid and write the next layer's operand rows. Each
// thread then composites its own sample front to back and stops its ray when
// transmittance drops below T_eps; the PQ decode (Eq. 1-2) runs when the ray
// finishes. Slots whose rays end take new rays from a global counter, so the
// tile stays full until the frame runs out of rays.
//
// Shared memory per CTA: MLP weights in the MMA operand layout (18-20 KB),
// one 128 x 64 activation tile (16 KB, reused by every layer), the sample
// distance table, an mbarrier. TMEM: 64 columns (every layer writes columns
// 0 .. N-1 after the previous layer's values have been read).
//
// Look-ahead march (contracted scenes). The samples a ray evaluates do not
// depend on compositing (only early termination cuts the list short), so a
// lane may find its ray's next samples before the current one is shaded. The
// warp marches one iteration at a time and stops once every lane has a
// sample queued; lanes that already have one keep marching meanwhile and
// queue up to kLookahead samples; a ray that terminates drops what it
// queued. This pays where rays are long (an unbounded scene's far field:
// tens of samples per ray), and costs more than it saves on the few samples
// per ray of a bounded room, whose lanes march in chunks of kTcChunk
// iterations and hold one sample.
#include "field.h"
#include "tc_mlp.cuh"

namespace vrn {

#ifndef VRN_LOOKAHEAD
#define VRN_LOOKAHEAD 32
#endif
constexpr int kLookahead = VRN_LOOKAHEAD;  // samples a lane may hold found ahead of shading

// Tiles per CTA (NT): each 128-thread warpgroup runs its own 128-row tile
// (its own activation tile, mbarrier, TMEM columns and named barrier) and
// the tiles share one weight image, so more tiles per CTA leave more of the
// SM's shared memory to L1 for the hash-grid gather. Bounded scenes with
// fp16 or bf16 operands run four tiles per 16-warp CTA, two CTAs per SM at
// 64 registers a thread: 32 warps and 168 KB of shared memory per SM,
// against six 4-warp CTAs at 80 registers (24 warps, 228 KB); measured 6 %
// faster on the room frame despite the extra register spills. The fp8 path
// spills far more at 64 registers (7 % slower) and keeps one tile per CTA.
// Contracted scenes keep two tiles per 8-warp CTA, three CTAs per SM at 80
// registers, as their look-ahead queue lives in registers (10 % faster than
// one tile on the unbounded frame; four tiles: 4 % slower).
#ifndef VRN_TILES_BOUNDED
#define VRN_TILES_BOUNDED 4
#endif
template <bool CT, int FMT>
constexpr int render_tiles() { return CT ? 2 : (FMT == 2 ? 1 : VRN_TILES_BOUNDED); }
// resident CTAs per SM that the register budget is cut for
template <int NT>
constexpr int render_min_blocks() { return NT == 4 ? 2 : kTcMinBlocks / NT; }
static_assert((kLookahead & (kLookahead - 1)) == 0, "the look-ahead queue is a power-of-two ring");

template <int L, int FMT, bool CT, int NT = render_tiles<CT, FMT>()>
__global__ void __launch_bounds__(kTcThreads * NT, render_min_blocks<NT>())
render_tc_kernel(const FieldView f, const RaySource src, const RenderOut out,
                 unsigned long long *__restrict__ counter, const uint4 *__restrict__ wimg,
                 unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *unused;
    const TcShared S = tc_setup<D, FMT, NT>(smem, wimg, unused, nullptr, 0);
    const int row = tile_row();  // this thread's row of its tile
    const float *__restrict__ sT = f.t_tab;  // sample distances, read through L1

    constexpr unsigned FULL = 0xffffffffu;
    constexpr int LA = CT ? kLookahead : 1;  // 1: no look-ahead (bounded scenes)
    const int lane = threadIdx.x & 31;
    long long ray = -1, pix = 0;
    bool exhausted = false, ok = true;
    MarchRay mr;
    float r = 0.0f, T = 1.0f, C[3] = {0, 0, 0}, Dp = 0.0f;
    float adj[CT ? 6 : 1];  // contracted scenes: offsets to the adjacent pixels' rays
    bool has_adj = false;
    int n_eval = 0;
    int q[LA];              // look-ahead: ring of the step indices of the samples found ahead
    int qh = 0, nq = 0;     // look-ahead: oldest entry, how many are queued
    bool mend = false;      // look-ahead: the march of this ray has reached its end
    uint32_t phase = 0;
    unsigned st_samples = 0, st_levels = 0, st_steps = 0, st_rays = 0;

    while (true) {
        bool have = false;
        float p[3] = {0, 0, 0};
        // ---- march to the next occupied sample, refilling finished slots ----
        while (true) {
            const bool need = ray < 0 && !exhausted;
            const unsigned m = __ballot_sync(FULL, need);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
                base = __shfl_sync(FULL, base, leader);
                if (need) {
                    const long long slot = (long long)base + __popc(m & ((1u << lane) - 1u));
                    if (slot >= src.n_slots) {
                        exhausted = true;
                    } else if (slot_ray(src, f, slot, mr.o, mr.d, r, pix, CT ? adj : nullptr,
                                        CT ? &has_adj : nullptr)) {
                        march_init(f, mr);
                        ray = slot;
                        n_eval = 0;
                        qh = 0;
                        nq = 0;
                        mend = false;
                        T = 1.0f;
                        Dp = 0.0f;
                        C[0] = C[1] = C[2] = 0.0f;
                    }
                }
            }
            if constexpr (LA == 1) {
                if (ray >= 0 && !have) {
                    const int mres = march_next(f, sT, mr, p, kTcChunk, st_steps);
                    if (mres == MARCH_SAMPLE) {
                        have = true;
                    } else if (mres == MARCH_END) {
                        finish_outputs(out, pix, C, T, n_eval, Dp, nullptr, f.check);
                        ray = -1;
                        ++st_rays;
                    }
                }
                if (__all_sync(FULL, have || exhausted)) break;
            } else {
                for (int it = 0; it < kTcChunk; ++it) {
                    if (!__any_sync(FULL, ray >= 0 && nq == 0)) break;  // every live lane has a sample
                    if (ray >= 0 && !mend && nq < LA) {
                        float pq[3];
                        const int mres = march_next(f, sT, mr, pq, 1, st_steps);
                        if (mres == MARCH_SAMPLE) {
                            q[(qh + nq++) & (LA - 1)] = mr.step;
                            ++mr.step;
                        } else if (mres == MARCH_END) {
                            mend = true;
                            if (nq == 0) {
                                finish_outputs(out, pix, C, T, n_eval, Dp, nullptr, f.check);
                                ray = -1;
                                ++st_rays;
                            }
                        }
                    }
                }
                have = ray >= 0 && nq > 0;
                if (__all_sync(FULL, have || exhausted)) break;
            }
        }
        if (!tile_sync_or(S.bar, have) || *S.abort) break;
        // ---- features, tensor-core MLPs, compositing ----
        float t = 0.0f, delta = 0.0f;
        if (have) {
            int step = mr.step;
            if constexpr (LA > 1) {
                step = q[qh];
                t = sT[step];
#pragma unroll
                for (int k = 0; k < 3; ++k) p[k] = __fadd_rn(mr.o[k], __fmul_rn(t, mr.d[k]));  // as the march
            }
            t = sT[step];
            delta = sT[step + 1] - t;
            float r_norm;
            if constexpr (CT)
                r_norm = footprint(f, t, r, p, has_adj ? adj : nullptr, has_adj ? adj + 3 : nullptr);
            else
                r_norm = t * r * f.inv_ext;
            st_levels += gather_to_tile<L, FMT == 1 ? 1 : 0>(f, p, r_norm, S.act, row);
            ++st_samples;
        } else {
            uint32_t z[D / 2];
#pragma unroll
            for (int k = 0; k < D / 2; ++k) z[k] = 0u;
            store_row<D>(S.act, row, z);
        }
        float sigma, rgb[3];
        tc_mlp_any<D, FMT>(S, nullptr, mr.d, f.density_bias, sigma, rgb, phase, ok);
        if (have) {
            const float sd = sigma * delta;
            const float w = T * (-expm1f(-sd));
            C[0] += w * rgb[0];
            C[1] += w * rgb[1];
            C[2] += w * rgb[2];
            Dp += w * t;
            T *= expf(-sd);
            ++n_eval;
            bool done = T < f.T_eps;
            if constexpr (LA == 1) {
                ++mr.step;
            } else {
                qh = (qh + 1) & (LA - 1);
                --nq;
                done = done || (nq == 0 && mend);
            }
            if (done) {
                finish_outputs(out, pix, C, T, n_eval, Dp, nullptr, f.check);
                ray = -1;
                ++st_rays;
            }
        }
    }
    add_stats(out.stats, st_samples, st_levels, st_steps, st_rays);
    tc_teardown(S, status);
}

template <int L, int FMT>
__global__ void __launch_bounds__(kTcThreads)
query_tc_kernel(const FieldView f, const float *__restrict__ pos, const float *__restrict__ dir,
                const float *__restrict__ radius, int n, float *__restrict__ sigma_out,
                float *__restrict__ rgb_out, float *__restrict__ feat_out, const uint4 *__restrict__ wimg,
                unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *sT;
    const TcShared S = tc_setup<D, FMT>(smem, wimg, sT, nullptr, 0);
    const int i = blockIdx.x * kTcThreads + threadIdx.x;
    const bool valid = i < n;
    float feat[D], dd[3] = {0, 0, 1};
    if (valid) {
        float p[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
        dd[0] = dir[3 * i];
        dd[1] = dir[3 * i + 1];
        dd[2] = dir[3 * i + 2];
        gather_features<L>(f, p, footprint(f, 1.0f, radius[i], p, nullptr, nullptr), feat);
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) feat[k] = 0.0f;
    }
    uint32_t phase = 0;
    bool ok = true;
    float sigma, rgb[3];
    tc_mlp_any<D, FMT>(S, feat, dd, f.density_bias, sigma, rgb, phase, ok);  // query keeps feat for output
    if (valid) {
        sigma_out[i] = sigma;
        for (int c = 0; c < 3; ++c) rgb_out[3 * i + c] = rgb[c];
        if (feat_out)
            for (int k = 0; k < D; ++k) feat_out[(long long)i * D + k] = feat[k];
    }
    tc_teardown(S, status);
}

// fp32 W1..W5 -> the K-major operand image of TcW<D>, fp16 or bf16.
__global__ void build_tc_image_kernel(const float *__restrict__ mlp, int D, int fmt,
                                      unsigned char *__restrict__ img) {
    const int sizes[5][3] = {{64, D, 64}, {16, 64, 16}, {64, 32, 64}, {64, 64, 64}, {16, 64, 3}};
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int off = 0, src = 0;
    for (int m = 0; m < 5; ++m) {
        const int N = sizes[m][0], K = sizes[m][1], rows = sizes[m][2];
        if (e < N * K) {
            const int row = e / K, col = e % K;
            const float v = row < rows ? mlp[src + row * K + col] : 0.0f;
            const int b = off + (row >> 3) * (K >> 3) * 128 + (col >> 3) * 128 + (row & 7) * 16 + (col & 7) * 2;
            if (fmt == 0)
                *reinterpret_cast<__half *>(img + b) = __float2half_rn(v);
            else
                *reinterpret_cast<__nv_bfloat16 *>(img + b) = __float2bfloat16_rn(v);
            return;
        }
        e -= N * K;
        off += N * K * 2;
        src += rows * K;
    }
}

// One CTA waits on an mbarrier that nothing completes; the bounded wait gives
// up after limit_ns, the CTA records the time-out and frees its TMEM.
__global__ void wait_timeout_kernel(unsigned long long limit_ns, unsigned long long *status) {
    __shared__ uint64_t mbar;
    __shared__ uint32_t holder;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&mbar, 1);
        abort_flag = 0;
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&holder, 32);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool ok = tc::mbar_wait_bounded(&mbar, 0u, &abort_flag, limit_ns);
    __syncthreads();
    if (threadIdx.x == 0 && (!ok || abort_flag)) atomicExch(status, (unsigned long long)(-VRNERF_ETIMEDOUT));
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x < 32) tc::tmem_dealloc(holder, 32);
}

// fp32 W1..W5 -> the fp8-mode image (TcW8): W1, W5 fp16; W2..W4 e4m3 with a
// power-of-two scale per matrix (max |w| * s in [128, 256)); one CTA per matrix.
__global__ void build_tc_image_fp8_kernel(const float *__restrict__ mlp, int D, unsigned char *__restrict__ img) {
    const int m = blockIdx.x;
    const int Ns[5] = {64, 16, 64, 64, 16}, Ks[5] = {D, 64, 32, 64, 64}, Rs[5] = {64, 16, 64, 64, 3};
    const int w2 = 64 * D * 2, w3 = w2 + 16 * 64, w4 = w3 + 64 * 32, w5 = w4 + 64 * 64, sc = w5 + 16 * 64 * 2;
    const int offs[5] = {0, w2, w3, w4, w5};
    int src = 0;
    for (int i = 0; i < m; ++i) src += Rs[i] * Ks[i];
    const int N = Ns[m], K = Ks[m], R = Rs[m];
    unsigned char *dst = img + offs[m];
    if (m == 0 || m == 4) {
        for (int e = threadIdx.x; e < N * K; e += blockDim.x) {
            const int row = e / K, col = e % K;
            const float v = row < R ? mlp[src + row * K + col] : 0.0f;
            *reinterpret_cast<__half *>(dst + (row >> 3) * (K >> 3) * 128 + (col >> 3) * 128 + (row & 7) * 16 +
                                        (col & 7) * 2) = __float2half_rn(v);
        }
        return;
    }
    __shared__ float red[256];
    float mx = 0.0f;
    for (int e = threadIdx.x; e < R * K; e += blockDim.x) mx = fmaxf(mx, fabsf(mlp[src + e]));
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + st]);
        __syncthreads();
    }
    float s, inv;
    row_scale(red[0], s, inv);
    for (int e = threadIdx.x; e < N * K; e += blockDim.x) {
        const int row = e / K, col = e % K;
        const float v = row < R ? mlp[src + row * K + col] * s : 0.0f;
        dst[(row >> 3) * (K >> 4) * 128 + (col >> 4) * 128 + (row & 7) * 16 + (col & 15)] =
            (unsigned char)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
    if (threadIdx.x == 0) reinterpret_cast<float *>(img + sc)[m - 1] = inv;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int L, int FMT, bool CT>
static cudaError_t render_tc_ct(vrnerf_field *F, const RaySource &src, const RenderOut &out, cudaStream_t st) {
    constexpr int NT = render_tiles<CT, FMT>();
    const size_t smem = tc_smem_bytes(2 * L, 0, NT);
    auto kern = render_tc_kernel<L, FMT, CT, NT>;
    int bps = 0;
    cudaError_t e = prepare_tc(kern, smem, bps, NT);
    if (e != cudaSuccess) return e;
    long long want = (src.n_slots + kTcThreads * NT - 1) / (kTcThreads * NT);
    long long grid = (long long)num_sms() * bps;
    if (want < grid) grid = want;
    if (grid < 1) grid = 1;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(F->counter);
    kern<<<(unsigned)grid, kTcThreads * NT, smem, st>>>(F->view, src, out, cnt, static_cast<const uint4 *>(F->tc_w),
                                                        cnt + 1);
    return cudaGetLastError();
}

template <int L, int FMT>
static cudaError_t render_tc_t(vrnerf_field *F, const RaySource &src, const RenderOut &out, cudaStream_t st) {
    return F->view.contract ? render_tc_ct<L, FMT, true>(F, src, out, st) : render_tc_ct<L, FMT, false>(F, src, out, st);
}

static int fmt_of(int prec) { return prec == VRNERF_BF16 ? 1 : (prec == VRNERF_FP8 ? 2 : 0); }

cudaError_t launch_render_tc(vrnerf_field *F, const RaySource &src, const RenderOut &out, int prec,
                             cudaStream_t st) {
    if (prec != VRNERF_FP16 && prec != VRNERF_BF16 && prec != VRNERF_FP8) return cudaErrorNotSupported;
    const int fmt = fmt_of(prec);
    cudaError_t e = ensure_tc_image(F, fmt, st);
    if (e != cudaSuccess) return e;
    if (F->view.L == 8)
        return fmt == 1 ? render_tc_t<8, 1>(F, src, out, st)
                        : (fmt == 2 ? render_tc_t<8, 2>(F, src, out, st) : render_tc_t<8, 0>(F, src, out, st));
    return fmt == 1 ? render_tc_t<16, 1>(F, src, out, st)
                    : (fmt == 2 ? render_tc_t<16, 2>(F, src, out, st) : render_tc_t<16, 0>(F, src, out, st));
}

template <int L, int FMT>
static cudaError_t query_tc_t(vrnerf_field *F, const float *pos, const float *dir, const float *radius, int n,
                              float *sigma, float *rgb, float *feat, cudaStream_t st) {
    const size_t smem = tc_smem_bytes(2 * L, 0);
    auto kern = query_tc_kernel<L, FMT>;
    int bps = 0;
    cudaError_t e = prepare_tc(kern, smem, bps);
    if (e != cudaSuccess) return e;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(F->counter);
    kern<<<(n + kTcThreads - 1) / kTcThreads, kTcThreads, smem, st>>>(
        F->view, pos, dir, radius, n, sigma, rgb, feat, static_cast<const uint4 *>(F->tc_w), cnt + 1);
    return cudaGetLastError();
}

cudaError_t launch_query_tc(vrnerf_field *F, const float *pos, const float *dir, const float *radius, int n,
                            float *sigma, float *rgb, float *feat, int prec, cudaStream_t st) {
    if (prec != VRNERF_FP16 && prec != VRNERF_BF16 && prec != VRNERF_FP8) return cudaErrorNotSupported;
    const int fmt = fmt_of(prec);
    cudaError_t e = ensure_tc_image(F, fmt, st);
    if (e != cudaSuccess) return e;
    if (F->view.L == 8)
        return fmt == 1 ? query_tc_t<8, 1>(F, pos, dir, radius, n, sigma, rgb, feat, st)
                        : (fmt == 2 ? query_tc_t<8, 2>(F, pos, dir, radius, n, sigma, rgb, feat, st)
                                    : query_tc_t<8, 0>(F, pos, dir, radius, n, sigma, rgb, feat, st));
    return fmt == 1 ? query_tc_t<16, 1>(F, pos, dir, radius, n, sigma, rgb, feat, st)
                    : (fmt == 2 ? query_tc_t<16, 2>(F, pos, dir, radius, n, sigma, rgb, feat, st)
                                : query_tc_t<16, 0>(F, pos, dir, radius, n, sigma, rgb, feat, st));
}

cudaError_t launch_wait_timeout(vrnerf_field *F, unsigned long long limit_ns, cudaStream_t st) {
    wait_timeout_kernel<<<1, 128, 0, st>>>(limit_ns, reinterpret_cast<unsigned long long *>(F->counter) + 1);
    return cudaGetLastError();
}

}  // namespace vrn

extern "C" int vrnerf_debug_wait_timeout(vrnerf_field *F, uint32_t limit_us, void *stream) {
    if (!F) return vrn::fail(VRNERF_EINVAL, "field is NULL");
    if (limit_us < 1 || limit_us > 2000000) return vrn::fail(VRNERF_EINVAL, "limit_us must be in [1, 2000000]");
    cudaError_t e = vrn::launch_wait_timeout(F, 1000ull * limit_us, (cudaStream_t)stream);
    if (e != cudaSuccess) return vrn::cuda_fail(e, "debug_wait_timeout");
    return VRNERF_OK;
}
