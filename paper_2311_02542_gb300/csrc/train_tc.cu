// train_tc.cu -- the per-sample MLP backward of the training step on tcgen05
// tensor cores, bf16 operands and fp32 accumulation (the mixed-precision
// option of the training path; the fp32 CUDA-core kernel stays the default).
//
// Persistent CTAs (two per SM) walk tiles of 128 samples (row r = thread r):
//  forward recompute   F (bf16 features kept by the forward pass)
//                                              -> L1: H  = relu(F W1^T)
//                                              -> L2: O  = H W2^T
//                      X = [O, SH(d)]          -> L3: H1 = relu(X W3^T)
//                                              -> L4: H2 = relu(H1 W4^T)
//  backward            dH2 = relu'(H2) (dZ W5)         (CUDA cores, 3 x 64)
//                      dW4 += dH2^T H1, dW5 += dZ^T H2, dH1 = relu'(H1) (dH2 W4)
//                      dW3 += dH1^T X,                  dX  = dH1 W3
//                      dO = dX[:16] + e_0 dL/do_0   (dL/dsigma sigma, fp32, from the ray pass)
//                      dW2 += dO^T H,                   dH  = relu'(H) (dO W2)
//                      dW1 += dH^T F,                   dF  = dH W1  -> hash-grid scatter
// Every product is a 128-row MMA on tiles that the epilogues write once, as
// rows ([128 samples][units], 16-byte stores). The forward and data-gradient
// products read them K-major; the weight gradients sum over the samples, so
// they read the same tiles MN-major (A = the delta tile, rows = output units,
// K = samples; B = the input tile), and the data gradients read the forward
// weight image MN-major as W instead of W^T: no transposed copies. dH2 and dZ
// share one [128][80] tile (units 0..63 and 64..66), so one A operand serves
// dW4 and dW5; an MMA's rows past a tile's units read the next rows of shared
// memory and land in TMEM lanes that its result does not use.
// dW1, dW3, dW4 accumulate in TMEM across all tiles of the CTA; dW2 and dW5
// go to one scratch accumulator per tile and are added into fp32 sums in
// shared memory, which keeps the CTA at 256 TMEM columns and ~110 KB of shared
// memory: two CTAs share an SM, so one CTA's epilogues overlap the other's
// MMAs. The sums reach global memory once at the end.
#include "field.h"
#include "tc_mlp.cuh"

namespace vrn {

namespace {

constexpr int kTile = 128;
constexpr int kBwdPerSm = 2;  // resident CTAs per SM (shared memory and TMEM are sized for two)

// Shared-memory carve-up of the backward CTA (bytes). Every MN-major read of
// a delta tile as a 128-row A operand runs past the tile's end by less than
// 1 KB (rows = units beyond the tile's width); the buffer after it absorbs that.
template <int D>
struct BwdSm {
    static constexpr int w = 0;                                     // forward image (bf16)
    static constexpr int F = (TcW<D>::bytes + 1023) & ~1023;        // [128][D]
    static constexpr int H = F + kTile * D * 2;                     // [128][64]: H, then dH
    static constexpr int X = H + kTile * 64 * 2;                    // [128][32]: X, then dO [128][16]
    static constexpr int H1 = X + kTile * 32 * 2;                   // [128][64]: H1, then dH1
    static constexpr int H2 = H1 + kTile * 64 * 2;                  // [128][64]
    static constexpr int G = H2 + kTile * 64 * 2;                   // [128][80]: dH2 | dZ | 0
    static constexpr int acc2 = G + kTile * 80 * 2;                 // fp32 dW2 [16][64]
    static constexpr int acc5 = acc2 + 16 * 64 * 4;                 // fp32 dW5 [3][64]
    static constexpr int w5 = acc5 + 3 * 64 * 4;                    // fp32 W5 [3][64]
    static constexpr int misc = w5 + 3 * 64 * 4;                    // mbarrier, TMEM holder, abort
    static constexpr int bytes = misc + 64;
    // a 128-row MN-major read of a [128][U] tile ends 2048 - (U / 8) * 128 bytes past it
    static_assert(acc5 - acc2 >= 2048 - 80 / 8 * 128, "the overrun of G stays in acc2");
    static_assert(X - H >= 2048 - 64 / 8 * 128 && H2 - H1 >= 2048 - 64 / 8 * 128, "overruns of dH, dH1");
    static_assert(kTile * 32 * 2 >= kTile * 16 * 2 + 2048 - 16 / 8 * 128, "the overrun of dO stays in X");
};

// TMEM columns (256 per CTA, so that two CTAs fit the SM's 512).
constexpr uint32_t kColData = 0;    // data products, 64 columns
constexpr uint32_t kColScr = 64;    // dW5 (lanes 64..66) or dW2 (lanes 0..15) of the current tile
constexpr uint32_t kColW4 = 128;    // lanes 0..63 x 64
constexpr uint32_t kColW1 = 192;    // lanes 0..63 x D (D <= 32)
constexpr uint32_t kColW3 = 224;    // lanes 0..63 x 32
constexpr uint32_t kBwdCols = 256;

// One operand of an MMA: start address, descriptor strides and the byte step
// to the next 16 values of K.
struct Opnd {
    uint32_t addr, lbo, sbo, kstep;
    bool mn;
};

// Tile [rows][U] (16-bit elements, row length U) read K-major: K runs along U.
__device__ __forceinline__ Opnd kmaj(uint32_t addr, int U) {
    return {addr, 128u, (uint32_t)(U / 8) * 128u, 256u, false};
}
// The same tile read MN-major: K runs along its rows, M or N along U.
__device__ __forceinline__ Opnd mnmaj(uint32_t addr, int U) {
    const uint32_t g = (uint32_t)(U / 8) * 128u;
    return {addr, g, 128u, 2u * g, true};
}

// D[tmem] (+)= A[128 x K] * B[K x N], K a multiple of 16.
template <int K, int N>
__device__ __forceinline__ void issue(const Opnd &a, const Opnd &b, uint32_t d, bool acc) {
    const uint32_t idesc = tc::idesc_f16(N, 1) | tc::idesc_mn(a.mn, b.mn);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
        tc::mma_f16(d, tc::smem_desc(a.addr + ks * a.kstep, a.lbo, a.sbo),
                    tc::smem_desc(b.addr + ks * b.kstep, b.lbo, b.sbo), idesc, (ks > 0 || acc) ? 1u : 0u);
}

// Row r, units 8j..8j+7 of a [128][U] tile: one 16-byte store of bf16 values.
__device__ __forceinline__ void store8(unsigned char *tile, int U, int r, int j, const float *v) {
    uint4 w;
    uint32_t *p = &w.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
        p[e] = *reinterpret_cast<const uint32_t *>(&b);
    }
    *reinterpret_cast<uint4 *>(tile + (r >> 3) * (U / 8) * 128 + j * 128 + (r & 7) * 16) = w;
}

struct Sync {
    uint64_t *mbar;
    volatile int *abort;
    uint32_t phase;
};

// Shared-memory operands written by this CTA -> tensor core; thread 0 issues
// the batch `issue`, commits, and every thread waits (bounded) for it. A wait
// that runs out sets s.abort; control flow stays the same for every thread
// (the tile loop checks the flag CTA-wide).
template <typename F>
__device__ __forceinline__ void mma_batch(Sync &s, F issue_fn) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        issue_fn();
        tc::mma_commit(s.mbar);
    }
    tc::mbar_wait_bounded(s.mbar, s.phase, s.abort);
    s.phase ^= 1u;
    tc::fence_after_sync();
}

__device__ __forceinline__ void tmem_row(uint32_t taddr, int ncols, float *v) {
    for (int c = 0; c < ncols; c += 16) {
        float t[16];
        tc::tmem_ld16(taddr + c, t);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[c + i] = t[i];
    }
}

// Adds this tile's scratch accumulator (lanes lo..lo+n-1, 64 columns) into
// the CTA's fp32 sums; called by the warp that owns those TMEM lanes.
__device__ __forceinline__ void drain_scratch(uint32_t lane_addr, int r, int lo, int n, float *sum) {
    float s[64];
    tmem_row(lane_addr + kColScr, 64, s);
    if (r >= lo && r < lo + n) {
        float *row = sum + (r - lo) * 64;
#pragma unroll
        for (int k = 0; k < 64; ++k) row[k] += s[k];
    }
}

}  // namespace

template <int L>
__global__ void __launch_bounds__(kTile, kBwdPerSm)
bwd_tc_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
              const float *__restrict__ r_in, const int2 *__restrict__ rec, const long long *__restrict__ off,
              const int *__restrict__ n_used, long long n_samples, const float4 *__restrict__ grad_s,
              const uint4 *__restrict__ feat_in, const uint4 *__restrict__ wimg, float4 *__restrict__ dfeat_out,
              float *__restrict__ mlp_grad, unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    using M = BwdSm<D>;
    using W = TcW<D>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int r = threadIdx.x, warp = r >> 5;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + M::misc);
    uint32_t *holder = reinterpret_cast<uint32_t *>(smem + M::misc + 8);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + M::misc + 12);
    float *acc2 = reinterpret_cast<float *>(smem + M::acc2);
    float *acc5 = reinterpret_cast<float *>(smem + M::acc5);
    float *w5 = reinterpret_cast<float *>(smem + M::w5);
    const float *W5 = f.mlp + 64 * D + 16 * 64 + 64 * 32 + 64 * 64;
    for (int i = r; i < W::bytes / 16; i += kTile) reinterpret_cast<uint4 *>(smem + M::w)[i] = wimg[i];
    for (int i = r; i < 16 * 64 + 3 * 64; i += kTile) acc2[i] = 0.0f;  // acc2 and acc5 are adjacent
    for (int i = r; i < 3 * 64; i += kTile) w5[i] = W5[i];
    if (r == 0) {
        tc::mbar_init(mbar, 1);
        *abort = 0;
    }
    if (r < 32) {
        tc::tmem_alloc(holder, kBwdCols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *holder;
    const uint32_t lane_addr = tbase + ((uint32_t)(r & ~31) << 16);
    Sync sy{mbar, abort, 0u};
    const uint32_t s0 = tc::smem_u32(smem);
    unsigned char *tF = smem + M::F, *tH = smem + M::H, *tX = smem + M::X, *tH1 = smem + M::H1;
    unsigned char *tH2 = smem + M::H2, *tG = smem + M::G;
    // operands: activation and delta tiles, and the forward weight image read as W (MN-major)
    const Opnd F_k = kmaj(s0 + M::F, D), F_mn = mnmaj(s0 + M::F, D);
    const Opnd H_k = kmaj(s0 + M::H, 64), H_mn = mnmaj(s0 + M::H, 64);
    const Opnd X_k = kmaj(s0 + M::X, 32), X_mn = mnmaj(s0 + M::X, 32);
    const Opnd dO_k = kmaj(s0 + M::X, 16), dO_mn = mnmaj(s0 + M::X, 16);
    const Opnd H1_k = kmaj(s0 + M::H1, 64), H1_mn = mnmaj(s0 + M::H1, 64);
    const Opnd H2_mn = mnmaj(s0 + M::H2, 64);
    const Opnd G_k = kmaj(s0 + M::G, 80), G_mn = mnmaj(s0 + M::G, 80);
    const uint32_t wb = s0 + M::w;
    const Opnd W1_k = kmaj(wb + W::w1, D), W2_k = kmaj(wb + W::w2, 64), W3_k = kmaj(wb + W::w3, 32),
               W4_k = kmaj(wb + W::w4, 64);
    const Opnd W1_mn = mnmaj(wb + W::w1, D), W2_mn = mnmaj(wb + W::w2, 64), W3_mn = mnmaj(wb + W::w3, 32),
               W4_mn = mnmaj(wb + W::w4, 64);
    bool acc = false;  // TMEM weight-gradient accumulators hold this CTA's sums

    const long long tiles = (n_samples + kTile - 1) / kTile;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        if (__syncthreads_or(*abort)) break;
        const long long i = tile * kTile + r;
        bool have = false;
        float dir[3] = {0.0f, 0.0f, 1.0f}, dsig = 0.0f, dz[3] = {0, 0, 0};
        if (i < n_samples) {
            const int2 q = rec[i];
            const long long b = q.x;
            if (i - off[b] < n_used[b]) {
                have = true;
                dir[0] = d_in[3 * b];
                dir[1] = d_in[3 * b + 1];
                dir[2] = d_in[3 * b + 2];
                const float4 gs = grad_s[i];
                dsig = gs.x;
                dz[0] = gs.y;
                dz[1] = gs.z;
                dz[2] = gs.w;
            }
        }
        // ---- features (bf16 rows, kept by the forward pass) ----
#pragma unroll
        for (int k = 0; k < D / 8; ++k) {
            const uint4 w = have ? __ldg(feat_in + i * (D / 8) + k) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(tF + (r >> 3) * (D / 8) * 128 + k * 128 + (r & 7) * 16) = w;
        }
        // ---- L1: H = relu(F W1^T) ----
        mma_batch(sy, [&] { issue<D, 64>(F_k, W1_k, tbase + kColData, false); });
        uint64_t m0 = 0, m1 = 0;  // ReLU masks of H, H1
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                v[k] = fmaxf(v[k], 0.0f);
                if (v[k] > 0.0f) m0 |= 1ull << k;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) store8(tH, 64, r, j, v + 8 * j);
        }
        // ---- L2: O = H W2^T; X = [O, SH(d)] ----
        mma_batch(sy, [&] { issue<64, 16>(H_k, W2_k, tbase + kColData, false); });
        {
            float x[32];
            tmem_row(lane_addr + kColData, 16, x);
            sh16(dir[0], dir[1], dir[2], x + 16);
#pragma unroll
            for (int j = 0; j < 4; ++j) store8(tX, 32, r, j, x + 8 * j);
        }
        // ---- L3: H1 = relu(X W3^T) ----
        mma_batch(sy, [&] { issue<32, 64>(X_k, W3_k, tbase + kColData, false); });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                v[k] = fmaxf(v[k], 0.0f);
                if (v[k] > 0.0f) m1 |= 1ull << k;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) store8(tH1, 64, r, j, v + 8 * j);
        }
        // ---- L4: H2 = relu(H1 W4^T); dH2 = relu'(H2) (dZ W5) and dZ into G ----
        mma_batch(sy, [&] { issue<64, 64>(H1_k, W4_k, tbase + kColData, false); });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float h[8], g[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = 8 * j + e;
                    h[e] = fmaxf(v[k], 0.0f);
                    const float a = w5[k] * dz[0] + w5[64 + k] * dz[1] + w5[128 + k] * dz[2];
                    g[e] = h[e] > 0.0f ? a : 0.0f;
                }
                store8(tH2, 64, r, j, h);
                store8(tG, 80, r, j, g);
            }
            const float z8[8] = {dz[0], dz[1], dz[2], 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            const float zero[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            store8(tG, 80, r, 8, z8);
            store8(tG, 80, r, 9, zero);
        }
        // ---- dW4 += dH2^T H1, dW5 = dZ^T H2 (scratch), dH1 = dH2 W4 ----
        mma_batch(sy, [&] {
            issue<kTile, 64>(G_mn, H1_mn, tbase + kColW4, acc);
            issue<kTile, 64>(G_mn, H2_mn, tbase + kColScr, false);
            issue<64, 64>(G_k, W4_mn, tbase + kColData, false);
        });
        if (warp == 2) drain_scratch(lane_addr, r, 64, 3, acc5);
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = (m1 >> k) & 1ull ? v[k] : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) store8(tH1, 64, r, j, v + 8 * j);  // dH1
        }
        // ---- dW3 += dH1^T X, dX = dH1 W3 (its first 16 columns: dO) ----
        mma_batch(sy, [&] {
            issue<kTile, 32>(H1_mn, X_mn, tbase + kColW3, acc);
            issue<64, 16>(H1_k, W3_mn, tbase + kColData, false);
        });
        {
            float v[16];
            tmem_row(lane_addr + kColData, 16, v);
            v[0] += dsig;  // dL/do_0 = dL/dsigma * sigma, from the ray pass (fp32)
            store8(tX, 16, r, 0, v);
            store8(tX, 16, r, 1, v + 8);  // dO as a [128][16] tile
        }
        // ---- dW2 = dO^T H (scratch), dH = dO W2 ----
        mma_batch(sy, [&] {
            issue<kTile, 64>(dO_mn, H_mn, tbase + kColScr, false);
            issue<16, 64>(dO_k, W2_mn, tbase + kColData, false);
        });
        if (warp == 0) drain_scratch(lane_addr, r, 0, 16, acc2);
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = (m0 >> k) & 1ull ? v[k] : 0.0f;
#pragma unroll
            for (int j = 0; j < 8; ++j) store8(tH, 64, r, j, v + 8 * j);  // dH
        }
        // ---- dW1 += dH^T F, dF = dH W1 ----
        mma_batch(sy, [&] {
            issue<kTile, D>(H_mn, F_mn, tbase + kColW1, acc);
            issue<64, D>(H_k, W1_mn, tbase + kColData, false);
        });
        acc = true;
        {  // dL/dfeatures (fp32) for the grid scatter; the TMEM load is warp-wide
            float dfeat[D];
            tmem_row(lane_addr + kColData, D, dfeat);
            if (have) {
#pragma unroll
                for (int k = 0; k < D / 4; ++k)
                    dfeat_out[i * (D / 4) + k] =
                        make_float4(dfeat[4 * k], dfeat[4 * k + 1], dfeat[4 * k + 2], dfeat[4 * k + 3]);
            }
        }
        tc::fence_before_sync();  // this tile's TMEM reads precede the next tile's MMAs
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // ---- weight gradients: TMEM lane = output unit -> global [out][in] ----
    if (acc && !*abort) {
        float *g1 = mlp_grad, *g2 = g1 + 64 * D, *g3 = g2 + 16 * 64, *g4 = g3 + 64 * 32, *g5 = g4 + 64 * 64;
        float v[64];
        tmem_row(lane_addr + kColW4, 64, v);
        if (r < 64)
            for (int k = 0; k < 64; ++k) atomicAdd(g4 + r * 64 + k, v[k]);
        tmem_row(lane_addr + kColW1, D, v);
        if (r < 64)
            for (int k = 0; k < D; ++k) atomicAdd(g1 + r * D + k, v[k]);
        tmem_row(lane_addr + kColW3, 32, v);
        if (r < 64)
            for (int k = 0; k < 32; ++k) atomicAdd(g3 + r * 32 + k, v[k]);
        for (int e = r; e < 16 * 64; e += kTile) atomicAdd(g2 + e, acc2[e]);
        for (int e = r; e < 3 * 64; e += kTile) atomicAdd(g5 + e, acc5[e]);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (r == 0 && *abort && status) atomicExch(status, (unsigned long long)(-VRNERF_ETIMEDOUT));
    if (r < 32) tc::tmem_dealloc(tbase, kBwdCols);
}

// Grid-gradient scatter after either backward kernel: one thread per sample
// (consecutive samples in a warp, so the dense-level runs still merge), at
// full occupancy so that the atomics' latency is hidden; dL/dfeatures come
// from the backward kernel in fp32. The levels are taken in groups of LG,
// blockIdx.y = group: blocks start in linear order, so the whole batch
// scatters into one group's levels before the next group's blocks run, and
// the fp32 gradient lines of those levels (16 MB per hashed level) stay in L2
// under the atomics instead of every sample touching all L levels at once.
// Each group recomputes the sample's position and footprint.
template <int L, int LG>
__global__ void __launch_bounds__(128)
grid_scatter_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                    const float *__restrict__ r_in, const int2 *__restrict__ rec, const long long *__restrict__ off,
                    const int *__restrict__ n_used, long long n, const float4 *__restrict__ dfeat_in,
                    float *__restrict__ grid_grad) {
    constexpr int D = 2 * L;
    static_assert(L % LG == 0 && LG % 2 == 0, "levels split into groups of whole float4s");
    const int l0 = blockIdx.y * LG;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // uniform per block
        const long long i = i0 + threadIdx.x;
        bool have = false;
        float p[3] = {0.0f, 0.0f, 0.0f}, rn = 0.0f, dfeat[2 * LG];
        if (i < n) {
            const int2 q = rec[i];
            const long long b = q.x;
            if (i - off[b] < n_used[b]) {
                have = true;
                const float o[3] = {o_in[3 * b], o_in[3 * b + 1], o_in[3 * b + 2]};
                const float d[3] = {d_in[3 * b], d_in[3 * b + 1], d_in[3 * b + 2]};
                const float t = f.t_tab[q.y];
                int vox;
                sample_voxel(f, o, d, t, p, vox);
                rn = footprint(f, t, r_in[b], p, nullptr, nullptr);
            }
        }
#pragma unroll
        for (int k = 0; k < LG / 2; ++k) {  // read once: streaming loads leave L2 to the gradient
            const float4 v = have ? __ldcs(dfeat_in + i * (D / 4) + l0 / 2 + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dfeat[4 * k] = v.x;
            dfeat[4 * k + 1] = v.y;
            dfeat[4 * k + 2] = v.z;
            dfeat[4 * k + 3] = v.w;
        }
        scatter_grid_grad<LG>(f, p, rn, dfeat, have, grid_grad, l0);
    }
}

// Sample forward of the bf16 training precision: one thread per sample of a
// 128-sample tile gathers its features straight into the bf16 operand tile
// (kept in global memory for the backward) and the tile runs the MLPs on the
// tensor cores; sigma and PQ colour per sample. Like the render kernel, a
// CTA runs kFwdTiles tiles (one per 4-warp group, each with its own tiles of
// the batch) that share one weight image, two CTAs per SM.
constexpr int kFwdTiles = 4;

template <int L, int NT>
__global__ void __launch_bounds__(kTcThreads * NT, NT == 4 ? 2 : kTcMinBlocks / NT)
sample_fwd_tc_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                     const float *__restrict__ r_in, const int2 *__restrict__ rec, long long n,
                     float4 *__restrict__ sc, uint4 *__restrict__ feat_out, const uint4 *__restrict__ wimg,
                     unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *unused;
    const TcShared S = tc_setup<D, 1, NT>(smem, wimg, unused, nullptr, 0);
    const int r = tile_row();
    const int g = NT == 1 ? 0 : (int)(threadIdx.x >> 7);
    uint32_t phase = 0;
    bool ok = true;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    for (long long tile = (long long)blockIdx.x * NT + g; tile < tiles; tile += (long long)gridDim.x * NT) {
        if (tile_sync_or(S.bar, *S.abort != 0)) break;
        const long long i = tile * kTcThreads + r;
        const bool have = i < n;
        float dir[3] = {0.0f, 0.0f, 1.0f};
        if (have) {
            const int2 q = rec[i];
            const long long b = q.x;
            const float o[3] = {o_in[3 * b], o_in[3 * b + 1], o_in[3 * b + 2]};
            dir[0] = d_in[3 * b];
            dir[1] = d_in[3 * b + 1];
            dir[2] = d_in[3 * b + 2];
            const float t = f.t_tab[q.y];
            float p[3];
            int vox;
            sample_voxel(f, o, dir, t, p, vox);
            gather_to_tile<L, 1>(f, p, footprint(f, t, r_in[b], p, nullptr, nullptr), S.act, r);
            const unsigned char *row = S.act + (r >> 3) * (D / 8) * 128 + (r & 7) * 16;
#pragma unroll
            for (int j = 0; j < D / 8; ++j) feat_out[i * (D / 8) + j] = *reinterpret_cast<const uint4 *>(row + j * 128);
        } else {
            uint32_t z[D / 2];
#pragma unroll
            for (int k = 0; k < D / 2; ++k) z[k] = 0u;
            store_row<D>(S.act, r, z);
        }
        float sigma, rgb[3];
        tc_mlp_any<D, 1>(S, nullptr, dir, f.density_bias, sigma, rgb, phase, ok);
        if (have) sc[i] = make_float4(sigma, rgb[0], rgb[1], rgb[2]);
    }
    tc_teardown(S, status);
}

// bf16 weight image of the tensor-core training kernels (the forward image;
// the backward reads it MN-major for the data gradients), rebuilt when the
// fp32 weights change.
static cudaError_t ensure_bwd_images(vrnerf_field *F, cudaStream_t st) {
    const int D = F->view.d_in;
    const size_t fwd = (size_t)(64 * D * 2 + 16 * 64 * 2 + 64 * 32 * 2 + 64 * 64 * 2 + 16 * 64 * 2);
    if (F->tcb_w && F->tcb_version == F->mlp_version) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!F->tcb_w && (e = cudaMalloc(&F->tcb_w, fwd)) != cudaSuccess) return e;
    unsigned char *img = static_cast<unsigned char *>(F->tcb_w);
    build_tc_image_kernel<<<(int)((fwd / 2 + 255) / 256), 256, 0, st>>>(F->mlp, D, 1, img);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    F->tcb_version = F->mlp_version;
    return cudaSuccess;
}

template <int L>
static cudaError_t launch_bwd_tc_t(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                                   const long long *off, const int *n_used, long long n, const float4 *grad_s,
                                   const uint4 *feat, float4 *dfeat, cudaStream_t st) {
    constexpr int D = 2 * L;
    cudaError_t e = ensure_bwd_images(F, st);
    if (e != cudaSuccess) return e;
    const size_t smem = BwdSm<D>::bytes;
    auto kern = bwd_tc_kernel<L>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    // resident CTAs per SM from registers, shared memory and TMEM (kBwdCols
    // of the SM's 512 columns per CTA), at most kBwdPerSm
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    int dev = 0, regs_sm = 65536, smem_sm = 233472;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int by_regs = regs_sm / (((fa.numRegs + 7) / 8) * 8 * kTile);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    int per_sm = by_regs < by_smem ? by_regs : by_smem;
    if (per_sm > (int)(512 / kBwdCols)) per_sm = (int)(512 / kBwdCols);
    per_sm = per_sm < 1 ? 1 : (per_sm > kBwdPerSm ? kBwdPerSm : per_sm);
    const long long tiles = (n + kTile - 1) / kTile, cap = (long long)num_sms() * per_sm;
    const int grid = (int)(tiles < cap ? tiles : cap);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    kern<<<grid, kTile, smem, st>>>(F->view, o, d, r, rec, off, n_used, n, grad_s, feat,
                                    static_cast<const uint4 *>(F->tcb_w), dfeat, F->mlp_grad, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_grid_scatter(F, o, d, r, rec, off, n_used, n, dfeat, st);
}

#ifndef VRN_SCATTER_LEVELS
#define VRN_SCATTER_LEVELS 8  // levels per group of the grid-gradient scatter
#endif

template <int L>
static cudaError_t launch_grid_scatter_t(vrnerf_field *F, const float *o, const float *d, const float *r,
                                         const int2 *rec, const long long *off, const int *n_used, long long n,
                                         const float4 *dfeat, cudaStream_t st) {
    constexpr int LG = VRN_SCATTER_LEVELS < L ? VRN_SCATTER_LEVELS : L;
    auto kern = grid_scatter_kernel<L, LG>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0);
    if (e != cudaSuccess) return e;
    const long long blocks = (n + 127) / 128, cap = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    const dim3 grid((unsigned)(blocks < cap ? blocks : cap), L / LG);
    kern<<<grid, 128, 0, st>>>(F->view, o, d, r, rec, off, n_used, n, dfeat, F->grid_grad);
    return cudaGetLastError();
}

cudaError_t launch_grid_scatter(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                                const long long *off, const int *n_used, long long n, const float4 *dfeat,
                                cudaStream_t st) {
    return F->view.L == 8 ? launch_grid_scatter_t<8>(F, o, d, r, rec, off, n_used, n, dfeat, st)
                          : launch_grid_scatter_t<16>(F, o, d, r, rec, off, n_used, n, dfeat, st);
}

template <int L>
static cudaError_t launch_fwd_tc_t(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                                   long long n, float4 *sc, uint4 *feat, cudaStream_t st) {
    constexpr int D = 2 * L;
    cudaError_t e = ensure_bwd_images(F, st);
    if (e != cudaSuccess) return e;
    constexpr int NT = kFwdTiles;
    const size_t smem = tc_smem_bytes(D, 0, NT);
    auto kern = sample_fwd_tc_kernel<L, NT>;
    int bps = 0;
    if ((e = prepare_tc(kern, smem, bps, NT)) != cudaSuccess) return e;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads, cap = (long long)num_sms() * bps;
    const long long want = (tiles + NT - 1) / NT;
    const int grid = (int)(want < cap ? (want < 1 ? 1 : want) : cap);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    kern<<<grid, kTcThreads * NT, smem, st>>>(F->view, o, d, r, rec, n, sc, feat,
                                              reinterpret_cast<const uint4 *>(F->tcb_w), status);
    return cudaGetLastError();
}

cudaError_t launch_fwd_tc(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                          long long n, float4 *sc, uint4 *feat, cudaStream_t st) {
    return F->view.L == 8 ? launch_fwd_tc_t<8>(F, o, d, r, rec, n, sc, feat, st)
                          : launch_fwd_tc_t<16>(F, o, d, r, rec, n, sc, feat, st);
}

cudaError_t launch_bwd_tc(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                          const long long *off, const int *n_used, long long n, const float4 *grad_s,
                          const uint4 *feat, float4 *dfeat, cudaStream_t st) {
    return F->view.L == 8 ? launch_bwd_tc_t<8>(F, o, d, r, rec, off, n_used, n, grad_s, feat, dfeat, st)
                          : launch_bwd_tc_t<16>(F, o, d, r, rec, off, n_used, n, grad_s, feat, dfeat, st);
}

}  // namespace vrn
