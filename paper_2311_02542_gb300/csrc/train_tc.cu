// train_tc.cu -- the per-sample MLP backward of the training step on tcgen05
// tensor cores, bf16 operands and fp32 accumulation (the mixed-precision
// option of the training path; the fp32 CUDA-core kernel stays the default).
//
// One persistent CTA per SM walks tiles of 128 samples (row r = thread r):
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
// Every product is a 128-row MMA: the data gradients take the activations'
// row tiles as A and a transposed weight image as B; the weight gradients
// sum over the tile's samples, so their A is the delta tile transposed (rows
// = output units, K = the 128 samples) and their B the input tile
// transposed, both written by the epilogues as columns. The weight gradients
// accumulate in TMEM across all tiles of the CTA and are added to global
// memory once at the end. The transposed deltas of one batch share one
// buffer (dH2^T in rows 0..63, dZ^T in rows 64..66): an MMA's rows that
// belong to another product land in TMEM lanes its result does not use.
#include "field.h"
#include "tc_mlp.cuh"

namespace vrn {

namespace {

constexpr int kTile = 128;

// Transposed weight image (K-major B operands of the data-gradient MMAs):
// W4^T [64 in][64 out], W3^T [32 in][64 out], W2^T [64 in][16 out], W1^T [D][64].
template <int D>
struct TcWT {
    static constexpr int w4 = 0;
    static constexpr int w3 = w4 + 64 * 64 * 2;
    static constexpr int w2 = w3 + 32 * 64 * 2;
    static constexpr int w1 = w2 + 64 * 16 * 2;
    static constexpr int bytes = w1 + D * 64 * 2;
};

// Shared-memory carve-up of the backward CTA (bytes).
template <int D>
struct BwdSm {
    static constexpr int w = 0;                                        // forward image (bf16)
    static constexpr int wt = (TcW<D>::bytes + 1023) & ~1023;          // transposed image
    static constexpr int F = (wt + TcWT<D>::bytes + 1023) & ~1023;     // [128][D]
    static constexpr int FT = F + kTile * D * 2;                        // [D][128]
    static constexpr int H = FT + D * kTile * 2;                        // [128][64]: H, dH2, dH
    static constexpr int HT = H + kTile * 64 * 2;                       // [64][128]
    static constexpr int X = HT + 64 * kTile * 2;                       // [128][32]: X, dO [128][16]
    static constexpr int XT = X + kTile * 32 * 2;                       // [32][128]
    static constexpr int H1 = XT + 32 * kTile * 2;                      // [128][64]: H1, dH1
    static constexpr int H1T = H1 + kTile * 64 * 2;                     // [64][128]
    static constexpr int H2T = H1T + 64 * kTile * 2;                    // [64][128]
    static constexpr int AT = H2T + 64 * kTile * 2;                     // [128][128] transposed deltas
    static constexpr int misc = AT + kTile * kTile * 2;                 // mbarrier, TMEM holder, abort
    static constexpr int bytes = misc + 64;
};

// TMEM columns: the data products' accumulator and the weight gradients.
constexpr uint32_t kColData = 0;    // 64 columns
constexpr uint32_t kColW4 = 64;     // lanes 0..63  x 64
constexpr uint32_t kColW2 = 128;    // lanes 0..15  x 64
constexpr uint32_t kColW5 = 192;    // lanes 64..66 x 64
constexpr uint32_t kColW1 = 256;    // lanes 0..63  x D
constexpr uint32_t kColW3 = 288;    // lanes 0..63  x 32
constexpr uint32_t kBwdCols = 512;

__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// element (row, col) of a K-major [rows][K] 16-bit tile
__device__ __forceinline__ void put16(unsigned char *tile, int row, int col, int K, uint16_t v) {
    *reinterpret_cast<uint16_t *>(tile + tc::kmajor_offset(row, col, K)) = v;
}

// D[tmem] (+)= A[128 x K] * B[N x K]^T, both K-major in shared memory.
template <int K, int N>
__device__ __forceinline__ void issue_mma(uint32_t a, uint32_t b, uint32_t d, bool acc) {
    constexpr uint32_t sbo = (K / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_f16(N, 1);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
        tc::mma_f16(d, tc::smem_desc(a + ks * 256, 128, sbo), tc::smem_desc(b + ks * 256, 128, sbo), idesc,
                    (ks > 0 || acc) ? 1u : 0u);
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
__device__ __forceinline__ void mma_batch(Sync &s, F issue) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        issue();
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

}  // namespace

template <int L>
__global__ void __launch_bounds__(kTile, 1)
bwd_tc_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
              const float *__restrict__ r_in, const int2 *__restrict__ rec, const long long *__restrict__ off,
              const int *__restrict__ n_used, long long n_samples, const float4 *__restrict__ grad_s,
              const uint4 *__restrict__ feat_in, const uint4 *__restrict__ wimg, const uint4 *__restrict__ wtimg,
              float4 *__restrict__ dfeat_out,
              float *__restrict__ mlp_grad, unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    using M = BwdSm<D>;
    using W = TcW<D>;
    using WT = TcWT<D>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int r = threadIdx.x;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + M::misc);
    uint32_t *holder = reinterpret_cast<uint32_t *>(smem + M::misc + 8);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + M::misc + 12);
    for (int i = r; i < W::bytes / 16; i += kTile) reinterpret_cast<uint4 *>(smem + M::w)[i] = wimg[i];
    for (int i = r; i < WT::bytes / 16; i += kTile) reinterpret_cast<uint4 *>(smem + M::wt)[i] = wtimg[i];
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
    unsigned char *tF = smem + M::F, *tFT = smem + M::FT, *tH = smem + M::H, *tHT = smem + M::HT;
    unsigned char *tX = smem + M::X, *tXT = smem + M::XT, *tH1 = smem + M::H1, *tH1T = smem + M::H1T;
    unsigned char *tH2T = smem + M::H2T, *tAT = smem + M::AT;
    const float *W5 = f.mlp + 64 * D + 16 * 64 + 64 * 32 + 64 * 64;
    bool acc = false;  // weight-gradient accumulators hold this CTA's sums

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
        // ---- features (bf16, kept by the forward pass): F row and F^T column ----
#pragma unroll
        for (int k = 0; k < D / 8; ++k) {
            const uint4 w = have ? __ldg(feat_in + i * (D / 8) + k) : make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(tF + tc::kmajor_offset(r, 8 * k, D)) = w;  // one core-matrix row
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) put16(tFT, 8 * k + j, r, kTile, (uint16_t)(ws[j >> 1] >> (16 * (j & 1))));
        }
        // ---- L1: H = relu(F W1^T) ----
        mma_batch(sy, [&] { issue_mma<D, 64>(s0 + M::F, s0 + M::w + W::w1, tbase + kColData, false); });
        uint64_t m0 = 0, m1 = 0, m2 = 0;  // ReLU masks of H, H1, H2
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const float h = fmaxf(v[k], 0.0f);
                if (h > 0.0f) m0 |= 1ull << k;
                const uint16_t b = bf16_bits(h);
                put16(tH, r, k, 64, b);
                put16(tHT, k, r, kTile, b);
            }
        }
        // ---- L2: O = H W2^T ----
        mma_batch(sy, [&] { issue_mma<64, 16>(s0 + M::H, s0 + M::w + W::w2, tbase + kColData, false); });
        {
            float o[16], sh[16];
            tmem_row(lane_addr + kColData, 16, o);
            sh16(dir[0], dir[1], dir[2], sh);
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const uint16_t b = bf16_bits(k < 16 ? o[k] : sh[k - 16]);
                put16(tX, r, k, 32, b);
                put16(tXT, k, r, kTile, b);
            }
        }
        // ---- L3: H1 = relu(X W3^T) ----
        mma_batch(sy, [&] { issue_mma<32, 64>(s0 + M::X, s0 + M::w + W::w3, tbase + kColData, false); });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const float h = fmaxf(v[k], 0.0f);
                if (h > 0.0f) m1 |= 1ull << k;
                const uint16_t b = bf16_bits(h);
                put16(tH1, r, k, 64, b);
                put16(tH1T, k, r, kTile, b);
            }
        }
        // ---- L4: H2 = relu(H1 W4^T); dH2 = relu'(H2) (dZ W5), dZ^T, dH2^T ----
        mma_batch(sy, [&] { issue_mma<64, 64>(s0 + M::H1, s0 + M::w + W::w4, tbase + kColData, false); });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const float h = fmaxf(v[k], 0.0f);
                if (h > 0.0f) m2 |= 1ull << k;
                put16(tH2T, k, r, kTile, bf16_bits(h));
                const float a = __ldg(W5 + k) * dz[0] + __ldg(W5 + 64 + k) * dz[1] + __ldg(W5 + 128 + k) * dz[2];
                const uint16_t g = bf16_bits(h > 0.0f ? a : 0.0f);
                put16(tH, r, k, 64, g);  // dH2 (H itself is no longer an operand)
                put16(tAT, k, r, kTile, g);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) put16(tAT, 64 + c, r, kTile, bf16_bits(dz[c]));
        }
        // ---- dW4 += dH2^T H1, dW5 += dZ^T H2, dH1 = dH2 W4 ----
        mma_batch(sy, [&] {
                issue_mma<kTile, 64>(s0 + M::AT, s0 + M::H1T, tbase + kColW4, acc);
                issue_mma<kTile, 64>(s0 + M::AT, s0 + M::H2T, tbase + kColW5, acc);
                issue_mma<64, 64>(s0 + M::H, s0 + M::wt + WT::w4, tbase + kColData, false);
        });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const uint16_t g = bf16_bits((m1 >> k) & 1ull ? v[k] : 0.0f);
                put16(tH1, r, k, 64, g);  // dH1
                put16(tAT, k, r, kTile, g);
            }
        }
        // ---- dW3 += dH1^T X, dX = dH1 W3 ----
        mma_batch(sy, [&] {
                issue_mma<kTile, 32>(s0 + M::AT, s0 + M::XT, tbase + kColW3, acc);
                issue_mma<64, 32>(s0 + M::H1, s0 + M::wt + WT::w3, tbase + kColData, false);
        });
        {
            float v[16];
            tmem_row(lane_addr + kColData, 16, v);
            v[0] += dsig;  // dL/do_0 = dL/dsigma * sigma, from the ray pass (fp32)
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const uint16_t g = bf16_bits(v[k]);
                put16(tX, r, k, 16, g);  // dO as a [128][16] operand
                put16(tAT, k, r, kTile, g);
            }
        }
        // ---- dW2 += dO^T H, dH = dO W2 ----
        mma_batch(sy, [&] {
                issue_mma<kTile, 64>(s0 + M::AT, s0 + M::HT, tbase + kColW2, acc);
                issue_mma<16, 64>(s0 + M::X, s0 + M::wt + WT::w2, tbase + kColData, false);
        });
        {
            float v[64];
            tmem_row(lane_addr + kColData, 64, v);
#pragma unroll
            for (int k = 0; k < 64; ++k) {
                const uint16_t g = bf16_bits((m0 >> k) & 1ull ? v[k] : 0.0f);
                put16(tH, r, k, 64, g);  // dH
                put16(tAT, k, r, kTile, g);
            }
        }
        // ---- dW1 += dH^T F, dF = dH W1 ----
        mma_batch(sy, [&] {
                issue_mma<kTile, D>(s0 + M::AT, s0 + M::FT, tbase + kColW1, acc);
                issue_mma<64, D>(s0 + M::H, s0 + M::wt + WT::w1, tbase + kColData, false);
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
        tmem_row(lane_addr + kColW2, 64, v);
        if (r < 16)
            for (int k = 0; k < 64; ++k) atomicAdd(g2 + r * 64 + k, v[k]);
        tmem_row(lane_addr + kColW5, 64, v);
        if (r >= 64 && r < 67)
            for (int k = 0; k < 64; ++k) atomicAdd(g5 + (r - 64) * 64 + k, v[k]);
        tmem_row(lane_addr + kColW1, D, v);
        if (r < 64)
            for (int k = 0; k < D; ++k) atomicAdd(g1 + r * D + k, v[k]);
        tmem_row(lane_addr + kColW3, 32, v);
        if (r < 64)
            for (int k = 0; k < 32; ++k) atomicAdd(g3 + r * 32 + k, v[k]);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (r == 0 && *abort && status) atomicExch(status, (unsigned long long)(-VRNERF_ETIMEDOUT));
    if (r < 32) tc::tmem_dealloc(tbase, kBwdCols);
}

// Grid-gradient scatter of the tensor-core backward: one thread per sample
// (consecutive samples in a warp, so the dense-level runs still merge), at
// full occupancy so that the atomics' latency is hidden; dL/dfeatures come
// from the backward kernel in fp32.
template <int L>
__global__ void __launch_bounds__(128)
grid_scatter_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                    const float *__restrict__ r_in, const int2 *__restrict__ rec, const long long *__restrict__ off,
                    const int *__restrict__ n_used, long long n, const float4 *__restrict__ dfeat_in,
                    float *__restrict__ grid_grad) {
    constexpr int D = 2 * L;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {  // uniform per block
        const long long i = i0 + threadIdx.x;
        bool have = false;
        float p[3] = {0.0f, 0.0f, 0.0f}, rn = 0.0f, dfeat[D];
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
        for (int k = 0; k < D / 4; ++k) {
            const float4 v = have ? __ldg(dfeat_in + i * (D / 4) + k) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            dfeat[4 * k] = v.x;
            dfeat[4 * k + 1] = v.y;
            dfeat[4 * k + 2] = v.z;
            dfeat[4 * k + 3] = v.w;
        }
        scatter_grid_grad<L>(f, p, rn, dfeat, have, grid_grad);
    }
}

// Sample forward of the bf16 training precision: one thread per sample of a
// 128-sample tile gathers its features straight into the bf16 operand tile
// (kept in global memory for the backward) and the tile runs the MLPs on the
// tensor cores; sigma and PQ colour per sample.
template <int L>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks)
sample_fwd_tc_kernel(const FieldView f, const float *__restrict__ o_in, const float *__restrict__ d_in,
                     const float *__restrict__ r_in, const int2 *__restrict__ rec, long long n,
                     float4 *__restrict__ sc, uint4 *__restrict__ feat_out, const uint4 *__restrict__ wimg,
                     unsigned long long *__restrict__ status) {
    constexpr int D = 2 * L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *unused;
    const TcShared S = tc_setup<D, 1>(smem, wimg, unused, nullptr, 0);
    const int r = threadIdx.x;
    uint32_t phase = 0;
    bool ok = true;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        if (__syncthreads_or(*S.abort)) break;
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

// fp32 W1..W4 -> the transposed bf16 image TcWT<D>.
__global__ void build_wt_image_kernel(const float *__restrict__ mlp, int D, unsigned char *__restrict__ img) {
    // (matrix, rows N = inputs, K = outputs, source offset, source row length)
    const int w1 = 0, w2 = 64 * D, w3 = w2 + 16 * 64, w4 = w3 + 64 * 32;
    const int spec[4][4] = {{64, 64, w4, 64}, {32, 64, w3, 32}, {64, 16, w2, 64}, {D, 64, w1, D}};
    int e = blockIdx.x * blockDim.x + threadIdx.x, base = 0;
    for (int m = 0; m < 4; ++m) {
        const int N = spec[m][0], K = spec[m][1];
        if (e < N * K) {
            const int n = e / K, k = e % K;  // element (n = input, k = output) = W[k][n]
            const float v = mlp[spec[m][2] + k * spec[m][3] + n];
            const int b = base + (n >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
            *reinterpret_cast<__nv_bfloat16 *>(img + b) = __float2bfloat16_rn(v);
            return;
        }
        e -= N * K;
        base += N * K * 2;
    }
}

// Weight images of the tensor-core backward (forward bf16 image, transposed
// image), rebuilt when the fp32 weights change.
static cudaError_t ensure_bwd_images(vrnerf_field *F, cudaStream_t st) {
    const int D = F->view.d_in;
    const size_t fwd = (size_t)(64 * D * 2 + 16 * 64 * 2 + 64 * 32 * 2 + 64 * 64 * 2 + 16 * 64 * 2);
    const size_t wt = (size_t)(64 * 64 * 2 + 32 * 64 * 2 + 64 * 16 * 2 + D * 64 * 2);
    if (F->tcb_w && F->tcb_version == F->mlp_version) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!F->tcb_w && (e = cudaMalloc(&F->tcb_w, fwd + wt)) != cudaSuccess) return e;
    unsigned char *img = static_cast<unsigned char *>(F->tcb_w);
    build_tc_image_kernel<<<(int)((fwd / 2 + 255) / 256), 256, 0, st>>>(F->mlp, D, 1, img);
    build_wt_image_kernel<<<(int)((wt / 2 + 255) / 256), 256, 0, st>>>(F->mlp, D, img + fwd);
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
    const long long tiles = (n + kTile - 1) / kTile;
    const int grid = (int)(tiles < num_sms() ? tiles : num_sms());
    const unsigned char *img = static_cast<const unsigned char *>(F->tcb_w);
    const size_t fwd = (size_t)TcW<D>::bytes;
    unsigned long long *status = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    kern<<<grid, kTile, smem, st>>>(F->view, o, d, r, rec, off, n_used, n, grad_s, feat,
                                    reinterpret_cast<const uint4 *>(img), reinterpret_cast<const uint4 *>(img + fwd),
                                    dfeat, F->mlp_grad, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_grid_scatter(F, o, d, r, rec, off, n_used, n, dfeat, st);
}

template <int L>
static cudaError_t launch_grid_scatter_t(vrnerf_field *F, const float *o, const float *d, const float *r,
                                         const int2 *rec, const long long *off, const int *n_used, long long n,
                                         const float4 *dfeat, cudaStream_t st) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grid_scatter_kernel<L>, 128, 0);
    if (e != cudaSuccess) return e;
    const long long blocks = (n + 127) / 128, cap = (long long)num_sms() * (per_sm > 0 ? per_sm : 1);
    grid_scatter_kernel<L><<<(int)(blocks < cap ? blocks : cap), 128, 0, st>>>(F->view, o, d, r, rec, off, n_used, n,
                                                                               dfeat, F->grid_grad);
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
    const size_t smem = tc_smem_bytes(D, 0);
    auto kern = sample_fwd_tc_kernel<L>;
    int bps = 0;
    if ((e = prepare_tc(kern, smem, bps)) != cudaSuccess) return e;
    const long long tiles = (n + kTcThreads - 1) / kTcThreads, cap = (long long)num_sms() * bps;
    const int grid = (int)(tiles < cap ? tiles : cap);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    kern<<<grid, kTcThreads, smem, st>>>(F->view, o, d, r, rec, n, sc, feat,
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
