// tc_mlp.cuh -- the density and colour MLPs (Sec. 6) on tcgen05 tensor
// cores for one 128-row tile per CTA, shared by the render, query and
// serving kernels: operand layout, per-layer issue / commit / wait, TMEM
// epilogues, CTA set-up and tear-down, and the host-side launch helpers.
#pragma once
#include <cuda_fp8.h>

#include "field.h"
#include "tc.cuh"

namespace vrn {

constexpr int kTcThreads = 128;
constexpr int kTcMinBlocks = 6;  // resident CTAs per SM the register budget is cut for
constexpr int kTcChunk = 8;      // march iterations between warp refill points
constexpr uint32_t kTmemCols = 64;

template <int D>
struct TcW {  // byte offsets of the weight image (K-major operands)
    static constexpr int w1 = 0;                 // [64][D]
    static constexpr int w2 = w1 + 64 * D * 2;   // [16][64]
    static constexpr int w3 = w2 + 16 * 64 * 2;  // [64][32]
    static constexpr int w4 = w3 + 64 * 32 * 2;  // [64][64]
    static constexpr int w5 = w4 + 64 * 64 * 2;  // [16][64], rows 3..15 zero
    static constexpr int bytes = w5 + 16 * 64 * 2;
};

// Weight image of the fp8 mode: W1 and W5 fp16, W2..W4 e4m3 (K-major,
// 16-byte core-matrix rows), then the inverse weight scales of W2..W4.
template <int D>
struct TcW8 {
    static constexpr int w1 = 0;                  // [64][D] fp16
    static constexpr int w2 = w1 + 64 * D * 2;    // [16][64] e4m3
    static constexpr int w3 = w2 + 16 * 64;       // [64][32] e4m3
    static constexpr int w4 = w3 + 64 * 32;       // [64][64] e4m3
    static constexpr int w5 = w4 + 64 * 64;       // [16][64] fp16
    static constexpr int scales = w5 + 16 * 64 * 2;  // float inv_s2, inv_s3, inv_s4, pad
    static constexpr int bytes = scales + 16;
};

template <int D, int FMT>
struct TcImage {
    static constexpr int bytes = FMT == 2 ? TcW8<D>::bytes : TcW<D>::bytes;
};

struct TcShared {
    unsigned char *w;     // weight image (shared by the CTA's tiles)
    unsigned char *act;   // this tile's 128 x 64 operand tile
    uint64_t *mbar;       // this tile's mbarrier
    volatile int *abort;
    uint32_t tbase;       // this tile's TMEM columns (lane 0)
    uint32_t talloc;      // the CTA's TMEM allocation and its columns
    uint32_t tcols;
    int bar;              // named barrier of the tile's 128 threads (0: the whole CTA of one tile)
};

// The tile's 128 threads meet (a CTA of one tile: the whole CTA). Barrier
// ids are immediates, so that the kernel reserves only the barriers it uses.
__device__ __forceinline__ void tile_sync(int bar) {
    switch (bar) {
    case 0: asm volatile("bar.sync 0, 128;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 1, 128;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 2, 128;" ::: "memory"); break;
    case 3: asm volatile("bar.sync 3, 128;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 128;" ::: "memory"); break;
    }
}

// bar.red.or over the tile's 128 threads: true if any of them passes true.
template <int ID>
__device__ __forceinline__ bool tile_sync_or_id(bool pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((int)pred), "n"(ID)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool tile_sync_or(int bar, bool pred) {
    switch (bar) {
    case 0: return tile_sync_or_id<0>(pred);
    case 1: return tile_sync_or_id<1>(pred);
    case 2: return tile_sync_or_id<2>(pred);
    case 3: return tile_sync_or_id<3>(pred);
    default: return tile_sync_or_id<4>(pred);
    }
}

// Row of this thread in its tile, and whether it issues the tile's MMAs.
__device__ __forceinline__ int tile_row() { return threadIdx.x & (kTcThreads - 1); }

template <int FMT>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if (FMT == 0) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

// ReLU and fp32 -> packed 16-bit pair in one instruction (a in the low half).
template <int FMT>
__device__ __forceinline__ uint32_t pack2_relu(float a, float b) {
    uint32_t d;
    if (FMT == 0)
        asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    else
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

// LOD-weighted hash-grid features of one sample (Sec. 4.2.1, Eq. 3), written
// as row r of the first layer's 128 x 2L operand (16-bit pairs); levels with
// zero weight are not fetched and give zeros. The level loop is kept rolled
// (one level per iteration): the kernel's code stays small and its registers
// free, which measured 2.5-5 % faster on 2048^2 frames than two levels per
// iteration (four: 8-11 % slower). Returns the number of levels fetched.
template <int L, int FMT16>
__device__ __forceinline__ int gather_to_tile(const FieldView &f, const float p[3], float r_norm,
                                              unsigned char *tile, int r) {
    constexpr int D = 2 * L;
    const float Ls = lod_star(f, r_norm);
    unsigned char *row = tile + (r >> 3) * (D / 8) * 128 + (r & 7) * 16;
    float ph[3];
    grid_position(f, p, ph);
    int fetched = 0;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const float w = lod_weight(Ls, l);
        uint32_t word = 0u;
        if (w > 0.0f) {
            ++fetched;
            uint32_t idx[8];
            float fr[3];
            level_corners_ph(f, l, ph, idx, fr);
            const float x0 = 1.0f - fr[0], y0 = 1.0f - fr[1], z0 = 1.0f - fr[2];
            const float w00 = y0 * z0, w10 = fr[1] * z0, w01 = y0 * fr[2], w11 = fr[1] * fr[2];
            const float cw[8] = {x0 * w00, fr[0] * w00, x0 * w10, fr[0] * w10,
                                 x0 * w01, fr[0] * w01, x0 * w11, fr[0] * w11};
            if (f.feat_fp16) {
                // both features of a corner in one half2; interpolate with HFMA2
                const unsigned int *base = reinterpret_cast<const unsigned int *>(f.grid) +
                                           (size_t)l * (f.T_mask + 1u);
                uint32_t e[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) e[b] = __ldg(base + idx[b]);
                __half2 acc = __float2half2_rn(0.0f);
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    acc = __hfma2(__float2half2_rn(cw[b]), *reinterpret_cast<const __half2 *>(&e[b]), acc);
                acc = __hmul2(acc, __float2half2_rn(w));
                if (FMT16 == 0) {
                    word = *reinterpret_cast<uint32_t *>(&acc);
                } else {
                    const float2 v = __half22float2(acc);
                    word = pack2<1>(v.x, v.y);
                }
            } else {
                float2 e[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) e[b] = load_feat(f, l, idx[b]);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    a0 = fmaf(cw[b], e[b].x, a0);
                    a1 = fmaf(cw[b], e[b].y, a1);
                }
                word = pack2<FMT16>(w * a0, w * a1);
            }
        }
        const int c = 2 * l;
        *reinterpret_cast<uint32_t *>(row + (c >> 3) * 128 + (c & 7) * 2) = word;
    }
    return fetched;
}

// Row r of a 128 x K operand tile (K-major core matrices).
template <int K>
__device__ __forceinline__ void store_row(unsigned char *base, int r, const uint32_t (&pk)[K / 2]) {
#pragma unroll
    for (int j = 0; j < K / 8; ++j) {
        uint4 v = make_uint4(pk[4 * j], pk[4 * j + 1], pk[4 * j + 2], pk[4 * j + 3]);
        *reinterpret_cast<uint4 *>(base + (r >> 3) * (K / 8) * 128 + j * 128 + (r & 7) * 16) = v;
    }
}

// ReLU(k x) of this thread's 64 accumulator columns (TMEM) -> row r of the
// 128 x 64 16-bit operand tile, 16 columns (two 16-byte core-matrix rows) at
// a time: only 8 packed words are live at once instead of the whole row,
// which took the 64-register render kernel's spills from 236 to 148 bytes and
// its 2048^2 frame from 2.56 to 2.47 ms.
template <int FMT>
__device__ __forceinline__ void relu_row64(unsigned char *act, int r, uint32_t taddr, float k) {
    unsigned char *row = act + (r >> 3) * (64 / 8) * 128 + (r & 7) * 16;
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
        float v[16];
        tc::tmem_ld16(taddr + c, v);
        uint32_t pk[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) pk[i] = pack2_relu<FMT>(v[2 * i] * k, v[2 * i + 1] * k);
        *reinterpret_cast<uint4 *>(row + (c / 8) * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4 *>(row + (c / 8 + 1) * 128) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    }
}

template <int K, int N, int FMT>
__device__ __forceinline__ void issue_layer(uint32_t a_addr, uint32_t b_addr, uint32_t tmem) {
    constexpr uint32_t sbo = (K / 8) * 128;
    constexpr uint32_t idesc = tc::idesc_f16(N, FMT);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
        tc::mma_f16(tmem, tc::smem_desc(a_addr + ks * 256, 128, sbo), tc::smem_desc(b_addr + ks * 256, 128, sbo),
                    idesc, ks > 0 ? 1u : 0u);
}

// e4m3 operands: 16 elements per core-matrix row, K = 32 per instruction.
template <int K, int N>
__device__ __forceinline__ void issue_layer_e4m3(uint32_t a_addr, uint32_t b_addr, uint32_t tmem) {
    constexpr uint32_t sbo = (K / 16) * 128;
    constexpr uint32_t idesc = tc::idesc_e4m3(N);
#pragma unroll
    for (int ks = 0; ks < K / 32; ++ks)
        tc::mma_f8(tmem, tc::smem_desc(a_addr + ks * 256, 128, sbo), tc::smem_desc(b_addr + ks * 256, 128, sbo),
                   idesc, ks > 0 ? 1u : 0u);
}

template <int K, int N>
__device__ __forceinline__ void run_layer_e4m3(const TcShared &S, int w_off, uint32_t &phase, bool &ok) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    tile_sync(S.bar);
    if (tile_row() == 0) {
        tc::fence_after_sync();
        issue_layer_e4m3<K, N>(tc::smem_u32(S.act), tc::smem_u32(S.w) + w_off, S.tbase);
        tc::mma_commit(S.mbar);
    }
    ok = tc::mbar_wait_bounded(S.mbar, phase, S.abort) && ok;
    phase ^= 1u;
    tc::fence_after_sync();
}

// Power-of-two scale that maps the row maximum m into [128, 256) (e4m3
// holds up to 448), and its inverse.
__device__ __forceinline__ void row_scale(float m, float &s, float &inv) {
    const int e = (int)((__float_as_uint(m) >> 23) & 255u);
    if (m > 0.0f && e > 0 && e < 255) {
        const int k = 7 - (e - 127);                   // s = 2^k, m * s in [128, 256)
        const int kk = k > 126 ? 126 : (k < -126 ? -126 : k);
        s = __uint_as_float((uint32_t)(127 + kk) << 23);
        inv = __uint_as_float((uint32_t)(127 - kk) << 23);
    } else {
        s = 1.0f;
        inv = 1.0f;
    }
}

// Row r of a 128 x K e4m3 operand (16-byte core-matrix rows): K / 16 chunks.
template <int K>
__device__ __forceinline__ void store_row_e4m3(unsigned char *base, int r, const float *v, float s) {
#pragma unroll
    for (int j = 0; j < K / 16; ++j) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(
                make_float2(v[16 * j + 4 * q] * s, v[16 * j + 4 * q + 1] * s), __NV_SATFINITE, __NV_E4M3);
            const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(
                make_float2(v[16 * j + 4 * q + 2] * s, v[16 * j + 4 * q + 3] * s), __NV_SATFINITE, __NV_E4M3);
            w[q] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
        *reinterpret_cast<uint4 *>(base + (r >> 3) * (K / 16) * 128 + j * 128 + (r & 7) * 16) =
            make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Runs one layer: the tile's rows are written; all threads sync, thread 0
// issues and commits, everyone waits for the accumulators.
template <int K, int N, int FMT>
__device__ __forceinline__ void run_layer(const TcShared &S, int w_off, uint32_t &phase, bool &ok) {
    tc::fence_proxy_async();
    tc::fence_before_sync();
    tile_sync(S.bar);
    if (tile_row() == 0) {
        tc::fence_after_sync();
        issue_layer<K, N, FMT>(tc::smem_u32(S.act), tc::smem_u32(S.w) + w_off, S.tbase);
        tc::mma_commit(S.mbar);
    }
    ok = tc::mbar_wait_bounded(S.mbar, phase, S.abort) && ok;
    phase ^= 1u;
    tc::fence_after_sync();
}

// Density MLP (D -> 64 -> 16, ReLU; sigma = exp(o_0 + bias)) and colour MLP
// ([o, SH(d)] 32 -> 64 -> 64 -> 3, ReLU, sigmoid) for the 128 rows of the
// CTA; this thread's row is `feat`, or, when feat is null, has already been
// written into the first operand (gather_to_tile). All 128 threads must call it.
template <int D, int FMT>
__device__ __forceinline__ void tc_mlp(const TcShared &S, const float *feat, const float dir[3],
                                       float density_bias, float &sigma, float rgb[3], uint32_t &phase,
                                       bool &ok) {
    using W = TcW<D>;
    const int r = tile_row();
    const uint32_t taddr = S.tbase + ((uint32_t)(r & ~31) << 16);
    if (feat) {
        uint32_t pk[D / 2];
#pragma unroll
        for (int i = 0; i < D / 2; ++i) pk[i] = pack2<FMT>(feat[2 * i], feat[2 * i + 1]);
        store_row<D>(S.act, r, pk);
    }
    run_layer<D, 64, FMT>(S, W::w1, phase, ok);
    relu_row64<FMT>(S.act, r, taddr, 1.0f);
    run_layer<64, 16, FMT>(S, W::w2, phase, ok);
    {
        float o[16], sh[16];
        tc::tmem_ld16(taddr, o);
        sigma = expf(o[0] + density_bias);
        sh16(dir[0], dir[1], dir[2], sh);
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            pk[i] = pack2<FMT>(o[2 * i], o[2 * i + 1]);
            pk[8 + i] = pack2<FMT>(sh[2 * i], sh[2 * i + 1]);
        }
        store_row<32>(S.act, r, pk);
    }
    run_layer<32, 64, FMT>(S, W::w3, phase, ok);
    relu_row64<FMT>(S.act, r, taddr, 1.0f);
    run_layer<64, 64, FMT>(S, W::w4, phase, ok);
    relu_row64<FMT>(S.act, r, taddr, 1.0f);
    run_layer<64, 16, FMT>(S, W::w5, phase, ok);
    {
        float z[16];
        tc::tmem_ld16(taddr, z);
        rgb[0] = 1.0f / (1.0f + expf(-z[0]));
        rgb[1] = 1.0f / (1.0f + expf(-z[1]));
        rgb[2] = 1.0f / (1.0f + expf(-z[2]));
    }
    tc::fence_before_sync();  // this tile's TMEM reads precede the next tile's MMAs
}

// fp8 mode: the density MLP's output layer and the colour MLP's two hidden
// layers (W2, W3, W4) take e4m3 operands with a power-of-two scale per row
// (this thread's sample) and per weight matrix, undone on the fp32
// accumulator; the first layer (W1) and the colour output (W5) stay fp16.
template <int D>
__device__ __forceinline__ void tc_mlp_fp8(const TcShared &S, const float *feat, const float dir[3],
                                           float density_bias, float &sigma, float rgb[3], uint32_t &phase,
                                           bool &ok) {
    using W = TcW8<D>;
    const int r = tile_row();
    const uint32_t taddr = S.tbase + ((uint32_t)(r & ~31) << 16);
    const float *inv_w = reinterpret_cast<const float *>(S.w + W::scales);
    if (feat) {
        uint32_t pk[D / 2];
#pragma unroll
        for (int i = 0; i < D / 2; ++i) pk[i] = pack2<0>(feat[2 * i], feat[2 * i + 1]);
        store_row<D>(S.act, r, pk);
    }
    run_layer<D, 64, 0>(S, W::w1, phase, ok);
    float s_in, inv_in;
    {
        float h[64], m = 0.0f;
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                h[c + i] = fmaxf(v[i], 0.0f);
                m = fmaxf(m, h[c + i]);
            }
        }
        row_scale(m, s_in, inv_in);
        store_row_e4m3<64>(S.act, r, h, s_in);
    }
    run_layer_e4m3<64, 16>(S, W::w2, phase, ok);
    {
        float o[16], x[32];
        tc::tmem_ld16(taddr, o);
        const float k = inv_in * inv_w[0];
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            o[i] *= k;
            x[i] = o[i];
        }
        sigma = expf(o[0] + density_bias);
        sh16(dir[0], dir[1], dir[2], x + 16);
#pragma unroll
        for (int i = 0; i < 32; ++i) m = fmaxf(m, fabsf(x[i]));
        row_scale(m, s_in, inv_in);
        store_row_e4m3<32>(S.act, r, x, s_in);
    }
    run_layer_e4m3<32, 64>(S, W::w3, phase, ok);
    {
        float h[64], m = 0.0f;
        const float k = inv_in * inv_w[1];
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                h[c + i] = fmaxf(v[i] * k, 0.0f);
                m = fmaxf(m, h[c + i]);
            }
        }
        row_scale(m, s_in, inv_in);
        store_row_e4m3<64>(S.act, r, h, s_in);
    }
    run_layer_e4m3<64, 64>(S, W::w4, phase, ok);
    {
        uint32_t pk[32];
        const float k = inv_in * inv_w[2];
#pragma unroll
        for (int c = 0; c < 64; c += 16) {
            float v[16];
            tc::tmem_ld16(taddr + c, v);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                pk[c / 2 + i] = pack2_relu<0>(v[2 * i] * k, v[2 * i + 1] * k);
        }
        store_row<64>(S.act, r, pk);
    }
    run_layer<64, 16, 0>(S, W::w5, phase, ok);
    {
        float z[16];
        tc::tmem_ld16(taddr, z);
        rgb[0] = 1.0f / (1.0f + expf(-z[0]));
        rgb[1] = 1.0f / (1.0f + expf(-z[1]));
        rgb[2] = 1.0f / (1.0f + expf(-z[2]));
    }
    tc::fence_before_sync();
}

template <int D, int FMT>
__device__ __forceinline__ void tc_mlp_any(const TcShared &S, const float *feat, const float dir[3],
                                           float density_bias, float &sigma, float rgb[3], uint32_t &phase,
                                           bool &ok) {
    if constexpr (FMT == 2)
        tc_mlp_fp8<D>(S, feat, dir, density_bias, sigma, rgb, phase, ok);
    else
        tc_mlp<D, FMT>(S, feat, dir, density_bias, sigma, rgb, phase, ok);
}

// Shared-memory carve-up, weight upload, mbarriers and TMEM set-up for a
// CTA of NT tiles (NT x 128 threads): one weight image, then NT activation
// tiles, the sample table, and the misc block (NT mbarriers, the TMEM
// holder, the abort flag). Tile g = threadIdx.x / 128 gets activation tile
// g, mbarrier g, TMEM columns [64 g, 64 g + 64) and named barrier g + 1
// (barrier 0, the whole CTA, when NT = 1).
template <int D, int FMT = 0, int NT = 1>
__device__ __forceinline__ TcShared tc_setup(unsigned char *smem, const uint4 *__restrict__ wimg,
                                             float *&sT, const float *__restrict__ t_tab, int S_steps) {
    using W = TcImage<D, FMT>;
    constexpr uint32_t kCols = NT == 1 ? kTmemCols : (NT == 2 ? 128u : 256u);
    static_assert(NT >= 1 && NT <= 4, "1 to 4 tiles per CTA");
    const int g = NT == 1 ? 0 : (int)(threadIdx.x >> 7);
    TcShared S;
    S.w = smem;
    unsigned char *act0 = smem + ((W::bytes + 1023) & ~1023);
    S.act = act0 + g * (128 * 64 * 2);
    sT = reinterpret_cast<float *>(act0 + NT * (128 * 64 * 2));
    const int nt = S_steps + 1;
    unsigned char *misc = reinterpret_cast<unsigned char *>(sT + ((nt + 3) & ~3));
    uint64_t *mbars = reinterpret_cast<uint64_t *>(misc);
    S.mbar = mbars + g;
    uint32_t *holder = reinterpret_cast<uint32_t *>(misc + 8 * NT);
    S.abort = reinterpret_cast<volatile int *>(misc + 8 * NT + 4);
    for (int i = threadIdx.x; i < W::bytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(S.w)[i] = wimg[i];
    if (t_tab)
        for (int i = threadIdx.x; i < nt; i += blockDim.x) sT[i] = t_tab[i];
    if (threadIdx.x == 0) {
        for (int k = 0; k < NT; ++k) tc::mbar_init(mbars + k, 1);
        *S.abort = 0;
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(holder, kCols);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    S.talloc = *holder;
    S.tcols = kCols;
    S.tbase = S.talloc + (uint32_t)(64 * g);
    S.bar = NT == 1 ? 0 : 1 + g;
    return S;
}

__device__ __forceinline__ void tc_teardown(const TcShared &S, unsigned long long *status) {
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0 && *S.abort && status) atomicExch(status, (unsigned long long)(-VRNERF_ETIMEDOUT));
    if (threadIdx.x < 32) tc::tmem_dealloc(S.talloc, S.tcols);
}


// fp32 W1..W5 -> the K-major operand image of TcW<D>, fp16 or bf16.
__global__ void build_tc_image_kernel(const float *__restrict__ mlp, int D, int fmt,
                                      unsigned char *__restrict__ img);
// fp32 W1..W5 -> the image of TcW8<D> (one CTA per weight matrix).
__global__ void build_tc_image_fp8_kernel(const float *__restrict__ mlp, int D, unsigned char *__restrict__ img);

inline size_t tc_smem_bytes(int D, int S_steps, int NT = 1) {
    const size_t wb = (size_t)(64 * D * 2 + 16 * 64 * 2 + 64 * 32 * 2 + 64 * 64 * 2 + 16 * 64 * 2);
    size_t b = ((wb + 1023) & ~(size_t)1023) + (size_t)NT * 128 * 64 * 2 +
               sizeof(float) * (size_t)((S_steps + 1 + 3) & ~3) + 64;
    // at most 512 / cols CTAs per SM by shared memory (228 KB usable, 1 KB
    // reserved per CTA), so that tcgen05.alloc never waits
    const size_t cols = NT == 1 ? kTmemCols : (NT == 2 ? 128 : 256);
    const size_t floor_bytes = (size_t)233472 / (512 / cols + 1) - 1024 + 16;
    return b > floor_bytes ? b : floor_bytes;
}

inline cudaError_t ensure_tc_image(vrnerf_field *F, int fmt, cudaStream_t st) {
    const int D = F->view.d_in;
    const size_t bytes = (size_t)(64 * D * 2 + 16 * 64 * 2 + 64 * 32 * 2 + 64 * 64 * 2 + 16 * 64 * 2);
    if (F->tc_w && F->tc_prec == fmt && F->tc_version == F->mlp_version) return cudaSuccess;
    if (!F->tc_w) {
        cudaError_t e = cudaMalloc(&F->tc_w, bytes);
        if (e != cudaSuccess) return e;
        F->tc_w_bytes = bytes;
    }
    if (fmt == 2) {
        build_tc_image_fp8_kernel<<<5, 256, 0, st>>>(F->mlp, D, static_cast<unsigned char *>(F->tc_w));
    } else {
        const int n = (int)(bytes / 2);
        build_tc_image_kernel<<<(n + 255) / 256, 256, 0, st>>>(F->mlp, D, fmt, static_cast<unsigned char *>(F->tc_w));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    F->tc_prec = fmt;
    F->tc_version = F->mlp_version;
    return cudaSuccess;
}

// Resident CTAs per SM from the kernel's registers and shared memory (the
// runtime's occupancy query under-reports kernels that allocate TMEM), capped
// so that the CTAs on one SM never ask for more than its 512 TMEM columns.
template <typename K>
inline cudaError_t prepare_tc(K kern, size_t smem, int &blocks_per_sm, int NT = 1) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    int dev = 0, regs_sm = 65536, smem_sm = 233472;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int regs = ((fa.numRegs + 7) / 8) * 8 * kTcThreads * NT;
    const int by_regs = regs > 0 ? regs_sm / regs : 8;
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    blocks_per_sm = by_regs < by_smem ? by_regs : by_smem;
    const int cols = NT == 1 ? (int)kTmemCols : (NT == 2 ? 128 : 256);
    if (blocks_per_sm > 512 / cols) blocks_per_sm = 512 / cols;
    if (blocks_per_sm < 1) return cudaErrorInvalidConfiguration;
    return cudaSuccess;
}

}  // namespace vrn
