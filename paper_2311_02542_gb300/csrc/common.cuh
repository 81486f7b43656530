// common.cuh -- device-side building blocks of the per-ray field renderer.
//
// Geometry that decides integers (ray directions, sample positions, occupancy
// voxels, hash-grid corners) is computed in fp32 with each operation rounded
// on its own (__fadd_rn / __fmul_rn / __fdiv_rn / __fsqrt_rn): nvcc would
// otherwise contract a*b+c into one FMA and change which voxel or corner a
// sample lands in. Everything continuous (LOD weights, interpolation, MLP,
// compositing, PQ) uses ordinary fp32 arithmetic and CUDA's math functions.
#pragma once
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

namespace vrn {

constexpr int kMaxLevels = 16;
constexpr int kMaxViews = 256;
constexpr int kTileW = 8;   // rays of one warp cover an 8 x 4 pixel tile
constexpr int kTileH = 4;
constexpr int kDistCap = 32;  // the occupancy distance field saturates at this many voxels

// Everything a kernel needs to read the field; passed by value.
struct FieldView {
    const void *grid;       // [L][T][F] fp32 or fp16
    const float *mlp;       // fp32 W1..W5, [out][in]
    const uint32_t *occ;    // occupancy bits
    const float *t_tab;     // sample distances t_0..t_S
    int L, F, d_in, log2_T, feat_fp16, S;
    uint32_t T_mask;
    int N[kMaxLevels];
    uint32_t dense_mask;
    float mn[3], inv_cell[3], res_f[3];
    int res[3];
    float inv_ext;
    float two_s, inv_ln_f, lod_bias, T_eps, density_bias, radius_scale;
    int n_mlp;
    // empty-space skipping: per voxel v, the distance d to the nearest occupied
    // voxel u in the metric max_k ceil(|u_k - v_k| / dstep[k]) (an L-infinity
    // distance that counts dstep[k] voxels as one unit along axis k, so that
    // skip boxes of anisotropic cells reach about as far along every axis),
    // saturated at kDistCap; 0 = occupied
    const uint8_t *dist;
    int dstep[3];             // voxels per distance unit along each axis (>= 1)
    int skip;                 // 0: test every sample against the occupancy bits
    float skip_eps;           // margin (voxels) kept from the faces of an empty cube
    float ln_tn, inv_ln_q;    // ln t_near and S / ln(t_far / t_near)
    // unbounded scenes (Sec. 4): x = (p - cen) inv_h, y = C(x) (L-infinity
    // contraction), normalised grid position y / 4 + 1/2
    int contract;
    float cen[3], inv_h;
    // checked builds (VRNERF_CHECKED): bounds-check failures are OR-ed in here
    unsigned long long *check;
};

// Checked builds: a failed bounds check records its bit in f.check (read by
// vrnerf_field_status) and the caller skips or clamps the access; nothing
// traps. Release builds compile the checks away.
enum : unsigned long long {
    kCheckHash = 1ull,    // hash-grid index beyond the table
    kCheckVoxel = 2ull,   // occupancy voxel index beyond the grid
    kCheckStep = 4ull,    // sample index beyond the table of distances
    kCheckPixel = 8ull,   // output pixel beyond the launch's rays
    kCheckRecord = 16ull, // training record beyond its buffers
    kCheckTrigger = 32ull // set on purpose by vrnerf_debug_check_trigger
};
#if defined(VRNERF_CHECKED) && VRNERF_CHECKED
#define VRN_CHECKED 1
__device__ __forceinline__ bool vrn_check(const unsigned long long *flag, bool ok, unsigned long long bit) {
    if (!ok && flag) atomicOr(const_cast<unsigned long long *>(flag), bit);
    return ok;
}
#else
#define VRN_CHECKED 0
__device__ __forceinline__ bool vrn_check(const unsigned long long *, bool ok, unsigned long long) { return ok; }
#endif

// One launch's rays: either camera views (pixels in 8x4 tiles) or explicit arrays.
struct ViewInfo {
    int W, H, tiles_x;
    int slot_begin;       // first ray slot of this view
    long long pix_begin;  // first output pixel of this view
};

struct RaySource {
    // camera mode
    const float *c2w;     // [n][12]
    const float *K;       // [n][4]
    int n_views;
    ViewInfo views[kMaxViews];
    // explicit mode (n_views == 0)
    const float *o, *d, *r;
    long long n_slots;    // ray slots to process (camera mode: padded to whole tiles)
};

struct RenderOut {
    float *lin;   // [rays][3]
    float *pq;    // optional
    float *T;     // optional
    int *n;       // optional
    unsigned long long *stats;  // optional [4]: samples, levels fetched, steps tested, rays
    float *depth;               // optional: sum_i w_i t_i
    float *normal;              // optional [rays][3]: sum_i w_i n_i (fp32 kernel only)
    unsigned int *rgba8;        // optional [rays]: sRGB8 + coverage at `exposure`
    float exposure;             // 2^ev, linear scale applied before the sRGB encoding
    long long n_pix;            // rays of the launch (checked builds verify writes; 0: unknown)
};

// Warp-aggregated add of per-thread counters into stats (all lanes call).
__device__ __forceinline__ void add_stats(unsigned long long *stats, unsigned a, unsigned b,
                                          unsigned c, unsigned d) {
    if (!stats) return;
    unsigned long long v[4] = {a, b, c, d};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        unsigned long long x = v[k];
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) x += __shfl_xor_sync(0xffffffffu, x, s);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(stats + k, x);
    }
}

// ---------------------------------------------------------------------------
// fp32 geometry with separate rounding
// ---------------------------------------------------------------------------
__device__ __forceinline__ void camera_ray(const float *__restrict__ c2w, const float *__restrict__ K,
                                           int u, int v, float o[3], float d[3]) {
    float x = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), K[2]), K[0]);
    float y = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), K[3]), K[1]);
    float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), 1.0f));
    float cx = __fdiv_rn(x, n), cy = __fdiv_rn(y, n), cz = __fdiv_rn(1.0f, n);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = __fadd_rn(__fadd_rn(__fmul_rn(c2w[4 * k + 0], cx), __fmul_rn(c2w[4 * k + 1], cy)),
                         __fmul_rn(c2w[4 * k + 2], cz));
        o[k] = c2w[4 * k + 3];
    }
}

// Cubic space contraction with the L-infinity norm (Sec. 4): m = |x|_inf,
// C(x) = x for m <= 1, else (2 - 1/m) x / m, computed as x ((2 - 1/m) (1/m))
// with every operation rounded on its own. Returns the normalised grid
// position ph = C(x) / 4 + 1/2 of world position p.
__device__ __forceinline__ void contracted_position(const FieldView &f, const float p[3], float ph[3]) {
    float x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = __fmul_rn(__fsub_rn(p[k], f.cen[k]), f.inv_h);
    const float m = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fabsf(x[2]));
    if (m > 1.0f) {
        const float inv = __fdiv_rn(1.0f, m);
        const float sc = __fmul_rn(__fsub_rn(2.0f, inv), inv);
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = __fmul_rn(x[k], sc);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ph[k] = __fadd_rn(__fmul_rn(x[k], 0.25f), 0.5f);
}

// p = o + t d and its occupancy voxel; false once the sample leaves the grid.
// The grid of a contracted scene covers all of space (coordinates clamped to
// the last voxel, reached only where 2 - 1/m rounds to 2).
__device__ __forceinline__ bool sample_voxel(const FieldView &f, const float o[3], const float d[3],
                                             float t, float p[3], int &vox, int v[3], float *gc = nullptr) {
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = __fadd_rn(o[k], __fmul_rn(t, d[k]));
    if (f.contract) {
        float ph[3];
        contracted_position(f, p, ph);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float g = __fmul_rn(ph[k], f.res_f[k]);
            if (gc) gc[k] = g;
            const int c = (int)floorf(g);
            v[k] = c < 0 ? 0 : (c > f.res[k] - 1 ? f.res[k] - 1 : c);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float g = __fmul_rn(__fsub_rn(p[k], f.mn[k]), f.inv_cell[k]);
            if (!(g >= 0.0f) || !(g < f.res_f[k])) return false;
            v[k] = (int)g;
        }
    }
    vox = v[0] + f.res[0] * (v[1] + f.res[1] * v[2]);
    if (VRN_CHECKED && !vrn_check(f.check, vox >= 0 && (long long)vox < (long long)f.res[0] * f.res[1] * f.res[2],
                                  kCheckVoxel))
        vox = 0;
    return true;
}
__device__ __forceinline__ bool sample_voxel(const FieldView &f, const float o[3], const float d[3],
                                             float t, float p[3], int &vox) {
    int v[3];
    return sample_voxel(f, o, d, t, p, vox, v);
}

__device__ __forceinline__ bool occupied(const uint32_t *__restrict__ occ, int vox) {
    return (__ldg(occ + (vox >> 5)) >> (vox & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Occupancy march (Sec. 4.3) with exact empty-space skipping.
//
// The evaluated samples are defined per sample: sample i is evaluated iff its
// fp32 position falls in an occupied voxel, and the march ends at the first
// sample outside the grid. The skip never changes that set. A sample's voxel
// v has distance d = dist[v] to the nearest occupied voxel, so every voxel u
// with |u_k - v_k| <= (d - 1) dstep[k] on every axis is empty: the box
// [v_k - (d-1) dstep[k], v_k + (d-1) dstep[k] + 1) of grid coordinates
// (clipped to the grid) holds no occupied voxel. The march shrinks that box
// by skip_eps voxels on every face and jumps to the first sample at or past
// the ray's exit from it.
// Every sample jumped over lies, exactly, at least skip_eps inside the cube;
// skip_eps is far above the rounding error of the fp32 position and of the
// exit distance (checked when the field is created), so each of those
// samples would have been found, one by one, in an empty voxel of the cube.
//
// Contracted scenes: the ray is a curve in the grid, so the exit is bounded
// instead of solved. With a = |x(s) - x(t)|_inf (x = (p - cen) / h), the
// contracted point moves by at most K a in the L-infinity norm, K the largest
// row sum of J_C on the way: 1 inside the inner cube, 4/m - 3/m^2 <= 4/3
// outside, and <= 4/m for m >= 3; m >= m(t) - a along the segment. So with D
// the clearance (grid cube shrunk by skip_eps, in contracted units) every
// sample with a <= max(3D/4, D m / (4 + D) when m(t) >= 3 (4 + D) / 4) lies
// in the cube; the faces on the grid's outer boundary are never crossed.
// ---------------------------------------------------------------------------
struct MarchRay {
    float o[3], d[3];
    float g0[3], inv_s[3];  // grid coordinate at t = 0 and 1 / (grid units per unit t)
    int step;
};

__device__ __forceinline__ void march_init(const FieldView &f, MarchRay &m) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m.g0[k] = (m.o[k] - f.mn[k]) * f.inv_cell[k];
        const float s = m.d[k] * f.inv_cell[k];
        m.inv_s[k] = s != 0.0f ? 1.0f / s : 0.0f;
    }
    m.step = 0;
}

// First sample index j >= lo whose distance is >= t (S if none).
__device__ __forceinline__ int first_sample_at(const FieldView &f, const float *__restrict__ sT,
                                               float t, int lo) {
    int j = (int)ceilf((__logf(t) - f.ln_tn) * f.inv_ln_q);  // estimate, corrected below
    j = j < lo ? lo : (j > f.S ? f.S : j);
    while (j > lo && sT[j - 1] >= t) --j;
    while (j < f.S && sT[j] < t) ++j;
    return j;
}

enum { MARCH_END = 0, MARCH_SAMPLE = 1, MARCH_MORE = 2 };

// Advances m.step to the next evaluated sample (MARCH_SAMPLE, p set,
// m.step = its index), to the end of the ray (MARCH_END), or stops after
// max_iter iterations (MARCH_MORE). tested counts sample tests.
__device__ __forceinline__ int march_next(const FieldView &f, const float *__restrict__ sT,
                                          MarchRay &m, float p[3], int max_iter,
                                          unsigned &tested) {
    for (int it = 0; it < max_iter; ++it) {
        if (m.step >= f.S) return MARCH_END;
        if (VRN_CHECKED && !vrn_check(f.check, m.step >= 0, kCheckStep)) return MARCH_END;
        const float t = sT[m.step];
        int vox, v[3];
        float gc[3];
        if (!sample_voxel(f, m.o, m.d, t, p, vox, v, gc)) return MARCH_END;
        ++tested;
        if (!f.skip) {
            if (occupied(f.occ, vox)) return MARCH_SAMPLE;
            ++m.step;
            continue;
        }
        const int dv = (int)__ldg(f.dist + vox);
        if (dv == 0) return MARCH_SAMPLE;
        if (f.contract) {
            float D = INFINITY, mx = 0.0f, dinf = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int ext = (dv - 1) * f.dstep[k];
                const int lo_i = v[k] - ext, hi_i = v[k] + ext + 1;
                const float cu = 4.0f / f.res_f[k];  // contracted units per voxel
                if (lo_i > 0) D = fminf(D, (gc[k] - ((float)lo_i + f.skip_eps)) * cu);
                if (hi_i < f.res[k]) D = fminf(D, (((float)hi_i - f.skip_eps) - gc[k]) * cu);
                mx = fmaxf(mx, fabsf((p[k] - f.cen[k]) * f.inv_h));
                dinf = fmaxf(dinf, fabsf(m.d[k]));
            }
            if (D > 0.0f && dinf > 0.0f) {
                float a = 0.75f * D;
                if (mx >= 0.75f * (4.0f + D)) a = fmaxf(a, D * mx / (4.0f + D));
                const float t_skip = t + a / (dinf * f.inv_h);
                m.step = first_sample_at(f, sT, t_skip, m.step + 1);
            } else {
                ++m.step;
            }
            continue;
        }
        float t_in = -INFINITY, t_out = INFINITY;
        bool ok = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int ext = (dv - 1) * f.dstep[k];
            const int lo_i = max(v[k] - ext, 0), hi_i = min(v[k] + ext + 1, f.res[k]);
            const float lo = (float)lo_i + f.skip_eps, hi = (float)hi_i - f.skip_eps;
            if (m.inv_s[k] != 0.0f) {
                const float ta = (lo - m.g0[k]) * m.inv_s[k], tb = (hi - m.g0[k]) * m.inv_s[k];
                t_in = fmaxf(t_in, fminf(ta, tb));
                t_out = fminf(t_out, fmaxf(ta, tb));
            } else if (!(m.g0[k] >= lo && m.g0[k] <= hi)) {
                ok = false;
            }
        }
        if (ok && t_in <= t && t_out > t)
            m.step = first_sample_at(f, sT, t_out, m.step + 1);
        else
            ++m.step;
    }
    return MARCH_MORE;
}

// Normalised grid position p^ = (p - box_min) / largest extent, or the
// contracted position of an unbounded scene; fp32 with separate rounding
// (shared by every level of a sample).
__device__ __forceinline__ void grid_position(const FieldView &f, const float p[3], float ph[3]) {
    if (f.contract) {
        contracted_position(f, p, ph);
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) ph[k] = __fmul_rn(__fsub_rn(p[k], f.mn[k]), f.inv_ext);
}

// Contraction Jacobian applied to v at x (k: the axis of the largest |x_k|,
// the first on ties): v inside the inner cube, else s v + s'(m) x sign(x_k) v_k
// with s(m) = 2/m - 1/m^2.
__device__ __forceinline__ void contract_jv(const float x[3], const float v[3], float out[3]) {
    float m = fabsf(x[0]);
    int k = 0;
    if (fabsf(x[1]) > m) { m = fabsf(x[1]); k = 1; }
    if (fabsf(x[2]) > m) { m = fabsf(x[2]); k = 2; }
    if (m <= 1.0f) {
        out[0] = v[0]; out[1] = v[1]; out[2] = v[2];
        return;
    }
    const float im = 1.0f / m;
    const float sc = im * (2.0f - im), ds = 2.0f * im * im * (im - 1.0f);
    const float vk = x[k] >= 0.0f ? v[k] : -v[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = fmaf(ds * x[a], vk, sc * v[a]);
}

// Transposed Jacobian applied to a gradient g at x: the gradient with respect
// to x of a function whose gradient with respect to C(x) is g.
__device__ __forceinline__ void contract_jtv(const float x[3], float g[3]) {
    float m = fabsf(x[0]);
    int k = 0;
    if (fabsf(x[1]) > m) { m = fabsf(x[1]); k = 1; }
    if (fabsf(x[2]) > m) { m = fabsf(x[2]); k = 2; }
    if (m <= 1.0f) return;
    const float im = 1.0f / m;
    const float sc = im * (2.0f - im), ds = 2.0f * im * im * (im - 1.0f);
    const float gx = fmaf(g[0], x[0], fmaf(g[1], x[1], g[2] * x[2]));
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] *= sc;
    g[k] += (x[k] >= 0.0f ? ds : -ds) * gx;
}

// Footprint radius in normalised grid units of the sample at distance t
// (Sec. 4.2.1). Plain scenes: t r / largest extent. Contracted scenes with
// adjacent-ray offsets (du, dv: the directions of the pixels to the right and
// below minus the ray's own): radius_scale times the mean first-order
// distance |J_C (t inv_h du)| to the adjacent rays' contracted samples, over
// 4. Contracted scenes, explicit rays: t r inv_h det(J_C)^(1/3) / 4 with
// det(J_C)^(1/3) = (2m - 1)^(2/3) / m^2 outside the inner cube.
__device__ __forceinline__ float footprint(const FieldView &f, float t, float r, const float p[3],
                                           const float *du, const float *dv) {
    if (!f.contract) return t * r * f.inv_ext;
    float x[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) x[k] = (p[k] - f.cen[k]) * f.inv_h;
    if (du) {
        const float st = t * f.inv_h;
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float *da = a ? dv : du;
            const float v[3] = {st * da[0], st * da[1], st * da[2]};
            float jv[3];
            contract_jv(x, v, jv);
            acc += sqrtf(fmaf(jv[0], jv[0], fmaf(jv[1], jv[1], jv[2] * jv[2])));
        }
        return f.radius_scale * 0.125f * acc;
    }
    const float m = fmaxf(fmaxf(fabsf(x[0]), fabsf(x[1])), fabsf(x[2]));
    const float j = m <= 1.0f ? 1.0f : cbrtf((2.0f * m - 1.0f) * (2.0f * m - 1.0f)) / (m * m);
    return t * r * f.inv_h * j * 0.25f;
}

// Corner indices of level l (corner b at offset (b&1, b>>1&1, b>>2&1)) and
// the position inside the cell, from the normalised position ph.
__device__ __forceinline__ void level_corners_ph(const FieldView &f, int l, const float ph[3],
                                                 uint32_t idx[8], float fr[3]) {
    const int N = f.N[l];
    int c0[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float x = __fmul_rn(ph[k], (float)N);
        int c = (int)floorf(x);
        c = c < 0 ? 0 : (c > N - 1 ? N - 1 : c);
        c0[k] = c;
        fr[k] = __fsub_rn(x, (float)c);
    }
    if ((f.dense_mask >> l) & 1u) {
        const uint32_t n1 = (uint32_t)N + 1u;
#pragma unroll
        for (int b = 0; b < 8; ++b)
            idx[b] = (uint32_t)(c0[0] + (b & 1)) +
                     n1 * ((uint32_t)(c0[1] + ((b >> 1) & 1)) + n1 * (uint32_t)(c0[2] + ((b >> 2) & 1)));
    } else {
        // instant-NGP spatial hash, primes (1, 2654435761, 805459861)
        const uint32_t hx0 = (uint32_t)c0[0], hx1 = hx0 + 1u;
        const uint32_t hy0 = (uint32_t)c0[1] * 2654435761u, hy1 = hy0 + 2654435761u;
        const uint32_t hz0 = (uint32_t)c0[2] * 805459861u, hz1 = hz0 + 805459861u;
        const uint32_t yz[4] = {hy0 ^ hz0, hy1 ^ hz0, hy0 ^ hz1, hy1 ^ hz1};
#pragma unroll
        for (int b = 0; b < 8; ++b) idx[b] = ((b & 1 ? hx1 : hx0) ^ yz[b >> 1]) & f.T_mask;
    }
#if VRN_CHECKED
#pragma unroll
    for (int b = 0; b < 8; ++b)
        if (!vrn_check(f.check, idx[b] <= f.T_mask, kCheckHash)) idx[b] = 0;
#endif
}

__device__ __forceinline__ void level_corners(const FieldView &f, int l, const float p[3],
                                              uint32_t idx[8], float fr[3]) {
    float ph[3];
    grid_position(f, p, ph);
    level_corners_ph(f, l, ph, idx, fr);
}

// Eq. 3 as a clamp: w_l = clamp(L* - l + 1, 0, 1).
__device__ __forceinline__ float lod_star(const FieldView &f, float r_norm) {
    return -logf(f.two_s * r_norm) * f.inv_ln_f + f.lod_bias;
}
__device__ __forceinline__ float lod_weight(float Lstar, int l) {
    return fminf(fmaxf(Lstar - (float)l + 1.0f, 0.0f), 1.0f);
}

// ---------------------------------------------------------------------------
// PQ (Eq. 1-2), fp32
// ---------------------------------------------------------------------------
constexpr float kPqM1 = 1305.0f / 8192.0f;
constexpr float kPqM2 = 2523.0f / 32.0f;
constexpr float kPqInvM1 = 8192.0f / 1305.0f;
constexpr float kPqInvM2 = 32.0f / 2523.0f;
constexpr float kPqC1 = 107.0f / 128.0f;
constexpr float kPqC2 = 2413.0f / 128.0f;
constexpr float kPqC3 = 2392.0f / 128.0f;

// CUDA's __powf (error within 2 + 1.16 |y| ulp) keeps the decode within
// ~1e-5 relative even after the cancellation in e - c1.
__device__ __forceinline__ float pq_to_linear(float E) {
    E = fminf(fmaxf(E, 0.0f), 1.0f);
    float e = __powf(E, kPqInvM2);
    float num = fmaxf(e - kPqC1, 0.0f);
    return 100.0f * __powf(num / (kPqC2 - kPqC3 * e), kPqInvM1);
}

__device__ __forceinline__ float linear_to_pq(float c) {
    float Y = fminf(fmaxf(c * 0.01f, 0.0f), 1.0f);
    float ym = powf(Y, kPqM1);
    return powf((kPqC1 + kPqC2 * ym) / (1.0f + kPqC3 * ym), kPqM2);
}

// Display encoding: sRGB transfer function (IEC 61966-2-1) of a relative
// linear value clamped to [0, 1], 8 bits rounded half up.
__device__ __forceinline__ unsigned int srgb8(float v) {
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    const float s = v <= 0.0031308f ? 12.92f * v : 1.055f * powf(v, 1.0f / 2.4f) - 0.055f;
    return (unsigned int)(255.0f * s + 0.5f);
}

__device__ __forceinline__ unsigned int tonemap_rgba8(const float lin[3], float T, float exposure) {
    unsigned int w = srgb8(lin[0] * exposure) | srgb8(lin[1] * exposure) << 8 | srgb8(lin[2] * exposure) << 16;
    const float a = fminf(fmaxf(1.0f - T, 0.0f), 1.0f);  // coverage, not display-encoded
    return w | (unsigned int)(255.0f * a + 0.5f) << 24;
}

// Per-ray epilogue shared by the render kernels: PQ decode (Eq. 1-2) and the
// optional outputs.
__device__ __forceinline__ void finish_outputs(const RenderOut &out, long long pix, const float C[3], float T,
                                               int n, float depth, const float *N, const unsigned long long *check) {
    if (VRN_CHECKED && out.n_pix > 0 && !vrn_check(check, pix >= 0 && pix < out.n_pix, kCheckPixel)) return;
    float lin[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lin[c] = pq_to_linear(C[c]);
        out.lin[3 * pix + c] = lin[c];
        if (out.pq) out.pq[3 * pix + c] = C[c];
    }
    if (out.T) out.T[pix] = T;
    if (out.n) out.n[pix] = n;
    if (out.depth) out.depth[pix] = depth;
    if (out.rgba8) out.rgba8[pix] = tonemap_rgba8(lin, T, out.exposure);
    if (N && out.normal) {
        out.normal[3 * pix] = N[0];
        out.normal[3 * pix + 1] = N[1];
        out.normal[3 * pix + 2] = N[2];
    }
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, bands 0..3, Condon-Shortley phase, index l^2+l+m.
// Coefficients: sqrt(2) N_lm (-1)^m d^m P_l / dz^m, N_lm^2 = (2l+1)/(4 pi)
// (l-m)!/(l+m)!, times Re / Im of (x + i y)^m.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sh16(float x, float y, float z, float s[16]) {
    const float xx = x * x, yy = y * y, zz = z * z;
    s[0] = 0.28209479177387814f;                 // 1 / (2 sqrt(pi))
    s[1] = -0.48860251190291987f * y;            // sqrt(3 / 4pi)
    s[2] = 0.48860251190291987f * z;
    s[3] = -0.48860251190291987f * x;
    s[4] = 1.0925484305920792f * x * y;          // sqrt(15 / 4pi)
    s[5] = -1.0925484305920792f * y * z;
    s[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);  // sqrt(5 / 16pi)
    s[7] = -1.0925484305920792f * x * z;
    s[8] = 0.54627421529603959f * (xx - yy);     // sqrt(15 / 16pi)
    s[9] = -0.59004358992664352f * y * (3.0f * xx - yy);   // sqrt(35 / 32pi)
    s[10] = 2.8906114426405538f * x * y * z;     // sqrt(105 / 4pi)
    s[11] = -0.45704579946446572f * y * (5.0f * zz - 1.0f);  // sqrt(21 / 32pi)
    s[12] = 0.37317633259011540f * z * (5.0f * zz - 3.0f);  // sqrt(7 / 16pi)
    s[13] = -0.45704579946446572f * x * (5.0f * zz - 1.0f);
    s[14] = 1.4453057213202769f * z * (xx - yy); // sqrt(105 / 16pi)
    s[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
}

// ---------------------------------------------------------------------------
// Ray slots: camera mode maps slot -> (view, pixel) in 8x4 tiles.
// ---------------------------------------------------------------------------
// adj (optional, camera mode only): the direction offsets to the pixels to
// the right and below, d(u+1, v) - d(u, v) and d(u, v+1) - d(u, v), which set
// the footprint of a contracted scene; returns *has_adj = false for explicit rays.
__device__ __forceinline__ bool slot_ray(const RaySource &src, const FieldView &f, long long slot,
                                         float o[3], float d[3], float &r, long long &pix,
                                         float *adj = nullptr, bool *has_adj = nullptr) {
    if (has_adj) *has_adj = src.n_views != 0;
    if (src.n_views == 0) {
        pix = slot;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[k] = __ldg(src.o + 3 * slot + k);
            d[k] = __ldg(src.d + 3 * slot + k);
        }
        r = __ldg(src.r + slot);
        return true;
    }
    int v = 0;
    while (v + 1 < src.n_views && slot >= src.views[v + 1].slot_begin) ++v;
    const ViewInfo &vi = src.views[v];
    int q = (int)(slot - vi.slot_begin);
    int tile = q >> 5, lane = q & 31;
    int px = (tile % vi.tiles_x) * kTileW + (lane & (kTileW - 1));
    int py = (tile / vi.tiles_x) * kTileH + (lane >> 3);
    if (px >= vi.W || py >= vi.H) return false;
    const float *K = src.K + 4 * v;
    camera_ray(src.c2w + 12 * v, K, px, py, o, d);
    if (adj) {
        float oo[3], du[3], dv[3];
        camera_ray(src.c2w + 12 * v, K, px + 1, py, oo, du);
        camera_ray(src.c2w + 12 * v, K, px, py + 1, oo, dv);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            adj[k] = __fsub_rn(du[k], d[k]);
            adj[3 + k] = __fsub_rn(dv[k], d[k]);
        }
    }
    r = __fdiv_rn(f.radius_scale, __ldg(K));
    pix = vi.pix_begin + (long long)py * vi.W + px;
    return true;
}

__device__ __forceinline__ float2 load_feat(const FieldView &f, int l, uint32_t idx) {
    size_t e = (size_t)l * (f.T_mask + 1u) + idx;
    if (f.feat_fp16) {
        uint32_t bits = __ldg(reinterpret_cast<const unsigned int *>(f.grid) + e);
        __half2 h = *reinterpret_cast<__half2 *>(&bits);
        return __half22float2(h);
    }
    return __ldg(reinterpret_cast<const float2 *>(f.grid) + e);
}

// LOD-weighted hash-grid features of one sample (Eq. 3): levels with zero
// weight are not fetched and give zeros.
template <int L>
__device__ __forceinline__ int gather_features(const FieldView &f, const float p[3], float r_norm,
                                               float feat[2 * L]) {
    const float Ls = lod_star(f, r_norm);
    int fetched = 0;
#pragma unroll
    for (int l = 0; l < L; ++l) {
        const float w = lod_weight(Ls, l);
        float a0 = 0.0f, a1 = 0.0f;
        if (w > 0.0f) {
            ++fetched;
            uint32_t idx[8];
            float fr[3];
            level_corners(f, l, p, idx, fr);
            float2 e[8];
#pragma unroll
            for (int b = 0; b < 8; ++b) e[b] = load_feat(f, l, idx[b]);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                float cw = (b & 1 ? fr[0] : 1.0f - fr[0]) * (b & 2 ? fr[1] : 1.0f - fr[1]) *
                           (b & 4 ? fr[2] : 1.0f - fr[2]);
                a0 += cw * e[b].x;
                a1 += cw * e[b].y;
            }
        }
        feat[2 * l] = w * a0;
        feat[2 * l + 1] = w * a1;
    }
    return fetched;
}


// Hash-grid gradient scatter of one sample per lane (all 32 lanes call it,
// `have` false for lanes without a sample) over levels l0 .. l0 + LG - 1:
// dL/dfeat (dfeat[2 (l - l0) + c]) times the level weight w_l and the
// trilinear weight of each corner, added into grid_grad [L][T][F=2].
// On dense levels neighbouring lanes (consecutive samples of a ray) often hit
// the same corners, and thousands of samples per batch meet on the few
// coarse vertices, so runs of equal indices in consecutive lanes are summed
// with shuffles first and only the run's first lane issues the atomic.
template <int LG>
__device__ __forceinline__ void scatter_grid_grad(const FieldView &f, const float p[3], float rn,
                                                  const float *dfeat, bool have, float *grid_grad, int l0) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float Ls = have ? lod_star(f, rn) : -1.0e30f;
#pragma unroll
    for (int q = 0; q < LG; ++q) {  // unrolled: dfeat stays in registers
        const int l = l0 + q;
        const float wl = lod_weight(Ls, l);
        const bool act = have && wl > 0.0f;
        if (!__any_sync(FULL, act)) break;  // weights fall with l for every lane
        uint32_t idx[8];
        float fr[3] = {0.0f, 0.0f, 0.0f};
        if (act) level_corners(f, l, p, idx, fr);
        float2 *gbase = reinterpret_cast<float2 *>(grid_grad) + (size_t)l * (f.T_mask + 1u);
        const bool dense = (f.dense_mask >> l) & 1u;
        if (!dense) {
            // hashed level: the x-adjacent corners (b, b + 1) of a cell often fall on
            // the two halves of one aligned 16-byte pair of entries (indices that
            // differ only in bit 0), which one four-wide atomic updates
            if (act) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float wyz = (j & 1 ? fr[1] : 1.0f - fr[1]) * (j & 2 ? fr[2] : 1.0f - fr[2]) * wl;
                    const float c0 = (1.0f - fr[0]) * wyz, c1 = fr[0] * wyz;
                    const float2 g0 = make_float2(c0 * dfeat[2 * q], c0 * dfeat[2 * q + 1]);
                    const float2 g1 = make_float2(c1 * dfeat[2 * q], c1 * dfeat[2 * q + 1]);
                    const uint32_t i0 = idx[2 * j], i1 = idx[2 * j + 1];
                    if ((i0 ^ i1) == 1u) {
                        const float4 v = (i0 & 1u) ? make_float4(g1.x, g1.y, g0.x, g0.y)
                                                   : make_float4(g0.x, g0.y, g1.x, g1.y);
                        atomicAdd(reinterpret_cast<float4 *>(gbase + (i0 & ~1u)), v);
                    } else {
                        atomicAdd(gbase + i0, g0);
                        atomicAdd(gbase + i1, g1);
                    }
                }
            }
            continue;
        }
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const float cw = (b & 1 ? fr[0] : 1.0f - fr[0]) * (b & 2 ? fr[1] : 1.0f - fr[1]) *
                             (b & 4 ? fr[2] : 1.0f - fr[2]) * wl;
            float gx = act ? cw * dfeat[2 * q] : 0.0f, gy = act ? cw * dfeat[2 * q + 1] : 0.0f;
            const uint32_t key = act ? idx[b] : 0xffffffffu;
            const uint32_t prev = __shfl_up_sync(FULL, key, 1);
            const bool head = lane == 0 || prev != key;
            const unsigned heads = __ballot_sync(FULL, head);
            const unsigned above = heads & ~((2u << lane) - 1u);  // heads after this lane
            const int next = above ? __ffs(above) - 1 : 32;       // end of this lane's run
#pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const float ox = __shfl_down_sync(FULL, gx, s), oy = __shfl_down_sync(FULL, gy, s);
                if (lane + s < next) {
                    gx += ox;
                    gy += oy;
                }
            }
            if (head && act) atomicAdd(gbase + idx[b], make_float2(gx, gy));
        }
    }
}

}  // namespace vrn
