// prune.cu -- occupancy-grid pruning (Sec. 4.3.2): joint history- and
// grid-based pruning, then the distance field is rebuilt.
//
// Grid part: one warp per voxel; its lanes evaluate the density at the k^3
// sub-cell centres of the voxel (full detail: zero footprint, so every
// level is fetched), the warp takes the maximum, and lane 0 turns it into an
// opacity with the smallest step a training ray can take in the voxel: the
// spacing of the exponential sample interval holding the distance from the
// nearest camera centre to the voxel box. History part: the largest opacity
// of any sample composited in the voxel during training (recorded by
// vrnerf_backward once vrnerf_history_reset has been called). A voxel stays
// occupied iff it was, and either opacity reaches the threshold.
#include <cstring>
#include <vector>

#include "field.h"

namespace vrn {

cudaError_t launch_build_dist(const FieldView &f, uint8_t *dist, cudaStream_t st);

// World position of a contracted point y (|y|_inf < 2): the inverse
// contraction x = y for |y|_inf <= 1, else y / (m (2 - m)); false at m >= 2.
__device__ __forceinline__ bool uncontract_world(const FieldView &f, const float y[3], float p[3]) {
    const float m = fmaxf(fmaxf(fabsf(y[0]), fabsf(y[1])), fabsf(y[2]));
    if (m >= 2.0f) return false;
    const float sc = m <= 1.0f ? 1.0f : 1.0f / (m * (2.0f - m));
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = f.cen[a] + y[a] * sc / f.inv_h;
    return true;
}

template <int L>
__global__ void __launch_bounds__(256)
prune_kernel(const FieldView f, const float *__restrict__ cams, int n_cams, int k, float threshold,
             const float *__restrict__ hist, float *__restrict__ alpha_out, uint32_t *__restrict__ occ_out,
             unsigned long long *__restrict__ kept) {
    constexpr int D = 2 * L;
    const int lane = threadIdx.x & 31;
    const long long nvox = (long long)f.res[0] * f.res[1] * f.res[2];
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const float *W1 = f.mlp, *W2 = W1 + 64 * D;
    unsigned int kept_here = 0;
    for (long long v = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); v < nvox; v += warps) {
        if (alpha_out && lane == 0) alpha_out[v] = 0.0f;
        if (!occupied(f.occ, (int)v)) continue;
        const int vx = (int)(v % f.res[0]), vy = (int)((v / f.res[0]) % f.res[1]),
                  vz = (int)(v / ((long long)f.res[0] * f.res[1]));
        const int vv[3] = {vx, vy, vz};
        float lo[3], cell[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cell[a] = 1.0f / f.inv_cell[a];
            lo[a] = f.mn[a] + (float)vv[a] * cell[a];
        }
        float smax = 0.0f, dmin = INFINITY;
        for (int i = lane; i < k * k * k; i += 32) {
            const int j[3] = {i % k, (i / k) % k, i / (k * k)};
            float p[3];
            if (f.contract) {
                // lattice point of the contracted voxel, mapped back to world space
                float y[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    y[a] = 4.0f * ((float)vv[a] + ((float)j[a] + 0.5f) / (float)k) / f.res_f[a] - 2.0f;
                uncontract_world(f, y, p);
                for (int c = 0; c < n_cams; ++c) {
                    float s2 = 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float e = p[a] - __ldg(cams + 3 * c + a);
                        s2 = fmaf(e, e, s2);
                    }
                    dmin = fminf(dmin, sqrtf(s2));
                }
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) p[a] = lo[a] + ((float)j[a] + 0.5f) / (float)k * cell[a];
            }
            float feat[D];
            gather_features<L>(f, p, 0.0f, feat);
            float o0 = 0.0f;
            for (int jj = 0; jj < 64; ++jj) {
                float a = 0.0f;
#pragma unroll
                for (int q = 0; q < D; ++q) a = fmaf(__ldg(W1 + jj * D + q), feat[q], a);
                o0 = fmaf(__ldg(W2 + jj), fmaxf(a, 0.0f), o0);
            }
            smax = fmaxf(smax, expf(o0 + f.density_bias));
        }
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) {
            smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, s));
            dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, s));
        }
        if (lane == 0) {
            if (f.contract) {
                // the voxel's world region: a box inside the inner cube, else the
                // lattice points (above) and the finite corner pre-images
                float ylo[3], yhi[3];
                bool inner = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    ylo[a] = 4.0f * (float)vv[a] / f.res_f[a] - 2.0f;
                    yhi[a] = 4.0f * (float)(vv[a] + 1) / f.res_f[a] - 2.0f;
                    if (ylo[a] < -1.0f || yhi[a] > 1.0f) inner = false;
                }
                if (inner) {
                    dmin = INFINITY;
                    for (int c = 0; c < n_cams; ++c) {
                        float s2 = 0.0f;
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float l = f.cen[a] + ylo[a] / f.inv_h, h = f.cen[a] + yhi[a] / f.inv_h;
                            const float cc = __ldg(cams + 3 * c + a);
                            const float dd = cc < l ? l - cc : (cc > h ? cc - h : 0.0f);
                            s2 = fmaf(dd, dd, s2);
                        }
                        dmin = fminf(dmin, sqrtf(s2));
                    }
                } else {
                    for (int b = 0; b < 8; ++b) {
                        float y[3], q[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) y[a] = (b >> a) & 1 ? yhi[a] : ylo[a];
                        if (!uncontract_world(f, y, q)) continue;
                        for (int c = 0; c < n_cams; ++c) {
                            float s2 = 0.0f;
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                const float e = q[a] - __ldg(cams + 3 * c + a);
                                s2 = fmaf(e, e, s2);
                            }
                            dmin = fminf(dmin, sqrtf(s2));
                        }
                    }
                }
            } else {
                for (int c = 0; c < n_cams; ++c) {
                    float s2 = 0.0f;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float cc = __ldg(cams + 3 * c + a), l = lo[a], h = lo[a] + cell[a];
                        const float dd = cc < l ? l - cc : (cc > h ? cc - h : 0.0f);
                        s2 = fmaf(dd, dd, s2);
                    }
                    dmin = fminf(dmin, sqrtf(s2));
                }
            }
            // interval [t_i, t_i+1) holding dmin (i clamped to [0, S-1])
            int lo_i = 0, hi_i = f.S - 1;
            while (lo_i < hi_i) {
                const int mid = (lo_i + hi_i + 1) >> 1;
                if (__ldg(f.t_tab + mid) <= dmin) lo_i = mid;
                else hi_i = mid - 1;
            }
            const float delta = __ldg(f.t_tab + lo_i + 1) - __ldg(f.t_tab + lo_i);
            const float alpha = -expm1f(-smax * delta);
            if (alpha_out) alpha_out[v] = alpha;
            if (alpha >= threshold || (hist && hist[v] >= threshold)) {
                atomicOr(occ_out + (v >> 5), 1u << (v & 31));
                ++kept_here;
            }
        }
    }
    if (lane == 0 && kept_here) atomicAdd(kept, (unsigned long long)kept_here);
}

// Nearest-neighbour refinement of the occupancy grid by an integer factor:
// a child voxel takes its parent's bit (one thread per output word) and, when
// a history is kept, its parent's history value.
__global__ void upsample_bits_kernel(const uint32_t *__restrict__ occ, int3 r0, int fac, int3 r1, long long nvox1,
                                     uint32_t *__restrict__ out) {
    const long long words = (nvox1 + 31) / 32;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < words;
         w += (long long)gridDim.x * blockDim.x) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const long long v = w * 32 + b;
            if (v >= nvox1) break;
            const long long x = v % r1.x, y = (v / r1.x) % r1.y, z = v / ((long long)r1.x * r1.y);
            const long long p = x / fac + r0.x * (y / fac + r0.y * (z / fac));
            word |= ((__ldg(occ + (p >> 5)) >> (p & 31)) & 1u) << b;
        }
        out[w] = word;
    }
}

__global__ void upsample_hist_kernel(const float *__restrict__ h0, int3 r0, int fac, int3 r1, long long nvox1,
                                     float *__restrict__ h1) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox1;
         v += (long long)gridDim.x * blockDim.x) {
        const long long x = v % r1.x, y = (v / r1.x) % r1.y, z = v / ((long long)r1.x * r1.y);
        h1[v] = __ldg(h0 + x / fac + r0.x * (y / fac + r0.y * (z / fac)));
    }
}

}  // namespace vrn

using namespace vrn;

extern "C" {

int vrnerf_history_reset(vrnerf_field *F) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    const size_t n = (size_t)F->desc.occ_res[0] * F->desc.occ_res[1] * F->desc.occ_res[2];
    cudaError_t e = cudaSuccess;
    if (!F->hist && (e = cudaMalloc(&F->hist, n * sizeof(float))) != cudaSuccess)
        return fail(VRNERF_ENOMEM, "history: %s", cudaGetErrorString(e));
    if ((e = cudaMemset(F->hist, 0, n * sizeof(float))) != cudaSuccess) return cuda_fail(e, "history_reset");
    return VRNERF_OK;
}

int vrnerf_field_get_history(vrnerf_field *F, float *hist_host) {
    if (!F || !hist_host) return fail(VRNERF_EINVAL, "NULL argument");
    if (!F->hist) return fail(VRNERF_EINVAL, "no history: call vrnerf_history_reset first");
    const size_t n = (size_t)F->desc.occ_res[0] * F->desc.occ_res[1] * F->desc.occ_res[2];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(hist_host, F->hist, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "get_history");
    return VRNERF_OK;
}

int vrnerf_prune(vrnerf_field *F, const float *camera_centres_host, int32_t n_cameras, int32_t points_per_axis,
                 float threshold, int32_t apply, float *alpha_out, uint32_t *occ_bits_out, uint64_t *kept_host) {
    NvtxRange nvtx_range("vrnerf_prune");
    if (!F || !camera_centres_host) return fail(VRNERF_EINVAL, "NULL argument");
    if (n_cameras < 1 || n_cameras > 65536) return fail(VRNERF_EINVAL, "n_cameras must be in [1, 65536]");
    if (points_per_axis < 1 || points_per_axis > 16) return fail(VRNERF_EINVAL, "points_per_axis must be in [1, 16]");
    if (!(threshold >= 0.0f)) return fail(VRNERF_EINVAL, "threshold must be >= 0");
    const vrnerf_field_desc &d = F->desc;
    const long long nvox = (long long)d.occ_res[0] * d.occ_res[1] * d.occ_res[2];
    const size_t words = (size_t)((nvox + 31) / 32);
    float *cams = nullptr;
    uint32_t *occ_new = nullptr;
    unsigned long long *kept = nullptr;
    cudaError_t e = cudaMalloc(&cams, sizeof(float) * 3 * n_cameras);
    if (e == cudaSuccess) e = cudaMalloc(&occ_new, words * 4);
    if (e == cudaSuccess) e = cudaMalloc(&kept, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(cams, camera_centres_host, sizeof(float) * 3 * n_cameras, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(occ_new, 0, words * 4);
    if (e == cudaSuccess) e = cudaMemset(kept, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        const int blocks = num_sms() * 8;
        if (F->view.L == 8)
            prune_kernel<8><<<blocks, 256>>>(F->view, cams, n_cameras, points_per_axis, threshold, F->hist,
                                             alpha_out, occ_new, kept);
        else
            prune_kernel<16><<<blocks, 256>>>(F->view, cams, n_cameras, points_per_axis, threshold, F->hist,
                                              alpha_out, occ_new, kept);
        e = cudaGetLastError();
    }
    unsigned long long kept_h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&kept_h, kept, sizeof kept_h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && occ_bits_out) e = cudaMemcpy(occ_bits_out, occ_new, words * 4, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && apply) {
        e = cudaMemcpy(F->occ, occ_new, words * 4, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = launch_build_dist(F->view, F->dist, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(cams);
    cudaFree(occ_new);
    cudaFree(kept);
    if (e != cudaSuccess) return cuda_fail(e, "prune");
    if (kept_host) *kept_host = kept_h;
    return VRNERF_OK;
}

int vrnerf_field_get_occupancy(vrnerf_field *F, uint32_t *occ_bits_host) {
    if (!F || !occ_bits_host) return fail(VRNERF_EINVAL, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(occ_bits_host, F->occ, occ_words(F->desc) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "get_occupancy");
    return VRNERF_OK;
}

int vrnerf_occupancy_upsample(vrnerf_field *F, int32_t factor) {
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (factor < 2 || factor > 8) return fail(VRNERF_EINVAL, "factor must be in [2, 8]");
    vrnerf_field_desc d = F->desc;
    long long nvox1 = 1;
    for (int k = 0; k < 3; ++k) {
        d.occ_res[k] *= factor;
        nvox1 *= d.occ_res[k];
    }
    int rc = check_desc(&d);
    if (rc) return rc;
    const int3 r0{F->desc.occ_res[0], F->desc.occ_res[1], F->desc.occ_res[2]};
    const int3 r1{d.occ_res[0], d.occ_res[1], d.occ_res[2]};
    uint32_t *occ1 = nullptr;
    uint8_t *dist1 = nullptr;
    float *hist1 = nullptr;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMalloc(&occ1, occ_words(d) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dist1, (size_t)nvox1);
    if (e == cudaSuccess && F->hist) e = cudaMalloc(&hist1, (size_t)nvox1 * sizeof(float));
    if (e == cudaSuccess) {
        const int blocks = num_sms() * 4;
        upsample_bits_kernel<<<blocks, 256>>>(F->occ, r0, factor, r1, nvox1, occ1);
        if (hist1) upsample_hist_kernel<<<blocks, 256>>>(F->hist, r0, factor, r1, nvox1, hist1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(occ1);
        cudaFree(dist1);
        cudaFree(hist1);
        return cuda_fail(e, "occupancy_upsample");
    }
    cudaFree(F->occ);
    cudaFree(F->dist);
    cudaFree(F->hist);
    F->occ = occ1;
    F->dist = dist1;
    F->hist = hist1;
    F->desc = d;
    std::vector<float> t_tab;
    derive_view(d, F->view, t_tab);
    F->view.grid = F->grid;
    F->view.mlp = F->mlp;
    F->view.occ = F->occ;
    F->view.t_tab = F->t_tab;
    F->view.dist = F->dist;
    F->view.check = reinterpret_cast<unsigned long long *>(F->counter) + 2;
    e = launch_build_dist(F->view, F->dist, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "occupancy_upsample: distance field");
    return VRNERF_OK;
}

}  // extern "C"
