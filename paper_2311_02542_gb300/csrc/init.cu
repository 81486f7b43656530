// init.cu -- seeded field parameters from a counter-based SplitMix64 stream
// (Steele, Lea and Flood, OOPSLA 2014), so that a field created from a seed
// needs no host-side parameter upload.
//
// Stream s of seed z: key = mix(z ^ (s * 0xD1B54A32D192ED03)); draw k =
// mix(key + (k + 1) * 0x9E3779B97F4A7C15); u_k = (draw_k >> 40) * 2^-24.
// Grid: U(lo, hi) in fp64 rounded to fp32 (then fp16 for fp16 storage).
// Weight matrix m (stream 2 + m): Xavier-uniform (2 u - 1) sqrt(6 / (in + out)).
#include <utility>

#include "internal.h"

namespace vrn {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double draw01(uint64_t key, long long k) {
    uint64_t z = mix64(key + (uint64_t)(k + 1) * 0x9E3779B97F4A7C15ull);
    return (double)(z >> 40) * 0x1p-24;
}

__global__ void seeded_grid_kernel(void *grid, int fp16, long long n, uint64_t key, double lo,
                                   double hi) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double u = draw01(key, k);
        float v = __double2float_rn(__dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u)));
        if (fp16)
            reinterpret_cast<__half *>(grid)[k] = __float2half_rn(v);
        else
            reinterpret_cast<float *>(grid)[k] = v;
    }
}

__global__ void seeded_matrix_kernel(float *w, long long n, uint64_t key, double bound) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double u = draw01(key, k);
        w[k] = __double2float_rn(__dmul_rn(__dsub_rn(__dmul_rn(2.0, u), 1.0), bound));
    }
}

static uint64_t host_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return host_mix64(seed ^ (stream * 0xD1B54A32D192ED03ull));
}

cudaError_t launch_seeded_grid(void *grid, int fp16, long long n, uint64_t seed, double lo,
                               double hi, cudaStream_t st) {
    int blocks = num_sms() * 8;
    seeded_grid_kernel<<<blocks, 256, 0, st>>>(grid, fp16, n, stream_key(seed, 1), lo, hi);
    return cudaGetLastError();
}

cudaError_t launch_seeded_mlp(float *mlp, const int (*shapes)[2], int n_mats, uint64_t seed,
                              cudaStream_t st) {
    long long off = 0;
    for (int m = 0; m < n_mats; ++m) {
        const int fo = shapes[m][0], fi = shapes[m][1];
        const long long n = (long long)fo * fi;
        const double bound = sqrt(6.0 / (double)(fi + fo));
        seeded_matrix_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
            mlp + off, n, stream_key(seed, 2 + m), bound);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        off += n;
    }
    return cudaSuccess;
}

// Occupancy distance field: dist[v] = min(kDistCap, d(v)), 0 for occupied
// voxels, with d(v) the distance from v to the nearest occupied voxel u in
// the metric max_k ceil(|u_k - v_k| / dstep[k]). After r dilations of the
// occupancy by the box of half-extent dstep[k] voxels along axis k, a voxel
// is covered iff an occupied voxel lies within distance r; its distance is
// the first r that covers it. Each dilation is dstep[0] + dstep[1] + dstep[2]
// separable 3-tap passes.
__global__ void dist_init_kernel(const uint32_t *__restrict__ occ, long long n, uint8_t *__restrict__ mask,
                                 uint8_t *__restrict__ dist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint8_t o = (occ[i >> 5] >> (i & 31)) & 1u;
        mask[i] = o;
        dist[i] = o ? 0 : (uint8_t)kDistCap;
    }
}

__global__ void dilate_axis_kernel(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int rx, int ry,
                                   int rz, int axis) {
    const long long n = (long long)rx * ry * rz;
    const long long stride = axis == 0 ? 1 : (axis == 1 ? rx : (long long)rx * ry);
    const int len = axis == 0 ? rx : (axis == 1 ? ry : rz);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)((i / stride) % len);
        uint8_t v = in[i];
        if (c > 0) v |= in[i - stride];
        if (c + 1 < len) v |= in[i + stride];
        out[i] = v;
    }
}

__global__ void dist_assign_kernel(const uint8_t *__restrict__ mask, long long n, int r, uint8_t *__restrict__ dist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (mask[i] && dist[i] == (uint8_t)kDistCap) dist[i] = (uint8_t)r;
}

cudaError_t launch_build_dist(const FieldView &f, uint8_t *dist, cudaStream_t st) {
    const int rx = f.res[0], ry = f.res[1], rz = f.res[2];
    const long long n = (long long)rx * ry * rz;
    uint8_t *a = nullptr, *b = nullptr;
    cudaError_t e = cudaMallocAsync(&a, (size_t)n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&b, (size_t)n, st);
    const int grid = num_sms() * 8;
    if (e == cudaSuccess) {
        dist_init_kernel<<<grid, 256, 0, st>>>(f.occ, n, a, dist);
        for (int r = 1; r < kDistCap && e == cudaSuccess; ++r) {
            for (int k = 0; k < 3; ++k)
                for (int j = 0; j < f.dstep[k]; ++j) {
                    dilate_axis_kernel<<<grid, 256, 0, st>>>(a, b, rx, ry, rz, k);
                    std::swap(a, b);  // a holds the dilated mask
                }
            dist_assign_kernel<<<grid, 256, 0, st>>>(a, n, r, dist);
            e = cudaGetLastError();
        }
    }
    if (a) cudaFreeAsync(a, st);
    if (b) cudaFreeAsync(b, st);
    return e;
}

}  // namespace vrn
