// init.cu -- seeded field parameters from a counter-based SplitMix64 stream
// (Steele, Lea and Flood, OOPSLA 2014), so that a field created from a seed
// needs no host-side parameter upload.
//
// Stream s of seed z: key = mix(z ^ (s * 0xD1B54A32D192ED03)); draw k =
// mix(key + (k + 1) * 0x9E3779B97F4A7C15); u_k = (draw_k >> 40) * 2^-24.
// Grid: U(lo, hi) in fp64 rounded to fp32 (then fp16 for fp16 storage).
// Weight matrix m (stream 2 + m): Xavier-uniform (2 u - 1) sqrt(6 / (in + out)).
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

// Level m of the occupancy pyramid from level m - 1: bit = OR of the (up to)
// 2x2x2 child bits. One thread per output word.
__global__ void mip_level_kernel(const uint32_t *__restrict__ prev, int prx, int pry, int prz,
                                 uint32_t *__restrict__ out, int rx, int ry, int rz) {
    const long long n = (long long)rx * ry * rz;
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w * 32 >= n) return;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
        const long long i = w * 32 + b;
        if (i >= n) break;
        const int bx = (int)(i % rx), by = (int)((i / rx) % ry), bz = (int)(i / ((long long)rx * ry));
        uint32_t any = 0;
        for (int c = 0; c < 8; ++c) {
            const int cx = 2 * bx + (c & 1), cy = 2 * by + ((c >> 1) & 1), cz = 2 * bz + (c >> 2);
            if (cx < prx && cy < pry && cz < prz) {
                const long long j = cx + (long long)prx * (cy + (long long)pry * cz);
                any |= (prev[j >> 5] >> (j & 31)) & 1u;
            }
        }
        bits |= any << b;
    }
    out[w] = bits;
}

cudaError_t launch_build_mip(const FieldView &f, uint32_t *mip, cudaStream_t st) {
    const uint32_t *prev = f.occ;
    int prx = f.res[0], pry = f.res[1], prz = f.res[2];
    for (int m = 1; m <= f.n_mip; ++m) {
        const int rx = (f.res[0] + (1 << m) - 1) >> m, ry = (f.res[1] + (1 << m) - 1) >> m,
                  rz = (f.res[2] + (1 << m) - 1) >> m;
        const long long words = ((long long)rx * ry * rz + 31) / 32;
        uint32_t *out = mip + f.mip_off[m];
        mip_level_kernel<<<(unsigned)((words + 127) / 128), 128, 0, st>>>(prev, prx, pry, prz, out, rx,
                                                                         ry, rz);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        prev = out;
        prx = rx;
        pry = ry;
        prz = rz;
    }
    return cudaSuccess;
}

}  // namespace vrn
