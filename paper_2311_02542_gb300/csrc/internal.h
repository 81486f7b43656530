// internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace vrn {

// NVTX range over an entry point or a stage (header-only NVTX 3: free unless
// a profiler is attached), so that timelines show the library's calls.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Per-kernel launch shape, filled on first use for the current device.
struct Launch {
    int blocks_per_sm = 0;
    int smem = 0;
};

int num_sms();

// render_simt.cu: plain fp32 path (MLP on the CUDA cores)
size_t simt_smem_bytes(const FieldView &f);
cudaError_t launch_render_simt(const FieldView &f, const RaySource &src, const RenderOut &out,
                               unsigned long long *counter, cudaStream_t st);
cudaError_t launch_query_simt(const FieldView &f, const float *pos, const float *dir,
                              const float *radius, int n, float *sigma, float *rgb, float *feat,
                              cudaStream_t st);
cudaError_t launch_debug_march(const FieldView &f, const float *o, const float *d, int B, int cap,
                               int *rec_i, int *rec_vox, int *count, cudaStream_t st);
cudaError_t launch_tonemap(const float *pq, const float *T, long long n, float exposure, unsigned int *rgba8,
                           cudaStream_t st);
cudaError_t launch_debug_corners(const FieldView &f, const float *pos, int n, uint32_t *idx,
                                 cudaStream_t st);

// init.cu: seeded parameters (SplitMix64) and format conversion
cudaError_t launch_seeded_grid(void *grid, int fp16, long long n, uint64_t seed, double lo,
                               double hi, cudaStream_t st);
cudaError_t launch_seeded_mlp(float *mlp, const int (*shapes)[2], int n_mats, uint64_t seed,
                              cudaStream_t st);
// occupancy distance field (res_x * res_y * res_z bytes) from f.occ
cudaError_t launch_build_dist(const FieldView &f, uint8_t *dist, cudaStream_t st);

}  // namespace vrn
