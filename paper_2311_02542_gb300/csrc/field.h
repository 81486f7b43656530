// field.h -- the opaque vrnerf_field of the C ABI and the host-side helpers
// that the translation units share.
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/vrnerf.h"
#include "internal.h"

struct vrnerf_field {
    vrnerf_field_desc desc{};
    int device = 0;
    vrn::FieldView view{};
    // parameters and occupancy
    void *grid = nullptr;         // [L][T][F] fp32 or fp16
    float *mlp = nullptr;         // fp32 W1..W5
    uint32_t *occ = nullptr;
    float *t_tab = nullptr;       // [S+1]
    void *counter = nullptr;      // ray-slot counter of the persistent kernels (scratch)
    uint8_t *dist = nullptr;      // occupancy distance field (one byte per voxel)
    float *hist = nullptr;        // training history: max composited opacity per voxel
    // tensor-core weight images, rebuilt when the fp32 weights change
    void *tc_w = nullptr;
    size_t tc_w_bytes = 0;
    int tc_prec = -1;
    uint64_t mlp_version = 1, tc_version = 0;
    // tensor-core backward (bf16 training precision): forward + transposed images
    void *tcb_w = nullptr;
    uint64_t tcb_version = 0;
    int train_prec = VRNERF_FP32;
    uint64_t sample_budget = 0;     // samples per pass of the training pipeline (0: default)
    // training state
    float *grid_grad = nullptr, *mlp_grad = nullptr;
    float *grid_master = nullptr;  // fp32 master copy when the grid is stored in fp16
    float *m_grid = nullptr, *v_grid = nullptr, *m_mlp = nullptr, *v_mlp = nullptr;
    float *loss_acc = nullptr;
    void *train_scratch = nullptr;  // per-batch forward results (C, n, dL/dC)
    int adam_t = 0;
    // render_host staging
    float *stage_cam = nullptr, *stage_out = nullptr;
    size_t stage_cam_bytes = 0, stage_out_bytes = 0;
    vrn::RaySource src_scratch{};

    void release();
    int ensure_staging(size_t cam_bytes, size_t out_bytes);
};

namespace vrn {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
uint64_t grid_bytes(const vrnerf_field_desc &d);
uint64_t grid_entries(const vrnerf_field_desc &d);
uint64_t occ_words(const vrnerf_field_desc &d);
int check_desc(const vrnerf_field_desc *d);
// The field geometry a description implies (levels, grids, skip settings),
// the table of sample distances t_0..t_S written to any array of S + 1
// floats, and both together.
void derive_geometry(const vrnerf_field_desc &d, FieldView &f);
void fill_sample_table(const vrnerf_field_desc &d, float *t_tab);
void derive_view(const vrnerf_field_desc &d, FieldView &f, std::vector<float> &t_tab);
void release_train_scratch(vrnerf_field *F);

// render_tc.cu, train_tc.cu: tcgen05 tensor-core MLP path
cudaError_t launch_fwd_tc(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                          long long n, float4 *sc, uint4 *feat, cudaStream_t st);
cudaError_t launch_bwd_tc(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                          const long long *off, const int *n_used, long long n, const float4 *grad_s,
                          const uint4 *feat, float4 *dfeat, cudaStream_t st);
cudaError_t launch_grid_scatter(vrnerf_field *F, const float *o, const float *d, const float *r, const int2 *rec,
                                const long long *off, const int *n_used, long long n, const float4 *dfeat,
                                cudaStream_t st);
cudaError_t launch_render_tc(vrnerf_field *F, const RaySource &src, const RenderOut &out, int prec,
                             cudaStream_t st);
cudaError_t launch_query_tc(vrnerf_field *F, const float *pos, const float *dir, const float *radius,
                            int n, float *sigma, float *rgb, float *feat, int prec, cudaStream_t st);

}  // namespace vrn
