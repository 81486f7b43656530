// noalloc.cu -- vrnerf_render_noalloc: the fp32 render for callers that may
// not allocate GPU memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- a frame
// callback of a real-time compositor or VR runtime with a hard per-frame
// budget (an allocation can synchronise the device and stall the frame), a
// process whose device memory is carved up up front by another allocator,
// or a plug-in inside a host application that owns all allocations. Such a
// caller keeps the field's parameters in buffers it already owns and
// passes them in; this entry point then allocates nothing.
//
// The render kernel needs a little scratch besides its inputs and outputs:
// the ray-slot counter of the persistent kernel and the table of sample
// distances. Here that scratch is one file-scope __device__ array of
// kScratchBytes, which every GPU that loads the library holds until the
// process exits. Its device address is looked up once per device, with that
// device current, on the first call made on that device; make that first
// call outside any CUDA stream capture.
//
// All calls share the array and it keeps what the last call left in it, so
// the counter is cleared on every call. Calls whose work overlaps on the GPU
// (on different streams, or from different host threads) race on it: order
// them on one stream or synchronise in between.
#include <cmath>
#include <cstring>
#include <mutex>

#include "field.h"

namespace vrn {

int check_desc(const vrnerf_field_desc *d);
int check_views(const int32_t *res, int32_t n, long long &rays);
void make_camera_source(const float *c2w, const float *K, const int32_t *res, int32_t n,
                        RaySource &src);

namespace {

constexpr size_t kScratchBytes = 32 * 1024;      // 32 KiB per device
constexpr size_t kCounterBytes = 256;            // ray-slot counter, padded
constexpr int kMaxSteps = (int)((kScratchBytes - kCounterBytes) / sizeof(float)) - 1;  // 8127
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set-up on first use).
int scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(VRNERF_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "render_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return VRNERF_OK;
}

// The field geometry of a description, with the sample-distance table
// written to a caller-provided array (no heap use).
void derive_view_fixed(const vrnerf_field_desc &d, FieldView &f, float *t_tab) {
    memset(&f, 0, sizeof f);
    f.L = d.levels;
    f.F = d.feats;
    f.d_in = d.levels * d.feats;
    f.log2_T = d.log2_T;
    f.T_mask = (1u << d.log2_T) - 1u;
    f.feat_fp16 = d.feat_fp16 ? 1 : 0;
    f.S = d.max_steps;
    const long long T = 1ll << d.log2_T;
    for (int l = 0; l < d.levels; ++l) {
        const int N = (int)floor(d.base_res * pow(d.growth, (double)l) + 1e-6);
        f.N[l] = N;
        const long long n1 = (long long)N + 1;
        if (n1 * n1 * n1 <= T) f.dense_mask |= 1u << l;
    }
    double ext_max = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double ext = (double)d.aabb_max[k] - (double)d.aabb_min[k];
        f.mn[k] = d.aabb_min[k];
        f.inv_cell[k] = (float)((double)d.occ_res[k] / ext);
        f.res[k] = d.occ_res[k];
        f.res_f[k] = (float)d.occ_res[k];
        if (ext > ext_max) ext_max = ext;
    }
    f.inv_ext = (float)(1.0 / ext_max);
    f.contract = d.contract;
    for (int k = 0; k < 3; ++k) f.cen[k] = (float)(0.5 * ((double)d.aabb_min[k] + (double)d.aabb_max[k]));
    f.inv_h = (float)(2.0 / ext_max);
    f.two_s = (float)(2.0 * d.base_res);
    f.inv_ln_f = (float)(1.0 / log(d.growth));
    f.lod_bias = d.lod_bias;
    f.T_eps = d.T_eps;
    f.density_bias = d.density_bias;
    f.radius_scale = d.radius_scale;
    f.n_mlp = 64 * f.d_in + 16 * 64 + 64 * 32 + 64 * 64 + 3 * 64;
    const double tn = d.t_near, tf = d.t_far;
    for (int i = 0; i <= d.max_steps; ++i)
        t_tab[i] = (float)(tn * pow(tf / tn, (double)i / (double)d.max_steps));
}

}  // namespace
}  // namespace vrn

using namespace vrn;

extern "C" int vrnerf_render_noalloc(const vrnerf_field_desc *desc, const void *grid,
                                     const float *mlp, const uint32_t *occ_bits,
                                     const float *cameras, const float *intrinsics,
                                     const int32_t *resolution_host, int32_t n, float *out,
                                     void *stream) {
    try {
        int rc = check_desc(desc);
        if (rc) return rc;
        if (!grid || !mlp || !occ_bits || !cameras || !intrinsics || !out)
            return fail(VRNERF_EINVAL, "render_noalloc: NULL argument");
        if (desc->max_steps > kMaxSteps)
            return fail(VRNERF_EINVAL,
                        "render_noalloc: max_steps %d exceeds the %d that its %zu-byte scratch holds",
                        desc->max_steps, kMaxSteps, kScratchBytes);
        long long rays = 0;
        if ((rc = check_views(resolution_host, n, rays))) return rc;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "render_noalloc: cudaGetDevice");
        unsigned char *scratch = nullptr;
        if ((rc = scratch_address(dev, &scratch))) return rc;

        float t_host[kMaxSteps + 1];
        FieldView view;
        derive_view_fixed(*desc, view, t_host);
        float *t_dev = reinterpret_cast<float *>(scratch + kCounterBytes);
        unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
        view.grid = grid;
        view.mlp = mlp;
        view.occ = occ_bits;
        view.t_tab = t_dev;

        cudaStream_t st = (cudaStream_t)stream;
        // pageable source: the call returns once t_host has been staged
        e = cudaMemcpyAsync(t_dev, t_host, sizeof(float) * (desc->max_steps + 1),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned long long), st);
        view.check = counter + 1;  // bounds-check bits of checked builds (not reported by this entry)
        if (e != cudaSuccess) return cuda_fail(e, "render_noalloc: scratch set-up");
        RaySource src;
        make_camera_source(cameras, intrinsics, resolution_host, n, src);
        RenderOut ro{out, nullptr, nullptr, nullptr, nullptr};
        ro.n_pix = rays;
        e = launch_render_simt(view, src, ro, counter, st);
        if (e != cudaSuccess) return cuda_fail(e, "render_noalloc: launch");
        return VRNERF_OK;
    } catch (...) {
        return fail(VRNERF_EINVAL, "render_noalloc: unexpected C++ exception");
    }
}
