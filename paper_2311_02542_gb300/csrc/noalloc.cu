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
// the counter is cleared on every call; the sample-distance table is copied
// in only when t_near, t_far or max_steps differ from the last call on the
// device. Calls whose work overlaps on the GPU (on different streams, or from
// different host threads) race on it: order them on one stream or
// synchronise in between.
//
// With no distance field (it would need memory of its own) the march tests
// every sample against the occupancy bits instead of skipping empty space,
// which costs more march work than vrnerf_render on sparse scenes.
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

// Key of the sample-distance table last uploaded to each device's scratch:
// the table is copied again only when t_near, t_far or max_steps change.
struct TableKey {
    bool valid = false;
    float t_near = 0.0f, t_far = 0.0f;
    int max_steps = 0;
};
TableKey g_table_key[kMaxDevices];

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

        FieldView view;
        derive_geometry(*desc, view);
        // No distance field exists here (building one would need its own
        // device memory): every sample is tested against the occupancy bits.
        view.skip = 0;
        view.dist = nullptr;
        float *t_dev = reinterpret_cast<float *>(scratch + kCounterBytes);
        unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
        view.grid = grid;
        view.mlp = mlp;
        view.occ = occ_bits;
        view.t_tab = t_dev;

        cudaStream_t st = (cudaStream_t)stream;
        {
            std::lock_guard<std::mutex> lock(g_setup_mutex);
            TableKey &key = g_table_key[dev];
            if (!key.valid || key.t_near != desc->t_near || key.t_far != desc->t_far ||
                key.max_steps != desc->max_steps) {
                float t_host[kMaxSteps + 1];
                fill_sample_table(*desc, t_host);
                // pageable source: the call returns once t_host has been staged
                e = cudaMemcpyAsync(t_dev, t_host, sizeof(float) * (desc->max_steps + 1),
                                    cudaMemcpyHostToDevice, st);
                key.valid = e == cudaSuccess;
                key.t_near = desc->t_near;
                key.t_far = desc->t_far;
                key.max_steps = desc->max_steps;
            }
        }
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
