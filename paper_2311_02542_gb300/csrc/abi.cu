// abi.cu -- the C ABI (include/vrnerf.h): field lifetime, argument checking
// and launches. Host code only; kernels live in the other translation units.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/vrnerf.h"
#include "internal.h"
#include "field.h"

namespace vrn {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(VRNERF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_err.clear(); }

int num_sms() {
    static int dev_cached = -1, sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != dev_cached) {
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        dev_cached = dev;
    }
    return sms > 0 ? sms : 1;
}

// ---------------------------------------------------------------------------
// description checks and derived geometry
// ---------------------------------------------------------------------------
// Sets the test bit of the bounds-check word (checked builds only).
__global__ void check_trigger_kernel(const FieldView f) { vrn_check(f.check, threadIdx.x != 0, kCheckTrigger); }

int check_desc(const vrnerf_field_desc *d) {
    if (!d) return fail(VRNERF_EINVAL, "desc is NULL");
    if (d->feats != 2) return fail(VRNERF_EINVAL, "feats must be 2 (got %d)", d->feats);
    if (d->levels * d->feats != 16 && d->levels * d->feats != 32)
        return fail(VRNERF_EINVAL, "levels * feats must be 16 or 32 (got %d)", d->levels * d->feats);
    if (d->log2_T < 4 || d->log2_T > 24) return fail(VRNERF_EINVAL, "log2_T must be in [4, 24]");
    if (d->d_hidden != 64 || d->d_out != 16 || d->c_hidden != 64 || d->c_layers != 2)
        return fail(VRNERF_EINVAL, "MLP widths must be 64 / 16 / 64 x 2 (Sec. 6)");
    if (!(d->base_res >= 1.0) || !(d->growth >= 1.0) || !std::isfinite(d->growth))
        return fail(VRNERF_EINVAL, "base_res and growth must be >= 1");
    for (int k = 0; k < 3; ++k) {
        if (!(d->aabb_max[k] > d->aabb_min[k])) return fail(VRNERF_EINVAL, "empty AABB on axis %d", k);
        if (d->occ_res[k] < 1 || d->occ_res[k] > 2048)
            return fail(VRNERF_EINVAL, "occ_res must be in [1, 2048]");
    }
    if (d->contract != 0 && d->contract != 1) return fail(VRNERF_EINVAL, "contract must be 0 or 1");
    if ((long long)d->occ_res[0] * d->occ_res[1] * d->occ_res[2] > 0x7fffffffll)
        return fail(VRNERF_EINVAL, "occupancy grid must hold fewer than 2^31 voxels");
    if (d->max_steps < 1 || d->max_steps > 8192) return fail(VRNERF_EINVAL, "max_steps must be in [1, 8192]");
    if (!(d->t_near > 0.0f) || !(d->t_far > d->t_near))
        return fail(VRNERF_EINVAL, "need 0 < t_near < t_far");
    if (!(d->T_eps >= 0.0f) || !(d->radius_scale >= 0.0f) || !std::isfinite(d->lod_bias) ||
        !std::isfinite(d->density_bias))
        return fail(VRNERF_EINVAL, "bad T_eps / radius_scale / lod_bias / density_bias");
    const double top = d->base_res * pow(d->growth, (double)(d->levels - 1));
    if (top > 1.0e6) return fail(VRNERF_EINVAL, "finest level resolution too large");
    return VRNERF_OK;
}

void derive_geometry(const vrnerf_field_desc &d, FieldView &f) {
    memset(&f, 0, sizeof f);
    f.L = d.levels;
    f.F = d.feats;
    f.d_in = d.levels * d.feats;
    f.log2_T = d.log2_T;
    f.T_mask = (1u << d.log2_T) - 1u;
    f.feat_fp16 = d.feat_fp16 ? 1 : 0;
    f.S = d.max_steps;
    f.dense_mask = 0;
    const long long T = 1ll << d.log2_T;
    for (int l = 0; l < d.levels; ++l) {
        // N_l = floor(s f^l + 1e-6); dense when (N_l + 1)^3 <= T
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
    // distance-field units: dstep[k] voxels along axis k, about the largest
    // cell's size (1 on a contracted grid, whose cells are cubes)
    double cell_max = 0.0;
    for (int k = 0; k < 3; ++k)
        cell_max = fmax(cell_max, ((double)d.aabb_max[k] - (double)d.aabb_min[k]) / d.occ_res[k]);
    for (int k = 0; k < 3; ++k) {
        const double cell = ((double)d.aabb_max[k] - (double)d.aabb_min[k]) / d.occ_res[k];
        const int r = d.contract ? 1 : (int)floor(cell_max / cell + 1e-9);
        f.dstep[k] = r < 1 ? 1 : (r > 64 ? 64 : r);
    }
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
    const int res_max = max(d.occ_res[0], max(d.occ_res[1], d.occ_res[2]));
    // Skipping is exact when skip_eps exceeds the rounding error of the fp32
    // grid coordinate of a sample and of a cube-exit distance, both below
    // 2^-24 (c (t_far + 2 A + ext) + res) up to a small factor (A: largest
    // |coordinate| of the box, c: largest voxels per unit); keep a 16x margin.
    f.skip_eps = 1.0f / 16.0f;
    double A = 0.0, c_max = 0.0;
    for (int k = 0; k < 3; ++k) {
        A = fmax(A, fmax(fabs((double)d.aabb_min[k]), fabs((double)d.aabb_max[k])));
        c_max = fmax(c_max, (double)f.inv_cell[k]);
    }
    const double err = ldexp(1.0, -24) * (c_max * ((double)d.t_far + 2.0 * A + ext_max) + res_max);
    f.skip = (16.0 * err < (double)f.skip_eps) ? 1 : 0;
    if (d.contract) {
        // contracted coordinates stay within [-2, 2]: a sample's rounding
        // error there is a few ulps of 2 plus that of x = (p - cen) / h near
        // the inner cube; the skip bound itself keeps a relative slack
        const double err_c = ldexp(1.0, -24) * (8.0 + 4.0 * A * (double)f.inv_h) * res_max / 4.0;
        f.skip = (16.0 * err_c < (double)f.skip_eps) ? 1 : 0;
    }
    f.ln_tn = logf(d.t_near);
    f.inv_ln_q = (float)((double)d.max_steps / log((double)d.t_far / (double)d.t_near));
}

void fill_sample_table(const vrnerf_field_desc &d, float *t_tab) {
    // exponential sample distances t_i = t_near (t_far / t_near)^(i / S), fp64 -> fp32
    const double tn = d.t_near, tf = d.t_far;
    for (int i = 0; i <= d.max_steps; ++i)
        t_tab[i] = (float)(tn * pow(tf / tn, (double)i / (double)d.max_steps));
}

void derive_view(const vrnerf_field_desc &d, FieldView &f, std::vector<float> &t_tab) {
    derive_geometry(d, f);
    t_tab.resize(d.max_steps + 1);
    fill_sample_table(d, t_tab.data());
}

uint64_t grid_bytes(const vrnerf_field_desc &d) {
    return (uint64_t)d.levels * (1ull << d.log2_T) * d.feats * (d.feat_fp16 ? 2 : 4);
}
uint64_t grid_entries(const vrnerf_field_desc &d) {
    return (uint64_t)d.levels * (1ull << d.log2_T) * d.feats;
}
uint64_t occ_words(const vrnerf_field_desc &d) {
    return ((uint64_t)d.occ_res[0] * d.occ_res[1] * d.occ_res[2] + 31) / 32;
}

int check_views(const int32_t *res, int32_t n, long long &rays) {
    if (n < 1 || n > VRNERF_MAX_VIEWS) return fail(VRNERF_EINVAL, "n views must be in [1, %d]", VRNERF_MAX_VIEWS);
    if (!res) return fail(VRNERF_EINVAL, "resolution is NULL");
    rays = 0;
    for (int v = 0; v < n; ++v) {
        if (res[2 * v] < 1 || res[2 * v] > 16384 || res[2 * v + 1] < 1 || res[2 * v + 1] > 16384)
            return fail(VRNERF_EINVAL, "view %d: resolution must be in [1, 16384]", v);
        rays += (long long)res[2 * v] * res[2 * v + 1];
    }
    if (rays >= (1ll << 31)) return fail(VRNERF_EINVAL, "too many rays in one call");
    return VRNERF_OK;
}

void make_camera_source(const float *c2w, const float *K, const int32_t *res, int32_t n, RaySource &src) {
    memset(&src, 0, sizeof src);
    src.c2w = c2w;
    src.K = K;
    src.n_views = n;
    long long slots = 0, pix = 0;
    for (int v = 0; v < n; ++v) {
        ViewInfo &vi = src.views[v];
        vi.W = res[2 * v];
        vi.H = res[2 * v + 1];
        vi.tiles_x = (vi.W + kTileW - 1) / kTileW;
        const int tiles_y = (vi.H + kTileH - 1) / kTileH;
        vi.slot_begin = (int)slots;
        vi.pix_begin = pix;
        slots += (long long)vi.tiles_x * tiles_y * 32;
        pix += (long long)vi.W * vi.H;
    }
    src.n_slots = slots;
}

}  // namespace vrn

using namespace vrn;

void vrnerf_field::release() {
    release_train_scratch(this);
    void *ptrs[] = {grid,     mlp,      occ,         t_tab,  counter, tc_w,   grid_grad, mlp_grad,
                    grid_master, m_grid, v_grid, m_mlp, v_mlp, loss_acc, stage_cam, stage_out, dist, hist, tcb_w};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    grid = nullptr;
    mlp = nullptr;
    occ = nullptr;
    t_tab = nullptr;
    counter = nullptr;
    dist = nullptr;
    hist = nullptr;
    tcb_w = nullptr;
    tc_w = nullptr;
    grid_grad = mlp_grad = grid_master = m_grid = v_grid = m_mlp = v_mlp = loss_acc = nullptr;
    stage_cam = stage_out = nullptr;
}

int vrnerf_field::ensure_staging(size_t cam_bytes, size_t out_bytes) {
    cudaError_t e = cudaSuccess;
    if (cam_bytes > stage_cam_bytes) {
        if (stage_cam) cudaFree(stage_cam);
        stage_cam = nullptr;
        stage_cam_bytes = 0;
        if ((e = cudaMalloc(&stage_cam, cam_bytes)) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "staging allocation failed: %s", cudaGetErrorString(e));
        stage_cam_bytes = cam_bytes;
    }
    if (out_bytes > stage_out_bytes) {
        if (stage_out) cudaFree(stage_out);
        stage_out = nullptr;
        stage_out_bytes = 0;
        if ((e = cudaMalloc(&stage_out, out_bytes)) != cudaSuccess)
            return fail(VRNERF_ENOMEM, "staging allocation failed: %s", cudaGetErrorString(e));
        stage_out_bytes = out_bytes;
    }
    return VRNERF_OK;
}

#define ABI_GUARD_BEGIN \
    try {               \
        clear_error();
#define ABI_GUARD_END                                                 \
    }                                                                 \
    catch (const std::bad_alloc &) {                                  \
        return fail(VRNERF_ENOMEM, "host allocation failed");         \
    }                                                                 \
    catch (...) {                                                     \
        return fail(VRNERF_EINVAL, "unexpected C++ exception");       \
    }

extern "C" {

const char *vrnerf_last_error(void) { return g_err.c_str(); }

int vrnerf_field_sizes(const vrnerf_field_desc *desc, uint64_t *gb, uint64_t *mf, uint64_t *ow) {
    ABI_GUARD_BEGIN
    int rc = check_desc(desc);
    if (rc) return rc;
    if (gb) *gb = grid_bytes(*desc);
    if (mf) *mf = (uint64_t)(64 * desc->levels * desc->feats + 16 * 64 + 64 * 32 + 64 * 64 + 3 * 64);
    if (ow) *ow = occ_words(*desc);
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_field_create(const vrnerf_field_desc *desc, const void *grid_host, const float *mlp_host,
                        const uint32_t *occ_bits_host, uint64_t seed, vrnerf_field **out) {
    ABI_GUARD_BEGIN
    if (!out) return fail(VRNERF_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_desc(desc);
    if (rc) return rc;
    if (!occ_bits_host) return fail(VRNERF_EINVAL, "occ_bits_host is NULL");
    vrnerf_field *F = new vrnerf_field();
    F->desc = *desc;
    cudaGetDevice(&F->device);
    std::vector<float> t_tab;
    derive_view(*desc, F->view, t_tab);
    const uint64_t gbytes = grid_bytes(*desc);
    const uint64_t nmlp = (uint64_t)F->view.n_mlp;
    const uint64_t nocc = occ_words(*desc);
    cudaError_t e;
    if ((e = cudaMalloc(&F->grid, gbytes)) != cudaSuccess ||
        (e = cudaMalloc(&F->mlp, nmlp * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&F->occ, nocc * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc(&F->t_tab, t_tab.size() * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&F->counter, 64)) != cudaSuccess ||
        (e = cudaMalloc(&F->dist, (size_t)desc->occ_res[0] * desc->occ_res[1] * desc->occ_res[2])) != cudaSuccess) {
        vrnerf_field_destroy(F);
        cudaGetLastError();
        return fail(VRNERF_ENOMEM, "device allocation failed: %s", cudaGetErrorString(e));
    }
    if (grid_host)
        e = cudaMemcpy(F->grid, grid_host, gbytes, cudaMemcpyHostToDevice);
    else
        e = launch_seeded_grid(F->grid, desc->feat_fp16, (long long)grid_entries(*desc), seed,
                               (double)-1e-2f, (double)1e-2f, 0);
    if (e == cudaSuccess) {
        if (mlp_host) {
            e = cudaMemcpy(F->mlp, mlp_host, nmlp * sizeof(float), cudaMemcpyHostToDevice);
        } else {
            const int din = desc->levels * desc->feats;
            const int shapes[5][2] = {{64, din}, {16, 64}, {64, 32}, {64, 64}, {3, 64}};
            e = launch_seeded_mlp(F->mlp, shapes, 5, seed, 0);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpy(F->occ, occ_bits_host, nocc * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(F->counter, 0, 64);
    if (e == cudaSuccess)
        e = cudaMemcpy(F->t_tab, t_tab.data(), t_tab.size() * 4, cudaMemcpyHostToDevice);
    F->view.grid = F->grid;
    F->view.mlp = F->mlp;
    F->view.occ = F->occ;
    F->view.t_tab = F->t_tab;
    F->view.dist = F->dist;
    F->view.check = reinterpret_cast<unsigned long long *>(F->counter) + 2;
    if (e == cudaSuccess) e = launch_build_dist(F->view, F->dist, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        vrnerf_field_destroy(F);
        return cuda_fail(e, "field_create");
    }
    *out = F;
    return VRNERF_OK;
    ABI_GUARD_END
}

void vrnerf_field_destroy(vrnerf_field *F) {
    if (!F) return;
    try {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(F->device);
        cudaDeviceSynchronize();
        F->release();
        cudaSetDevice(prev);
        delete F;
    } catch (...) {
    }
}

int vrnerf_field_status(vrnerf_field *F) {
    ABI_GUARD_BEGIN
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    unsigned long long w[2] = {0, 0};  // status word, bounds-check bits (checked builds)
    unsigned long long *dev = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(w, dev, sizeof w, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && (w[0] || w[1])) e = cudaMemset(dev, 0, sizeof w);
    if (e != cudaSuccess) return cuda_fail(e, "field_status");
    if (w[0]) return fail(-(int)w[0], "a device-side wait timed out; the last kernel stopped early");
    if (w[1]) return fail(VRNERF_ECHECK, "bounds checks failed (bits 0x%llx: 1 hash index, 2 voxel, 4 sample, "
                                         "8 pixel, 16 training record, 32 test trigger)", w[1]);
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_field_get_params(vrnerf_field *F, void *grid_host, float *mlp_host) {
    ABI_GUARD_BEGIN
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    cudaError_t e = cudaSuccess;
    if (grid_host) e = cudaMemcpy(grid_host, F->grid, grid_bytes(F->desc), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && mlp_host)
        e = cudaMemcpy(mlp_host, F->mlp, sizeof(float) * F->view.n_mlp, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "get_params");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_tonemap(const float *pq, const float *T, int64_t n, float exposure_ev, uint32_t *rgba8, void *stream) {
    ABI_GUARD_BEGIN
    if (n < 0) return fail(VRNERF_EINVAL, "n must be >= 0");
    if (n > 0 && (!pq || !rgba8)) return fail(VRNERF_EINVAL, "NULL argument");
    if (!std::isfinite(exposure_ev)) return fail(VRNERF_EINVAL, "exposure_ev must be finite");
    cudaError_t e = launch_tonemap(pq, T, n, exp2f(exposure_ev), reinterpret_cast<unsigned int *>(rgba8),
                                   static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "tonemap");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_build_checked(void) { return VRN_CHECKED; }

int vrnerf_debug_check_trigger(vrnerf_field *F, void *stream) {
    ABI_GUARD_BEGIN
    if (!F) return fail(VRNERF_EINVAL, "field is NULL");
    if (!VRN_CHECKED) return fail(VRNERF_EINVAL, "not a checked build");
    check_trigger_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(F->view);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "debug_check_trigger");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_field_set_occupancy(vrnerf_field *F, const uint32_t *occ) {
    ABI_GUARD_BEGIN
    if (!F || !occ) return fail(VRNERF_EINVAL, "NULL argument");
    cudaError_t e = cudaMemcpy(F->occ, occ, occ_words(F->desc) * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_build_dist(F->view, F->dist, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "set_occupancy");
    return VRNERF_OK;
    ABI_GUARD_END
}

static int check_precision(int p) {
    if (p < VRNERF_FP32 || p > VRNERF_FP8) return fail(VRNERF_EINVAL, "unknown precision %d", p);
    return VRNERF_OK;
}

static int render_common(vrnerf_field *F, const RaySource &src, float *out,
                         const vrnerf_render_opts *opts, cudaStream_t st, long long n_pix) {
    const int prec = opts ? opts->precision : VRNERF_FP32;
    int rc = check_precision(prec);
    if (rc) return rc;
    if (opts && opts->out_normal && prec != VRNERF_FP32)
        return fail(VRNERF_EINVAL, "out_normal needs the fp32 path (precision VRNERF_FP32)");
    if (opts && opts->out_rgba8 && !std::isfinite(opts->exposure_ev))
        return fail(VRNERF_EINVAL, "exposure_ev must be finite");
    RenderOut ro{out, opts ? opts->out_pq : nullptr, opts ? opts->out_T : nullptr,
                 opts ? opts->out_n : nullptr,
                 opts ? reinterpret_cast<unsigned long long *>(opts->stats) : nullptr,
                 opts ? opts->out_depth : nullptr,
                 opts ? opts->out_normal : nullptr,
                 opts ? reinterpret_cast<unsigned int *>(opts->out_rgba8) : nullptr,
                 opts ? exp2f(opts->exposure_ev) : 1.0f,
                 n_pix};
    cudaError_t e = cudaMemsetAsync(F->counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_fail(e, "render: reset counter");
    if (prec == VRNERF_FP32)
        e = launch_render_simt(F->view, src, ro, reinterpret_cast<unsigned long long *>(F->counter), st);
    else
        e = launch_render_tc(F, src, ro, prec, st);
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    return VRNERF_OK;
}

int vrnerf_render(vrnerf_field *F, const float *cameras, const float *intrinsics,
                  const int32_t *resolution_host, int32_t n, float *out,
                  const vrnerf_render_opts *opts, void *stream) {
    ABI_GUARD_BEGIN
    NvtxRange nvtx_range("vrnerf_render");
    if (!F || !cameras || !intrinsics || !out) return fail(VRNERF_EINVAL, "NULL argument");
    long long rays = 0;
    int rc = check_views(resolution_host, n, rays);
    if (rc) return rc;
    RaySource *src = &F->src_scratch;
    make_camera_source(cameras, intrinsics, resolution_host, n, *src);
    return render_common(F, *src, out, opts, (cudaStream_t)stream, rays);
    ABI_GUARD_END
}

int vrnerf_render_host(vrnerf_field *F, const float *cameras_host, const float *intrinsics_host,
                       const int32_t *resolution_host, int32_t n, float *out_host,
                       const vrnerf_render_opts *opts, void *stream) {
    ABI_GUARD_BEGIN
    NvtxRange nvtx_range("vrnerf_render_host");
    if (!F || !cameras_host || !intrinsics_host || !out_host) return fail(VRNERF_EINVAL, "NULL argument");
    long long rays = 0;
    int rc = check_views(resolution_host, n, rays);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cam_bytes = (size_t)n * 16 * sizeof(float);
    const size_t out_bytes = (size_t)rays * 3 * sizeof(float);
    // pinned host memory the GPU can address: the kernel writes the image
    // there itself, overlapping the transfer with the render (no staging
    // buffer, no copy after the kernel); pageable memory goes through staging
    float *out_dev = nullptr;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
        out_dev = static_cast<float *>(pa.devicePointer);
    else
        cudaGetLastError();
    if ((rc = F->ensure_staging(cam_bytes, out_dev ? 0 : out_bytes))) return rc;
    cudaError_t e = cudaMemcpyAsync(F->stage_cam, cameras_host, (size_t)n * 12 * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(F->stage_cam + (size_t)n * 12, intrinsics_host, (size_t)n * 4 * 4,
                            cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "render_host: upload");
    RaySource *src = &F->src_scratch;
    make_camera_source(F->stage_cam, F->stage_cam + (size_t)n * 12, resolution_host, n, *src);
    vrnerf_render_opts o2{};
    if (opts) o2.precision = opts->precision;
    if ((rc = render_common(F, *src, out_dev ? out_dev : F->stage_out, &o2, st, rays))) return rc;
    if (!out_dev) e = cudaMemcpyAsync(out_host, F->stage_out, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "render_host: download");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_render_rays(vrnerf_field *F, const float *o, const float *d, const float *r, int32_t B,
                       float *out, const vrnerf_render_opts *opts, void *stream) {
    ABI_GUARD_BEGIN
    NvtxRange nvtx_range("vrnerf_render_rays");
    if (!F || !o || !d || !r || !out) return fail(VRNERF_EINVAL, "NULL argument");
    if (B < 1) return fail(VRNERF_EINVAL, "B must be >= 1");
    RaySource *src = &F->src_scratch;
    memset(src, 0, sizeof *src);
    src->o = o;
    src->d = d;
    src->r = r;
    src->n_slots = B;
    return render_common(F, *src, out, opts, (cudaStream_t)stream, B);
    ABI_GUARD_END
}

int vrnerf_query(vrnerf_field *F, const float *pos, const float *dir, const float *radius, int32_t n,
                 float *sigma, float *rgb, float *feat, int32_t precision, void *stream) {
    ABI_GUARD_BEGIN
    if (!F || !pos || !dir || !radius || !sigma || !rgb) return fail(VRNERF_EINVAL, "NULL argument");
    if (n < 1) return fail(VRNERF_EINVAL, "n must be >= 1");
    int rc = check_precision(precision);
    if (rc) return rc;
    cudaError_t e;
    if (precision == VRNERF_FP32)
        e = launch_query_simt(F->view, pos, dir, radius, n, sigma, rgb, feat, (cudaStream_t)stream);
    else
        e = launch_query_tc(F, pos, dir, radius, n, sigma, rgb, feat, precision, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "query");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_debug_march(vrnerf_field *F, const float *o, const float *d, int32_t B, int32_t cap,
                       int32_t *rec_i, int32_t *rec_vox, int32_t *count, void *stream) {
    ABI_GUARD_BEGIN
    if (!F || !o || !d || !count || (cap > 0 && (!rec_i || !rec_vox)))
        return fail(VRNERF_EINVAL, "NULL argument");
    if (B < 1 || cap < 0) return fail(VRNERF_EINVAL, "B must be >= 1 and cap >= 0");
    cudaError_t e = launch_debug_march(F->view, o, d, B, cap, rec_i, rec_vox, count, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "debug_march");
    return VRNERF_OK;
    ABI_GUARD_END
}

int vrnerf_debug_corners(vrnerf_field *F, const float *pos, int32_t n, uint32_t *idx, void *stream) {
    ABI_GUARD_BEGIN
    if (!F || !pos || !idx) return fail(VRNERF_EINVAL, "NULL argument");
    if (n < 1) return fail(VRNERF_EINVAL, "n must be >= 1");
    cudaError_t e = launch_debug_corners(F->view, pos, n, idx, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "debug_corners");
    return VRNERF_OK;
    ABI_GUARD_END
}

}  // extern "C"
