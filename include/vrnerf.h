/*
 * vrnerf.h -- C ABI of the GB300 (sm_103a) renderer of VR-NeRF's field
 * ("VR-NeRF: High-Fidelity Virtualized Walkable Spaces", SIGGRAPH Asia 2023).
 *
 * The library renders an instant-NGP-style radiance field per ray: pinhole
 * ray generation, a march through a binary occupancy grid (Sec. 4.3),
 * multiresolution hash-grid features weighted by the level-of-detail scheme
 * of Sec. 4.2.1 (Eq. 3) with an optional LOD bias (Sec. 4.2.2), a density MLP
 * and a colour MLP (Sec. 6; the in-register tensor-core MLP of Sec. 5),
 * sigmoid colour in the PQ perceptual space (Sec. 4.1), front-to-back
 * compositing with early termination, and PQ decoding (Eq. 1-2) to linear
 * colour (1.0 = 100 cd/m^2). It also trains the field: the L1 loss in PQ
 * space (Sec. 4.1; supplement "Loss Design") back-propagated through the
 * compositor, the MLPs and the hash grid, and the Adam step of Sec. 6.
 *
 * Conventions for every entry point:
 *  - Return value: VRNERF_OK (0) or a negative VRNERF_E* code. The message
 *    of the last failure on the calling thread is vrnerf_last_error().
 *    No C++ exception crosses this interface.
 *  - Pointers named *_host are host memory; every other array pointer is
 *    device memory of the current CUDA device. The caller owns all buffers
 *    it passes; the library never frees or keeps them past the call (except
 *    where an entry point says so).
 *  - A field owns its device parameters, occupancy bits and scratch memory,
 *    allocated on the device that is current at vrnerf_field_create.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and is asynchronous unless stated otherwise: outputs are valid
 *    once the stream has been synchronised. Sizes and shapes are validated
 *    on the host before anything is launched; a rejected call enqueues
 *    nothing.
 *  - A field is not thread-safe: calls on one field must not overlap in
 *    time on different host threads, and work of different calls on one
 *    field must not run concurrently on different streams.
 *
 * Layouts:
 *  - hash grid [L][T][F], F contiguous, fp32 or IEEE fp16 (feat_fp16); every
 *    level holds T = 2^log2_T slots, dense levels use the first (N_l+1)^3.
 *  - MLP weights fp32, [out][in] row-major, concatenated W1 (64 x L*F),
 *    W2 (16 x 64), W3 (64 x 32), W4 (64 x 64), W5 (3 x 64); no biases.
 *  - occupancy bits: voxel (x, y, z) -> i = x + rx*(y + ry*z), word i >> 5,
 *    bit i & 31 (uint32 words).
 *  - cameras [n][3][4] fp32 camera-to-world (columns right, down, forward,
 *    centre; the camera looks down its +z axis); intrinsics [n][4] fp32
 *    (fx, fy, cx, cy) in pixels; resolution [n][2] int32 (W, H).
 *  - image outputs are packed per view, row-major, RGB interleaved: view v
 *    starts at pixel sum_{u<v} W_u*H_u.
 */
#ifndef VRNERF_H
#define VRNERF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VRNERF_OK 0
#define VRNERF_EINVAL (-1)    /* bad argument, shape or size */
#define VRNERF_ENOMEM (-2)    /* device or host allocation failed */
#define VRNERF_ECUDA (-3)     /* a CUDA call or kernel launch failed */
#define VRNERF_ETIMEDOUT (-4) /* a bounded wait ran out */
#define VRNERF_EBUSY (-5)     /* admission refused: over budget or queue full */
#define VRNERF_ENOTFOUND (-6) /* unknown ticket */
#define VRNERF_ECANCELED (-7) /* request was cancelled */
#define VRNERF_ECHECK (-8)    /* a bounds check of the checked build failed */
#define VRNERF_ELATE (-9)     /* request shed: its deadline passed before it reached the GPU */

/* Arithmetic of the MLP. Hash features, transmittance and PQ are always fp32. */
#define VRNERF_FP32 0 /* plain fp32 on the CUDA cores */
#define VRNERF_FP16 1 /* fp16 operands, fp32 accumulate, tcgen05 tensor cores */
#define VRNERF_BF16 2 /* bf16 operands, fp32 accumulate, tcgen05 tensor cores */
#define VRNERF_FP8 3  /* e4m3 hidden layers, fp16 first/last layers, fp32 accumulate */

#define VRNERF_MAX_LEVELS 16
#define VRNERF_MAX_VIEWS 256

typedef struct vrnerf_field vrnerf_field;

/* Field description. The MLP widths are fixed to the paper's (Sec. 6):
 * d_hidden = 64, d_out = 16, c_hidden = 64, c_layers = 2; levels * feats
 * must be 16 or 32 with feats = 2. Level l has resolution
 * N_l = floor(base_res * growth^l + 1e-6) and is dense when
 * (N_l + 1)^3 <= 2^log2_T, else hashed (instant-NGP spatial hash).
 * Samples sit at t_i = t_near (t_far / t_near)^(i / max_steps), i <
 * max_steps (Sec. 6: exponential distances); the march ends at the first
 * sample outside the occupancy grid's box [aabb_min, aabb_max]. Hash-grid
 * coordinates are (p - aabb_min) / max extent. The ray's base radius is
 * radius_scale / fx; L* = -log_growth(2 base_res r t / max extent) +
 * lod_bias (Eq. 3, Sec. 4.2.2). sigma = exp(o_0 + density_bias).
 * Compositing stops after the sample where transmittance < T_eps.
 * occ_res: occupancy voxels per axis, each in [1, 2048], fewer than 2^31 in
 * all (Sec. 4.3).
 * contract = 1 makes the scene unbounded (Sec. 4: L-infinity cubic
 * contraction): x = (p - centre) / h with the box's centre and half its
 * largest extent h, y = x for |x|_inf <= 1, else (2 - 1/|x|_inf) x / |x|_inf;
 * the hash grid and the occupancy grid span y in [-2, 2]^3 (normalised
 * position y / 4 + 1/2), the march runs to t_far, and the footprint of a
 * camera ray is the distance to its adjacent pixels' rays in contracted
 * space (Sec. 4.2.1), of an explicit ray t r det(J_C)^(1/3). */
typedef struct {
    int32_t levels, feats, log2_T, feat_fp16;
    double base_res, growth;
    int32_t d_hidden, d_out, c_hidden, c_layers;
    float aabb_min[3], aabb_max[3];
    int32_t occ_res[3];
    int32_t max_steps;
    float t_near, t_far;
    float lod_bias, T_eps, radius_scale, density_bias;
    int32_t contract; /* 0: bounded box, 1: unbounded (contracted) scene */
    int32_t reserved;
} vrnerf_field_desc;

/* Optional per-call render settings (NULL = fp32 MLP, linear output only). */
typedef struct {
    int32_t precision; /* VRNERF_FP32 / FP16 / BF16 / FP8 */
    int32_t reserved;
    float *out_pq;     /* optional [rays][3] PQ-space colour before decoding */
    float *out_T;      /* optional [rays] final transmittance */
    int32_t *out_n;    /* optional [rays] number of composited samples */
    uint64_t *stats;   /* optional [4] counters, added to (not reset): evaluated
                          samples, hash-grid levels fetched, march steps tested,
                          rays finished */
    float *out_depth;  /* optional [rays] expected distance sum_i w_i t_i of the
                          composited samples (divide by 1 - T for the distance
                          of the visible surface); the depth maps of the
                          paper's renders. */
    float *out_normal; /* optional [rays][3] composited normal sum_i w_i n_i,
                          n_i = -grad sigma / |grad sigma| at the sample's
                          position (fixed footprint); the normal maps of the
                          paper's renders. VRNERF_FP32 only (EINVAL otherwise). */
    uint32_t *out_rgba8; /* optional [rays] display pixels: sRGB (IEC 61966-2-1)
                          of clamp(linear 2^exposure_ev, 0, 1), 8 bits per
                          channel rounded half up, alpha = 1 - T; packed
                          R | G << 8 | B << 16 | A << 24 (the exposure sweep
                          of the paper's tonemapping from PQ to sRGB). */
    float exposure_ev; /* exposure in stops for out_rgba8 (0: 100 cd/m^2 = white) */
    int32_t reserved2;
} vrnerf_render_opts;

/* Message of the last failed call on this thread ("" if none). */
const char *vrnerf_last_error(void);

/* Bytes of the hash grid, floats of the MLP and uint32 words of the
 * occupancy bits that a description needs. Any output may be NULL.
 * EINVAL for an unsupported description. */
int vrnerf_field_sizes(const vrnerf_field_desc *desc, uint64_t *grid_bytes, uint64_t *mlp_floats,
                       uint64_t *occ_words);

/* Creates a field on the current device (Sec. 4, the model of Sec. 6).
 * grid_host / mlp_host: initial parameters in the layouts above, or NULL to
 * draw them from `seed` with the library's SplitMix64 stream (grid
 * U(-1e-2, 1e-2), Xavier-uniform weights). occ_bits_host: required.
 * *out receives the field; destroy it with vrnerf_field_destroy.
 * Synchronous. EINVAL, ENOMEM, ECUDA. */
int vrnerf_field_create(const vrnerf_field_desc *desc, const void *grid_host, const float *mlp_host,
                        const uint32_t *occ_bits_host, uint64_t seed, vrnerf_field **out);

/* VRNERF_OK, or the error a kernel of this field recorded since the last
 * call (VRNERF_ETIMEDOUT when a bounded device-side wait of the tensor-core
 * kernels ran out; the kernel then stopped early and its output is
 * incomplete), and clears it. Synchronises the field's device. */
int vrnerf_field_status(vrnerf_field *field);

/* Frees the field and all its device memory (synchronises its device). */
void vrnerf_field_destroy(vrnerf_field *field);

/* Copies the current parameters (after training) to host buffers of the
 * sizes vrnerf_field_sizes gives; either may be NULL. Synchronous. */
int vrnerf_field_get_params(vrnerf_field *field, void *grid_host, float *mlp_host);

/* Checkpoint (no counterpart in the paper): writes the description, the
 * hash grid, the MLP weights, the occupancy bits and, after training, the
 * Adam step count, moments and fp32 master grid to one flat little-endian
 * file ("VRNF" header, version 1, then the arrays in that order).
 * Synchronous. EINVAL (NULL argument, file cannot be written), ECUDA. */
int vrnerf_field_save(vrnerf_field *field, const char *path);

/* Creates a field on the current device from a file written by
 * vrnerf_field_save, Adam state included, so training resumes where it
 * stopped. Synchronous. EINVAL (unreadable or malformed file), ENOMEM, ECUDA. */
int vrnerf_field_load(const char *path, vrnerf_field **out);

/* Replaces the occupancy bits (Sec. 4.3). Synchronous. */
int vrnerf_field_set_occupancy(vrnerf_field *field, const uint32_t *occ_bits_host);

/* Renders n views (Sec. 5): cameras / intrinsics in device memory,
 * resolution_host in host memory, out = device [sum W*H][3] linear colour
 * (1.0 = 100 cd/m^2), decoded from PQ per channel (Eq. 1-2). n <=
 * VRNERF_MAX_VIEWS, W, H in [1, 16384], fx, fy > 0. EINVAL, ECUDA. */
int vrnerf_render(vrnerf_field *field, const float *cameras, const float *intrinsics,
                  const int32_t *resolution_host, int32_t n, float *out,
                  const vrnerf_render_opts *opts, void *stream);

/* vrnerf_render (Sec. 5) with every array in host memory: copies the cameras in and
 * the image out on `stream` through the field's device staging buffers and
 * returns after the stream has finished (synchronous). When out_host is
 * pinned host memory the GPU can address (cudaHostAlloc / cudaHostRegister,
 * mapped), the kernel writes the image into it directly and no staging
 * buffer or copy is used; the values are the same. The optional outputs of
 * opts are ignored. EINVAL, ENOMEM, ECUDA. */
int vrnerf_render_host(vrnerf_field *field, const float *cameras_host, const float *intrinsics_host,
                       const int32_t *resolution_host, int32_t n, float *out_host,
                       const vrnerf_render_opts *opts, void *stream);

/* Renders B explicit rays: origins / unit directions [B][3], base radii [B]
 * (footprint radius at unit distance, Sec. 4.2.1), device memory;
 * out [B][3] linear colour. EINVAL, ECUDA. */
int vrnerf_render_rays(vrnerf_field *field, const float *rays_o, const float *rays_d,
                       const float *radii, int32_t B, float *out, const vrnerf_render_opts *opts,
                       void *stream);

/* Evaluates the field at n points (Sec. 4.2.1 and Sec. 6): world positions
 * [n][3], unit directions [n][3], footprint radii [n] in world units (t r).
 * Outputs: sigma [n], PQ colour rgb [n][3], optional LOD-weighted features
 * feat [n][L*F] (may be NULL). Points outside the box are clamped to the
 * grid's edge cells. precision as in vrnerf_render_opts. EINVAL, ECUDA. */
int vrnerf_query(vrnerf_field *field, const float *pos, const float *dir, const float *radius,
                 int32_t n, float *sigma, float *rgb, float *feat, int32_t precision, void *stream);

/* Occupancy visits (Sec. 4.3) of B explicit rays, without early
 * termination: for ray b, the step index i and voxel index of each
 * evaluated sample in order, into rec_i / rec_vox [B][cap] (records past
 * cap are dropped), and count [B] = the full number. Device memory.
 * EINVAL, ECUDA. */
int vrnerf_debug_march(vrnerf_field *field, const float *rays_o, const float *rays_d, int32_t B,
                       int32_t cap, int32_t *rec_i, int32_t *rec_vox, int32_t *count, void *stream);

/* Hash-grid corner indices (Sec. 4, instant-NGP encoding; dense coarse
 * levels per the supplement) of n world positions: idx [n][L][8], corner b
 * at offset (b & 1, b >> 1 & 1, b >> 2 & 1). Device memory. EINVAL, ECUDA. */
int vrnerf_debug_corners(vrnerf_field *field, const float *pos, int32_t n, uint32_t *idx,
                         void *stream);

/* Training (Sec. 6; Sec. 4.1 and supplement "Loss Design"): renders B
 * explicit rays, and computes loss = mean over rays and channels of
 * |C_pq - PQ(target / 100)| and its gradient with respect to every hash-grid
 * entry and MLP weight into the field's gradient buffers (overwritten).
 * target_linear [B][3] device memory. loss_host (may be NULL) receives the
 * loss. The batch runs sample-parallel: rays are marched and their samples
 * listed, evaluated one thread per sample, composited per ray, and
 * back-propagated one thread per sample (recomputing features and
 * activations). The call waits for `stream` once (the sample count sizes
 * its buffers). EINVAL, ENOMEM, ECUDA. */
int vrnerf_backward(vrnerf_field *field, const float *rays_o, const float *rays_d,
                    const float *radii, const float *target_linear, int32_t B, float *loss_host,
                    void *stream);

/* The forward of the training path for explicit rays (Sec. 4.1, Sec. 6):
 * PQ colour out_pq [B][3] and composited sample count out_n [B] (the render
 * of vrnerf_render_rays with VRNERF_FP32, early termination included),
 * computed sample-parallel like vrnerf_backward, so that small batches fill
 * the GPU. Device memory; waits for `stream` once. EINVAL, ENOMEM, ECUDA. */
int vrnerf_forward_rays(vrnerf_field *field, const float *rays_o, const float *rays_d,
                        const float *radii, int32_t B, float *out_pq, int32_t *out_n, void *stream);

/* Backward for an arbitrary loss on the PQ colours (the hand-written
 * backward behind an autograd function): the gradient of
 * sum_i grad_pq[i] . C_pq(ray i) with respect to every hash-grid entry and
 * MLP weight into the field's gradient buffers (overwritten). n_fwd [B] are
 * the sample counts that vrnerf_forward_rays (or vrnerf_render_rays with
 * VRNERF_FP32) returned for the same rays and parameters: ray i composites
 * exactly n_fwd[i] samples, as in that forward pass; samples are recomputed, only sigma, colour and their
 * gradients are kept per sample. All arrays device memory; the call waits
 * for `stream` once (the sample count sizes its buffers). EINVAL, ENOMEM,
 * ECUDA. */
int vrnerf_backward_from_grad(vrnerf_field *field, const float *rays_o, const float *rays_d,
                              const float *radii, int32_t B, const int32_t *n_fwd,
                              const float *grad_pq, void *stream);

/* Most samples one pass of the training pipeline (vrnerf_backward,
 * vrnerf_train_step, vrnerf_forward_rays, vrnerf_backward_from_grad) holds
 * at once; 0 restores the default (2^26). The pipeline keeps per-sample
 * buffers on the device: 152 bytes per evaluated sample, 216 with the bf16
 * training precision. A batch with more samples than the budget, or whose
 * buffers cannot be allocated, is processed in ray ranges that fit, one
 * after the other, with gradients, loss and history accumulated over them:
 * the same result as one pass up to the order of float additions. ENOMEM
 * only when a single ray's samples do not fit. No counterpart in the paper
 * (Sec. 6 trains on 12 800 rays per step). EINVAL for a NULL field. */
int vrnerf_field_set_sample_budget(vrnerf_field *field, uint64_t max_samples);

/* Arithmetic of the MLPs in training (Sec. 6, A9): VRNERF_FP32 (default;
 * CUDA cores, gradients within 1e-4 of the fp64 reference) or VRNERF_BF16
 * (tcgen05 tensor cores for the per-sample forward and backward: bf16
 * features, activations, deltas and weights, fp32 accumulation; the
 * compositing, the loss and the hash-grid scatter stay fp32). Applies to
 * vrnerf_backward, vrnerf_train_step and vrnerf_backward_from_grad
 * (vrnerf_forward_rays stays fp32). EINVAL for other precisions. */
int vrnerf_field_set_train_precision(vrnerf_field *field, int32_t precision);

/* Device pointers of the field's parameters ([L][T][F] grid in its storage
 * type, fp32 MLP) and fp32 gradient buffers (allocated on the first call
 * that asks for them), valid until vrnerf_field_destroy; any output may be
 * NULL. For frameworks that view them as tensors. A caller that writes the
 * parameters must then call vrnerf_field_params_changed, which refreshes the
 * derived copies (tensor-core weight images, the fp32 master of an fp16
 * grid). EINVAL, ENOMEM. */
int vrnerf_field_param_ptrs(vrnerf_field *field, void **grid, float **mlp, float **grid_grad,
                            float **mlp_grad);
int vrnerf_field_params_changed(vrnerf_field *field);

/* Checked builds (libvrnerf_checked.so, compiled with VRNERF_CHECKED=1)
 * verify hash-grid indices, occupancy voxels, sample indices, output pixels
 * and training records on the device; a failed check sets a bit that the
 * next vrnerf_field_status reports as VRNERF_ECHECK, and the access is
 * skipped or clamped (no trap). vrnerf_build_checked returns 1 in such a
 * build, else 0. vrnerf_debug_check_trigger sets the test bit (32) through
 * a kernel, so that the reporting path can be tested; EINVAL in release
 * builds. */
int vrnerf_build_checked(void);
int vrnerf_debug_check_trigger(vrnerf_field *field, void *stream);

/* Display tonemapping of an existing PQ image (Sec. 4.1: the exposure sweep
 * at rendering time; Sec. 6 evaluates in tonemapped sRGB): PQ colour to sRGB
 * at a chosen exposure, without re-rendering. pq [n][3] and optional T [n] (NULL: alpha 255) in device
 * memory; rgba8 [n] as vrnerf_render_opts.out_rgba8. Asynchronous on
 * `stream`. EINVAL (n < 0, NULL pointers), ECUDA. */
int vrnerf_tonemap(const float *pq, const float *T, int64_t n, float exposure_ev, uint32_t *rgba8,
                   void *stream);

/* Occupancy-grid pruning (Sec. 4.3.2). vrnerf_history_reset allocates (on
 * the first call) and zeroes the field's training history: from then on
 * every vrnerf_backward records, per occupancy voxel, the largest opacity
 * 1 - exp(-sigma delta) of the samples it composites there.
 * vrnerf_field_get_history copies it to hist_host [voxels] (synchronous). */
int vrnerf_history_reset(vrnerf_field *field);
int vrnerf_field_get_history(vrnerf_field *field, float *hist_host);

/* Joint history- and grid-based pruning (Sec. 4.3.2). For every occupied
 * voxel: the largest density over the points_per_axis^3 sub-cell centres
 * (full detail), as an opacity with the smallest sample spacing a training
 * ray has there (the exponential spacing at the distance from the nearest of
 * the n_cameras camera centres, host [n][3], to the voxel). A voxel stays
 * occupied iff that opacity or its recorded history reaches `threshold`
 * (the paper anneals it from 0 to 0.2). Optional outputs, device memory:
 * alpha_out [voxels] the grid opacity, occ_bits_out the new bits; kept_host
 * the number of voxels kept. apply != 0 replaces the field's occupancy and
 * rebuilds its distance field. Synchronous. EINVAL, ENOMEM, ECUDA. */
int vrnerf_prune(vrnerf_field *field, const float *camera_centres_host, int32_t n_cameras,
                 int32_t points_per_axis, float threshold, int32_t apply, float *alpha_out,
                 uint32_t *occ_bits_out, uint64_t *kept_host);

/* Refines the occupancy grid by an integer factor in [2, 8] per axis
 * (Sec. 4.3.2: a coarse grid upsampled at training milestones): every child
 * voxel takes its parent's bit and, if a history is kept, its history value;
 * the field's occ_res is multiplied by factor and its distance field
 * rebuilt. Synchronous; no render, training call or server may be using the
 * field meanwhile. EINVAL (factor, resulting occ_res), ENOMEM, ECUDA; on an
 * error the field is unchanged. */
int vrnerf_occupancy_upsample(vrnerf_field *field, int32_t factor);

/* Copies the field's occupancy bits (layout of vrnerf_field_create) to
 * occ_bits_host [ceil(voxels / 32)] words. Synchronous. EINVAL, ECUDA. */
int vrnerf_field_get_occupancy(vrnerf_field *field, uint32_t *occ_bits_host);

/* Copies the gradient buffers of the last vrnerf_backward to the host:
 * grid_grad_host [L][T][F] fp32, mlp_grad_host fp32 (either may be NULL).
 * Synchronous. */
int vrnerf_field_get_grads(vrnerf_field *field, float *grid_grad_host, float *mlp_grad_host);

/* One Adam step (Sec. 6: beta1 = 0.9, beta2 = 0.99, eps = 1e-15) on all
 * parameters from the gradient buffers; learning rate lr_grid for the hash
 * grid and lr_mlp for the MLP weights (paper: 0.01 and 0.005). The field
 * keeps fp32 master weights and the first and second moments. */
int vrnerf_adam_step(vrnerf_field *field, float lr_grid, float lr_mlp, void *stream);

/* vrnerf_backward followed by vrnerf_adam_step: one training iteration of
 * Sec. 6. */
int vrnerf_train_step(vrnerf_field *field, const float *rays_o, const float *rays_d,
                      const float *radii, const float *target_linear, int32_t B, float lr_grid,
                      float lr_mlp, float *loss_host, void *stream);

/* Loads a gradient buffer from the host into the field (for testing the
 * optimiser on given gradients). Synchronous. */
int vrnerf_field_set_grads(vrnerf_field *field, const float *grid_grad_host,
                           const float *mlp_grad_host);

/* Failure detection without a GPU fault (no counterpart in the paper):
 * launches one CTA that allocates TMEM and waits, through the same bounded
 * mbarrier wait the tensor-core kernels use, on an mbarrier that nothing
 * completes. After limit_us microseconds it gives up, records
 * VRNERF_ETIMEDOUT in the field's status word, frees its TMEM and returns;
 * vrnerf_field_status then reports ETIMEDOUT and the context stays usable.
 * limit_us in [1, 2000000]. EINVAL, ECUDA. */
int vrnerf_debug_wait_timeout(vrnerf_field *field, uint32_t limit_us, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of render requests (stereo eye pairs and
 * single views of any resolution) through one persistent tensor-core render
 * kernel that keeps the field resident and takes rays of newly admitted
 * requests while earlier ones are still on the GPU; the interactive VR
 * rendering of Sec. 5 on one GPU.
 * ------------------------------------------------------------------------- */
typedef struct vrnerf_server vrnerf_server;

typedef struct {
    uint64_t completed;        /* requests finished since the last reset */
    uint64_t rays;             /* their rays */
    uint64_t kernel_launches;  /* persistent-kernel launches (it leaves when idle) */
    uint64_t pending, inflight;
    double p50_ms, p99_ms, max_ms; /* submit-to-output-on-host latency */
    double wall_s;             /* since the first request after the last reset */
    uint64_t max_inflight;     /* most requests admitted to the GPU at once since the last reset */
    uint64_t tile_rounds;      /* 128-row MLP tiles the kernel has run since the server
                                  was created (updated as requests finish) */
    uint64_t mixed_tile_rounds; /* of those, tiles whose rows held samples of two or more
                                   requests: work of different requests overlapping on the
                                   device, in the same tensor-core MMAs */
    uint64_t late;             /* requests with a deadline that finished after it */
    uint64_t shed;             /* requests dropped because their deadline passed first */
    double wait_p50_ms, wait_p99_ms; /* submit to admission (queueing for budget or ring) */
    double gpu_p50_ms, gpu_p99_ms;   /* admission to every ray rendered */
    double copy_p50_ms, copy_p99_ms; /* rendered to output in host memory */
} vrnerf_serve_stats;

/* Serving (Sec. 5: real-time rendering of stereo eye buffers, here as
 * continuous batching on one GPU). Starts a server for `field` on its
 * device: a scheduler thread, two streams and an output arena of
 * hbm_budget_bytes on the device. A request is admitted when its output
 * (12 bytes per ray; none for an output in pinned host memory) fits in the arena's free space and the in-flight views
 * fit the server's view ring (256); otherwise it waits in arrival order. precision: VRNERF_FP16 or VRNERF_BF16. The server
 * owns the field until vrnerf_server_destroy: make no other call on the
 * field meanwhile. EINVAL, ENOMEM. */
int vrnerf_server_create(vrnerf_field *field, uint64_t hbm_budget_bytes, int32_t precision,
                         vrnerf_server **out);

/* Queues a request of n_views (1..16) views; every array is host memory and
 * is copied, except out_host ([sum W*H][3] linear colour, may be NULL),
 * which must stay valid until vrnerf_poll reports the request. When out_host
 * is pinned (page-locked) host memory that the device can address, the
 * kernel writes the pixels into it directly: such a request takes no part
 * of the HBM budget and has no copy-out (a cancelled request that is
 * already running may still write its pixels); other outputs are rendered
 * into the budget's arena and copied out. Non-blocking. *ticket identifies
 * the request. EINVAL (bad view, or an arena output larger than the whole
 * budget), EBUSY (1024 requests already waiting). */
int vrnerf_submit(vrnerf_server *server, int32_t n_views, const float *cameras_host,
                  const float *intrinsics_host, const int32_t *resolution_host, float *out_host,
                  uint64_t *ticket);

/* vrnerf_submit with a deadline (Sec. 6.2 paces stereo frames at 36 Hz and
 * reports p99 frame rates): the request is due deadline_ms after submission
 * (0: no deadline). Waiting requests are admitted earliest deadline first;
 * requests without one follow in arrival order. With shed_if_late != 0 a
 * request still waiting when its deadline passes is dropped (vrnerf_poll
 * returns VRNERF_ELATE); otherwise it runs and, if it finishes after its
 * deadline, counts as late in vrnerf_serve_stats. EINVAL, EBUSY as
 * vrnerf_submit. */
int vrnerf_submit_deadline(vrnerf_server *server, int32_t n_views, const float *cameras_host,
                           const float *intrinsics_host, const int32_t *resolution_host, float *out_host,
                           double deadline_ms, int32_t shed_if_late, uint64_t *ticket);

/* Waits up to timeout_ms for the request; VRNERF_OK when its output is in
 * out_host (the ticket is then released; *latency_ms, if non-NULL, gets the
 * submit-to-done time), ETIMEDOUT if not yet done, ECANCELED if it was
 * cancelled (ticket released), ELATE if it was shed (ticket released),
 * ENOTFOUND for an unknown ticket. */
int vrnerf_poll(vrnerf_server *server, uint64_t ticket, int32_t timeout_ms, double *latency_ms);

/* Cancels a request: a waiting request is dropped, a running one finishes on
 * the GPU but its output is not copied (an output in pinned host memory,
 * written directly, may already hold pixels). Poll it to release the
 * ticket. */
int vrnerf_cancel(vrnerf_server *server, uint64_t ticket);

/* Latency percentiles and throughput of the requests finished so far. */
int vrnerf_server_stats(vrnerf_server *server, vrnerf_serve_stats *out);
int vrnerf_server_reset_stats(vrnerf_server *server);

/* Stops the scheduler, lets the kernel drain and frees the server. */
void vrnerf_server_destroy(vrnerf_server *server);

/* The fp32 render of vrnerf_render for callers that cannot allocate GPU
 * memory: it calls no cudaMalloc, cudaFree or other allocating routine.
 * The paper has no counterpart; this exists for callers such as a VR
 * compositor's frame callback, where an allocation could stall the frame,
 * or a plug-in whose host application owns every device allocation.
 * The caller passes the field's parameters in device buffers it owns, in the
 * layouts above, of exactly these sizes (the library sees only pointers and
 * cannot check them): grid L * 2^log2_T * F elements, fp16 when feat_fp16
 * else fp32; mlp 64 L F + 16*64 + 64*32 + 64*64 + 3*64 fp32 weights;
 * occ_bits ceil(rx ry rz / 32) words; cameras [n][3][4], intrinsics [n][4]
 * and out [sum W*H][3] as in vrnerf_render (device), resolution_host on the
 * host. With no distance field (it would need device memory of its own) the
 * march tests every sample against the occupancy bits instead of skipping
 * empty space: the same result as vrnerf_render, with more march work on
 * sparse scenes. The kernel's scratch (ray-slot counter and sample-distance
 * table) lives in one 32 KiB static device array that every GPU loading the
 * library keeps until the process exits; its address is looked up on the
 * first call made on each device (make that call outside stream capture),
 * and the table is copied in again only when t_near, t_far or max_steps
 * differ from the previous call on that device. max_steps above 8127 is
 * rejected with EINVAL. Calls share the scratch: calls whose work overlaps on
 * the GPU race, so order them on one stream. EINVAL, ECUDA. */
int vrnerf_render_noalloc(const vrnerf_field_desc *desc, const void *grid, const float *mlp,
                          const uint32_t *occ_bits, const float *cameras, const float *intrinsics,
                          const int32_t *resolution_host, int32_t n, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VRNERF_H */
