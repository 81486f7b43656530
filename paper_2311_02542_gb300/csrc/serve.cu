// serve.cu -- continuous-batching render server.
//
// The paper renders each VR frame as soon as it is asked for (Sec. 5: dual
// 2K x 2K eye buffers at interactive rates); on one GB300 a stream of stereo
// and single-view requests of mixed resolution is served by ONE persistent
// tensor-core render kernel that keeps the field resident and takes work as
// it arrives:
//  - the host scheduler admits waiting requests earliest deadline first
//    (requests without a deadline in arrival order) when the output fits in
//    the HBM budget (a pre-allocated arena) and the view ring has room,
//    copies its views (camera, intrinsics, resolution, output slice) into a
//    ring in device memory and then the number of published views into a
//    control block in device memory, in stream order;
//  - the kernel's warps take ray slots by fetch-and-add on the slot counter of
//    the oldest published view that still has slots (a monotonic view cursor
//    skips exhausted views; overshoot on an exhausted view is ignored). Rays
//    of different requests share 128-row MLP tiles, so requests that arrive
//    while others are on the GPU overlap with them on the device;
//  - every thread counts the slots it finished per view and adds them to
//    that view's counter in device memory after a fence; the thread that
//    completes the view raises the view's flag in host-mapped memory after a
//    system-scope fence, so the host sees a view complete only after its
//    output is written; the host then copies the output slice to the
//    request's buffer;
//  - when a CTA has no rays and nothing is published, it polls with
//    __nanosleep; the launch leaves as a whole once every CTA has been idle
//    past a time limit (or on stop), and the host relaunches the kernel when
//    new work arrives and none is running.
// No device-side wait is unbounded.
#include <algorithm>
#include <cstddef>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "tc_mlp.cuh"

namespace vrn {

constexpr int kRing = 256;  // views the ring holds; in-flight views stay below this

struct __align__(16) ServeView {
    float c2w[12];
    float K[4];
    int W, H, tiles_x;
    unsigned int req;      // sequence number of the request the view belongs to
    unsigned long long slot_begin, slot_end;
    float *out;            // device [W*H][3]
    unsigned int *done;    // host-mapped flag: set to the slot count when the view is finished
    unsigned long long taken;  // slots handed out (fetch-and-add; may overshoot)
    unsigned long long finished;  // slots finished (device counter)
};

// A warp's copy of the view it last took slots from (the first 104 bytes
// of ServeView: pose, intrinsics, sizes, request, slot range, output), keyed
// by the view's sequence number, so that refills from the same view read
// shared memory instead of the ring in global memory.
struct __align__(16) ViewCache {
    unsigned int words[26];
    unsigned int seq;  // view sequence number held (0xffffffff: none)
    unsigned int pad;
};

static_assert(offsetof(ServeView, W) == 64 && offsetof(ServeView, H) == 68 && offsetof(ServeView, tiles_x) == 72 &&
                  offsetof(ServeView, req) == 76 && offsetof(ServeView, out) == 96,
              "ViewCache word indices follow the ServeView layout");

struct __align__(16) ServeShared {
    int quit;
    unsigned int rmin, rmax, pad;
    ViewCache vc[kTcThreads / 32];
};
constexpr size_t kServeSharedBytes = (sizeof(ServeShared) + 15) & ~(size_t)15;

struct ServeCtl {                  // device memory, written by the host's copies
    unsigned long long published;  // ray slots published so far (statistics)
    unsigned int n_views;          // views published so far
    int stop;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_acquire_sys_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_acquire_gpu_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_gpu_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_acquire_sys_s32(const int *p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__device__ __forceinline__ T *ldcg_ptr(T *const *p) {
    return reinterpret_cast<T *>(__ldcg(reinterpret_cast<const unsigned long long *>(p)));
}

template <int L, int FMT, bool CT>
__global__ void __launch_bounds__(kTcThreads, kTcMinBlocks)
serve_kernel(const FieldView f, ServeView *__restrict__ ring, const ServeCtl *__restrict__ ctl,
             unsigned int *__restrict__ cursor, const uint4 *__restrict__ wimg,
             unsigned long long idle_ns, unsigned long long *__restrict__ status,
             unsigned long long *__restrict__ tile_stats) {
    unsigned int *idle = cursor + 1;  // idle CTAs of this launch | quitting bit
    constexpr int D = 2 * L;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *unused;
    const TcShared S = tc_setup<D, FMT>(smem, wimg, unused, nullptr, 0);
    const float *__restrict__ sT = f.t_tab;  // sample distances, read through L1
    // the serving kernel's own shared variables sit in the dynamic allocation
    // after the tensor-core carve-up (static shared memory would be padded to
    // the dynamic region's 1 KB alignment and cost a resident CTA per SM)
    ServeShared &SS = *reinterpret_cast<ServeShared *>(reinterpret_cast<unsigned char *>(S.mbar) + 64);
    int &s_quit = SS.quit;
    // smallest and largest request number among the rows of this tile round
    unsigned int &s_rmin = SS.rmin, &s_rmax = SS.rmax;
    ViewCache &vc = SS.vc[threadIdx.x >> 5];
    if ((threadIdx.x & 31) == 0) vc.seq = 0xffffffffu;
    __syncwarp();
    if (threadIdx.x == 0) {
        s_rmin = 0xffffffffu;
        s_rmax = 0u;
    }

    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    bool live = false, ok = true;
    MarchRay mr;
    float r = 0.0f, T = 1.0f, C[3] = {0, 0, 0};
    float adj[CT ? 6 : 1];  // contracted scenes: offsets to the adjacent pixels' rays
    float *dst = nullptr;
    int view = -1, cnt_view = -1;
    unsigned int my_req = 0;  // request of this thread's ray
    unsigned int cnt = 0;  // finished slots of cnt_view not yet reported
    uint32_t phase = 0;
    unsigned tested = 0;
    unsigned int nv_seen = 0;  // published views last read from the control block

    // Reports this thread's finished slots of cnt_view; the thread that
    // completes the view raises the view's host-visible flag.
    auto flush = [&]() {
        if (cnt && cnt_view >= 0) {
            ServeView *sv = ring + cnt_view;
            __threadfence_system();  // this thread's pixels (device or mapped host memory) before its count
            const unsigned long long total =
                (unsigned long long)__ldcg(&sv->tiles_x) * ((__ldcg(&sv->H) + kTileH - 1) / kTileH) * 32ull;
            if (atomicAdd(&sv->finished, (unsigned long long)cnt) + cnt == total) {
                __threadfence_system();
                atomicExch_system(ldcg_ptr(&sv->done), (unsigned int)total);
            }
        }
        cnt = 0;
    };
    auto count_slot = [&](int v) {
        if (v != cnt_view) {
            flush();
            cnt_view = v;
        }
        ++cnt;
    };
    auto finish = [&]() {
        dst[0] = pq_to_linear(C[0]);
        dst[1] = pq_to_linear(C[1]);
        dst[2] = pq_to_linear(C[2]);
        count_slot(view);
        live = false;
    };

    while (true) {
        bool have = false, starved = false;
        float p[3] = {0, 0, 0};
        while (true) {
            const bool need = !live && !starved;
            const unsigned m = __ballot_sync(FULL, need);
            if (m) {
                const int leader = __ffs(m) - 1;
                unsigned long long base = 0, got = 0;
                int v = -1;
                unsigned int vseq = 0;
                if (lane == leader) {
                    // take up to popc(m) slots from the oldest view that has any left
                    unsigned int c = atomicAdd(cursor, 0u);
                    if (c >= nv_seen) nv_seen = ld_acquire_gpu_u32(&ctl->n_views);
                    const unsigned int nv = nv_seen;
                    for (int tries = 0; tries < 2 * kRing && c < nv; ++tries) {
                        ServeView *sv = ring + (c % kRing);
                        const unsigned long long total =
                            c == vc.seq ? (unsigned long long)vc.words[18] * ((vc.words[17] + kTileH - 1) / kTileH) * 32ull
                                        : (unsigned long long)__ldcg(&sv->tiles_x) *
                                              ((__ldcg(&sv->H) + kTileH - 1) / kTileH) * 32ull;
                        const unsigned long long start = atomicAdd(&sv->taken, (unsigned long long)__popc(m));
                        if (start < total) {
                            base = start;
                            got = min((unsigned long long)__popc(m), total - start);
                            v = (int)(c % kRing);
                            vseq = c;
                            break;
                        }
                        atomicMax(cursor, c + 1);
                        c = max(c + 1, atomicAdd(cursor, 0u));
                    }
                }
                base = __shfl_sync(FULL, base, leader);
                got = __shfl_sync(FULL, got, leader);
                v = __shfl_sync(FULL, v, leader);
                vseq = __shfl_sync(FULL, vseq, leader);
                if (v >= 0 && vseq != vc.seq) {  // another view: load its descriptor once for the warp
                    __syncwarp();
                    if (lane < 26) vc.words[lane] = __ldcg(reinterpret_cast<const unsigned int *>(ring + v) + lane);
                    __syncwarp();
                    if (lane == 0) vc.seq = vseq;
                    __syncwarp();
                }
                if (need) {
                    const unsigned rank = __popc(m & ((1u << lane) - 1u));
                    if (rank >= got) {
                        starved = true;
                    } else {
                        const int q = (int)(base + rank);
                        const float *cw = reinterpret_cast<const float *>(vc.words);
                        const int W = (int)vc.words[16], H = (int)vc.words[17], tx = (int)vc.words[18];
                        const int tile = q >> 5, ln = q & 31;
                        const int px = (tile % tx) * kTileW + (ln & (kTileW - 1));
                        const int py = (tile / tx) * kTileH + (ln >> 3);
                        if (px < W && py < H) {
                            const float *c2w = cw, *K = cw + 12;
                            camera_ray(c2w, K, px, py, mr.o, mr.d);
                            if constexpr (CT) {
                                float oo[3], du[3], dv[3];
                                camera_ray(c2w, K, px + 1, py, oo, du);
                                camera_ray(c2w, K, px, py + 1, oo, dv);
#pragma unroll
                                for (int k = 0; k < 3; ++k) {
                                    adj[k] = __fsub_rn(du[k], mr.d[k]);
                                    adj[3 + k] = __fsub_rn(dv[k], mr.d[k]);
                                }
                            }
                            r = __fdiv_rn(f.radius_scale, K[0]);
                            march_init(f, mr);
                            float *vout;
                            memcpy(&vout, &vc.words[24], sizeof vout);
                            dst = vout + 3ll * ((long long)py * W + px);
                            view = v;
                            my_req = vc.words[19];
                            live = true;
                            T = 1.0f;
                            C[0] = C[1] = C[2] = 0.0f;
                        } else {
                            count_slot(v);  // padding slot of the 8x4 tiling
                        }
                    }
                }
            }
            if (live && !have) {
                const int mres = march_next(f, sT, mr, p, kTcChunk, tested);
                if (mres == MARCH_SAMPLE) have = true;
                else if (mres == MARCH_END) finish();
            }
            if (__all_sync(FULL, have || starved)) break;
        }
        if (!__syncthreads_or(have)) {
            // Nothing to shade in this CTA: report, then wait for work or stop.
            // The kernel leaves as a whole: a CTA may only quit once every CTA
            // of the launch is idle (idle[0] counts them; bit 31 marks the
            // launch as quitting, after which no CTA takes work again). A CTA
            // that left alone would shrink the kernel for as long as the
            // others stay busy, and the host relaunches only a finished kernel.
            flush();
            if (threadIdx.x == 0) {
                constexpr unsigned kQuit = 1u << 31;
                s_quit = 0;
                atomicAdd(idle, 1u);
                const uint64_t t0 = tc::globaltimer_ns();
                while (true) {
                    const uint64_t waited = tc::globaltimer_ns() - t0;
                    // after 500 idle limits a CTA quits whatever the others do
                    // (bounded wait) and takes the launch with it
                    if (ld_acquire_gpu_s32(&ctl->stop) || waited > 500ull * idle_ns) {
                        atomicOr(idle, kQuit);
                        s_quit = 1;
                        break;
                    }
                    const unsigned st = ld_acquire_gpu_u32(idle);
                    if (st & kQuit) { s_quit = 1; break; }
                    if (ld_acquire_gpu_u32(cursor) < ld_acquire_gpu_u32(&ctl->n_views)) {
                        // back to work: one unconditional decrement (a compare-and-swap
                        // here made hundreds of waking CTAs retry against each other);
                        // a launch already quitting takes this CTA with it
                        if (atomicSub(idle, 1u) & kQuit) s_quit = 1;
                        break;
                    }
                    // every CTA idle past the limit: the launch quits
                    if (waited > idle_ns && atomicCAS(idle, gridDim.x, gridDim.x | kQuit) == gridDim.x) {
                        s_quit = 1;
                        break;
                    }
                    __nanosleep(2000);
                }
            }
            __syncthreads();
            const bool quit = s_quit != 0 && !__syncthreads_or(live);
            if (quit || *S.abort) break;
            continue;
        }
        if (*S.abort) break;
        float delta = 0.0f;
        if (have) {
            const float t = sT[mr.step];
            delta = sT[mr.step + 1] - t;
            float r_norm;
            if constexpr (CT)
                r_norm = footprint(f, t, r, p, adj, adj + 3);
            else
                r_norm = t * r * f.inv_ext;
            gather_to_tile<L, FMT == 1 ? 1 : 0>(f, p, r_norm, S.act, threadIdx.x);
        } else {
            uint32_t z[D / 2];
#pragma unroll
            for (int k = 0; k < D / 2; ++k) z[k] = 0u;
            store_row<D>(S.act, threadIdx.x, z);
        }
        {
            // which requests share this tile's MLP rows (read after the MMAs'
            // barriers; reset by thread 0 before the next round's barrier)
            const unsigned lo = __reduce_min_sync(FULL, have ? my_req : 0xffffffffu);
            const unsigned hi = __reduce_max_sync(FULL, have ? my_req : 0u);
            if (lane == 0 && lo != 0xffffffffu) {
                atomicMin(&s_rmin, lo);
                atomicMax(&s_rmax, hi);
            }
        }
        float sigma, rgb[3];
        tc_mlp_any<D, FMT>(S, nullptr, mr.d, f.density_bias, sigma, rgb, phase, ok);
        if (threadIdx.x == 0) {
            atomicAdd(tile_stats, 1ull);
            if (s_rmin != s_rmax) atomicAdd(tile_stats + 1, 1ull);
            s_rmin = 0xffffffffu;
            s_rmax = 0u;
        }
        if (have) {
            const float sd = sigma * delta;
            const float w = T * (-expm1f(-sd));
            C[0] += w * rgb[0];
            C[1] += w * rgb[1];
            C[2] += w * rgb[2];
            T *= expf(-sd);
            ++mr.step;
            if (T < f.T_eps) finish();
        }
    }
    flush();
    tc_teardown(S, status);
}

template <int L, int FMT, bool CT>
static cudaError_t launch_serve_ct(vrnerf_field *F, ServeView *ring, const ServeCtl *ctl,
                                   unsigned int *cursor, unsigned long long idle_ns,
                                   unsigned long long *tile_stats, cudaStream_t st) {
    const size_t smem = tc_smem_bytes(2 * L, 0) + kServeSharedBytes;
    auto kern = serve_kernel<L, FMT, CT>;
    int bps = 0;
    cudaError_t e = prepare_tc(kern, smem, bps);
    if (e != cudaSuccess) return e;
    unsigned long long *status = reinterpret_cast<unsigned long long *>(F->counter) + 1;
    kern<<<num_sms() * bps, kTcThreads, smem, st>>>(F->view, ring, ctl, cursor,
                                                    static_cast<const uint4 *>(F->tc_w), idle_ns, status,
                                                    tile_stats);
    return cudaGetLastError();
}

template <int L, int FMT>
static cudaError_t launch_serve_t(vrnerf_field *F, ServeView *ring, const ServeCtl *ctl,
                                  unsigned int *cursor, unsigned long long idle_ns,
                                  unsigned long long *tile_stats, cudaStream_t st) {
    return F->view.contract ? launch_serve_ct<L, FMT, true>(F, ring, ctl, cursor, idle_ns, tile_stats, st)
                            : launch_serve_ct<L, FMT, false>(F, ring, ctl, cursor, idle_ns, tile_stats, st);
}

}  // namespace vrn

using namespace vrn;

// ---------------------------------------------------------------------------
// host scheduler
// ---------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int n = 0;
    std::vector<float> c2w, K;
    std::vector<int32_t> res;
    float *out_host = nullptr;
    float *out_dev = nullptr;     // out_host as the GPU addresses it, when it is mapped pinned memory
    bool zero_copy = false;       // the kernel writes the output straight into out_host
    uint64_t rays = 0, bytes = 0;
    size_t arena_off = 0;
    Clock::time_point t_submit, t_admit, t_gpu, t_done;
    Clock::time_point deadline;   // valid when has_deadline
    bool has_deadline = false;
    bool shed_if_late = false;    // drop it if the deadline passes before admission
    int views_left = 0;
    std::vector<int> ring_idx;
    cudaEvent_t copied = nullptr;
    int state = 0;  // 0 pending, 1 in flight, 2 copying, 3 done, 4 cancelled, 5 shed (late)
    bool cancel = false;
};

struct Arena {  // first-fit sub-allocator over one device buffer (the HBM budget)
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void init(size_t n) {
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(size_t n, size_t &off) {
        n = (n + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                return true;
            }
        return false;
    }
    void release(size_t off, size_t n) {
        n = (n + 255) & ~(size_t)255;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace

struct vrnerf_server {
    vrnerf_field *F = nullptr;
    int prec = VRNERF_FP16;
    uint64_t budget = 0;
    int max_pending = 1024;
    unsigned long long idle_ns = 20000000ull;
    cudaStream_t kst = nullptr, cst = nullptr;  // persistent kernel; output copies
    cudaStream_t pst = nullptr;                 // view descriptors and counters (never waits on copies)
    ServeView *ring_d = nullptr;
    ServeView *ring_h = nullptr;  // pinned staging
    ServeCtl *ctl_h = nullptr, *ctl_d = nullptr;
    unsigned int *done_h = nullptr, *done_d = nullptr;
    unsigned int *cursor = nullptr;  // device: oldest view that may have slots left
    unsigned long long *tile_stats_d = nullptr;  // device: tile rounds, rounds mixing requests
    unsigned long long *tile_stats_h = nullptr;  // pinned copy, refreshed as requests finish
    unsigned char *arena_d = nullptr;
    Arena arena;
    cudaEvent_t kernel_done = nullptr;
    bool kernel_launched = false;
    unsigned long long published = 0;
    unsigned int n_views = 0, oldest_live_view = 0;
    std::vector<unsigned long long> view_slots;  // per ring entry: slots of the view
    std::vector<Req *> view_req;                 // per ring entry
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Req *> pending;
    std::vector<Req *> inflight;
    std::map<uint64_t, Req *> by_ticket;
    std::vector<double> latencies_ms;
    std::vector<double> wait_ms, gpu_ms, copy_ms;  // per request: submit->admit, admit->rendered, ->copied
    uint64_t late = 0, shed = 0;
    uint64_t next_ticket = 1, rays_done = 0, completed = 0, launches = 0;
    uint64_t max_inflight = 0;        // most requests on the GPU at once
    unsigned int next_req = 0;        // request sequence numbers carried by the views
    Clock::time_point t_first;
    bool have_first = false;
    std::atomic<bool> quit{false};
    int error = 0;
    std::thread worker;

    void run();
    bool admit_locked(std::vector<int> &new_views);
    void publish(const std::vector<int> &new_views);
    void poll_completions();
    int ensure_kernel();
};

bool vrnerf_server::admit_locked(std::vector<int> &new_views) {
    bool any = false;
    const Clock::time_point now = Clock::now();
    while (!pending.empty()) {
        // drop cancelled requests, and late ones that asked to be shed
        for (auto it = pending.begin(); it != pending.end();) {
            Req *r = *it;
            if (r->cancel || (r->shed_if_late && r->has_deadline && r->deadline < now)) {
                r->state = r->cancel ? 4 : 5;
                if (!r->cancel) ++shed;
                it = pending.erase(it);
                done_cv.notify_all();
            } else {
                ++it;
            }
        }
        if (pending.empty()) break;
        // earliest deadline first; requests without one follow, in arrival order
        auto pick = pending.begin();
        for (auto it = pending.begin(); it != pending.end(); ++it)
            if ((*it)->has_deadline && (!(*pick)->has_deadline || (*it)->deadline < (*pick)->deadline)) pick = it;
        Req *q = *pick;
        // a ring entry is rewritten only long after its previous view finished
        if (n_views + q->n - oldest_live_view >= (unsigned)kRing / 2) break;
        size_t off = 0;
        if (!q->zero_copy && !arena.alloc(q->bytes, off)) break;  // HBM budget: wait for earlier requests
        pending.erase(pick);
        q->t_admit = now;
        q->arena_off = off;
        q->state = 1;
        q->views_left = q->n;
        size_t pix_off = 0;
        for (int v = 0; v < q->n; ++v) {
            const int idx = (int)(n_views % kRing);
            ServeView &sv = ring_h[idx];
            memcpy(sv.c2w, q->c2w.data() + 12 * v, sizeof sv.c2w);
            memcpy(sv.K, q->K.data() + 4 * v, sizeof sv.K);
            sv.W = q->res[2 * v];
            sv.H = q->res[2 * v + 1];
            sv.tiles_x = (sv.W + kTileW - 1) / kTileW;
            sv.req = next_req;
            const unsigned long long slots =
                (unsigned long long)sv.tiles_x * ((sv.H + kTileH - 1) / kTileH) * 32ull;
            sv.slot_begin = published;
            sv.slot_end = published + slots;
            sv.out = q->zero_copy ? q->out_dev + 3 * pix_off : reinterpret_cast<float *>(arena_d + off) + 3 * pix_off;
            sv.done = done_d + idx;
            sv.taken = 0;
            sv.finished = 0;
            done_h[idx] = 0;
            view_slots[idx] = slots;
            view_req[idx] = q;
            q->ring_idx.push_back(idx);
            published += slots;
            pix_off += (size_t)sv.W * sv.H;
            ++n_views;
            new_views.push_back(idx);
        }
        inflight.push_back(q);
        if (inflight.size() > max_inflight) max_inflight = inflight.size();
        ++next_req;
        any = true;
    }
    return any;
}

void vrnerf_server::publish(const std::vector<int> &new_views) {
    // view descriptors -> device ring, then the new totals -> control block,
    // both in device memory and in stream order: a kernel that sees the new
    // count finds the descriptors already written (and idle CTAs poll device
    // memory, not host memory across the chip-to-chip link)
    for (int idx : new_views)
        cudaMemcpyAsync(ring_d + idx, ring_h + idx, sizeof(ServeView), cudaMemcpyHostToDevice, pst);
    ctl_h->n_views = n_views;
    ctl_h->published = published;
    cudaMemcpyAsync(ctl_d, ctl_h, sizeof(ServeCtl), cudaMemcpyHostToDevice, pst);
    cudaStreamSynchronize(pst);
}

int vrnerf_server::ensure_kernel() {
    NvtxRange nvtx_range("serve: ensure kernel");
    if (kernel_launched && cudaEventQuery(kernel_done) != cudaSuccess) return VRNERF_OK;  // still running
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = ensure_tc_image(F, prec == VRNERF_BF16 ? 1 : 0, kst);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor + 1, 0, sizeof(unsigned int), kst);  // idle state
    if (e == cudaSuccess) {
        const int fmt = prec == VRNERF_BF16 ? 1 : 0;
        if (F->view.L == 8)
            e = fmt ? launch_serve_t<8, 1>(F, ring_d, ctl_d, cursor, idle_ns, tile_stats_d, kst)
                    : launch_serve_t<8, 0>(F, ring_d, ctl_d, cursor, idle_ns, tile_stats_d, kst);
        else
            e = fmt ? launch_serve_t<16, 1>(F, ring_d, ctl_d, cursor, idle_ns, tile_stats_d, kst)
                    : launch_serve_t<16, 0>(F, ring_d, ctl_d, cursor, idle_ns, tile_stats_d, kst);
    }
    if (e == cudaSuccess) e = cudaEventRecord(kernel_done, kst);
    if (e != cudaSuccess) return cuda_fail(e, "serve kernel launch");
    kernel_launched = true;
    ++launches;
    return VRNERF_OK;
}

void vrnerf_server::poll_completions() {
    std::vector<Req *> finished;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (Req *q : inflight) {
            if (q->state == 1) {
                bool all = true;
                for (int idx : q->ring_idx)
                    if (__atomic_load_n(&done_h[idx], __ATOMIC_ACQUIRE) < view_slots[idx]) all = false;
                if (all) {
                    q->t_gpu = Clock::now();
                    if (q->out_host && !q->zero_copy)
                        cudaMemcpyAsync(q->out_host, arena_d + q->arena_off, q->rays * 12, cudaMemcpyDeviceToHost, cst);
                    if (!q->zero_copy) cudaEventRecord(q->copied, cst);
                    q->state = 2;
                }
            }
            if (q->state == 2 && (q->zero_copy || cudaEventQuery(q->copied) == cudaSuccess)) finished.push_back(q);
        }
        for (Req *q : finished) {
            q->t_done = Clock::now();
            q->state = q->cancel ? 4 : 3;
            if (!q->zero_copy) arena.release(q->arena_off, q->bytes);
            for (int idx : q->ring_idx) view_req[idx] = nullptr;
            inflight.erase(std::find(inflight.begin(), inflight.end(), q));
            latencies_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
            wait_ms.push_back(std::chrono::duration<double, std::milli>(q->t_admit - q->t_submit).count());
            gpu_ms.push_back(std::chrono::duration<double, std::milli>(q->t_gpu - q->t_admit).count());
            copy_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_gpu).count());
            if (q->has_deadline && q->t_done > q->deadline) ++late;
            rays_done += q->rays;
            ++completed;
        }
        // the oldest view still referenced bounds ring reuse
        while (oldest_live_view < n_views && !view_req[oldest_live_view % kRing]) ++oldest_live_view;
    }
    if (!finished.empty()) {
        // the kernel's tile counters, for vrnerf_server_stats
        cudaMemcpyAsync(tile_stats_h, tile_stats_d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, pst);
        cudaStreamSynchronize(pst);
        done_cv.notify_all();
    }
}

void vrnerf_server::run() {
    cudaSetDevice(F->device);
    while (!quit.load()) {
        std::vector<int> nv;
        bool work;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (pending.empty() && inflight.empty())
                cv.wait_for(lk, std::chrono::milliseconds(5));
            admit_locked(nv);
            work = !inflight.empty();
        }
        if (!nv.empty()) publish(nv);
        if (work) {
            int rc = ensure_kernel();
            if (rc) {
                std::lock_guard<std::mutex> lk(mu);
                error = rc;
            }
        }
        poll_completions();
        if (work) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" {

int vrnerf_server_create(vrnerf_field *F, uint64_t hbm_budget_bytes, int32_t precision, vrnerf_server **out) {
    if (!F || !out) return fail(VRNERF_EINVAL, "NULL argument");
    *out = nullptr;
    if (precision != VRNERF_FP16 && precision != VRNERF_BF16)
        return fail(VRNERF_EINVAL, "the server renders with the fp16 or bf16 tensor-core path");
    if (hbm_budget_bytes < (1u << 20)) return fail(VRNERF_EINVAL, "budget below 1 MiB");
    vrnerf_server *S = new vrnerf_server();
    S->F = F;
    S->prec = precision;
    S->budget = hbm_budget_bytes;
    S->view_slots.assign(kRing, 0);
    S->view_req.assign(kRing, nullptr);
    cudaError_t e = cudaSetDevice(F->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->kst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->cst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->pst, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&S->ring_d, sizeof(ServeView) * kRing);
    if (e == cudaSuccess) e = cudaMallocHost(&S->ring_h, sizeof(ServeView) * kRing);
    if (e == cudaSuccess) e = cudaMallocHost(&S->ctl_h, sizeof(ServeCtl));
    if (e == cudaSuccess) e = cudaMalloc(&S->ctl_d, sizeof(ServeCtl));
    if (e == cudaSuccess) e = cudaMemset(S->ctl_d, 0, sizeof(ServeCtl));
    if (e == cudaSuccess) e = cudaHostAlloc(&S->done_h, sizeof(unsigned int) * kRing, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&S->done_d, S->done_h, 0);
    if (e == cudaSuccess) e = cudaMalloc(&S->cursor, 2 * sizeof(unsigned int));  // cursor, idle state
    if (e == cudaSuccess) e = cudaMemset(S->cursor, 0, 2 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&S->tile_stats_d, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(S->tile_stats_d, 0, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&S->tile_stats_h, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_d, hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->kernel_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        vrnerf_server_destroy(S);
        return fail(VRNERF_ENOMEM, "server resources: %s", cudaGetErrorString(e));
    }
    memset(S->ctl_h, 0, sizeof(ServeCtl));
    memset(S->done_h, 0, sizeof(unsigned int) * kRing);
    memset(S->tile_stats_h, 0, 2 * sizeof(unsigned long long));
    S->arena.init(hbm_budget_bytes);
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return VRNERF_OK;
}

}  // extern "C"

static int submit_impl(vrnerf_server *S, int32_t n_views, const float *cameras_host, const float *intrinsics_host,
                       const int32_t *resolution_host, float *out_host, double deadline_ms, int32_t shed_if_late,
                       uint64_t *ticket) {
    if (!S || !cameras_host || !intrinsics_host || !resolution_host || !ticket)
        return fail(VRNERF_EINVAL, "NULL argument");
    if (!(deadline_ms >= 0.0) || deadline_ms > 1.0e9) return fail(VRNERF_EINVAL, "deadline_ms must be in [0, 1e9]");
    if (n_views < 1 || n_views > 16) return fail(VRNERF_EINVAL, "a request holds 1 to 16 views");
    Req *q = new Req();
    q->n = n_views;
    q->c2w.assign(cameras_host, cameras_host + 12 * n_views);
    q->K.assign(intrinsics_host, intrinsics_host + 4 * n_views);
    q->res.assign(resolution_host, resolution_host + 2 * n_views);
    for (int v = 0; v < n_views; ++v) {
        if (q->res[2 * v] < 1 || q->res[2 * v] > 16384 || q->res[2 * v + 1] < 1 || q->res[2 * v + 1] > 16384 ||
            !(q->K[4 * v] > 0.0f) || !(q->K[4 * v + 1] > 0.0f)) {
            delete q;
            return fail(VRNERF_EINVAL, "view %d: bad resolution or focal length", v);
        }
        q->rays += (uint64_t)q->res[2 * v] * q->res[2 * v + 1];
    }
    q->bytes = q->rays * 12;
    if (out_host) {
        // pinned host memory the GPU can address: the kernel writes the
        // pixels there itself (no arena slice, no copy-out)
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer) {
            q->zero_copy = true;
            q->out_dev = static_cast<float *>(pa.devicePointer);
        } else {
            cudaGetLastError();
        }
    }
    if (!q->zero_copy && q->bytes > S->budget) {
        delete q;
        return fail(VRNERF_EINVAL, "request needs %llu bytes, more than the server's HBM budget",
                    (unsigned long long)q->rays * 12);
    }
    q->out_host = out_host;
    if (cudaEventCreateWithFlags(&q->copied, cudaEventDisableTiming) != cudaSuccess) {
        delete q;
        return fail(VRNERF_ENOMEM, "event");
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error) {
        cudaEventDestroy(q->copied);
        delete q;
        return fail(S->error, "server failed: %s", "kernel launch error");
    }
    if ((int)S->pending.size() >= S->max_pending) {
        cudaEventDestroy(q->copied);
        delete q;
        return fail(VRNERF_EBUSY, "admission queue full");
    }
    q->ticket = S->next_ticket++;
    q->t_submit = Clock::now();
    if (deadline_ms > 0.0) {
        q->has_deadline = true;
        q->shed_if_late = shed_if_late != 0;
        q->deadline = q->t_submit + std::chrono::duration_cast<Clock::duration>(
                                        std::chrono::duration<double, std::milli>(deadline_ms));
    }
    if (!S->have_first) {
        S->t_first = q->t_submit;
        S->have_first = true;
    }
    S->pending.push_back(q);
    S->by_ticket[q->ticket] = q;
    *ticket = q->ticket;
    S->cv.notify_all();
    return VRNERF_OK;
}

extern "C" {

int vrnerf_submit(vrnerf_server *S, int32_t n_views, const float *cameras_host, const float *intrinsics_host,
                  const int32_t *resolution_host, float *out_host, uint64_t *ticket) {
    return submit_impl(S, n_views, cameras_host, intrinsics_host, resolution_host, out_host, 0.0, 0, ticket);
}

int vrnerf_submit_deadline(vrnerf_server *S, int32_t n_views, const float *cameras_host,
                           const float *intrinsics_host, const int32_t *resolution_host, float *out_host,
                           double deadline_ms, int32_t shed_if_late, uint64_t *ticket) {
    return submit_impl(S, n_views, cameras_host, intrinsics_host, resolution_host, out_host, deadline_ms,
                       shed_if_late, ticket);
}

int vrnerf_poll(vrnerf_server *S, uint64_t ticket, int32_t timeout_ms, double *latency_ms) {
    if (!S) return fail(VRNERF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return fail(VRNERF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second;
    auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (q->state < 3 && !S->error) {
        if (S->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && q->state < 3) break;
    }
    if (q->state == 5) {
        S->by_ticket.erase(it);
        cudaEventDestroy(q->copied);
        delete q;
        return fail(VRNERF_ELATE, "request %llu was shed: its deadline passed before it reached the GPU",
                    (unsigned long long)ticket);
    }
    if (q->state < 3) {
        if (S->error) return fail(S->error, "server failed");
        return fail(VRNERF_ETIMEDOUT, "request %llu not finished", (unsigned long long)ticket);
    }
    const int state = q->state;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    S->by_ticket.erase(it);
    cudaEventDestroy(q->copied);
    delete q;
    return state == 4 ? fail(VRNERF_ECANCELED, "request %llu was cancelled", (unsigned long long)ticket)
                      : VRNERF_OK;
}

int vrnerf_cancel(vrnerf_server *S, uint64_t ticket) {
    if (!S) return fail(VRNERF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->by_ticket.find(ticket);
    if (it == S->by_ticket.end()) return fail(VRNERF_ENOTFOUND, "unknown ticket %llu", (unsigned long long)ticket);
    // pending: dropped at admission; in flight: rendered, but not copied out
    it->second->cancel = true;
    if (it->second->state <= 1) it->second->out_host = nullptr;
    S->cv.notify_all();
    return VRNERF_OK;
}

int vrnerf_server_stats(vrnerf_server *S, vrnerf_serve_stats *st) {
    if (!S || !st) return fail(VRNERF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof *st);
    st->completed = S->completed;
    st->rays = S->rays_done;
    st->kernel_launches = S->launches;
    st->pending = S->pending.size();
    st->inflight = S->inflight.size();
    st->max_inflight = S->max_inflight;
    st->tile_rounds = __atomic_load_n(&S->tile_stats_h[0], __ATOMIC_RELAXED);
    st->mixed_tile_rounds = __atomic_load_n(&S->tile_stats_h[1], __ATOMIC_RELAXED);
    std::vector<double> l = S->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        st->p50_ms = l[(size_t)(0.50 * (l.size() - 1))];
        st->p99_ms = l[(size_t)(0.99 * (l.size() - 1))];
        st->max_ms = l.back();
    }
    if (S->have_first)
        st->wall_s = std::chrono::duration<double>(Clock::now() - S->t_first).count();
    st->late = S->late;
    st->shed = S->shed;
    auto pct = [](std::vector<double> v, double *p50, double *p99) {
        if (v.empty()) return;
        std::sort(v.begin(), v.end());
        *p50 = v[(size_t)(0.50 * (v.size() - 1))];
        *p99 = v[(size_t)(0.99 * (v.size() - 1))];
    };
    pct(S->wait_ms, &st->wait_p50_ms, &st->wait_p99_ms);
    pct(S->gpu_ms, &st->gpu_p50_ms, &st->gpu_p99_ms);
    pct(S->copy_ms, &st->copy_p50_ms, &st->copy_p99_ms);
    return VRNERF_OK;
}

int vrnerf_server_reset_stats(vrnerf_server *S) {
    if (!S) return fail(VRNERF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies_ms.clear();
    S->wait_ms.clear();
    S->gpu_ms.clear();
    S->copy_ms.clear();
    S->late = 0;
    S->shed = 0;
    S->rays_done = 0;
    S->completed = 0;
    S->launches = 0;
    S->max_inflight = S->inflight.size();
    S->have_first = false;
    return VRNERF_OK;
}

void vrnerf_server_destroy(vrnerf_server *S) {
    if (!S) return;
    if (S->worker.joinable()) {
        S->quit.store(true);
        S->cv.notify_all();
        S->worker.join();
    }
    if (S->ctl_h && S->ctl_d && S->pst) {
        S->ctl_h->stop = 1;
        cudaMemcpyAsync(S->ctl_d, S->ctl_h, sizeof(ServeCtl), cudaMemcpyHostToDevice, S->pst);
        cudaStreamSynchronize(S->pst);
    }
    if (S->kst) cudaStreamSynchronize(S->kst);
    if (S->cst) cudaStreamSynchronize(S->cst);
    if (S->pst) cudaStreamSynchronize(S->pst);
    for (auto &kv : S->by_ticket) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    if (S->kernel_done) cudaEventDestroy(S->kernel_done);
    if (S->arena_d) cudaFree(S->arena_d);
    if (S->cursor) cudaFree(S->cursor);
    if (S->tile_stats_d) cudaFree(S->tile_stats_d);
    if (S->tile_stats_h) cudaFreeHost(S->tile_stats_h);
    if (S->done_h) cudaFreeHost(S->done_h);
    if (S->ctl_h) cudaFreeHost(S->ctl_h);
    if (S->ctl_d) cudaFree(S->ctl_d);
    if (S->ring_h) cudaFreeHost(S->ring_h);
    if (S->ring_d) cudaFree(S->ring_d);
    if (S->kst) cudaStreamDestroy(S->kst);
    if (S->cst) cudaStreamDestroy(S->cst);
    if (S->pst) cudaStreamDestroy(S->pst);
    delete S;
}

}  // extern "C"
