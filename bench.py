"""Benchmark of the per-ray VR-NeRF field renderer on one GB300.

Workload (the step): one render of a single 2048x2048 eye buffer in the
20 m x 20 m x 3 m synthetic room (L=16 hash levels, T=2^21, fp16 features,
256^3 occupancy, <= 1024 exponential samples per ray), camera at 1.7 m,
every step of the path (ray generation, occupancy march, LOD hash-grid
gather, density/colour MLP, compositing, PQ decode) in one launch.

Reports, as one JSON line:
  value            Mrays/s of the tuned path, inputs resident in HBM
  e2e              Mrays/s through vrnerf_render_host (host buffers, copies
                   inside the timed region)
  plain_fp32       the same for the fp32 MLP path
  stereo           2 x 2048^2 frame latency p50 / p99 (tuned path)
  roofline         dominant kernel (the fused render kernel) vs measured HBM peak
  cpu_baseline     the CPU oracle on a bounded crop of the same frame
  clocks           SM clocks sampled with nvidia-smi during the timed region

`--impl reference` times the CPU oracle instead (the only reference that
exists: the paper ships no code), on a 256x256 crop per step.
With --gpus N > 1 (torchrun) every rank renders its own frame: the path
shards by views with no collective (replicas only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "room_2048x2048_single_eye"
STEREO_BUDGET_MS = 1000.0 / 36.0  # one frame at the 36 Hz the paper's demo sustains


# DRAM bytes read + written by one 2048x2048 launch of render_tc_kernel<16, 0, 0, 4>
# (ncu dram__bytes_read.sum + dram__bytes_write.sum, one capture of the benchmark
# frame). NCU_TRAFFIC_CURRENT says whether the kernel is unchanged since that
# capture; when it is not, the bench line reports traffic null and the old
# figure beside it.
NCU_TRAFFIC_BYTES = 54128384 + 28538624
NCU_TRAFFIC_CURRENT = True  # captured on the current kernel (four tiles per CTA, chunked epilogue)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--variant", default="room",
                    choices=["room", "room_surface", "room_unbounded", "room_unbounded_surface"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serving-requests", type=int, default=300,
                    help="requests of the Poisson serving stream (0: skip)")
    ap.add_argument("--train-steps", type=int, default=5, help="timed 2^20-ray train steps (0: skip)")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the paper-grid / unbounded-room frames and the pruning pass")
    ap.add_argument("--profile-train", action="store_true",
                    help="small case for ncu: two 2^18-ray training steps on the room field")
    ap.add_argument("--train-prec", default="fp32", choices=("fp32", "bf16"),
                    help="training precision of --profile-train")
    ap.add_argument("--train-log2", type=int, default=18,
                    help="log2 of the --profile-train batch (rays)")
    ap.add_argument("--profile-case", action="store_true",
                    help="small case for ncu: two renders of a 1024x1024 window of the room frame")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, device=None):
    """Largest x over the ranks of the default process group (x alone)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mrays(rays_per_rank, world, ms_max):
    """Rays of all ranks (each renders its own frame) over the slowest rank's time."""
    return world * rays_per_rank / (ms_max * 1e-3) / 1e6


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler (every 50 ms) started before the warm-up; mark()
    at the start of the timed region, stop() at its end. The summary uses the
    samples taken between the two; when the region was shorter than one
    interval, the first sample after it (taken within 50 ms of its end, the
    GPU still at the region's clocks) and the last one before it."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.skip = 0

    def _lines(self):
        self.f.flush()
        self.f.seek(0)
        return [ln for ln in self.f.read().splitlines() if len(ln.split(",")) >= 9]

    def mark(self):
        """Waits (up to 3 s) for the sampler's first line, then records how
        many lines precede the timed region."""
        t0 = time.perf_counter()
        while self.p is not None and not self._lines() and time.perf_counter() - t0 < 3.0:
            time.sleep(0.02)
        self.skip = len(self._lines()) if self.p is not None else 0

    def stop(self):
        if self.p is None:
            self.f.close()
            os.unlink(self.f.name)
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        end = len(self._lines())
        in_region = end - self.skip
        if in_region <= 0:  # wait (at most 0.5 s) for the first sample after the region
            t0 = time.perf_counter()
            while len(self._lines()) <= end and time.perf_counter() - t0 < 0.5:
                time.sleep(0.005)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        lines = self._lines()
        if in_region > 0:
            lines = lines[self.skip:end]
        else:
            lines = lines[max(self.skip - 1, 0):self.skip] + lines[end:end + 1]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "in_region": max(in_region, 0),
                "interval_ms": 50}


# Keys printed last, in this order: a reader that keeps only the end of the
# line still sees the measurement record and the headline comparisons
# (stereo latency, tuned against plain fp32, the precision sweep).
TAIL_KEYS = ("work", "roofline", "e2e", "cpu_baseline", "clocks", "gpu_launches", "wall_s_timed",
             "serving_summary", "precision_sweep", "plain_fp32", "stereo_2x2048")


def tail_order(line):
    """The bench line with the bulky extras (serving runs, training steps,
    other workloads) first and TAIL_KEYS last."""
    head = {k: v for k, v in line.items() if k not in TAIL_KEYS}
    head.update({k: line[k] for k in TAIL_KEYS if k in line})
    return head


def pick_precision(V, arg):
    if arg != "auto":
        return V.PRECISIONS[arg]
    return V.FP16


def run_oracle_sample(sc, c2w, K, seconds, threads):
    """Renders 128x128 crops of the frame with the CPU oracle until about
    `seconds` have passed; returns (rays, elapsed)."""
    import oracle as O
    from paper_2311_02542_gb300 import synth as S
    F = O.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    rng = np.random.default_rng(0)
    rays, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        x0, y0 = rng.integers(0, 2048 - 128, 2)
        F.render(c2w, S.crop_camera(K, int(x0), int(y0)), np.array([[128, 128]], np.int32),
                 threads=threads)
        rays += 128 * 128
    return rays, time.perf_counter() - t0


def workload_config(cfg, variant, world):
    """The workload both arms measure: one 2048x2048 eye buffer of the room
    field per step and GPU."""
    return {"workload": WORKLOAD, "variant": variant, "resolution": [2048, 2048],
            "views_per_step": 1, "rays_per_step": 2048 * 2048, "levels": cfg.levels,
            "log2_T": cfg.log2_T, "occ_res": list(cfg.occ_res), "max_steps": cfg.max_steps,
            "parallelism": f"replicas{world}"}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2311_02542_gb300 import synth as S
    import oracle as O
    sc = S.make_scene(args.variant)
    c2w, K, res = S.camera_room(sc.occ, sc.cfg, 2, 2048, 2048)
    F = O.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    threads = os.cpu_count() or 1
    crop = np.array([[256, 256]], np.int32)
    rng = np.random.default_rng(1)

    def step():
        x0, y0 = rng.integers(0, 2048 - 256, 2)
        F.render(c2w, S.crop_camera(K, int(x0), int(y0)), crop, threads=threads)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    rays = 256 * 256 * args.steps
    v = rays / dt / 1e6
    line = {"impl": "reference", "metric": "Mrays/s", "value": round(v, 4), "unit": "Mrays/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**workload_config(sc.cfg, args.variant, args.gpus),
                       "sample": "one 256x256 crop of the 2048x2048 frame per step"},
            "cpu_baseline": {"value": round(v, 4), "unit": "Mrays/s", "cores": threads,
                             "kind": "oracle",
                             "sample": "one 256x256 crop of the 2048x2048 frame per step"},
            "e2e": {"value": round(v, 4), "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_bench(V, field, sc, n_req, warm=30, rate_hz=36.0 / 0.7, seed=4, in_flight=24):
    """Poisson stream of render requests (70 % stereo 2 x 2048^2, 30 % single
    views of side 512 / 1024 / 1536, random 6-DoF poses in the room) through
    the continuous-batching server; outputs are copied to pinned host buffers.
    Returns per-request latency percentiles and throughput."""
    import queue
    import threading

    import torch
    from paper_2311_02542_gb300 import synth as S
    reqs = S.request_stream(sc.occ, sc.cfg, n_req + warm, seed=seed, rate_hz=rate_hz)
    srv = V.Server(field, 6 << 30, V.FP16)
    maxr = max(r.rays for r in reqs)
    bufs = [torch.empty((maxr, 3), dtype=torch.float32, pin_memory=True).numpy()
            for _ in range(in_flight)]
    free, done, lat = queue.Queue(), queue.Queue(), {}
    for i in range(in_flight):
        free.put(i)

    def poller():
        while True:
            item = done.get()
            if item is None:
                return
            i, t, b = item
            lat[i] = srv.poll(t, 120000)
            free.put(b)

    th = threading.Thread(target=poller)
    th.start()
    t0 = time.perf_counter()
    t_meas = t0
    for i, r in enumerate(reqs):
        wait = t0 + r.arrival_s - time.perf_counter()
        if wait > 0 and rate_hz < 1e5:
            time.sleep(wait)
        if i == warm:
            srv.reset_stats()
            t_meas = time.perf_counter()
        b = free.get()
        # stereo frames are due within one 36 Hz frame time; single views carry no deadline
        dl = STEREO_BUDGET_MS if r.stereo else None
        done.put((i, srv.submit(r.c2w, r.intrinsics, r.resolution, bufs[b][:r.rays], deadline_ms=dl), b))
    done.put(None)
    th.join()
    wall = time.perf_counter() - t_meas
    st = srv.stats()
    srv.close()
    meas = range(warm, len(reqs))
    st_lat = np.array([lat[i] for i in meas if reqs[i].stereo])
    all_lat = np.array([lat[i] for i in meas])
    rays = sum(reqs[i].rays for i in meas)
    return {"requests": len(meas), "offered_req_s": round(rate_hz, 2) if rate_hz < 1e5 else "saturating",
            "stereo_p50_ms": round(float(np.percentile(st_lat, 50)), 3),
            "stereo_p99_ms": round(float(np.percentile(st_lat, 99)), 3),
            "all_p50_ms": round(float(np.percentile(all_lat, 50)), 3),
            "all_p99_ms": round(float(np.percentile(all_lat, 99)), 3),
            "stereo_within_budget": round(float(np.mean(st_lat <= STEREO_BUDGET_MS)), 4),
            "late_stereo": int(st["late"]),
            "stage_ms": {k: round(float(st[k]), 3) for k in ("wait_p50_ms", "wait_p99_ms", "gpu_p50_ms",
                                                               "gpu_p99_ms", "copy_p50_ms", "copy_p99_ms")},
            "Mrays_s": round(rays / wall / 1e6, 2), "wall_s": round(wall, 2),
            "kernel_launches": int(st["kernel_launches"]),
            "overlap": {"max_inflight": int(st["max_inflight"]), "mixed_tile_frac":
                        round(st["mixed_tile_rounds"] / max(st["tile_rounds"], 1), 4)},
            "note": ("latency = submit to image in pinned host memory; fp16 tensor-core MLP; stereo "
                     f"requests admitted earliest-deadline-first with a {STEREO_BUDGET_MS:.1f} ms deadline")}


def train_bench(V, sc, steps, batch=1 << 20, precision="fp32"):
    """Training step on a batch of rays drawn from 64 synthetic HDR views
    (targets log-uniform in [1e-3, 1e3]); forward, loss, backward, Adam.
    precision: arithmetic of the MLPs in the training forward and backward
    (fp32 CUDA cores or bf16 tcgen05 tensor cores)."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    field = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    V.vrnerf_field_set_train_precision(field, precision)
    poses, intr = S.training_views(sc.occ, sc.cfg, n_views=64)
    batches = []
    for k in range(2):
        o, d, r, tgt = S.training_batch(poses, intr, batch, seed=5, step=k)
        batches.append([torch.from_numpy(a).cuda() for a in (o, d, r, tgt)])
    for k in range(2):
        V.vrnerf_train_step(field, *batches[k % 2])
    torch.cuda.synchronize()
    ts, losses = [], []
    for k in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        V.vrnerf_train_step(field, *batches[k % 2], want_loss=False)
        b.record()
        ts.append((a, b))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ts]))
    loss = V.vrnerf_backward(field, *batches[0])
    field.close()
    return {"batch_rays": batch, "ms_per_step": round(ms, 3),
            "Mrays_s": round(batch / (ms * 1e-3) / 1e6, 2), "loss": round(float(loss), 6),
            "steps": steps,
            "mlp": "fp32 (CUDA cores)" if precision == "fp32"
            else "forward and backward: bf16 operands, fp32 accumulation (tcgen05)"}


def workload_bench(V, name, precision, steps, flush):
    """One 2048^2 eye buffer of another scene shape: Mrays/s and work counters."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    sc = S.make_scene(name)
    field = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, res = S.camera_room(sc.occ, sc.cfg, 2, 2048, 2048)
    cams, intr = torch.from_numpy(c2w).cuda(), torch.from_numpy(K).cuda()
    rays = 2048 * 2048
    out = torch.empty((rays, 3), device="cuda")
    stats = torch.zeros(4, dtype=torch.int64, device="cuda")
    V.vrnerf_render(field, cams, intr, res, out=out, precision=precision, stats=stats)
    for _ in range(2):
        V.vrnerf_render(field, cams, intr, res, out=out, precision=precision)
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        V.vrnerf_render(field, cams, intr, res, out=out, precision=precision)
        b.record()
        ts.append((a, b))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ts]))
    n_samples, n_levels, n_steps, _ = [int(x) for x in stats.cpu()]
    field.close()
    cfg = sc.cfg
    return {"Mrays_s": round(rays / (ms * 1e-3) / 1e6, 2), "ms_per_frame": round(ms, 3),
            "samples_per_ray": round(n_samples / rays, 3), "steps_per_ray": round(n_steps / rays, 2),
            "levels_per_sample": round(n_levels / max(n_samples, 1), 3),
            "grid": {"levels": cfg.levels, "base_res": cfg.base_res, "growth": round(cfg.growth, 4),
                     "log2_T": cfg.log2_T}, "contract": bool(cfg.contract), "t_far": cfg.t_far}


def prune_bench(V, sc, k=4):
    """One joint history/grid pruning pass (Sec. 4.3.2) over the scene's
    occupancy grid, k^3 density evaluations per occupied voxel."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    field = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    poses, _ = S.training_views(sc.occ, sc.cfg, n_views=64)
    cams = poses[:, :3, 3].astype(np.float32)
    V.vrnerf_history_reset(field)
    V.vrnerf_prune(field, cams, k, 0.2, apply=False)
    t0 = time.perf_counter()
    kept, _, _ = V.vrnerf_prune(field, cams, k, 0.2, apply=False)
    dt = time.perf_counter() - t0
    occupied = int(sc.occ.sum())
    field.close()
    return {"ms": round(dt * 1e3, 2), "points_per_voxel": k ** 3, "occupied_voxels": occupied,
            "kept_at_0.2": int(kept), "Mpoints_s": round(occupied * k ** 3 / dt / 1e6, 1)}


def profile_case(args):
    """Two renders of a 1024x1024 window of the benchmark frame (same field,
    about 140 MB on the device): the small case for ncu captures."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene(args.variant)
    field = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, _ = S.camera_room(sc.occ, sc.cfg, 2, 2048, 2048)
    K = S.crop_camera(K, 512, 512)
    res = np.array([[1024, 1024]], np.int32)
    prec = V.PRECISIONS["fp32" if args.precision == "auto" else args.precision]
    cams, intr = torch.from_numpy(c2w).cuda(), torch.from_numpy(K).cuda()
    out = torch.empty((1024 * 1024, 3), device="cuda")
    for _ in range(2):
        V.vrnerf_render(field, cams, intr, res, out=out, precision=prec)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "room 1024x1024 window", "precision": prec,
                      "mean_linear": float(out.mean())}))
    return 0


def profile_train(args):
    """Two training steps of 2^18 rays (--train-log2) on the room field (grid,
    gradients and moments about 1 GB on the device): the small case for ncu
    captures of the training kernels."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene(args.variant)
    field = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    V.vrnerf_field_set_train_precision(field, args.train_prec)
    poses, intr = S.training_views(sc.occ, sc.cfg, n_views=64)
    batch = [torch.from_numpy(a).cuda()
             for a in S.training_batch(poses, intr, 1 << args.train_log2, seed=5, step=0)]
    losses = [V.vrnerf_train_step(field, *batch) for _ in range(2)]
    print(json.dumps({"profile_train": f"room, 2^{args.train_log2} rays", "precision": args.train_prec,
                      "losses": losses}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile_case:
        return profile_case(args)
    if args.profile_train:
        return profile_train(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2311_02542_gb300 import synth as S
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    dev = torch.device("cuda", local)

    sc = S.make_scene(args.variant)
    cfg = sc.cfg
    field = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, res = S.camera_room(sc.occ, cfg, 2 + rank, 2048, 2048)
    cams, intr = torch.from_numpy(c2w).to(dev), torch.from_numpy(K).to(dev)
    rays = int(res[0, 0]) * int(res[0, 1])
    out = torch.empty((rays, 3), device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()
    tuned = pick_precision(V, args.precision)
    try:
        V.vrnerf_render(field, cams, intr, res, out=out, precision=tuned)
        torch.cuda.synchronize()
    except V.VrnerfError:
        tuned = V.FP32
    precision_name = {v: k for k, v in V.PRECISIONS.items()}[tuned]

    def timed(precision, steps, warmup, resolution=res, cam=cams, K_=intr, o=out):
        for _ in range(warmup):
            V.vrnerf_render(field, cam, K_, resolution, out=o, precision=precision)
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            V.vrnerf_render(field, cam, K_, resolution, out=o, precision=precision)
            b.record(stream)
            ts.append((a, b))
        torch.cuda.synchronize()
        return np.array([a.elapsed_time(b) for a, b in ts])

    # work statistics of one frame (untimed): samples, levels fetched, steps
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    n_per_ray = torch.empty(rays, dtype=torch.int32, device=dev)
    V.vrnerf_render(field, cams, intr, res, out=out, precision=tuned, stats=stats, out_n=n_per_ray)
    torch.cuda.synchronize()
    n_samples, n_levels, n_steps, n_rays_done = [int(x) for x in stats.cpu()]
    spr = n_per_ray.cpu().numpy()
    spr_hist = {f"p{q}": int(np.percentile(spr, q)) for q in (50, 90, 99)}
    spr_hist["max"] = int(spr.max())
    spr_hist["zero_frac"] = round(float((spr == 0).mean()), 4)

    # timed region: tuned path (its warm-up steps run first, untimed),
    # bracketed by barrier + synchronize on both sides
    clk = Clocks(local)
    for _ in range(args.warmup):
        V.vrnerf_render(field, cams, intr, res, out=out, precision=tuned)
    torch.cuda.synchronize()
    clk.mark()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    ms = timed(tuned, args.steps, 0)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - t_wall0
    clocks = clk.stop()
    ms_step = max_over_ranks(float(ms.mean()), dev)
    value = whole_job_mrays(rays, world, ms_step)

    # plain fp32 path on the same frame
    ms32 = timed(V.FP32, 10, 2) if tuned != V.FP32 else ms

    # precision sweep on the same frame: throughput (median frame, so that one
    # host stall between the start event and the launch does not count), and PQ-space PSNR against
    # the fp32 render (the tests hold each precision to >= 50 dB against the
    # fp64 CPU oracle on 256^2 crops)
    ref_pq = torch.empty((rays, 3), device=dev)
    V.vrnerf_render(field, cams, intr, res, out=out, precision=V.FP32, out_pq=ref_pq)
    sweep = {}
    for name in ("fp32", "fp16", "bf16", "fp8"):
        p = V.PRECISIONS[name]
        t = timed(p, 5, 2)
        pq = torch.empty((rays, 3), device=dev)
        V.vrnerf_render(field, cams, intr, res, out=out, precision=p, out_pq=pq)
        mse = float(((pq - ref_pq).double() ** 2).mean())
        sweep[name] = {"Mrays_s": round(rays / (float(np.median(t)) * 1e-3) / 1e6, 2),
                       "psnr_pq_vs_fp32_db": (round(10 * np.log10(1.0 / mse), 2) if mse > 0 else "inf")}


    # stereo 2 x 2048^2 frame latency (tuned)
    st_c2w = S.stereo_pair(c2w[0])
    st_K = np.concatenate([K, K])
    st_res = np.array([[2048, 2048], [2048, 2048]], np.int32)
    st_out = torch.empty((2 * rays, 3), device=dev)
    st_ms = timed(tuned, 50, 10, st_res, torch.from_numpy(st_c2w).to(dev),
                  torch.from_numpy(st_K).to(dev), st_out)

    # end to end through the host-buffer entry point (pinned host memory)
    h_out = torch.empty((rays, 3), dtype=torch.float32, pin_memory=True).numpy()
    h_cam = torch.from_numpy(c2w.copy()).pin_memory().numpy()
    h_K = torch.from_numpy(K.copy()).pin_memory().numpy()
    for _ in range(2):
        V.vrnerf_render_host(field, h_cam, h_K, res, out=h_out, precision=tuned)
    e2e_t = []
    for _ in range(10):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        V.vrnerf_render_host(field, h_cam, h_K, res, out=h_out, precision=tuned)
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = world * rays / float(np.mean(e2e_t)) / 1e6

    hbm_peak, peak_kind = load_peaks()
    feat_bytes = 2 if cfg.feat_fp16 else 4
    # algorithmic bytes of one launch: 8 corners x F features per fetched
    # level, 12 B of output per ray, 1 byte of distance field per march step
    alg_bytes = n_levels * 8 * cfg.feats * feat_bytes + rays * 12 + n_steps
    achieved = alg_bytes / (ms_step * 1e-3) / 1e9

    line = {
        "metric": "Mrays/s", "value": round(value, 3), "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16+f32acc", "bf16": "bf16+f32acc",
                  "fp8": "e4m3+f16+f32acc"}[precision_name],
        "data": "synthetic",
        "config": {**workload_config(cfg, args.variant, world),
                   "l2": "256 MB buffer written between timed steps"},
        "mlp_precision": precision_name,
        "work": {"samples_per_ray": round(n_samples / rays, 3), "samples_per_ray_hist": spr_hist,
                 "levels_per_sample": round(n_levels / max(n_samples, 1), 3),
                 "steps_per_ray": round(n_steps / rays, 2), "rays_finished": n_rays_done},
        "precision_sweep": sweep,
        "plain_fp32": {"value": round(world * rays / (float(ms32.mean()) * 1e-3) / 1e6, 3),
                       "unit": "Mrays/s", "ms_per_step": round(float(ms32.mean()), 4)},
        "stereo_2x2048": {"p50_ms": round(float(np.percentile(st_ms, 50)), 4),
                          "p99_ms": round(float(np.percentile(st_ms, 99)), 4),
                          "fps_p99": round(1e3 / float(np.percentile(st_ms, 99)), 2),
                          "frames": int(st_ms.size)},
        "e2e": {"value": round(e2e_v, 3), "unit": "Mrays/s", "h2d_bytes_per_step": 64,
                "d2h_bytes_per_step": rays * 12,
                "note": "vrnerf_render_host with pinned host arrays: cameras copied in, the image written "
                        "by the kernel into the pinned output (zero-copy), timed to the call's return"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak,
                     "unit": "GB/s", "frac": round(achieved / hbm_peak, 5),
                     "traffic": (NCU_TRAFFIC_BYTES if NCU_TRAFFIC_CURRENT and precision_name == "fp16"
                                 and args.variant == "room" else None),
                     "traffic_note": ("ncu dram__bytes_read + dram__bytes_write of one 2048^2 fp16 launch "
                                      "(the gather is served from L2)"),
                     "peak_kind": peak_kind, "kernel": "render (fused march+gather+MLP+composite)"},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "wall_s_timed": round(wall, 3),
    }
    if args.serving_requests > 0:
        line["serving"] = serving_bench(V, field, sc, args.serving_requests)
        sc_s = S.make_scene("room_surface")  # opaque occupied voxels, as in a trained scene
        field_s = V.Field(sc_s.cfg, sc_s.grid, sc_s.mlp, sc_s.occ_bits)
        line["serving_surface_variant"] = serving_bench(V, field_s, sc_s, args.serving_requests)
        field_s.close()
        n_sat = max(60, args.serving_requests // 3)
        line["serving_saturated"] = serving_bench(V, field, sc, n_sat, warm=10, rate_hz=1e9)
        # the same requests rendered one by one without the server (device
        # buffers): the server's efficiency on this mix
        reqs = S.request_stream(sc.occ, cfg, n_sat + 10, seed=4, rate_hz=1e9)[10:]
        direct_rays, direct_ms = 0, 0.0
        for rq in reqs:
            nr = int((rq.resolution[:, 0].astype(np.int64) * rq.resolution[:, 1]).sum())
            o_d = torch.empty((nr, 3), device=dev)
            c_d, k_d = torch.from_numpy(rq.c2w).to(dev), torch.from_numpy(rq.intrinsics).to(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            V.vrnerf_render(field, c_d, k_d, rq.resolution, out=o_d, precision=V.FP16)
            b.record()
            torch.cuda.synchronize()
            direct_ms += a.elapsed_time(b)
            direct_rays += nr
        line["serving_saturated"]["direct_render_Mrays_s"] = round(direct_rays / (direct_ms * 1e-3) / 1e6, 2)
        line["serving_summary"] = {
            k: {"stereo_p50_ms": line[k]["stereo_p50_ms"], "stereo_p99_ms": line[k]["stereo_p99_ms"],
                "Mrays_s": line[k]["Mrays_s"]} for k in ("serving", "serving_surface_variant")}
        line["serving_summary"]["budget_ms"] = round(STEREO_BUDGET_MS, 2)
    if args.train_steps > 0:
        line["train_step"] = train_bench(V, sc, args.train_steps)
        # the paper's batch: 12 800 rays (256 rays from each of 50 images)
        line["train_step_paper_batch"] = train_bench(V, sc, max(args.train_steps, 20), batch=12800)
        line["train_step_bf16_tc"] = train_bench(V, sc, args.train_steps, precision="bf16")
    if not args.no_extra_workloads:
        line["workloads"] = {
            "room_paper_grid_2048": workload_bench(V, "room_paper_grid", tuned, 10, flush),
            "room_unbounded_2048": workload_bench(V, "room_unbounded", tuned, 10, flush),
            "room_unbounded_surface_2048": workload_bench(V, "room_unbounded_surface", tuned,
                                                          10, flush),
        }
        line["prune_room_surface_k4"] = prune_bench(V, S.make_scene("room_surface"))
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        crays, cdt = run_oracle_sample(sc, c2w, K, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": round(crays / cdt / 1e6, 5), "unit": "Mrays/s",
                                "cores": threads, "kind": "oracle",
                                "sample": f"{crays // (128 * 128)} random 128x128 crops of the "
                                          f"2048x2048 frame ({cdt:.1f} s)"}
        # the same on one host core (a shorter sample)
        crays1, cdt1 = run_oracle_sample(sc, c2w, K, min(4.0, args.cpu_seconds / 3), 1)
        line["cpu_baseline"]["single_core_Mrays_s"] = round(crays1 / cdt1 / 1e6, 5)
        # the oracle's 256^2 window of the frame against each GPU precision
        import oracle as O
        crop_K = S.crop_camera(K, 896, 896)
        crop_res = np.array([[256, 256]], np.int32)
        oracle_pq = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits).render(c2w, crop_K, crop_res,
                                                                      threads=threads)["pq"]
        psnr = {}
        for name in ("fp32", "fp16", "bf16", "fp8"):
            cpq = torch.empty((256 * 256, 3), device=dev)
            V.vrnerf_render(field, cams, torch.from_numpy(crop_K).to(dev), crop_res,
                            out=torch.empty((256 * 256, 3), device=dev), precision=V.PRECISIONS[name],
                            out_pq=cpq)
            mse_o = float(np.mean((cpq.cpu().numpy().astype(np.float64) - oracle_pq) ** 2))
            psnr[name] = round(10 * np.log10(1.0 / mse_o), 2) if mse_o > 0 else "inf"
        line["cpu_baseline"]["gpu_psnr_pq_vs_oracle_db"] = psnr
        line["cpu_baseline"]["psnr_sample"] = "256x256 window at (896, 896) of the frame, PQ peak 1.0"
    if rank == 0:
        print(json.dumps(tail_order(line)), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
