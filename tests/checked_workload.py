"""Runs the library's entry points through the checked build (device-side
bounds checks on hash indices, voxels, sample indices, output pixels and
training records) and fails if any check fired. Started by
tests/test_gpu_checked.py with VRNERF_CHECKED=1."""
import os
import sys
from dataclasses import replace

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2311_02542_gb300 import synth as S  # noqa: E402
from paper_2311_02542_gb300 import vrnerf as V  # noqa: E402


def cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def main():
    V.load()
    assert V.lib_path().endswith("libvrnerf_checked.so") and V.vrnerf_build_checked()
    sc = S.make_scene("unit_cube")
    for cfg in (sc.cfg, replace(sc.cfg, contract=True, t_far=100.0)):
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, 64, 64)
        cams = np.concatenate([c2w, c2w])
        Ks = np.concatenate([K, S.intrinsics_fov(33, 17)[None]])
        res2 = np.array([[64, 64], [33, 17]], np.int32)
        rays = 64 * 64 + 33 * 17
        for prec in ("fp32", "fp16", "bf16", "fp8"):
            V.vrnerf_render(f, cuda(cams), cuda(Ks), res2, precision=prec,
                            out_depth=torch.empty(rays, device="cuda"),
                            out_rgba8=torch.empty(rays, device="cuda", dtype=torch.int32))
        V.vrnerf_render(f, cuda(c2w), cuda(K), res, out_normal=torch.empty((4096, 3), device="cuda"))
        V.vrnerf_field_status(f)
        poses = c2w[:, :, 3]
        rng = np.random.default_rng(1)
        o = (poses[0] + 0 * rng.normal(size=(4096, 3))).astype(np.float32)
        d = rng.normal(size=(4096, 3))
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
        r = np.full(4096, 1e-3, np.float32)
        tgt = np.exp(rng.uniform(-3, 3, (4096, 3))).astype(np.float32)
        o, d, r, tgt = cuda(o), cuda(d), cuda(r), cuda(tgt)
        V.vrnerf_render_rays(f, o, d, r, precision="fp16")
        V.vrnerf_query(f, o, d, r)
        V.vrnerf_debug_march(f, o, d, 64)
        V.vrnerf_debug_corners(f, o)
        V.vrnerf_history_reset(f)
        V.vrnerf_train_step(f, o, d, r, tgt)
        V.vrnerf_field_set_train_precision(f, "bf16")  # the tensor-core backward
        V.vrnerf_train_step(f, o, d, r, tgt)
        V.vrnerf_field_set_train_precision(f, "fp32")
        pq, n = V.vrnerf_forward_rays(f, o, d, r)
        V.vrnerf_backward_from_grad(f, o, d, r, n, torch.randn_like(pq))
        V.vrnerf_field_status(f)
        V.vrnerf_prune(f, poses, 2, 0.01, apply=True)
        V.vrnerf_occupancy_upsample(f, 2)
        V.vrnerf_render(f, cuda(c2w), cuda(K), res, precision="fp16")
        V.vrnerf_field_status(f)
        f.close()
    room = S.make_scene("room")
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, _ = S.camera_room(room.occ, room.cfg, 2, 2048, 2048)
    Kc = S.crop_camera(K, 896, 896)
    V.vrnerf_render(f, cuda(c2w), cuda(Kc), np.array([[256, 256]], np.int32), precision="fp16")
    srv = V.Server(f, 64 << 20, "fp16")
    out = np.zeros((160 * 128, 3), np.float32)
    srv.poll(srv.submit(c2w, S.intrinsics_fov(160, 128)[None], np.array([[160, 128]], np.int32), out), 20000)
    srv.close()
    V.vrnerf_field_status(f)
    # the reporting path: a kernel sets the test bit, the status call reports
    # it once and clears it
    V.vrnerf_debug_check_trigger(f)
    try:
        V.vrnerf_field_status(f)
        raise AssertionError("check bit not reported")
    except V.VrnerfError as e:
        assert e.code == V.ECHECK, e
    V.vrnerf_field_status(f)
    f.close()
    print("checked workload OK")


if __name__ == "__main__":
    main()
