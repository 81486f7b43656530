"""Continuous-batching server: every request's image equals the same views
rendered alone (vrnerf_render, same precision) within the tensor-core
tolerance; admission by HBM budget; cancel, unknown tickets, timeouts; the
persistent kernel leaves when idle and is relaunched for new work."""
import time

import numpy as np
import pytest
import torch

from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu

TC_RTOL, TC_ATOL = 2e-3, 1e-5


@pytest.fixture(scope="module")
def V():
    from paper_2311_02542_gb300 import vrnerf
    vrnerf.load()
    return vrnerf


@pytest.fixture(scope="module")
def room():
    return S.make_scene("room")


def _alone(V, f, c2w, K, res):
    return V.vrnerf_render(f, torch.from_numpy(c2w).cuda(), torch.from_numpy(K).cuda(), res,
                           precision="fp16").cpu().numpy()


def _mix(room, rng):
    cfg = room.cfg
    reqs = []
    for i, (w, h) in enumerate([(192, 160), (64, 64), (96, 80), (192, 160), (33, 17), (128, 128),
                                (192, 160), (250, 7)]):
        p = S.room_position(room.occ, cfg, rng)
        pose = S.pose_from_angles(p, rng.uniform(0, 6.28), rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5))
        if i % 3 == 0:  # stereo pair
            c2w = S.stereo_pair(pose)
            K = np.stack([S.intrinsics_fov(w, h)] * 2)
            res = np.array([[w, h]] * 2, np.int32)
        else:
            c2w, K, res = pose[None], S.intrinsics_fov(w, h)[None], np.array([[w, h]], np.int32)
        reqs.append((c2w, K, res))
    return reqs


def test_serving_matches_rendering_alone(V, room):
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    reqs = _mix(room, np.random.default_rng(41))
    want = [_alone(V, f, *r) for r in reqs]
    srv = V.Server(f, 256 << 20, "fp16")
    outs, tickets = [], []
    for c2w, K, res in reqs:  # submitted back to back: they share the GPU
        out = np.full((int((res[:, 0] * res[:, 1]).sum()), 3), np.nan, np.float32)
        outs.append(out)
        tickets.append(srv.submit(c2w, K, res, out))
    for t in tickets:
        srv.poll(t, 20000)
    for got, ref in zip(outs, want):
        assert np.isfinite(got).all()
        assert np.all(np.abs(got - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    V.vrnerf_field_status(f)
    f.close()


def test_serving_admits_by_hbm_budget(V, room):
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 256, 256)
    ref = _alone(V, f, c2w, K, res)
    one = 256 * 256 * 12
    srv = V.Server(f, one + one // 2, "fp16")  # room for one request's output at a time
    outs = [np.zeros((256 * 256, 3), np.float32) for _ in range(4)]
    ts = [srv.submit(c2w, K, res, o) for o in outs]
    for t in ts:
        srv.poll(t, 20000)
    for o in outs:
        assert np.all(np.abs(o - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
    big = np.array([[512, 512]], np.int32)
    with pytest.raises(V.VrnerfError) as e:
        srv.submit(c2w, S.intrinsics_fov(512, 512)[None], big, None)
    assert e.value.code == V.EINVAL
    srv.close()
    f.close()


def test_serving_cancel_unknown_and_timeout(V, room):
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 2048, 2048)
    srv = V.Server(f, 200 << 20, "fp16")
    t_big = srv.submit(c2w, K, res, np.zeros((2048 * 2048, 3), np.float32))
    t_cancel = srv.submit(c2w, K, res, np.zeros((2048 * 2048, 3), np.float32))
    srv.cancel(t_cancel)
    with pytest.raises(V.VrnerfError) as e:
        srv.poll(t_big, 0)
    assert e.value.code in (V.ETIMEDOUT,)
    srv.poll(t_big, 20000)
    with pytest.raises(V.VrnerfError) as e:
        srv.poll(t_cancel, 20000)
    assert e.value.code == V.ECANCELED
    with pytest.raises(V.VrnerfError) as e:
        srv.poll(123456789, 0)
    assert e.value.code == V.ENOTFOUND
    srv.close()
    f.close()


def test_serving_relaunches_after_idle_exit(V, room):
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 64, 64)
    ref = _alone(V, f, c2w, K, res)
    srv = V.Server(f, 16 << 20, "fp16")
    for _ in range(3):
        out = np.zeros((64 * 64, 3), np.float32)
        srv.poll(srv.submit(c2w, K, res, out), 20000)
        assert np.all(np.abs(out - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
        time.sleep(0.1)  # longer than the kernel's idle limit
    assert srv.stats()["kernel_launches"] >= 2
    srv.close()
    f.close()
