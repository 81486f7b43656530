"""The seeded synthetic inputs follow their stated recipe: serving request mix
(Poisson arrivals at 36/0.7 req/s, 70 % stereo pairs 63 mm apart, singles of
side 512 / 1024 / 1536, pitch and roll within 30 degrees), training batches
(90 degree frusta, HDR targets log-uniform in [1e-3, 1e3]) and the benchmark
camera (1.7 m eye height, level)."""
import math

import numpy as np
import pytest

from paper_2311_02542_gb300 import synth as S


@pytest.fixture(scope="module")
def room():
    return S.make_scene("room", with_params=False)


def _orthonormal(m):
    R = m[:, :3].astype(np.float64)
    return np.allclose(R.T @ R, np.eye(3), atol=1e-6)


def test_pose_frame_is_orthonormal_and_right_handed():
    for yaw, pitch, roll in ((0.3, 0.2, -0.4), (2.0, -0.5, 0.1), (5.0, 0.0, 0.0)):
        m = S.pose_from_angles(np.zeros(3), yaw, pitch, roll)
        assert _orthonormal(m)
        right, down, fwd = (m[:, k].astype(np.float64) for k in range(3))
        assert np.allclose(np.cross(fwd, right), down, atol=1e-6)  # x right, y down, z forward
        assert fwd[2] == pytest.approx(math.sin(pitch), abs=1e-6)


def test_request_stream_mix_rate_and_poses(room):
    rate = 36.0 / 0.7
    reqs = S.request_stream(room.occ, room.cfg, 2000, rate_hz=rate)
    t = np.array([r.arrival_s for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert gaps.mean() == pytest.approx(1.0 / rate, rel=0.06)
    assert gaps.std() == pytest.approx(1.0 / rate, rel=0.1)  # exponential: std = mean
    stereo = [r for r in reqs if r.stereo]
    assert len(stereo) / len(reqs) == pytest.approx(0.7, abs=0.03)
    sides = [int(r.resolution[0, 0]) for r in reqs if not r.stereo]
    counts = {s: sides.count(s) for s in (512, 1024, 1536)}
    assert sum(counts.values()) == len(sides) and min(counts.values()) > 0.25 * len(sides)
    for r in stereo[:200]:
        assert r.resolution.tolist() == [[2048, 2048], [2048, 2048]]
        left, right = r.c2w[0].astype(np.float64), r.c2w[1].astype(np.float64)
        assert np.linalg.norm(right[:, 3] - left[:, 3]) == pytest.approx(0.063, abs=1e-5)
        assert np.allclose(left[:, :3], right[:, :3])
    s30 = math.sin(math.radians(30)) + 1e-6
    for r in reqs[:300]:
        m = r.c2w[0].astype(np.float64)
        assert _orthonormal(r.c2w[0])
        assert abs(m[2, 2]) <= s30  # pitch
        assert np.all((m[:, 3] > 0) & (m[:, 3] < np.array(room.cfg.aabb_max)))


def test_training_batch_frusta_and_targets(room):
    poses, intr = S.training_views(room.occ, room.cfg, n_views=64)
    assert poses.shape == (64, 3, 4)
    o, d, r, tgt = S.training_batch(poses, intr, 1 << 16, seed=5, step=3)
    assert np.allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.all(r == np.float32(0.5 / float(intr[0])))
    # every ray lies in the 90 degree frustum of the view it starts from
    k = np.array([np.flatnonzero((poses[:, :, 3] == oi).all(axis=1))[0] for oi in o[:2000]])
    P = poses[k].astype(np.float64)
    dd = d[:2000].astype(np.float64)
    fwd = np.einsum("ij,ij->i", dd, P[:, :, 2])
    assert np.all(fwd > 0)
    for axis in (0, 1):
        assert np.all(np.abs(np.einsum("ij,ij->i", dd, P[:, :, axis]) / fwd) <= 1.0 + 1e-6)
    assert tgt.min() >= 1e-3 * (1 - 1e-6) and tgt.max() <= 1e3 * (1 + 1e-6)
    lg = np.log(tgt.astype(np.float64))
    assert lg.mean() == pytest.approx(0.0, abs=0.05)
    assert lg.std() == pytest.approx(2 * math.log(1e3) / math.sqrt(12), rel=0.02)  # uniform in log
    # another step draws another batch
    o2, _, _, _ = S.training_batch(poses, intr, 1 << 16, seed=5, step=4)
    assert not np.array_equal(o, o2)


def test_benchmark_camera_is_level_at_eye_height(room):
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 2048, 2048)
    m = c2w[0].astype(np.float64)
    assert m[2, 3] == pytest.approx(1.7, abs=1e-6)
    assert abs(m[2, 2]) < 1e-6  # forward is horizontal
    assert res.tolist() == [[2048, 2048]]
    assert float(K[0, 0]) == pytest.approx(1024.0, rel=1e-6)  # 90 degree field of view


def test_unbounded_room_has_windows_ground_and_far_buildings():
    sc = S.make_scene("room_unbounded", with_params=False)
    cfg = sc.cfg
    assert cfg.contract and sc.occ.shape == (256, 256, 256)
    cen = (np.array(cfg.aabb_min) + np.array(cfg.aabb_max)) / 2
    h = 0.5 * max(np.array(cfg.aabb_max) - np.array(cfg.aabb_min))

    def occupied(p):
        x = (np.asarray(p, np.float64) - cen) / h
        m = np.abs(x).max()
        y = x if m <= 1 else (2 - 1 / m) * x / m
        i = np.minimum(((y + 2) / 4 * 256).astype(int), 255)
        return bool(sc.occ[i[2], i[1], i[0]])

    assert occupied((10.0, 10.0, -0.5))      # floor / ground under the room
    assert occupied((-0.1, 1.5, 1.6))        # wall between windows
    assert not occupied((-0.1, 5.0, 1.6))    # window opening in the same wall
    assert not occupied((10.0, 10.0, 1.7))   # eye height in the room
    assert occupied((400.0, 10.0, -0.5))     # ground far outside (the slab -1 <= z <= 0)
    # buildings: occupied voxels above the horizon outside the inner cube
    n = 256
    yc = (np.arange(n) + 0.5) / n * 4 - 2
    far = (np.abs(yc)[None, :] > 1.2) | (np.abs(yc)[:, None] > 1.2)  # [y][x]
    above = yc > 0.02
    assert sc.occ[above][:, far].any()
