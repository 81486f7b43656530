"""Continuous-batching server: every request's image equals the same views
rendered alone (vrnerf_render, same precision) within the tensor-core
tolerance, and the fp64 oracle's render within 2e-3 |ref| + 1e-5 (rays whose
early termination flips at T_eps, found from the alone render's sample
counts, within T_eps + 1e-4 in PQ); requests overlap on the device (tiles
whose MLP rows mix requests); admission by HBM budget; cancel, unknown
tickets, timeouts; the persistent kernel leaves when idle and is relaunched
for new work."""
import time

import numpy as np
import pytest
import torch

import oracle as O
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


def _alone_n(V, f, c2w, K, res):
    """Linear colour and per-ray sample counts of the fp16 render alone."""
    rays = int((res[:, 0] * res[:, 1]).sum())
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(f, torch.from_numpy(c2w).cuda(), torch.from_numpy(K).cuda(), res,
                          precision="fp16", out_n=n)
    return lin.cpu().numpy(), n.cpu().numpy()


def _check_against_oracle(got_lin, n_gpu, ref, T_eps):
    """Served linear colour against the oracle: fp16 tolerance, with the
    rays whose sample count differs at T_eps held to T_eps in PQ."""
    flip = n_gpu != ref["n"]
    ok = np.abs(got_lin.astype(np.float64) - ref["linear"]) <= TC_RTOL * np.abs(ref["linear"]) + TC_ATOL
    bad = ~ok.all(1) & ~flip
    assert not bad.any(), (bad.sum(), np.abs(got_lin - ref["linear"])[bad].max())
    if flip.any():
        pq = np.array([[O.linear_to_pq(float(c)) for c in row] for row in got_lin[flip]])
        assert np.abs(pq - ref["pq"][flip]).max() <= T_eps + 1e-4
        assert flip.mean() <= 0.01


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
    # the requests shared the GPU: several were admitted at once, and MLP
    # tiles held samples of more than one request
    print(f"serving overlap: max in flight {st['max_inflight']}, tile rounds {st['tile_rounds']}, "
          f"mixed {st['mixed_tile_rounds']}")
    assert st["max_inflight"] >= 2
    assert st["mixed_tile_rounds"] >= 1 and st["tile_rounds"] > st["mixed_tile_rounds"]
    srv.close()
    V.vrnerf_field_status(f)
    # every served image against the fp64 oracle
    F = O.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    for (c2w, K, res), got in zip(reqs, outs):
        _, n_gpu = _alone_n(V, f, c2w, K, res)
        _check_against_oracle(got, n_gpu, F.render(c2w, K, res), room.cfg.T_eps)
    f.close()


@pytest.mark.parametrize("variant", ["room", "room_surface"])
def test_serving_stereo_2048_against_oracle(V, variant):
    """One stereo pair of 2048^2 eye buffers (Sec. 5) through the server: 4 000
    sampled pixels of each eye against the fp64 oracle."""
    sc = S.make_scene(variant)
    f = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    pose, _, _ = S.camera_room(sc.occ, sc.cfg, 2, 2048, 2048)
    c2w = S.stereo_pair(pose[0])
    K = np.stack([S.intrinsics_fov(2048, 2048)] * 2)
    res = np.array([[2048, 2048]] * 2, np.int32)
    srv = V.Server(f, 256 << 20, "fp16")
    out = np.full((2 * 2048 * 2048, 3), np.nan, np.float32)
    srv.poll(srv.submit(c2w, K, res, out), 30000)
    srv.close()
    assert np.isfinite(out).all()
    _, n_gpu = _alone_n(V, f, c2w, K, res)
    o, d, r = O.camera_rays(sc.cfg, c2w, K, res)
    pick = np.sort(np.random.default_rng(43).choice(o.shape[0], 8000, replace=False))
    F = O.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    ref = F.render_rays(o[pick], d[pick], r[pick])
    _check_against_oracle(out[pick], n_gpu[pick], ref, sc.cfg.T_eps)
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


def test_serving_deadlines_order_and_shed(V, room):
    """Waiting requests are admitted earliest deadline first, and a request
    whose deadline passes while it waits is shed when it asked to be. The
    budget holds one 512^2 output at a time, so admission is sequential."""
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 512, 512)
    one = 512 * 512 * 12
    srv = V.Server(f, one + one // 2, "fp16")
    outs = [np.zeros((512 * 512, 3), np.float32) for _ in range(4)]
    t_a = srv.submit(c2w, K, res, outs[0])                          # admitted at once
    t_b = srv.submit(c2w, K, res, outs[1])                          # no deadline, arrives first
    t_c = srv.submit(c2w, K, res, outs[2], deadline_ms=10000.0)     # deadline: goes ahead of b
    t_d = srv.submit(c2w, K, res, outs[3], deadline_ms=0.001, shed_if_late=True)
    lat = {t: srv.poll(t, 20000) for t in (t_a, t_c, t_b)}
    with pytest.raises(V.VrnerfError) as e:
        srv.poll(t_d, 20000)
    assert e.value.code == V.ELATE
    # c was submitted after b and finished before it
    assert lat[t_c] < lat[t_b]
    ref = _alone(V, f, c2w, K, res)
    for o in outs[:3]:
        assert np.all(np.abs(o - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
    st = srv.stats()
    assert st["shed"] == 1 and st["late"] == 0 and st["completed"] == 3
    assert st["gpu_p99_ms"] >= st["gpu_p50_ms"] > 0 and st["wait_p99_ms"] > 0 and st["copy_p50_ms"] > 0
    with pytest.raises(V.VrnerfError):
        srv.submit(c2w, K, res, None, deadline_ms=-1.0)
    srv.close()
    f.close()


def test_serving_writes_pinned_outputs_directly(V, room):
    """An output buffer in pinned host memory is written by the kernel itself:
    it takes no part of the HBM budget (here 1 MiB, far below the outputs)
    and needs no copy-out; the images equal rendering alone. A pageable
    buffer of the same size is still refused against that budget."""
    f = V.Field(room.cfg, room.grid, room.mlp, room.occ_bits)
    srv = V.Server(f, 1 << 20, "fp16")
    reqs = _mix(room, np.random.default_rng(47))[:5]
    outs, tickets = [], []
    for c2w, K, res in reqs:
        out = torch.empty((int((res[:, 0] * res[:, 1]).sum()), 3), dtype=torch.float32, pin_memory=True).numpy()
        out.fill(np.nan)
        outs.append(out)
        tickets.append(srv.submit(c2w, K, res, out))
    for t in tickets:
        srv.poll(t, 20000)
    for (c2w, K, res), got in zip(reqs, outs):
        ref = _alone(V, f, c2w, K, res)
        assert np.isfinite(got).all()
        assert np.all(np.abs(got - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["copy_p99_ms"] < 1.0
    c2w, K, res = S.camera_room(room.occ, room.cfg, 2, 512, 512)   # 3 MB of output
    with pytest.raises(V.VrnerfError) as e:
        srv.submit(c2w, K, res, np.zeros((512 * 512, 3), np.float32))
    assert e.value.code == V.EINVAL
    pinned = torch.empty((512 * 512, 3), dtype=torch.float32, pin_memory=True).numpy()
    srv.poll(srv.submit(c2w, K, res, pinned), 20000)
    ref = _alone(V, f, c2w, K, res)
    assert np.all(np.abs(pinned - ref) <= TC_RTOL * np.abs(ref) + TC_ATOL)
    srv.close()
    f.close()
