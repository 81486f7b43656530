"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on
the same seeded inputs.

Bit-exact: seeded parameters, hash-grid corner indices, occupancy visits,
per-ray sample counts. fp32 radiance: |gpu - oracle| <= 1e-4 |oracle| + 1e-6
in PQ space and in linear colour, except rays whose early-termination
decision flips at T_eps, which must agree within T_eps * max colour in PQ
space and are counted.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-6


@pytest.fixture(scope="module")
def V():
    from paper_2311_02542_gb300 import vrnerf
    vrnerf.load()
    return vrnerf


@pytest.fixture(scope="module")
def cube():
    return S.make_scene("unit_cube")


@pytest.fixture(scope="module")
def room():
    return S.make_scene("room")


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _close(gpu, ref, rtol=RTOL, atol=ATOL):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    return np.abs(gpu - ref) <= rtol * np.abs(ref) + atol


def check_render(gpu_pq, gpu_lin, gpu_n, ref, T_eps, rtol=RTOL, max_flip_frac=0.01):
    """Element-wise render parity with the early-termination allowance."""
    flip = gpu_n != ref["n"]
    ok_pq = _close(gpu_pq, ref["pq"], rtol).all(axis=1)
    ok_lin = _close(gpu_lin, ref["linear"], rtol).all(axis=1)
    good = ok_pq & ok_lin
    bad = ~good & ~flip
    assert not bad.any(), (f"{bad.sum()} rays out of tolerance; worst pq err "
                           f"{np.max(np.abs(gpu_pq - ref['pq'])[bad])}")
    if flip.any():
        d = np.abs(gpu_pq[flip] - ref["pq"][flip]).max()
        assert d <= T_eps * 1.0 + 1e-5, d
        assert flip.mean() <= max_flip_frac
    return int(flip.sum())


def render_gpu(V, field, c2w, K, res, precision=0):
    res = np.asarray(res, np.int32).reshape(-1, 2)
    rays = int((res[:, 0] * res[:, 1]).sum())
    pq = torch.empty((rays, 3), device="cuda")
    T = torch.empty(rays, device="cuda")
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(field, _cuda(c2w), _cuda(K), res, precision=precision, out_pq=pq,
                          out_T=T, out_n=n)
    torch.cuda.synchronize()
    return lin.cpu().numpy(), pq.cpu().numpy(), T.cpu().numpy(), n.cpu().numpy()


# ---------------------------------------------------------------------------
def test_seeded_init_matches_generator(V, cube, room):
    for sc in (cube, room):
        f = V.Field(sc.cfg, None, None, sc.occ_bits, seed=sc.seed)
        g, m = V.vrnerf_field_get_params(f)
        assert (g.view(np.uint16 if sc.cfg.feat_fp16 else np.uint32) ==
                sc.grid.view(np.uint16 if sc.cfg.feat_fp16 else np.uint32)).all()
        assert (m.view(np.uint32) == sc.mlp.view(np.uint32)).all()
        f.close()


def test_corner_indices_bit_exact(V, cube, room):
    rng = np.random.default_rng(11)
    for sc in (cube, room):
        cfg = sc.cfg
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        lo, hi = np.array(cfg.aabb_min), np.array(cfg.aabb_max)
        pos = (lo + (hi - lo) * rng.uniform(0, 1, (20000, 3))).astype(np.float32)
        pos[:8] = np.array([lo, hi, [lo[0], hi[1], lo[2]], hi - 1e-6, lo + 1e-7, (lo + hi) / 2,
                            [hi[0], lo[1], hi[2]], [lo[0], lo[1], hi[2]]], np.float32)
        ref, _ = O.corners(cfg, pos)
        got = V.vrnerf_debug_corners(f, _cuda(pos)).cpu().numpy().view(np.uint32)
        assert (got == ref).all()
        f.close()


def _rays_for_march(cfg, sc, n_side):
    if cfg.occ_res[0] == 64:
        c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, n_side, n_side)
    else:
        c2w, K, res = S.camera_room(sc.occ, cfg, 2, 2048, 2048)
        K = S.crop_camera(K, 1024 - n_side // 2, 1024 - n_side // 2)
        res = np.array([[n_side, n_side]], np.int32)
    return c2w, K, res


def test_march_visits_bit_exact(V, cube, room):
    for sc, side in ((cube, 64), (room, 96)):
        cfg = sc.cfg
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        c2w, K, res = _rays_for_march(cfg, sc, side)
        o, d, r = O.camera_rays(cfg, c2w, K, res)
        rng = np.random.default_rng(12)
        # add grazing rays along voxel faces and axis-parallel rays
        extra_o = (np.array(cfg.aabb_min) + rng.integers(1, 8, (64, 3)) /
                   np.array(cfg.occ_res) * (np.array(cfg.aabb_max) - np.array(cfg.aabb_min)))
        extra_d = np.zeros((64, 3))
        extra_d[np.arange(64), rng.integers(0, 3, 64)] = rng.choice([-1.0, 1.0], 64)
        o = np.concatenate([o, extra_o.astype(np.float32)])
        d = np.concatenate([d, extra_d.astype(np.float32)])
        cap = cfg.max_steps
        ri, rv, cnt = F.march(o, d, cap)
        gi, gv, gc = V.vrnerf_debug_march(f, _cuda(o), _cuda(d), cap)
        gi, gv, gc = gi.cpu().numpy(), gv.cpu().numpy(), gc.cpu().numpy()
        assert (gc == cnt).all()
        assert (gi == ri).all() and (gv == rv).all()
        assert cnt.sum() > 1000
        f.close()


def test_march_skip_stress_bit_exact(V, cube, room):
    """Empty-space skipping must reproduce the per-sample occupancy rule on
    arbitrary rays: random origins and directions, directions close to the
    axes and to the diagonals, origins on voxel faces and pyramid-block
    faces, origins outside the box."""
    rng = np.random.default_rng(21)
    for sc in (cube, room):
        cfg = sc.cfg
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        lo, hi = np.array(cfg.aabb_min), np.array(cfg.aabb_max)
        res = np.array(cfg.occ_res)
        n = 12000
        o = lo + (hi - lo) * rng.uniform(-0.05, 1.05, (n, 3))
        # a third of the origins exactly on voxel or block faces
        k = n // 3
        cells = rng.integers(0, res, (k, 3)) // rng.choice([1, 2, 4, 8, 16], (k, 1)) * 1.0
        o[:k] = lo + (hi - lo) * cells / res
        d = rng.normal(size=(n, 3))
        m = n // 4
        d[k:k + m] = np.eye(3)[rng.integers(0, 3, m)] * rng.choice([-1, 1], (m, 1)) + \
            rng.normal(scale=1e-4, size=(m, 3)) * rng.integers(0, 2, (m, 1))
        d[k + m:k + 2 * m] = rng.choice([-1.0, 1.0], (m, 3)) + rng.normal(scale=1e-5, size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        o, d = o.astype(np.float32), d.astype(np.float32)
        cap = 64
        ri, rv, cnt = F.march(o, d, cap)
        gi, gv, gc = V.vrnerf_debug_march(f, _cuda(o), _cuda(d), cap)
        gi, gv, gc = gi.cpu().numpy(), gv.cpu().numpy(), gc.cpu().numpy()
        bad = np.nonzero((gc != cnt) | (gi != ri).any(1) | (gv != rv).any(1))[0]
        assert bad.size == 0, (bad[:5], o[bad[:2]], d[bad[:2]], cnt[bad[:2]], gc[bad[:2]])
        assert cnt.sum() > 10000
        f.close()


def test_query_parity(V, cube, room):
    rng = np.random.default_rng(13)
    for sc in (cube, room):
        cfg = sc.cfg
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        n = 3000
        lo, hi = np.array(cfg.aabb_min), np.array(cfg.aabb_max)
        pos = (lo + (hi - lo) * rng.uniform(0, 1, (n, 3))).astype(np.float32)
        d = rng.normal(size=(n, 3))
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
        rad = (10 ** rng.uniform(-6, -1, n)).astype(np.float32)
        rad[:10] = 0.0
        sig, rgb, feat = F.query(pos, d, rad)
        gs, gr, gf = V.vrnerf_query(f, _cuda(pos), _cuda(d), _cuda(rad), with_feat=True)
        assert _close(gs.cpu().numpy(), sig).all()
        assert _close(gr.cpu().numpy(), rgb).all()
        assert _close(gf.cpu().numpy(), feat, atol=1e-8).all()
        f.close()


def test_render_unit_cube_parity(V, cube):
    cfg = cube.cfg
    for c in (cfg, replace(cfg, density_bias=4.0)):
        f = V.Field(c, cube.grid, cube.mlp, cube.occ_bits)
        F = O.Field(c, cube.grid, cube.mlp, cube.occ_bits)
        c2w, K, res = S.camera_unit_cube(cube.occ, c, 1, 64, 64)
        ref = F.render(c2w, K, res)
        lin, pq, T, n = render_gpu(V, f, c2w, K, res)
        check_render(pq, lin, n, ref, c.T_eps)
        assert ref["n"].max() > 5
        f.close()


@pytest.mark.parametrize("variant", ["room", "room_surface"])
def test_render_room_crop_parity(V, room, variant):
    cfg = S.cfg_room(surface=(variant == "room_surface"))
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, _ = S.camera_room(room.occ, cfg, 2, 2048, 2048)
    rng = np.random.default_rng(14)
    flips = 0
    for _ in range(3):
        x0, y0 = rng.integers(0, 2048 - 100, 2)
        Kc = S.crop_camera(K, int(x0), int(y0))
        res = np.array([[100, 61]], np.int32)  # ragged against the 8 x 4 ray tiles
        ref = F.render(c2w, Kc, res)
        lin, pq, T, n = render_gpu(V, f, c2w, Kc, res)
        flips += check_render(pq, lin, n, ref, cfg.T_eps)
    f.close()


def test_render_full_frame_sampled(V, room):
    cfg = room.cfg
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, cfg, 2, 2048, 2048)
    lin, pq, T, n = render_gpu(V, f, c2w, K, res)
    o, d, r = O.camera_rays(cfg, c2w, K, res)
    pick = np.random.default_rng(15).choice(o.shape[0], 4000, replace=False)
    ref = F.render_rays(o[pick], d[pick], r[pick])
    check_render(pq[pick], lin[pick], n[pick], ref, cfg.T_eps)
    assert np.isfinite(lin).all() and (lin >= 0).all()
    f.close()


def test_render_multiview_ragged_and_tiny(V, cube):
    cfg = cube.cfg
    f = V.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
    F = O.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
    views = [S.camera_unit_cube(cube.occ, cfg, s, w, h) for s, w, h in ((3, 37, 23), (4, 1, 1), (5, 64, 9))]
    c2w = np.concatenate([v[0] for v in views])
    K = np.concatenate([v[1] for v in views])
    res = np.concatenate([v[2] for v in views])
    ref = F.render(c2w, K, res)
    lin, pq, T, n = render_gpu(V, f, c2w, K, res)
    check_render(pq, lin, n, ref, cfg.T_eps)
    f.close()


def test_empty_occupancy_is_black(V, cube):
    cfg = cube.cfg
    f = V.Field(cfg, cube.grid, cube.mlp, S.pack_bits(np.zeros_like(cube.occ)))
    c2w, K, res = S.camera_unit_cube(cube.occ, cfg, 1, 40, 24)
    lin, pq, T, n = render_gpu(V, f, c2w, K, res)
    assert (lin == 0).all() and (pq == 0).all() and (n == 0).all() and (T == 1).all()
    f.close()


def test_render_host_matches_device(V, cube):
    cfg = cube.cfg
    f = V.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
    c2w, K, res = S.camera_unit_cube(cube.occ, cfg, 1, 64, 48)
    a = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res).cpu().numpy()
    b = V.vrnerf_render_host(f, c2w, K, res)  # pageable output: staging buffer and copy
    assert (a == b).all()
    # pinned output: the kernel writes into host memory itself
    pinned = torch.full((a.shape[0], 3), -1.0, dtype=torch.float32).pin_memory().numpy()
    c = V.vrnerf_render_host(f, c2w, K, res, out=pinned)
    assert c is pinned and (a == c).all()
    for prec in ("fp16", "bf16"):
        ref = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=prec).cpu().numpy()
        pinned[:] = -1.0
        V.vrnerf_render_host(f, c2w, K, res, out=pinned, precision=prec)
        assert (ref == pinned).all()
    f.close()


def test_invalid_arguments_are_rejected(V, cube):
    cfg = cube.cfg
    f = V.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
    c2w, K, res = S.camera_unit_cube(cube.occ, cfg, 1, 8, 8)
    for bad in (np.array([[0, 8]]), np.array([[8, 20000]])):
        with pytest.raises(V.VrnerfError) as e:
            V.vrnerf_render(f, _cuda(c2w), _cuda(K), bad, out=torch.empty((64, 3), device="cuda"))
        assert e.value.code == V.EINVAL
    with pytest.raises(V.VrnerfError):
        V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=9)
    f.close()


@pytest.mark.parametrize("prec,rtol", [("fp32", 1e-4), ("fp16", 2e-3)])
def test_render_depth_parity(V, cube, room, prec, rtol):
    """Expected depth sum_i w_i t_i (the paper's depth maps) against the oracle."""
    cases = [(cube, S.cfg_unit_cube(), S.camera_unit_cube(cube.occ, cube.cfg, 1, 48, 40))]
    cfg_s = S.cfg_room(surface=True)
    c2w, K, _ = S.camera_room(room.occ, cfg_s, 2, 2048, 2048)
    cases.append((room, cfg_s, (c2w, S.crop_camera(K, 700, 900), np.array([[96, 72]], np.int32))))
    for sc, cfg, (c2w, K, res) in cases:
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        ref = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits).render(c2w, K, res)
        rays = int(res[0, 0] * res[0, 1])
        dep = torch.empty(rays, device="cuda")
        n = torch.empty(rays, device="cuda", dtype=torch.int32)
        V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=prec, out_depth=dep, out_n=n)
        dep, n = dep.cpu().numpy(), n.cpu().numpy()
        same = n == ref["n"]
        assert same.mean() > 0.99 and ref["depth"].max() > 0
        assert np.all(np.abs(dep[same] - ref["depth"][same]) <= rtol * np.abs(ref["depth"][same]) + 1e-6)
        f.close()
