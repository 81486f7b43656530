"""GPU parity of unbounded (contracted) scenes against the oracle: the
L-infinity contraction (Sec. 4) in the march and the hash grid, the
adjacent-ray footprint of camera rays and the Jacobian footprint of
explicit rays (Sec. 4.2.1), through every kernel family.

Bars as for bounded scenes: corner indices and occupancy visits bit-exact;
fp32 radiance <= 1e-4 |ref| + 1e-6; fp16 tensor cores <= 2e-3 |ref| + 1e-5;
gradients <= 1e-4 |ref| + 1e-5 max|ref|; rays whose sample count differs at
T_eps excluded (<= 1 %) and held to T_eps in PQ.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-6
TC_RTOL, TC_ATOL = 2e-3, 1e-5


@pytest.fixture(scope="module")
def V():
    from paper_2311_02542_gb300 import vrnerf
    vrnerf.load()
    return vrnerf


@pytest.fixture(scope="module")
def unit():
    """Unit box inside an unbounded scene: 32^3 contracted occupancy with
    15 % of the voxels set, random fp32 features and weights, samples to
    t = 200."""
    cfg = replace(S.cfg_unit_cube(), contract=True, t_far=200.0, max_steps=128, occ_res=(32, 32, 32),
                  density_bias=1.0)
    rng = np.random.default_rng(12)
    occ = rng.uniform(size=(32, 32, 32)) < 0.15
    occ[8:24, 8:24, 8:24] &= rng.uniform(size=(16, 16, 16)) < 0.3  # inner cube sparser
    grid = rng.uniform(-1, 1, (cfg.levels, cfg.T, cfg.feats)).astype(np.float32)
    mlp = (rng.normal(size=O.mlp_count(cfg)) * 0.5).astype(np.float32)
    return cfg, occ, grid, mlp


@pytest.fixture(scope="module")
def room():
    return S.make_scene("room_unbounded_surface")


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _close(gpu, ref, rtol, atol):
    return np.abs(np.asarray(gpu, np.float64) - ref) <= rtol * np.abs(ref) + atol


def _check(lin, pq, n, ref, T_eps, rtol=RTOL, atol=ATOL, max_flip=0.01):
    flip = n != ref["n"]
    good = _close(pq, ref["pq"], rtol, atol).all(1) & _close(lin, ref["linear"], rtol, atol).all(1)
    bad = ~good & ~flip
    assert not bad.any(), (bad.sum(), np.abs(pq - ref["pq"])[bad].max())
    if flip.any():
        assert np.abs(pq[flip] - ref["pq"][flip]).max() <= T_eps + 1e-4
    assert flip.mean() <= max_flip


def _render(V, f, c2w, K, res, precision=0):
    res = np.asarray(res, np.int32).reshape(-1, 2)
    rays = int((res[:, 0] * res[:, 1]).sum())
    pq = torch.empty((rays, 3), device="cuda")
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=precision, out_pq=pq, out_n=n)
    V.vrnerf_field_status(f)
    return lin.cpu().numpy(), pq.cpu().numpy(), n.cpu().numpy()


def _far_rays(cfg, rng, n):
    """Origins inside and far outside the inner cube, random directions plus
    axis-parallel ones."""
    o = np.concatenate([rng.uniform(0.1, 0.9, (n // 2, 3)), 0.5 + rng.normal(size=(n - n // 2, 3)) * 20])
    d = rng.normal(size=(n, 3))
    d[: n // 8] = 0
    d[np.arange(n // 8), rng.integers(0, 3, n // 8)] = rng.choice([-1.0, 1.0], n // 8)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)


def test_contracted_corners_bit_exact(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    rng = np.random.default_rng(1)
    pos = (0.5 + rng.normal(size=(20000, 3)) * rng.choice([0.3, 3.0, 300.0], (20000, 1))).astype(np.float32)
    pos[:4] = [[0.5, 0.5, 0.5], [1.0, 0.5, 0.5], [1e6, -3.0, 2.0], [0.0, 1.0, 0.0]]
    ref, _ = O.corners(cfg, pos)
    got = V.vrnerf_debug_corners(f, _cuda(pos)).cpu().numpy().view(np.uint32)
    assert (got == ref).all()
    f.close()


def test_contracted_march_bit_exact(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    o, d = _far_rays(cfg, np.random.default_rng(2), 4000)
    ri, rv, cnt = F.march(o, d, cfg.max_steps)
    gi, gv, gc = (t.cpu().numpy() for t in V.vrnerf_debug_march(f, _cuda(o), _cuda(d), cfg.max_steps))
    assert (gc == cnt).all() and (gi == ri).all() and (gv == rv).all()
    assert cnt.sum() > 10000
    f.close()


def test_contracted_render_fp32_camera_adjacent_footprint(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    for seed in (1, 2):
        c2w, K, res = S.camera_unit_cube(occ, cfg, seed, 48, 40)
        lin, pq, n = _render(V, f, c2w, K, res)
        ref = F.render(c2w, K, res)
        assert (ref["n"] > 0).mean() > 0.5
        _check(lin, pq, n, ref, cfg.T_eps)
    f.close()


def test_contracted_render_rays_jacobian_footprint(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    o, d = _far_rays(cfg, np.random.default_rng(3), 2000)
    r = np.full(2000, 1e-3, np.float32)
    ref = F.render_rays(o, d, r)
    pq = torch.empty((2000, 3), device="cuda")
    n = torch.empty(2000, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render_rays(f, _cuda(o), _cuda(d), _cuda(r), out_pq=pq, out_n=n)
    _check(lin.cpu().numpy(), pq.cpu().numpy(), n.cpu().numpy(), ref, cfg.T_eps)
    # the camera-ray footprint differs from the explicit-ray one: a camera
    # render is not the same as rendering its rays explicitly
    c2w, K, res = S.camera_unit_cube(occ, cfg, 1, 48, 40)
    oc, dc, rc = O.camera_rays(cfg, c2w, K, res)
    a = F.render_rays(oc, dc, rc)["pq"]
    b = F.render(c2w, K, res)["pq"]
    assert np.abs(a - b).max() > 1e-6
    f.close()


def test_contracted_query(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    rng = np.random.default_rng(4)
    pos = (0.5 + rng.normal(size=(5000, 3)) * rng.choice([0.3, 3.0, 30.0], (5000, 1))).astype(np.float32)
    dirs = rng.normal(size=(5000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    rad = np.exp(rng.uniform(np.log(1e-4), np.log(1.0), 5000))
    sig, rgb, _ = F.query(pos, dirs, rad)
    gs, grgb, _ = V.vrnerf_query(f, _cuda(pos), _cuda(dirs), _cuda(rad))
    assert _close(gs.cpu().numpy(), sig, RTOL, ATOL).all()
    assert _close(grgb.cpu().numpy(), rgb, RTOL, ATOL).all()
    f.close()


def _relu_margin(F, cfg, mlp, o, d, r):
    """Smallest |pre-activation| / (|W| |input|) over the ReLUs of every
    sample the rays composite (T_eps = 0): below ~1e-6 fp32 and fp64 may take
    different subgradients there, and a gradient comparison is ill-posed."""
    ri, rv, cnt = F.march(o, d, cfg.max_steps)
    t = O.sample_table(cfg)
    P, R, Dd = [], [], []
    for b in range(o.shape[0]):
        for k in range(cnt[b]):
            i = ri[b, k]
            P.append((o[b] + np.float32(t[i]) * d[b]).astype(np.float32))
            R.append(float(t[i]) * float(r[b]))
            Dd.append(d[b])
    Dd = np.array(Dd, np.float64)
    _, _, feat = F.query(np.array(P), Dd, np.array(R))
    D = cfg.d_in
    m = mlp.astype(np.float64)
    W1 = m[:64 * D].reshape(64, D)
    W2 = m[64 * D:64 * D + 1024].reshape(16, 64)
    W3 = m[64 * D + 1024:64 * D + 3072].reshape(64, 32)
    W4 = m[64 * D + 3072:64 * D + 7168].reshape(64, 64)
    x = np.concatenate([np.maximum(feat @ W1.T, 0) @ W2.T, np.stack([O.sh16(v) for v in Dd])], 1)
    h1 = np.maximum(x @ W3.T, 0)
    margins = []
    for W, inp in ((W1, feat), (W3, x), (W4, h1)):
        margins.append((np.abs(inp @ W.T) / (np.abs(inp) @ np.abs(W).T + 1e-30)).min())
    return min(margins)


def test_contracted_backward(V, unit):
    """Explicit rays with the Jacobian footprint through the training path.
    The view (12 x 12 pixels) is the first seeded one whose samples keep every
    ReLU at least 3e-6 (relative) away from its kink, ten times the fp32
    rounding of a 64-term pre-activation."""
    cfg, occ, grid, mlp = unit
    cfg = replace(cfg, T_eps=0.0)  # no early-termination flips: the same samples on both sides
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    for seed in range(2, 30):
        c2w, K, res = S.camera_unit_cube(occ, cfg, seed, 12, 12)
        o, d, r = O.camera_rays(cfg, c2w, K, res)
        if _relu_margin(F, cfg, mlp, o, d, r) > 3e-6:
            break
    else:
        pytest.fail("no well-conditioned view among the seeds")
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    tgt = np.exp(np.random.default_rng(5).uniform(-3, 3, (o.shape[0], 3))).astype(np.float32)
    loss_ref, rg, rm = F.backward(o, d, r, tgt)
    loss = V.vrnerf_backward(f, _cuda(o), _cuda(d), _cuda(r), _cuda(tgt))
    gg, gm = V.vrnerf_field_get_grads(f)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    for got, ref in ((gm, rm), (gg.reshape(-1), rg.reshape(-1))):
        scale = np.abs(ref).max()
        assert scale > 0
        ok = np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * scale
        assert ok.all(), (np.count_nonzero(~ok), np.abs(got - ref)[~ok].max(), scale)
    f.close()


def test_contracted_normals(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    c2w, K, res = S.camera_unit_cube(occ, cfg, 3, 32, 32)
    nrm = torch.empty((32 * 32, 3), device="cuda")
    n = torch.empty(32 * 32, device="cuda", dtype=torch.int32)
    V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, out_normal=nrm, out_n=n)
    ref = F.render(c2w, K, res, normals=True)
    same = n.cpu().numpy() == ref["n"]
    assert same.mean() > 0.99
    err = np.abs(nrm.cpu().numpy() - ref["normal"])[same]
    assert (err <= 2e-3).all(), err.max()
    f.close()


def test_contracted_prune(V, unit):
    cfg, occ, grid, mlp = unit
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    cams = np.array([[0.5, 0.5, 0.5], [0.2, 0.7, 0.4]], np.float32)
    _, alpha_ref = O.prune(F, cams, 2, 0.0)
    _, alpha, _ = V.vrnerf_prune(f, cams, 2, 0.0, apply=False, want_alpha=True)
    alpha = alpha.reshape(occ.shape)
    assert (alpha[~occ] == 0).all()
    # Outside the inner cube the k^3 lattice points are mapped back through the
    # inverse contraction, whose conditioning near the cube's edge amplifies
    # the fp32 rounding of a point, and their camera distance comes from
    # sampled points: fp32 against fp64 can pick a neighbouring sample interval
    # where the distance sits on a sample boundary. So every voxel matches
    # within 1e-4, or its optical depth -ln(1 - alpha) differs from the
    # oracle's by the ratio q of adjacent exponential intervals
    # (delta_{i+1} / delta_i = q), or, outside the inner cube only, by 1e-3.
    ok = np.abs(alpha - alpha_ref) <= 1e-4 * alpha_ref + 1e-6
    assert ok[occ].mean() > 0.99, ok[occ].mean()
    q = (cfg.t_far / cfg.t_near) ** (1.0 / cfg.max_steps)
    inner = np.zeros(occ.shape, bool)
    inner[8:24, 8:24, 8:24] = True  # the inner cube |x|_inf <= 1 of the 32^3 contracted grid
    bad = occ & ~ok
    tau = -np.log1p(-alpha[bad].astype(np.float64))
    tau_ref = -np.log1p(-alpha_ref[bad])
    ratio = tau / tau_ref
    neighbour = (np.abs(ratio - q) <= 1e-3 * q) | (np.abs(ratio - 1 / q) <= 1e-3 / q)
    near = (np.abs(ratio - 1) <= 1e-3) & ~inner[bad]
    assert (neighbour | near).all(), (bad.sum(), ratio[~(neighbour | near)][:5])
    f.close()


def test_contracted_room_fp32_and_fp16(V, room):
    cfg = room.cfg
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, _ = S.camera_room(room.occ, cfg, 2, 2048, 2048)
    K = S.crop_camera(K, 992, 992)
    res = np.array([[64, 64]], np.int32)
    ref = F.render(c2w, K, res)
    lin, pq, n = _render(V, f, c2w, K, res)
    _check(lin, pq, n, ref, cfg.T_eps)
    lin, pq, n = _render(V, f, c2w, K, res, precision=1)
    _check(lin, pq, n, ref, cfg.T_eps, TC_RTOL, TC_ATOL)
    f.close()


def test_contracted_serving_matches_rendering_alone(V, room):
    cfg = room.cfg
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, res = S.camera_room(room.occ, cfg, 3, 192, 160)
    want = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision="fp16").cpu().numpy()
    srv = V.Server(f, 64 << 20, "fp16")
    out = np.full((192 * 160, 3), np.nan, np.float32)
    srv.poll(srv.submit(c2w, K, res, out), 20000)
    assert np.all(np.abs(out - want) <= TC_RTOL * np.abs(want) + TC_ATOL)
    srv.close()
    f.close()


def test_contracted_skip_stress_room(V, room):
    """The contracted empty-space skip (a Lipschitz bound of the contraction
    along the ray) must reproduce the per-sample rule: camera rays through the
    windows out to 4 km, rays from far outside, grazing and axis-parallel rays."""
    cfg = room.cfg
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    rng = np.random.default_rng(22)
    c2w, K, _ = S.camera_room(room.occ, cfg, 5, 2048, 2048, n=4)
    o_list, d_list = [], []
    for v in range(4):
        Kc = S.crop_camera(K[v:v + 1], int(rng.integers(0, 1900)), int(rng.integers(0, 1900)))
        o, d, _ = O.camera_rays(cfg, c2w[v:v + 1], Kc, np.array([[64, 64]], np.int32))
        o_list.append(o)
        d_list.append(d)
    n = 6000
    far_o = (np.array([10.0, 10.0, 1.5]) + rng.normal(size=(n, 3)) * rng.choice([5.0, 100.0, 2000.0], (n, 1)))
    far_d = rng.normal(size=(n, 3))
    far_d[: n // 6] = 0
    far_d[np.arange(n // 6), rng.integers(0, 3, n // 6)] = rng.choice([-1.0, 1.0], n // 6)
    far_d[n // 6: n // 3, 2] = rng.uniform(-1e-3, 1e-3, n // 6)  # nearly horizontal
    far_d /= np.linalg.norm(far_d, axis=1, keepdims=True)
    o = np.concatenate(o_list + [far_o.astype(np.float32)])
    d = np.concatenate(d_list + [far_d.astype(np.float32)])
    cap = cfg.max_steps
    ri, rv, cnt = F.march(o, d, cap)
    gi, gv, gc = (t.cpu().numpy() for t in V.vrnerf_debug_march(f, _cuda(o), _cuda(d), cap))
    assert (gc == cnt).all()
    assert (gi == ri).all() and (gv == rv).all()
    assert cnt.sum() > 50000
    f.close()


def test_contracted_history(V, unit):
    """Training history of a contracted scene (Sec. 4.3.2, Sec. 4): after
    backward passes of rays from inside the box and from 20 units outside,
    every voxel of the contracted grid holds the largest composited opacity
    the oracle records there (T_eps = 0, so both sides composite the same
    samples)."""
    cfg, occ, grid, mlp = unit
    cfg = replace(cfg, T_eps=0.0)
    bits = S.pack_bits(occ)
    f = V.Field(cfg, grid, mlp, bits)
    F = O.Field(cfg, grid, mlp, bits)
    V.vrnerf_history_reset(f)
    rng = np.random.default_rng(21)
    c2w, K, res = S.camera_unit_cube(occ, cfg, 4, 24, 24)
    o1, d1, r1 = O.camera_rays(cfg, c2w, K, res)
    o2 = (0.5 + 20.0 * rng.normal(size=(400, 3))).astype(np.float32)
    d2 = 0.5 + 0.3 * rng.normal(size=(400, 3)) - o2
    d2 = (d2 / np.linalg.norm(d2, axis=1, keepdims=True)).astype(np.float32)
    r2 = np.full(400, 1e-3, np.float32)
    want = np.zeros(occ.size, np.float32)
    for o, d, r in ((o1, d1, r1), (o2, d2, r2)):
        tgt = np.full((o.shape[0], 3), 0.5, np.float32)
        V.vrnerf_backward(f, _cuda(o), _cuda(d), _cuda(r), _cuda(tgt))
        want = O.history(F, o, d, r, want)
    got = V.vrnerf_field_get_history(f)
    assert (want > 0).sum() > 200
    # voxels beyond the box's image in the contracted grid are recorded too
    outer = np.ones(occ.shape, bool)
    outer[8:24, 8:24, 8:24] = False
    assert (want.reshape(occ.shape)[outer] > 0).sum() > 50
    err = np.abs(got.astype(np.float64) - want)
    assert (err <= 1e-4 * want + 1e-6).all(), err.max()
    f.close()
