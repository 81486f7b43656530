"""GPU parity of occupancy-grid pruning (Sec. 4.3.2) against the oracle.

Grid opacities: |gpu - oracle| <= 1e-4 |oracle| + 1e-6 (fp32 features and
MLP against fp64). Keep decisions: identical for every voxel whose oracle
opacity is farther than that tolerance from the threshold. Training history:
the same bound per voxel, on rays whose sample sets match exactly (T_eps = 0,
march visits are bit-exact). After an applied prune, renders match the
oracle's on the pruned occupancy, which checks the rebuilt distance field.
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _small(seed=3, **kw):
    cfg = replace(S.cfg_unit_cube(), occ_res=(16, 16, 16), levels=8, **kw)
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=(16, 16, 16)) < 0.3
    grid = rng.uniform(-1, 1, (cfg.levels, cfg.T, cfg.feats)).astype(np.float32)
    mlp = (rng.normal(size=O.mlp_count(cfg)) * 0.5).astype(np.float32)
    return cfg, occ, grid, mlp


def _keep_matches(keep_gpu, keep_ref, alpha_ref, thr, hist=None):
    near = np.abs(alpha_ref - thr) <= RTOL * thr + ATOL
    if hist is not None:
        near |= np.abs(hist - thr) <= RTOL * thr + ATOL
    diff = (keep_gpu != keep_ref) & ~near
    assert not diff.any(), np.argwhere(diff)[:5]


@pytest.mark.parametrize("k", [2, 5])
def test_grid_opacity_and_keep_match_oracle(V, k):
    cfg, occ, grid, mlp = _small()
    bits = S.pack_bits(occ)
    f = V.Field(cfg, grid, mlp, bits)
    F = O.Field(cfg, grid, mlp, bits)
    cams = np.array([[0.5, 0.5, 0.5], [0.1, 0.9, 0.2], [0.95, 0.05, 0.6]], np.float32)
    _, alpha_ref = O.prune(F, cams, k, 0.0)
    thr = float(np.quantile(alpha_ref[occ], 0.5))
    hist = np.zeros(occ.shape, np.float32)
    rng = np.random.default_rng(6)
    hist[occ & (rng.uniform(size=occ.shape) < 0.2)] = 1.0
    keep_ref, alpha_ref = O.prune(F, cams, k, thr)
    kept, alpha, new_bits = V.vrnerf_prune(f, cams, k, thr, apply=False, want_alpha=True)
    alpha = alpha.reshape(occ.shape)
    assert (alpha[~occ] == 0).all()
    err = np.abs(alpha - alpha_ref)
    assert (err <= RTOL * alpha_ref + ATOL).all(), err.max()
    keep = S.unpack_bits(new_bits, cfg.occ_res)
    _keep_matches(keep, keep_ref, alpha_ref, thr)
    assert kept == keep.sum()
    # apply=False left the field's occupancy alone
    _, _, again = V.vrnerf_prune(f, cams, k, 0.0, apply=False)
    assert (again == bits).all()
    f.close()


def test_history_matches_oracle_and_joins_the_decision(V):
    cfg, occ, grid, mlp = _small(seed=4, T_eps=0.0)
    bits = S.pack_bits(occ)
    f = V.Field(cfg, grid, mlp, bits)
    F = O.Field(cfg, grid, mlp, bits)
    with pytest.raises(V.VrnerfError):
        V.vrnerf_field_get_history(f)
    V.vrnerf_history_reset(f)
    assert not V.vrnerf_field_get_history(f).any()
    want = np.zeros(occ.size, np.float32)
    for seed in (1, 2):
        c2w, K, res = S.camera_unit_cube(occ, cfg, seed, 24, 24)
        o, d, r = O.camera_rays(cfg, c2w, K, res)
        tgt = np.full((o.shape[0], 3), 0.5, np.float32)
        V.vrnerf_backward(f, _cuda(o), _cuda(d), _cuda(r), _cuda(tgt))
        want = O.history(F, o, d, r, want)
    got = V.vrnerf_field_get_history(f)
    assert (want > 0).sum() > 50
    assert (np.abs(got - want) <= RTOL * want + ATOL).all(), np.abs(got - want).max()
    # the history rescues voxels whose grid opacity is below the threshold
    cams = np.array([[0.5, 0.5, 0.5]], np.float32)
    _, alpha_ref = O.prune(F, cams, 2, 0.0)
    thr = float(np.quantile(alpha_ref[occ], 0.7))
    keep_ref, _ = O.prune(F, cams, 2, thr, want.reshape(occ.shape))
    keep_grid, _ = O.prune(F, cams, 2, thr)
    assert (keep_ref & ~keep_grid).any()
    kept, _, new_bits = V.vrnerf_prune(f, cams, 2, thr, apply=False)
    _keep_matches(S.unpack_bits(new_bits, cfg.occ_res), keep_ref, alpha_ref, thr, want.reshape(occ.shape))
    V.vrnerf_history_reset(f)
    assert not V.vrnerf_field_get_history(f).any()
    f.close()


def test_applied_prune_renders_like_oracle_on_pruned_occupancy(V):
    cfg, occ, grid, mlp = _small(seed=5, T_eps=0.0)
    bits = S.pack_bits(occ)
    f = V.Field(cfg, grid, mlp, bits)
    F = O.Field(cfg, grid, mlp, bits)
    cams = np.array([[0.3, 0.4, 0.5]], np.float32)
    _, alpha_ref = O.prune(F, cams, 3, 0.0)
    a = np.sort(alpha_ref[occ])
    i = int(np.argmax(np.diff(a[len(a) // 4: 3 * len(a) // 4]))) + len(a) // 4
    thr = float((a[i] + a[i + 1]) / 2)  # inside the widest gap: no voxel near it
    keep_ref, _ = O.prune(F, cams, 3, thr)
    assert 0 < keep_ref.sum() < occ.sum()
    kept, _, new_bits = V.vrnerf_prune(f, cams, 3, thr, apply=True)
    assert kept == keep_ref.sum() and (new_bits == S.pack_bits(keep_ref)).all()
    Fp = O.Field(cfg, grid, mlp, S.pack_bits(keep_ref))
    c2w, K, res = S.camera_unit_cube(occ, cfg, 3, 48, 48)
    ref = Fp.render(c2w, K, res)
    out = torch.empty((48 * 48, 3), device="cuda")
    n = torch.empty(48 * 48, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, out_pq=out, out_n=n)
    torch.cuda.synchronize()
    assert (n.cpu().numpy() == ref["n"]).all()
    lin = lin.cpu().numpy()
    assert (np.abs(lin - ref["linear"]) <= RTOL * np.abs(ref["linear"]) + ATOL).all()
    f.close()


def test_room_full_size_sampled_voxels(V):
    """Room field (L=16, T=2^21, fp16 features, 256^3 occupancy, the
    benchmark's scene) pruned with 4^3 points per voxel on the GPU; the oracle
    evaluates 300 sampled occupied voxels (an occupancy holding only those)."""
    sc = S.make_scene("room")
    cfg = sc.cfg
    f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    poses, _ = S.training_views(sc.occ, cfg, n_views=16)
    cams = poses[:, :3, 3].astype(np.float32)
    _, alpha, _ = V.vrnerf_prune(f, cams, 4, 0.0, apply=False, want_alpha=True)
    rng = np.random.default_rng(7)
    occ_idx = np.flatnonzero(sc.occ.reshape(-1))
    pick = rng.choice(occ_idx, 300, replace=False)
    sub = np.zeros(sc.occ.size, bool)
    sub[pick] = True
    F = O.Field(cfg, sc.grid, sc.mlp, S.pack_bits(sub.reshape(sc.occ.shape)))
    _, alpha_ref = O.prune(F, cams, 4, 0.0)
    ref = alpha_ref.reshape(-1)[pick]
    got = alpha[pick]
    assert (np.abs(got - ref) <= RTOL * ref + ATOL).all(), np.abs(got - ref).max()
    assert (alpha.reshape(-1)[~sc.occ.reshape(-1)] == 0).all()
    f.close()


def test_upsample_matches_oracle_and_renders(V):
    cfg, occ, grid, mlp = _small(seed=7, T_eps=0.0)
    f = V.Field(cfg, grid, mlp, S.pack_bits(occ))
    V.vrnerf_history_reset(f)
    c2w, K, res = S.camera_unit_cube(occ, cfg, 1, 16, 16)
    o, d, r = O.camera_rays(cfg, c2w, K, res)
    V.vrnerf_backward(f, _cuda(o), _cuda(d), _cuda(r), _cuda(np.full((o.shape[0], 3), 0.5)))
    h0 = V.vrnerf_field_get_history(f).reshape(occ.shape)
    assert (h0 > 0).any()
    with pytest.raises(V.VrnerfError):
        V.vrnerf_occupancy_upsample(f, 1)
    V.vrnerf_occupancy_upsample(f, 2)
    cfg2 = f.cfg
    assert cfg2.occ_res == (32, 32, 32)
    up = O.upsample_occupancy(occ, 2)
    assert (V.vrnerf_field_get_occupancy(f) == S.pack_bits(up)).all()
    assert (V.vrnerf_field_get_history(f) == O.upsample_occupancy(h0, 2).reshape(-1)).all()
    F2 = O.Field(cfg2, grid, mlp, S.pack_bits(up))
    c2w, K, res = S.camera_unit_cube(occ, cfg, 4, 40, 40)
    o, d, r = O.camera_rays(cfg2, c2w, K, res)
    ri, rv, cnt = F2.march(o, d, cfg2.max_steps)
    gi, gv, gc = (t.cpu().numpy() for t in V.vrnerf_debug_march(f, _cuda(o), _cuda(d), cfg2.max_steps))
    assert (gc == cnt).all() and (gi == ri).all() and (gv == rv).all()
    ref = F2.render(c2w, K, res)
    lin = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res).cpu().numpy()
    assert (np.abs(lin - ref["linear"]) <= RTOL * np.abs(ref["linear"]) + ATOL).all()
    f.close()


def test_pruning_schedule_during_training(V):
    """The loop of Sec. 4.3.2 at small scale on the opaque room: history on,
    train, prune every few steps with the threshold annealed towards 0.2,
    upsample the grid once at a milestone, keep training."""
    sc = S.make_scene("room_surface")
    cfg = sc.cfg
    f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    poses, intr = S.training_views(sc.occ, cfg, n_views=16)
    cams = poses[:, :3, 3].astype(np.float32)
    V.vrnerf_history_reset(f)
    count = int(sc.occ.sum())
    losses = []
    for it in range(12):
        batch = [_cuda(a) for a in S.training_batch(poses, intr, 1 << 13, seed=5, step=it)]
        losses.append(V.vrnerf_train_step(f, *batch))
        if it % 3 == 2:
            thr = 0.2 * (it + 1) / 12
            kept, _, _ = V.vrnerf_prune(f, cams, 4, thr, apply=True)
            assert 0 < kept <= count
            count = kept
            V.vrnerf_history_reset(f)
        if it == 5:
            V.vrnerf_occupancy_upsample(f, 2)
            count *= 8
            assert f.cfg.occ_res == (512, 512, 512)
            occ = S.unpack_bits(V.vrnerf_field_get_occupancy(f), f.cfg.occ_res)
            assert occ.sum() == count
    assert np.isfinite(losses).all()
    V.vrnerf_field_status(f)
    f.close()
