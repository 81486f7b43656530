"""GPU parity on the hash grid of the paper's experiments (Sec. 6): L = 16
levels of F = 2 features, base resolution 128, growth 1.4, T = 2^19 slots
per level, so every level is hashed (129^3 > 2^19), in the room.

- hash corner indices: bit-exact against the oracle;
- fp32 radiance of 100 x 61 windows: |gpu - oracle| <= 1e-4 |oracle| + 1e-6
  (rays whose early termination flips at T_eps within T_eps in PQ);
- fp16 tensor cores: <= 2e-3 |oracle| + 1e-5;
- the paper's training batch, 12 800 rays (256 rays from each of 50 views):
  fp32 gradients of the L1 loss in PQ space within 1e-4 |ref| + 1e-5 max|ref|
  of the oracle's, element-wise, and the loss within 1e-5 relative.
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
def scene():
    return S.make_scene("room_paper_grid")


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _close(gpu, ref, rtol, atol):
    return np.abs(np.asarray(gpu, np.float64) - ref) <= rtol * np.abs(ref) + atol


def _check(lin, pq, n, ref, T_eps, rtol, atol):
    flip = n != ref["n"]
    good = _close(pq, ref["pq"], rtol, atol).all(1) & _close(lin, ref["linear"], rtol, atol).all(1)
    bad = ~good & ~flip
    assert not bad.any(), (bad.sum(), np.abs(pq - ref["pq"])[bad].max())
    if flip.any():
        assert np.abs(pq[flip] - ref["pq"][flip]).max() <= T_eps + 1e-4
        assert flip.mean() <= 0.01


def test_paper_grid_is_all_hashed(scene):
    _, dense, _, _ = O.geometry(scene.cfg)
    assert not dense.any()


def test_paper_grid_corners_bit_exact(V, scene):
    cfg = scene.cfg
    f = V.Field(cfg, scene.grid, scene.mlp, scene.occ_bits)
    rng = np.random.default_rng(51)
    lo, hi = np.array(cfg.aabb_min), np.array(cfg.aabb_max)
    pos = (lo + (hi - lo) * rng.uniform(0, 1, (20000, 3))).astype(np.float32)
    pos[:8] = np.array([lo, hi, [lo[0], hi[1], lo[2]], hi - 1e-6, lo + 1e-7, (lo + hi) / 2,
                        [hi[0], lo[1], hi[2]], [lo[0], lo[1], hi[2]]], np.float32)
    ref, _ = O.corners(cfg, pos)
    got = V.vrnerf_debug_corners(f, _cuda(pos)).cpu().numpy().view(np.uint32)
    assert (got == ref).all()
    assert (ref < cfg.T).all()
    f.close()


@pytest.mark.parametrize("surface", [False, True])
def test_paper_grid_render_windows(V, scene, surface):
    cfg = replace(scene.cfg, density_bias=float(np.log(100.0)) if surface else 0.0)
    f = V.Field(cfg, scene.grid, scene.mlp, scene.occ_bits)
    F = O.Field(cfg, scene.grid, scene.mlp, scene.occ_bits)
    c2w, K, _ = S.camera_room(scene.occ, cfg, 2, 2048, 2048)
    rng = np.random.default_rng(52)
    res = np.array([[100, 61]], np.int32)  # ragged against the 8 x 4 ray tiles
    for _ in range(2):
        x0, y0 = rng.integers(0, 2048 - 100, 2)
        Kc = S.crop_camera(K, int(x0), int(y0))
        ref = F.render(c2w, Kc, res)
        for prec, rtol, atol in (("fp32", RTOL, ATOL), ("fp16", TC_RTOL, TC_ATOL)):
            pq = torch.empty((100 * 61, 3), device="cuda")
            n = torch.empty(100 * 61, device="cuda", dtype=torch.int32)
            lin = V.vrnerf_render(f, _cuda(c2w), _cuda(Kc), res, precision=prec, out_pq=pq, out_n=n)
            V.vrnerf_field_status(f)
            _check(lin.cpu().numpy(), pq.cpu().numpy(), n.cpu().numpy(), ref, cfg.T_eps, rtol, atol)
    f.close()


@pytest.mark.parametrize("surface", [False, True])
def test_paper_batch_gradients_against_oracle(V, scene, surface):
    """The paper's 12 800-ray batch (256 rays x 50 views, Sec. 6)."""
    cfg = replace(scene.cfg, density_bias=float(np.log(100.0)) if surface else 0.0)
    f = V.Field(cfg, scene.grid, scene.mlp, scene.occ_bits)
    F = O.Field(cfg, scene.grid, scene.mlp, scene.occ_bits)
    poses, intr = S.training_views(scene.occ, cfg, n_views=50, seed=5)
    o, d, r, tgt = S.training_batch(poses, intr, 12800, seed=5)
    loss_ref, rg, rm = F.backward(o, d, r, tgt)
    loss = V.vrnerf_backward(f, _cuda(o), _cuda(d), _cuda(r), _cuda(tgt))
    gg, gm = V.vrnerf_field_get_grads(f)
    V.vrnerf_field_status(f)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    for got, ref in ((gm, rm), (gg.reshape(-1), rg.reshape(-1))):
        scale = np.abs(ref).max()
        assert scale > 0
        ok = np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * scale
        assert ok.all(), (np.count_nonzero(~ok), np.abs(got - ref)[~ok].max(), scale)
    f.close()
