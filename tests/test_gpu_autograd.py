"""The hand-written backward behind torch.autograd: FieldModule /
RenderRaysFunction against the oracle's gradient of an arbitrary linear
functional of the PQ colours, against the fused L1 backward, and driven by a
torch optimiser.

Gradients: |gpu - oracle| <= 1e-4 |oracle| + 1e-5 max|oracle| element-wise
(fp32 accumulation in any order against fp64), as for vrnerf_backward.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    from paper_2311_02542_gb300 import vrnerf
    vrnerf.load()
    return vrnerf


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _scene():
    sc = S.make_scene("unit_cube")
    cfg = replace(sc.cfg, density_bias=3.0, T_eps=0.0)
    grid = (sc.grid * 50).astype(np.float32)
    return sc, cfg, grid


def _check_grads(got_g, got_m, ref_g, ref_m):
    for got, ref in ((got_m, ref_m), (got_g.reshape(-1), ref_g.reshape(-1))):
        scale = np.abs(ref).max()
        assert scale > 0
        ok = np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * scale
        assert ok.all(), (np.count_nonzero(~ok), np.abs(got - ref)[~ok].max(), scale)


def test_autograd_matches_oracle_for_any_upstream_gradient(V):
    sc, cfg, grid = _scene()
    f = V.Field(cfg, grid, sc.mlp, sc.occ_bits)
    F = O.Field(cfg, grid, sc.mlp, sc.occ_bits)
    module = V.FieldModule(f)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, 24, 24)
    o, d, r = O.camera_rays(cfg, c2w, K, res)
    G = np.random.default_rng(3).normal(size=(o.shape[0], 3))
    pq = module(_cuda(o), _cuda(d), _cuda(r))
    ref = F.render_rays(o, d, r)
    assert np.abs(pq.detach().cpu().numpy() - ref["pq"]).max() < 1e-4
    (pq * _cuda(G)).sum().backward()
    rg, rm = F.backward_grad(o, d, r, G)
    _check_grads(module.grid.grad.cpu().numpy(), module.mlp.grad.cpu().numpy(), rg, rm)
    f.close()


def test_autograd_l1_equals_fused_backward(V):
    """The L1 loss in PQ space written with torch ops gives the fused
    vrnerf_backward's gradients (same kernels, same upstream gradient)."""
    sc, cfg, grid = _scene()
    f = V.Field(cfg, grid, sc.mlp, sc.occ_bits)
    module = V.FieldModule(f)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 2, 32, 32)
    o, d, r = (_cuda(a) for a in O.camera_rays(cfg, c2w, K, res))
    tgt_lin = np.exp(np.random.default_rng(4).uniform(-3, 3, (o.shape[0], 3))).astype(np.float32)
    tgt_pq = np.array([[O.linear_to_pq(float(x)) for x in row] for row in tgt_lin], np.float32)
    loss = (module(o, d, r) - _cuda(tgt_pq)).abs().mean()
    loss.backward()
    fused = V.vrnerf_backward(f, o, d, r, _cuda(tgt_lin))
    gg, gm = V.vrnerf_field_get_grads(f)
    assert float(loss.detach()) == pytest.approx(fused, rel=1e-5)
    np.testing.assert_allclose(module.mlp.grad.cpu().numpy(), gm, rtol=1e-5, atol=1e-7 * np.abs(gm).max())
    np.testing.assert_allclose(module.grid.grad.cpu().numpy(), gg, rtol=1e-5, atol=1e-7 * np.abs(gg).max())
    f.close()


def test_torch_optimiser_trains_the_field(V):
    sc = S.make_scene("room")
    cfg = replace(sc.cfg, feat_fp16=False)
    f = V.Field(cfg, sc.grid.astype(np.float32), sc.mlp, sc.occ_bits)
    module = V.FieldModule(f)
    opt = torch.optim.Adam(module.parameters(), lr=5e-3, betas=(0.9, 0.99), eps=1e-15)
    poses, intr = S.training_views(sc.occ, cfg, n_views=16)
    o, d, r, tgt = S.training_batch(poses, intr, 1 << 13, seed=5, step=0)
    tgt_pq = _cuda(np.array([[O.linear_to_pq(float(x)) for x in row] for row in tgt], np.float32))
    o, d, r = _cuda(o), _cuda(d), _cuda(r)
    losses = []
    for _ in range(25):
        opt.zero_grad()
        loss = (module(o, d, r) - tgt_pq).abs().mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.9 * losses[0], losses[::6]
    # the tensor-core path sees the new weights once told
    module.params_changed()
    c2w, K, _ = S.camera_room(sc.occ, cfg, 2, 2048, 2048)
    K = S.crop_camera(K, 960, 960)
    res = np.array([[128, 128]], np.int32)
    a = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision="fp32").cpu().numpy()
    b = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision="fp16").cpu().numpy()
    assert np.all(np.abs(a - b) <= 2e-3 * np.abs(a) + 1e-4)
    V.vrnerf_field_status(f)
    f.close()


def test_forward_rays_equals_render_rays(V):
    """The sample-parallel forward gives the fp32 renderer's PQ colours and
    sample counts on the same rays (same arithmetic, another schedule)."""
    sc = S.make_scene("room")
    f = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    poses, intr = S.training_views(sc.occ, sc.cfg, n_views=16)
    o, d, r, _ = (_cuda(a) for a in S.training_batch(poses, intr, 12800, seed=5, step=1))
    pq_a, n_a = V.vrnerf_forward_rays(f, o, d, r)
    pq_b = torch.empty_like(pq_a)
    n_b = torch.empty_like(n_a)
    V.vrnerf_render_rays(f, o, d, r, precision="fp32", out_pq=pq_b, out_n=n_b)
    same = n_a == n_b
    assert same.float().mean() > 0.999  # a flip at T_eps only if fp32 rounding differs
    assert torch.allclose(pq_a[same], pq_b[same], rtol=1e-5, atol=1e-7)
    f.close()
