"""GPU parity of the auxiliary render outputs against the oracle: composited
normals (the fp32 path), display pixels (PQ to sRGB at an exposure, fused in
every render kernel and as a standalone kernel).

Normals: |gpu - oracle| <= 2e-3 per component (fp32 sums against fp64; a
normal is a unit vector, so the bound is absolute), rays whose sample count
differs (early termination at T_eps) excluded and counted; the axis field's
closed form (-(1 - T), 0, 0) within 1e-5. Display bytes: equal wherever the
oracle's unrounded 255 s is more than 0.02 from a rounding boundary, within
one step elsewhere.
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


def _bytes(words):
    w = np.asarray(words).astype(np.int64) & 0xFFFFFFFF
    return np.stack([(w >> (8 * c)) & 255 for c in range(4)], axis=1)


def _check_bytes(got_words, ref_words, pre, min_exact=0.99):
    got, ref = _bytes(got_words), _bytes(ref_words)
    near = np.abs(pre - np.floor(pre) - 0.5) < 0.02
    assert (got[~near] == ref[~near]).all(), np.argwhere((got != ref) & ~near)[:5]
    assert (np.abs(got - ref) <= 1).all()
    assert (got == ref).mean() >= min_exact


def _render_aux(V, f, c2w, K, res, precision=0, ev=0.0, normals=True):
    res = np.asarray(res, np.int32).reshape(-1, 2)
    rays = int((res[:, 0] * res[:, 1]).sum())
    pq = torch.empty((rays, 3), device="cuda")
    T = torch.empty(rays, device="cuda")
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    nrm = torch.empty((rays, 3), device="cuda") if normals else None
    rgba = torch.empty(rays, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=precision, out_pq=pq, out_T=T,
                          out_n=n, out_normal=nrm, out_rgba8=rgba, exposure_ev=ev)
    torch.cuda.synchronize()
    return dict(linear=lin.cpu().numpy(), pq=pq.cpu().numpy(), T=T.cpu().numpy(),
                n=n.cpu().numpy(), normal=None if nrm is None else nrm.cpu().numpy(),
                rgba=rgba.cpu().numpy())


def _random_cube(seed=3):
    sc = S.make_scene("unit_cube")
    cfg = replace(sc.cfg, density_bias=3.0)
    rng = np.random.default_rng(seed)
    grid = rng.uniform(-1, 1, sc.grid.shape).astype(np.float32)
    mlp = (rng.normal(size=O.mlp_count(cfg)) * 0.5).astype(np.float32)
    return sc, cfg, grid, mlp


def test_normals_match_oracle_unit_cube(V):
    sc, cfg, grid, mlp = _random_cube()
    f = V.Field(cfg, grid, mlp, sc.occ_bits)
    F = O.Field(cfg, grid, mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, 48, 48)
    got = _render_aux(V, f, c2w, K, res)
    ref = F.render(c2w, K, res, normals=True)
    same = got["n"] == ref["n"]
    assert same.mean() > 0.99
    assert np.abs(ref["normal"]).max() > 0.1
    err = np.abs(got["normal"] - ref["normal"])[same]
    assert (err <= 2e-3).all(), (err.max(), np.count_nonzero(err > 2e-3))
    # normals leave the colour untouched: same image as without them
    plain = _render_aux(V, f, c2w, K, res, normals=False)
    assert (plain["linear"] == got["linear"]).all() and (plain["n"] == got["n"]).all()
    with pytest.raises(V.VrnerfError):
        _render_aux(V, f, c2w, K, res, precision=1)
    f.close()


def test_normals_match_oracle_room_crop(V):
    sc = S.make_scene("room_surface")
    cfg = sc.cfg
    f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, _ = S.camera_room(sc.occ, cfg, 2, 2048, 2048)
    K = S.crop_camera(K, 1000, 1000)
    res = np.array([[40, 40]], np.int32)
    got = _render_aux(V, f, c2w, K, res)
    ref = F.render(c2w, K, res, normals=True)
    same = got["n"] == ref["n"]
    assert same.mean() > 0.98
    err = np.abs(got["normal"] - ref["normal"])[same]
    assert (err <= 2e-3).all(), (err.max(), np.count_nonzero(err > 2e-3))
    f.close()


def test_normals_axis_field_closed_form(V):
    """Level 0 holds the vertex's x coordinate / N_0 in feature 0, the density
    MLP passes it through one ReLU: every normal is -x, so the composited
    normal is (-(1 - T), 0, 0)."""
    sc = S.make_scene("unit_cube")
    cfg = replace(sc.cfg, density_bias=2.0)
    N0 = O.geometry(cfg)[0][0]
    grid = np.zeros(sc.grid.shape, np.float32)
    n1 = N0 + 1
    a = np.arange(n1 ** 3)
    grid[0, a, 0] = (a % n1) / N0
    mlp = np.zeros(O.mlp_count(cfg), np.float32)
    mlp[0] = 1.0                   # W1[0][0]
    mlp[64 * 2 * cfg.levels] = 1.0  # W2[0][0]
    f = V.Field(cfg, grid, mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 2, 32, 32)
    got = _render_aux(V, f, c2w, K, res)
    assert (got["n"] > 0).mean() > 0.5
    np.testing.assert_allclose(got["normal"][:, 0], -(1.0 - got["T"]), atol=1e-5)
    assert np.abs(got["normal"][:, 1:]).max() <= 1e-5  # fp32 cancellation of equal corners
    f.close()


@pytest.mark.parametrize("ev", [-1.0, 0.0, 2.5])
def test_rgba8_matches_oracle_tonemap(V, ev):
    sc, cfg, grid, mlp = _random_cube(seed=4)
    f = V.Field(cfg, grid, mlp, sc.occ_bits)
    F = O.Field(cfg, grid, mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 3, 48, 48)
    got = _render_aux(V, f, c2w, K, res, ev=ev, normals=False)
    ref = F.render(c2w, K, res)
    same = got["n"] == ref["n"]
    words, pre = O.tonemap(ref["pq"], ref["T"], ev)
    _check_bytes(got["rgba"][same], words[same], pre[same])
    f.close()


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_rgba8_tensor_core_epilogue_equals_standalone_tonemap(V, precision):
    sc = S.make_scene("room")
    f = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, _ = S.camera_room(sc.occ, sc.cfg, 2, 2048, 2048)
    K = S.crop_camera(K, 896, 896)
    res = np.array([[256, 256]], np.int32)
    got = _render_aux(V, f, c2w, K, res, precision=precision, ev=1.5, normals=False)
    again = V.vrnerf_tonemap(_cuda(got["pq"]), _cuda(got["T"]), 1.5).cpu().numpy()
    assert (again == got["rgba"]).all()
    f.close()


def test_standalone_tonemap_matches_oracle(V):
    rng = np.random.default_rng(9)
    n = 200_000
    pq = rng.uniform(0, 1, (n, 3))
    pq[:1000] = rng.uniform(0, 0.2, (1000, 3))  # the linear sRGB segment
    T = rng.uniform(0, 1, n)
    for ev in (-2.0, 0.0, 3.0):
        got = V.vrnerf_tonemap(_cuda(pq), _cuda(T), ev).cpu().numpy()
        words, pre = O.tonemap(pq.astype(np.float32), T.astype(np.float32), ev)
        _check_bytes(got, words, pre)
    got = V.vrnerf_tonemap(_cuda(pq[:10]), None, 0.0).cpu().numpy()
    assert ((got.astype(np.int64) & 0xFFFFFFFF) >> 24 == 255).all()
    V.vrnerf_tonemap(_cuda(np.zeros((0, 3))), None, 0.0)
    with pytest.raises(V.VrnerfError):
        V.vrnerf_tonemap(_cuda(pq[:10]), None, float("nan"))
