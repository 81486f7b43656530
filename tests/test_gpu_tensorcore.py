"""GPU parity of the tensor-core (tcgen05) MLP path against the CPU oracle.

fp16 operands with fp32 accumulation must agree with the fp64 oracle within
2e-3 relative (+1e-5 absolute) on sigma, PQ colour and linear colour; rays
whose early-termination decision flips at T_eps may differ by T_eps in PQ
space. bf16 and fp8 (e4m3 hidden layers) are held to a PQ-space PSNR of at
least 50 dB (peak 1.0) against the oracle, the fixed-quality bar of the
precision sweep.
"""
from dataclasses import replace

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
def cube():
    return S.make_scene("unit_cube")


@pytest.fixture(scope="module")
def room():
    return S.make_scene("room")


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _close(a, b, rtol=TC_RTOL, atol=TC_ATOL):
    return np.abs(np.asarray(a, np.float64) - b) <= rtol * np.abs(b) + atol


def psnr_pq(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - b) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def render(V, field, c2w, K, res, precision):
    res = np.asarray(res, np.int32).reshape(-1, 2)
    rays = int((res[:, 0] * res[:, 1]).sum())
    pq = torch.empty((rays, 3), device="cuda")
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    lin = V.vrnerf_render(field, _cuda(c2w), _cuda(K), res, precision=precision, out_pq=pq, out_n=n)
    V.vrnerf_field_status(field)
    return lin.cpu().numpy(), pq.cpu().numpy(), n.cpu().numpy()


def check_tc(lin, pq, n, ref, T_eps):
    flip = n != ref["n"]
    good = _close(pq, ref["pq"]).all(1) & _close(lin, ref["linear"]).all(1)
    bad = ~good & ~flip
    assert not bad.any(), (bad.sum(), np.abs(pq - ref["pq"])[bad].max())
    if flip.any():
        assert np.abs(pq[flip] - ref["pq"][flip]).max() <= T_eps + 1e-4
        assert flip.mean() <= 0.01


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
def test_query_tensorcore(V, cube, room, prec):
    rng = np.random.default_rng(31)
    for sc in (cube, room):
        cfg = sc.cfg
        f = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        n = 1000  # several 128-row tiles and a ragged last tile
        lo, hi = np.array(cfg.aabb_min), np.array(cfg.aabb_max)
        pos = (lo + (hi - lo) * rng.uniform(0, 1, (n, 3))).astype(np.float32)
        d = rng.normal(size=(n, 3))
        d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
        rad = (10 ** rng.uniform(-6, -1, n)).astype(np.float32)
        sig, rgb, ofeat = F.query(pos, d, rad)
        gs, gr, _ = V.vrnerf_query(f, _cuda(pos), _cuda(d), _cuda(rad), precision=prec)
        V.vrnerf_field_status(f)
        gs, gr = gs.cpu().numpy(), gr.cpu().numpy()
        if prec == "fp16":
            assert _close(gs, sig).all() and _close(gr, rgb).all()
        elif prec == "bf16":
            # sigma = exp(o_0), so its relative error is o_0's absolute error. With
            # unit roundoff u = 2^-9 for every bf16 rounding (feature, W1, hidden
            # h, W2) and the features' fp16 interpolation (8 HFMA2, 2^-11 each):
            #   |dh_k|  <= ((u + 8 2^-11) + u) sum_j |W1_kj f_j| + u |h_k|   (h_k > 0)
            #   |do_0|  <= sum_k |W2_0k| |dh_k| + u sum_k |W2_0k h_k|
            # per point, from the oracle's features; held at twice that bound
            D = cfg.d_in
            m = np.asarray(sc.mlp, np.float64)
            W1, W2 = m[:64 * D].reshape(64, D), m[64 * D:64 * D + 16 * 64].reshape(16, 64)
            fe = np.asarray(ofeat, np.float64).reshape(n, D)
            pre = fe @ W1.T
            hh = np.maximum(pre, 0.0)
            u = 2.0 ** -9
            dh = ((2 * u + 8 * 2.0 ** -11) * (np.abs(fe) @ np.abs(W1).T) + u * hh) * (pre > 0)
            bound = dh @ np.abs(W2[0]) + u * (np.abs(W2[0]) * hh).sum(1)
            rel = np.abs(gs - sig) / sig
            pos_b = bound > 0  # a point whose hidden units are all zero has o_0 = bias exactly
            ratio = float(np.max(rel[pos_b] / bound[pos_b])) if pos_b.any() else 0.0
            print(f"bf16 sigma: max rel err {rel.max():.3e}, max bound {bound.max():.3e}, "
                  f"worst err / bound {ratio:.3f}")
            assert np.all(rel <= 2 * bound + 1e-6), ratio
            assert np.max(np.abs(gr - rgb)) < 1e-2
        else:  # e4m3 hidden layers with per-row and per-matrix scales
            assert np.max(np.abs(gs - sig) / sig) < 5e-2
            assert np.max(np.abs(gr - rgb)) < 3e-2
        f.close()


def test_render_tensorcore_unit_cube(V, cube):
    for cfg in (cube.cfg, replace(cube.cfg, density_bias=4.0)):
        f = V.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
        F = O.Field(cfg, cube.grid, cube.mlp, cube.occ_bits)
        c2w, K, res = S.camera_unit_cube(cube.occ, cfg, 1, 64, 64)
        ref = F.render(c2w, K, res)
        check_tc(*render(V, f, c2w, K, res, "fp16"), ref, cfg.T_eps)
        f.close()


@pytest.mark.parametrize("variant", ["room", "room_surface"])
def test_render_tensorcore_room_crops(V, room, variant):
    cfg = S.cfg_room(surface=(variant == "room_surface"))
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, _ = S.camera_room(room.occ, cfg, 2, 2048, 2048)
    rng = np.random.default_rng(32)
    for _ in range(2):
        x0, y0 = rng.integers(0, 2048 - 100, 2)
        Kc = S.crop_camera(K, int(x0), int(y0))
        res = np.array([[100, 61]], np.int32)
        check_tc(*render(V, f, c2w, Kc, res, "fp16"), F.render(c2w, Kc, res), cfg.T_eps)
    f.close()


@pytest.mark.parametrize("variant", ["room", "room_surface"])
def test_precision_sweep_psnr(V, room, variant):
    """256x256 crops of the room frame: fp32, fp16 and bf16 MLPs against the
    fp64 oracle, PSNR in PQ space (peak 1)."""
    cfg = S.cfg_room(surface=(variant == "room_surface"))
    f = V.Field(cfg, room.grid, room.mlp, room.occ_bits)
    F = O.Field(cfg, room.grid, room.mlp, room.occ_bits)
    c2w, K, _ = S.camera_room(room.occ, cfg, 2, 2048, 2048)
    rng = np.random.default_rng(33)
    res = np.array([[256, 256]], np.int32)
    for _ in range(2):
        x0, y0 = rng.integers(0, 2048 - 256, 2)
        Kc = S.crop_camera(K, int(x0), int(y0))
        ref = F.render(c2w, Kc, res)
        for prec in ("fp32", "fp16", "bf16", "fp8"):
            _, pq, _ = render(V, f, c2w, Kc, res, prec)
            p = psnr_pq(pq, ref["pq"])
            err = np.abs(pq - ref["pq"])
            print(f"precision-sweep {variant} crop=({x0},{y0}) {prec}: PQ-PSNR {p:.2f} dB, "
                  f"max |err| {err.max():.3e}, mean |err| {err.mean():.3e}")
            assert p >= 50.0, prec
    f.close()
