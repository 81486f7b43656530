"""Full-frame parity of the tensor-core render against the CPU oracle.

The persistent tensor-core kernel launches at most SMs x (CTAs per SM) x 128
ray slots; a 2048 x 2048 frame (4.19 M rays) is ~36 times that, so every
slot finishes rays and takes new ones from the global counter in the middle
of other slots' tiles. These tests render whole 2048^2 frames in that launch
configuration (the one the benchmark times) and compare 4 000 sampled rays
with the fp64 oracle (Sec. 5: a full eye buffer):

- fp16: |gpu - oracle| <= 2e-3 |oracle| + 1e-5 on PQ and linear colour;
  rays whose early-termination decision flips at T_eps (<= 1 %) agree
  within T_eps + 1e-4 in PQ;
- bf16 and fp8 (e4m3 hidden layers): PQ-PSNR >= 50 dB over the sampled
  rays, and every sampled ray within a per-ray bound in PQ (bf16 5e-3,
  fp8 3e-2: ten and four times the largest error measured on these frames,
  5.2e-4 and 7.1e-3; a ray's colour is a convex combination of sigmoid
  outputs, so its error is bounded by the colour and opacity errors of its
  samples).

Scenes: the literal room (transparent: rays cross many occupied voxels),
the opaque room (rays stop at the first surface), and the opaque room
inside the unbounded outdoor scene (L-infinity contraction, adjacent-ray
footprints).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu

TC_RTOL, TC_ATOL = 2e-3, 1e-5
PER_RAY = {"bf16": 5e-3, "fp8": 3e-2}
N_SAMPLE = 4000
SIDE = 2048


@pytest.fixture(scope="module")
def V():
    from paper_2311_02542_gb300 import vrnerf
    vrnerf.load()
    return vrnerf


_REF = {}


def _scene_and_ref(name):
    """The scene, its benchmark camera, the sampled ray indices and the
    oracle's render of those rays (computed once per scene)."""
    if name not in _REF:
        sc = S.make_scene(name)
        c2w, K, res = S.camera_room(sc.occ, sc.cfg, 2, SIDE, SIDE)
        o, d, r = O.camera_rays(sc.cfg, c2w, K, res)
        pick = np.sort(np.random.default_rng(41).choice(o.shape[0], N_SAMPLE, replace=False))
        F = O.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
        adj = None
        if sc.cfg.contract:
            du, dv = O.camera_adjacent(c2w, K, res)
            adj = (du[pick], dv[pick])
        ref = F.render_rays(o[pick], d[pick], r[pick], adjacent=adj)
        _REF[name] = (sc, c2w, K, res, pick, ref)
    return _REF[name]


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _render_full(V, sc, c2w, K, res, prec):
    f = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    rays = int(res[0, 0]) * int(res[0, 1])
    pq = torch.empty((rays, 3), device="cuda")
    n = torch.empty(rays, device="cuda", dtype=torch.int32)
    stats = torch.zeros(4, device="cuda", dtype=torch.int64)
    lin = V.vrnerf_render(f, _cuda(c2w), _cuda(K), res, precision=prec, out_pq=pq, out_n=n, stats=stats)
    V.vrnerf_field_status(f)
    out = lin.cpu().numpy(), pq.cpu().numpy(), n.cpu().numpy(), stats.cpu().numpy()
    f.close()
    return out


@pytest.mark.parametrize("name", ["room", "room_surface", "room_unbounded_surface"])
@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp8"])
def test_full_frame_tensorcore_sampled(V, name, prec):
    sc, c2w, K, res, pick, ref = _scene_and_ref(name)
    lin, pq, n, stats = _render_full(V, sc, c2w, K, res, prec)
    rays = SIDE * SIDE
    # far more rays than the persistent grid has slots: slots refill
    slots = torch.cuda.get_device_properties(0).multi_processor_count * 6 * 128
    assert rays > 10 * slots
    assert stats[3] == rays  # every ray finished exactly once
    assert np.isfinite(lin).all() and (lin >= 0).all()
    assert ((pq >= 0) & (pq <= 1)).all()
    lin, pq, n = lin[pick], pq[pick], n[pick]
    err = np.abs(pq.astype(np.float64) - ref["pq"])
    mse = float(np.mean(err ** 2))
    psnr = float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)
    print(f"full-frame {name} {prec}: PQ-PSNR {psnr:.2f} dB over {N_SAMPLE} rays, max |err| "
          f"{err.max():.3e}, T_eps flips {(n != ref['n']).sum()}")
    if prec == "fp16":
        flip = n != ref["n"]
        close = lambda a, b: np.abs(np.asarray(a, np.float64) - b) <= TC_RTOL * np.abs(b) + TC_ATOL
        good = close(pq, ref["pq"]).all(1) & close(lin, ref["linear"]).all(1)
        bad = ~good & ~flip
        assert not bad.any(), (bad.sum(), err[bad].max())
        if flip.any():
            assert err[flip].max() <= sc.cfg.T_eps + 1e-4
            assert flip.mean() <= 0.01
    else:
        assert psnr >= 50.0, psnr
        assert err.max() <= PER_RAY[prec], err.max()
