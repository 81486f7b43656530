"""vrnerf_render_noalloc: the render entry point for callers that cannot
allocate GPU memory (for example a VR compositor's frame callback, where an
allocation could stall the frame, or a plug-in whose host application owns
every device allocation). It takes the field's parameters from buffers the
caller owns and keeps its scratch in a static device array.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test before it. It must pass both alone in a
fresh process and after the rest of the suite.
"""
from dataclasses import replace

import numpy as np
import pytest
import torch

from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-6


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def _caller_buffers(sc):
    grid = torch.from_numpy(np.ascontiguousarray(sc.grid)).cuda()
    mlp = _cuda(sc.mlp)
    occ = torch.from_numpy(sc.occ_bits.view(np.int32).copy()).cuda()
    return grid, mlp, occ


def test_noalloc_render_matches_render_on_consecutive_calls():
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene("unit_cube")
    cfg = sc.cfg
    field = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    grid, mlp, occ = _caller_buffers(sc)
    # two calls in a row, of different sizes: the shared counter must be
    # cleared by each call and the sample table rewritten
    for seed, w, h in ((1, 64, 48), (7, 37, 23), (1, 64, 48)):
        c2w, K, res = S.camera_unit_cube(sc.occ, cfg, seed, w, h)
        cams, intr = _cuda(c2w), _cuda(K)
        want = V.vrnerf_render(field, cams, intr, res).cpu().numpy()
        got = V.vrnerf_render_noalloc(cfg, grid, mlp, occ, cams, intr, res).cpu().numpy()
        assert np.all(np.abs(got - want) <= RTOL * np.abs(want) + ATOL)
    field.close()


def test_noalloc_render_room_fp16_features():
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene("room")
    cfg = sc.cfg
    field = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    grid, mlp, occ = _caller_buffers(sc)
    c2w, K, _ = S.camera_room(sc.occ, cfg, 2, 2048, 2048)
    res = np.array([[160, 96]], np.int32)
    cams, intr = _cuda(c2w), _cuda(S.crop_camera(K, 900, 1000))
    for _ in range(2):
        want = V.vrnerf_render(field, cams, intr, res).cpu().numpy()
        got = V.vrnerf_render_noalloc(cfg, grid, mlp, occ, cams, intr, res).cpu().numpy()
        assert np.all(np.abs(got - want) <= RTOL * np.abs(want) + ATOL)
    field.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene("unit_cube")
    grid, mlp, occ = _caller_buffers(sc)
    c2w, K, res = S.camera_unit_cube(sc.occ, sc.cfg, 1, 8, 8)
    with pytest.raises(V.VrnerfError) as e:
        V.vrnerf_render_noalloc(replace(sc.cfg, max_steps=8150), grid, mlp, occ, _cuda(c2w),
                                _cuda(K), res)
    assert e.value.code == V.EINVAL and "scratch" in str(e.value)


def test_noalloc_alternating_sample_counts():
    """Consecutive calls that change max_steps: the sample-distance table in
    the shared scratch is copied in again whenever its key changes, and the
    fp32 kernel's shared memory (weights plus the table) crosses 48 KB at
    about 3 900 steps, which needs the per-device launch attribute. Each call
    matches vrnerf_render of a field with the same description."""
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene("unit_cube")
    grid, mlp, occ = _caller_buffers(sc)
    c2w, K, res = S.camera_unit_cube(sc.occ, sc.cfg, 3, 40, 24)
    cams, intr = _cuda(c2w), _cuda(K)
    fields = {}
    for steps in (64, 4096, 64, 6000, 4096, 64):
        cfg = replace(sc.cfg, max_steps=steps)
        if steps not in fields:
            fields[steps] = V.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
        want = V.vrnerf_render(fields[steps], cams, intr, res).cpu().numpy()
        got = V.vrnerf_render_noalloc(cfg, grid, mlp, occ, cams, intr, res).cpu().numpy()
        assert np.all(np.abs(got - want) <= RTOL * np.abs(want) + ATOL), steps
    for f in fields.values():
        f.close()
