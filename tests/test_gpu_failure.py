"""Failure detection on the GPU without a fault: a device-side wait that can
never complete gives up after its time limit, reports ETIMEDOUT through the
field's status word, frees its TMEM, and the context keeps working."""
import numpy as np
import pytest
import torch

from paper_2311_02542_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    from paper_2311_02542_gb300 import vrnerf as V
    V.load()
    sc = S.make_scene("unit_cube")
    f = V.Field(sc.cfg, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, sc.cfg, 1, 32, 32)
    cams, intr = torch.from_numpy(c2w).cuda(), torch.from_numpy(K).cuda()
    before = V.vrnerf_render(f, cams, intr, res, precision="fp16").cpu().numpy()
    V.vrnerf_field_status(f)  # clean
    V.vrnerf_debug_wait_timeout(f, 20000)  # 20 ms
    with pytest.raises(V.VrnerfError) as e:
        V.vrnerf_field_status(f)
    assert e.value.code == V.ETIMEDOUT
    V.vrnerf_field_status(f)  # cleared by the read
    after = V.vrnerf_render(f, cams, intr, res, precision="fp16").cpu().numpy()
    assert np.array_equal(before, after)
    with pytest.raises(V.VrnerfError):
        V.vrnerf_debug_wait_timeout(f, 0)
    f.close()
