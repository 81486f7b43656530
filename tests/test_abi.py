"""C-ABI library: loads, exports every declared entry point, validates
descriptions on the host. No GPU compute."""
import ctypes
import glob
import os
import re

import pytest

from paper_2311_02542_gb300 import build as B
from paper_2311_02542_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(vrnerf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_checked_library_exports_the_same_symbols_and_says_so(lib):
    checked = ctypes.CDLL(B.LIB_CHECKED)
    missing = [n for n in sorted(_declared()) if not hasattr(checked, n)]
    assert not missing, missing
    assert checked.vrnerf_build_checked() == 1 and lib.vrnerf_build_checked() == 0


def test_field_sizes_and_validation_on_host(lib):
    from paper_2311_02542_gb300 import vrnerf as V
    cfg = S.cfg_room()
    gb, mf, ow = V.vrnerf_field_sizes(cfg)
    assert gb == 16 * (1 << 21) * 2 * 2
    assert mf == cfg.n_mlp() == 64 * 32 + 16 * 64 + 64 * 32 + 64 * 64 + 3 * 64
    assert ow == 256 ** 3 // 32
    from dataclasses import replace
    for bad in (replace(cfg, feats=4), replace(cfg, levels=5), replace(cfg, d_hidden=128),
                replace(cfg, t_near=0.0), replace(cfg, occ_res=(0, 4, 4)),
                replace(cfg, aabb_max=(0.0, 20.0, 3.0))):
        with pytest.raises(V.VrnerfError) as e:
            V.vrnerf_field_sizes(bad)
        assert e.value.code == V.EINVAL


def test_seeded_stream_is_deterministic_and_uniform():
    a = S.uniform01(7, 1, 0, 100000)
    b = S.uniform01(7, 1, 50000, 50000)
    assert (a[50000:] == b).all()
    assert 0.0 <= a.min() and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 5e-3
    assert not (S.uniform01(7, 2, 0, 1000) == a[:1000]).any()


def test_scene_generators_hit_their_targets():
    occ = S.occupancy_spheres((64, 64, 64), 0.10, 1)
    assert 0.095 <= occ.mean() <= 0.11
    room = S.occupancy_room((256, 256, 256), (20.0, 20.0, 3.0), 0.05, 2)
    assert 0.045 <= room.mean() <= 0.06
    assert room[0].all() and room[-1].all()
    bits = S.pack_bits(occ)
    assert (S.unpack_bits(bits, (64, 64, 64)) == occ).all()


def test_noalloc_wrapper_rejects_mismatched_buffers():
    """The binding checks the caller's buffers against the description before
    vrnerf_render_noalloc sees bare pointers (a short buffer would be read past
    its end on the device). CPU tensors of the right shape pass the size and
    type checks and fail only on the device check."""
    import torch
    from paper_2311_02542_gb300 import synth as S
    from paper_2311_02542_gb300 import vrnerf as V
    cfg = S.cfg_unit_cube()                          # fp32 grid, L=8, T=2^14, 64^3 occupancy
    n_grid = cfg.levels * cfg.T * cfg.feats
    good = dict(grid=torch.zeros(n_grid), mlp=torch.zeros(cfg.n_mlp()),
                occ_bits=torch.zeros(64 ** 3 // 32, dtype=torch.int32),
                cameras=torch.zeros(1, 3, 4), intrinsics=torch.zeros(1, 4))

    def check(**kw):
        a = {**good, **kw}
        V.check_noalloc_buffers(cfg, a["grid"], a["mlp"], a["occ_bits"], a["cameras"], a["intrinsics"],
                                1, a.get("out"), 64 * 64)

    bad = [dict(grid=torch.zeros(n_grid, dtype=torch.float16)),       # fp16 grid for an fp32 field
           dict(grid=torch.zeros(n_grid // 2)),                        # smaller table
           dict(mlp=torch.zeros(cfg.n_mlp() - 1)),                     # short weights
           dict(mlp=torch.zeros(cfg.n_mlp(), dtype=torch.float64)),
           dict(occ_bits=torch.zeros(64 ** 3 // 32 - 1, dtype=torch.int32)),
           dict(occ_bits=torch.zeros(64 ** 3 // 32, dtype=torch.float32)),
           dict(cameras=torch.zeros(2, 3)),
           dict(intrinsics=torch.zeros(3)),
           dict(out=torch.zeros(64 * 64, 2)),
           dict(grid=torch.zeros(2 * n_grid)[::2])]                    # not contiguous
    for kw in bad:
        with pytest.raises(ValueError) as e:
            check(**kw)
        assert "device memory" not in str(e.value), kw
    with pytest.raises(ValueError, match="device memory"):
        check()
