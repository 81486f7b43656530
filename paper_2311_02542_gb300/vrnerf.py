"""Thin Python binding of the C ABI in include/vrnerf.h.

Argument marshalling only: every step of rendering and training runs in the
CUDA library. PyTorch supplies device memory and streams. Importing this
module loads ``_build/libvrnerf.so`` and raises if it has not been built
(``python -m paper_2311_02542_gb300.build``); there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import replace
import os

import numpy as np
import torch

from . import build as _build

FP32, FP16, BF16, FP8 = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32, "fp16": FP16, "bf16": BF16, "fp8": FP8}
OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, EBUSY, ENOTFOUND, ECANCELED, ECHECK = 0, -1, -2, -3, -4, -5, -6, -7, -8
ELATE = -9


class VrnerfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"vrnerf error {code}: {msg}")
        self.code = code


class FieldDesc(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int32), ("feats", ctypes.c_int32), ("log2_T", ctypes.c_int32),
        ("feat_fp16", ctypes.c_int32),
        ("base_res", ctypes.c_double), ("growth", ctypes.c_double),
        ("d_hidden", ctypes.c_int32), ("d_out", ctypes.c_int32), ("c_hidden", ctypes.c_int32),
        ("c_layers", ctypes.c_int32),
        ("aabb_min", ctypes.c_float * 3), ("aabb_max", ctypes.c_float * 3),
        ("occ_res", ctypes.c_int32 * 3),
        ("max_steps", ctypes.c_int32),
        ("t_near", ctypes.c_float), ("t_far", ctypes.c_float),
        ("lod_bias", ctypes.c_float), ("T_eps", ctypes.c_float),
        ("radius_scale", ctypes.c_float), ("density_bias", ctypes.c_float),
        ("contract", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


class RenderOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("out_pq", ctypes.c_void_p), ("out_T", ctypes.c_void_p), ("out_n", ctypes.c_void_p),
                ("stats", ctypes.c_void_p), ("out_depth", ctypes.c_void_p),
                ("out_normal", ctypes.c_void_p), ("out_rgba8", ctypes.c_void_p),
                ("exposure_ev", ctypes.c_float), ("reserved2", ctypes.c_int32)]


_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_F = ctypes.c_float
_SIGS = {
    "vrnerf_last_error": (ctypes.c_char_p, []),
    "vrnerf_field_sizes": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "vrnerf_field_create": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_uint64, _VP]),
    "vrnerf_field_destroy": (None, [_VP]),
    "vrnerf_field_get_params": (ctypes.c_int, [_VP, _VP, _VP]),
    "vrnerf_field_status": (ctypes.c_int, [_VP]),
    "vrnerf_debug_wait_timeout": (ctypes.c_int, [_VP, ctypes.c_uint32, _VP]),
    "vrnerf_field_set_occupancy": (ctypes.c_int, [_VP, _VP]),
    "vrnerf_field_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "vrnerf_history_reset": (ctypes.c_int, [_VP]),
    "vrnerf_build_checked": (ctypes.c_int, []),
    "vrnerf_field_set_train_precision": (ctypes.c_int, [_VP, _I32]),
    "vrnerf_field_set_sample_budget": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "vrnerf_debug_check_trigger": (ctypes.c_int, [_VP, _VP]),
    "vrnerf_forward_rays": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "vrnerf_backward_from_grad": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "vrnerf_field_param_ptrs": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "vrnerf_field_params_changed": (ctypes.c_int, [_VP]),
    "vrnerf_tonemap": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _F, _VP, _VP]),
    "vrnerf_occupancy_upsample": (ctypes.c_int, [_VP, _I32]),
    "vrnerf_field_get_occupancy": (ctypes.c_int, [_VP, _VP]),
    "vrnerf_field_get_history": (ctypes.c_int, [_VP, _VP]),
    "vrnerf_prune": (ctypes.c_int, [_VP, _VP, _I32, _I32, _F, _I32, _VP, _VP, _VP]),
    "vrnerf_field_load": (ctypes.c_int, [ctypes.c_char_p, _VP]),
    "vrnerf_render": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "vrnerf_render_host": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "vrnerf_render_rays": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "vrnerf_query": (ctypes.c_int, [_VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP, _I32, _VP]),
    "vrnerf_debug_march": (ctypes.c_int, [_VP, _VP, _VP, _I32, _I32, _VP, _VP, _VP, _VP]),
    "vrnerf_debug_corners": (ctypes.c_int, [_VP, _VP, _I32, _VP, _VP]),
    "vrnerf_backward": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP]),
    "vrnerf_field_get_grads": (ctypes.c_int, [_VP, _VP, _VP]),
    "vrnerf_field_set_grads": (ctypes.c_int, [_VP, _VP, _VP]),
    "vrnerf_adam_step": (ctypes.c_int, [_VP, _F, _F, _VP]),
    "vrnerf_train_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _I32, _F, _F, _VP, _VP]),
    "vrnerf_render_noalloc": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP]),
    "vrnerf_server_create": (ctypes.c_int, [_VP, ctypes.c_uint64, _I32, _VP]),
    "vrnerf_submit": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "vrnerf_submit_deadline": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, ctypes.c_double, _I32, _VP]),
    "vrnerf_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _I32, _VP]),
    "vrnerf_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "vrnerf_server_stats": (ctypes.c_int, [_VP, _VP]),
    "vrnerf_server_reset_stats": (ctypes.c_int, [_VP]),
    "vrnerf_server_destroy": (None, [_VP]),
}


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("rays", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("pending", ctypes.c_uint64),
                ("inflight", ctypes.c_uint64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("max_inflight", ctypes.c_uint64), ("tile_rounds", ctypes.c_uint64),
                ("mixed_tile_rounds", ctypes.c_uint64), ("late", ctypes.c_uint64), ("shed", ctypes.c_uint64),
                ("wait_p50_ms", ctypes.c_double), ("wait_p99_ms", ctypes.c_double),
                ("gpu_p50_ms", ctypes.c_double), ("gpu_p99_ms", ctypes.c_double),
                ("copy_p50_ms", ctypes.c_double), ("copy_p99_ms", ctypes.c_double)]

_lib = None


def lib_path() -> str:
    """The release library, or the checked one (device-side bounds checks)
    when the environment sets VRNERF_CHECKED=1."""
    return _build.LIB_CHECKED if os.environ.get("VRNERF_CHECKED") == "1" else _build.LIB


def load():
    """Loads the CUDA library (torch is imported first so both share one CUDA runtime)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run "
                               "`python -m paper_2311_02542_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name, None)
            if fn is None:
                continue
            fn.restype, fn.argtypes = res, args
        _lib = L
    return _lib


def last_error() -> str:
    return load().vrnerf_last_error().decode()


def _check(rc):
    if rc != OK:
        raise VrnerfError(rc, last_error())


def desc(cfg) -> FieldDesc:
    d = FieldDesc()
    d.levels, d.feats, d.log2_T = cfg.levels, cfg.feats, cfg.log2_T
    d.feat_fp16 = int(cfg.feat_fp16)
    d.base_res, d.growth = cfg.base_res, cfg.growth
    d.d_hidden, d.d_out, d.c_hidden, d.c_layers = cfg.d_hidden, cfg.d_out, cfg.c_hidden, cfg.c_layers
    d.aabb_min[:] = list(cfg.aabb_min)
    d.aabb_max[:] = list(cfg.aabb_max)
    d.occ_res[:] = list(cfg.occ_res)
    d.max_steps = cfg.max_steps
    d.t_near, d.t_far = cfg.t_near, cfg.t_far
    d.lod_bias, d.T_eps = cfg.lod_bias, cfg.T_eps
    d.radius_scale, d.density_bias = cfg.radius_scale, cfg.density_bias
    d.contract = int(getattr(cfg, "contract", False))
    return d


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        assert t.is_contiguous(), "tensors passed to the library must be contiguous"
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype=torch.float32):
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()
    return t


class Field:
    """Owns a vrnerf_field* (device parameters, occupancy and scratch)."""

    def __init__(self, cfg, grid=None, mlp=None, occ_bits=None, seed=0):
        L = load()
        self.cfg = cfg
        self._desc = desc(cfg)
        h = ctypes.c_void_p()
        g = None if grid is None else np.ascontiguousarray(grid)
        m = None if mlp is None else np.ascontiguousarray(mlp, dtype=np.float32)
        o = np.ascontiguousarray(occ_bits, dtype=np.uint32)
        if g is not None:
            want = np.float16 if cfg.feat_fp16 else np.float32
            assert g.dtype == want and g.size == cfg.levels * cfg.T * cfg.feats
        _check(L.vrnerf_field_create(ctypes.byref(self._desc), _ptr(g), _ptr(m), _ptr(o),
                                     ctypes.c_uint64(seed), ctypes.byref(h)))
        self.h = h
        self.n_rays_last = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h and _lib is not None:
            _lib.vrnerf_field_destroy(h)
            self.h = None

    def close(self):
        self.__del__()


def vrnerf_field_sizes(cfg):
    gb, mf, ow = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    d = desc(cfg)
    _check(load().vrnerf_field_sizes(ctypes.byref(d), ctypes.byref(gb), ctypes.byref(mf), ctypes.byref(ow)))
    return gb.value, mf.value, ow.value


def vrnerf_field_create(cfg, grid=None, mlp=None, occ_bits=None, seed=0) -> Field:
    return Field(cfg, grid, mlp, occ_bits, seed)


def vrnerf_field_destroy(field: Field):
    field.close()


def vrnerf_field_status(field: Field):
    """Raises VrnerfError if a kernel of the field recorded an error (e.g. a
    bounded device wait that timed out); clears it."""
    _check(load().vrnerf_field_status(field.h))


def vrnerf_debug_wait_timeout(field: Field, limit_us: int, stream=None):
    _check(load().vrnerf_debug_wait_timeout(field.h, int(limit_us), _stream(stream)))


def vrnerf_field_get_params(field: Field):
    cfg = field.cfg
    g = np.empty((cfg.levels, cfg.T, cfg.feats), np.float16 if cfg.feat_fp16 else np.float32)
    m = np.empty(cfg.n_mlp(), np.float32)
    _check(load().vrnerf_field_get_params(field.h, _ptr(g), _ptr(m)))
    return g, m


def vrnerf_field_save(field: Field, path: str):
    _check(load().vrnerf_field_save(field.h, os.fsencode(path)))


def vrnerf_field_load(path: str, cfg) -> Field:
    """Loads a checkpoint; `cfg` is the FieldConfig it was written from (the
    binding keeps it for array shapes)."""
    f = Field.__new__(Field)
    h = ctypes.c_void_p()
    _check(load().vrnerf_field_load(os.fsencode(path), ctypes.byref(h)))
    f.cfg, f.h, f._desc, f.n_rays_last = cfg, h, desc(cfg), 0
    return f


def vrnerf_tonemap(pq, T=None, exposure_ev=0.0, out=None, stream=None):
    """pq [n][3] (and T [n]) CUDA tensors -> packed sRGB8 + coverage int32 [n]."""
    n = pq.shape[0]
    if out is None:
        out = torch.empty(n, device=pq.device, dtype=torch.int32)
    _check(load().vrnerf_tonemap(_ptr(_dev(pq)), _ptr(None if T is None else _dev(T)), n,
                                 float(exposure_ev), _ptr(_dev(out, torch.int32)), _stream(stream)))
    return out


def vrnerf_forward_rays(field: Field, rays_o, rays_d, radii, out_pq=None, out_n=None, stream=None):
    """PQ colours [B][3] and sample counts [B] of explicit rays, sample-parallel."""
    B = rays_o.shape[0]
    if out_pq is None:
        out_pq = torch.empty((B, 3), device=rays_o.device, dtype=torch.float32)
    if out_n is None:
        out_n = torch.empty(B, device=rays_o.device, dtype=torch.int32)
    _check(load().vrnerf_forward_rays(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)), _ptr(_dev(radii)), B,
                                      _ptr(_dev(out_pq)), _ptr(_dev(out_n, torch.int32)), _stream(stream)))
    return out_pq, out_n


def vrnerf_backward_from_grad(field: Field, rays_o, rays_d, radii, n_fwd, grad_pq, stream=None):
    B = rays_o.shape[0]
    _check(load().vrnerf_backward_from_grad(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)), _ptr(_dev(radii)),
                                            B, _ptr(_dev(n_fwd, torch.int32)), _ptr(_dev(grad_pq)),
                                            _stream(stream)))


class _DeviceArray:
    """A device buffer of the library described by __cuda_array_interface__,
    so that torch.as_tensor views it without a copy."""

    def __init__(self, ptr, shape, typestr, owner):
        self.owner = owner  # keeps the field alive as long as the view
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def vrnerf_field_param_views(field: Field, grads=True):
    """Zero-copy torch views of the field's parameters (grid [L][T][F] in its
    storage type, mlp fp32) and, with grads, of its fp32 gradient buffers."""
    cfg = field.cfg
    g, m, gg, gm = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().vrnerf_field_param_ptrs(field.h, ctypes.byref(g), ctypes.byref(m),
                                          ctypes.byref(gg) if grads else None,
                                          ctypes.byref(gm) if grads else None))
    shape = (cfg.levels, cfg.T, cfg.feats)
    out = {"grid": torch.as_tensor(_DeviceArray(g.value, shape, "<f2" if cfg.feat_fp16 else "<f4", field),
                                   device="cuda"),
           "mlp": torch.as_tensor(_DeviceArray(m.value, (cfg.n_mlp(),), "<f4", field), device="cuda")}
    if grads:
        out["grid_grad"] = torch.as_tensor(_DeviceArray(gg.value, shape, "<f4", field), device="cuda")
        out["mlp_grad"] = torch.as_tensor(_DeviceArray(gm.value, (cfg.n_mlp(),), "<f4", field), device="cuda")
    return out


def vrnerf_field_params_changed(field: Field):
    _check(load().vrnerf_field_params_changed(field.h))


class RenderRaysFunction(torch.autograd.Function):
    """PQ colours of explicit rays (fp32 path) as a differentiable function of
    the field's parameters: forward and backward run the library's
    sample-parallel training kernels (samples recomputed in backward)."""

    @staticmethod
    def forward(ctx, field, rays_o, rays_d, radii, grid, mlp):
        pq, n = vrnerf_forward_rays(field, rays_o, rays_d, radii)
        ctx.field = field
        ctx.save_for_backward(rays_o, rays_d, radii, n)
        return pq

    @staticmethod
    def backward(ctx, grad_pq):
        o, d, r, n = ctx.saved_tensors
        field = ctx.field
        vrnerf_backward_from_grad(field, o, d, r, n, grad_pq.contiguous())
        v = vrnerf_field_param_views(field)
        gg = v["grid_grad"].clone()
        if field.cfg.feat_fp16:
            gg = gg.to(torch.float16)
        return None, None, None, None, gg, v["mlp_grad"].clone()


class FieldModule(torch.nn.Module):
    """The field as a torch module: parameters are views of the library's
    buffers, forward(rays_o, rays_d, radii) returns PQ colours [B][3]. After
    changing the parameters outside the library (a torch optimiser step),
    call params_changed() before rendering with the tensor-core paths."""

    def __init__(self, field: Field):
        super().__init__()
        self.field = field
        v = vrnerf_field_param_views(field, grads=False)
        self.grid = torch.nn.Parameter(v["grid"])
        self.mlp = torch.nn.Parameter(v["mlp"])

    def forward(self, rays_o, rays_d, radii):
        return RenderRaysFunction.apply(self.field, rays_o, rays_d, radii, self.grid, self.mlp)

    def params_changed(self):
        vrnerf_field_params_changed(self.field)


def vrnerf_field_set_sample_budget(field: Field, max_samples: int):
    """Most samples one training pass holds (0: the library's default)."""
    _check(load().vrnerf_field_set_sample_budget(field.h, int(max_samples)))


def vrnerf_field_set_train_precision(field: Field, precision):
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    _check(load().vrnerf_field_set_train_precision(field.h, p))


def vrnerf_build_checked() -> bool:
    return bool(load().vrnerf_build_checked())


def vrnerf_debug_check_trigger(field: Field, stream=None):
    _check(load().vrnerf_debug_check_trigger(field.h, _stream(stream)))


def vrnerf_history_reset(field: Field):
    _check(load().vrnerf_history_reset(field.h))


def vrnerf_field_get_history(field: Field):
    cfg = field.cfg
    h = np.empty(cfg.occ_res[0] * cfg.occ_res[1] * cfg.occ_res[2], np.float32)
    _check(load().vrnerf_field_get_history(field.h, _ptr(h)))
    return h


def vrnerf_prune(field: Field, camera_centres, points_per_axis=4, threshold=0.2, apply=True,
                 want_alpha=False):
    """Returns (kept voxel count, alpha [voxels] or None, new occupancy bits)."""
    cfg = field.cfg
    cams = np.ascontiguousarray(camera_centres, np.float32).reshape(-1, 3)
    nvox = cfg.occ_res[0] * cfg.occ_res[1] * cfg.occ_res[2]
    alpha = torch.empty(nvox, device="cuda") if want_alpha else None
    bits = torch.empty((nvox + 31) // 32, device="cuda", dtype=torch.int32)
    kept = ctypes.c_uint64()
    _check(load().vrnerf_prune(field.h, _ptr(cams), cams.shape[0], int(points_per_axis),
                               float(threshold), int(bool(apply)), _ptr(alpha), _ptr(bits),
                               ctypes.byref(kept)))
    return kept.value, (alpha.cpu().numpy() if want_alpha else None), bits.cpu().numpy().view(np.uint32)


def vrnerf_occupancy_upsample(field: Field, factor=2):
    _check(load().vrnerf_occupancy_upsample(field.h, int(factor)))
    field.cfg = replace(field.cfg, occ_res=tuple(int(r) * int(factor) for r in field.cfg.occ_res))


def vrnerf_field_get_occupancy(field: Field):
    r = field.cfg.occ_res
    bits = np.empty((r[0] * r[1] * r[2] + 31) // 32, np.uint32)
    _check(load().vrnerf_field_get_occupancy(field.h, _ptr(bits)))
    return bits


def vrnerf_field_set_occupancy(field: Field, occ_bits):
    o = np.ascontiguousarray(occ_bits, dtype=np.uint32)
    _check(load().vrnerf_field_set_occupancy(field.h, _ptr(o)))


def _opts(precision, out_pq=None, out_T=None, out_n=None, stats=None, out_depth=None,
          out_normal=None, out_rgba8=None, exposure_ev=0.0):
    o = RenderOpts()
    o.out_normal = None if out_normal is None else _dev(out_normal).data_ptr()
    o.out_rgba8 = None if out_rgba8 is None else _dev(out_rgba8, torch.int32).data_ptr()
    o.exposure_ev = float(exposure_ev)
    o.out_depth = None if out_depth is None else _dev(out_depth).data_ptr()
    o.stats = None if stats is None else _dev(stats, torch.int64).data_ptr()
    o.precision = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    o.out_pq = None if out_pq is None else _dev(out_pq).data_ptr()
    o.out_T = None if out_T is None else _dev(out_T).data_ptr()
    o.out_n = None if out_n is None else _dev(out_n, torch.int32).data_ptr()
    return o


def vrnerf_render(field: Field, cameras, intrinsics, resolution, out=None, precision=FP32,
                  out_pq=None, out_T=None, out_n=None, stats=None, out_depth=None, out_normal=None,
                  out_rgba8=None, exposure_ev=0.0, stream=None):
    """cameras [n][3][4], intrinsics [n][4]: float32 CUDA tensors; resolution
    [n][2] (W, H) on the host. Returns out [sum W*H][3] linear colour."""
    res = np.ascontiguousarray(resolution, dtype=np.int32).reshape(-1, 2)
    rays = int((res[:, 0].astype(np.int64) * res[:, 1]).sum())
    if out is None:
        out = torch.empty((rays, 3), device=cameras.device, dtype=torch.float32)
    o = _opts(precision, out_pq, out_T, out_n, stats, out_depth, out_normal, out_rgba8, exposure_ev)
    _check(load().vrnerf_render(field.h, _ptr(_dev(cameras)), _ptr(_dev(intrinsics)), _ptr(res),
                                res.shape[0], _ptr(_dev(out)), ctypes.byref(o), _stream(stream)))
    return out


def vrnerf_render_host(field: Field, cameras, intrinsics, resolution, out=None, precision=FP32,
                       stream=None):
    """All arrays on the host (numpy); copies in and out inside the call."""
    res = np.ascontiguousarray(resolution, dtype=np.int32).reshape(-1, 2)
    rays = int((res[:, 0].astype(np.int64) * res[:, 1]).sum())
    cams = np.ascontiguousarray(cameras, dtype=np.float32)
    K = np.ascontiguousarray(intrinsics, dtype=np.float32)
    if out is None:
        out = np.empty((rays, 3), np.float32)
    o = _opts(precision)
    _check(load().vrnerf_render_host(field.h, _ptr(cams), _ptr(K), _ptr(res), res.shape[0],
                                     _ptr(out), ctypes.byref(o), _stream(stream)))
    return out


def vrnerf_render_rays(field: Field, rays_o, rays_d, radii, out=None, precision=FP32, out_pq=None,
                       out_T=None, out_n=None, stats=None, out_depth=None, out_normal=None,
                       out_rgba8=None, exposure_ev=0.0, stream=None):
    B = rays_o.shape[0]
    if out is None:
        out = torch.empty((B, 3), device=rays_o.device, dtype=torch.float32)
    o = _opts(precision, out_pq, out_T, out_n, stats, out_depth, out_normal, out_rgba8, exposure_ev)
    _check(load().vrnerf_render_rays(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)),
                                     _ptr(_dev(radii)), B, _ptr(_dev(out)), ctypes.byref(o),
                                     _stream(stream)))
    return out


def vrnerf_query(field: Field, pos, direction, radius, precision=FP32, with_feat=False, stream=None):
    n = pos.shape[0]
    dev = pos.device
    sigma = torch.empty(n, device=dev)
    rgb = torch.empty((n, 3), device=dev)
    feat = torch.empty((n, field.cfg.d_in), device=dev) if with_feat else None
    p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
    _check(load().vrnerf_query(field.h, _ptr(_dev(pos)), _ptr(_dev(direction)), _ptr(_dev(radius)),
                               n, _ptr(sigma), _ptr(rgb), _ptr(feat), p, _stream(stream)))
    return sigma, rgb, feat


def vrnerf_debug_march(field: Field, rays_o, rays_d, cap, stream=None):
    B = rays_o.shape[0]
    dev = rays_o.device
    rec_i = torch.full((B, cap), -1, device=dev, dtype=torch.int32)
    rec_v = torch.full((B, cap), -1, device=dev, dtype=torch.int32)
    cnt = torch.empty(B, device=dev, dtype=torch.int32)
    _check(load().vrnerf_debug_march(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)), B, cap,
                                     _ptr(rec_i), _ptr(rec_v), _ptr(cnt), _stream(stream)))
    return rec_i, rec_v, cnt


def vrnerf_debug_corners(field: Field, pos, stream=None):
    n = pos.shape[0]
    idx = torch.empty((n, field.cfg.levels, 8), device=pos.device, dtype=torch.int32)
    _check(load().vrnerf_debug_corners(field.h, _ptr(_dev(pos)), n, _ptr(idx), _stream(stream)))
    return idx


def vrnerf_backward(field: Field, rays_o, rays_d, radii, target_linear, stream=None):
    B = rays_o.shape[0]
    loss = ctypes.c_float()
    _check(load().vrnerf_backward(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)), _ptr(_dev(radii)),
                                  _ptr(_dev(target_linear)), B, ctypes.byref(loss), _stream(stream)))
    return loss.value


def vrnerf_field_get_grads(field: Field):
    cfg = field.cfg
    g = np.empty((cfg.levels, cfg.T, cfg.feats), np.float32)
    m = np.empty(cfg.n_mlp(), np.float32)
    _check(load().vrnerf_field_get_grads(field.h, _ptr(g), _ptr(m)))
    return g, m


def vrnerf_field_set_grads(field: Field, grid_grad, mlp_grad):
    g = np.ascontiguousarray(grid_grad, dtype=np.float32)
    m = np.ascontiguousarray(mlp_grad, dtype=np.float32)
    _check(load().vrnerf_field_set_grads(field.h, _ptr(g), _ptr(m)))


def vrnerf_adam_step(field: Field, lr_grid=0.01, lr_mlp=0.005, stream=None):
    _check(load().vrnerf_adam_step(field.h, lr_grid, lr_mlp, _stream(stream)))


def vrnerf_train_step(field: Field, rays_o, rays_d, radii, target_linear, lr_grid=0.01,
                      lr_mlp=0.005, want_loss=True, stream=None):
    B = rays_o.shape[0]
    loss = ctypes.c_float()
    _check(load().vrnerf_train_step(field.h, _ptr(_dev(rays_o)), _ptr(_dev(rays_d)),
                                    _ptr(_dev(radii)), _ptr(_dev(target_linear)), B, lr_grid,
                                    lr_mlp, ctypes.byref(loss) if want_loss else None,
                                    _stream(stream)))
    return loss.value if want_loss else None


def check_noalloc_buffers(cfg, grid, mlp, occ_bits, cameras, intrinsics, n_views, out, rays):
    """Checks the caller-owned buffers of vrnerf_render_noalloc against the
    description before the call: the C entry point receives bare pointers and
    cannot see their sizes, so a short or mistyped buffer would be read past
    its end on the device. Raises ValueError."""
    def need(t, name, dtypes, numel, at_least=False):
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if t.dtype not in dtypes:
            raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
        if (t.numel() < numel) if at_least else (t.numel() != numel):
            raise ValueError(f"{name} holds {t.numel()} elements, expected {'at least ' if at_least else ''}{numel}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    grid_dtype = (torch.float16,) if cfg.feat_fp16 else (torch.float32,)
    need(grid, "grid", grid_dtype, cfg.levels * cfg.T * cfg.feats)
    need(mlp, "mlp", (torch.float32,), cfg.n_mlp())
    nvox = int(cfg.occ_res[0]) * int(cfg.occ_res[1]) * int(cfg.occ_res[2])
    occ_types = tuple(t for t in (torch.int32, getattr(torch, "uint32", None)) if t is not None)
    need(occ_bits, "occ_bits", occ_types, (nvox + 31) // 32, at_least=True)
    need(cameras, "cameras", (torch.float32,), 12 * n_views)
    need(intrinsics, "intrinsics", (torch.float32,), 4 * n_views)
    if out is not None:
        need(out, "out", (torch.float32,), 3 * rays)
    for name, t in (("grid", grid), ("mlp", mlp), ("occ_bits", occ_bits), ("cameras", cameras),
                    ("intrinsics", intrinsics), ("out", out)):
        if t is not None and not t.is_cuda:
            raise ValueError(f"{name} must be in device memory")


def vrnerf_render_noalloc(cfg, grid, mlp, occ_bits, cameras, intrinsics, resolution, out=None,
                          stream=None):
    """fp32 render that allocates nothing in the library: grid / mlp / occ_bits
    are caller-owned CUDA tensors (fp16 or fp32 grid, fp32 weights, occupancy
    words as int32 or uint32). `out` is allocated here only when not given."""
    res = np.ascontiguousarray(resolution, dtype=np.int32).reshape(-1, 2)
    rays = int((res[:, 0].astype(np.int64) * res[:, 1]).sum())
    check_noalloc_buffers(cfg, grid, mlp, occ_bits, cameras, intrinsics, res.shape[0], out, rays)
    if out is None:
        out = torch.empty((rays, 3), device=cameras.device, dtype=torch.float32)
    d = desc(cfg)
    _check(load().vrnerf_render_noalloc(ctypes.byref(d), _ptr(grid), _ptr(_dev(mlp)), _ptr(occ_bits),
                                        _ptr(_dev(cameras)), _ptr(_dev(intrinsics)), _ptr(res),
                                        res.shape[0], _ptr(_dev(out)), _stream(stream)))
    return out


class Server:
    """Continuous-batching render server (vrnerf_server_*). Holds references
    to the host arrays of every request until it is polled."""

    def __init__(self, field: Field, hbm_budget_bytes: int, precision=FP16):
        self.field = field
        h = ctypes.c_void_p()
        p = PRECISIONS.get(precision, precision) if isinstance(precision, str) else int(precision)
        _check(load().vrnerf_server_create(field.h, ctypes.c_uint64(int(hbm_budget_bytes)), p,
                                           ctypes.byref(h)))
        self.h = h
        self._keep = {}

    def submit(self, cameras, intrinsics, resolution, out=None, deadline_ms=None, shed_if_late=False):
        """Queues a request; with deadline_ms it is admitted earliest deadline
        first (vrnerf_submit_deadline), and shed_if_late drops it if the
        deadline passes while it waits."""
        cams = np.ascontiguousarray(cameras, np.float32).reshape(-1, 3, 4)
        K = np.ascontiguousarray(intrinsics, np.float32).reshape(-1, 4)
        res = np.ascontiguousarray(resolution, np.int32).reshape(-1, 2)
        t = ctypes.c_uint64()
        o = _ptr(out) if out is not None else None
        if deadline_ms is None:
            _check(load().vrnerf_submit(self.h, cams.shape[0], _ptr(cams), _ptr(K), _ptr(res), o, ctypes.byref(t)))
        else:
            _check(load().vrnerf_submit_deadline(self.h, cams.shape[0], _ptr(cams), _ptr(K), _ptr(res), o,
                                                 float(deadline_ms), int(bool(shed_if_late)), ctypes.byref(t)))
        self._keep[t.value] = out
        return t.value

    def poll(self, ticket, timeout_ms=10000):
        lat = ctypes.c_double()
        rc = load().vrnerf_poll(self.h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(lat))
        if rc in (OK, ECANCELED, ELATE):
            self._keep.pop(ticket, None)
        _check(rc)
        return lat.value

    def cancel(self, ticket):
        _check(load().vrnerf_cancel(self.h, ctypes.c_uint64(ticket)))

    def stats(self):
        st = ServerStats()
        _check(load().vrnerf_server_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(load().vrnerf_server_reset_stats(self.h))

    def close(self):
        if getattr(self, "h", None):
            load().vrnerf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        if _lib is not None:
            self.close()


def vrnerf_server_create(field: Field, hbm_budget_bytes: int, precision=FP16) -> Server:
    return Server(field, hbm_budget_bytes, precision)
