"""CPU oracle of VR-NeRF's per-ray field rendering -- TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline load this package. The product path (the CUDA library and its
binding) never imports it and shares no code with it.

The arithmetic lives in ``vrnerf_oracle.c`` (plain C, fp64 radiance, fp32
decisions for voxel visits and hash corners); this module compiles it with
gcc and marshals numpy arrays through ctypes.

Parity status per function (what pins it, see tests/test_oracle_*.py):
  pq_encode / pq_decode   ST 2084 anchor values, PQ(1) = 1, round trip, monotone
  lod_weights / lod_level Eq. 3 hand-worked cases, sum rule, closed-form L*
  level_res / dense rule  hand-derived level tables of both configurations
  corners                 brute-force vertex enumeration, bijection, linear-field
                          interpolation exactness
  sh16                    orthonormality by quadrature, addition theorem
  query (MLP)             hand-set weights with closed forms, independent matmul
  render_rays / render    constant-density closed form, opacity invariants,
                          empty grid, early-termination bound, slab brute force;
                          depth: opaque first sample, bounds by t and opacity
  march                   brute-force occupancy visits on tiny grids
  backward / backward_grad central finite differences in fp64 (of the L1 loss, and of a
                          random linear functional of the PQ colours)
  adam                    closed-form first and second steps
  prune / history         thresholds 0 and > 1, monotone in the threshold, constant-density
                          opacity against a brute-force nearest-camera spacing; history
                          against the march's own visit records
  upsample_occupancy      brute-force child-to-parent loop on a tiny grid
  density_grad / normals  central differences of sigma in fp64; a field whose density
                          grows along one axis gives normals -axis, composited to (1 - T)
  grid_position / uncontract / footprint (contracted scenes)
                          closed-form contractions on and off the axes, continuity at the
                          inner cube, round trip through the inverse, first-order footprint
                          against finite differences of the contraction, det(J)^(1/3)
                          against a finite-difference Jacobian, contracted march by brute force
  tonemap                 sRGB anchors of IEC 61966-2-1 at PQ inputs of known luminance,
                          exposure doubling, coverage from T
Parity unpinned: the appearance of a random field (nothing in the paper fixes it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vrnerf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc_vrnerf.so")
_lib = None
_lock = threading.Lock()

CFLAGS = ["-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
          "-fopenmp"]


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Desc(ctypes.Structure):
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
        ("lod_bias", ctypes.c_double), ("T_eps", ctypes.c_double),
        ("radius_scale", ctypes.c_double), ("density_bias", ctypes.c_double),
        ("contract", ctypes.c_int32), ("pad", ctypes.c_int32),
    ]


def desc(cfg) -> Desc:
    d = Desc()
    d.levels, d.feats, d.log2_T = cfg.levels, cfg.feats, cfg.log2_T
    d.feat_fp16 = int(cfg.feat_fp16)
    d.base_res, d.growth = cfg.base_res, cfg.growth
    d.d_hidden, d.d_out, d.c_hidden, d.c_layers = cfg.d_hidden, cfg.d_out, cfg.c_hidden, cfg.c_layers
    d.aabb_min[:] = [float(np.float32(v)) for v in cfg.aabb_min]
    d.aabb_max[:] = [float(np.float32(v)) for v in cfg.aabb_max]
    d.occ_res[:] = list(cfg.occ_res)
    d.max_steps = cfg.max_steps
    d.t_near, d.t_far = float(np.float32(cfg.t_near)), float(np.float32(cfg.t_far))
    d.lod_bias, d.T_eps = cfg.lod_bias, cfg.T_eps
    d.radius_scale, d.density_bias = cfg.radius_scale, cfg.density_bias
    d.contract = int(getattr(cfg, "contract", False))
    return d


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


_F32 = ctypes.POINTER(ctypes.c_float)
_F64 = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_DP = ctypes.POINTER(Desc)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_pq_encode": (ctypes.c_double, [ctypes.c_double]),
                "orc_pq_decode": (ctypes.c_double, [ctypes.c_double]),
                "orc_linear_to_pq": (ctypes.c_double, [ctypes.c_double]),
                "orc_pq_to_linear": (ctypes.c_double, [ctypes.c_double]),
                "orc_lod_weights": (None, [ctypes.c_double, ctypes.c_int32, _F64]),
                "orc_lod_level": (ctypes.c_double, [_DP, ctypes.c_double]),
                "orc_level_res": (ctypes.c_int32, [_DP, ctypes.c_int32]),
                "orc_level_dense": (ctypes.c_int32, [_DP, ctypes.c_int32]),
                "orc_sample_table": (None, [_DP, _F32]),
                "orc_ray": (None, [_F32, _F32, ctypes.c_int32, ctypes.c_int32, _F32, _F32]),
                "orc_corners": (None, [_DP, _F32, ctypes.c_int32, _U32, _F32]),
                "orc_sh16": (None, [_F64, _F64]),
                "orc_mlp_count": (ctypes.c_int32, [_DP]),
                "orc_query": (None, [_DP, _F64, _F64, _F32, _F64, _F64, ctypes.c_int32, _F64,
                                     _F64, _F64]),
                "orc_render_rays": (None, [_DP, _F64, _F64, _U32, _F32, _F32, _F32,
                                           ctypes.c_int32, _F64, _F64, _F64, _I32, _F64, _F64,
                                           ctypes.c_int32]),
                "orc_render_rays_adjacent": (None, [_DP, _F64, _F64, _U32, _F32, _F32, _F32, _F64,
                                                    _F64, ctypes.c_int32, _F64, _F64, _F64, _I32,
                                                    _F64, _F64, ctypes.c_int32]),
                "orc_grid_position": (None, [_DP, _F32, ctypes.c_int32, _F32]),
                "orc_uncontract": (ctypes.c_int32, [_F64, _F64]),
                "orc_footprint": (ctypes.c_double, [_DP, _F64, _F64, ctypes.c_float, _F32,
                                                    ctypes.c_double]),
                "orc_camera_adjacent": (None, [_F32, _F32, _I32, ctypes.c_int32, _F64, _F64]),
                "orc_density_grad": (None, [_DP, _F64, _F64, _F32, _F64, ctypes.c_int32, _F64,
                                            _F64]),
                "orc_tonemap": (None, [_F64, _F64, ctypes.c_int64, ctypes.c_double, _U32, _F64]),
                "orc_render": (None, [_DP, _F64, _F64, _U32, _F32, _F32, _I32, ctypes.c_int32,
                                      _F64, _F64, _F64, _I32, _F64, ctypes.c_int32]),
                "orc_camera_rays": (None, [_DP, _F32, _F32, _I32, ctypes.c_int32, _F32, _F32,
                                           _F32]),
                "orc_march": (None, [_DP, _U32, _F32, _F32, ctypes.c_int32, ctypes.c_int32, _I32,
                                     _I32, _I32]),
                "orc_backward": (ctypes.c_double, [_DP, _F64, _F64, _U32, _F32, _F32, _F32, _F32,
                                                   ctypes.c_int32, _F64, _F64]),
                "orc_backward_grad": (None, [_DP, _F64, _F64, _U32, _F32, _F32, _F32, _F64,
                                             ctypes.c_int32, _F64, _F64]),
                "orc_adam": (None, [_F64, _F64, _F64, _F64, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double]),
                "orc_geometry": (None, [_DP, _I32, _I32, _F32, _F32]),
                "orc_prune": (None, [_DP, _F64, _F64, _U32, _F32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_double, _F32, ctypes.POINTER(ctypes.c_uint8), _F64]),
                "orc_history": (None, [_DP, _F64, _F64, _U32, _F32, _F32, _F32, ctypes.c_int32,
                                       _F32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype, fn.argtypes = res, args
            _lib = L
    return _lib


# ----------------------------------------------------------------------------
# numpy-facing helpers
# ----------------------------------------------------------------------------
def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def pq_encode(Y):
    return lib().orc_pq_encode(float(Y))


def pq_decode(E):
    return lib().orc_pq_decode(float(E))


def linear_to_pq(c):
    return lib().orc_linear_to_pq(float(c))


def pq_to_linear(E):
    return lib().orc_pq_to_linear(float(E))


def lod_weights(Lstar, levels):
    w = np.zeros(levels, np.float64)
    lib().orc_lod_weights(float(Lstar), levels, _p(w, ctypes.c_double))
    return w


def lod_level(cfg, r_norm):
    d = desc(cfg)
    return lib().orc_lod_level(ctypes.byref(d), float(r_norm))


def geometry(cfg):
    d = desc(cfg)
    N = np.zeros(cfg.levels, np.int32)
    dense = np.zeros(cfg.levels, np.int32)
    ic = np.zeros(3, np.float32)
    ie = np.zeros(1, np.float32)
    lib().orc_geometry(ctypes.byref(d), _p(N, ctypes.c_int32), _p(dense, ctypes.c_int32),
                       _p(ic, ctypes.c_float), _p(ie, ctypes.c_float))
    return N, dense.astype(bool), ic, float(ie[0])


def sample_table(cfg):
    d = desc(cfg)
    t = np.zeros(cfg.max_steps + 1, np.float32)
    lib().orc_sample_table(ctypes.byref(d), _p(t, ctypes.c_float))
    return t


def ray(c2w, K, u, v):
    o = np.zeros(3, np.float32)
    dd = np.zeros(3, np.float32)
    lib().orc_ray(_p(_f32(c2w), ctypes.c_float), _p(_f32(K), ctypes.c_float), int(u), int(v),
                  _p(o, ctypes.c_float), _p(dd, ctypes.c_float))
    return o, dd


def camera_rays(cfg, c2w, K, res):
    c2w, K, res = _f32(c2w), _f32(K), _i32(res)
    n = int(res.shape[0])
    total = int((res[:, 0].astype(np.int64) * res[:, 1]).sum())
    o = np.zeros((total, 3), np.float32)
    dd = np.zeros((total, 3), np.float32)
    r = np.zeros(total, np.float32)
    d = desc(cfg)
    lib().orc_camera_rays(ctypes.byref(d), _p(c2w, ctypes.c_float), _p(K, ctypes.c_float),
                          _p(res, ctypes.c_int32), n, _p(o, ctypes.c_float),
                          _p(dd, ctypes.c_float), _p(r, ctypes.c_float))
    return o, dd, r


def grid_position(cfg, pos):
    """Normalised grid position in [0, 1]^3 (fp32) of world points [n][3]:
    scaled box, or the contracted cube of an unbounded scene."""
    pos = _f32(pos).reshape(-1, 3)
    ph = np.zeros_like(pos)
    lib().orc_grid_position(ctypes.byref(desc(cfg)), _p(pos, ctypes.c_float), pos.shape[0],
                            _p(ph, ctypes.c_float))
    return ph


def uncontract(y):
    """Pre-image of a contracted point (fp64), None at |y|_inf >= 2."""
    y = _f64(y).reshape(3)
    x = np.zeros(3)
    ok = lib().orc_uncontract(_p(y, ctypes.c_double), _p(x, ctypes.c_double))
    return x if ok else None


def footprint(cfg, p, t, r, adjacent=None):
    """Normalised footprint radius of the sample at distance t and position p
    (adjacent = (du, dv) for a camera ray of a contracted scene)."""
    p = _f32(p).reshape(3)
    du, dv = (None, None) if adjacent is None else (_f64(a).reshape(3) for a in adjacent)
    return lib().orc_footprint(ctypes.byref(desc(cfg)), _p(du, ctypes.c_double),
                               _p(dv, ctypes.c_double), float(np.float32(t)),
                               _p(p, ctypes.c_float), float(r))


def camera_adjacent(c2w, K, res):
    """Per camera ray: offsets du, dv [total][3] to the directions of the
    pixels to the right and below (fp32 directions, difference in fp64)."""
    c2w, K = _f32(c2w).reshape(-1, 3, 4), _f32(K).reshape(-1, 4)
    res = _i32(res).reshape(-1, 2)
    total = int((res[:, 0].astype(np.int64) * res[:, 1]).sum())
    du = np.zeros((total, 3), np.float64)
    dv = np.zeros((total, 3), np.float64)
    lib().orc_camera_adjacent(_p(c2w, ctypes.c_float), _p(K, ctypes.c_float),
                              _p(res, ctypes.c_int32), res.shape[0], _p(du, ctypes.c_double),
                              _p(dv, ctypes.c_double))
    return du, dv


def corners(cfg, pos):
    pos = _f32(pos).reshape(-1, 3)
    n = pos.shape[0]
    idx = np.zeros((n, cfg.levels, 8), np.uint32)
    frac = np.zeros((n, cfg.levels, 3), np.float32)
    d = desc(cfg)
    lib().orc_corners(ctypes.byref(d), _p(pos, ctypes.c_float), n, _p(idx, ctypes.c_uint32),
                      _p(frac, ctypes.c_float))
    return idx, frac


def sh16(direction):
    out = np.zeros(16, np.float64)
    lib().orc_sh16(_p(_f64(direction), ctypes.c_double), _p(out, ctypes.c_double))
    return out


def mlp_count(cfg):
    d = desc(cfg)
    return lib().orc_mlp_count(ctypes.byref(d))


class Field:
    """Parameters held in fp64 (exact copies of the fp16 / fp32 inputs)."""

    def __init__(self, cfg, grid, mlp, occ_bits):
        self.cfg = cfg
        self.d = desc(cfg)
        self.grid = _f64(np.asarray(grid, dtype=np.float64).reshape(-1))
        self.mlp = _f64(np.asarray(mlp, dtype=np.float64).reshape(-1))
        self.occ = _u32(occ_bits)
        assert self.grid.size == cfg.levels * cfg.T * cfg.feats
        assert self.mlp.size == mlp_count(cfg)

    def _args(self):
        return (ctypes.byref(self.d), _p(self.grid, ctypes.c_double),
                _p(self.mlp, ctypes.c_double))

    def query(self, pos, direction, radius):
        pos = _f32(pos).reshape(-1, 3)
        n = pos.shape[0]
        sig = np.zeros(n, np.float64)
        rgb = np.zeros((n, 3), np.float64)
        feat = np.zeros((n, self.cfg.d_in), np.float64)
        lib().orc_query(*self._args(), _p(pos, ctypes.c_float),
                        _p(_f64(direction).reshape(-1, 3), ctypes.c_double),
                        _p(_f64(radius).reshape(-1), ctypes.c_double), n,
                        _p(sig, ctypes.c_double), _p(rgb, ctypes.c_double),
                        _p(feat, ctypes.c_double))
        return sig, rgb, feat

    def render_rays(self, o, dd, r, threads=None, normals=False, adjacent=None):
        """adjacent = (du, dv) [B][3] direction offsets to the adjacent pixels'
        rays (the camera-ray footprint of a contracted scene), else None."""
        o, dd, r = _f32(o).reshape(-1, 3), _f32(dd).reshape(-1, 3), _f32(r).reshape(-1)
        B = o.shape[0]
        pq = np.zeros((B, 3), np.float64)
        lin = np.zeros((B, 3), np.float64)
        T = np.zeros(B, np.float64)
        n = np.zeros(B, np.int32)
        depth = np.zeros(B, np.float64)
        nrm = np.zeros((B, 3), np.float64) if normals else None
        outs = (_p(pq, ctypes.c_double), _p(lin, ctypes.c_double), _p(T, ctypes.c_double),
                _p(n, ctypes.c_int32), _p(depth, ctypes.c_double), _p(nrm, ctypes.c_double),
                threads or os.cpu_count() or 1)
        if adjacent is None:
            lib().orc_render_rays(*self._args(), _p(self.occ, ctypes.c_uint32),
                                  _p(o, ctypes.c_float), _p(dd, ctypes.c_float),
                                  _p(r, ctypes.c_float), B, *outs)
        else:
            du, dv = (_f64(a).reshape(-1, 3) for a in adjacent)
            lib().orc_render_rays_adjacent(*self._args(), _p(self.occ, ctypes.c_uint32),
                                           _p(o, ctypes.c_float), _p(dd, ctypes.c_float),
                                           _p(r, ctypes.c_float), _p(du, ctypes.c_double),
                                           _p(dv, ctypes.c_double), B, *outs)
        out = dict(pq=pq, linear=lin, T=T, n=n, depth=depth)
        if normals:
            out["normal"] = nrm
        return out

    def render(self, c2w, K, res, threads=None, normals=False):
        o, dd, r = camera_rays(self.cfg, c2w, K, res)
        adj = camera_adjacent(c2w, K, res) if getattr(self.cfg, "contract", False) else None
        return self.render_rays(o, dd, r, threads, normals, adj)

    def density_grad(self, pos, radius):
        """sigma [n] and d sigma / d position [n][3] at a fixed footprint."""
        pos = _f32(pos).reshape(-1, 3)
        radius = _f64(np.broadcast_to(np.asarray(radius, np.float64), (pos.shape[0],)))
        n = pos.shape[0]
        sigma = np.zeros(n, np.float64)
        grad = np.zeros((n, 3), np.float64)
        lib().orc_density_grad(*self._args(), _p(pos, ctypes.c_float), _p(radius, ctypes.c_double),
                               n, _p(sigma, ctypes.c_double), _p(grad, ctypes.c_double))
        return sigma, grad

    def march(self, o, dd, cap):
        o, dd = _f32(o).reshape(-1, 3), _f32(dd).reshape(-1, 3)
        B = o.shape[0]
        rec_i = np.full((B, cap), -1, np.int32)
        rec_v = np.full((B, cap), -1, np.int32)
        cnt = np.zeros(B, np.int32)
        lib().orc_march(ctypes.byref(self.d), _p(self.occ, ctypes.c_uint32),
                        _p(o, ctypes.c_float), _p(dd, ctypes.c_float), B, cap,
                        _p(rec_i, ctypes.c_int32), _p(rec_v, ctypes.c_int32),
                        _p(cnt, ctypes.c_int32))
        return rec_i, rec_v, cnt

    def backward(self, o, dd, r, target_lin):
        o, dd, r = _f32(o).reshape(-1, 3), _f32(dd).reshape(-1, 3), _f32(r).reshape(-1)
        tgt = _f32(target_lin).reshape(-1, 3)
        B = o.shape[0]
        gg = np.zeros_like(self.grid)
        gm = np.zeros_like(self.mlp)
        loss = lib().orc_backward(*self._args(), _p(self.occ, ctypes.c_uint32),
                                  _p(o, ctypes.c_float), _p(dd, ctypes.c_float),
                                  _p(r, ctypes.c_float), _p(tgt, ctypes.c_float), B,
                                  _p(gg, ctypes.c_double), _p(gm, ctypes.c_double))
        return loss, gg, gm

    def backward_grad(self, o, dd, r, gC):
        """Gradients of sum_i gC_i . C_pq(ray i) for an upstream gradient gC [B][3]."""
        o, dd, r = _f32(o).reshape(-1, 3), _f32(dd).reshape(-1, 3), _f32(r).reshape(-1)
        g = _f64(gC).reshape(-1, 3)
        gg = np.zeros_like(self.grid)
        gm = np.zeros_like(self.mlp)
        lib().orc_backward_grad(*self._args(), _p(self.occ, ctypes.c_uint32), _p(o, ctypes.c_float),
                                _p(dd, ctypes.c_float), _p(r, ctypes.c_float), _p(g, ctypes.c_double),
                                o.shape[0], _p(gg, ctypes.c_double), _p(gm, ctypes.c_double))
        return gg, gm


def prune(F, cams, k, threshold, hist=None):
    """Joint grid / history pruning of F's occupancy (Sec. 4.3.2); returns
    (keep [rz][ry][rx] bool, alpha_grid [rz][ry][rx])."""
    cfg = F.cfg
    nvox = cfg.occ_res[0] * cfg.occ_res[1] * cfg.occ_res[2]
    keep = np.zeros(nvox, np.uint8)
    alpha = np.zeros(nvox, np.float64)
    cams = _f32(cams).reshape(-1, 3)
    h = None if hist is None else _f32(hist).reshape(-1)
    lib().orc_prune(ctypes.byref(F.d), _p(F.grid, ctypes.c_double), _p(F.mlp, ctypes.c_double),
                    _p(F.occ, ctypes.c_uint32), _p(cams, ctypes.c_float), cams.shape[0], int(k),
                    float(threshold), _p(h, ctypes.c_float), _p(keep, ctypes.c_uint8),
                    _p(alpha, ctypes.c_double))
    shape = tuple(cfg.occ_res[::-1])
    return keep.reshape(shape).astype(bool), alpha.reshape(shape)


def tonemap(pq, T=None, ev=0.0):
    """PQ colour [n][3] (and transmittance [n]) -> packed sRGB8 + coverage
    words [n] and the unrounded 255 s values [n][4] at exposure ev stops."""
    pq = _f64(pq).reshape(-1, 3)
    n = pq.shape[0]
    Tm = None if T is None else _f64(T).reshape(-1)
    rgba = np.zeros(n, np.uint32)
    pre = np.zeros((n, 4), np.float64)
    lib().orc_tonemap(_p(pq, ctypes.c_double), _p(Tm, ctypes.c_double), n, float(ev),
                      _p(rgba, ctypes.c_uint32), _p(pre, ctypes.c_double))
    return rgba, pre


def upsample_occupancy(values, factor):
    """Occupancy grid refined by an integer factor per axis (Sec. 4.3.2: the
    coarse grid is upsampled at training milestones): the voxel (x, y, z) of
    the fine grid takes the value of (x // factor, y // factor, z // factor).
    values: [rz][ry][rx] bits or per-voxel history."""
    v = np.asarray(values)
    for axis in range(3):
        v = np.repeat(v, factor, axis=axis)
    return v


def history(F, o, dd, r, hist=None):
    """Largest composited-sample opacity per voxel for explicit rays."""
    cfg = F.cfg
    nvox = cfg.occ_res[0] * cfg.occ_res[1] * cfg.occ_res[2]
    h = np.zeros(nvox, np.float32) if hist is None else _f32(hist).reshape(-1).copy()
    o, dd, r = _f32(o).reshape(-1, 3), _f32(dd).reshape(-1, 3), _f32(r).reshape(-1)
    lib().orc_history(ctypes.byref(F.d), _p(F.grid, ctypes.c_double), _p(F.mlp, ctypes.c_double),
                      _p(F.occ, ctypes.c_uint32), _p(o, ctypes.c_float), _p(dd, ctypes.c_float),
                      _p(r, ctypes.c_float), o.shape[0], _p(h, ctypes.c_float))
    return h


def adam(param, grad, m, v, t, lr, beta1=0.9, beta2=0.99, eps=1e-15):
    """In-place Adam step on float64 arrays."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(_p(param, ctypes.c_double), _p(grad, ctypes.c_double),
                   _p(m, ctypes.c_double), _p(v, ctypes.c_double), param.size, int(t),
                   float(lr), float(beta1), float(beta2), float(eps))
