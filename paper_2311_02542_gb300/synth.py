"""Seeded synthetic inputs for the VR-NeRF field renderer.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests. It draws random numbers and lays out scene geometry, camera
poses and parameter blobs. It contains none of the rendering method's
arithmetic: no ray generation, marching, hashing, level-of-detail, MLP,
compositing or PQ transform.

Random parameters come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014). The
library's seeded initialisation implements the same published generator, so a
field created from a seed holds exactly the blob that ``field_params`` returns.
Scene geometry (occupancy blobs, furniture, poses) uses numpy's Philox
generator and is only ever produced here.

The paper's datasets (Eyeful Tower, Sec. 3) are not available; these seeded
scenes stand in with the paper's shapes: rooms of tens of square metres, a
1.7 m eye height and 2K eye buffers (Sec. 5), hash grid L=16, F=2 (Sec. 6).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# ----------------------------------------------------------------------------
# SplitMix64 counter-based stream
# ----------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_STREAM_MUL = 0xD1B54A32D192ED03
_MASK64 = (1 << 64) - 1

# stream ids of the parameter blob
STREAM_GRID = 1
STREAM_W = (2, 3, 4, 5, 6)  # W1..W5


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (variant 13 of Stafford's mixers)."""
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    z = np.array([(int(seed) ^ ((int(stream) * _STREAM_MUL) & _MASK64)) & _MASK64],
                 dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(_mix(z)[0])


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws k = start .. start+count-1 of a stream as float64 in [0, 1).

    draw_k = mix(key + (k + 1) * gamma); u_k = (draw_k >> 40) * 2^-24.
    """
    key = np.uint64(stream_key(seed, stream))
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(key + k * _GAMMA)
    return (z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)


# ----------------------------------------------------------------------------
# Field configurations
# ----------------------------------------------------------------------------
@dataclass
class FieldConfig:
    """Hash grid + MLP + occupancy + sampling settings of one field.

    The MLP widths are the paper's (Sec. 6): density 1 hidden layer of 64 to
    16 outputs, colour 2 hidden layers of 64 to 3 outputs.
    """
    levels: int = 8
    feats: int = 2
    log2_T: int = 14
    feat_fp16: bool = False
    base_res: float = 16.0
    growth: float = 1.5
    d_hidden: int = 64
    d_out: int = 16
    c_hidden: int = 64
    c_layers: int = 2
    aabb_min: tuple = (0.0, 0.0, 0.0)
    aabb_max: tuple = (1.0, 1.0, 1.0)
    occ_res: tuple = (64, 64, 64)
    max_steps: int = 64
    t_near: float = 0.01
    t_far: float = math.sqrt(3.0)
    lod_bias: float = 0.0
    T_eps: float = 1e-4
    radius_scale: float = 0.5
    density_bias: float = 0.0
    feat_lo: float = -1e-2
    feat_hi: float = 1e-2
    contract: bool = False  # unbounded scene: L-infinity contraction around the box (Sec. 4)

    @property
    def d_in(self) -> int:
        return self.levels * self.feats

    @property
    def T(self) -> int:
        return 1 << self.log2_T

    def mlp_shapes(self):
        return [(self.d_hidden, self.d_in), (self.d_out, self.d_hidden),
                (self.c_hidden, self.d_out + 16), (self.c_hidden, self.c_hidden),
                (3, self.c_hidden)]

    def n_mlp(self) -> int:
        return sum(a * b for a, b in self.mlp_shapes())

    def as_dict(self):
        return asdict(self)


def cfg_unit_cube() -> FieldConfig:
    """64x64 render in a unit cube: L=8, T=2^14, F=2 fp32, s=16, f=1.5,
    occupancy 64^3, <=64 samples per ray."""
    return FieldConfig()


def cfg_room(surface: bool = False) -> FieldConfig:
    """20 m x 20 m x 3 m room: L=16, T=2^21, F=2 fp16, s=16 to finest 8192,
    occupancy 256^3, <=1024 samples per ray (Sec. 6: 1024 exponential samples).

    ``surface=True`` adds a constant density offset of ln(100) so that occupied
    voxels are close to opaque (sigma ~ 100 per metre), which makes rays stop
    at the first surface as in a trained walkable scene.
    """
    diag = math.sqrt(20.0 ** 2 + 20.0 ** 2 + 3.0 ** 2)
    return FieldConfig(levels=16, feats=2, log2_T=21, feat_fp16=True, base_res=16.0,
                       growth=math.exp(math.log(8192.0 / 16.0) / 15.0),
                       aabb_min=(0.0, 0.0, 0.0), aabb_max=(20.0, 20.0, 3.0),
                       occ_res=(256, 256, 256), max_steps=1024, t_near=0.05,
                       t_far=diag, density_bias=(math.log(100.0) if surface else 0.0))


def cfg_room_paper_grid(surface: bool = False) -> FieldConfig:
    """The room with the hash grid of the paper's experiments (Sec. 6): L=16
    levels of F=2 features, base resolution 128, growth 1.4 (every level
    hashed), here with T=2^19 slots per level and fp16 features."""
    c = cfg_room(surface)
    c.base_res, c.growth, c.log2_T = 128.0, 1.4, 19
    return c


def cfg_room_unbounded(surface: bool = False) -> FieldConfig:
    """The room of cfg_room with windows, inside an unbounded outdoor scene
    (Sec. 4: far field through the L-infinity contraction; most of the
    paper's scenes with views through windows use it, Table 5). Occupancy
    256^3 over the contracted cube [-2, 2]^3 around the room's centre (inner
    cube: 20 m wide), samples out to 4 km."""
    c = cfg_room(surface)
    c.contract = True
    c.t_far = 4000.0
    return c


# ----------------------------------------------------------------------------
# Parameter blob
# ----------------------------------------------------------------------------
def grid_params(cfg: FieldConfig, seed: int, chunk: int = 1 << 22) -> np.ndarray:
    """Hash-grid table [L][T][F]: U(feat_lo, feat_hi), rounded to fp32 and,
    for fp16 storage, then to fp16 (round to nearest even).

    Every level holds T slots; dense levels use the first (N+1)^3 of them.
    """
    n = cfg.levels * cfg.T * cfg.feats
    out = np.empty(n, dtype=np.float16 if cfg.feat_fp16 else np.float32)
    lo, hi = float(np.float32(cfg.feat_lo)), float(np.float32(cfg.feat_hi))
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        u = uniform01(seed, STREAM_GRID, s, c)
        v = (lo + (hi - lo) * u).astype(np.float32)
        out[s:s + c] = v.astype(out.dtype)
    return out.reshape(cfg.levels, cfg.T, cfg.feats)


def mlp_params(cfg: FieldConfig, seed: int) -> list:
    """W1..W5 as [out][in] fp32 arrays, Xavier-uniform: U(-b, b),
    b = sqrt(6 / (fan_in + fan_out)); no biases."""
    ws = []
    for sid, (fo, fi) in zip(STREAM_W, cfg.mlp_shapes()):
        b = math.sqrt(6.0 / (fi + fo))
        u = uniform01(seed, sid, 0, fo * fi)
        ws.append(((2.0 * u - 1.0) * b).astype(np.float32).reshape(fo, fi))
    return ws


def pack_mlp(ws) -> np.ndarray:
    return np.concatenate([w.reshape(-1) for w in ws]).astype(np.float32)


def unpack_mlp(cfg: FieldConfig, flat: np.ndarray) -> list:
    out, o = [], 0
    for fo, fi in cfg.mlp_shapes():
        out.append(np.asarray(flat[o:o + fo * fi], dtype=np.float32).reshape(fo, fi))
        o += fo * fi
    return out


# ----------------------------------------------------------------------------
# Occupancy grids (bit-packed: voxel (x,y,z) -> i = x + rx*(y + ry*z),
# word i >> 5, bit i & 31)
# ----------------------------------------------------------------------------
def pack_bits(occ: np.ndarray) -> np.ndarray:
    """occ: bool [rz][ry][rx] -> uint32 words."""
    flat = np.ascontiguousarray(occ, dtype=bool).reshape(-1)
    pad = (-flat.size) % 32
    if pad:
        flat = np.concatenate([flat, np.zeros(pad, bool)])
    bits = flat.reshape(-1, 32).astype(np.uint64)
    w = (bits << np.arange(32, dtype=np.uint64)).sum(axis=1)
    return w.astype(np.uint32)


def unpack_bits(words: np.ndarray, res) -> np.ndarray:
    rx, ry, rz = res
    b = ((words[:, None].astype(np.uint64) >> np.arange(32, dtype=np.uint64)) & 1).astype(bool)
    return b.reshape(-1)[: rx * ry * rz].reshape(rz, ry, rx)


def occupancy_spheres(res=(64, 64, 64), target=0.10, seed=1) -> np.ndarray:
    """Seeded spheres (radius U(2, 8) voxels) added until >= target - 0.5 %."""
    rng = np.random.Generator(np.random.Philox(seed))
    rx, ry, rz = res
    occ = np.zeros((rz, ry, rx), bool)
    zz, yy, xx = np.meshgrid(np.arange(rz) + 0.5, np.arange(ry) + 0.5,
                             np.arange(rx) + 0.5, indexing="ij")
    while occ.mean() < target - 0.005:
        c = rng.uniform(0, 1, 3) * np.array([rx, ry, rz])
        r = rng.uniform(2.0, 8.0)
        occ |= (xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= r * r
    return occ


def occupancy_room(res=(256, 256, 256), aabb_max=(20.0, 20.0, 3.0), target=0.05,
                   seed=2, return_boxes=False):
    """Room shell (floor, ceiling and four walls, one voxel thick) plus seeded
    axis-aligned furniture boxes (0.3-2 m footprint, 0.4-2 m tall, standing on
    the floor) until >= target - 0.5 % of the voxels are occupied."""
    rng = np.random.Generator(np.random.Philox(seed))
    rx, ry, rz = res
    X, Y, Z = aabb_max
    occ = np.zeros((rz, ry, rx), bool)
    occ[0] = occ[-1] = True
    occ[:, 0, :] = occ[:, -1, :] = True
    occ[:, :, 0] = occ[:, :, -1] = True
    boxes = []
    while occ.mean() < target - 0.005:
        w, d = rng.uniform(0.3, 2.0, 2)
        h = rng.uniform(0.4, 2.0)
        x0 = rng.uniform(0.2, X - 0.2 - w)
        y0 = rng.uniform(0.2, Y - 0.2 - d)
        ix0, ix1 = int(x0 / X * rx), int(math.ceil((x0 + w) / X * rx))
        iy0, iy1 = int(y0 / Y * ry), int(math.ceil((y0 + d) / Y * ry))
        iz1 = int(math.ceil(h / Z * rz))
        occ[0:iz1, iy0:iy1, ix0:ix1] = True
        boxes.append((x0, y0, 0.0, x0 + w, y0 + d, h))
    return (occ, boxes) if return_boxes else occ


def _uncontract_np(y):
    m = np.maximum(np.abs(y).max(axis=-1, keepdims=True), 1.0)
    return y / (m * (2.0 - np.minimum(m, 2.0 - 1e-9)))


def unbounded_boxes(cfg: FieldConfig, seed=2, furniture=40, buildings=60):
    """World-space boxes (lo, hi) of the unbounded room: ground (z <= 0
    everywhere), the room's walls (0.2 m thick, windows 1.4 m tall at 0.9 m
    on every wall), its ceiling, seeded furniture, and seeded buildings 40 m
    to 1.5 km away (8-40 m footprint, 5-80 m tall)."""
    rng = np.random.Generator(np.random.Philox(seed + 7000))
    X, Y, Z = cfg.aabb_max
    big = 1e7
    boxes = [((-big, -big, -1.0), (big, big, 0.0)),           # ground / floor
             ((-0.2, -0.2, Z), (X + 0.2, Y + 0.2, Z + 0.2))]  # ceiling
    win_lo, win_hi = 0.9, 2.3
    spans = [(0.0, 3.0), (7.0, 9.0), (11.0, 13.0), (17.0, 20.0)]  # wall between windows
    for wall in range(4):
        # full-height pieces between windows, sill and lintel pieces under / over them
        pieces = [(a, b, 0.0, Z) for a, b in spans]
        for a, b in ((3.0, 7.0), (9.0, 11.0), (13.0, 17.0)):
            pieces += [(a, b, 0.0, win_lo), (a, b, win_hi, Z)]
        for a, b, z0, z1 in pieces:
            if wall == 0:
                boxes.append(((-0.2, a, z0), (0.0, b, z1)))
            elif wall == 1:
                boxes.append(((X, a, z0), (X + 0.2, b, z1)))
            elif wall == 2:
                boxes.append(((a, -0.2, z0), (b, 0.0, z1)))
            else:
                boxes.append(((a, Y, z0), (b, Y + 0.2, z1)))
    for _ in range(furniture):
        w, d = rng.uniform(0.3, 2.0, 2)
        h = rng.uniform(0.4, 2.0)
        x0 = rng.uniform(0.2, X - 0.2 - w)
        y0 = rng.uniform(0.2, Y - 0.2 - d)
        boxes.append(((x0, y0, 0.0), (x0 + w, y0 + d, h)))
    for _ in range(buildings):
        dist = math.exp(rng.uniform(math.log(40.0), math.log(1500.0)))
        ang = rng.uniform(0, 2 * math.pi)
        w, d = rng.uniform(8.0, 40.0, 2)
        h = rng.uniform(5.0, 80.0)
        cx, cy = X / 2 + dist * math.cos(ang), Y / 2 + dist * math.sin(ang)
        boxes.append(((cx - w / 2, cy - d / 2, 0.0), (cx + w / 2, cy + d / 2, h)))
    return boxes


def occupancy_unbounded(cfg: FieldConfig, seed=2, build_res=128):
    """Contracted-grid occupancy of unbounded_boxes: a voxel of a
    build_res^3 grid over [-2, 2]^3 is occupied when the bounding box of its
    corners' pre-images overlaps a box; then repeated up to cfg.occ_res."""
    boxes = unbounded_boxes(cfg, seed)
    lo_b = np.array([b[0] for b in boxes])
    hi_b = np.array([b[1] for b in boxes])
    cen = (np.array(cfg.aabb_min) + np.array(cfg.aabb_max)) / 2
    h = 0.5 * max(cfg.aabb_max[k] - cfg.aabb_min[k] for k in range(3))
    n = build_res
    e = 4.0 * np.arange(n + 1) / n - 2.0
    occ = np.zeros((n, n, n), bool)
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for z in range(n):
        corners = []
        for c in range(8):
            y = np.stack([e[xx + (c & 1)], e[yy + ((c >> 1) & 1)],
                          np.full(xx.shape, e[z + ((c >> 2) & 1)])], axis=-1)
            y = np.clip(y, -2.0 + 1e-9, 2.0 - 1e-9)
            corners.append(_uncontract_np(y) * h + cen)
        corners = np.stack(corners)
        vlo, vhi = corners.min(axis=0), corners.max(axis=0)     # [n][n][3]
        slo, shi = vlo.reshape(-1, 3).min(0), vhi.reshape(-1, 3).max(0)
        hit = np.zeros((n, n), bool)
        for blo, bhi in zip(lo_b, hi_b):
            if (blo > shi).any() or (bhi < slo).any():
                continue
            hit |= ((vlo[..., 0] <= bhi[0]) & (vhi[..., 0] >= blo[0]) & (vlo[..., 1] <= bhi[1]) &
                    (vhi[..., 1] >= blo[1]) & (vlo[..., 2] <= bhi[2]) & (vhi[..., 2] >= blo[2]))
        occ[z] = hit
    f = [cfg.occ_res[k] // n for k in range(3)]
    return occ.repeat(f[2], 0).repeat(f[1], 1).repeat(f[0], 2)


# ----------------------------------------------------------------------------
# Cameras: c2w [3][4] fp32 (columns: right, down, forward, centre; OpenCV
# convention, the camera looks down +z of its own frame), intrinsics
# (fx, fy, cx, cy) fp32, resolution (W, H) int32.
# ----------------------------------------------------------------------------
def pose_from_angles(centre, yaw, pitch=0.0, roll=0.0) -> np.ndarray:
    """World frame z-up. forward = (cos p cos y, cos p sin y, sin p)."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([cp * cy_, cp * sy_, sp])
    right = np.array([sy_, -cy_, 0.0])
    down = np.cross(fwd, right)
    cr, sr = math.cos(roll), math.sin(roll)
    r2 = cr * right + sr * down
    d2 = -sr * right + cr * down
    m = np.zeros((3, 4), np.float64)
    m[:, 0], m[:, 1], m[:, 2], m[:, 3] = r2, d2, fwd, centre
    return m.astype(np.float32)


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation (Shoemake's quaternion method)."""
    u1, u2, u3 = rng.uniform(0, 1, 3)
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def intrinsics_fov(width, height, fov_deg=90.0) -> np.ndarray:
    f = 0.5 * width / math.tan(math.radians(fov_deg) * 0.5)
    return np.array([f, f, 0.5 * width, 0.5 * height], np.float32)


def _free_at(occ, cfg: FieldConfig, p) -> bool:
    rx, ry, rz = cfg.occ_res
    if getattr(cfg, "contract", False):
        cen = [(cfg.aabb_min[k] + cfg.aabb_max[k]) / 2 for k in range(3)]
        h = 0.5 * max(cfg.aabb_max[k] - cfg.aabb_min[k] for k in range(3))
        x = np.array([(p[k] - cen[k]) / h for k in range(3)])
        m = np.abs(x).max()
        y = x if m <= 1 else (2 - 1 / m) * x / m
        g = [(y[k] + 2) / 4 * cfg.occ_res[k] for k in range(3)]
    else:
        g = [(p[k] - cfg.aabb_min[k]) / (cfg.aabb_max[k] - cfg.aabb_min[k]) * cfg.occ_res[k]
             for k in range(3)]
    i = [int(math.floor(v)) for v in g]
    if any(i[k] < 0 or i[k] >= cfg.occ_res[k] for k in range(3)):
        return False
    return not occ[i[2], i[1], i[0]]


def camera_unit_cube(occ, cfg: FieldConfig, seed=1, width=64, height=64, fov=90.0):
    """One camera at a random free voxel with a uniformly random orientation."""
    rng = np.random.Generator(np.random.Philox(seed + 1000))
    while True:
        p = rng.uniform(0.1, 0.9, 3)
        if _free_at(occ, cfg, p):
            break
    m = np.zeros((3, 4), np.float64)
    m[:, :3] = random_rotation(rng)
    m[:, 3] = p
    return (m.astype(np.float32)[None], intrinsics_fov(width, height, fov)[None],
            np.array([[width, height]], np.int32))


def room_position(occ, cfg: FieldConfig, rng, z=None):
    X, Y, Z = cfg.aabb_max
    while True:
        p = np.array([rng.uniform(0.5, X - 0.5), rng.uniform(0.5, Y - 0.5),
                      z if z is not None else rng.uniform(0.5, Z - 0.5)])
        if _free_at(occ, cfg, p):
            return p


def camera_room(occ, cfg: FieldConfig, seed=2, width=2048, height=2048, fov=90.0, n=1):
    """n cameras at 1.7 m eye height, random free (x, y), random yaw, pitch 0."""
    rng = np.random.Generator(np.random.Philox(seed + 2000))
    cams, intr, res = [], [], []
    for _ in range(n):
        p = room_position(occ, cfg, rng, z=1.7)
        cams.append(pose_from_angles(p, rng.uniform(0, 2 * math.pi)))
        intr.append(intrinsics_fov(width, height, fov))
        res.append((width, height))
    return np.stack(cams), np.stack(intr), np.array(res, np.int32)


def stereo_pair(c2w: np.ndarray, ipd: float = 0.063) -> np.ndarray:
    """Left/right eye poses: the centre moves by -/+ ipd/2 along the right axis."""
    out = np.stack([c2w.copy(), c2w.copy()])
    right = c2w[:, 0].astype(np.float64)
    out[0, :, 3] = (c2w[:, 3] - 0.5 * ipd * right).astype(np.float32)
    out[1, :, 3] = (c2w[:, 3] + 0.5 * ipd * right).astype(np.float32)
    return out


def crop_camera(intr: np.ndarray, x0: int, y0: int) -> np.ndarray:
    """Intrinsics of a window whose top-left pixel is (x0, y0) of the full image."""
    out = np.array(intr, np.float32).copy()
    out[..., 2] -= np.float32(x0)
    out[..., 3] -= np.float32(y0)
    return out


# ----------------------------------------------------------------------------
# Serving requests: 70 % stereo pairs of 2048^2 eyes, 30 % single views with a
# side uniform in {512, 1024, 1536}, Poisson arrivals, 6-DoF poses in the room.
# ----------------------------------------------------------------------------
@dataclass
class Request:
    arrival_s: float
    c2w: np.ndarray           # [n][3][4]
    intrinsics: np.ndarray    # [n][4]
    resolution: np.ndarray    # [n][2]
    stereo: bool = False

    @property
    def rays(self) -> int:
        return int(np.prod(self.resolution, axis=1).sum())


def request_stream(occ, cfg: FieldConfig, n: int, seed=4, rate_hz=36.0 / 0.7,
                   stereo_frac=0.7, eye=2048, singles=(512, 1024, 1536)):
    rng = np.random.Generator(np.random.Philox(seed + 4000))
    t = 0.0
    out = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate_hz)
        p = room_position(occ, cfg, rng)
        pose = pose_from_angles(p, rng.uniform(0, 2 * math.pi),
                                math.radians(rng.uniform(-30, 30)),
                                math.radians(rng.uniform(-30, 30)))
        if rng.uniform() < stereo_frac:
            c = stereo_pair(pose)
            i = np.stack([intrinsics_fov(eye, eye)] * 2)
            r = np.array([[eye, eye]] * 2, np.int32)
            out.append(Request(t, c, i, r, True))
        else:
            s = int(rng.choice(singles))
            out.append(Request(t, pose[None], intrinsics_fov(s, s)[None],
                               np.array([[s, s]], np.int32), False))
    return out


# ----------------------------------------------------------------------------
# Training batches: rays from 64 synthetic views, HDR targets log-uniform in
# [1e-3, 1e3] linear units (1.0 = 100 cd/m^2).
# ----------------------------------------------------------------------------
def training_views(occ, cfg: FieldConfig, n_views=64, seed=5, size=256):
    rng = np.random.Generator(np.random.Philox(seed + 5000))
    poses = [pose_from_angles(room_position(occ, cfg, rng, z=rng.uniform(1.0, 2.2)),
                              rng.uniform(0, 2 * math.pi), math.radians(rng.uniform(-20, 20)))
             for _ in range(n_views)]
    return np.stack(poses), intrinsics_fov(size, size)


def training_batch(poses: np.ndarray, intr: np.ndarray, n_rays: int, seed=5, step=0):
    """Rays drawn uniformly over views and over each view's 90 degree frustum.

    Directions are normalised here (input preparation); the radius is the
    view's pixel half-pitch at unit distance, 0.5 / fx.
    """
    rng = np.random.Generator(np.random.Philox(seed * 1000003 + step))
    k = rng.integers(0, poses.shape[0], n_rays)
    u = rng.uniform(-1.0, 1.0, (n_rays, 2))
    P = poses[k].astype(np.float64)
    d = P[:, :, 2] + u[:, :1] * P[:, :, 0] + u[:, 1:] * P[:, :, 1]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = P[:, :, 3]
    r = np.full(n_rays, 0.5 / float(intr[0]), np.float32)
    target = np.exp(rng.uniform(math.log(1e-3), math.log(1e3), (n_rays, 3)))
    return (o.astype(np.float32), d.astype(np.float32), r, target.astype(np.float32))


# ----------------------------------------------------------------------------
# Convenience bundles
# ----------------------------------------------------------------------------
@dataclass
class Scene:
    cfg: FieldConfig
    grid: np.ndarray
    mlp: np.ndarray
    occ: np.ndarray          # bool [rz][ry][rx]
    occ_bits: np.ndarray     # uint32
    seed: int = 0
    extra: dict = field(default_factory=dict)


def make_scene(name: str, seed: int | None = None, with_params: bool = True) -> Scene:
    if name == "unit_cube":
        cfg, s = cfg_unit_cube(), 1 if seed is None else seed
        occ = occupancy_spheres(cfg.occ_res, 0.10, s)
    elif name in ("room", "room_surface"):
        cfg, s = cfg_room(surface=(name == "room_surface")), 2 if seed is None else seed
        occ = occupancy_room(cfg.occ_res, cfg.aabb_max, 0.05, s)
    elif name == "room_paper_grid":
        cfg, s = cfg_room_paper_grid(), 2 if seed is None else seed
        occ = occupancy_room(cfg.occ_res, cfg.aabb_max, 0.05, s)
    elif name in ("room_unbounded", "room_unbounded_surface"):
        cfg, s = cfg_room_unbounded(surface=name.endswith("surface")), 2 if seed is None else seed
        occ = occupancy_unbounded(cfg, s)
    else:
        raise ValueError(name)
    grid = grid_params(cfg, s) if with_params else None
    mlp = pack_mlp(mlp_params(cfg, s)) if with_params else None
    return Scene(cfg, grid, mlp, occ, pack_bits(occ), s)
