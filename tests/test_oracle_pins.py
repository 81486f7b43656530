"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
anchor values, hand-worked cases, closed forms, invariants and brute force on
tiny inputs. None of these needs a GPU.
"""
import math
import os
from dataclasses import replace

import numpy as np
import pytest

import oracle as O
from paper_2311_02542_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ----------------------------------------------------------------------------
# PQ (Sec. 4.1, Eq. 1-2)
# ----------------------------------------------------------------------------
def test_pq_anchor_values():
    for lum, pq in _rows("pq_anchors.txt"):
        assert abs(O.pq_encode(float(lum) / 10000.0) - float(pq)) < 1e-4, lum


def test_pq_full_scale_is_exactly_one():
    # c1 + c2 = 1 + c3 = 2520/128, so PQ(1) is exactly 1
    assert O.pq_encode(1.0) == 1.0
    assert O.pq_decode(1.0) == pytest.approx(1.0, abs=1e-15)


def test_pq_round_trip_and_monotone():
    Y = np.logspace(-7, 0, 400)
    E = np.array([O.pq_encode(y) for y in Y])
    back = np.array([O.pq_decode(e) for e in E])
    assert np.max(np.abs(back - Y) / Y) < 1e-9
    assert np.all(np.diff(E) > 0)


def test_pq_clamps_and_zero():
    assert O.pq_decode(-0.25) == 0.0
    assert O.pq_decode(0.0) == 0.0
    assert O.pq_decode(1.5) == pytest.approx(1.0)
    assert O.pq_encode(2.0) == 1.0
    # 1.0 linear is 100 cd/m^2 (Sec. 4.1)
    assert O.linear_to_pq(1.0) == pytest.approx(O.pq_encode(0.01), rel=1e-15)
    assert O.pq_to_linear(O.linear_to_pq(3.7)) == pytest.approx(3.7, rel=1e-9)


# ----------------------------------------------------------------------------
# Level of detail (Sec. 4.2.1 Eq. 3, Sec. 4.2.2)
# ----------------------------------------------------------------------------
def test_lod_weights_hand_cases():
    for row in _rows("lod_eq3_cases.txt"):
        Ls, n = float(row[0]), int(row[1])
        want = np.array([float(x) for x in row[2:]])
        np.testing.assert_allclose(O.lod_weights(Ls, n), want, atol=1e-12, err_msg=str(Ls))


def test_lod_weight_sum_rule():
    rng = np.random.default_rng(0)
    for Ls in rng.uniform(-3, 20, 500):
        w = O.lod_weights(Ls, 16)
        assert w.sum() == pytest.approx(min(max(Ls + 1.0, 0.0), 16.0), abs=1e-12)
        assert np.all(np.diff(w) <= 0)
        assert np.all((w >= 0) & (w <= 1))


def test_lod_level_closed_form():
    # f = 2: a footprint of 2^-k / (2 s) puts the Nyquist level at exactly k
    cfg = replace(S.cfg_unit_cube(), growth=2.0)
    for k in range(0, 8):
        assert O.lod_level(cfg, 2.0 ** -k / (2 * cfg.base_res)) == pytest.approx(k, abs=1e-12)
    cfg = S.cfg_unit_cube()  # f = 1.5
    assert O.lod_level(cfg, 1.5 ** -3 / (2 * 16)) == pytest.approx(3.0, abs=1e-12)
    # LOD bias adds to L* (Sec. 4.2.2)
    cfgb = replace(cfg, lod_bias=-1.25)
    assert O.lod_level(cfgb, 1.5 ** -3 / 32) == pytest.approx(1.75, abs=1e-12)
    # a vanishing footprint resolves every level
    assert np.all(O.lod_weights(O.lod_level(cfg, 0.0), 8) == 1.0)


def test_level_resolutions_and_dense_rule():
    rows = {(r[0], r[1]): [int(x) for x in r[2:]] for r in _rows("level_res.txt")}
    for name, cfg in (("unit_cube", S.cfg_unit_cube()), ("room", S.cfg_room()),
                      ("room_paper_grid", S.cfg_room_paper_grid())):
        N, dense, _, _ = O.geometry(cfg)
        assert list(N) == rows[(name, "N")]
        assert list(dense.astype(int)) == rows[(name, "dense")]


# ----------------------------------------------------------------------------
# Sample distances and rays
# ----------------------------------------------------------------------------
def test_sample_table_exponential():
    for cfg in (S.cfg_unit_cube(), S.cfg_room()):
        t = O.sample_table(cfg).astype(np.float64)
        assert t[0] == np.float32(cfg.t_near)
        assert t[-1] == pytest.approx(float(np.float32(cfg.t_far)), rel=2e-7)
        ratio = t[1:] / t[:-1]
        q = (cfg.t_far / cfg.t_near) ** (1.0 / cfg.max_steps)
        assert np.max(np.abs(ratio - q)) < 1e-5
        assert np.all(np.diff(t) > 0)


def test_ray_principal_axis_and_corner_angle():
    rng = np.random.Generator(np.random.Philox(3))
    R = S.random_rotation(rng)
    c2w = np.zeros((3, 4), np.float32)
    c2w[:, :3] = R
    c2w[:, 3] = (0.1, 0.2, 0.3)
    K = np.array([1.5, 1.5, 1.5, 1.5], np.float32)  # 3x3 image, fov 90 degrees
    o, d = O.ray(c2w, K, 1, 1)
    np.testing.assert_allclose(d, R[:, 2], atol=2e-7)
    np.testing.assert_array_equal(o, c2w[:, 3])
    o, d = O.ray(c2w, K, 0, 0)  # pixel centre at (-1, -1)/1.5 in the image plane
    x = y = (0.5 - 1.5) / 1.5
    assert np.linalg.norm(d) == pytest.approx(1.0, abs=3e-7)
    assert float(d @ R[:, 2]) == pytest.approx(1.0 / math.sqrt(1 + x * x + y * y), abs=3e-7)
    assert float(d @ R[:, 0]) == pytest.approx(x / math.sqrt(1 + x * x + y * y), abs=3e-7)


# ----------------------------------------------------------------------------
# Hash-grid corners (brute force on tiny grids)
# ----------------------------------------------------------------------------
def _tiny(base_res, log2_T, levels=1):
    return replace(S.cfg_unit_cube(), levels=levels, base_res=float(base_res), growth=1.5,
                   log2_T=log2_T)


def test_dense_corners_bijection_brute_force():
    cfg = _tiny(3, 8)  # N = 3, (N+1)^3 = 64 <= 256: dense
    N, dense, _, _ = O.geometry(cfg)
    assert N[0] == 3 and dense[0]
    seen = set()
    for k in range(3):
        for j in range(3):
            for i in range(3):
                p = np.array([(i + 0.5) / 3, (j + 0.5) / 3, (k + 0.5) / 3], np.float32)
                idx, _ = O.corners(cfg, p)
                for b in range(8):
                    a, bb, c = i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)
                    # x-fastest enumeration of the 4^3 vertices
                    assert idx[0, 0, b] == a + 4 * bb + 16 * c
                    seen.add(int(idx[0, 0, b]))
    assert seen == set(range(64))


def test_hashed_corners_brute_force():
    cfg = _tiny(7, 6)  # N = 7, 8^3 = 512 > 64: hashed
    N, dense, _, _ = O.geometry(cfg)
    assert N[0] == 7 and not dense[0]
    for k in range(7):
        for j in range(7):
            for i in range(7):
                p = np.array([(i + 0.5) / 7, (j + 0.5) / 7, (k + 0.5) / 7], np.float32)
                idx, _ = O.corners(cfg, p)
                for b in range(8):
                    a, bb, c = i + (b & 1), j + ((b >> 1) & 1), k + ((b >> 2) & 1)
                    h = (a ^ (bb * 2654435761) ^ (c * 805459861)) % (1 << 32) % 64
                    assert idx[0, 0, b] == h
                    # pi_1 = 1: stepping x flips only the low bits of x itself
                    if b & 1:
                        assert int(idx[0, 0, b]) ^ int(idx[0, 0, b - 1]) == (a ^ (a - 1)) & 63


def test_hash_wraps_at_32_bits():
    cfg = replace(S.cfg_room(), levels=16)
    N, dense, _, _ = O.geometry(cfg)
    p = np.array([[19.99, 19.99, 2.99]], np.float32)
    idx, frac = O.corners(cfg, p)
    ph = (p[0] - np.float32(0)) * np.float32(1 / 20)
    c = np.floor(ph.astype(np.float32) * np.float32(N[15])).astype(np.int64)
    h = (int(c[0]) ^ (int(c[1]) * 2654435761) ^ (int(c[2]) * 805459861)) % (1 << 32) % (1 << 21)
    assert idx[0, 15, 0] == h
    assert (idx < (1 << 21)).all()


def test_trilinear_reproduces_linear_field():
    """Trilinear interpolation is exact for a field linear in the vertex
    coordinates, which pins frac, the corner weights and their order."""
    cfg = _tiny(5, 10)  # dense, 6^3 vertices
    occ = np.ones((1, 1, 1), bool)
    grid = np.zeros((1, cfg.T, 2))
    for c in range(6):
        for b in range(6):
            for a in range(6):
                grid[0, a + 6 * b + 36 * c] = (0.3 * a - 0.7 * b + 1.1 * c, 2.0)
    mlp = np.zeros(O.mlp_count(cfg))
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    rng = np.random.default_rng(1)
    pos = rng.uniform(0, 1, (200, 3)).astype(np.float32)
    dirs = np.tile([0, 0, 1.0], (200, 1))
    _, _, feat = F.query(pos, dirs, np.zeros(200))
    x = pos.astype(np.float64) * 5
    np.testing.assert_allclose(feat[:, 0], 0.3 * x[:, 0] - 0.7 * x[:, 1] + 1.1 * x[:, 2],
                               atol=1e-5)
    np.testing.assert_allclose(feat[:, 1], 2.0, atol=1e-12)


# ----------------------------------------------------------------------------
# Spherical harmonics (direction encoding)
# ----------------------------------------------------------------------------
def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    phis = np.arange(24) * (2 * math.pi / 24)
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        s = math.sqrt(1 - z * z)
        for ph in phis:
            y = O.sh16([s * math.cos(ph), s * math.sin(ph), z])
            G += w * (2 * math.pi / 24) * np.outer(y, y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_addition_theorem_and_phase():
    rng = np.random.default_rng(2)
    for _ in range(50):
        a, b = rng.normal(size=3), rng.normal(size=3)
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        ya, yb = O.sh16(a), O.sh16(b)
        for l in range(4):
            sl = slice(l * l, (l + 1) * (l + 1))
            Pl = np.polynomial.legendre.legval(a @ b, [0] * l + [1])
            assert ya[sl] @ yb[sl] == pytest.approx((2 * l + 1) / (4 * math.pi) * Pl, abs=1e-12)
    # Condon-Shortley phase: Y_{1,1}(x) = -sqrt(3 / 4 pi)
    assert O.sh16([1.0, 0, 0])[3] == pytest.approx(-math.sqrt(3 / (4 * math.pi)))
    assert O.sh16([0, 1.0, 0])[1] == pytest.approx(-math.sqrt(3 / (4 * math.pi)))


# ----------------------------------------------------------------------------
# MLPs (Sec. 6) with hand-set weights and against an independent matmul
# ----------------------------------------------------------------------------
def _const_field(cfg, value, mlp, occ=None):
    grid = np.full((cfg.levels, cfg.T, cfg.feats), value, np.float64)
    occ = np.ones(tuple(cfg.occ_res[::-1]), bool) if occ is None else occ
    return O.Field(cfg, grid, mlp, S.pack_bits(occ))


def _mlp_views(cfg, flat):
    out, o = [], 0
    for fo, fi in cfg.mlp_shapes():
        out.append(flat[o:o + fo * fi].reshape(fo, fi))
        o += fo * fi
    return out


def test_mlp_hand_set_weights():
    cfg = S.cfg_unit_cube()
    mlp = np.zeros(O.mlp_count(cfg))
    W1, W2, W3, W4, W5 = _mlp_views(cfg, mlp)
    a, k = 0.02, 60.0
    W1[0, 0] = 1.0          # h_0 = relu(feature 0 of level 0) = a
    W2[0, 0] = k            # o_0 = k a -> sigma = exp(k a)
    W3[0, 16] = 1.0         # h1_0 = relu(SH_0) = 1 / (2 sqrt(pi))
    W4[0, 0] = 1.0          # h2_0 = h1_0
    W5[:, 0] = (1.0, -2.0, 3.0)
    F = _const_field(cfg, a, mlp)
    sig, rgb, feat = F.query(np.array([[0.3, 0.4, 0.5]], np.float32), [[0.0, 0.6, 0.8]], [0.0])
    assert sig[0] == pytest.approx(math.exp(k * a), rel=1e-12)
    y0 = 0.5 / math.sqrt(math.pi)
    want = 1.0 / (1.0 + np.exp(-np.array([1.0, -2.0, 3.0]) * y0))
    np.testing.assert_allclose(rgb[0], want, rtol=1e-12)
    np.testing.assert_allclose(feat[0], a, rtol=1e-12)
    # all-zero weights: sigma = exp(0) = 1, colour = sigmoid(0) = 1/2 exactly
    F0 = _const_field(cfg, a, np.zeros(O.mlp_count(cfg)))
    sig, rgb, _ = F0.query(np.array([[0.3, 0.4, 0.5]], np.float32), [[0.0, 0.6, 0.8]], [0.0])
    assert sig[0] == 1.0 and np.all(rgb == 0.5)


def test_mlp_against_independent_matmul():
    cfg = S.cfg_unit_cube()
    sc = S.make_scene("unit_cube")
    F = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits)
    rng = np.random.default_rng(3)
    n = 64
    pos = rng.uniform(0.05, 0.95, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = rng.uniform(0, 3e-3, n)
    sig, rgb, feat = F.query(pos, d, rad)
    W1, W2, W3, W4, W5 = [w.astype(np.float64) for w in S.unpack_mlp(cfg, sc.mlp)]
    h = np.maximum(feat @ W1.T, 0)
    o = h @ W2.T
    sh = np.stack([O.sh16(x) for x in d])
    x = np.concatenate([o, sh], axis=1)
    h2 = np.maximum(np.maximum(x @ W3.T, 0) @ W4.T, 0)
    np.testing.assert_allclose(sig, np.exp(o[:, 0]), rtol=1e-12)
    np.testing.assert_allclose(rgb, 1 / (1 + np.exp(-(h2 @ W5.T))), rtol=1e-12)


# ----------------------------------------------------------------------------
# Compositing: closed forms and invariants
# ----------------------------------------------------------------------------
def _slab_exit(o, d, lo, hi):
    t = np.inf
    for k in range(3):
        if d[k] > 0:
            t = min(t, (hi[k] - o[k]) / d[k])
        elif d[k] < 0:
            t = min(t, (lo[k] - o[k]) / d[k])
    return t


def test_constant_density_closed_form():
    """All features 0 and no biases: sigma = exp(0) = 1; W5 = 0 gives c = 1/2.
    In a fully occupied cube C = 1/2 (1 - exp(-(t_n - t_0))), the sum of the
    deltas of the n samples inside telescoping."""
    cfg = S.cfg_unit_cube()
    rng = np.random.default_rng(4)
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.3
    _mlp_views(cfg, mlp)[4][:] = 0.0
    F = _const_field(cfg, 0.0, mlp)
    t = O.sample_table(cfg).astype(np.float64)
    checked = 0
    for _ in range(200):
        o = rng.uniform(0.2, 0.8, 3).astype(np.float32)
        d = rng.normal(size=3)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        te = _slab_exit(o.astype(np.float64), d.astype(np.float64), [0, 0, 0], [1, 1, 1])
        if np.min(np.abs(t - te)) < 1e-4:
            continue  # a sample on the boundary: rounding decides, skip
        n = int(np.sum(t[:-1] < te))
        out = F.render_rays(o[None], d[None], np.zeros(1, np.float32), threads=1)
        assert out["n"][0] == n
        np.testing.assert_allclose(out["pq"][0], 0.5 * (1 - math.exp(-(t[n] - t[0]))), rtol=1e-12)
        checked += 1
    assert checked > 150


def test_opaque_closed_form_and_early_termination():
    cfg = S.cfg_unit_cube()
    mlp = np.zeros(O.mlp_count(cfg))
    W1, W2, *_ = _mlp_views(cfg, mlp)
    a = 0.02
    W1[0, 0] = 1.0
    W2[0, 0] = math.log(200.0) / a  # sigma = 200 per unit
    F = _const_field(cfg, a, mlp)
    o = np.array([[0.5, 0.5, 0.5]], np.float32)
    d = np.array([[0.0, 0.0, 1.0]], np.float32)
    out = F.render_rays(o, d, np.zeros(1, np.float32), threads=1)
    t = O.sample_table(cfg).astype(np.float64)
    n = int(out["n"][0])
    T = math.exp(-200.0 * (t[n] - t[0]))
    assert out["T"][0] == pytest.approx(T, rel=1e-9)
    assert T < cfg.T_eps <= math.exp(-200.0 * (t[n - 1] - t[0]))
    np.testing.assert_allclose(out["pq"][0], 0.5 * (1 - T), rtol=1e-12)
    assert abs(out["pq"][0][0] - 0.5) <= 0.5 * cfg.T_eps


def test_weights_plus_transmittance_is_one_on_random_field():
    """With W5 = 0 every colour is 1/2, so C = (sum_i w_i) / 2 and the
    invariant sum_i w_i + T_final = 1 reads C = (1 - T) / 2 for every ray."""
    sc = S.make_scene("unit_cube")
    cfg = replace(sc.cfg, density_bias=2.5)
    mlp = sc.mlp.astype(np.float64).copy()
    _mlp_views(cfg, mlp)[4][:] = 0.0
    grid = sc.grid.astype(np.float64) * 300  # make sigma vary strongly
    F = O.Field(cfg, grid, mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, 32, 32)
    out = F.render(c2w, K, res)
    assert np.all((out["T"] >= 0) & (out["T"] <= 1))
    np.testing.assert_allclose(out["pq"], np.repeat((1 - out["T"])[:, None] / 2, 3, 1), atol=1e-13)
    assert out["n"].max() > 3 and out["T"].min() < 0.5


def test_early_termination_error_bound():
    sc = S.make_scene("unit_cube")
    cfg = replace(sc.cfg, density_bias=3.0)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg, 1, 32, 32)
    a = O.Field(cfg, sc.grid, sc.mlp, sc.occ_bits).render(c2w, K, res)
    b = O.Field(replace(cfg, T_eps=0.0), sc.grid, sc.mlp, sc.occ_bits).render(c2w, K, res)
    assert np.max(np.abs(a["pq"] - b["pq"])) <= cfg.T_eps
    assert (a["n"] < b["n"]).any()


def test_empty_grid_renders_black():
    sc = S.make_scene("unit_cube")
    occ = np.zeros_like(sc.occ)
    F = O.Field(sc.cfg, sc.grid, sc.mlp, S.pack_bits(occ))
    c2w, K, res = S.camera_unit_cube(sc.occ, sc.cfg, 1, 16, 16)
    out = F.render(c2w, K, res)
    assert np.all(out["pq"] == 0) and np.all(out["linear"] == 0)
    assert np.all(out["n"] == 0) and np.all(out["T"] == 1)


# ----------------------------------------------------------------------------
# Occupancy march (Sec. 4.3): brute force in fp64 away from voxel faces
# ----------------------------------------------------------------------------
def test_march_single_voxel_brute_force():
    cfg = replace(S.cfg_unit_cube(), occ_res=(8, 8, 8), max_steps=64)
    rng = np.random.default_rng(5)
    t = O.sample_table(cfg).astype(np.float64)
    checked = 0
    for trial in range(60):
        occ = np.zeros((8, 8, 8), bool)
        v = rng.integers(0, 8, 3)
        occ[v[2], v[1], v[0]] = True
        F = O.Field(cfg, np.zeros((cfg.levels, cfg.T, 2)), np.zeros(O.mlp_count(cfg)),
                    S.pack_bits(occ))
        o = rng.uniform(0.05, 0.95, (20, 3)).astype(np.float32)
        target = (v + 0.5) / 8
        d = target - o
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        d = d.astype(np.float32)
        rec_i, rec_v, cnt = F.march(o, d, 64)
        for r in range(20):
            P = o[r].astype(np.float64) + t[:-1, None] * d[r].astype(np.float64)
            G = P * 8
            if np.min(np.abs(G - np.round(G))) < 1e-4:
                continue
            inside = np.all((G >= 0) & (G < 8), axis=1)
            n_in = int(np.argmin(inside)) if not inside.all() else len(inside)
            vox = np.floor(G[:n_in]).astype(int)
            lin = vox[:, 0] + 8 * (vox[:, 1] + 8 * vox[:, 2])
            want = np.nonzero(lin == v[0] + 8 * (v[1] + 8 * v[2]))[0]
            assert cnt[r] == len(want)
            np.testing.assert_array_equal(rec_i[r, :cnt[r]], want)
            assert np.all(rec_v[r, :cnt[r]] == v[0] + 8 * (v[1] + 8 * v[2]))
            checked += 1
    assert checked > 500


# ----------------------------------------------------------------------------
# Backward (central finite differences, fp64) and Adam (closed form)
# ----------------------------------------------------------------------------
def test_backward_matches_finite_differences():
    """Central differences (fp64, step 1e-6) of the L1 loss on 1 000 randomly
    chosen parameters, 300 hash-grid entries touched by the batch and 700
    MLP weights, the count the training configuration names."""
    cfg = replace(S.cfg_unit_cube(), levels=4, log2_T=9, occ_res=(16, 16, 16), max_steps=48,
                  T_eps=0.0)
    rng = np.random.default_rng(6)
    grid = rng.uniform(-1, 1, (cfg.levels, cfg.T, cfg.feats))
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.4
    occ = rng.uniform(size=(16, 16, 16)) < 0.4
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    B = 6
    o = rng.uniform(0.3, 0.7, (B, 3)).astype(np.float32)
    d = rng.normal(size=(B, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r = np.full(B, 2e-3, np.float32)
    tgt = np.full((B, 3), 1e-3, np.float32)  # far below every rendered colour
    loss, gg, gm = F.backward(o, d, r, tgt)

    def loss_at(g, m):
        return O.Field(cfg, g, m, S.pack_bits(occ)).backward(o, d, r, tgt)[0]

    h = 1e-6
    touched = np.nonzero(gg.reshape(-1))[0]
    assert touched.size >= 300
    picks = [("g", i) for i in rng.choice(touched, 300, replace=False)]
    picks += [("m", i) for i in rng.choice(mlp.size, 700, replace=False)]
    bad = 0
    for kind, i in picks:
        g2, m2 = grid.reshape(-1).copy(), mlp.copy()
        arr = g2 if kind == "g" else m2
        arr[i] += h
        lp = loss_at(g2, m2)
        arr[i] -= 2 * h
        lm = loss_at(g2, m2)
        fd = (lp - lm) / (2 * h)
        an = (gg.reshape(-1) if kind == "g" else gm)[i]
        if abs(fd - an) > 1e-7 + 1e-4 * abs(an):
            bad += 1
    print("finite differences on", len(picks), "parameters:", bad, "outside the bound")
    assert bad <= 2, bad  # at most a ReLU kink crossed by the finite step


def test_backward_grad_matches_finite_differences():
    """Gradient of a random linear functional sum_i gC_i . C_pq(ray i) of the
    PQ colours (the upstream gradient of an arbitrary loss) against central
    differences of that functional through the fp64 render."""
    cfg = replace(S.cfg_unit_cube(), levels=4, log2_T=9, occ_res=(16, 16, 16), max_steps=48,
                  T_eps=0.0)
    rng = np.random.default_rng(16)
    grid = rng.uniform(-1, 1, (cfg.levels, cfg.T, cfg.feats))
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.4
    occ = rng.uniform(size=(16, 16, 16)) < 0.4
    F = O.Field(cfg, grid, mlp, S.pack_bits(occ))
    B = 6
    o = rng.uniform(0.3, 0.7, (B, 3)).astype(np.float32)
    d = rng.normal(size=(B, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r = np.full(B, 2e-3, np.float32)
    gC = rng.normal(size=(B, 3))
    gg, gm = F.backward_grad(o, d, r, gC)

    def functional(g, m):
        return float((O.Field(cfg, g, m, S.pack_bits(occ)).render_rays(o, d, r, threads=1)["pq"] * gC).sum())

    h = 1e-6
    touched = np.nonzero(gg.reshape(-1))[0]
    picks = [("g", i) for i in rng.choice(touched, 40, replace=False)]
    picks += [("m", i) for i in rng.choice(mlp.size, 100, replace=False)]
    bad = 0
    for kind, i in picks:
        g2, m2 = grid.reshape(-1).copy(), mlp.copy()
        arr = g2 if kind == "g" else m2
        arr[i] += h
        fp = functional(g2, m2)
        arr[i] -= 2 * h
        fm = functional(g2, m2)
        fd = (fp - fm) / (2 * h)
        an = (gg.reshape(-1) if kind == "g" else gm)[i]
        if abs(fd - an) > 1e-7 + 1e-4 * abs(an):
            bad += 1
    assert bad <= 2, bad  # at most a ReLU kink crossed by the finite step
    # with the L1 loss's upstream gradient it is the fused L1 backward
    tgt = np.full((B, 3), 1e-3, np.float32)
    C = F.render_rays(o, d, r, threads=1)["pq"]
    g1 = np.sign(C - np.array([O.linear_to_pq(1e-3)] * 3)) / (3 * B)
    _, ga, ma = F.backward(o, d, r, tgt)
    gb, mb = F.backward_grad(o, d, r, g1)
    np.testing.assert_allclose(gb, ga, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(mb, ma, rtol=1e-12, atol=1e-15)


def test_adam_closed_form():
    g1 = np.array([0.5, -2e-3, 0.0, 7.0])
    g2 = np.array([-0.25, 4e-3, 1.0, 7.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m, v = np.zeros(4), np.zeros(4)
    lr, eps = 0.01, 1e-15
    O.adam(p, g1, m, v, 1, lr)
    # first step: m_hat = g, v_hat = g^2, step = lr g / (|g| + eps)
    want1 = np.array([1.0, 2.0, 3.0, 4.0]) - lr * g1 / (np.abs(g1) + eps)
    np.testing.assert_allclose(p, want1, rtol=0, atol=1e-15)
    O.adam(p, g2, m, v, 2, lr)
    mm = 0.9 * 0.1 * g1 + 0.1 * g2
    vv = 0.99 * 0.01 * g1 ** 2 + 0.01 * g2 ** 2
    want2 = want1 - lr * (mm / (1 - 0.81)) / (np.sqrt(vv / (1 - 0.9801)) + eps)
    np.testing.assert_allclose(p, want2, rtol=0, atol=1e-14)


def test_depth_opaque_first_sample_and_bounds():
    """Expected depth sum_i w_i t_i: a sample that absorbs (all but e^-200 of)
    the light puts the depth at its own distance; in general the depth lies
    between (1 - T) t_first and (1 - T) t_last of the composited samples."""
    cfg = replace(S.cfg_unit_cube(), T_eps=0.0)
    mlp = np.zeros(O.mlp_count(cfg))
    W1, W2, *_ = _mlp_views(cfg, mlp)
    a = 0.02
    W1[0, 0] = 1.0
    W2[0, 0] = math.log(1e7) / a  # sigma = 1e7 per unit: one sample is opaque
    occ = np.zeros((64, 64, 64), bool)
    occ[:, :, 40:] = True         # slab x >= 40/64
    F = _const_field(cfg, a, mlp, occ)
    o = np.array([[0.1, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    out = F.render_rays(o, d, np.zeros(1, np.float32), threads=1)
    rec_i, _, cnt = F.march(o, d, 64)
    t = O.sample_table(cfg).astype(np.float64)
    assert out["depth"][0] == pytest.approx(t[rec_i[0, 0]], rel=1e-12)
    sc = S.make_scene("unit_cube")
    cfg2 = replace(sc.cfg, density_bias=3.0)
    F2 = O.Field(cfg2, sc.grid, sc.mlp, sc.occ_bits)
    c2w, K, res = S.camera_unit_cube(sc.occ, cfg2, 1, 24, 24)
    o, dd, r = O.camera_rays(cfg2, c2w, K, res)
    out = F2.render_rays(o, dd, r)
    rec_i, _, cnt = F2.march(o, dd, 64)
    for k in np.nonzero(out["n"] > 1)[0][:200]:
        ti = t[rec_i[k, :out["n"][k]]]
        op = 1.0 - out["T"][k]
        assert op * ti[0] - 1e-12 <= out["depth"][k] <= op * ti[-1] + 1e-12


# ----------------------------------------------------------------------------
# Occupancy pruning (Sec. 4.3.2)
# ----------------------------------------------------------------------------
def _small_field(seed=3):
    cfg = replace(S.cfg_unit_cube(), occ_res=(16, 16, 16), levels=8)
    rng = np.random.default_rng(seed)
    occ = rng.uniform(size=(16, 16, 16)) < 0.3
    grid = rng.uniform(-1, 1, (cfg.levels, cfg.T, cfg.feats))
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.5
    return cfg, occ, O.Field(cfg, grid, mlp, S.pack_bits(occ))


def test_prune_threshold_limits_and_monotone():
    cfg, occ, F = _small_field()
    cams = np.array([[0.5, 0.5, 0.5], [0.1, 0.9, 0.2]], np.float32)
    keep0, alpha = O.prune(F, cams, 2, 0.0)
    assert (keep0 == occ).all()
    keep_hi, _ = O.prune(F, cams, 2, 1.5)
    assert not keep_hi.any()
    prev = occ.sum()
    for thr in np.quantile(alpha[occ], [0.1, 0.3, 0.5, 0.7, 0.9]):
        keep, _ = O.prune(F, cams, 2, thr)
        assert keep.sum() <= prev and not (keep & ~occ).any()
        assert (keep == (occ & (alpha >= thr))).all()
        prev = keep.sum()
    # history keeps a voxel the grid part would prune
    thr = np.quantile(alpha[occ], 0.9)
    keep, _ = O.prune(F, cams, 2, thr)
    v = np.argwhere(occ & ~keep)[0]
    hist = np.zeros(occ.shape, np.float32)
    hist[tuple(v)] = 1.0
    keep_h, _ = O.prune(F, cams, 2, thr, hist)
    assert keep_h[tuple(v)] and keep_h.sum() == keep.sum() + 1


def test_prune_constant_density_brute_force():
    """All-zero parameters: sigma = exp(density_bias) everywhere, so the grid
    opacity is 1 - exp(-sigma delta(t_min)), t_min the distance from the
    nearest camera to the voxel box and delta the spacing of the sample
    interval holding it (found here by brute force)."""
    cfg = replace(S.cfg_unit_cube(), occ_res=(8, 8, 8), levels=8, density_bias=2.0)
    occ = np.ones((8, 8, 8), bool)
    F = O.Field(cfg, np.zeros((cfg.levels, cfg.T, 2)), np.zeros(O.mlp_count(cfg)), S.pack_bits(occ))
    cams = np.array([[0.3, 0.6, 0.45]], np.float32)
    _, alpha = O.prune(F, cams, 3, 0.0)
    t = O.sample_table(cfg).astype(np.float64)
    sig = np.exp(2.0)
    for vz in range(8):
        for vy in range(8):
            for vx in range(8):
                lo = np.array([vx, vy, vz]) / 8.0
                hi = lo + 1 / 8.0
                c = cams[0].astype(np.float64)
                dist = np.linalg.norm(np.maximum(0, np.maximum(lo - c, c - hi)))
                i = max(0, min(int(np.searchsorted(t, dist, side="right")) - 1, cfg.max_steps - 1))
                want = 1 - np.exp(-sig * (t[i + 1] - t[i]))
                assert alpha[vz, vy, vx] == pytest.approx(want, rel=1e-12)


def test_history_matches_march_records():
    """Constant density: every composited sample's opacity is
    1 - exp(-sigma delta_i), so each voxel's history is the largest of those
    over the samples the march records in it."""
    cfg = replace(S.cfg_unit_cube(), occ_res=(16, 16, 16), density_bias=0.5, T_eps=0.0)
    rng = np.random.default_rng(4)
    occ = rng.uniform(size=(16, 16, 16)) < 0.3
    F = O.Field(cfg, np.zeros((cfg.levels, cfg.T, 2)), np.zeros(O.mlp_count(cfg)), S.pack_bits(occ))
    o = rng.uniform(0.2, 0.8, (50, 3)).astype(np.float32)
    d = rng.normal(size=(50, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r = np.zeros(50, np.float32)
    h = O.history(F, o, d, r)
    rec_i, rec_v, cnt = F.march(o, d, 64)
    t = O.sample_table(cfg).astype(np.float64)
    want = np.zeros(16 ** 3)
    for b in range(50):
        for k in range(cnt[b]):
            i, v = rec_i[b, k], rec_v[b, k]
            want[v] = max(want[v], 1 - np.exp(-np.exp(0.5) * (t[i + 1] - t[i])))
    np.testing.assert_allclose(h, want.astype(np.float32), rtol=1e-6, atol=0)


def test_upsample_occupancy_brute_force():
    rng = np.random.default_rng(2)
    occ = rng.uniform(size=(2, 3, 4)) < 0.5
    up = O.upsample_occupancy(occ, 3)
    assert up.shape == (6, 9, 12)
    for z in range(6):
        for y in range(9):
            for x in range(12):
                assert up[z, y, x] == occ[z // 3, y // 3, x // 3]


# ----------------------------------------------------------------------------
# Auxiliary outputs: density gradient / normals, display tonemapping
# ----------------------------------------------------------------------------
def test_density_grad_matches_central_differences():
    """Positive features; hidden units 0-31 have positive input weights (always
    active), 32-63 negative ones (never active), so log sigma = o_0 + bias is
    trilinear inside each cell of every level with no ReLU switch, and central
    differences of log sigma inside one cell of every level give
    grad sigma / sigma up to the fp32 rounding of the grid coordinates
    (~1e-5 of a finest cell against a 0.13-cell stencil). A dropped level,
    feature, ReLU mask or W2 term fails."""
    cfg = replace(S.cfg_unit_cube(), occ_res=(16, 16, 16), levels=8)
    rng = np.random.default_rng(8)
    grid = rng.uniform(0.1, 1.0, (cfg.levels, cfg.T, cfg.feats))
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.3
    W1 = np.abs(mlp[:64 * 16].reshape(64, 16))
    W1[32:] *= -1
    mlp[:64 * 16] = W1.reshape(-1)
    F = O.Field(cfg, grid, mlp, S.pack_bits(np.ones((16, 16, 16), bool)))
    n = 4000
    pos = rng.uniform(0.05, 0.95, (n, 3)).astype(np.float32)
    _, frac = O.corners(cfg, pos)
    inner = ((frac > 0.08) & (frac < 0.92)).reshape(n, -1).all(axis=1)
    radius = 1e-4
    sig, grad = F.density_grad(pos, radius)
    h = 2.0 ** -12
    idx = np.flatnonzero(inner)
    assert idx.size > 50, idx.size
    for i in idx:
        fd = np.zeros(3)
        for k in range(3):
            pp, pm = pos[i].copy(), pos[i].copy()
            pp[k] += h
            pm[k] -= h
            ls = np.log(F.density_grad(np.stack([pp, pm]), radius)[0])
            fd[k] = (ls[0] - ls[1]) / (float(pp[k]) - float(pm[k]))
        np.testing.assert_allclose(grad[i] / sig[i], fd, rtol=0, atol=2e-4 * np.abs(fd).max())


def _axis_field(density_bias):
    """Level 0 dense (N = 5) with feature 0 = the vertex's x coordinate / 5,
    the density MLP passes it through one ReLU: o_0 = p_x, so grad sigma
    points along +x and every normal is -x."""
    cfg = replace(_tiny(5, 10), occ_res=(8, 8, 8), density_bias=density_bias, T_eps=0.0)
    grid = np.zeros((1, cfg.T, 2))
    for c in range(6):
        for b in range(6):
            for a in range(6):
                grid[0, a + 6 * b + 36 * c] = (a / 5.0, 0.0)
    mlp = np.zeros(O.mlp_count(cfg))
    mlp[0] = 1.0            # W1[0][0]
    mlp[64 * 2 + 0] = 1.0   # W2[0][0]
    return cfg, O.Field(cfg, grid, mlp, S.pack_bits(np.ones((8, 8, 8), bool)))


def test_density_grad_closed_form_axis_field():
    cfg, F = _axis_field(1.0)
    pos = np.array([[0.3, 0.5, 0.5], [0.71, 0.2, 0.9]], np.float32)
    sig, grad = F.density_grad(pos, 0.0)
    np.testing.assert_allclose(sig, np.exp(pos[:, 0].astype(np.float64) + 1.0), rtol=1e-6)
    np.testing.assert_allclose(grad[:, 0], sig, rtol=1e-6)
    assert (grad[:, 1:] == 0).all()


def test_composited_normal_closed_form():
    """sum_i w_i n_i with n_i = -x for every sample: (-(1 - T), 0, 0)."""
    cfg, F = _axis_field(2.0)
    rng = np.random.default_rng(5)
    o = rng.uniform(0.3, 0.7, (40, 3)).astype(np.float32)
    d = rng.normal(size=(40, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    out = F.render_rays(o, d, np.zeros(40, np.float32), threads=1, normals=True)
    assert (out["n"] > 3).all()
    np.testing.assert_allclose(out["normal"][:, 0], -(1.0 - out["T"]), rtol=1e-9, atol=1e-12)
    assert (out["normal"][:, 1:] == 0).all()
    # normals do not change the rest of the render
    plain = F.render_rays(o, d, np.zeros(40, np.float32), threads=1)
    assert (plain["pq"] == out["pq"]).all() and (plain["T"] == out["T"]).all()


def test_tonemap_srgb_anchors_exposure_and_coverage():
    rows = [tuple(map(float, ln.split())) for ln in open(os.path.join(GOLDEN, "srgb_anchors.txt"))
            if ln.strip() and not ln.startswith("#")]
    v = np.array([r[0] for r in rows])
    s = np.array([r[1] for r in rows])
    pq = np.repeat(np.array([O.linear_to_pq(x) for x in v])[:, None], 3, axis=1)
    rgba, pre = O.tonemap(pq)
    np.testing.assert_allclose(pre[:, :3] / 255.0, s[:, None].repeat(3, 1), atol=2e-6)
    assert ((rgba >> 24) == 255).all()
    assert [int(x & 255) for x in rgba] == [int(np.floor(255 * x + 0.5)) for x in s]
    # +1 stop of exposure on half the luminance gives the same pixels
    pq_half = np.repeat(np.array([O.linear_to_pq(x / 2) for x in v])[:, None], 3, axis=1)
    rgba2, pre2 = O.tonemap(pq_half, ev=1.0)
    np.testing.assert_allclose(pre2, pre, rtol=1e-5)
    # over-exposure clamps to white, PQ 0 is black, coverage is 1 - T
    rgba3, _ = O.tonemap([[1.0, 0.0, 0.5]], T=[0.25], ev=0.0)
    assert int(rgba3[0]) & 255 == 255 and (int(rgba3[0]) >> 8) & 255 == 0
    assert int(rgba3[0]) >> 24 == int(np.floor(0.75 * 255 + 0.5))


# ----------------------------------------------------------------------------
# Unbounded scenes: L-infinity contraction (Sec. 4) and the contracted
# footprint (Sec. 4.2.1)
# ----------------------------------------------------------------------------
def _contracted_cfg(**kw):
    # unit box: centre 0.5, x = 2 (p - 0.5), so the inner cube is the box itself
    return replace(S.cfg_unit_cube(), contract=True, t_far=1000.0, max_steps=256, **kw)


def test_contraction_closed_forms():
    cfg = _contracted_cfg()
    x = np.array([[0.0, 0.0, 0.0], [0.5, -0.25, 1.0], [2.0, 0.0, 0.0], [-4.0, 1.0, 0.5],
                  [3.0, 1.5, 0.0], [0.0, 0.0, -1e4]])
    # (2 - 1/m) x / m beyond the inner cube, identity inside
    want = []
    for v in x:
        m = np.abs(v).max()
        want.append(v if m <= 1 else (2 - 1 / m) * v / m)
    want = np.array(want) / 4 + 0.5
    ph = O.grid_position(cfg, (x / 2 + 0.5).astype(np.float32))
    np.testing.assert_allclose(ph, want, atol=2e-7)
    # specific values: x = (2, 0, 0) -> y_x = 1.5; (3, 1.5, 0) -> (5/3, 5/6, 0)
    assert ph[2, 0] == pytest.approx(0.875, abs=1e-7)
    np.testing.assert_allclose(ph[4], [5 / 12 + 0.5, 5 / 24 + 0.5, 0.5], atol=2e-7)


def test_contraction_continuous_bounded_monotone():
    cfg = _contracted_cfg()
    rng = np.random.default_rng(1)
    d = rng.normal(size=(50, 3))
    d /= np.abs(d).max(axis=1, keepdims=True)  # |d|_inf = 1
    s = np.concatenate([np.linspace(0, 3, 301), np.geomspace(3, 1e5, 200)])
    for v in d:
        p = (0.5 + 0.5 * s[:, None] * v[None, :]).astype(np.float32)
        ph = O.grid_position(cfg, p).astype(np.float64)
        y = 4 * ph - 2
        assert (np.abs(y) <= 2).all()
        r = np.abs(y).max(axis=1)
        assert (np.diff(r) >= -1e-6).all()                  # monotone along the ray
        np.testing.assert_allclose(r[s <= 1], s[s <= 1], atol=1e-6)  # identity inside
        k = np.searchsorted(s, 1.0)
        assert abs(r[k + 1] - r[k]) < 0.02                  # continuous at the inner cube


def test_uncontract_round_trip():
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.normal(size=3) * rng.choice([0.3, 3.0, 30.0])
        m = np.abs(x).max()
        y = x if m <= 1 else (2 - 1 / m) * x / m
        np.testing.assert_allclose(O.uncontract(y), x, rtol=1e-12, atol=1e-12)
    assert O.uncontract(np.array([2.0, 0.0, 0.0])) is None


def test_contracted_footprint_inner_cube_and_plain():
    cfg = _contracted_cfg()
    p = np.array([0.6, 0.45, 0.3], np.float32)
    du, dv = np.array([1e-3, 0, 0]), np.array([0, 2e-3, 0])
    t, r = 0.7, 0.0005
    # inside: t r inv_h / 4 (explicit), radius_scale * t * mean|d_adj| inv_h / 4 (camera)
    assert O.footprint(cfg, p, t, r) == pytest.approx(t * r * 2 / 4, rel=1e-6)
    assert O.footprint(cfg, p, t, r, (du, dv)) == pytest.approx(
        cfg.radius_scale * np.float32(t) * 1.5e-3 * 2 / 4, rel=1e-6)
    plain = replace(cfg, contract=False)
    assert O.footprint(plain, p, t, r) == pytest.approx(np.float32(t) * r, rel=1e-6)


def test_contracted_footprint_against_finite_differences():
    """Outside the inner cube: the camera footprint is the first-order distance
    between adjacent rays' contracted samples (finite difference of C with a
    tiny offset), and det(J_C)^(1/3) matches a finite-difference Jacobian."""
    cfg = _contracted_cfg()
    rng = np.random.default_rng(3)

    def C(x):
        m = np.abs(x).max()
        return x if m <= 1 else (2 - 1 / m) * x / m

    for _ in range(100):
        x = rng.normal(size=3) * 4
        if np.abs(x).max() < 1.2:
            continue
        p = (0.5 + x / 2).astype(np.float32)
        x = (p.astype(np.float64) - 0.5) * 2
        t = 2.0
        du = rng.normal(size=3) * 1e-7
        dv = rng.normal(size=3) * 1e-7
        want = np.mean([np.linalg.norm(C(x + t * dd * 2) - C(x)) for dd in (du, dv)])
        got = O.footprint(cfg, p, t, 0.0, (du, dv))
        assert got == pytest.approx(cfg.radius_scale * want / 4, rel=1e-4)
        h = 1e-6
        J = np.stack([(C(x + h * e) - C(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        want_j = np.cbrt(np.linalg.det(J))
        assert O.footprint(cfg, p, t, 1e-3) == pytest.approx(t * 1e-3 * 2 * want_j / 4, rel=1e-5)


def test_contracted_march_brute_force():
    cfg = _contracted_cfg(occ_res=(16, 16, 16))
    rng = np.random.default_rng(4)
    occ = rng.uniform(size=(16, 16, 16)) < 0.15
    F = O.Field(cfg, np.zeros((cfg.levels, cfg.T, 2)), np.zeros(O.mlp_count(cfg)), S.pack_bits(occ))
    o = rng.uniform(0.2, 0.8, (30, 3)).astype(np.float32)
    d = rng.normal(size=(30, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    ri, rv, cnt = F.march(o, d, cfg.max_steps)
    t = O.sample_table(cfg)
    flat = occ.reshape(-1)
    for b in range(30):
        # every sample stays on the grid (the contracted cube covers space)
        p = (o[b][None, :] + t[:-1, None] * d[b][None, :]).astype(np.float32)
        ph = O.grid_position(cfg, p)
        v = np.clip(np.floor(ph * np.float32(16)).astype(np.int64), 0, 15)
        vox = v[:, 0] + 16 * (v[:, 1] + 16 * v[:, 2])
        want = [(i, vx) for i, vx in enumerate(vox) if flat[vx]]
        assert cnt[b] == len(want)
        assert [(int(a), int(c)) for a, c in zip(ri[b, :cnt[b]], rv[b, :cnt[b]])] == want
    assert cnt.sum() > 100


def test_contracted_history_brute_force():
    """History of a contracted scene (Sec. 4.3.2 with the contraction of
    Sec. 4): with constant density every composited sample's opacity is
    1 - exp(-sigma delta_i), recorded in the voxel of the contracted grid the
    sample falls in (found here by brute force from the contracted position);
    the bounded rule (p - box_min) / cell would put it elsewhere or drop it.
    Rays start inside the box and 20 units outside it."""
    cfg = _contracted_cfg(occ_res=(16, 16, 16), density_bias=0.5, T_eps=0.0)
    rng = np.random.default_rng(6)
    occ = rng.uniform(size=(16, 16, 16)) < 0.2
    F = O.Field(cfg, np.zeros((cfg.levels, cfg.T, 2)), np.zeros(O.mlp_count(cfg)), S.pack_bits(occ))
    n = 120
    o = np.concatenate([rng.uniform(0.2, 0.8, (n // 2, 3)),
                        0.5 + 20 * rng.normal(size=(n // 2, 3))]).astype(np.float32)
    d = np.where(np.arange(n)[:, None] < n // 2, rng.normal(size=(n, 3)), 0.5 - o)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    h = O.history(F, o, d, np.zeros(n, np.float32))
    t = O.sample_table(cfg).astype(np.float64)
    flat = occ.reshape(-1)
    want = np.zeros(16 ** 3)
    for b in range(n):
        p = (o[b][None, :] + t[:-1, None].astype(np.float32) * d[b][None, :]).astype(np.float32)
        v = np.clip(np.floor(O.grid_position(cfg, p) * np.float32(16)).astype(np.int64), 0, 15)
        vox = v[:, 0] + 16 * (v[:, 1] + 16 * v[:, 2])
        for i, vx in enumerate(vox):
            if flat[vx]:
                want[vx] = max(want[vx], 1 - np.exp(-np.exp(0.5) * (t[i + 1] - t[i])))
    assert (want > 0).sum() > 100
    # voxels outside the box's image [4, 12)^3 are reached too
    assert (want.reshape(16, 16, 16)[:4] > 0).any()
    np.testing.assert_allclose(h, want.astype(np.float32), rtol=1e-6, atol=0)


def test_contracted_density_grad_matches_central_differences():
    """As the plain-scene pin, with the gradient chained through J_C: points in
    the outer shell and in the inner cube, away from cell faces and from the
    planes where the largest |x_k| changes axis (J_C jumps there). Coarse
    levels (finest N = 13) let the stencil span 1e-3 of the grid, so the fp32
    rounding of the grid position stays below 1e-4 of it."""
    cfg = replace(_contracted_cfg(occ_res=(16, 16, 16)), levels=4, base_res=4.0, growth=1.5)
    rng = np.random.default_rng(8)
    grid = rng.uniform(0.1, 1.0, (cfg.levels, cfg.T, cfg.feats))
    mlp = rng.normal(size=O.mlp_count(cfg)) * 0.3
    din = cfg.levels * cfg.feats
    W1 = np.abs(mlp[:64 * din].reshape(64, din))
    W1[32:] *= -1
    mlp[:64 * din] = W1.reshape(-1)
    F = O.Field(cfg, grid, mlp, S.pack_bits(np.ones((16, 16, 16), bool)))
    n = 8000
    pos = (0.5 + rng.normal(size=(n, 3)) * rng.choice([0.2, 1.5], (n, 1))).astype(np.float32)
    _, frac = O.corners(cfg, pos)
    x = np.abs((pos.astype(np.float64) - 0.5) * 2)
    xs = np.sort(x, axis=1)
    ok = ((frac > 0.1) & (frac < 0.9)).reshape(n, -1).all(axis=1) & (xs[:, 2] - xs[:, 1] > 0.05 * xs[:, 2])
    ok &= np.abs(xs[:, 2] - 1.0) > 0.05  # not at the inner cube's faces
    sig, grad = F.density_grad(pos, 1e-5)
    idx = np.flatnonzero(ok)
    outer = xs[idx, 2] > 1.0
    assert idx.size > 100 and outer.sum() > 30, (idx.size, outer.sum())
    for i in idx:
        h = 1e-3 * max(1.0, xs[i, 2])  # at most 1e-3 of the grid, tangential or radial
        fd = np.zeros(3)
        for k in range(3):
            pp, pm = pos[i].copy(), pos[i].copy()
            pp[k] += h
            pm[k] -= h
            ls = np.log(F.density_grad(np.stack([pp, pm]), 1e-5)[0])
            fd[k] = (ls[0] - ls[1]) / (float(pp[k]) - float(pm[k]))
        np.testing.assert_allclose(grad[i] / sig[i], fd, rtol=0, atol=1e-3 * np.abs(fd).max())
