/*
 * vrnerf_oracle.c -- plain CPU oracle of VR-NeRF's per-ray field rendering
 * ("VR-NeRF: High-Fidelity Virtualized Walkable Spaces", Sec. 4-6).
 *
 * TEST INFRASTRUCTURE ONLY. It is loaded by the test suite, by the smoke
 * check and by the benchmark's CPU-baseline leg, never by the product path,
 * and it shares no code, header, table or constant with the CUDA library.
 *
 * What it computes, one ray at a time and in the paper's order:
 *   ray -> exponential samples -> occupancy test (Sec. 4.3) -> LOD level and
 *   weights (Sec. 4.2.1, Eq. 3) -> multiresolution hash-grid features ->
 *   density MLP and colour MLP (Sec. 6) -> sigmoid colour in PQ space
 *   (Sec. 4.1) -> front-to-back compositing with early termination -> PQ
 *   decode (Eq. 1-2); and the L1 loss in PQ space with its gradient and the
 *   Adam step (Sec. 6, supplement "Loss Design").
 *
 * Precision. Parameters, interpolation, MLPs, compositing and PQ run in
 * fp64. The decisions that floating point turns into integers -- which
 * occupancy voxel a sample falls in and which hash-grid corners it reads --
 * are taken in fp32 with every multiply, add, divide and square root rounded
 * on its own (no fused multiply-add: build with -ffp-contract=off), i.e. in
 * the kernels' precision, so both sides take the same decision.
 *
 * Readings where the paper is silent (S) or ambiguous (A); each is listed
 * with its reason in the design notes:
 *  - (S) pinhole rays through pixel centres, camera looking down +z of its
 *    frame; base radius r = radius_scale / fx (0.5: half a pixel);
 *  - (S) sample i sits at t_i = t_near (t_far/t_near)^(i/S), delta_i =
 *    t_{i+1} - t_i; the march ends when a sample leaves the occupancy grid;
 *  - (S) level resolution N_l = floor(s f^l + 1e-6); level l is dense when
 *    (N_l+1)^3 <= T, else hashed with the instant-NGP spatial hash;
 *  - (A) hash-grid coordinates are normalised by the largest AABB extent;
 *  - (S) no biases; sigma = exp(o_0 + density_bias); direction encoding =
 *    real spherical harmonics of bands 0-3 (16 values);
 *  - (S) compositing stops after the sample at which T < T_eps; black
 *    background; compositing happens in PQ space, then PQ is decoded per
 *    channel with 1.0 linear = 100 cd/m^2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_LEVELS 32

typedef struct {
    int32_t levels, feats, log2_T, feat_fp16;
    double base_res, growth;
    int32_t d_hidden, d_out, c_hidden, c_layers;
    float aabb_min[3], aabb_max[3];
    int32_t occ_res[3];
    int32_t max_steps;
    float t_near, t_far;
    double lod_bias, T_eps, radius_scale, density_bias;
    int32_t contract; /* 1: unbounded scene, L-infinity contraction (Sec. 4) */
    int32_t pad;
} orc_desc;

/* ------------------------------------------------------------------------
 * PQ transfer function, Sec. 4.1 Eq. 1-2 (SMPTE ST 2084).
 * Y in [0,1] stands for 0..10 000 cd/m^2; linear colour 1 is 100 cd/m^2.
 * --------------------------------------------------------------------- */
static const double PQ_M1 = 1305.0 / 8192.0;
static const double PQ_M2 = 2523.0 / 32.0;
static const double PQ_C1 = 107.0 / 128.0;
static const double PQ_C2 = 2413.0 / 128.0;
static const double PQ_C3 = 2392.0 / 128.0;

/* Eq. 1: PQ(Y), Y clamped to [0, 1]. */
double orc_pq_encode(double Y)
{
    if (!(Y > 0.0)) Y = 0.0;
    if (Y > 1.0) Y = 1.0;
    double ym = pow(Y, PQ_M1);
    return pow((PQ_C1 + PQ_C2 * ym) / (1.0 + PQ_C3 * ym), PQ_M2);
}

/* Inverse of Eq. 1 solved for Y: with e = E^(1/m2), e (1 + c3 Y^m1) =
 * c1 + c2 Y^m1, so Y^m1 = (e - c1) / (c2 - c3 e). E clamped to [0, 1]. */
double orc_pq_decode(double E)
{
    if (!(E > 0.0)) E = 0.0;
    if (E > 1.0) E = 1.0;
    double e = pow(E, 1.0 / PQ_M2);
    double num = e - PQ_C1;
    if (num < 0.0) num = 0.0;
    return pow(num / (PQ_C2 - PQ_C3 * e), 1.0 / PQ_M1);
}

/* linear colour (1.0 = 100 cd/m^2) -> PQ and back. */
double orc_linear_to_pq(double c) { return orc_pq_encode(c / 100.0); }
double orc_pq_to_linear(double E) { return 100.0 * orc_pq_decode(E); }

/* ------------------------------------------------------------------------
 * Level-of-detail weights, Sec. 4.2.1 Eq. 3, written as its three cases.
 * --------------------------------------------------------------------- */
void orc_lod_weights(double Lstar, int32_t levels, double *w)
{
    double fl = floor(Lstar), ce = ceil(Lstar);
    for (int32_t l = 0; l < levels; ++l) {
        double L = (double)l;
        if (L <= fl)
            w[l] = 1.0;
        else if (L <= ce)
            w[l] = Lstar - fl;
        else
            w[l] = 0.0;
    }
}

/* Optimal level L* = -log_f(2 s r) + dL (Sec. 4.2.1 and 4.2.2); r is the
 * footprint radius in normalised grid units. */
double orc_lod_level(const orc_desc *D, double r_norm)
{
    return -log(2.0 * D->base_res * r_norm) / log(D->growth) + D->lod_bias;
}

/* ------------------------------------------------------------------------
 * Grid geometry.
 * --------------------------------------------------------------------- */
int32_t orc_level_res(const orc_desc *D, int32_t l)
{
    return (int32_t)floor(D->base_res * pow(D->growth, (double)l) + 1e-6);
}

int32_t orc_level_dense(const orc_desc *D, int32_t l)
{
    int64_t n1 = (int64_t)orc_level_res(D, l) + 1;
    return n1 * n1 * n1 <= ((int64_t)1 << D->log2_T);
}

/* Exponentially spaced sample distances (Sec. 6), t[0..S], fp64 rounded to fp32. */
void orc_sample_table(const orc_desc *D, float *t)
{
    int32_t S = D->max_steps;
    double tn = (double)D->t_near, tf = (double)D->t_far;
    for (int32_t i = 0; i <= S; ++i)
        t[i] = (float)(tn * pow(tf / tn, (double)i / (double)S));
}

typedef struct {
    float mn[3], inv_cell[3], inv_ext;
    float cen[3], inv_h; /* contraction: x = (p - cen) inv_h, inner cube |x|_inf <= 1 */
    int32_t contract;
    int32_t N[ORC_MAX_LEVELS], dense[ORC_MAX_LEVELS];
    uint32_t T;
} orc_geom;

static void geom_init(const orc_desc *D, orc_geom *g)
{
    double ext_max = 0.0;
    for (int k = 0; k < 3; ++k) {
        double ext = (double)D->aabb_max[k] - (double)D->aabb_min[k];
        g->mn[k] = D->aabb_min[k];
        g->inv_cell[k] = (float)((double)D->occ_res[k] / ext);
        if (ext > ext_max) ext_max = ext;
    }
    g->inv_ext = (float)(1.0 / ext_max);
    g->contract = D->contract;
    for (int k = 0; k < 3; ++k)
        g->cen[k] = (float)(0.5 * ((double)D->aabb_min[k] + (double)D->aabb_max[k]));
    g->inv_h = (float)(2.0 / ext_max);
    for (int32_t l = 0; l < D->levels; ++l) {
        g->N[l] = orc_level_res(D, l);
        g->dense[l] = orc_level_dense(D, l);
    }
    g->T = 1u << D->log2_T;
}

/* Pinhole ray through the centre of pixel (u, v), in fp32 with separate
 * rounding of each operation. c2w is [3][4] (columns right, down, forward,
 * centre); K = (fx, fy, cx, cy). */
void orc_ray(const float *c2w, const float *K, int32_t u, int32_t v, float *o, float *d)
{
    float x = ((float)u + 0.5f - K[2]) / K[0];
    float y = ((float)v + 0.5f - K[3]) / K[1];
    float n = sqrtf(x * x + y * y + 1.0f);
    float cx = x / n, cy = y / n, cz = 1.0f / n;
    for (int k = 0; k < 3; ++k) {
        d[k] = c2w[4 * k + 0] * cx + c2w[4 * k + 1] * cy + c2w[4 * k + 2] * cz;
        o[k] = c2w[4 * k + 3];
    }
}

/* Cubic space contraction with the L-infinity norm (Sec. 4, unbounded
 * scenes): with m = |x|_inf, C(x) = x for m <= 1, else (2 - 1/m) x / m, so
 * the whole space maps into the cube |y|_inf < 2 and the inner cube stays
 * as it is. fp32 with every operation rounded on its own (voxel decisions):
 * s = (2 - 1/m) (1/m), y = x s. */
static float linf(const float *x)
{
    float m = fabsf(x[0]);
    if (fabsf(x[1]) > m) m = fabsf(x[1]);
    if (fabsf(x[2]) > m) m = fabsf(x[2]);
    return m;
}

static void contract_pt(const float *x, float *y)
{
    float m = linf(x);
    if (m <= 1.0f) {
        for (int k = 0; k < 3; ++k) y[k] = x[k];
        return;
    }
    float inv = 1.0f / m;
    float sc = (2.0f - inv) * inv;
    for (int k = 0; k < 3; ++k) y[k] = x[k] * sc;
}

/* Normalised grid position in [0, 1]^3 of world position p: the scene box
 * scaled by its largest extent, or (contracted scenes) the contracted point
 * of the cube [-2, 2]^3, ph = y / 4 + 1/2. */
static void grid_ph(const orc_geom *g, const float *p, float *ph)
{
    if (!g->contract) {
        for (int k = 0; k < 3; ++k) ph[k] = (p[k] - g->mn[k]) * g->inv_ext;
        return;
    }
    float x[3], y[3];
    for (int k = 0; k < 3; ++k) x[k] = (p[k] - g->cen[k]) * g->inv_h;
    contract_pt(x, y);
    for (int k = 0; k < 3; ++k) ph[k] = y[k] * 0.25f + 0.5f;
}

/* Sample position p = o + t d and its occupancy voxel, fp32. Returns 0 when
 * any voxel coordinate falls outside [0, res): the march ends there. The
 * grid of a contracted scene covers all of space: its coordinates are
 * clamped to the last voxel (reached only where 2 - 1/m rounds to 2). */
static int sample_voxel(const orc_desc *D, const orc_geom *g, const float *o, const float *d,
                        float t, float *p, int32_t *vox)
{
    int32_t v[3];
    for (int k = 0; k < 3; ++k) p[k] = o[k] + t * d[k];
    if (g->contract) {
        float ph[3];
        grid_ph(g, p, ph);
        for (int k = 0; k < 3; ++k) {
            float gk = ph[k] * (float)D->occ_res[k];
            int32_t c = (int32_t)floorf(gk);
            v[k] = c < 0 ? 0 : (c > D->occ_res[k] - 1 ? D->occ_res[k] - 1 : c);
        }
    } else {
        for (int k = 0; k < 3; ++k) {
            float gk = (p[k] - g->mn[k]) * g->inv_cell[k];
            if (!(gk >= 0.0f) || !(gk < (float)D->occ_res[k])) return 0;
            v[k] = (int32_t)floorf(gk);
        }
    }
    *vox = v[0] + D->occ_res[0] * (v[1] + D->occ_res[1] * v[2]);
    return 1;
}

/* Contraction Jacobian applied to a vector, fp64: J v = v inside the inner
 * cube, else s v + s'(m) x sign(x_k) v_k with s(m) = 2/m - 1/m^2 and k the
 * axis of the largest |x_k| (the first one on ties). */
static void contract_jv(const double *x, const double *v, double *out)
{
    double m = fabs(x[0]);
    int k = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(x[a]) > m) {
            m = fabs(x[a]);
            k = a;
        }
    if (m <= 1.0) {
        for (int a = 0; a < 3; ++a) out[a] = v[a];
        return;
    }
    const double sc = 2.0 / m - 1.0 / (m * m), ds = -2.0 / (m * m) + 2.0 / (m * m * m);
    const double vk = x[k] >= 0.0 ? v[k] : -v[k];
    for (int a = 0; a < 3; ++a) out[a] = sc * v[a] + ds * x[a] * vk;
}

/* Footprint radius in normalised grid units at distance t (Sec. 4.2.1).
 * Plain scenes: t r / max extent. Contracted scenes, camera rays (du, dv: the
 * direction of the pixel to the right and below minus the ray's own): the
 * distance between the sample and the corresponding samples of the two
 * adjacent rays in contracted space, to first order |J_C (t du inv_h)|,
 * averaged, times radius_scale (so that it is t r without contraction), over
 * 4 (the cube [-2, 2] spans the unit grid). Contracted scenes, explicit rays:
 * t r inv_h det(J_C)^(1/3) / 4, with det(J_C)^(1/3) = (2m - 1)^(2/3) / m^2
 * for m = |x|_inf > 1. */
static double footprint(const orc_desc *D, const orc_geom *g, const double *du, const double *dv,
                        float t, const float *p, double r)
{
    if (!g->contract) return (double)t * r * (double)g->inv_ext;
    double x[3], m = 0.0;
    for (int k = 0; k < 3; ++k) {
        x[k] = ((double)p[k] - (double)g->cen[k]) * (double)g->inv_h;
        if (fabs(x[k]) > m) m = fabs(x[k]);
    }
    if (du && dv) {
        double acc = 0.0;
        for (int a = 0; a < 2; ++a) {
            const double *da = a ? dv : du;
            double v[3], jv[3];
            for (int k = 0; k < 3; ++k) v[k] = (double)t * da[k] * (double)g->inv_h;
            contract_jv(x, v, jv);
            acc += sqrt(jv[0] * jv[0] + jv[1] * jv[1] + jv[2] * jv[2]);
        }
        return D->radius_scale * 0.5 * acc * 0.25;
    }
    double j = m <= 1.0 ? 1.0 : pow(2.0 * m - 1.0, 2.0 / 3.0) / (m * m);
    return (double)t * r * (double)g->inv_h * j * 0.25;
}

static int occupied(const uint32_t *occ, int32_t vox)
{
    return (occ[vox >> 5] >> (vox & 31)) & 1u;
}

/* Eight corner indices of level l for world position p (fp32 decisions) and
 * the fractional position inside the cell. Corner b has offset
 * (b & 1, (b >> 1) & 1, (b >> 2) & 1). */
static void level_corners(const orc_geom *g, int32_t l, const float *p, uint32_t *idx, float *frac)
{
    int32_t N = g->N[l];
    int32_t c0[3];
    float phv[3];
    grid_ph(g, p, phv);
    for (int k = 0; k < 3; ++k) {
        float ph = phv[k];
        float x = ph * (float)N;
        int32_t c = (int32_t)floorf(x);
        if (c < 0) c = 0;
        if (c > N - 1) c = N - 1;
        c0[k] = c;
        frac[k] = x - (float)c;
    }
    for (int b = 0; b < 8; ++b) {
        uint32_t cx = (uint32_t)(c0[0] + (b & 1));
        uint32_t cy = (uint32_t)(c0[1] + ((b >> 1) & 1));
        uint32_t cz = (uint32_t)(c0[2] + ((b >> 2) & 1));
        if (g->dense[l]) {
            uint32_t n1 = (uint32_t)N + 1u;
            idx[b] = cx + n1 * (cy + n1 * cz);
        } else {
            /* instant-NGP spatial hash: XOR of coordinates times large primes,
             * pi_1 = 1, modulo the table size. */
            idx[b] = (cx * 1u ^ cy * 2654435761u ^ cz * 805459861u) & (g->T - 1u);
        }
    }
}

/* Corner indices for n world positions: idx [n][L][8]. */
void orc_corners(const orc_desc *D, const float *pos, int32_t n, uint32_t *idx, float *frac)
{
    orc_geom g;
    geom_init(D, &g);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t l = 0; l < D->levels; ++l)
            level_corners(&g, l, pos + 3 * i, idx + ((int64_t)i * D->levels + l) * 8,
                          frac ? frac + ((int64_t)i * D->levels + l) * 3 : NULL);
}

/* ------------------------------------------------------------------------
 * Real spherical harmonics, bands 0..3 (16 values), from the general
 * definition: Y_lm = N_lm P_l^|m|(z) {sqrt2 cos(m phi), 1, sqrt2 sin(|m| phi)}
 * with the Condon-Shortley phase, N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!).
 * Index l^2 + l + m. The azimuthal factor is taken from (x + i y)^m =
 * sin^m(theta) e^{i m phi}, and P_l^m(z) = (-1)^m sin^m(theta) d^m P_l/dz^m.
 * --------------------------------------------------------------------- */
static double fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

/* m-th derivative of the Legendre polynomial P_l at z, from
 * P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) z^(l-2k). */
static double legendre_deriv(int l, int m, double z)
{
    double s = 0.0;
    for (int k = 0; 2 * k <= l; ++k) {
        int p = l - 2 * k;
        if (p < m) continue;
        double c = ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
        double dc = fact(p) / fact(p - m);
        s += c * dc * pow(z, (double)(p - m));
    }
    return s / pow(2.0, (double)l);
}

void orc_sh16(const double *dir, double *out)
{
    double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= 3; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * fact(l - am) / fact(l + am));
            /* (x + i y)^am */
            double re = 1.0, im = 0.0;
            for (int j = 0; j < am; ++j) {
                double r2 = re * x - im * y, i2 = re * y + im * x;
                re = r2;
                im = i2;
            }
            double cs = (am & 1) ? -1.0 : 1.0;
            double Pd = legendre_deriv(l, am, z);
            double v;
            if (m == 0)
                v = N * Pd;
            else if (m > 0)
                v = sqrt(2.0) * N * cs * Pd * re;
            else
                v = sqrt(2.0) * N * cs * Pd * im;
            out[l * l + l + m] = v;
        }
    }
}

/* ------------------------------------------------------------------------
 * Field evaluation at one sample: LOD-weighted hash-grid features (Eq. 3),
 * density MLP and colour MLP (Sec. 6), fp64.
 * --------------------------------------------------------------------- */
typedef struct {
    double feat[ORC_MAX_LEVELS * 2];
    double wl[ORC_MAX_LEVELS];
    uint32_t idx[ORC_MAX_LEVELS][8];
    double cw[ORC_MAX_LEVELS][8];
    double h[64], o[16], x[32], h1[64], h2[64], z[3];
    double sigma, c[3];
} orc_sample;

static double relu(double v) { return v > 0.0 ? v : 0.0; }

static const double *mlp_W(const orc_desc *D, const double *mlp, int which)
{
    int din = D->levels * D->feats;
    const double *p = mlp;
    int sizes[5] = {64 * din, 16 * 64, 64 * 32, 64 * 64, 3 * 64};
    for (int i = 0; i < which; ++i) p += sizes[i];
    return p;
}

int32_t orc_mlp_count(const orc_desc *D)
{
    return 64 * D->levels * D->feats + 16 * 64 + 64 * 32 + 64 * 64 + 3 * 64;
}

/* Features at world position p with normalised footprint radius r_norm. */
static void sample_feats(const orc_desc *D, const orc_geom *g, const double *grid,
                         const float *p, double r_norm, orc_sample *s)
{
    int32_t L = D->levels, F = D->feats;
    orc_lod_weights(orc_lod_level(D, r_norm), L, s->wl);
    for (int32_t l = 0; l < L; ++l) {
        for (int f = 0; f < F; ++f) s->feat[l * F + f] = 0.0;
        if (s->wl[l] == 0.0) {
            /* level not resolvable at this footprint: not fetched, zeros */
            for (int b = 0; b < 8; ++b) {
                s->idx[l][b] = 0;
                s->cw[l][b] = 0.0;
            }
            continue;
        }
        float fr[3];
        level_corners(g, l, p, s->idx[l], fr);
        for (int b = 0; b < 8; ++b) {
            double w = 1.0;
            for (int k = 0; k < 3; ++k) {
                double t = (double)fr[k];
                w *= ((b >> k) & 1) ? t : 1.0 - t;
            }
            s->cw[l][b] = w;
            const double *e = grid + ((int64_t)l * g->T + s->idx[l][b]) * F;
            for (int f = 0; f < F; ++f) s->feat[l * F + f] += w * e[f];
        }
        for (int f = 0; f < F; ++f) s->feat[l * F + f] *= s->wl[l];
    }
}

static void mlp_forward(const orc_desc *D, const double *mlp, const double *dir, orc_sample *s)
{
    int din = D->levels * D->feats;
    const double *W1 = mlp_W(D, mlp, 0), *W2 = mlp_W(D, mlp, 1), *W3 = mlp_W(D, mlp, 2);
    const double *W4 = mlp_W(D, mlp, 3), *W5 = mlp_W(D, mlp, 4);
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int k = 0; k < din; ++k) a += W1[j * din + k] * s->feat[k];
        s->h[j] = relu(a);
    }
    for (int i = 0; i < 16; ++i) {
        double a = 0.0;
        for (int j = 0; j < 64; ++j) a += W2[i * 64 + j] * s->h[j];
        s->o[i] = a;
    }
    s->sigma = exp(s->o[0] + D->density_bias);
    double sh[16];
    orc_sh16(dir, sh);
    for (int i = 0; i < 16; ++i) {
        s->x[i] = s->o[i];
        s->x[16 + i] = sh[i];
    }
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int k = 0; k < 32; ++k) a += W3[j * 32 + k] * s->x[k];
        s->h1[j] = relu(a);
    }
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int k = 0; k < 64; ++k) a += W4[j * 64 + k] * s->h1[k];
        s->h2[j] = relu(a);
    }
    for (int c = 0; c < 3; ++c) {
        double a = 0.0;
        for (int k = 0; k < 64; ++k) a += W5[c * 64 + k] * s->h2[k];
        s->z[c] = a;
        s->c[c] = 1.0 / (1.0 + exp(-a)); /* sigmoid -> PQ-space colour */
    }
}

/* Gradient of sigma with respect to the world position p at a fixed
 * footprint (the LOD weights w_l depend on the ray distance, not on p):
 * sigma = exp(o_0 + bias), o_0 = W2[0] relu(W1 feat), and feature (l, f) is
 * w_l times the trilinear interpolation of its cell's corners in the level's
 * coordinate x = N_l (p - aabb_min) / max extent, whose derivative along
 * axis k replaces the corner weight's factor of axis k by +-1. */
static void density_grad(const orc_desc *D, const orc_geom *g, const double *grid, const double *mlp,
                         const float *p, const orc_sample *s, double *grad)
{
    int32_t L = D->levels, F = D->feats, din = L * F;
    const double *W1 = mlp_W(D, mlp, 0), *W2 = mlp_W(D, mlp, 1);
    double dfeat[ORC_MAX_LEVELS * 2][3];
    for (int32_t l = 0; l < L; ++l) {
        for (int f = 0; f < F; ++f)
            for (int k = 0; k < 3; ++k) dfeat[l * F + f][k] = 0.0;
        if (s->wl[l] == 0.0) continue;
        uint32_t idx[8];
        float fr[3];
        level_corners(g, l, p, idx, fr);
        const double dxdp = (double)g->N[l]; /* d (level coordinate) / d ph */
        for (int b = 0; b < 8; ++b) {
            const double *e = grid + ((int64_t)l * g->T + idx[b]) * F;
            for (int k = 0; k < 3; ++k) {
                double dw = ((b >> k) & 1) ? 1.0 : -1.0;
                for (int m = 0; m < 3; ++m) {
                    if (m == k) continue;
                    double t = (double)fr[m];
                    dw *= ((b >> m) & 1) ? t : 1.0 - t;
                }
                for (int f = 0; f < F; ++f) dfeat[l * F + f][k] += s->wl[l] * dxdp * dw * e[f];
            }
        }
    }
    for (int k = 0; k < 3; ++k) {
        double do0 = 0.0;
        for (int j = 0; j < 64; ++j) {
            double pre = 0.0, dpre = 0.0;
            for (int q = 0; q < din; ++q) {
                pre += W1[j * din + q] * s->feat[q];
                dpre += W1[j * din + q] * dfeat[q][k];
            }
            if (pre > 0.0) do0 += W2[j] * dpre;
        }
        grad[k] = s->sigma * do0; /* d sigma / d ph_k */
    }
    /* chain to the world position: d ph / d p = inv_ext I, or for a
     * contracted scene inv_h J_C(x) / 4 (grad_p = (d ph / d p)^T grad_ph) */
    if (!g->contract) {
        for (int k = 0; k < 3; ++k) grad[k] *= (double)g->inv_ext;
        return;
    }
    double x[3], m = 0.0;
    int kk = 0;
    for (int k = 0; k < 3; ++k) {
        x[k] = ((double)p[k] - (double)g->cen[k]) * (double)g->inv_h;
        if (fabs(x[k]) > m) {
            m = fabs(x[k]);
            kk = k;
        }
    }
    const double sc = 0.25 * (double)g->inv_h;
    if (m <= 1.0) {
        for (int k = 0; k < 3; ++k) grad[k] *= sc;
        return;
    }
    const double s0 = 2.0 / m - 1.0 / (m * m), ds = -2.0 / (m * m) + 2.0 / (m * m * m);
    double gx = 0.0;
    for (int b = 0; b < 3; ++b) gx += grad[b] * x[b];
    for (int k = 0; k < 3; ++k) grad[k] *= s0;
    grad[kk] += (x[kk] >= 0.0 ? ds : -ds) * gx;
    for (int k = 0; k < 3; ++k) grad[k] *= sc;
}

/* sigma and its position gradient at n points (footprint radius in world
 * units per point): grad [n][3]. */
void orc_density_grad(const orc_desc *D, const double *grid, const double *mlp, const float *pos,
                      const double *radius, int32_t n, double *sigma, double *grad)
{
    orc_geom g;
    geom_init(D, &g);
    const double dir[3] = {0.0, 0.0, 1.0};
    for (int32_t i = 0; i < n; ++i) {
        orc_sample s;
        sample_feats(D, &g, grid, pos + 3 * i, footprint(D, &g, NULL, NULL, 1.0f, pos + 3 * i, radius[i]), &s);
        mlp_forward(D, mlp, dir, &s);
        sigma[i] = s.sigma;
        density_grad(D, &g, grid, mlp, pos + 3 * i, &s, grad + 3 * i);
    }
}

/* Field query at n points: world position, unit direction, footprint radius
 * (world units) -> sigma, PQ colour, and the 32 LOD-weighted features. */
void orc_query(const orc_desc *D, const double *grid, const double *mlp, const float *pos,
               const double *dir, const double *radius, int32_t n, double *sigma, double *rgb,
               double *feat)
{
    orc_geom g;
    geom_init(D, &g);
    int din = D->levels * D->feats;
    for (int32_t i = 0; i < n; ++i) {
        orc_sample s;
        sample_feats(D, &g, grid, pos + 3 * i, footprint(D, &g, NULL, NULL, 1.0f, pos + 3 * i, radius[i]), &s);
        mlp_forward(D, mlp, dir + 3 * i, &s);
        sigma[i] = s.sigma;
        for (int c = 0; c < 3; ++c) rgb[3 * i + c] = s.c[c];
        if (feat)
            for (int k = 0; k < din; ++k) feat[(int64_t)i * din + k] = s.feat[k];
    }
}

/* ------------------------------------------------------------------------
 * One ray: march, evaluate, composite front to back, stop when T < T_eps.
 * --------------------------------------------------------------------- */
typedef struct {
    double C[3];
    double T;
    double depth;     /* sum_i w_i t_i: expected distance of the composited samples */
    double normal[3]; /* sum_i w_i n_i, n_i = -grad sigma / |grad sigma| (when asked for) */
    int32_t n_eval;
} orc_ray_out;

/* Per-sample tape entry for the backward pass. */
typedef struct {
    float p[3];
    int32_t vox; /* the sample's occupancy voxel, as the march found it */
    double r_norm, delta, sigma, alpha, Tin, c[3];
} orc_tape;

static void render_one(const orc_desc *D, const orc_geom *g, const double *grid, const double *mlp,
                       const uint32_t *occ, const float *t_tab, const float *o, const float *d,
                       double r, const double *du, const double *dv, orc_ray_out *out,
                       orc_tape *tape, int normals)
{
    double dir[3] = {d[0], d[1], d[2]};
    double T = 1.0, C[3] = {0, 0, 0}, depth = 0.0, Nrm[3] = {0, 0, 0};
    int32_t n = 0;
    for (int32_t i = 0; i < D->max_steps; ++i) {
        float p[3];
        int32_t vox;
        if (!sample_voxel(D, g, o, d, t_tab[i], p, &vox)) break;
        if (!occupied(occ, vox)) continue;
        double t = (double)t_tab[i];
        double delta = (double)t_tab[i + 1] - (double)t_tab[i];
        double r_norm = footprint(D, g, du, dv, t_tab[i], p, r);
        orc_sample s;
        sample_feats(D, g, grid, p, r_norm, &s);
        mlp_forward(D, mlp, dir, &s);
        double alpha = 1.0 - exp(-s.sigma * delta);
        double w = T * alpha;
        if (tape) {
            orc_tape *e = &tape[n];
            memcpy(e->p, p, sizeof p);
            e->vox = vox;
            e->r_norm = r_norm;
            e->delta = delta;
            e->sigma = s.sigma;
            e->alpha = alpha;
            e->Tin = T;
            for (int c = 0; c < 3; ++c) e->c[c] = s.c[c];
        }
        for (int c = 0; c < 3; ++c) C[c] += w * s.c[c];
        depth += w * t;
        if (normals) {
            double gs[3];
            density_grad(D, g, grid, mlp, p, &s, gs);
            const double len = sqrt(gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2]);
            if (len > 0.0)
                for (int k = 0; k < 3; ++k) Nrm[k] += w * (-gs[k] / len);
        }
        T *= 1.0 - alpha;
        ++n;
        if (T < D->T_eps) break;
    }
    for (int c = 0; c < 3; ++c) out->C[c] = C[c];
    out->T = T;
    out->depth = depth;
    for (int k = 0; k < 3; ++k) out->normal[k] = Nrm[k];
    out->n_eval = n;
}

static void render_rays_impl(const orc_desc *D, const double *grid, const double *mlp,
                             const uint32_t *occ, const float *o, const float *d, const float *r,
                             const double *du, const double *dv, int32_t B, double *out_pq,
                             double *out_lin, double *out_T, int32_t *out_n, double *out_depth,
                             double *out_normal, int32_t threads)
{
    orc_geom g;
    geom_init(D, &g);
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
#pragma omp parallel for schedule(dynamic, 16) num_threads(threads > 0 ? threads : 1)
    for (int32_t i = 0; i < B; ++i) {
        orc_ray_out ro;
        render_one(D, &g, grid, mlp, occ, t_tab, o + 3 * i, d + 3 * i, (double)r[i],
                   du ? du + 3 * i : NULL, dv ? dv + 3 * i : NULL, &ro, NULL, out_normal != NULL);
        for (int c = 0; c < 3; ++c) {
            if (out_pq) out_pq[3 * i + c] = ro.C[c];
            if (out_lin) out_lin[3 * i + c] = orc_pq_to_linear(ro.C[c]);
            if (out_normal) out_normal[3 * i + c] = ro.normal[c];
        }
        if (out_T) out_T[i] = ro.T;
        if (out_n) out_n[i] = ro.n_eval;
        if (out_depth) out_depth[i] = ro.depth;
    }
    free(t_tab);
}

/* Explicit rays: o, d [B][3] fp32, r [B] (base radius at unit distance).
 * Outputs (any may be NULL): PQ colour [B][3], linear colour [B][3],
 * final transmittance [B], composited sample count [B], expected depth
 * sum_i w_i t_i [B], composited normal [B][3]. */
void orc_render_rays(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
                     const float *o, const float *d, const float *r, int32_t B, double *out_pq,
                     double *out_lin, double *out_T, int32_t *out_n, double *out_depth,
                     double *out_normal, int32_t threads)
{
    render_rays_impl(D, grid, mlp, occ, o, d, r, NULL, NULL, B, out_pq, out_lin, out_T, out_n,
                     out_depth, out_normal, threads);
}

/* Camera rays of a contracted scene: as orc_render_rays plus, per ray, the
 * direction offsets du, dv [B][3] to the adjacent pixels' rays, which set
 * the footprint in contracted space. */
void orc_render_rays_adjacent(const orc_desc *D, const double *grid, const double *mlp,
                              const uint32_t *occ, const float *o, const float *d, const float *r,
                              const double *du, const double *dv, int32_t B, double *out_pq,
                              double *out_lin, double *out_T, int32_t *out_n, double *out_depth,
                              double *out_normal, int32_t threads)
{
    render_rays_impl(D, grid, mlp, occ, o, d, r, du, dv, B, out_pq, out_lin, out_T, out_n,
                     out_depth, out_normal, threads);
}

/* Direction offsets to the adjacent pixels' rays, du = d(u + 1, v) - d(u, v)
 * and dv = d(u, v + 1) - d(u, v), per pixel in orc_camera_rays order (the
 * difference of the fp32 directions, taken in fp64). */
void orc_camera_adjacent(const float *c2w, const float *K, const int32_t *res, int32_t n_views,
                         double *du, double *dv)
{
    int64_t q = 0;
    for (int32_t v = 0; v < n_views; ++v) {
        int32_t W = res[2 * v], H = res[2 * v + 1];
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x, ++q) {
                float o[3], d0[3], d1[3], d2[3];
                orc_ray(c2w + 12 * v, K + 4 * v, x, y, o, d0);
                orc_ray(c2w + 12 * v, K + 4 * v, x + 1, y, o, d1);
                orc_ray(c2w + 12 * v, K + 4 * v, x, y + 1, o, d2);
                for (int k = 0; k < 3; ++k) {
                    du[3 * q + k] = (double)d1[k] - (double)d0[k];
                    dv[3 * q + k] = (double)d2[k] - (double)d0[k];
                }
            }
    }
}

/* Cameras c2w [n][3][4], K [n][4], res [n][2] = (W, H). Pixels of view v are
 * packed row-major after those of views 0..v-1. Optional window (x0, y0, w, h)
 * per view renders only that crop: win = NULL renders everything. */
void orc_render(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
                const float *c2w, const float *K, const int32_t *res, int32_t n_views,
                double *out_pq, double *out_lin, double *out_T, int32_t *out_n, double *out_depth,
                int32_t threads)
{
    int64_t total = 0;
    for (int32_t v = 0; v < n_views; ++v) total += (int64_t)res[2 * v] * res[2 * v + 1];
    float *o = (float *)malloc(sizeof(float) * 3 * total);
    float *d = (float *)malloc(sizeof(float) * 3 * total);
    float *r = (float *)malloc(sizeof(float) * total);
    int64_t q = 0;
    for (int32_t v = 0; v < n_views; ++v) {
        int32_t W = res[2 * v], H = res[2 * v + 1];
        float rr = (float)(D->radius_scale / (double)K[4 * v]);
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x, ++q) {
                orc_ray(c2w + 12 * v, K + 4 * v, x, y, o + 3 * q, d + 3 * q);
                r[q] = rr;
            }
    }
    double *du = NULL, *dv = NULL;
    if (D->contract) {
        du = (double *)malloc(sizeof(double) * 3 * total);
        dv = (double *)malloc(sizeof(double) * 3 * total);
        orc_camera_adjacent(c2w, K, res, n_views, du, dv);
    }
    render_rays_impl(D, grid, mlp, occ, o, d, r, du, dv, (int32_t)total, out_pq, out_lin, out_T,
                     out_n, out_depth, NULL, threads);
    free(du);
    free(dv);
    free(o);
    free(d);
    free(r);
}

/* Rays of n views -> o, d [total][3] and r [total] exactly as orc_render makes them. */
void orc_camera_rays(const orc_desc *D, const float *c2w, const float *K, const int32_t *res,
                     int32_t n_views, float *o, float *d, float *r)
{
    int64_t q = 0;
    for (int32_t v = 0; v < n_views; ++v) {
        int32_t W = res[2 * v], H = res[2 * v + 1];
        float rr = (float)(D->radius_scale / (double)K[4 * v]);
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x, ++q) {
                orc_ray(c2w + 12 * v, K + 4 * v, x, y, o + 3 * q, d + 3 * q);
                r[q] = rr;
            }
    }
}

/* Occupancy visits of explicit rays without early termination: for each ray
 * the ordered sample indices i and voxels of every evaluated sample, up to
 * cap records per ray; count[ray] is the full number. */
void orc_march(const orc_desc *D, const uint32_t *occ, const float *o, const float *d, int32_t B,
               int32_t cap, int32_t *rec_i, int32_t *rec_vox, int32_t *count)
{
    orc_geom g;
    geom_init(D, &g);
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
    for (int32_t r = 0; r < B; ++r) {
        int32_t n = 0;
        for (int32_t i = 0; i < D->max_steps; ++i) {
            float p[3];
            int32_t vox;
            if (!sample_voxel(D, &g, o + 3 * r, d + 3 * r, t_tab[i], p, &vox)) break;
            if (!occupied(occ, vox)) continue;
            if (n < cap) {
                rec_i[(int64_t)r * cap + n] = i;
                rec_vox[(int64_t)r * cap + n] = vox;
            }
            ++n;
        }
        count[r] = n;
    }
    free(t_tab);
}

/* ------------------------------------------------------------------------
 * Training: L1 loss in PQ space (supplement, "Loss Design"; Sec. 4.1),
 * its gradient through compositing, MLPs and the hash grid, and Adam
 * (Sec. 6: beta = (0.9, 0.99), eps = 1e-15).
 *
 * loss = 1/(3B) sum_rays sum_ch |C_pq - PQ(target / 100)|, subgradient 0 at 0.
 * Compositing gradient, with w_i = T_i a_i, T_{i+1} = T_i (1 - a_i),
 * a_i = 1 - exp(-sigma_i delta_i), C = sum_i w_i c_i:
 *   dC/dc_i     = w_i
 *   dC/dsigma_i = delta_i (T_{i+1} c_i - sum_{j>i} w_j c_j).
 * --------------------------------------------------------------------- */
static void mlp_backward(const orc_desc *D, const double *mlp, orc_sample *s, double dsigma,
                         const double *dc, double *gmlp, double *dfeat)
{
    int din = D->levels * D->feats;
    const double *W1 = mlp_W(D, mlp, 0), *W2 = mlp_W(D, mlp, 1), *W3 = mlp_W(D, mlp, 2);
    const double *W4 = mlp_W(D, mlp, 3), *W5 = mlp_W(D, mlp, 4);
    double *G1 = gmlp + (W1 - mlp), *G2 = gmlp + (W2 - mlp), *G3 = gmlp + (W3 - mlp);
    double *G4 = gmlp + (W4 - mlp), *G5 = gmlp + (W5 - mlp);
    double dz[3], dh2[64], dh1[64], dx[32], dout[16], dh[64];
    for (int c = 0; c < 3; ++c) dz[c] = dc[c] * s->c[c] * (1.0 - s->c[c]);
    for (int k = 0; k < 64; ++k) {
        double a = 0.0;
        for (int c = 0; c < 3; ++c) {
            a += W5[c * 64 + k] * dz[c];
            G5[c * 64 + k] += dz[c] * s->h2[k];
        }
        dh2[k] = s->h2[k] > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < 64; ++k) {
        double a = 0.0;
        for (int j = 0; j < 64; ++j) {
            a += W4[j * 64 + k] * dh2[j];
            G4[j * 64 + k] += dh2[j] * s->h1[k];
        }
        dh1[k] = s->h1[k] > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < 32; ++k) {
        double a = 0.0;
        for (int j = 0; j < 64; ++j) {
            a += W3[j * 32 + k] * dh1[j];
            G3[j * 32 + k] += dh1[j] * s->x[k];
        }
        dx[k] = a;
    }
    for (int i = 0; i < 16; ++i) dout[i] = dx[i];
    dout[0] += dsigma * s->sigma; /* sigma = exp(o_0 + bias) */
    for (int j = 0; j < 64; ++j) {
        double a = 0.0;
        for (int i = 0; i < 16; ++i) {
            a += W2[i * 64 + j] * dout[i];
            G2[i * 64 + j] += dout[i] * s->h[j];
        }
        dh[j] = s->h[j] > 0.0 ? a : 0.0;
    }
    for (int k = 0; k < din; ++k) {
        double a = 0.0;
        for (int j = 0; j < 64; ++j) {
            a += W1[j * din + k] * dh[j];
            G1[j * din + k] += dh[j] * s->feat[k];
        }
        dfeat[k] = a;
    }
}

/* Loss and gradients for a batch of explicit rays. grid_grad [L][T][F] and
 * mlp_grad are overwritten. Returns the loss. */
/* Back-propagates dL/dC_pq = gC of one ray through compositing (suffix
 * sums S_i = sum_{j>i} w_j c_j, walked from the back), the MLPs and the
 * hash-grid interpolation, adding into grid_grad and mlp_grad. */
static void backprop_ray(const orc_desc *D, const orc_geom *g, const double *grid, const double *mlp,
                         const double *dir, const orc_ray_out *ro, const orc_tape *tape, const double *gC,
                         double *grid_grad, double *mlp_grad)
{
    int F = D->feats;
    double suffix[3] = {0, 0, 0};
    for (int32_t k = ro->n_eval - 1; k >= 0; --k) {
        const orc_tape *e = &tape[k];
        double w = e->Tin * e->alpha, Tout = e->Tin * (1.0 - e->alpha);
        double dc[3], dsig = 0.0;
        for (int c = 0; c < 3; ++c) {
            dc[c] = w * gC[c];
            dsig += gC[c] * e->delta * (Tout * e->c[c] - suffix[c]);
        }
        orc_sample s;
        sample_feats(D, g, grid, e->p, e->r_norm, &s);
        mlp_forward(D, mlp, dir, &s);
        double dfeat[ORC_MAX_LEVELS * 2];
        mlp_backward(D, mlp, &s, dsig, dc, mlp_grad, dfeat);
        for (int32_t l = 0; l < D->levels; ++l) {
            if (s.wl[l] == 0.0) continue;
            for (int b = 0; b < 8; ++b) {
                double *gg = grid_grad + ((int64_t)l * g->T + s.idx[l][b]) * F;
                for (int f = 0; f < F; ++f) gg[f] += s.wl[l] * s.cw[l][b] * dfeat[l * F + f];
            }
        }
        for (int c = 0; c < 3; ++c) suffix[c] += w * e->c[c];
    }
}

double orc_backward(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
                    const float *o, const float *d, const float *r, const float *target_lin,
                    int32_t B, double *grid_grad, double *mlp_grad)
{
    orc_geom g;
    geom_init(D, &g);
    int64_t ngrid = (int64_t)D->levels * g.T * D->feats;
    memset(grid_grad, 0, sizeof(double) * ngrid);
    memset(mlp_grad, 0, sizeof(double) * orc_mlp_count(D));
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
    orc_tape *tape = (orc_tape *)malloc(sizeof(orc_tape) * D->max_steps);
    double loss = 0.0;
    for (int32_t i = 0; i < B; ++i) {
        const float *oi = o + 3 * i, *di = d + 3 * i;
        double dir[3] = {di[0], di[1], di[2]};
        orc_ray_out ro;
        render_one(D, &g, grid, mlp, occ, t_tab, oi, di, (double)r[i], NULL, NULL, &ro, tape, 0);
        double gC[3];
        for (int c = 0; c < 3; ++c) {
            double tgt = orc_linear_to_pq((double)target_lin[3 * i + c]);
            double diff = ro.C[c] - tgt;
            loss += fabs(diff);
            gC[c] = (diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0)) / (3.0 * B);
        }
        backprop_ray(D, &g, grid, mlp, dir, &ro, tape, gC, grid_grad, mlp_grad);
    }
    free(tape);
    free(t_tab);
    return loss / (3.0 * B);
}

/* Gradient of sum_i gC_i . C_pq(ray i) for a given upstream gradient gC
 * [B][3] (any loss on the PQ colours): grid_grad and mlp_grad overwritten. */
void orc_backward_grad(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
                       const float *o, const float *d, const float *r, const double *gC, int32_t B,
                       double *grid_grad, double *mlp_grad)
{
    orc_geom g;
    geom_init(D, &g);
    int64_t ngrid = (int64_t)D->levels * g.T * D->feats;
    memset(grid_grad, 0, sizeof(double) * ngrid);
    memset(mlp_grad, 0, sizeof(double) * orc_mlp_count(D));
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
    orc_tape *tape = (orc_tape *)malloc(sizeof(orc_tape) * D->max_steps);
    for (int32_t i = 0; i < B; ++i) {
        const float *oi = o + 3 * i, *di = d + 3 * i;
        double dir[3] = {di[0], di[1], di[2]};
        orc_ray_out ro;
        render_one(D, &g, grid, mlp, occ, t_tab, oi, di, (double)r[i], NULL, NULL, &ro, tape, 0);
        backprop_ray(D, &g, grid, mlp, dir, &ro, tape, gC + 3 * i, grid_grad, mlp_grad);
    }
    free(tape);
    free(t_tab);
}

/* Adam (Kingma and Ba 2015) on one parameter array, step number t >= 1. */
void orc_adam(double *param, const double *grad, double *m, double *v, int64_t n, int32_t t,
              double lr, double beta1, double beta2, double eps)
{
    double bc1 = 1.0 - pow(beta1, (double)t), bc2 = 1.0 - pow(beta2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------
 * Occupancy-grid pruning (Sec. 4.3.2), joint history and grid pruning.
 *
 * Grid part: for every occupied voxel, the maximum density over a k x k x k
 * lattice of points inside it (cell centres of the voxel's k^3 sub-cells;
 * full detail: footprint 0), turned into an opacity with the smallest step a
 * training ray can take there -- the sample spacing at the distance from the
 * nearest camera centre to the voxel (the spacing grows with distance):
 *     alpha_grid = 1 - exp(-sigma_max * delta_min).
 * History part: hist[v], the largest opacity 1 - exp(-sigma delta) of any
 * sample composited in v during training (NULL: none recorded).
 * A voxel stays occupied iff it was occupied and alpha_grid >= threshold or
 * hist >= threshold. keep_out [voxels] (0/1), alpha_out [voxels] (may be NULL).
 * --------------------------------------------------------------------- */
/* Inverse contraction, fp64: y with m = |y|_inf <= 1 is its own pre-image,
 * 1 < m < 2 comes from x = y / (m (2 - m)); returns 0 for m >= 2 (infinity). */
static int uncontract(const double *y, double *x)
{
    double m = fabs(y[0]);
    if (fabs(y[1]) > m) m = fabs(y[1]);
    if (fabs(y[2]) > m) m = fabs(y[2]);
    if (m >= 2.0) return 0;
    const double sc = m <= 1.0 ? 1.0 : 1.0 / (m * (2.0 - m));
    for (int a = 0; a < 3; ++a) x[a] = y[a] * sc;
    return 1;
}

static double box_distance(const double *c, const double *lo, const double *hi)
{
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double d = 0.0;
        if (c[k] < lo[k]) d = lo[k] - c[k];
        else if (c[k] > hi[k]) d = c[k] - hi[k];
        s += d * d;
    }
    return sqrt(s);
}

void orc_prune(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
               const float *cams, int32_t n_cams, int32_t k, double threshold, const float *hist,
               uint8_t *keep_out, double *alpha_out)
{
    orc_geom g;
    geom_init(D, &g);
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
    const int32_t rx = D->occ_res[0], ry = D->occ_res[1], rz = D->occ_res[2];
    double cell[3];
    for (int a = 0; a < 3; ++a) cell[a] = ((double)D->aabb_max[a] - (double)D->aabb_min[a]) / D->occ_res[a];
    for (int32_t vz = 0; vz < rz; ++vz)
        for (int32_t vy = 0; vy < ry; ++vy)
            for (int32_t vx = 0; vx < rx; ++vx) {
                const int32_t v = vx + rx * (vy + ry * vz);
                if (alpha_out) alpha_out[v] = 0.0;
                if (!occupied(occ, v)) {
                    keep_out[v] = 0;
                    continue;
                }
                const int32_t vv[3] = {vx, vy, vz};
                double lo[3], hi[3];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = D->aabb_min[a] + vv[a] * cell[a];
                    hi[a] = lo[a] + cell[a];
                }
                double sig_max = 0.0, dmin = INFINITY;
                for (int32_t i = 0; i < k * k * k; ++i) {
                    const int32_t j[3] = {i % k, (i / k) % k, i / (k * k)};
                    float p[3];
                    if (g.contract) {
                        double y[3];
                        for (int a = 0; a < 3; ++a)
                            y[a] = 4.0 * (vv[a] + (j[a] + 0.5) / k) / D->occ_res[a] - 2.0;
                        double x[3];
                        uncontract(y, x);
                        for (int a = 0; a < 3; ++a) p[a] = (float)(g.cen[a] + x[a] / (double)g.inv_h);
                        for (int32_t c = 0; c < n_cams; ++c) {
                            double s2 = 0.0;
                            for (int a = 0; a < 3; ++a) {
                                double e = (double)p[a] - (double)cams[3 * c + a];
                                s2 += e * e;
                            }
                            if (sqrt(s2) < dmin) dmin = sqrt(s2);
                        }
                    } else {
                        for (int a = 0; a < 3; ++a) p[a] = (float)(lo[a] + (j[a] + 0.5) / k * cell[a]);
                    }
                    orc_sample s;
                    sample_feats(D, &g, grid, p, 0.0, &s);
                    const double dir[3] = {0.0, 0.0, 1.0};
                    mlp_forward(D, mlp, dir, &s);
                    if (s.sigma > sig_max) sig_max = s.sigma;
                }
                if (g.contract) {
                    /* distance to the voxel's world region: exact for a voxel of
                     * the inner cube (its pre-image is a box), else the smallest
                     * distance to a lattice point or a finite corner pre-image */
                    double ylo[3], yhi[3], clo[3], chi[3];
                    int inner = 1;
                    for (int a = 0; a < 3; ++a) {
                        ylo[a] = 4.0 * vv[a] / D->occ_res[a] - 2.0;
                        yhi[a] = 4.0 * (vv[a] + 1) / D->occ_res[a] - 2.0;
                        if (ylo[a] < -1.0 || yhi[a] > 1.0) inner = 0;
                        clo[a] = g.cen[a] + ylo[a] / (double)g.inv_h;
                        chi[a] = g.cen[a] + yhi[a] / (double)g.inv_h;
                    }
                    if (inner) {
                        dmin = INFINITY;
                        for (int32_t c = 0; c < n_cams; ++c) {
                            const double cc[3] = {cams[3 * c], cams[3 * c + 1], cams[3 * c + 2]};
                            const double dd = box_distance(cc, clo, chi);
                            if (dd < dmin) dmin = dd;
                        }
                    } else {
                        for (int b = 0; b < 8; ++b) {
                            double y[3], x[3];
                            for (int a = 0; a < 3; ++a) y[a] = ((b >> a) & 1) ? yhi[a] : ylo[a];
                            if (!uncontract(y, x)) continue;
                            for (int32_t c = 0; c < n_cams; ++c) {
                                double s2 = 0.0;
                                for (int a = 0; a < 3; ++a) {
                                    double e = g.cen[a] + x[a] / (double)g.inv_h - (double)cams[3 * c + a];
                                    s2 += e * e;
                                }
                                if (sqrt(s2) < dmin) dmin = sqrt(s2);
                            }
                        }
                    }
                } else {
                    for (int32_t c = 0; c < n_cams; ++c) {
                        const double cc[3] = {cams[3 * c], cams[3 * c + 1], cams[3 * c + 2]};
                        const double dd = box_distance(cc, lo, hi);
                        if (dd < dmin) dmin = dd;
                    }
                }
                /* spacing of the sample interval holding distance dmin */
                int32_t i = 0;
                while (i + 1 < D->max_steps && (double)t_tab[i + 1] <= dmin) ++i;
                const double delta = (double)t_tab[i + 1] - (double)t_tab[i];
                const double alpha = 1.0 - exp(-sig_max * delta);
                if (alpha_out) alpha_out[v] = alpha;
                keep_out[v] = (alpha >= threshold || (hist && (double)hist[v] >= threshold)) ? 1 : 0;
            }
    free(t_tab);
}

/* Training history (Sec. 4.3.2): for explicit rays, the largest opacity
 * 1 - exp(-sigma delta) of any composited sample, per voxel; hist [voxels]
 * is raised, not reset. A sample's voxel is the one the occupancy march
 * found it in (sample_voxel), so a contracted scene (Sec. 4) records it in
 * the contracted grid. */
void orc_history(const orc_desc *D, const double *grid, const double *mlp, const uint32_t *occ,
                 const float *o, const float *d, const float *r, int32_t B, float *hist)
{
    orc_geom g;
    geom_init(D, &g);
    float *t_tab = (float *)malloc(sizeof(float) * (D->max_steps + 1));
    orc_sample_table(D, t_tab);
    orc_tape *tape = (orc_tape *)malloc(sizeof(orc_tape) * D->max_steps);
    for (int32_t b = 0; b < B; ++b) {
        orc_ray_out ro;
        render_one(D, &g, grid, mlp, occ, t_tab, o + 3 * b, d + 3 * b, (double)r[b], NULL, NULL, &ro, tape, 0);
        for (int32_t k = 0; k < ro.n_eval; ++k) {
            /* the voxel the march tested the sample in (contraction-aware) */
            const int32_t vox = tape[k].vox;
            const float a = (float)tape[k].alpha;
            if (a > hist[vox]) hist[vox] = a;
        }
    }
    free(tape);
    free(t_tab);
}

/* Display tonemapping (the paper's exposure sweep: PQ colour to sRGB at a
 * chosen exposure). Per channel: linear = PQ^-1(C) in units of 100 cd/m^2,
 * v = clamp(linear 2^ev, 0, 1), the sRGB transfer function of IEC 61966-2-1
 * (12.92 v up to 0.0031308, else 1.055 v^(1/2.4) - 0.055), 8 bits by
 * round-half-up of 255 s. Alpha = coverage 1 - T (255 when T is NULL).
 * rgba [n] packs R | G << 8 | B << 16 | A << 24; pre [n][4] (optional)
 * holds the unrounded 255 s values. */
static double srgb_oetf(double v)
{
    return v <= 0.0031308 ? 12.92 * v : 1.055 * pow(v, 1.0 / 2.4) - 0.055;
}

void orc_tonemap(const double *pq, const double *T, int64_t n, double ev, uint32_t *rgba, double *pre)
{
    const double scale = pow(2.0, ev);
    for (int64_t i = 0; i < n; ++i) {
        double q[4];
        for (int c = 0; c < 3; ++c) {
            double v = orc_pq_to_linear(pq[3 * i + c]) * scale;
            v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
            q[c] = 255.0 * srgb_oetf(v);
        }
        double a = T ? 1.0 - T[i] : 1.0;
        a = a < 0.0 ? 0.0 : (a > 1.0 ? 1.0 : a);
        q[3] = 255.0 * a;
        uint32_t word = 0;
        for (int c = 0; c < 4; ++c) {
            word |= (uint32_t)floor(q[c] + 0.5) << (8 * c);
            if (pre) pre[4 * i + c] = q[c];
        }
        rgba[i] = word;
    }
}

/* Introspection for the tests: normalised grid positions [n][3] (fp32, as
 * the march and the hash grid see them), inverse contraction [n][3] of
 * contracted points (fp64; 0 where |y|_inf >= 2), footprint radius of one
 * sample (du, dv may be NULL). */
void orc_grid_position(const orc_desc *D, const float *pos, int32_t n, float *ph)
{
    orc_geom g;
    geom_init(D, &g);
    for (int32_t i = 0; i < n; ++i) grid_ph(&g, pos + 3 * i, ph + 3 * i);
}

int32_t orc_uncontract(const double *y, double *x) { return uncontract(y, x); }

double orc_footprint(const orc_desc *D, const double *du, const double *dv, float t, const float *p,
                     double r)
{
    orc_geom g;
    geom_init(D, &g);
    return footprint(D, &g, du, dv, t, p, r);
}

/* Introspection for the tests. */
void orc_geometry(const orc_desc *D, int32_t *N, int32_t *dense, float *inv_cell, float *inv_ext)
{
    orc_geom g;
    geom_init(D, &g);
    for (int32_t l = 0; l < D->levels; ++l) {
        N[l] = g.N[l];
        dense[l] = g.dense[l];
    }
    for (int k = 0; k < 3; ++k) inv_cell[k] = g.inv_cell[k];
    *inv_ext = g.inv_ext;
}
