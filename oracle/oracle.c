/*
 * oracle.c -- FP64 brute-force CPU oracle for multi-depth ray casting with a depth-sensor model.
 *
 * TEST INFRASTRUCTURE. This is the slow, plain reference that the CUDA path is checked against.
 * Only the tests, the package smoke check and the benchmark's CPU-baseline leg build, load or call
 * it; the product path never links it and shares no code, header, table or helper with it.
 *
 * What it computes (Sec. 3.2.2 "Efficient Multi-Depth System Simulation", Algorithm 1, and the
 * perception rows of the domain-randomisation table in Appendix A.2):
 *   for every requested (env e, camera c, pixel x, y) at step s:
 *     1. camera pose   : link pose (t_l, q_l) of the mounting link composed with the mount offset;
 *     2. BuildDepthRay : r = ((x - c_x)/f_x, (y - c_y)/f_y, 1) in the optical frame (x right,
 *                        y down, z forward), d = R_c r / |r|, o = p_c, m = 1/|r|          (Alg. 1)
 *     3. closest hit   : every triangle of env e's link meshes (placed in the world by the link
 *                        poses) and every triangle of the shared terrain, intersected in FP64,
 *                        z_raw = min(d_max, min over hits of m*t)          (Alg. 1, far plane Sec. 3.2.2)
 *     4. downsample    : a camera rendered at raw resolution W x H and downsampled by f gives the
 *                        (W/f) x (H/f) image whose pixel is the mean of its f x f raw block
 *                        (240x135 raw to 48x27, Sec. 4.1, perception settings)
 *     5. sensor        : latency k ~ U{0..Lmax} per (env, camera, step); source step
 *                        s' = max(s - k, s_first[e]); z = z_raw(s'); Gaussian noise on hits,
 *                        clip to [d_min, d_max], pixel dropout                   (Appendix A.2)
 *     6. side masking  : an env in mask mode 1 (small) or 2 (large) has the outer n_mode columns on
 *                        both sides of every image filled with uniform values in [d_min, d_max]
 *                        (Random Side Masking, Sec. 3.2.4)
 *   Camera randomisation (Appendix A.2, perception rows): the mount of camera c in env e may be
 *   perturbed per env by (dp, dq): offset p_off + dp in the link frame, rotation R(q_off) R(dq), so
 *   dq rotates about the camera's own axes; FOV randomisation is per-env intrinsics.
 *   Random words come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
 *   (global env, camera, pixel, step).
 *
 * Readings where the paper is silent (each is listed with its reason in the design notes):
 *   - depth is z-depth along the optical axis, m*t (range t is an option);
 *   - triangles are two-sided and closed (edges and vertices belong to the triangle); t > 0;
 *   - z_raw at the far plane counts as a miss: noise is added only when z_raw < d_max;
 *   - noise sigma = sigma_abs + sigma_rel * z (the paper's preset is sigma_rel = 0.1);
 *   - n = sqrt(-2 ln u1) cos(2 pi u2), u1 = (w1 + 1) 2^-32, u2 = w2 2^-32 (Box-Muller);
 *   - dropout after clipping: if w0 < floor(p 2^32) the pixel becomes `fill`;
 *   - latency word: Philox with pixel field 0xFFFFFFFF, k = (w0 * (Lmax + 1)) >> 32;
 *   - counter (ge, c, pixel, step_lo), key (seed0 ^ step_hi, seed1); the pixel index is that of
 *     the output (downsampled) image;
 *   - downsampling is the plain mean of the f x f raw depths (misses count as d_max), taken before
 *     the sensor model, so the latency ring and the noise act on the policy-resolution image;
 *   - side-mask fill: d_min + (d_max - d_min) (w3 + 1/2) 2^-32 with w3 the fourth word of the keyed
 *     stream at the current step s (not the source step), applied after dropout.
 *
 * Besides the depth, each ray gets flags that say where FP32 arithmetic may legitimately decide
 * differently: the ray passes within eps of a silhouette edge (boundary edge or crease) of a
 * triangle whose plane it meets no farther than the visible surface; its raw depth lies within
 * 1e-4 of the far plane (the hit-or-miss decision that gates the noise); or the visible hit is so
 * oblique that FP32 rounding of the ray direction alone moves the depth by more than 2.5e-5 m.
 *
 * No acceleration structure, no blocking: each ray loops over every triangle.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EXPORT __attribute__((visibility("default")))

/* ---------------------------------------------------------------------------------------------
 * Philox4x32-10, from the SC'11 description: ten rounds of two 32x32->64 multiplies, each round
 *   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * with the key bumped by the Weyl constants between rounds.
 * ------------------------------------------------------------------------------------------- */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

ORACLE_EXPORT void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* The keyed stream: counter (env, cam, pixel, step_lo), key (seed0 ^ step_hi, seed1). */
static void keyed_words(uint32_t ge, uint32_t cam, uint32_t pix, int64_t step,
                        const uint32_t seed[2], uint32_t w[4])
{
    uint64_t s = (uint64_t)step;
    uint32_t ctr[4] = {ge, cam, pix, (uint32_t)(s & 0xFFFFFFFFu)};
    uint32_t key[2] = {seed[0] ^ (uint32_t)(s >> 32), seed[1]};
    oracle_philox4x32_10(ctr, key, w);
}

/* ---------------------------------------------------------------------------------------------
 * Small FP64 vector helpers
 * ------------------------------------------------------------------------------------------- */
typedef struct { double x, y, z; } vec3;

static vec3 v3(double x, double y, double z) { vec3 r = {x, y, z}; return r; }
static vec3 vsub(vec3 a, vec3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
static vec3 vadd(vec3 a, vec3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
static vec3 vscale(vec3 a, double s) { return v3(a.x * s, a.y * s, a.z * s); }
static double vdot(vec3 a, vec3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec3 vcross(vec3 a, vec3 b)
{
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double vnorm(vec3 a) { return sqrt(vdot(a, a)); }
static double vmaxabs(vec3 a)
{
    double m = fabs(a.x);
    if (fabs(a.y) > m) m = fabs(a.y);
    if (fabs(a.z) > m) m = fabs(a.z);
    return m;
}

/* Row-major 3x3 rotation of a unit quaternion (x, y, z, w), normalised here in FP64. */
static void quat_to_mat(const float qf[4], double R[9])
{
    double x = qf[0], y = qf[1], z = qf[2], w = qf[3];
    double n = sqrt(x * x + y * y + z * z + w * w);
    x /= n; y /= n; z /= n; w /= n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - z * w);     R[2] = 2 * (x * z + y * w);
    R[3] = 2 * (x * y + z * w);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - x * w);
    R[6] = 2 * (x * z - y * w);     R[7] = 2 * (y * z + x * w);     R[8] = 1 - 2 * (x * x + y * y);
}

static vec3 mat_vec(const double R[9], vec3 v)
{
    return v3(R[0] * v.x + R[1] * v.y + R[2] * v.z,
              R[3] * v.x + R[4] * v.y + R[5] * v.z,
              R[6] * v.x + R[7] * v.y + R[8] * v.z);
}

static void mat_mul(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            C[3 * i + j] = A[3 * i + 0] * B[0 + j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}

/* Spacing of float32 numbers at magnitude a (a > 0). */
static double ulp_f32(double a)
{
    int e;
    if (a < 1e-30) a = 1e-30;
    frexp(a, &e);          /* a = f 2^e, f in [0.5, 1) */
    return ldexp(1.0, e - 24);
}

/* Distance from p to segment [a, b]. */
static double point_segment_dist(vec3 p, vec3 a, vec3 b)
{
    vec3 ab = vsub(b, a), ap = vsub(p, a);
    double L2 = vdot(ab, ab);
    double u = L2 > 0 ? vdot(ap, ab) / L2 : 0.0;
    if (u < 0) u = 0;
    if (u > 1) u = 1;
    return vnorm(vsub(ap, vscale(ab, u)));
}

/* ---------------------------------------------------------------------------------------------
 * Scene: FP32 inputs kept as given, plus per-triangle silhouette-edge bits.
 * An edge is a silhouette edge when no other triangle shares it (a boundary), when more than two
 * triangles share it, or when its two triangles are not coplanar (a crease: |n1 x n2| > 1e-4 for
 * unit normals; below that the difference is FP32 rounding of a flat surface).
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    int64_t n_verts, n_tris;
    float *verts;        /* [V,3] */
    int32_t *tris;       /* [T,3] */
    uint8_t *sil;        /* [T] bit k: edge (v_k, v_{k+1 mod 3}) is a silhouette edge */
} mesh_t;

typedef struct {
    mesh_t terrain;
    int32_t n_links;
    mesh_t *links;
} oracle_scene;

typedef struct { uint64_t key; uint64_t ref; } edge_rec;

static void radix_sort_edges(edge_rec *a, edge_rec *tmp, int64_t n, int64_t *count)
{
    for (int pass = 0; pass < 4; ++pass) {
        int shift = 16 * pass;
        memset(count, 0, 65537 * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) count[((a[i].key >> shift) & 0xFFFF) + 1]++;
        for (int d = 0; d < 65536; ++d) count[d + 1] += count[d];
        for (int64_t i = 0; i < n; ++i) tmp[count[(a[i].key >> shift) & 0xFFFF]++] = a[i];
        memcpy(a, tmp, (size_t)n * sizeof(edge_rec));
    }
}

static vec3 vert_of(const mesh_t *m, int64_t vi)
{
    return v3(m->verts[3 * vi + 0], m->verts[3 * vi + 1], m->verts[3 * vi + 2]);
}

static vec3 unit_normal(const mesh_t *m, int64_t t, int *ok)
{
    vec3 a = vert_of(m, m->tris[3 * t + 0]);
    vec3 b = vert_of(m, m->tris[3 * t + 1]);
    vec3 c = vert_of(m, m->tris[3 * t + 2]);
    vec3 n = vcross(vsub(b, a), vsub(c, a));
    double l = vnorm(n);
    *ok = l > 0;
    return l > 0 ? vscale(n, 1.0 / l) : n;
}

static int mesh_init(mesh_t *m, const float *verts, int64_t n_verts, const int32_t *tris, int64_t n_tris)
{
    m->n_verts = n_verts;
    m->n_tris = n_tris;
    m->verts = (float *)malloc((size_t)(n_verts > 0 ? n_verts : 1) * 3 * sizeof(float));
    m->tris = (int32_t *)malloc((size_t)(n_tris > 0 ? n_tris : 1) * 3 * sizeof(int32_t));
    m->sil = (uint8_t *)calloc((size_t)(n_tris > 0 ? n_tris : 1), 1);
    if (!m->verts || !m->tris || !m->sil) return -1;
    if (n_verts) memcpy(m->verts, verts, (size_t)n_verts * 3 * sizeof(float));
    if (n_tris) memcpy(m->tris, tris, (size_t)n_tris * 3 * sizeof(int32_t));
    for (int64_t i = 0; i < 3 * n_tris; ++i)
        if (m->tris[i] < 0 || m->tris[i] >= n_verts) return -2;
    if (n_tris == 0) return 0;

    int64_t ne = 3 * n_tris;
    edge_rec *e = (edge_rec *)malloc((size_t)ne * sizeof(edge_rec));
    edge_rec *tmp = (edge_rec *)malloc((size_t)ne * sizeof(edge_rec));
    int64_t *count = (int64_t *)malloc(65537 * sizeof(int64_t));
    if (!e || !tmp || !count) { free(e); free(tmp); free(count); return -1; }
    for (int64_t t = 0; t < n_tris; ++t)
        for (int k = 0; k < 3; ++k) {
            uint64_t a = (uint32_t)m->tris[3 * t + k], b = (uint32_t)m->tris[3 * t + (k + 1) % 3];
            uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
            e[3 * t + k].key = (hi << 32) | lo;
            e[3 * t + k].ref = (uint64_t)(3 * t + k);
        }
    radix_sort_edges(e, tmp, ne, count);
    for (int64_t i = 0; i < ne;) {
        int64_t j = i;
        while (j < ne && e[j].key == e[i].key) ++j;
        int silhouette = 1;
        if (j - i == 2) {
            int ok0, ok1;
            vec3 n0 = unit_normal(m, (int64_t)(e[i].ref / 3), &ok0);
            vec3 n1 = unit_normal(m, (int64_t)(e[i + 1].ref / 3), &ok1);
            silhouette = !(ok0 && ok1 && vnorm(vcross(n0, n1)) <= 1e-4);
        }
        if (silhouette)
            for (int64_t q = i; q < j; ++q) m->sil[e[q].ref / 3] |= (uint8_t)(1u << (e[q].ref % 3));
        i = j;
    }
    free(e);
    free(tmp);
    free(count);
    return 0;
}

static void mesh_free(mesh_t *m)
{
    free(m->verts);
    free(m->tris);
    free(m->sil);
}

ORACLE_EXPORT void oracle_scene_destroy(oracle_scene *s)
{
    if (!s) return;
    mesh_free(&s->terrain);
    for (int l = 0; l < s->n_links; ++l) mesh_free(&s->links[l]);
    free(s->links);
    free(s);
}

/* Link meshes are given concatenated: link l owns verts [vo[l], vo[l+1]) and tris [to[l], to[l+1])
 * whose indices are local to the link. Returns NULL on bad input or allocation failure. */
ORACLE_EXPORT oracle_scene *oracle_scene_create(const float *terrain_verts, int64_t n_tverts,
                                                const int32_t *terrain_tris, int64_t n_ttris,
                                                const float *link_verts, const int64_t *link_vert_off,
                                                const int32_t *link_tris, const int64_t *link_tri_off,
                                                int32_t n_links)
{
    oracle_scene *s = (oracle_scene *)calloc(1, sizeof(oracle_scene));
    if (!s) return NULL;
    s->n_links = n_links;
    s->links = (mesh_t *)calloc((size_t)(n_links > 0 ? n_links : 1), sizeof(mesh_t));
    if (!s->links || mesh_init(&s->terrain, terrain_verts, n_tverts, terrain_tris, n_ttris) != 0) {
        oracle_scene_destroy(s);
        return NULL;
    }
    for (int l = 0; l < n_links; ++l) {
        int64_t v0 = link_vert_off[l], v1 = link_vert_off[l + 1];
        int64_t t0 = link_tri_off[l], t1 = link_tri_off[l + 1];
        if (mesh_init(&s->links[l], link_verts + 3 * v0, v1 - v0, link_tris + 3 * t0, t1 - t0) != 0) {
            oracle_scene_destroy(s);
            return NULL;
        }
    }
    return s;
}

/* ---------------------------------------------------------------------------------------------
 * Ray against one triangle: plane intersection plus closed inside test, both in FP64.
 * Returns 1 and the ray parameter t of the plane hit when the plane is met at t > 0
 * (inside or not), with *inside set when the point lies in the closed triangle.
 * ------------------------------------------------------------------------------------------- */
static int ray_plane_triangle(vec3 o, vec3 d, vec3 a, vec3 b, vec3 c, double *t_out, int *inside)
{
    vec3 n = vcross(vsub(b, a), vsub(c, a));
    double denom = vdot(n, d);
    if (denom == 0.0 || vdot(n, n) == 0.0) return 0;
    double t = vdot(n, vsub(a, o)) / denom;
    if (!(t > 0.0)) return 0;
    vec3 p = vadd(o, vscale(d, t));
    double ea = vdot(vcross(vsub(b, a), vsub(p, a)), n);
    double eb = vdot(vcross(vsub(c, b), vsub(p, b)), n);
    double ec = vdot(vcross(vsub(a, c), vsub(p, c)), n);
    *inside = (ea >= 0.0 && eb >= 0.0 && ec >= 0.0);
    *t_out = t;
    return 1;
}

/* Per-ray record of the nearest hit and of the silhouette proximity. */
typedef struct {
    vec3 o, d;
    double m;          /* depth per unit of t (1/|r| for z-depth, 1 for range) */
    double t_best;     /* nearest hit parameter, +inf if none */
    vec3 n_best;       /* unit normal of the nearest hit triangle */
} ray_t;

/* Pass 1: nearest hit over all triangles of one mesh placed by (R, t); R = NULL for the identity. */
static void mesh_closest(const mesh_t *m, const double *R, vec3 tr, ray_t *ray)
{
    for (int64_t i = 0; i < m->n_tris; ++i) {
        vec3 p[3];
        for (int k = 0; k < 3; ++k) {
            vec3 v = vert_of(m, m->tris[3 * i + k]);
            p[k] = R ? vadd(mat_vec(R, v), tr) : v;
        }
        double t;
        int inside;
        if (ray_plane_triangle(ray->o, ray->d, p[0], p[1], p[2], &t, &inside) && inside && t < ray->t_best) {
            vec3 n = vcross(vsub(p[1], p[0]), vsub(p[2], p[0]));
            ray->t_best = t;
            ray->n_best = vscale(n, 1.0 / vnorm(n));
        }
    }
}

/* Pass 2: smallest distance from a plane-hit point to a silhouette edge, over triangles whose plane
 * the ray meets no farther than depth z_lim; also reports the scale used for eps. */
static void mesh_silhouette(const mesh_t *m, const double *R, vec3 tr, const ray_t *ray, double z_lim,
                            double eps_probe, double *g_rel, double *g_abs)
{
    for (int64_t i = 0; i < m->n_tris; ++i) {
        if (!m->sil[i]) continue;
        vec3 p[3];
        for (int k = 0; k < 3; ++k) {
            vec3 v = vert_of(m, m->tris[3 * i + k]);
            p[k] = R ? vadd(mat_vec(R, v), tr) : v;
        }
        double t;
        int inside;
        if (!ray_plane_triangle(ray->o, ray->d, p[0], p[1], p[2], &t, &inside)) continue;
        if (ray->m * t > z_lim) continue;
        vec3 q = vadd(ray->o, vscale(ray->d, t));
        /* skip triangles whose box, grown by the probe radius, does not contain q */
        int far = 0;
        double qc[3] = {q.x, q.y, q.z};
        for (int ax = 0; ax < 3 && !far; ++ax) {
            double lo = ax == 0 ? p[0].x : ax == 1 ? p[0].y : p[0].z, hi = lo;
            for (int k = 1; k < 3; ++k) {
                double v = ax == 0 ? p[k].x : ax == 1 ? p[k].y : p[k].z;
                if (v < lo) lo = v;
                if (v > hi) hi = v;
            }
            if (qc[ax] < lo - eps_probe || qc[ax] > hi + eps_probe) far = 1;
        }
        if (far) continue;
        double scale = vmaxabs(ray->o);
        if (vmaxabs(q) > scale) scale = vmaxabs(q);
        double eps = 4.0 * ulp_f32(scale);
        if (eps < 1e-6) eps = 1e-6;
        for (int k = 0; k < 3; ++k) {
            if (!(m->sil[i] & (1u << k))) continue;
            double dist = point_segment_dist(q, p[k], p[(k + 1) % 3]);
            if (dist / eps < *g_rel) *g_rel = dist / eps;
            if (dist < *g_abs) *g_abs = dist;
        }
    }
}

/* ---------------------------------------------------------------------------------------------
 * Cameras and sensor
 * ------------------------------------------------------------------------------------------- */
/* cam_i [C,4] = (raw width, raw height, mount_link, downsample factor f >= 1);
 * cam_f [C,13] = (fx, fy, cx, cy, off_x, off_y, off_z, q_x, q_y, q_z, q_w, d_min, d_max). */
typedef struct {
    float sigma_abs, sigma_rel, p_drop, fill;
    int32_t max_latency;
    uint32_t seed[2];
    int32_t depth_kind;    /* 0 = z-depth (m t), 1 = range (t) */
} oracle_sensor;

enum {
    ORACLE_FLAG_EDGE = 1,        /* within eps_edge = max(1e-6, 4 ulp_f32(|coords|)) of a silhouette edge */
    ORACLE_FLAG_EDGE_1E6 = 2,    /* within 1e-6 m of a silhouette edge */
    ORACLE_FLAG_FAR = 4,         /* |z_raw - d_max| <= 1e-4: the hit-or-miss decision gating noise */
    ORACLE_FLAG_DROPPED = 8,     /* dropout replaced the pixel by `fill` */
    ORACLE_FLAG_GRAZING = 16,    /* the visible hit is so oblique that FP32 rounding of the ray alone can
                                    move the depth by more than 2.5e-5 m (a quarter of the tolerance) */
    ORACLE_FLAG_MASKED = 32,     /* side masking replaced the pixel by a uniform value */
};

/* Raw depth of one pixel from the poses of one step; fills flags bits 0..2 when want_flags. */
static double raw_depth(const oracle_scene *S, const int32_t *cam_i, const float *cam_f, int32_t C,
                        const float *intr_env, const float *mount_dr, const float *poses_step, int32_t L,
                        int32_t e, int32_t c, int32_t x, int32_t y, int32_t depth_kind, int want_flags,
                        int *flags)
{
    const float *cf = cam_f + 13 * c;
    double fx = cf[0], fy = cf[1], cx = cf[2], cy = cf[3];
    if (intr_env) {
        const float *k = intr_env + 4 * ((int64_t)e * C + c);
        fx = k[0]; fy = k[1]; cx = k[2]; cy = k[3];
    }
    double d_max = cf[12];
    int32_t mount = cam_i[4 * c + 2];

    /* 1. camera pose = mounting link pose composed with the mount offset */
    const float *lp = poses_step + 7 * ((int64_t)e * L + mount);
    double Rl[9], Roff[9], Rc[9];
    quat_to_mat(lp + 3, Rl);
    quat_to_mat(cf + 7, Roff);
    vec3 p_off = v3(cf[4], cf[5], cf[6]);
    if (mount_dr) {
        /* randomised mount: offset p_off + dp, rotation R(q_off) R(dq) */
        const float *dr = mount_dr + 7 * ((int64_t)e * C + c);
        double Rdq[9], Rm[9];
        quat_to_mat(dr + 3, Rdq);
        mat_mul(Roff, Rdq, Rm);
        memcpy(Roff, Rm, sizeof Rm);
        p_off = vadd(p_off, v3(dr[0], dr[1], dr[2]));
    }
    mat_mul(Rl, Roff, Rc);
    vec3 p_c = vadd(v3(lp[0], lp[1], lp[2]), mat_vec(Rl, p_off));

    /* 2. BuildDepthRay */
    vec3 r = v3((x - cx) / fx, (y - cy) / fy, 1.0);
    double rn = vnorm(r);
    ray_t ray;
    ray.o = p_c;
    ray.d = vscale(mat_vec(Rc, r), 1.0 / rn);
    ray.m = depth_kind == 0 ? 1.0 / rn : 1.0;
    ray.t_best = INFINITY;

    /* 3. closest hit over env e's links (placed in the world) and over the terrain */
    for (int32_t l = 0; l < S->n_links && l < L; ++l) {
        const float *bp = poses_step + 7 * ((int64_t)e * L + l);
        double Rb[9];
        quat_to_mat(bp + 3, Rb);
        mesh_closest(&S->links[l], Rb, v3(bp[0], bp[1], bp[2]), &ray);
    }
    mesh_closest(&S->terrain, NULL, v3(0, 0, 0), &ray);
    double z_hit = ray.m * ray.t_best;     /* +inf when nothing was hit */
    double z = z_hit < d_max ? z_hit : d_max;

    if (want_flags) {
        double g_rel = INFINITY, g_abs = INFINITY;
        double z_lim = z + 1e-3;
        /* every plane-hit point considered lies within |o| + z_lim/m of the origin, so a box test
         * with this radius never skips a triangle whose eps could reach the point */
        double probe = 4.0 * ulp_f32(vmaxabs(ray.o) + z_lim / ray.m);
        if (probe < 1e-6) probe = 1e-6;
        for (int32_t l = 0; l < S->n_links && l < L; ++l) {
            const float *bp = poses_step + 7 * ((int64_t)e * L + l);
            double Rb[9];
            quat_to_mat(bp + 3, Rb);
            mesh_silhouette(&S->links[l], Rb, v3(bp[0], bp[1], bp[2]), &ray, z_lim, probe, &g_rel, &g_abs);
        }
        mesh_silhouette(&S->terrain, NULL, v3(0, 0, 0), &ray, z_lim, probe, &g_rel, &g_abs);
        if (g_rel <= 1.0) *flags |= ORACLE_FLAG_EDGE;
        if (g_abs <= 1e-6) *flags |= ORACLE_FLAG_EDGE_1E6;
        if (fabs(z_hit - d_max) <= 1e-4) *flags |= ORACLE_FLAG_FAR;
        if (z_hit < d_max) {
            /* conditioning: a unit direction carried in FP32 is off by about 2^-22 rad, which moves a
             * hit at incidence cos c by (t + 1 m) 2^-22 sqrt(1 - c^2) / c along the ray */
            double c = fabs(vdot(ray.n_best, ray.d));
            double u = ray.m * (ray.t_best + 1.0) * ldexp(1.0, -22) * sqrt(fmax(0.0, 1.0 - c * c)) / fmax(c, 1e-300);
            if (u > 2.5e-5) *flags |= ORACLE_FLAG_GRAZING;
        }
    }
    return z;
}

/* Depth of output pixel (x, y) of camera c before the sensor: the raw depth when the camera is not
 * downsampled, else the mean of the f x f raw pixels (f x + i, f y + j); flags are OR-ed. */
static double image_depth(const oracle_scene *S, const int32_t *cam_i, const float *cam_f, int32_t C,
                          const float *intr_env, const float *mount_dr, const float *poses_step, int32_t L,
                          int32_t e, int32_t c, int32_t x, int32_t y, int32_t depth_kind, int want_flags,
                          int *flags)
{
    int32_t f = cam_i[4 * c + 3];
    if (f <= 1)
        return raw_depth(S, cam_i, cam_f, C, intr_env, mount_dr, poses_step, L, e, c, x, y, depth_kind,
                         want_flags, flags);
    double sum = 0.0;
    for (int32_t j = 0; j < f; ++j)
        for (int32_t i = 0; i < f; ++i)
            sum += raw_depth(S, cam_i, cam_f, C, intr_env, mount_dr, poses_step, L, e, c, f * x + i, f * y + j,
                             depth_kind, want_flags, flags);
    return sum / ((double)f * (double)f);
}

/*
 * Render the requested rays at step `step`.
 *   poses     [S,E,L,7] float32, poses[i] belongs to step step0 + i
 *   s_first   [E] first step of each env since its reset (NULL: all step0)
 *   rays      [N,4] int64 (e, c, x, y), (x, y) a pixel of the output (downsampled) image
 *   mount_dr  [E,C,7] float32 per-env mount perturbation (dp xyz, dq xyzw) or NULL
 *   rsm_mode  [E] uint8 side-mask mode (0 none, 1 small, 2 large; larger values count as 2) or NULL
 *   rsm_cols  [3] columns masked on each side for modes 0, 1, 2 (ignored when rsm_mode is NULL)
 *   outputs   depth [N] (sensor applied), raw [N] (z_raw of the source step), k [N], flags [N]
 * Returns 0, or -1 for a bad argument (a source step without poses, an index out of range).
 */
ORACLE_EXPORT int oracle_render(const oracle_scene *S, const int32_t *cam_i, const float *cam_f,
                                int32_t n_cams, const float *intr_env, const float *poses,
                                int64_t n_steps, int32_t n_envs, int32_t n_links, int64_t step0,
                                const int64_t *s_first, const oracle_sensor *sensor, int32_t env_offset,
                                const int64_t *rays, int64_t n_rays, int64_t step, int32_t want_flags,
                                const float *mount_dr, const uint8_t *rsm_mode, const int32_t *rsm_cols,
                                double *depth, double *raw, int32_t *k_out, int32_t *flags_out,
                                int32_t n_threads)
{
    for (int32_t c = 0; c < n_cams; ++c) {
        int32_t f = cam_i[4 * c + 3];
        if (f < 1 || cam_i[4 * c] % f != 0 || cam_i[4 * c + 1] % f != 0) return -1;
    }
    for (int64_t i = 0; i < n_rays; ++i) {
        const int64_t *q = rays + 4 * i;
        if (q[0] < 0 || q[0] >= n_envs || q[1] < 0 || q[1] >= n_cams) return -1;
        const int32_t *ci = cam_i + 4 * q[1];
        if (q[2] < 0 || q[2] >= ci[0] / ci[3] || q[3] < 0 || q[3] >= ci[1] / ci[3]) return -1;
        if (ci[2] < 0 || ci[2] >= n_links) return -1;
    }
    if (step < step0 || step >= step0 + n_steps) return -1;
    for (int32_t e = 0; e < n_envs; ++e)
        if (s_first && s_first[e] > step) return -1;
    int err = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const uint64_t span = (uint64_t)sensor->max_latency + 1u;
    double thr_d = floor((double)sensor->p_drop * 4294967296.0);
    if (thr_d < 0) thr_d = 0;
    if (thr_d > 4294967296.0) thr_d = 4294967296.0;
    const uint64_t drop_thr = (uint64_t)thr_d;
    const int64_t stride = (int64_t)n_envs * n_links * 7;

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_rays; ++i) {
        const int64_t *q = rays + 4 * i;
        int32_t e = (int32_t)q[0], c = (int32_t)q[1], x = (int32_t)q[2], y = (int32_t)q[3];
        int32_t W = cam_i[4 * c] / cam_i[4 * c + 3];   /* output width */
        const float *cf = cam_f + 13 * c;
        double d_min = cf[11], d_max = cf[12];
        uint32_t ge = (uint32_t)(env_offset + e);

        /* latency: one draw per (env, camera, step) */
        uint32_t w[4];
        keyed_words(ge, (uint32_t)c, 0xFFFFFFFFu, step, sensor->seed, w);
        int32_t k = (int32_t)(((uint64_t)w[0] * span) >> 32);
        int64_t sf = s_first ? s_first[e] : step0;
        int64_t src = step - k;
        if (src < sf) src = sf;
        if (src < step0) { err = 1; continue; }

        int flags = 0;
        double zr = image_depth(S, cam_i, cam_f, n_cams, intr_env, mount_dr, poses + (src - step0) * stride,
                                n_links, e, c, x, y, sensor->depth_kind, want_flags, &flags);

        /* noise, clip and dropout keyed by the source step */
        keyed_words(ge, (uint32_t)c, (uint32_t)(y * W + x), src, sensor->seed, w);
        double z = zr;
        if (zr < d_max) {
            double u1 = ((double)w[1] + 1.0) * (1.0 / 4294967296.0);
            double u2 = (double)w[2] * (1.0 / 4294967296.0);
            double n = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
            z = zr + ((double)sensor->sigma_abs + (double)sensor->sigma_rel * zr) * n;
        }
        if (z < d_min) z = d_min;
        if (z > d_max) z = d_max;
        if ((uint64_t)w[0] < drop_thr) {
            z = sensor->fill;
            flags |= ORACLE_FLAG_DROPPED;
        }
        if (rsm_mode) {
            /* side masking: the outer n columns on both sides, n by the env's mode */
            int32_t mode = rsm_mode[e] > 2 ? 2 : rsm_mode[e];
            int32_t n = rsm_cols[mode];
            if (x < n || x >= W - n) {
                keyed_words(ge, (uint32_t)c, (uint32_t)(y * W + x), step, sensor->seed, w);
                z = d_min + (d_max - d_min) * (((double)w[3] + 0.5) * (1.0 / 4294967296.0));
                flags |= ORACLE_FLAG_MASKED;
            }
        }
        depth[i] = z;
        if (raw) raw[i] = zr;
        if (k_out) k_out[i] = k;
        if (flags_out) flags_out[i] = flags;
    }
    return err ? -1 : 0;
}
