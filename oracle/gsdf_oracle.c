/*
 * Gradient-SDF CPU oracle -- TEST INFRASTRUCTURE ONLY (see gsdf_oracle.h).
 *
 * Plain restatement of the paper's definitions:
 *   Sec. 3.1, Eq. (sdf_update)       psi <- (W psi + w d)/(W + w),  W <- W + w
 *   Sec. 3.2, Eq. (gradient_update)  g <- g + w n,  ghat = g/|g|
 *   Sec. 4.1, Eq. (tracking)         E(R,t) = sum_k w_k d_S(R p_k + t)^2
 *   Sec. 4.1, Eq. (taylor)           d(p) = psi_j* + (p - v_j*)^T ghat_j*,  grad d = ghat_j*,
 *                                    j* = nearest grid voxel = round(p / v_s)
 *   Sec. 5.1                         Gauss-Newton, Cholesky solve of the normal equations
 *   Sec. 5.3                         pixel-driven integration: each pixel updates the voxels on
 *                                    its viewing ray within the truncation band; linear weight;
 *                                    depth cutoff 3.5 m; normals with angle to the ray < 75 deg.
 * Readings where the paper is silent (all stated in the header comments of each function):
 *   - inside-positive sign (Sec. 3.1): d(v) = z_v - D(u), z_v the camera-space depth of the voxel
 *     centre; normals oriented away from the camera;
 *   - ray sampling: samples z_k = D + (k - K) v_s/2, k = 0..2K, K = ceil(T / (v_s/2)), each sample
 *     rounded to its voxel; consecutive duplicates collapsed (a ray visits a voxel once);
 *   - linear weight: w = 1 for d <= eps, (T - d)/(T - eps) for eps < d <= T, none for |d| > T;
 *   - normals: cross product of central differences of back-projected neighbours;
 *   - tracking weight w_k: Huber with threshold delta, recomputed each Gauss-Newton step;
 *     a pixel whose nearest voxel is missing, has W = 0 or g = 0 is skipped;
 *   - pose update: left-multiplicative, T <- exp(xi^) T with xi = (omega, upsilon) = -H^-1 b.
 */
#include "gsdf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* per-voxel hash map (one voxel per entry, Sec. 5.1)                                          */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int32_t m[3];
    int32_t used;
    double psi;
    double g[3];
    double w;
} orc_entry;

struct orc_map {
    orc_params prm;
    int dense;
    int dims[3];
    int origin[3];
    orc_entry* tab;
    size_t cap; /* power of two */
    size_t count;
};

static uint64_t orc_hash(const int32_t m[3]) {
    uint64_t k = ((uint64_t)(uint32_t)m[0] * 0x9E3779B97F4A7C15ull) ^
                 ((uint64_t)(uint32_t)m[1] * 0xC2B2AE3D27D4EB4Full) ^
                 ((uint64_t)(uint32_t)m[2] * 0x165667B19E3779F9ull);
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    return k;
}

static orc_entry* orc_find(const orc_map* map, const int32_t m[3]) {
    size_t mask = map->cap - 1;
    size_t i = (size_t)orc_hash(m) & mask;
    for (;;) {
        orc_entry* e = &map->tab[i];
        if (!e->used) return NULL;
        if (e->m[0] == m[0] && e->m[1] == m[1] && e->m[2] == m[2]) return e;
        i = (i + 1) & mask;
    }
}

static int orc_grow(orc_map* map) {
    size_t ncap = map->cap * 2;
    orc_entry* nt = (orc_entry*)calloc(ncap, sizeof(orc_entry));
    if (!nt) return -1;
    for (size_t j = 0; j < map->cap; ++j) {
        if (!map->tab[j].used) continue;
        size_t i = (size_t)orc_hash(map->tab[j].m) & (ncap - 1);
        while (nt[i].used) i = (i + 1) & (ncap - 1);
        nt[i] = map->tab[j];
    }
    free(map->tab);
    map->tab = nt;
    map->cap = ncap;
    return 0;
}

/* find or insert a zero voxel (psi = 0, g = 0, W = 0) */
static orc_entry* orc_get(orc_map* map, const int32_t m[3]) {
    orc_entry* e = orc_find(map, m);
    if (e) return e;
    if (2 * (map->count + 1) > map->cap && orc_grow(map) != 0) return NULL;
    size_t mask = map->cap - 1;
    size_t i = (size_t)orc_hash(m) & mask;
    while (map->tab[i].used) i = (i + 1) & mask;
    e = &map->tab[i];
    memset(e, 0, sizeof(*e));
    e->m[0] = m[0];
    e->m[1] = m[1];
    e->m[2] = m[2];
    e->used = 1;
    map->count++;
    return e;
}

orc_map* orc_map_new(const orc_params* prm) {
    orc_map* map = (orc_map*)calloc(1, sizeof(orc_map));
    if (!map) return NULL;
    map->prm = *prm;
    map->cap = 1024;
    map->tab = (orc_entry*)calloc(map->cap, sizeof(orc_entry));
    if (!map->tab) {
        free(map);
        return NULL;
    }
    return map;
}

orc_map* orc_map_new_dense(const orc_params* prm, const int dims[3], const int origin[3]) {
    orc_map* map = orc_map_new(prm);
    if (!map) return NULL;
    map->dense = 1;
    for (int i = 0; i < 3; ++i) {
        map->dims[i] = dims[i];
        map->origin[i] = origin[i];
    }
    return map;
}

void orc_map_free(orc_map* map) {
    if (!map) return;
    free(map->tab);
    free(map);
}

size_t orc_map_count(const orc_map* map) {
    size_t n = 0;
    for (size_t i = 0; i < map->cap; ++i) n += map->tab[i].used && map->tab[i].w > 0.0;
    return n;
}

static int orc_in_dense(const orc_map* map, const int32_t m[3]) {
    if (!map->dense) return 1;
    for (int i = 0; i < 3; ++i)
        if (m[i] < map->origin[i] || m[i] >= map->origin[i] + map->dims[i]) return 0;
    return 1;
}

int orc_map_set_dense(orc_map* map, const float* psi, const float* g, const float* w) {
    if (!map->dense) return -1;
    size_t idx = 0;
    for (int z = 0; z < map->dims[2]; ++z)
        for (int y = 0; y < map->dims[1]; ++y)
            for (int x = 0; x < map->dims[0]; ++x, ++idx) {
                if (!(w[idx] > 0.0f)) continue;
                int32_t m[3] = {map->origin[0] + x, map->origin[1] + y, map->origin[2] + z};
                orc_entry* e = orc_get(map, m);
                if (!e) return -1;
                e->psi = psi[idx];
                e->g[0] = g[3 * idx + 0];
                e->g[1] = g[3 * idx + 1];
                e->g[2] = g[3 * idx + 2];
                e->w = w[idx];
            }
    return 0;
}

void orc_block_of(const int32_t m[3], int32_t b[3], int32_t local[3]) {
    for (int i = 0; i < 3; ++i) {
        int32_t q = m[i] >= 0 ? m[i] / 8 : -((-m[i] + 7) / 8); /* floor(m / 8) */
        b[i] = q;
        local[i] = m[i] - 8 * q;
    }
}

/* ------------------------------------------------------------------------------------------ */
/* FP32 index path                                                                             */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    float R[9], t[3];      /* camera -> world, rounded once from FP64 */
    float RT[9], tinv[3];  /* world -> camera: R^T and -R^T t (FP64, then rounded once) */
} orc_pose32;

static void orc_round_pose(const double T[16], orc_pose32* q) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            q->R[3 * i + j] = (float)T[4 * i + j];
            q->RT[3 * i + j] = (float)T[4 * j + i];
        }
        q->t[i] = (float)T[4 * i + 3];
        double s = T[0 * 4 + i] * T[3];
        s = s + T[1 * 4 + i] * T[7];
        s = s + T[2 * 4 + i] * T[11];
        q->tinv[i] = (float)(-s);
    }
}

/* j* of Eq. (taylor): nearest grid voxel, m = floor(P / v_s + 1/2) with 1/v_s rounded to FP32 */
static void orc_round_voxel(const float P[3], float inv_vs, int32_t m[3]) {
    for (int i = 0; i < 3; ++i) {
        float s = P[i] * inv_vs;
        s = s + 0.5f;
        m[i] = (int32_t)floorf(s);
    }
}

static int orc_depth_ok(float D, float dmax) { return D > 0.0f && D <= dmax; }

typedef struct {
    float ifx, ify, inv_vs;
} orc_recip;

static orc_recip orc_recips(const orc_intrinsics* K, float vs) {
    orc_recip r;
    r.ifx = (float)(1.0 / (double)K->fx);
    r.ify = (float)(1.0 / (double)K->fy);
    r.inv_vs = (float)(1.0 / (double)vs);
    return r;
}

/* back-projection of pixel (u, v) at depth z: z * ((u - cx)/fx, (v - cy)/fy, 1) */
static void orc_backproject(const orc_intrinsics* K, const orc_recip* rc, int u, int v, float z, float p[3]) {
    float xn = ((float)u - K->cx) * rc->ifx;
    float yn = ((float)v - K->cy) * rc->ify;
    p[0] = z * xn;
    p[1] = z * yn;
    p[2] = z;
}

/* world direction of pixel (u, v): d = R ray, ray = ((u - cx)/fx, (v - cy)/fy, 1);
 * d_i = (R_i0 ray_0 + R_i1 ray_1) + R_i2, each operation rounded to FP32 */
static void orc_ray_world(const orc_intrinsics* K, const orc_recip* rc, const float R[9], int u, int v, float d[3]) {
    float xn = ((float)u - K->cx) * rc->ifx;
    float yn = ((float)v - K->cy) * rc->ify;
    for (int i = 0; i < 3; ++i) {
        float a = R[3 * i + 0] * xn;
        float b = R[3 * i + 1] * yn;
        float s = a + b;
        d[i] = s + R[3 * i + 2];
    }
}

/* world point at depth z along that ray: P_i = z d_i + t_i (product, then sum, in FP32) */
static void orc_ray_point(const float d[3], const float t[3], float z, float P[3]) {
    for (int i = 0; i < 3; ++i) {
        float a = z * d[i];
        P[i] = a + t[i];
    }
}

void orc_pixel_point(const orc_intrinsics* K, const double T_wc[16], int u, int v, float D,
                     float P_out[3], int32_t m_out[3], float voxel_size) {
    orc_pose32 q;
    orc_round_pose(T_wc, &q);
    orc_recip rc = orc_recips(K, voxel_size);
    float d[3];
    orc_ray_world(K, &rc, q.R, u, v, d);
    orc_ray_point(d, q.t, D, P_out);
    orc_round_voxel(P_out, rc.inv_vs, m_out);
}

static float orc_dot32(const float a[3], const float b[3]) {
    float s = a[0] * b[0];
    s = s + a[1] * b[1];
    s = s + a[2] * b[2];
    return s;
}

/* Normal of pixel (u, v), Sec. 5.3 (75 degree filter).  Reading: central differences of the
 * back-projected 4-neighbours, n = (p_r - p_l) x (p_d - p_u), normalised, oriented so that
 * n . p > 0 (away from the camera, i.e. along the inside-positive SDF gradient).  Rejected at the
 * image border, if a neighbour is invalid or differs from the centre depth by more than T, if
 * the cross product vanishes, or if n . p / |p| < cos(75 deg). */
int orc_normal(const float* depth, const orc_intrinsics* K, const orc_params* prm, int u, int v,
               float n_out[3]) {
    const int W = K->width, H = K->height;
    if (u < 1 || u >= W - 1 || v < 1 || v >= H - 1) return 0;
    const float D = depth[(size_t)v * W + u];
    if (!orc_depth_ok(D, K->depth_max)) return 0;
    const float Dl = depth[(size_t)v * W + u - 1], Dr = depth[(size_t)v * W + u + 1];
    const float Du = depth[(size_t)(v - 1) * W + u], Dd = depth[(size_t)(v + 1) * W + u];
    const float nb[4] = {Dl, Dr, Du, Dd};
    for (int i = 0; i < 4; ++i) {
        if (!orc_depth_ok(nb[i], K->depth_max)) return 0;
        float diff = nb[i] - D;
        if (diff > prm->truncation || diff < -prm->truncation) return 0;
    }
    orc_recip rc = orc_recips(K, prm->voxel_size);
    float pl[3], pr[3], pu[3], pd[3], p[3];
    orc_backproject(K, &rc, u - 1, v, Dl, pl);
    orc_backproject(K, &rc, u + 1, v, Dr, pr);
    orc_backproject(K, &rc, u, v - 1, Du, pu);
    orc_backproject(K, &rc, u, v + 1, Dd, pd);
    orc_backproject(K, &rc, u, v, D, p);
    float a[3] = {pr[0] - pl[0], pr[1] - pl[1], pr[2] - pl[2]};
    float b[3] = {pd[0] - pu[0], pd[1] - pu[1], pd[2] - pu[2]};
    float n[3];
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    float nn = orc_dot32(n, n);
    if (!(nn > 0.0f)) return 0;
    float s = sqrtf(nn);
    n[0] = n[0] / s;
    n[1] = n[1] / s;
    n[2] = n[2] / s;
    float dp = orc_dot32(n, p);
    if (dp < 0.0f) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
        dp = -dp;
    }
    float c = dp / sqrtf(orc_dot32(p, p));
    if (!(c >= prm->cos_max_angle)) return 0;
    n_out[0] = n[0];
    n_out[1] = n[1];
    n_out[2] = n[2];
    return 1;
}

/* half-width K of the ray band in samples of v_s / 2: ceil(T / (v_s/2)), in FP64 with a 1e-6
 * guard so that T = 5 v_s gives exactly 10 */
static int orc_band_half(float vs, float T) {
    double h = (double)(0.5f * vs);
    return (int)ceil((double)T / h - 1e-6);
}

/* ------------------------------------------------------------------------------------------ */
/* integration: Eqs. (sdf_update), (gradient_update), pixel-driven as in Sec. 5.3             */
/* ------------------------------------------------------------------------------------------ */

int orc_integrate(orc_map* map, const float* depth, const orc_intrinsics* K, const double T_wc[16],
                  orc_integrate_stats* st) {
    const orc_params* prm = &map->prm;
    orc_pose32 q;
    orc_round_pose(T_wc, &q);
    orc_recip rc = orc_recips(K, prm->voxel_size);
    const float vs = prm->voxel_size, T = prm->truncation, eps = prm->weight_eps;
    const float h = 0.5f * vs;
    const int Kb = orc_band_half(vs, T);
    int64_t n_rays = 0, n_visits = 0;
    for (int v = 0; v < K->height; ++v) {
        for (int u = 0; u < K->width; ++u) {
            const float D = depth[(size_t)v * K->width + u];
            float n[3];
            if (!orc_normal(depth, K, prm, u, v, n)) continue; /* includes the depth test */
            n_rays++;
            /* world normal n_w = R n (values in FP64 from the FP32 rotation) */
            double nw[3];
            for (int i = 0; i < 3; ++i)
                nw[i] = (double)q.R[3 * i] * n[0] + (double)q.R[3 * i + 1] * n[1] + (double)q.R[3 * i + 2] * n[2];
            float dw[3];
            orc_ray_world(K, &rc, q.R, u, v, dw);
            int32_t prev[3] = {0, 0, 0};
            int have_prev = 0;
            for (int k = 0; k <= 2 * Kb; ++k) {
                float step = (float)(k - Kb) * h;
                float z = D + step;
                float P[3];
                orc_ray_point(dw, q.t, z, P);
                int32_t m[3];
                orc_round_voxel(P, rc.inv_vs, m);
                if (have_prev && m[0] == prev[0] && m[1] == prev[1] && m[2] == prev[2]) continue;
                prev[0] = m[0];
                prev[1] = m[1];
                prev[2] = m[2];
                have_prev = 1;
                /* distance estimate d(v) = z_v - D (projective, inside-positive) */
                float vc[3] = {(float)m[0] * vs, (float)m[1] * vs, (float)m[2] * vs};
                float zv = q.RT[6] * vc[0];
                zv = zv + q.RT[7] * vc[1];
                zv = zv + q.RT[8] * vc[2];
                zv = zv + q.tinv[2];
                float d = zv - D;
                if (d > T || d < -T) continue;
                if (!orc_in_dense(map, m)) continue;
                double w = (d <= eps) ? 1.0 : ((double)T - (double)d) / ((double)T - (double)eps);
                if (!(w > 0.0)) continue;
                orc_entry* e = orc_get(map, m);
                if (!e) return -1;
                /* Eq. (sdf_update) and Eq. (gradient_update), applied in ray order */
                e->psi = (e->w * e->psi + w * (double)d) / (e->w + w);
                e->w = e->w + w;
                e->g[0] += w * nw[0];
                e->g[1] += w * nw[1];
                e->g[2] += w * nw[2];
                n_visits++;
            }
        }
    }
    if (st) {
        st->n_rays = n_rays;
        st->n_visits = n_visits;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* tracking: Eq. (tracking) with the Taylor model Eq. (taylor)                                 */
/* ------------------------------------------------------------------------------------------ */

int orc_taylor(const orc_map* map, const double P[3], const int32_t m[3], double* r, double ghat[3]) {
    const orc_entry* e = orc_find(map, m);
    if (!e || !(e->w > 0.0)) return 1;
    double gn = sqrt(e->g[0] * e->g[0] + e->g[1] * e->g[1] + e->g[2] * e->g[2]);
    if (!(gn > 0.0)) return 1;
    const double vs = (double)map->prm.voxel_size;
    double s = e->psi;
    for (int i = 0; i < 3; ++i) {
        ghat[i] = e->g[i] / gn;
        s += ghat[i] * (P[i] - vs * (double)m[i]);
    }
    *r = s;
    return 0;
}

int orc_trilinear(const orc_map* map, const double P[3], const int32_t b[3], double* d, double grad[3]) {
    const double vs = (double)map->prm.voxel_size;
    double a[3], c[8];
    for (int k = 0; k < 3; ++k) a[k] = (P[k] - vs * (double)b[k]) / vs;
    for (int q = 0; q < 8; ++q) {
        const int32_t m[3] = {b[0] + (q & 1), b[1] + ((q >> 1) & 1), b[2] + ((q >> 2) & 1)};
        const orc_entry* e = orc_find(map, m);
        if (!e || !(e->w > 0.0)) return 1;
        c[q] = e->psi;
    }
    double s = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int q = 0; q < 8; ++q) {
        const int ix = q & 1, iy = (q >> 1) & 1, iz = (q >> 2) & 1;
        const double wx = ix ? a[0] : 1.0 - a[0], wy = iy ? a[1] : 1.0 - a[1], wz = iz ? a[2] : 1.0 - a[2];
        const double sx = ix ? 1.0 : -1.0, sy = iy ? 1.0 : -1.0, sz = iz ? 1.0 : -1.0;
        s += c[q] * wx * wy * wz;
        gx += c[q] * sx * wy * wz;
        gy += c[q] * wx * sy * wz;
        gz += c[q] * wx * wy * sz;
    }
    *d = s;
    grad[0] = gx / vs;
    grad[1] = gy / vs;
    grad[2] = gz / vs;
    return 0;
}

/* lowest corner of the interpolation cell of P on the FP32 index path: floor(P (1/v_s)) */
static void orc_cell(const float P[3], float inv_vs, int32_t b[3]) {
    for (int i = 0; i < 3; ++i) {
        const float s = P[i] * inv_vs;
        b[i] = (int32_t)floorf(s);
    }
}

int orc_track_reduce(const orc_map* map, const float* depth, const orc_intrinsics* K,
                     const double T_wc[16], orc_track_stats* st) {
    const orc_params* prm = &map->prm;
    orc_pose32 q;
    orc_round_pose(T_wc, &q);
    orc_recip rc = orc_recips(K, prm->voxel_size);
    const double delta = prm->huber_delta;
    double A[6][6] = {{0}};
    double b[6] = {0};
    double E = 0.0;
    int64_t n = 0, nh = 0;
    for (int v = 0; v < K->height; ++v) {
        for (int u = 0; u < K->width; ++u) {
            const float D = depth[(size_t)v * K->width + u];
            if (!orc_depth_ok(D, K->depth_max)) continue;
            float dw[3], Pf[3];
            int32_t m[3];
            orc_ray_world(K, &rc, q.R, u, v, dw);
            orc_ray_point(dw, q.t, D, Pf);
            double P[3] = {Pf[0], Pf[1], Pf[2]}, gh[3], r;
            if (prm->tracker == 1) {
                /* direct SDF baseline: trilinear d and its gradient (not normalised) */
                orc_cell(Pf, rc.inv_vs, m);
                if (orc_trilinear(map, P, m, &r, gh) != 0) continue;
            } else {
                orc_round_voxel(Pf, rc.inv_vs, m);
                if (orc_taylor(map, P, m, &r, gh) != 0) continue;
            }
            /* J = d r / d xi for T <- exp(xi^) T, xi = (omega, upsilon): (P x ghat, ghat), ghat
             * standing for the gradient of the residual's model (grad d for the trilinear one) */
            double J[6] = {P[1] * gh[2] - P[2] * gh[1], P[2] * gh[0] - P[0] * gh[2],
                           P[0] * gh[1] - P[1] * gh[0], gh[0], gh[1], gh[2]};
            double ar = fabs(r);
            double w = ar <= delta ? 1.0 : delta / ar;
            if (ar > delta) nh++;
            for (int i = 0; i < 6; ++i) {
                for (int j = i; j < 6; ++j) A[i][j] += w * J[i] * J[j];
                b[i] += w * J[i] * r;
            }
            E += w * r * r;
            n++;
        }
    }
    int idx = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) st->H[idx++] = A[i][j];
    for (int i = 0; i < 6; ++i) st->b[i] = b[i];
    st->energy = E;
    st->n_valid = n;
    st->n_huber = nh;
    st->status = 0;
    for (int i = 0; i < 6; ++i) st->xi[i] = 0.0;
    return 0;
}

/* Cholesky solve of (H + lambda I) xi = -b (Sec. 5.1).  lambda = damping * mean(diag H).
 * Degenerate (returns 1, xi = 0) if fewer than 6 residuals or a pivot <= 1e-12 max diag. */
int orc_solve6(const double H21[21], const double b[6], double damping, int64_t n_valid, double xi[6]) {
    double A[6][6];
    int idx = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) {
            A[i][j] = H21[idx];
            A[j][i] = H21[idx];
            idx++;
        }
    for (int i = 0; i < 6; ++i) xi[i] = 0.0;
    if (damping > 0.0) {
        double tr = 0.0;
        for (int i = 0; i < 6; ++i) tr += A[i][i];
        double lam = damping * tr / 6.0;
        for (int i = 0; i < 6; ++i) A[i][i] += lam;
    }
    if (n_valid < 6) return 1;
    double maxd = 0.0;
    for (int i = 0; i < 6; ++i) maxd = A[i][i] > maxd ? A[i][i] : maxd;
    if (!(maxd > 0.0)) return 1;
    double L[6][6] = {{0}};
    for (int j = 0; j < 6; ++j) {
        double s = A[j][j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 1e-12 * maxd)) return 1;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < 6; ++i) {
            double t = A[i][j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double t = -b[i];
        for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
        y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < 6; ++k) t -= L[k][i] * xi[k];
        xi[i] = t / L[i][i];
    }
    return 0;
}

/* SE(3) exponential of xi = (omega, upsilon): R by Rodrigues, t = V upsilon with
 * V = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2 (series for small th) */
void orc_se3_exp(const double xi[6], double T[16]) {
    const double* w = xi;
    const double* u = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-4) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    double Wx[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    double W2[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Wx[i][k] * Wx[k][j];
            W2[i][j] = s;
        }
    double R[3][3], V[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double I = (i == j) ? 1.0 : 0.0;
            R[i][j] = I + A * Wx[i][j] + B * W2[i][j];
            V[i][j] = I + B * Wx[i][j] + C * W2[i][j];
        }
    memset(T, 0, 16 * sizeof(double));
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) T[4 * i + j] = R[i][j];
        T[4 * i + 3] = V[i][0] * u[0] + V[i][1] * u[1] + V[i][2] * u[2];
    }
    T[15] = 1.0;
}

int orc_track_step(const orc_map* map, const float* depth, const orc_intrinsics* K, double T_wc[16],
                   orc_track_stats* st) {
    orc_track_reduce(map, depth, K, T_wc, st);
    double xi[6];
    int bad = orc_solve6(st->H, st->b, map->prm.damping, st->n_valid, xi);
    st->status = bad;
    for (int i = 0; i < 6; ++i) st->xi[i] = xi[i];
    if (bad) return 0;
    double dT[16], Tn[16];
    orc_se3_exp(xi, dT);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += dT[4 * i + k] * T_wc[4 * k + j];
            Tn[4 * i + j] = s;
        }
    memcpy(T_wc, Tn, sizeof(Tn));
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* extraction                                                                                  */
/* ------------------------------------------------------------------------------------------ */

static int orc_cmp_voxel(const void* pa, const void* pb) {
    const orc_voxel_out* a = (const orc_voxel_out*)pa;
    const orc_voxel_out* b = (const orc_voxel_out*)pb;
    for (int i = 0; i < 3; ++i) {
        if (a->m[i] < b->m[i]) return -1;
        if (a->m[i] > b->m[i]) return 1;
    }
    return 0;
}

size_t orc_extract(const orc_map* map, orc_voxel_out* out, size_t cap) {
    size_t n = 0;
    for (size_t i = 0; i < map->cap; ++i) {
        const orc_entry* e = &map->tab[i];
        if (!e->used || !(e->w > 0.0)) continue;
        if (n < cap) {
            orc_voxel_out* o = &out[n];
            o->m[0] = e->m[0];
            o->m[1] = e->m[1];
            o->m[2] = e->m[2];
            o->psi = e->psi;
            o->g[0] = e->g[0];
            o->g[1] = e->g[1];
            o->g[2] = e->g[2];
            o->w = e->w;
        }
        n++;
    }
    size_t k = n < cap ? n : cap;
    qsort(out, k, sizeof(orc_voxel_out), orc_cmp_voxel);
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* photometric + geometric voxel energy (Sec. 4.2) and its gradient                            */
/* ------------------------------------------------------------------------------------------ */

/* surface point p = v - psi ghat of voxel j (Eq. grad_sdf_project); 0 if g = 0 */
static int orc_surface_point(const int32_t* m, const double* psi, const double* g, int64_t j, double vs,
                             double p[3], double gh[3], double* gn) {
    const double* gj = g + 3 * j;
    double n = sqrt(gj[0] * gj[0] + gj[1] * gj[1] + gj[2] * gj[2]);
    if (!(n > 0.0)) return 0;
    for (int k = 0; k < 3; ++k) {
        gh[k] = gj[k] / n;
        p[k] = vs * (double)m[3 * j + k] - psi[j] * gh[k];
    }
    *gn = n;
    return 1;
}

/* camera coordinates x = R^T (p - t) of a world point for pose T (camera -> world) */
static void orc_to_camera(const double* T, const double p[3], double x[3]) {
    const double d[3] = {p[0] - T[3], p[1] - T[7], p[2] - T[11]};
    for (int i = 0; i < 3; ++i) x[i] = T[0 * 4 + i] * d[0] + T[1 * 4 + i] * d[1] + T[2 * 4 + i] * d[2];
}

/* FP32 index path of the energy's pixel decisions for voxel j in a keyframe: the surface point,
 * its camera coordinates and its projection, every operation rounded to FP32 in the order
 * written, from psi and g rounded to FP32 and the pose rounded once (orc_round_pose):
 *   n2 = (g0 g0 + g1 g1) + g2 g2,  ghat_k = g_k / sqrt(n2),  s_k = psi ghat_k,  p_k = v_s m_k - s_k
 *   d = p - t,  x_i = (R_0i d_0 + R_1i d_1) + R_2i d_2,  u = (f_x x_0) / x_2 + c_x,  v likewise.
 * Returns 0 if g rounds to zero or the point is not in front of the camera (x_2 <= 0). */
typedef struct {
    float s[3], x[3], u, v;
} orc_proj32;

static int orc_project32(const int32_t* m, const double* psi, const double* g, int64_t j, float vs,
                         const orc_pose32* q, const orc_intrinsics* K, orc_proj32* o) {
    const float gj[3] = {(float)g[3 * j], (float)g[3 * j + 1], (float)g[3 * j + 2]};
    const float ps = (float)psi[j];
    float n2 = gj[0] * gj[0];
    n2 = n2 + gj[1] * gj[1];
    n2 = n2 + gj[2] * gj[2];
    if (!(n2 > 0.0f)) return 0;
    const float nr = sqrtf(n2);
    float d[3];
    for (int k = 0; k < 3; ++k) {
        const float gh = gj[k] / nr;
        o->s[k] = ps * gh;
        const float v = vs * (float)m[3 * j + k];
        const float p = v - o->s[k];
        d[k] = p - q->t[k];
    }
    for (int i = 0; i < 3; ++i) {
        float a = q->R[0 * 3 + i] * d[0];
        a = a + q->R[1 * 3 + i] * d[1];
        o->x[i] = a + q->R[2 * 3 + i] * d[2];
    }
    if (!(o->x[2] > 0.0f)) return 0;
    o->u = (K->fx * o->x[0]) / o->x[2] + K->cx;
    o->v = (K->fy * o->x[1]) / o->x[2] + K->cy;
    return 1;
}

void orc_visibility(int64_t n, const int32_t* m, const double* psi, const double* g, float voxel_size, int n_frames,
                    const orc_intrinsics* K, const double* poses, const float* const* depth, uint8_t* nu) {
    const float vs = voxel_size, half = 0.5f * voxel_size;
    for (int i = 0; i < n_frames; ++i) {
        orc_pose32 q;
        orc_round_pose(poses + 16 * i, &q);
        for (int64_t j = 0; j < n; ++j) {
            uint8_t vis = 0;
            orc_proj32 o;
            if (orc_project32(m, psi, g, j, vs, &q, K, &o)) {
                const int surface = fabsf(o.s[0]) <= half && fabsf(o.s[1]) <= half && fabsf(o.s[2]) <= half;
                if (surface && o.u >= 1.0f && o.u <= (float)(K->width - 2) && o.v >= 1.0f &&
                    o.v <= (float)(K->height - 2)) {
                    const int iu = (int)floorf(o.u + 0.5f), iv = (int)floorf(o.v + 0.5f);
                    const float D = depth[i][(size_t)iv * K->width + iu];
                    if (orc_depth_ok(D, K->depth_max) && fabsf(o.x[2] - D) <= vs) vis = 1;
                }
            }
            nu[(size_t)i * n + j] = vis;
        }
    }
}

typedef struct {
    int32_t m[3];
    int64_t idx;
} orc_key_index;

static int orc_cmp_key(const void* pa, const void* pb) {
    const orc_key_index* a = (const orc_key_index*)pa;
    const orc_key_index* b = (const orc_key_index*)pb;
    for (int k = 0; k < 3; ++k) {
        if (a->m[k] < b->m[k]) return -1;
        if (a->m[k] > b->m[k]) return 1;
    }
    return 0;
}

int orc_energy(int64_t n, const int32_t* m, const double* psi, const double* g, const double* rho, float voxel_size,
               int n_frames, const orc_intrinsics* K, const double* poses, const float* const* rgb,
               const float* const* depth, const uint8_t* nu, double lambda_geo, double E[3], double* dpsi,
               double* dg, double* drho, double* dxi, double* dT) {
    const double vs = (double)voxel_size;
    const int grad = dpsi != NULL;
    const int Wd = K->width, Hd = K->height;
    if (grad) {
        for (int64_t j = 0; j < n; ++j) {
            dpsi[j] = 0.0;
            for (int k = 0; k < 3; ++k) dg[3 * j + k] = drho[3 * j + k] = 0.0;
        }
        for (int k = 0; k < 6 * n_frames; ++k) dxi[k] = 0.0;
        if (dT)
            for (int k = 0; k < 16 * n_frames; ++k) dT[k] = 0.0;
    }
    double Ep = 0.0, Eg = 0.0;
    /* photometric term, Eqs. (rgb_cost), (intensity_proj) with an explicit colour rho_j */
    for (int i = 0; i < n_frames; ++i) {
        const double* T = poses + 16 * i;
        const float* img = rgb[i];
        orc_pose32 q32;
        orc_round_pose(T, &q32);
        for (int64_t j = 0; j < n; ++j) {
            if (!nu[(size_t)i * n + j]) continue;
            /* decisions on the FP32 index path: the pair counts while its point projects into the
             * image at the evaluated pose; the bilinear cell is (floor u, floor v), kept inside */
            orc_proj32 o;
            if (!orc_project32(m, psi, g, j, voxel_size, &q32, K, &o)) continue;
            if (!(o.u >= 0.0f && o.u <= (float)(Wd - 1) && o.v >= 0.0f && o.v <= (float)(Hd - 1))) continue;
            int x0 = (int)floorf(o.u), y0 = (int)floorf(o.v);
            if (x0 > Wd - 2) x0 = Wd - 2;
            if (y0 > Hd - 2) y0 = Hd - 2;
            /* values in FP64 */
            double p[3], gh[3], gn, x[3];
            if (!orc_surface_point(m, psi, g, j, vs, p, gh, &gn)) continue;
            orc_to_camera(T, p, x);
            const double z = x[2];
            const double u = K->fx * x[0] / z + K->cx, v = K->fy * x[1] / z + K->cy;
            const double a = u - x0, b = v - y0;
            double dEdu = 0.0, dEdv = 0.0;
            for (int c = 0; c < 3; ++c) {
                const double I00 = img[((size_t)y0 * Wd + x0) * 3 + c], I01 = img[((size_t)y0 * Wd + x0 + 1) * 3 + c];
                const double I10 = img[((size_t)(y0 + 1) * Wd + x0) * 3 + c];
                const double I11 = img[((size_t)(y0 + 1) * Wd + x0 + 1) * 3 + c];
                const double I = (1 - a) * (1 - b) * I00 + a * (1 - b) * I01 + (1 - a) * b * I10 + a * b * I11;
                const double r = I - rho[3 * j + c];
                Ep += r * r;
                if (grad) {
                    drho[3 * j + c] -= 2.0 * r;
                    dEdu += 2.0 * r * ((1 - b) * (I01 - I00) + b * (I11 - I10));
                    dEdv += 2.0 * r * ((1 - a) * (I10 - I00) + a * (I11 - I01));
                }
            }
            if (!grad) continue;
            /* chain rule: (u, v) <- x (pinhole) <- p (x = R^T (p - t)) <- (psi, g) and the pose */
            const double dx[3] = {dEdu * K->fx / z, dEdv * K->fy / z,
                                  -(dEdu * K->fx * x[0] + dEdv * K->fy * x[1]) / (z * z)};
            double q[3];  /* dE/dp = R dE/dx */
            for (int r_ = 0; r_ < 3; ++r_) q[r_] = T[4 * r_ + 0] * dx[0] + T[4 * r_ + 1] * dx[1] + T[4 * r_ + 2] * dx[2];
            const double qg = q[0] * gh[0] + q[1] * gh[1] + q[2] * gh[2];
            dpsi[j] += -qg;                                            /* dp/dpsi = -ghat */
            for (int k = 0; k < 3; ++k) dg[3 * j + k] += -psi[j] * (q[k] - gh[k] * qg) / gn;  /* dghat/dg */
            /* left perturbation of the pose: dx/domega = R^T [p]x, dx/dupsilon = -R^T */
            double* dx_i = dxi + 6 * i;
            dx_i[0] += q[1] * p[2] - q[2] * p[1];
            dx_i[1] += q[2] * p[0] - q[0] * p[2];
            dx_i[2] += q[0] * p[1] - q[1] * p[0];
            dx_i[3] -= q[0];
            dx_i[4] -= q[1];
            dx_i[5] -= q[2];
            if (dT) { /* entries of T: dE/dR_ab = (p - t)_a dE/dx_b, dE/dt = -R dE/dx */
                double* G = dT + 16 * i;
                for (int a_ = 0; a_ < 3; ++a_) {
                    const double pa = p[a_] - T[4 * a_ + 3];
                    for (int b_ = 0; b_ < 3; ++b_) G[4 * a_ + b_] += pa * dx[b_];
                    G[4 * a_ + 3] -= q[a_];
                }
            }
        }
    }
    /* geometric term, Eq. (tracking) with Eq. (taylor), squared residuals, every keyframe */
    orc_key_index* keys = (orc_key_index*)malloc(sizeof(orc_key_index) * (size_t)(n > 0 ? n : 1));
    if (!keys) return -1;
    for (int64_t j = 0; j < n; ++j) {
        keys[j].m[0] = m[3 * j];
        keys[j].m[1] = m[3 * j + 1];
        keys[j].m[2] = m[3 * j + 2];
        keys[j].idx = j;
    }
    qsort(keys, (size_t)n, sizeof(orc_key_index), orc_cmp_key);
    orc_recip rc = orc_recips(K, voxel_size);
    for (int i = 0; i < n_frames && lambda_geo != 0.0; ++i) {
        orc_pose32 q32;
        orc_round_pose(poses + 16 * i, &q32);
        for (int v = 0; v < Hd; ++v) {
            for (int u = 0; u < Wd; ++u) {
                const float D = depth[i][(size_t)v * Wd + u];
                if (!orc_depth_ok(D, K->depth_max)) continue;
                float dw[3], Pf[3];
                orc_key_index key;
                orc_ray_world(K, &rc, q32.R, u, v, dw);
                orc_ray_point(dw, q32.t, D, Pf);
                orc_round_voxel(Pf, rc.inv_vs, key.m);
                const orc_key_index* hit = (const orc_key_index*)bsearch(&key, keys, (size_t)n, sizeof(orc_key_index),
                                                                         orc_cmp_key);
                if (!hit) continue;
                const int64_t j = hit->idx;
                const double* gj = g + 3 * j;
                const double gn = sqrt(gj[0] * gj[0] + gj[1] * gj[1] + gj[2] * gj[2]);
                if (!(gn > 0.0)) continue;
                const double P[3] = {Pf[0], Pf[1], Pf[2]};
                double gh[3], d[3], r = psi[j];
                for (int k = 0; k < 3; ++k) {
                    gh[k] = gj[k] / gn;
                    d[k] = P[k] - vs * (double)key.m[k];
                    r += gh[k] * d[k];
                }
                Eg += r * r;
                if (!grad) continue;
                const double s = 2.0 * lambda_geo * r;
                dpsi[j] += s;
                const double gd = gh[0] * d[0] + gh[1] * d[1] + gh[2] * d[2];
                for (int k = 0; k < 3; ++k) dg[3 * j + k] += s * (d[k] - gh[k] * gd) / gn;
                double* dx_i = dxi + 6 * i;
                dx_i[0] += s * (P[1] * gh[2] - P[2] * gh[1]);
                dx_i[1] += s * (P[2] * gh[0] - P[0] * gh[2]);
                dx_i[2] += s * (P[0] * gh[1] - P[1] * gh[0]);
                dx_i[3] += s * gh[0];
                dx_i[4] += s * gh[1];
                dx_i[5] += s * gh[2];
                if (dT) { /* P = R p_c + t with the camera point p_c = D ((u - c_x)/f_x, (v - c_y)/f_y, 1) */
                    const double pc[3] = {D * ((u - (double)K->cx) / K->fx), D * ((v - (double)K->cy) / K->fy), D};
                    double* G = dT + 16 * i;
                    for (int a_ = 0; a_ < 3; ++a_) {
                        for (int b_ = 0; b_ < 3; ++b_) G[4 * a_ + b_] += s * gh[a_] * pc[b_];
                        G[4 * a_ + 3] += s * gh[a_];
                    }
                }
            }
        }
    }
    free(keys);
    E[0] = Ep + lambda_geo * Eg;
    E[1] = Ep;
    E[2] = Eg;
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* photometric bundle adjustment step (Sec. 4.2)                                                */
/* ------------------------------------------------------------------------------------------ */

/* Colour and its image gradient at the projection of voxel j in keyframe i, if the pair counts:
 * FP32 index path for the decisions (orc_project32, in-image test, cell), FP64 values.  Returns 0
 * if the pair does not count.  p, gh: the surface point and ghat; x: camera coordinates. */
static int orc_pair_colour(const int32_t* m, const double* psi, const double* g, int64_t j, float voxel_size,
                           const double* T, const orc_pose32* q32, const orc_intrinsics* K, const float* img,
                           double I[3], double dIdu[3], double dIdv[3], double p[3], double gh[3], double x[3]) {
    const int Wd = K->width, Hd = K->height;
    orc_proj32 o;
    if (!orc_project32(m, psi, g, j, voxel_size, q32, K, &o)) return 0;
    if (!(o.u >= 0.0f && o.u <= (float)(Wd - 1) && o.v >= 0.0f && o.v <= (float)(Hd - 1))) return 0;
    int x0 = (int)floorf(o.u), y0 = (int)floorf(o.v);
    if (x0 > Wd - 2) x0 = Wd - 2;
    if (y0 > Hd - 2) y0 = Hd - 2;
    double gn;
    if (!orc_surface_point(m, psi, g, j, (double)voxel_size, p, gh, &gn)) return 0;
    orc_to_camera(T, p, x);
    const double u = K->fx * x[0] / x[2] + K->cx, v = K->fy * x[1] / x[2] + K->cy;
    const double a = u - x0, b = v - y0;
    for (int c = 0; c < 3; ++c) {
        const double I00 = img[((size_t)y0 * Wd + x0) * 3 + c], I01 = img[((size_t)y0 * Wd + x0 + 1) * 3 + c];
        const double I10 = img[((size_t)(y0 + 1) * Wd + x0) * 3 + c];
        const double I11 = img[((size_t)(y0 + 1) * Wd + x0 + 1) * 3 + c];
        I[c] = (1 - a) * (1 - b) * I00 + a * (1 - b) * I01 + (1 - a) * b * I10 + a * b * I11;
        dIdu[c] = (1 - b) * (I01 - I00) + b * (I11 - I10);
        dIdv[c] = (1 - a) * (I10 - I00) + a * (I11 - I01);
    }
    return 1;
}

static void orc_add_normal(double A[6][6], double bb[6], const double J[6], double r, double w) {
    for (int i = 0; i < 6; ++i) {
        for (int k = i; k < 6; ++k) A[i][k] += w * J[i] * J[k];
        bb[i] += w * J[i] * r;
    }
}

int orc_ba_step(int64_t n, const int32_t* m, double* psi, const double* g, double* rho, float voxel_size, int n_frames,
                const orc_intrinsics* K, double* poses, const float* const* rgb, const float* const* depth,
                const uint8_t* nu, double lambda_geo, double damping, int flags, orc_track_stats* st, double* psi_H,
                double* psi_b) {
    const double vs = (double)voxel_size;
    double* sum = (double*)calloc((size_t)(n > 0 ? n : 1) * 4, sizeof(double));
    double* hp = (double*)calloc((size_t)(n > 0 ? n : 1) * 2, sizeof(double));
    orc_key_index* keys = (orc_key_index*)malloc(sizeof(orc_key_index) * (size_t)(n > 0 ? n : 1));
    if (!sum || !hp || !keys) {
        free(sum);
        free(hp);
        free(keys);
        return -1;
    }
    /* 1. mean colour, Eq. (mean_color), over the pairs that count */
    for (int i = 0; i < n_frames; ++i) {
        orc_pose32 q32;
        orc_round_pose(poses + 16 * i, &q32);
        for (int64_t j = 0; j < n; ++j) {
            if (!nu[(size_t)i * n + j]) continue;
            double I[3], du[3], dv[3], p[3], gh[3], x[3];
            if (!orc_pair_colour(m, psi, g, j, voxel_size, poses + 16 * i, &q32, K, rgb[i], I, du, dv, p, gh, x))
                continue;
            for (int c = 0; c < 3; ++c) sum[4 * j + c] += I[c];
            sum[4 * j + 3] += 1.0;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int c = 0; c < 3; ++c) rho[3 * j + c] = sum[4 * j + 3] > 0.0 ? sum[4 * j + c] / sum[4 * j + 3] : 0.0;
    /* 2. Gauss-Newton terms with rho fixed (the decoupled energies of Eq. rgb_cost_pose) */
    for (int64_t j = 0; j < n; ++j) {
        keys[j].m[0] = m[3 * j];
        keys[j].m[1] = m[3 * j + 1];
        keys[j].m[2] = m[3 * j + 2];
        keys[j].idx = j;
    }
    qsort(keys, (size_t)n, sizeof(orc_key_index), orc_cmp_key);
    const orc_recip rc = orc_recips(K, voxel_size);
    for (int i = 0; i < n_frames; ++i) {
        const double* T = poses + 16 * i;
        orc_pose32 q32;
        orc_round_pose(T, &q32);
        double A[6][6] = {{0}}, bb[6] = {0}, E = 0.0;
        int64_t nres = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (!nu[(size_t)i * n + j]) continue;
            double I[3], du[3], dv[3], p[3], gh[3], x[3];
            if (!orc_pair_colour(m, psi, g, j, voxel_size, T, &q32, K, rgb[i], I, du, dv, p, gh, x)) continue;
            const double z = x[2];
            for (int c = 0; c < 3; ++c) {
                const double r = I[c] - rho[3 * j + c];
                /* dI/dx through the pinhole, then q = R dI/dx = dI/dp */
                const double dx[3] = {du[c] * K->fx / z, dv[c] * K->fy / z,
                                      -(du[c] * K->fx * x[0] + dv[c] * K->fy * x[1]) / (z * z)};
                double qv[3];
                for (int r_ = 0; r_ < 3; ++r_)
                    qv[r_] = T[4 * r_ + 0] * dx[0] + T[4 * r_ + 1] * dx[1] + T[4 * r_ + 2] * dx[2];
                /* left perturbation: dp_cam/domega via x = R^T (p - t): dI/domega = q x p, dI/dupsilon = -q */
                const double J[6] = {qv[1] * p[2] - qv[2] * p[1], qv[2] * p[0] - qv[0] * p[2],
                                     qv[0] * p[1] - qv[1] * p[0], -qv[0], -qv[1], -qv[2]};
                orc_add_normal(A, bb, J, r, 1.0);
                E += r * r;
                ++nres;
                const double jp = -(qv[0] * gh[0] + qv[1] * gh[1] + qv[2] * gh[2]); /* dp/dpsi = -ghat */
                hp[2 * j] += jp * jp;
                hp[2 * j + 1] += jp * r;
            }
        }
        for (int v = 0; v < K->height && lambda_geo != 0.0; ++v) {
            for (int u = 0; u < K->width; ++u) {
                const float D = depth[i][(size_t)v * K->width + u];
                if (!orc_depth_ok(D, K->depth_max)) continue;
                float dw[3], Pf[3];
                orc_key_index key;
                orc_ray_world(K, &rc, q32.R, u, v, dw);
                orc_ray_point(dw, q32.t, D, Pf);
                orc_round_voxel(Pf, rc.inv_vs, key.m);
                const orc_key_index* hit =
                    (const orc_key_index*)bsearch(&key, keys, (size_t)n, sizeof(orc_key_index), orc_cmp_key);
                if (!hit) continue;
                const int64_t j = hit->idx;
                const double* gj = g + 3 * j;
                const double gn = sqrt(gj[0] * gj[0] + gj[1] * gj[1] + gj[2] * gj[2]);
                if (!(gn > 0.0)) continue;
                const double P[3] = {Pf[0], Pf[1], Pf[2]};
                double gh[3], r = psi[j];
                for (int k = 0; k < 3; ++k) {
                    gh[k] = gj[k] / gn;
                    r += gh[k] * (P[k] - vs * (double)key.m[k]);
                }
                const double J[6] = {P[1] * gh[2] - P[2] * gh[1], P[2] * gh[0] - P[0] * gh[2],
                                     P[0] * gh[1] - P[1] * gh[0], gh[0], gh[1], gh[2]};
                orc_add_normal(A, bb, J, r, lambda_geo);
                E += lambda_geo * r * r;
                ++nres;
                hp[2 * j] += lambda_geo; /* dr/dpsi = 1 */
                hp[2 * j + 1] += lambda_geo * r;
            }
        }
        orc_track_stats* s = st + i;
        int idx = 0;
        for (int a = 0; a < 6; ++a)
            for (int k = a; k < 6; ++k) s->H[idx++] = A[a][k];
        for (int a = 0; a < 6; ++a) {
            s->b[a] = bb[a];
            s->xi[a] = 0.0;
        }
        s->energy = E;
        s->n_valid = nres;
        s->n_huber = 0;
        s->status = 0;
    }
    /* 3. updates */
    for (int i = 0; i < n_frames && (flags & ORC_BA_POSES); ++i) {
        orc_track_stats* s = st + i;
        double xi[6];
        s->status = orc_solve6(s->H, s->b, damping, s->n_valid, xi);
        for (int a = 0; a < 6; ++a) s->xi[a] = xi[a];
        if (s->status) continue;
        double dT[16], Tn[16];
        double* T = poses + 16 * i;
        orc_se3_exp(xi, dT);
        for (int a = 0; a < 4; ++a)
            for (int k = 0; k < 4; ++k) {
                double acc = 0.0;
                for (int l = 0; l < 4; ++l) acc += dT[4 * a + l] * T[4 * l + k];
                Tn[4 * a + k] = acc;
            }
        memcpy(T, Tn, sizeof(Tn));
    }
    for (int64_t j = 0; j < n; ++j) {
        if (psi_H) psi_H[j] = hp[2 * j];
        if (psi_b) psi_b[j] = hp[2 * j + 1];
        if ((flags & ORC_BA_PSI) && hp[2 * j] > 0.0) psi[j] -= hp[2 * j + 1] / ((1.0 + damping) * hp[2 * j]);
    }
    free(sum);
    free(hp);
    free(keys);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* oriented point cloud and its 2x2x2 upsampling (Sec. 4.3)                                    */
/* ------------------------------------------------------------------------------------------ */

size_t orc_points(int64_t n, const int32_t* m, const double* psi, const double* g, float voxel_size, int level,
                  orc_point* out, size_t cap) {
    const float half = 0.5f * voxel_size, quarter = 0.25f * voxel_size;
    const double vs64 = (double)voxel_size;
    size_t count = 0;
    for (int64_t j = 0; j < n; ++j) {
        /* FP32 index path: ghat and psi ghat of the voxel */
        const float gj[3] = {(float)g[3 * j], (float)g[3 * j + 1], (float)g[3 * j + 2]};
        const float ps = (float)psi[j];
        float n2 = gj[0] * gj[0];
        n2 = n2 + gj[1] * gj[1];
        n2 = n2 + gj[2] * gj[2];
        if (!(n2 > 0.0f)) continue;
        const float nr = sqrtf(n2);
        float gh[3];
        for (int k = 0; k < 3; ++k) gh[k] = gj[k] / nr;
        /* FP64 values */
        const double* g64 = g + 3 * j;
        const double gn = sqrt(g64[0] * g64[0] + g64[1] * g64[1] + g64[2] * g64[2]);
        const double gh64[3] = {g64[0] / gn, g64[1] / gn, g64[2] / gn};
        if (level == 0) {
            int keep = 1;
            for (int k = 0; k < 3; ++k) {
                const float sk = ps * gh[k];
                keep &= fabsf(sk) <= half;
            }
            if (!keep) continue;
            if (count < cap) {
                orc_point* o = out + count;
                o->sub = -1;
                for (int k = 0; k < 3; ++k) {
                    o->m[k] = m[3 * j + k];
                    o->p[k] = vs64 * (double)m[3 * j + k] - psi[j] * gh64[k];
                    o->n[k] = -gh64[k];
                }
            }
            ++count;
            continue;
        }
        for (int sub = 0; sub < 8; ++sub) {
            float d[3];
            for (int k = 0; k < 3; ++k) d[k] = ((sub >> k) & 1) ? quarter : -quarter;
            /* Taylor distance of the subvoxel centre, Eq. (taylor): psi + ghat . delta */
            float t = gh[0] * d[0];
            t = t + gh[1] * d[1];
            t = t + gh[2] * d[2];
            const float pc = ps + t;
            int keep = 1;
            for (int k = 0; k < 3; ++k) {
                const float sk = pc * gh[k];
                keep &= fabsf(sk) <= quarter;
            }
            if (!keep) continue;
            if (count < cap) {
                orc_point* o = out + count;
                o->sub = sub;
                double pc64 = psi[j];
                for (int k = 0; k < 3; ++k) pc64 += gh64[k] * (double)d[k];
                for (int k = 0; k < 3; ++k) {
                    o->m[k] = m[3 * j + k];
                    o->p[k] = vs64 * (double)m[3 * j + k] + (double)d[k] - pc64 * gh64[k];
                    o->n[k] = -gh64[k];
                }
            }
            ++count;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------------------------ */
/* layered marching cubes (Sec. 4.3)                                                           */
/* ------------------------------------------------------------------------------------------ */

/* corners of edge e: the corner with the edge's axis bit 0, and the one with it 1 */
static void orc_edge_corners(int e, int* a, int* b) {
    const int axis = e >> 2, k = e & 3;
    int lo = 0;
    if (axis == 0) lo = ((k & 1) << 1) | ((k >> 1) << 2);  /* dy = k&1, dz = k>>1 */
    if (axis == 1) lo = (k & 1) | ((k >> 1) << 2);         /* dx = k&1, dz = k>>1 */
    if (axis == 2) lo = (k & 1) | ((k >> 1) << 1);         /* dx = k&1, dy = k>>1 */
    *a = lo;
    *b = lo | (1 << axis);
}

/* triangles (edge triples) of case `inside` (bit c = corner c inside); returns their number */
static int orc_mc_case(int inside, int tri[][3]) {
    int nb[12][2], deg[12];
    for (int e = 0; e < 12; ++e) deg[e] = 0;
    for (int axis = 0; axis < 3; ++axis) {
        for (int side = 0; side < 2; ++side) {
            /* the face's 4 corners in cyclic order and the edge between consecutive ones */
            const int u = (axis + 1) % 3, w = (axis + 2) % 3;
            int cs[4], es[4];
            const int du[4] = {0, 1, 1, 0}, dw[4] = {0, 0, 1, 1};
            for (int q = 0; q < 4; ++q) cs[q] = (side << axis) | (du[q] << u) | (dw[q] << w);
            for (int q = 0; q < 4; ++q) {
                const int c0 = cs[q], c1 = cs[(q + 1) % 4];
                for (int e = 0; e < 12; ++e) {
                    int a, b;
                    orc_edge_corners(e, &a, &b);
                    if ((a == c0 && b == c1) || (a == c1 && b == c0)) es[q] = e;
                }
            }
            int cross[4], nc = 0;
            for (int q = 0; q < 4; ++q) {
                const int i0 = (inside >> cs[q]) & 1, i1 = (inside >> cs[(q + 1) % 4]) & 1;
                if (i0 != i1) cross[nc++] = q;
            }
            int pairs[2][2], np = 0;
            if (nc == 2) {
                pairs[0][0] = es[cross[0]];
                pairs[0][1] = es[cross[1]];
                np = 1;
            } else if (nc == 4) {
                /* inside corners on a diagonal: each is cut off by joining its two edges
                 * (edge q joins corners q and q+1, so corner q lies between edges q-1 and q) */
                for (int q = 0; q < 4; ++q) {
                    if ((inside >> cs[q]) & 1) {
                        pairs[np][0] = es[(q + 3) % 4];
                        pairs[np][1] = es[q];
                        ++np;
                    }
                }
            }
            for (int p = 0; p < np; ++p) {
                const int e0 = pairs[p][0], e1 = pairs[p][1];
                nb[e0][deg[e0]++] = e1;
                nb[e1][deg[e1]++] = e0;
            }
        }
    }
    int used[12] = {0}, nt = 0;
    for (int start = 0; start < 12; ++start) {
        if (deg[start] != 2 || used[start]) continue;
        int loop[12], len = 0, prev = -1, cur = start;
        int next = nb[start][0] < nb[start][1] ? nb[start][0] : nb[start][1];
        for (;;) {
            loop[len++] = cur;
            used[cur] = 1;
            if (prev >= 0) next = nb[cur][0] == prev ? nb[cur][1] : nb[cur][0];
            prev = cur;
            cur = next;
            if (cur == start) break;
        }
        for (int k = 1; k + 1 < len; ++k) {
            tri[nt][0] = loop[0];
            tri[nt][1] = loop[k];
            tri[nt][2] = loop[k + 1];
            ++nt;
        }
    }
    return nt;
}

typedef struct {
    int32_t m[3];
    double psi;
} orc_zvox;

static int orc_cmp_zvox(const void* pa, const void* pb) {
    const orc_zvox* a = (const orc_zvox*)pa;
    const orc_zvox* b = (const orc_zvox*)pb;
    for (int k = 2; k >= 0; --k) {
        if (a->m[k] < b->m[k]) return -1;
        if (a->m[k] > b->m[k]) return 1;
    }
    return 0;
}

size_t orc_marching_cubes(int64_t n, const int32_t* m, const double* psi, float voxel_size, orc_triangle* out,
                          size_t cap) {
    if (n <= 0) return 0;
    const double vs = (double)voxel_size;
    int lo[3], hi[3];
    for (int k = 0; k < 3; ++k) lo[k] = hi[k] = m[k];
    for (int64_t j = 1; j < n; ++j)
        for (int k = 0; k < 3; ++k) {
            if (m[3 * j + k] < lo[k]) lo[k] = m[3 * j + k];
            if (m[3 * j + k] > hi[k]) hi[k] = m[3 * j + k];
        }
    orc_zvox* zs = (orc_zvox*)malloc(sizeof(orc_zvox) * (size_t)n);
    const size_t nx = (size_t)(hi[0] - lo[0] + 1), ny = (size_t)(hi[1] - lo[1] + 1);
    double* layer[2];
    unsigned char* have[2];
    layer[0] = (double*)malloc(sizeof(double) * nx * ny);
    layer[1] = (double*)malloc(sizeof(double) * nx * ny);
    have[0] = (unsigned char*)calloc(nx * ny, 1);
    have[1] = (unsigned char*)calloc(nx * ny, 1);
    if (!zs || !layer[0] || !layer[1] || !have[0] || !have[1]) {
        free(zs);
        free(layer[0]);
        free(layer[1]);
        free(have[0]);
        free(have[1]);
        return 0;
    }
    for (int64_t j = 0; j < n; ++j) {
        for (int k = 0; k < 3; ++k) zs[j].m[k] = m[3 * j + k];
        zs[j].psi = psi[j];
    }
    qsort(zs, (size_t)n, sizeof(orc_zvox), orc_cmp_zvox);
    int table[256][12][3], counts[256];
    for (int c = 0; c < 256; ++c) counts[c] = orc_mc_case(c, table[c]);
    /* two z-layers of the bounding box at a time: layer 1 holds z, layer 0 holds z - 1 */
    int64_t pos = 0;
    size_t count = 0;
    for (int z = lo[2]; z <= hi[2]; ++z) {
        double* tl = layer[0];
        unsigned char* th = have[0];
        layer[0] = layer[1];
        have[0] = have[1];
        layer[1] = tl;
        have[1] = th;
        memset(have[1], 0, nx * ny);
        while (pos < n && zs[pos].m[2] == z) {
            const size_t at = (size_t)(zs[pos].m[1] - lo[1]) * nx + (size_t)(zs[pos].m[0] - lo[0]);
            layer[1][at] = zs[pos].psi;
            have[1][at] = 1;
            ++pos;
        }
        if (z == lo[2]) continue;
        /* cubes with lowest corner in layer z - 1 */
        for (size_t y = 0; y + 1 < ny; ++y) {
            for (size_t x = 0; x + 1 < nx; ++x) {
                double cp[8];
                int ok = 1, inside = 0;
                for (int c = 0; c < 8; ++c) {
                    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
                    const size_t at = (y + dy) * nx + (x + dx);
                    if (!have[dz][at]) {
                        ok = 0;
                        break;
                    }
                    cp[c] = layer[dz][at];
                    if (cp[c] > 0.0) inside |= 1 << c;
                }
                if (!ok || counts[inside] == 0) continue;
                const int32_t mc[3] = {lo[0] + (int32_t)x, lo[1] + (int32_t)y, z - 1};
                for (int t = 0; t < counts[inside]; ++t) {
                    if (count < cap) {
                        orc_triangle* o = out + count;
                        o->m[0] = mc[0];
                        o->m[1] = mc[1];
                        o->m[2] = mc[2];
                        o->edges = table[inside][t][0] | (table[inside][t][1] << 4) | (table[inside][t][2] << 8);
                        for (int k = 0; k < 3; ++k) {
                            int a, b;
                            orc_edge_corners(table[inside][t][k], &a, &b);
                            const double tt = cp[a] / (cp[a] - cp[b]);
                            for (int d = 0; d < 3; ++d) {
                                const double va = vs * (double)(mc[d] + ((a >> d) & 1));
                                const double vb = vs * (double)(mc[d] + ((b >> d) & 1));
                                o->v[3 * k + d] = va + tt * (vb - va);
                            }
                        }
                    }
                    ++count;
                }
            }
        }
    }
    free(zs);
    free(layer[0]);
    free(layer[1]);
    free(have[0]);
    free(have[1]);
    return count;
}
