/*
 * Gradient-SDF CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C restatement of the method's definitions, used to check the
 * CUDA library.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it; the product path never does.  It shares no code with the CUDA library.
 *
 * Numerics: every value (psi, g, W, residuals, Jacobians, normal equations, Cholesky, SE(3)
 * exponential) is FP64.  Every *discrete decision* (which pixel is valid, which voxel a point
 * rounds to, whether a normal passes the 75 degree test, whether a voxel lies inside the
 * truncation band) is taken on an explicit FP32 "index path" whose operations and their order are
 * fixed, so that any implementation doing the same correctly rounded FP32 operations takes the
 * same decisions bit for bit.  Compile with -ffp-contract=off and without -ffast-math.
 *
 * Map storage follows Sec. 5.1 of the paper: one hash-map entry per voxel holding
 * (psi, g, W).  A "dense" map is the same storage restricted to a box of voxel coordinates.
 */
#ifndef GSDF_ORACLE_H
#define GSDF_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_map orc_map;

/* camera intrinsics; pixel (u, v) has integer coordinates; depth_max is the 3.5 m cutoff of Sec. 5.3 */
typedef struct {
    float fx, fy, cx, cy;
    int width, height;
    float depth_max;
} orc_intrinsics;

/* method parameters (Sec. 5.3): voxel size v_s, truncation T, linear-weight knee eps,
 * Huber threshold delta, cos of the maximum normal/ray angle (75 degrees) */
typedef struct {
    float voxel_size;
    float truncation;
    float weight_eps;
    float huber_delta;
    float cos_max_angle;
    double damping; /* relative Levenberg-Marquardt damping, 0 = plain Gauss-Newton */
    int tracker;    /* 0: Eq. (taylor), one voxel; 1: trilinear interpolation of psi over the 8 voxels
                       of the cell, Eqs. (dir_dist), (dir_grad) (the direct SDF tracker baseline) */
} orc_params;

typedef struct {
    int32_t m[3];
    double psi;
    double g[3];
    double w;
} orc_voxel_out;

typedef struct {
    double H[21]; /* upper triangle of sum w J J^T, row-major */
    double b[6];  /* sum w J r */
    double energy;
    int64_t n_valid;
    int64_t n_huber;
    int status;   /* 0 ok, 1 degenerate (pose unchanged) */
    double xi[6]; /* applied increment (omega, upsilon) */
} orc_track_stats;

typedef struct {
    int64_t n_rays;   /* pixels that passed the depth and normal tests */
    int64_t n_visits; /* ray-voxel updates with w > 0 */
} orc_integrate_stats;

orc_map* orc_map_new(const orc_params* prm);
/* dense box [origin, origin + dims); integration outside it is skipped */
orc_map* orc_map_new_dense(const orc_params* prm, const int dims[3], const int origin[3]);
void orc_map_free(orc_map* map);
size_t orc_map_count(const orc_map* map);
/* set voxel values directly (analytic maps); psi/g/w arrays are x-fastest over dims */
int orc_map_set_dense(orc_map* map, const float* psi, const float* g, const float* w);

/* Eqs. sdf_update / gradient_update, pixel-driven as in Sec. 5.3 */
int orc_integrate(orc_map* map, const float* depth, const orc_intrinsics* K, const double T_wc[16],
                  orc_integrate_stats* st);
/* normal equations of Eq. (tracking) with the Taylor model Eq. (taylor) at pose T_wc */
int orc_track_reduce(const orc_map* map, const float* depth, const orc_intrinsics* K,
                     const double T_wc[16], orc_track_stats* st);
/* one Gauss-Newton step: reduce, Cholesky solve, left-multiplicative SE(3) update */
int orc_track_step(const orc_map* map, const float* depth, const orc_intrinsics* K, double T_wc[16],
                   orc_track_stats* st);

/* pieces exposed for the pins */
int orc_solve6(const double H21[21], const double b[6], double damping, int64_t n_valid, double xi[6]);
void orc_se3_exp(const double xi[6], double T[16]);
/* Taylor model at world point P using voxel m: returns 0 if usable, fills r and ghat */
int orc_taylor(const orc_map* map, const double P[3], const int32_t m[3], double* r, double ghat[3]);
/* Eqs. (dir_dist), (dir_grad) with trilinear interpolation over the cell whose lowest corner is
 * voxel b: with a = P / v_s - b, d(P) = sum_c psi_c prod_k (a_k or 1 - a_k) over the 8 corners, and
 * grad d its exact gradient (differences of psi along each axis, bilinearly weighted, / v_s).
 * Returns 0 if all 8 corners exist with W > 0. */
int orc_trilinear(const orc_map* map, const double P[3], const int32_t b[3], double* d, double grad[3]);
/* FP32 index path: world point of pixel (u, v) at depth D and its rounded voxel coordinate */
void orc_pixel_point(const orc_intrinsics* K, const double T_wc[16], int u, int v, float D,
                     float P_out[3], int32_t m_out[3], float voxel_size);
/* FP32 normal of pixel (u, v) in camera coordinates; returns 1 if it passes every test */
int orc_normal(const float* depth, const orc_intrinsics* K, const orc_params* prm, int u, int v,
               float n_out[3]);
/* voxels with W > 0 sorted by (x, y, z); returns the number written (<= cap) */
size_t orc_extract(const orc_map* map, orc_voxel_out* out, size_t cap);
/* block coordinate (floor division by 8) and local index of a voxel coordinate */
void orc_block_of(const int32_t m[3], int32_t b[3], int32_t local[3]);

/* ---------------------------------------------------------------------------------------------
 * Photometric + geometric voxel energy (Sec. 4.2, Eqs. rgb_cost, intensity_proj, mean_color,
 * variance; Eq. tracking) and its gradient, in FP64.
 *   surface point of voxel j:  p_j = v_j - psi_j ghat_j,  ghat = g / |g|   (Eq. grad_sdf_project)
 *   photometric:  E_p = sum_{i,j,c} nu_ij (I_i^c(pi(R_i^T (p_j - t_i))) - rho_j^c)^2, bilinear I
 *   geometric:    E_g = sum_i sum_k r_ik^2, r = psi_m + ghat_m . (P - v_m) at the nearest voxel m
 *                 of the back-projected pixel P (the FP32 index path), pixels without a voxel,
 *                 with W = 0 (not in the list) or g = 0 skipped
 *   E = E_p + lambda E_g.  Gradients: dE/dpsi, dE/dg (3n), dE/drho (3n) and, per keyframe, dE/dxi
 *   for a left perturbation T_i <- exp(xi^) T_i, xi = (omega, upsilon).
 * Voxels are given as a list (m[3n] integer coordinates, psi[n], g[3n], rho[3n]); images are
 * H x W x 3 FP32 (rgb) and H x W FP32 (depth), one per keyframe, all with intrinsics K.
 * ------------------------------------------------------------------------------------------- */

/* Discrete decisions (visibility, the photometric pair's bilinear cell) are taken on an FP32
 * index path from psi and g rounded to FP32 and the pose rounded to FP32 (order of operations in
 * the source); values stay FP64.
 * visibility nu[i * n + j] in {0, 1}: voxel j is a surface voxel (|psi_j ghat_j| <= v_s / 2 per
 * component, Sec. 4.3), its surface point projects into keyframe i with a one-pixel margin, in
 * front of the camera, and within v_s of the keyframe's depth at the nearest pixel.
 * In the energy a pair with nu_ij = 1 counts while its point projects into the image
 * (0 <= u <= W - 1, 0 <= v <= H - 1, in front) at the evaluated pose. */
void orc_visibility(int64_t n, const int32_t* m, const double* psi, const double* g, float voxel_size, int n_frames,
                    const orc_intrinsics* K, const double* poses, const float* const* depth, uint8_t* nu);

/* energy E[3] = (E, E_p, E_g) and, if dpsi != NULL, the full gradient; dT (may be NULL) gets, per
 * keyframe, dE/dT_ab for the 12 entries of T = [R t] as free variables (row-major 4 x 4, last row
 * zero), the gradient an autograd caller chains through */
int orc_energy(int64_t n, const int32_t* m, const double* psi, const double* g, const double* rho, float voxel_size,
               int n_frames, const orc_intrinsics* K, const double* poses, const float* const* rgb,
               const float* const* depth, const uint8_t* nu, double lambda_geo, double E[3], double* dpsi,
               double* dg, double* drho, double* dxi, double* dT);

/* ---------------------------------------------------------------------------------------------
 * One iteration of photometric bundle adjustment (Sec. 4.2, Eqs. rgb_cost, intensity_proj,
 * mean_color, rgb_cost_pose), optionally with lambda times the geometric term of Eq. (tracking):
 *   1. rho_j = mean colour of voxel j over the pairs that count (Eq. mean_color);
 *   2. with rho held fixed (the decoupled energies E_i of Eq. rgb_cost_pose), per keyframe the
 *      Gauss-Newton normal equations H_i = sum J J^T, b_i = sum J r of the residuals
 *      r = I_ij^c - rho_j^c with J = d r / d xi_i for the left perturbation T_i <- exp(xi^) T_i,
 *      plus lambda times the tracking terms of every keyframe pixel; per voxel the 1-D normal
 *      equations in psi_j (ghat held fixed, Sec. 4.2): psi_H = sum (dr/dpsi)^2, psi_b = sum
 *      dr/dpsi r, the geometric residual contributing lambda and lambda r;
 *   3. if flags & ORC_BA_POSES: xi_i = -(H_i + damping mean(diag H_i) I)^-1 b_i (orc_solve6) and
 *      T_i <- exp(xi_i^) T_i; if flags & ORC_BA_PSI: psi_j -= psi_b / ((1 + damping) psi_H) for
 *      psi_H > 0.
 * Pairs, cells and visibility as in orc_energy.  st[i] receives H, b, E_i (the step's starting
 * energy of keyframe i: its photometric residuals plus lambda times its geometric ones), the
 * residual count, the solve status and xi.  rho (3n) is written; psi_H, psi_b (n) may be NULL. */
#define ORC_BA_POSES 1
#define ORC_BA_PSI 2
int orc_ba_step(int64_t n, const int32_t* m, double* psi, const double* g, double* rho, float voxel_size, int n_frames,
                const orc_intrinsics* K, double* poses, const float* const* rgb, const float* const* depth,
                const uint8_t* nu, double lambda_geo, double damping, int flags, orc_track_stats* st, double* psi_H,
                double* psi_b);

/* ---------------------------------------------------------------------------------------------
 * Oriented point cloud (Sec. 4.3, "Oriented point cloud extraction") from a voxel list.
 *   level 0: voxel j gives the point v_j - psi_j ghat_j with normal -ghat_j when
 *            |psi_j ghat_j| <= v_s / 2 on every axis;
 *   level 1: each voxel is split into 2 x 2 x 2 subvoxels with centres c = v + delta,
 *            delta_k = +-v_s / 4; a subvoxel's distance is the Taylor value of Eq. (taylor),
 *            psi_c = psi + ghat . delta, and it gives the point c - psi_c ghat (normal -ghat) when
 *            |psi_c ghat| <= v_s / 4 on every axis.
 * Decisions on the FP32 index path (psi, g rounded to FP32; order of operations in the source),
 * values in FP64.  Points follow the list order, subvoxels in order sx + 2 sy + 4 sz.  Voxels with
 * g = 0 give nothing.  Returns the number of points (writes at most cap). */
typedef struct {
    int32_t m[3];
    int32_t sub; /* -1 at level 0, else the subvoxel index sx + 2 sy + 4 sz */
    double p[3];
    double n[3];
} orc_point;

size_t orc_points(int64_t n, const int32_t* m, const double* psi, const double* g, float voxel_size, int level,
                  orc_point* out, size_t cap);

/* ---------------------------------------------------------------------------------------------
 * Layered marching cubes (Sec. 4.3): the axis-aligned bounding box of the voxel list is swept two
 * z-layers at a time; every cube whose 8 corners (voxel centres m + {0,1}^3) are in the list gives
 * the triangles of its case.  A corner is inside when psi > 0; an edge with one inside corner
 * carries the vertex v_a + t (v_b - v_a), t = psi_a / (psi_a - psi_b).  Triangulation rule (any
 * marching-cubes table is such a rule; this one is stated so it can be reproduced): on each
 * face the crossing edges are joined in pairs -- a face with two crossings joins them, a face with
 * four (two inside corners on a diagonal) joins, for each inside corner, its two edges -- the
 * joins form closed loops through the crossing edges, each loop is walked from its smallest edge
 * id toward the smaller of that edge's two neighbours, and fanned from its first edge.
 * Edge ids: x-edges 0..3 (k = dy + 2 dz), y-edges 4..7 (k = dx + 2 dz), z-edges 8..11
 * (k = dx + 2 dy); corner index dx + 2 dy + 4 dz.  Cubes in z, y, x order; the triangles of a cube
 * in loop order.  Returns the number of triangles (writes at most cap). */
typedef struct {
    int32_t m[3];   /* the cube's lowest corner */
    int32_t edges;  /* e0 | e1 << 4 | e2 << 8 */
    double v[9];    /* the three vertices */
} orc_triangle;

size_t orc_marching_cubes(int64_t n, const int32_t* m, const double* psi, float voxel_size, orc_triangle* out,
                          size_t cap);

#ifdef __cplusplus
}
#endif
#endif
