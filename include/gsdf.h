/*
 * gsdf.h -- C ABI of the GB300 Gradient-SDF tracking and fusion library (libgsdf.so).
 *
 * The library implements the data-parallel hot path of "Gradient-SDF: A Semi-Implicit Surface
 * Representation for 3D Reconstruction" (Sommer et al., CVPR 2022):
 *   - a voxel map storing per voxel a signed distance psi, a gradient g and a weight W
 *     (Sec. 3.2, the GradSdfVoxel of Sec. 5.1), either a dense box of voxels or a hash table of
 *     8^3 voxel blocks (Sec. 3.1);
 *   - depth-image fusion, Eqs. (sdf_update) and (gradient_update), pixel-driven as in Sec. 5.3;
 *   - direct SDF camera tracking, Eq. (tracking), with the one-lookup first-order model
 *     Eq. (taylor), solved by Gauss-Newton with a Cholesky factorisation (Sec. 5.1).
 * Every step runs in the library's own CUDA kernels (sm_103a); there is no CPU fallback.
 *
 * Conventions
 *   - Depth images: FP32, row-major H x W, z-depth in metres, 0 (or anything outside
 *     (0, depth_max]) = no measurement.  Pixel (u, v) has integer coordinates.
 *   - Poses T_wc: 16 FP64 values, row-major 4x4, camera -> world (P = R p + t).
 *   - Voxel centres v = voxel_size * m, m in Z^3 (Sec. 3.1).  Block of m: floor(m / 8);
 *     local index (m mod 8): x + 8 y + 64 z.
 *   - Signed distances are inside-positive (negative in free space, Sec. 3.1); g points into
 *     the surface.
 *   - "_dev" pointers are CUDA device pointers; all other pointers are host pointers.
 *
 * Streams and ordering: every call is issued on the handle's stream (gsdf_create /
 * gsdf_set_stream) and returns without waiting, except gsdf_create, gsdf_destroy,
 * gsdf_upload_dense, gsdf_load_voxels, gsdf_extract_voxels, gsdf_num_blocks and gsdf_sync,
 * which synchronise the stream.  Caller-owned device buffers must stay valid until the stream
 * work that uses them has completed.  A handle must not be used from two threads at once.
 * gsdf_integrate, gsdf_track_step and gsdf_track allocate no device memory.
 *
 * Errors: argument errors are returned at once and leave the state unchanged.  Errors found on
 * the device (hash capacity exhausted) are recorded in a sticky device word, returned by the
 * next gsdf_sync (which clears it).  A degenerate tracking system is not an error of the map:
 * it is reported in gsdf_track_stats.status and leaves the pose unchanged.  Nothing aborts,
 * traps or prints.
 */
#ifndef GSDF_H
#define GSDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSDF_OK = 0,
    GSDF_ERR_INVALID_ARG = 1,  /* a null pointer, a bad size or an inconsistent configuration */
    GSDF_ERR_CUDA = 2,         /* a CUDA runtime call failed */
    GSDF_ERR_OOM = 3,          /* device allocation failed in gsdf_create / extraction */
    GSDF_ERR_CAPACITY = 4,     /* the hash table ran out of slots (probe limit reached) */
    GSDF_ERR_DEGENERATE = 5,   /* singular tracking system (see gsdf_track_stats.status) */
    GSDF_ERR_TIMEOUT = 6,      /* a bounded device wait gave up */
    GSDF_ERR_NO_VALID_PIXELS = 7
} gsdf_status;

enum { GSDF_GRID_DENSE = 0, GSDF_GRID_HASHED = 1 };
enum { GSDF_PAYLOAD_F32 = 0, GSDF_PAYLOAD_F16 = 1 };
enum { GSDF_TRACKER_TAYLOR = 0, GSDF_TRACKER_TRILINEAR = 1 };

/* Pinhole intrinsics (Sec. 5.3 uses 640x480 TUM frames, depth cut off at 3.5 m). */
typedef struct {
    float fx, fy, cx, cy;
    int32_t width, height;
    float depth_max;
} gsdf_intrinsics;

/* Map and method configuration.
 *   grid_kind      GSDF_GRID_DENSE or GSDF_GRID_HASHED
 *   dense_dims     dense grid size in voxels (x, y, z); dense only
 *   dense_origin   integer coordinate m of dense voxel (0, 0, 0); dense only
 *   voxel_size     v_s in metres (Sec. 3.1)
 *   truncation     T in metres (Sec. 5.3 uses 5 v_s); must be >= voxel_size / 2
 *   weight_eps     knee of the linear fusion weight: w = 1 for d <= eps, falling linearly to 0
 *                  at d = T (Sec. 5.3, "linear weight"); 0 <= eps < T
 *   huber_delta    threshold of the Huber tracking weight w_k of Eq. (tracking)
 *   cos_max_angle  cosine of the largest normal/viewing-ray angle integrated (Sec. 5.3: 75 deg)
 *   damping        relative Levenberg-Marquardt damping: H + damping * mean(diag H) * I;
 *                  0 = plain Gauss-Newton (Sec. 5.1)
 *   hash_slots     number of hash slots (power of two); each slot owns one 8^3 block payload
 *                  (10 KB); hashed only
 *   max_probe      linear-probe limit of the hash table (> 0); hashed only
 *   payload        voxel storage.  GSDF_PAYLOAD_F32: (W psi, g) and W in FP32, 20 bytes per voxel,
 *                  fused by atomic sums.  GSDF_PAYLOAD_F16 (hashed only): psi / sigma_b and
 *                  gbar = g / W as four FP16 values with one FP32 scale sigma_b per block (the
 *                  largest |psi| the block has held), and W in FP32: 12 bytes per voxel.  Per-pixel
 *                  arithmetic stays FP32; a frame is fused into FP32 accumulators of the touched
 *                  blocks, then folded into them and re-encoded with round-to-nearest, so psi
 *                  carries an error of at most 2^-11 sigma_b per frame and ghat about 5e-4.
 *   max_touched_blocks  FP16 payload only: entries of the per-frame accumulator table (a power
 *                  of two, at most hash_slots; keep it at least twice the blocks one frame
 *                  touches).  A frame whose blocks do not find an entry within 64 probes is fused
 *                  partially and reports GSDF_ERR_CAPACITY
 *   tracker        the model of gsdf_track_step.  GSDF_TRACKER_TAYLOR (the method, Eq. taylor):
 *                  one voxel lookup per pixel.  GSDF_TRACKER_TRILINEAR (the direct SDF tracker
 *                  the paper compares against, Eqs. dir_dist and dir_grad, Sec. 6): psi is
 *                  interpolated trilinearly over the 8 voxels of the cell containing P (lowest
 *                  corner floor(P (1/v_s)), FP32), r = d(P), J = (P x grad d, grad d) with the
 *                  interpolant's gradient; a pixel whose cell has an unobserved corner is
 *                  skipped.  FP32 payload only; not accepted by gsdf_batch_create.
 */
typedef struct {
    int32_t grid_kind;
    int32_t dense_dims[3];
    int32_t dense_origin[3];
    float voxel_size;
    float truncation;
    float weight_eps;
    float huber_delta;
    float cos_max_angle;
    double damping;
    int64_t hash_slots;
    int32_t max_probe;
    int32_t payload;             /* GSDF_PAYLOAD_F32 or GSDF_PAYLOAD_F16 (hashed maps only) */
    int32_t max_touched_blocks;  /* FP16 payload: blocks a single frame may update (>= 1) */
    int32_t tracker;             /* GSDF_TRACKER_TAYLOR or GSDF_TRACKER_TRILINEAR */
} gsdf_config;

/* Written by gsdf_track_step into device memory.  H is the upper triangle (row-major, 21
 * values) of sum_k w_k J_k J_k^T and b = sum_k w_k J_k r_k, both at the *input* pose;
 * J = (P x ghat, ghat) for the left increment T <- exp(xi^) T, xi = (omega, upsilon). */
typedef struct {
    double H[21];
    double b[6];
    double energy;    /* sum_k w_k r_k^2 */
    int64_t n_valid;  /* pixels with a usable voxel */
    int64_t n_huber;  /* of those, |r| > huber_delta */
    int32_t status;   /* GSDF_OK, or GSDF_ERR_DEGENERATE (pose left unchanged) */
    int32_t pad;
    double xi[6];     /* the increment applied (zero if degenerate) */
} gsdf_track_stats;

/* Written by gsdf_integrate into device memory (counts of this call, except n_blocks_total). */
typedef struct {
    int64_t n_rays;          /* pixels that passed the depth and normal tests */
    int64_t n_visits;        /* ray-voxel updates with weight > 0 */
    int64_t n_blocks_new;    /* hash blocks allocated by this call */
    int64_t n_blocks_total;  /* hash blocks allocated so far */
} gsdf_integrate_stats;

/* One voxel with W > 0, as returned by gsdf_extract_voxels (32 bytes).  psi is the fused
 * signed distance, g the unnormalised weighted sum of normals (ghat = g / |g|), w = W. */
typedef struct {
    int32_t m[3];
    float psi;
    float g[3];
    float w;
} gsdf_voxel;

/* One oriented surface point, as returned by gsdf_extract_points (40 bytes): the point p, its unit
 * normal n (= -ghat, pointing out of the surface), the voxel m it comes from and, after 2x2x2
 * upsampling, the subvoxel sub = sx + 2 sy + 4 sz (-1 without upsampling). */
typedef struct {
    int32_t m[3];
    int32_t sub;
    float p[3];
    float n[3];
} gsdf_point;

/* One triangle of the marching-cubes mesh, as returned by gsdf_extract_mesh (52 bytes): the cube's
 * lowest corner m, the cube edges its vertices lie on (e0 | e1 << 4 | e2 << 8, numbering in
 * gsdf_extract_mesh) and the three vertices. */
typedef struct {
    int32_t m[3];
    int32_t edges;
    float v[9];
} gsdf_triangle;

typedef struct gsdf_handle gsdf_handle;

/* Create a map on the current CUDA device.  Allocates the table, the voxel payload (zeroed:
 * psi = 0, g = 0, W = 0) and all scratch used by integrate/track; nothing is allocated later
 * on those paths.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Returns GSDF_ERR_INVALID_ARG on a bad configuration, GSDF_ERR_OOM if allocation fails. */
gsdf_status gsdf_create(const gsdf_config* cfg, void* cuda_stream, gsdf_handle** out);

/* Free every device and host resource of the handle (synchronises its stream first). */
gsdf_status gsdf_destroy(gsdf_handle* h);

/* Change the stream subsequent calls are issued on. */
gsdf_status gsdf_set_stream(gsdf_handle* h, void* cuda_stream);

/* Dense grids only: overwrite every voxel from host arrays (x fastest, then y, then z):
 * psi[n], g[3n] (xyz interleaved), w[n], n = dims[0] * dims[1] * dims[2].  Voxels with w = 0
 * count as unobserved.  Synchronous. */
gsdf_status gsdf_upload_dense(gsdf_handle* h, const float* psi, const float* g, const float* w);

/* Fuse one depth frame at pose T_wc_dev (Eqs. sdf_update, gradient_update; Sec. 5.3).
 * For every pixel whose depth is valid and whose normal (cross product of central differences
 * of its back-projected 4-neighbours, oriented away from the camera) makes an angle with the
 * viewing ray below acos(cos_max_angle), the samples z_k = D + (k - K) v_s / 2, k = 0..2K,
 * K = ceil(T / (v_s / 2)), are rounded to voxels; each distinct voxel of the ray with
 * d = z_v - D in [-T, T) (z_v: camera depth of the voxel centre) receives
 * (w d, w, w R n) with the linear weight w.  Hashed grids allocate the block of every voxel
 * that receives an update; dense grids skip voxels outside the box.  The result equals the
 * sequential running average of Eq. (sdf_update) up to floating-point summation order.
 * depth_dev: H*W FP32 on the device.  T_wc_dev: 16 FP64 on the device.
 * stats_dev: optional (NULL allowed) device gsdf_integrate_stats, overwritten. */
gsdf_status gsdf_integrate(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K,
                           const double* T_wc_dev, gsdf_integrate_stats* stats_dev);

/* One Gauss-Newton step of Eq. (tracking) with the model of Eq. (taylor) (Sec. 4.1, 5.1).
 * For every valid pixel, P = R p + t, the nearest voxel m = floor(P / v_s + 1/2) is looked up;
 * if it exists with W > 0 and g != 0, r = psi + ghat.(P - v_s m), J = (P x ghat, ghat),
 * w = Huber(r).  The normal equations are reduced on the device, (H + lambda I) xi = -b is
 * solved in FP64 (lambda = damping * trace(H) / 6) and T_wc_dev is replaced by
 * exp(xi^) T_wc_dev, all without a host round trip: the update of gsdf_gn_update.  If fewer
 * than 6 pixels are usable or an LDL^T pivot of H + lambda I is <= 1e-12 times its largest
 * diagonal entry, the pose is left unchanged and stats.status = GSDF_ERR_DEGENERATE.
 * T_wc_dev: 16 FP64 on the device, read and written.  stats_dev: optional (NULL allowed). */
gsdf_status gsdf_track_step(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K,
                            double* T_wc_dev, gsdf_track_stats* stats_dev);

/* n_iters consecutive Gauss-Newton steps, each exactly gsdf_track_step, in one call: the poses
 * and statistics equal those of n_iters gsdf_track_step calls bit for bit.
 * stats_dev: NULL or a device array of n_iters gsdf_track_stats (entry k describes step k).
 * With n_iters >= 2 the steps are chained: launch j first solves step j - 1's normal equations
 * (in every thread block, from the exact sums step j - 1 left in the handle's scratch) and then
 * tracks at the new pose, and one more launch solves the last step; the pose in T_wc_dev is
 * written by that last launch.  Unless the handle's stream is being captured by the caller (then
 * the kernels are simply launched into the caller's capture), the launches are recorded once into
 * a CUDA graph that is replayed while (depth_dev, *K, T_wc_dev, stats_dev, n_iters) stay the same;
 * a call with other arguments records a new graph (host-side cost, no device allocation by the
 * library).  Reusing one depth staging buffer and one stats buffer keeps every call a replay.
 * Calls on one handle are ordered by its stream; two calls of one handle must not run
 * concurrently (they share the chain's scratch).  1 <= n_iters <= 1024. */
gsdf_status gsdf_track(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K,
                       double* T_wc_dev, int32_t n_iters, gsdf_track_stats* stats_dev);

/* One damped Gauss-Newton update from given normal equations, for n independent systems on the
 * device (Sec. 4.1: the increment that minimises the linearised tracking energy, applied to the
 * pose as T <- exp(xi^) T; the last stage of every tracking step).  For system s:
 *   Hb_dev[27 s ..]   FP64, read: the 21 upper-triangle terms of H, row-major (H00 H01 .. H05
 *                     H11 .. H55), then the 6 of b -- the layout of gsdf_track_stats.H and .b;
 *   n_valid_dev[s]    residual count; fewer than 6 makes the system degenerate;
 *   damping           >= 0: solve (H + lambda I) xi = -b with lambda = damping * trace(H) / 6;
 *   T_dev[16 s ..]    FP64 row-major 4x4 camera-to-world pose, read and replaced by
 *                     exp(xi^) T (xi = (omega, upsilon), rotation first); unchanged if degenerate;
 *   xi_dev[6 s ..]    NULL or written: the increment (zeros if degenerate);
 *   status_dev[s]     NULL or written: GSDF_OK or GSDF_ERR_DEGENERATE.
 * Degenerate: n_valid < 6, a diagonal entry of H + lambda I that is not positive, or an LDL^T
 * pivot of H + lambda I at or below 1e-12 times its largest diagonal entry (as a Cholesky
 * factorisation would test it).  All pointers are device memory owned by the caller; the call is
 * asynchronous on cuda_stream (NULL: the legacy default stream) and allocates nothing.
 * GSDF_ERR_INVALID_ARG: n < 0, damping negative or not finite, or a required pointer NULL with
 * n > 0; GSDF_ERR_CUDA: the launch failed.  n = 0 does nothing. */
gsdf_status gsdf_gn_update(int32_t n, const double* Hb_dev, const int64_t* n_valid_dev, double damping,
                           double* T_dev, double* xi_dev, int32_t* status_dev, void* cuda_stream);

/* Copy every voxel with W > 0 to host_out, ordered by block (lexicographic block coordinate)
 * and then local index for hashed grids, by linear index (x fastest) for dense grids.
 * *count_out receives the number of such voxels even if it exceeds capacity (then only the
 * first `capacity` are written and GSDF_ERR_CAPACITY is returned).  Synchronous; may allocate
 * temporary device memory. */
gsdf_status gsdf_extract_voxels(gsdf_handle* h, gsdf_voxel* host_out, size_t capacity,
                                size_t* count_out);

/* Checkpoint restore: write n voxels (unique m; w > 0) into the map, allocating blocks as
 * needed.  Voxels of a dense map outside its box are rejected with GSDF_ERR_INVALID_ARG.
 * Round trip extract -> load -> extract reproduces m, g and w exactly and psi to within one
 * FP32 rounding.  Synchronous; may allocate temporary device memory. */
gsdf_status gsdf_load_voxels(gsdf_handle* h, const gsdf_voxel* host_in, size_t n);

/* Oriented point cloud of the map (Sec. 4.3).  level 0: every voxel with W > 0 and g != 0 whose
 * surface point lies in its own cube, |psi ghat| <= v_s / 2 on every axis, gives the point
 * v - psi ghat with normal -ghat.  level 1 (geometry upsampling): every such voxel is split into
 * 2 x 2 x 2 subvoxels with centres c = v + delta, delta_k = +-v_s / 4; a subvoxel's distance is the
 * Taylor value of Eq. (taylor), psi_c = psi + ghat . delta, and it gives c - psi_c ghat when
 * |psi_c ghat| <= v_s / 4 on every axis.  Decisions are taken in FP32 with correctly rounded
 * operations in a fixed order (ghat_k = g_k / sqrt((g0 g0 + g1 g1) + g2 g2), psi_c = psi +
 * ((ghat0 d0 + ghat1 d1) + ghat2 d2), psi = (W psi) / W as stored), so they are reproducible.
 * Order: the voxel order of gsdf_extract_voxels, subvoxels by increasing sub.  *count_out receives
 * the number of points even if it exceeds capacity (then only the first `capacity` are written and
 * GSDF_ERR_CAPACITY is returned).  Synchronous; may allocate temporary device memory. */
gsdf_status gsdf_extract_points(gsdf_handle* h, int32_t level, gsdf_point* host_out, size_t capacity,
                                size_t* count_out);

/* Marching-cubes mesh of the map (Sec. 4.3, the mesh the paper's layered marching cubes extracts):
 * every cube whose 8 corners m + {0,1}^3 (voxel centres) are observed (W > 0) gives the triangles
 * of its case.  A corner is inside when psi > 0; an edge between an inside and an outside corner
 * carries the vertex v_a + t (v_b - v_a), t = psi_a / (psi_a - psi_b).  Corner index c = dx + 2 dy
 * + 4 dz; edge ids: x-edges 0..3 (k = dy + 2 dz), y-edges 4..7 (k = dx + 2 dz), z-edges 8..11
 * (k = dx + 2 dy).  Triangulation rule: on each cube face the crossing edges are joined in pairs
 * (two crossings: joined; four, i.e. two inside corners on a diagonal: each inside corner's two
 * edges joined, which separates the inside corners), the joins close into loops, each loop is
 * walked from its smallest edge id toward the smaller of its two neighbours and fanned from its
 * first edge.  The rule depends only on a face's own corners, so neighbouring cubes agree and the
 * mesh of a closed surface is closed.  The paper sweeps a bounding box two z-layers at a time to
 * bound a CPU's memory; the library visits the same cubes directly through the map.  Order: the
 * voxel order of gsdf_extract_voxels (by lowest corner), then the case's triangle order.
 * Capacity semantics as gsdf_extract_voxels.  Synchronous; may allocate temporary device memory. */
gsdf_status gsdf_extract_mesh(gsdf_handle* h, gsdf_triangle* host_out, size_t capacity, size_t* count_out);

/* Number of allocated hash blocks (dense: number of 512-voxel chunks).  Synchronous. */
gsdf_status gsdf_num_blocks(gsdf_handle* h, int64_t* n_out);

/* Wait for the handle's stream; return (and clear) the first device-detected error. */
gsdf_status gsdf_sync(gsdf_handle* h);

/* Allocation-free tracking step (the paper has no counterpart; this is a deployment aid).
 * For callers that cannot call cudaMalloc -- code confined to a device-memory budget that a host
 * framework owns and hands out, or a real-time loop where an allocation, and the device-wide
 * synchronisation it may cause, is not allowed -- this entry point performs exactly one
 * gsdf_track_step on a dense grid that the caller owns, without a handle and without allocating
 * anything.  The caller passes every input and output:
 *   depth_dev   H*W FP32 depth (device), as for gsdf_track_step;
 *   A_dev       dims[0]*dims[1]*dims[2] float4 (device), x fastest: (W psi, g.x, g.y, g.z) of each
 *               voxel -- the library's own dense payload layout (psi times its weight, then the
 *               unnormalised gradient);
 *   W_dev       the matching weights (device); W = 0 marks an unobserved voxel;
 *   dims/origin grid size and integer coordinate of voxel (0,0,0) (host arrays of 3);
 *   voxel_size, huber_delta, damping: as in gsdf_config;
 *   T_wc_dev    pose, read and updated (device); stats_dev: NULL or device gsdf_track_stats;
 *   cuda_stream the stream to launch on (NULL = legacy default stream).
 * Scratch: a 16,640-byte array in the library's device memory (a static __device__ array that
 * every GPU which loads the library holds until the process exits).  The scratch this step
 * needs does not grow with the image or grid size: its fit is fixed when the library is built,
 * so this call never reports GSDF_ERR_CAPACITY.  Inputs beyond the limits gsdf_create and
 * gsdf_track_step accept (image sides > 32768, grid sides > 65536) return GSDF_ERR_INVALID_ARG.
 * The first call on a device resolves the array's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that first call before any
 * stream capture.  A reset of the device's context (cudaDeviceReset) invalidates the kept address:
 * after one, restart the process before calling this entry point again.  Every call clears the
 * array's accumulators on cuda_stream before using them, and all calls share the one array:
 * calls that may overlap on the GPU (different streams, or the same call issued into several
 * concurrently running graphs) race with each other and must be serialised by the caller. */
gsdf_status gsdf_track_step_dense_noalloc(const float* depth_dev, const gsdf_intrinsics* K,
                                          const void* A_dev, const float* W_dev,
                                          const int32_t dims[3], const int32_t origin[3],
                                          float voxel_size, float huber_delta, double damping,
                                          double* T_wc_dev, gsdf_track_stats* stats_dev,
                                          void* cuda_stream);

/* Measurement: the distinct voxels (out[0]) and distinct 8^3 blocks (out[1]; for a dense grid, the
 * 512-voxel chunks of its linear index) that one pass over a frame touches -- the compulsory
 * payload and table accesses of that pass, for roofline accounting (Sec. 5.3 tracks and fuses every
 * frame; these are the voxels each of those passes must read or write at least once).
 *   what = GSDF_FOOTPRINT_TRACK: the voxels gsdf_track_step at pose T_wc_dev reads: pixels with valid
 *          depth whose nearest voxel (Eq. taylor) exists, is observed and has g != 0;
 *   what = GSDF_FOOTPRINT_FUSE: the voxels gsdf_integrate of this frame at this pose updates.  Blocks
 *          are looked up, not inserted: call it after fusing the same frame at the same pose.
 * The map is not modified.  Synchronous; allocates and frees two bitmaps of n_voxels and n_voxels /
 * 512 bits, so it is not meant for the per-frame loop. */
enum { GSDF_FOOTPRINT_TRACK = 0, GSDF_FOOTPRINT_FUSE = 1 };
gsdf_status gsdf_footprint(gsdf_handle* h, int32_t what, const float* depth_dev, const gsdf_intrinsics* K,
                           const double* T_wc_dev, int64_t out[2]);

/* ---------------------------------------------------------------------------------------------
 * Batches: many independent scenes (maps of any kind, payload and voxel size, frames of any
 * resolution) tracked and fused together in batched launches (the tracking and fusion of
 * Sec. 5.3, run for many scenes at once).  Each Gauss-Newton step of every scene is one launch
 * over (scene, pixel-tile) items: for batches of up to 64 scenes and 4096 tiles a grid with one
 * thread block per tile, whose per-scene constants travel in the launch's parameters; larger
 * batches run a persistent kernel whose blocks pull items from a device counter.  A scene's 6x6
 * solve runs in the block that finishes its last tile while other blocks keep working, so the
 * per-scene FP64 tail overlaps the other scenes' pixel work.  Fusion runs the same way (a grid of
 * work items, or a persistent launch for larger batches).  Results per scene are those of gsdf_track_step / gsdf_integrate on that scene's handle, up to
 * FP32 summation order.
 * ------------------------------------------------------------------------------------------- */
typedef struct gsdf_batch gsdf_batch;

/* Group n handles (all on the current device; not used elsewhere while the batch is in use).
 * Dense, hashed FP32 and hashed FP16 maps may be mixed.  Allocates the batch's descriptor table
 * and counters.  cuda_stream: the stream of every batch call.  Handles with the trilinear tracker
 * are not accepted (GSDF_ERR_INVALID_ARG).  Synchronous. */
gsdf_status gsdf_batch_create(gsdf_handle* const* handles, int32_t n, void* cuda_stream, gsdf_batch** out);
gsdf_status gsdf_batch_destroy(gsdf_batch* b);

/* Set the frame of every scene: host arrays of n device pointers (depth_dev[s], T_wc_dev[s]) and
 * n intrinsics; track_stats_dev / integrate_stats_dev: NULL or device arrays of n entries.  The
 * descriptor table is copied to the device on the batch's stream.  A change of any frame size
 * rebuilds the tile table (host-synchronous, and uses an autotuned tile size when one is cached for
 * that set of sizes; otherwise 2048-px tiles, doubled up to 16384 px while a batch of at most 64
 * scenes would need more than 4096 tiles). */
gsdf_status gsdf_batch_set_frames(gsdf_batch* b, const float* const* depth_dev, const gsdf_intrinsics* K,
                                  double* const* T_wc_dev, gsdf_track_stats* track_stats_dev,
                                  gsdf_integrate_stats* integrate_stats_dev);

/* One Gauss-Newton step of every scene (one launch). */
gsdf_status gsdf_batch_track_step(gsdf_batch* b);

/* n_iters steps of every scene, recorded once into a CUDA graph and replayed while the tile
 * table and n_iters stay the same (frames may change between calls through
 * gsdf_batch_set_frames).  1 <= n_iters <= 1024. */
gsdf_status gsdf_batch_track(gsdf_batch* b, int32_t n_iters);

/* Fuse every scene's frame at its current pose (prologue, one fusion launch, for FP16 scenes one
 * persistent apply pass, epilogue). */
gsdf_status gsdf_batch_integrate(gsdf_batch* b);

/* Per-scene depth strides for gsdf_batch_frame: stride[s] (host array of n, in floats) is added
 * to scene s's depth pointer on the device after each frame, so that a sequence of frames stored
 * at a fixed distance from one another (e.g. an (F, H, W) tensor: stride H*W) is walked without
 * any call from the host.  0 keeps the pointer (the caller refills that buffer between frames,
 * e.g. with a copy on the batch's stream).  The caller keeps every frame that will be reached
 * valid.  Must follow gsdf_batch_set_frames; a later gsdf_batch_set_frames keeps the strides and
 * restarts the pointers from its arguments. */
gsdf_status gsdf_batch_set_depth_stride(gsdf_batch* b, const int64_t* stride);

/* One frame of every scene (the per-frame loop of Sec. 5.3): n_iters Gauss-Newton steps
 * (0 <= n_iters <= 1024; 0 fuses at the current poses), fusion at the tracked poses, then the depth
 * pointers' advance (gsdf_batch_set_depth_stride).  All of it is one CUDA graph, recorded on the
 * first call and replayed while n_iters and the tile table stay the same: one graph launch per
 * frame, and nothing copied from the host.  Statistics: the track_stats of the last step and the
 * frame's integrate_stats, as gsdf_batch_set_frames gave them. */
gsdf_status gsdf_batch_frame(gsdf_batch* b, int32_t n_iters);

/* Choose the tile size (pixels per work item) and the resident blocks per SM of the batched
 * tracking launch by timing candidates on the current frames: one Gauss-Newton step of every
 * scene per candidate, run on scratch copies of the poses without statistics, so maps, poses and
 * statistics are unchanged.  The choice is cached per shape class (the multiset of frame sizes).
 * Synchronous.  Optional outputs receive the choice. */
gsdf_status gsdf_batch_autotune(gsdf_batch* b, int32_t* tile_px_out, int32_t* ctas_per_sm_out);

/* ---------------------------------------------------------------------------------------------
 * Photometric + geometric voxel energy and its adjoint (Sec. 4.2, Eqs. rgb_cost, intensity_proj,
 * mean_color, variance; Eq. tracking with Eq. taylor), over an explicit list of n voxels.
 *   voxel j:    integer coordinate m_j, psi_j, g_j, colour rho_j (RGB); surface point
 *               p_j = v_s m_j - psi_j ghat_j, ghat = g / |g| (Eq. grad_sdf_project);
 *   keyframe i: pose T_i (camera -> world), RGB image I_i and depth image D_i, shared intrinsics;
 *   E   = E_p + lambda E_g,
 *   E_p = sum_{i,j,c} nu_ij (I_i^c(pi(R_i^T (p_j - t_i))) - rho_j^c)^2, I sampled bilinearly
 *         (Eq. rgb_cost with an explicit per-voxel colour rho; at rho = the mean colour of
 *         Eq. mean_color, E_p = sum_j N_j Var_j, Eq. variance);
 *   E_g = sum_i sum_pixels r^2, r = psi_m + ghat_m . (P - v_s m), P the back-projected pixel at
 *         T_i and m its nearest voxel (exactly the pixel path of gsdf_track_step), pixels whose
 *         voxel is not in the list or has g = 0 skipped.
 * Discrete decisions are taken on an FP32 index path with a fixed order of operations (psi, g
 * as given in FP32, T_i rounded once to FP32):
 *   n2 = (g0 g0 + g1 g1) + g2 g2, ghat_k = g_k / sqrt(n2), s_k = psi ghat_k, p_k = v_s m_k - s_k,
 *   d = p - t, x_i = (R_0i d_0 + R_1i d_1) + R_2i d_2, u = (f_x x_0) / x_2 + c_x, v likewise.
 * Visibility nu_ij = 1 iff n2 > 0, |s_k| <= v_s / 2 for every k (surface voxel, Sec. 4.3),
 * x_2 > 0, 1 <= u <= W - 2, 1 <= v <= H - 2, and at the nearest pixel (floor(u + 1/2),
 * floor(v + 1/2)) the depth D is valid and |x_2 - D| <= v_s.  In the energy a pair with
 * nu_ij = 1 counts while, at the evaluated pose, n2 > 0, x_2 > 0, 0 <= u <= W - 1 and
 * 0 <= v <= H - 1; its bilinear cell is (min(floor u, W - 2), min(floor v, H - 2)).
 * Per-pixel lookups are recomputed by every evaluation; nothing per pixel is stored.
 * Arithmetic: FP32 per voxel and per pixel, FP64 accumulation of the energies and pose terms.
 * ------------------------------------------------------------------------------------------- */
typedef struct gsdf_energy gsdf_energy;

/* Build an energy over n_voxels voxels (0 allowed) and n_frames keyframes (1..64):
 *   m_dev      3 n int32 (device), xyz per voxel, unique, each coordinate in [-2^23, 2^23);
 *   rgb_dev    n_frames x H x W x 3 FP32 (device), keyframe colours, row-major;
 *   depth_dev  n_frames x H x W FP32 (device), keyframe depths (as for gsdf_integrate);
 *   K          intrinsics shared by the keyframes, W, H >= 2.
 * The library copies m, rgb and depth (the caller's buffers may be freed afterwards) and builds
 * an index of the voxels by 8^3 block (a hash of block keys and a voxel table per block).  A
 * repeated or out-of-range coordinate returns GSDF_ERR_INVALID_ARG.  Synchronous on cuda_stream,
 * which later calls use.  Device memory: about 4 n (F + 8) bytes plus 2 KB per block and
 * 20 F H W bytes for the images. */
gsdf_status gsdf_energy_create(int64_t n_voxels, const int32_t* m_dev, float voxel_size, int32_t n_frames,
                               const gsdf_intrinsics* K, const float* rgb_dev, const float* depth_dev,
                               void* cuda_stream, gsdf_energy** out);
gsdf_status gsdf_energy_destroy(gsdf_energy* e);
gsdf_status gsdf_energy_set_stream(gsdf_energy* e, void* cuda_stream);

/* The visibility defined above at the poses T_dev (device, n_frames x 16 FP64) for psi_dev (n FP32)
 * and g_dev (3 n FP32), as a voxel-major bit set: nu_dev (device) holds ceil(n_frames / 32)
 * uint32 words per voxel, word k of voxel j at nu_dev[j * ceil(n_frames / 32) + k], and bit
 * (i mod 32) of word i / 32 is nu_ij. */
gsdf_status gsdf_energy_visibility(gsdf_energy* e, const float* psi_dev, const float* g_dev, const double* T_dev,
                                   uint32_t* nu_dev);

/* Evaluate E at (psi, g, rho, T) with visibility nu (all device; rho 3 n FP32; nu in the bit-set
 * layout of gsdf_energy_visibility, any bits the caller chooses; lambda_geo finite).  E_dev (device, 3 FP64) receives (E, E_p, E_g); E_g = 0 if lambda_geo = 0.
 * Gradients (device; NULL = not wanted; dpsi, dg, drho all or none):
 *   dpsi (n), dg (3 n), drho (3 n) FP32: dE/dpsi, dE/dg, dE/drho;
 *   dT   (n_frames x 16 FP64): dE/dT_ab for the 12 entries of each T = [R t] as free variables
 *        (row-major 4 x 4, last row 0) -- the gradient an autograd caller chains through;
 *   dxi  (n_frames x 6 FP64): dE/dxi for the left perturbation T_i <- exp(xi^) T_i at xi = 0,
 *        xi = (omega, upsilon).
 * grad_scale_dev: NULL or one device FP64 that multiplies every gradient (not E): the incoming
 * gradient of an autograd backward.  Asynchronous; no device allocation. */
gsdf_status gsdf_energy_eval(gsdf_energy* e, const float* psi_dev, const float* g_dev, const float* rho_dev,
                             const double* T_dev, const uint32_t* nu_dev, double lambda_geo,
                             const double* grad_scale_dev, double* E_dev, float* dpsi_dev, float* dg_dev,
                             float* drho_dev, double* dT_dev, double* dxi_dev);

/* One iteration of photometric bundle adjustment on the energy's voxels and keyframes (Sec. 4.2,
 * Eqs. rgb_cost, intensity_proj, mean_color, rgb_cost_pose), optionally with lambda_geo times the
 * geometric term (every keyframe pixel's Eq. tracking residual):
 *   1. rho_dev (3 n FP32, written) receives every voxel's mean colour over the pairs that count
 *      (Eq. mean_color; 0 where none counts);
 *   2. with rho held fixed -- the decoupled per-keyframe energies of Eq. rgb_cost_pose -- each
 *      keyframe's Gauss-Newton normal equations H_i = sum J J^T, b_i = sum J r are formed from its
 *      colour residuals r = I_ij^c - rho_j^c, J = d r / d xi for T_i <- exp(xi^) T_i, plus lambda
 *      times its pixels' tracking terms; and per voxel the 1-D normal equations in psi_j (ghat
 *      held fixed, as the paper does; the geometric residual contributes lambda and lambda r);
 *   3. if flags & GSDF_BA_POSES, every keyframe pose T_dev[i] (FP64, in place) is replaced by
 *      exp(xi_i^) T_i with (H_i + damping mean(diag H_i) I) xi_i = -b_i (FP64 Cholesky-equivalent
 *      solve of the tracking step; a degenerate system leaves the pose and sets the status); if
 *      flags & GSDF_BA_PSI, psi_dev (in place) takes the damped Newton step
 *      psi_j -= psi_b / ((1 + damping) psi_H) where psi_H > 0.  flags = 0 evaluates only.
 * Pairs, visibility (nu_dev, the bit set of gsdf_energy_visibility) and decisions as in
 * gsdf_energy_eval.  stats_dev: NULL or n_frames device gsdf_track_stats, entry i with H_i, b_i,
 * the keyframe's energy at the start of the step (colour residuals plus lambda times geometric),
 * the residual count in n_valid, the status and xi_i.  Asynchronous; no device allocation. */
enum { GSDF_BA_POSES = 1, GSDF_BA_PSI = 2 };
gsdf_status gsdf_energy_ba_step(gsdf_energy* e, float* psi_dev, const float* g_dev, float* rho_dev, double* T_dev,
                                const uint32_t* nu_dev, double lambda_geo, double damping, int32_t flags,
                                gsdf_track_stats* stats_dev);

/* Static description of a status code. */
const char* gsdf_status_string(gsdf_status s);

#ifdef __cplusplus
}
#endif
#endif /* GSDF_H */
