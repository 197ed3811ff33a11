// Device building blocks of the tracking step (Eq. (tracking) with the model Eq. (taylor),
// Gauss-Newton with an FP64 solve, Sec. 4.1 and 5.1), shared by the single-scene kernel
// (track.cu) and the batched persistent kernel (batch.cu).
#pragma once

#include "gsdf_internal.cuh"

namespace gsdf {

constexpr int kTrackThreads = 512;
constexpr int kTrackBlocksPerSM = 2;
constexpr int kTrackWarps = kTrackThreads / 32;
constexpr int kTerms = 30;
static_assert(kAccumCopies == kTrackWarps, "the finishing block reads one accumulator copy per warp");

// FP64 on this GPU: every FP64 warp instruction occupies the FP64 pipe for about 64 cycles,
// whatever the number of active lanes, so FP64 code is costed in warp instructions on the
// critical path.  The reduction and the solve keep the method's FP64 precision but use few of
// them:
//   * the grid-wide sum is exact fixed-point integer arithmetic (associative, hence deterministic
//     in any order, and off the FP64 pipe);
//   * the 6x6 system is solved by one warp holding one entry of the augmented upper triangle
//     [H | -b] per lane (27 lanes), so that an elimination step is three FP64 instructions.

// 2^k as a double (k within the normal exponent range)
__device__ __forceinline__ double exp2i(int k) { return __hiloint2double((1023 + k) << 20, 0); }
// e such that x * 2^-e lies in [0.5, 1), for finite x > 0 with a normal exponent
__device__ __forceinline__ int exponent_of(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1022; }

// Solve (H + lambda I) xi = -b, lambda = damping * mean(diag H), with one warp.  Hb (shared):
// the 21 upper-triangle terms of H (row-major) then the 6 of b.  Degenerate (returns false,
// xi = 0; uniform across the warp) if fewer than 6 residuals, a non-positive diagonal entry, or
// an LDL^T pivot d_j <= 1e-12 max diag (the test of the Cholesky factorisation).
//
// Method: the rows and columns are scaled by powers of two s_i ~ diag_i^-1/2 (exact), then
// eliminated without division: step j replaces every row i > j by
//     n_j (p_j row_i - a_ij row_j),   p_j = current pivot, n_j = 2^-e with p_j n_j in [1/2, 1),
// which equals the Schur-complement row times p_j n_j.  Row j is therefore row j of the LDL^T
// factor scaled by sigma_j = prod_{k<j} p_k n_k, so d_j (of the scaled matrix) = p_j / sigma_j
// and the pivot test is p_j > thr_j sigma_j with thr_j = 1e-12 maxd s_j^2, evaluated after the
// elimination.  Back-substitution uses the six pivot reciprocals, formed in parallel.
__device__ __forceinline__ bool solve6_warp(const double* Hb, double damping, long long n_valid, double* xi) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    // lane -> entry (i, k) of the augmented upper triangle, 0 <= i <= 5, i <= k <= 6 (k = 6: rhs)
    int ei = 0, ek = 0;
    {
        int base = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const int len = 7 - r;
            if (lane >= base && lane < base + len) {
                ei = r;
                ek = r + (lane - base);
            }
            base += len;
        }
    }
    const bool active = lane < 27;
    auto idx = [](int i, int k) { return i * 7 - i * (i - 1) / 2 + (k - i); };  // lane of entry (i, k), i <= k
    auto h21 = [](int i, int k) { return i * 6 - i * (i - 1) / 2 + (k - i); };  // index in the 21 terms

    // lane-parallel bookkeeping: lane j < 6 owns diagonal entry j
    const int dj = lane < 6 ? lane : 0;
    const double myd = lane < 6 ? Hb[h21(dj, dj)] : 0.0;
    double tr = myd;
    tr += __shfl_xor_sync(full, tr, 1);
    tr += __shfl_xor_sync(full, tr, 2);
    tr += __shfl_xor_sync(full, tr, 4);  // lanes 0..7 hold the trace (lanes 6, 7 contribute 0)
    tr = __shfl_sync(full, tr, 0);
    const double lam = damping > 0.0 ? damping * tr * (1.0 / 6.0) : 0.0;
    const double mydl = myd + lam;
    double mx = lane < 6 ? mydl : -1.0;
    mx = fmax(mx, __shfl_xor_sync(full, mx, 1));
    mx = fmax(mx, __shfl_xor_sync(full, mx, 2));
    mx = fmax(mx, __shfl_xor_sync(full, mx, 4));
    const double maxd = __shfl_sync(full, mx, 0);
    const bool bad_diag = __any_sync(full, lane < 6 && !(mydl > 0.0));
    if (lane < 6) xi[lane] = 0.0;
    if (n_valid < 6 || !(maxd > 0.0) || bad_diag) return false;
    // power-of-two scales s_j ~ diag_j^-1/2 (exact); lane j < 6 computes its own
    const double my_s = exp2i(-(exponent_of(lane < 6 ? mydl : 1.0) >> 1));
    const double s_i = __shfl_sync(full, my_s, ei);
    // (every lane must execute each shuffle: take it unconditionally, select afterwards)
    const double s_k_sh = __shfl_sync(full, my_s, ek < 6 ? ek : 0);
    const double s_k = ek < 6 ? s_k_sh : 1.0;
    double a = 0.0;
    if (active) a = ek < 6 ? (Hb[h21(ei, ek < 6 ? ek : 0)] + (ei == ek ? lam : 0.0)) : -Hb[21 + ei];
    a *= s_i * s_k;

    double pn_mine = 1.0;  // lane (j, j) keeps p_j n_j of its step
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const int jj = idx(j, j);
        const double p = __shfl_sync(full, a, jj);
        const double nrm = exp2i(-exponent_of(p > 0.0 ? p : 1.0));
        const double an = a * nrm;
        const double pn = __shfl_sync(full, an, jj);
        if (lane == jj) pn_mine = pn;
        const int src_n = idx(j, ei > j ? ei : j);
        const int src_k = idx(j, ek > j ? ek : j);
        const double aji_n = __shfl_sync(full, an, src_n);
        const double ajk = __shfl_sync(full, a, src_k);
        const double upd = fma(-aji_n, ajk, pn * a);
        if (active && ei > j) a = upd;
    }
    // pivot test, lane-parallel: lane j < 6 checks p_j > 1e-12 maxd s_j^2 sigma_j with
    // sigma_j = prod_{k<j} p_k n_k (exclusive prefix product by shuffles)
    const double pj = __shfl_sync(full, a, idx(dj, dj));
    const double pnj = __shfl_sync(full, pn_mine, idx(dj, dj));
    double pre = lane < 6 ? pnj : 1.0;  // inclusive prefix product over lanes 0..5
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const double up = __shfl_up_sync(full, pre, o);
        if (lane >= o) pre *= up;
    }
    double sigma = __shfl_up_sync(full, pre, 1);
    if (lane == 0) sigma = 1.0;
    const bool pivot_bad = __any_sync(full, lane < 6 && !(pj > (1e-12 * maxd) * (my_s * my_s) * sigma));
    if (pivot_bad) return false;
    // back-substitution on the rhs lanes (i, 6): x_k = c_k / p_k, c_i -= a_ik x_k
    const double rcp = 1.0 / (ei == ek ? a : 1.0);        // lanes (k, k): 1 / p_k, all at once
    double c = a;                                            // meaningful in lanes (i, 6)
#pragma unroll
    for (int k = 5; k >= 0; --k) {
        const double rk = __shfl_sync(full, rcp, idx(k, k));
        const double ck = __shfl_sync(full, c, idx(k, 6));
        const double xk = ck * rk;
        const double aik = __shfl_sync(full, a, idx(ei < k ? ei : k, k));
        if (ek == 6 && ei < k) c = fma(-aik, xk, c);
        if (ek == 6 && ei == k) c = xk;
    }
    if (active && ek == 6) xi[ei] = c * s_i;
    __syncwarp();
    return true;
}

// exp of the twist xi = (omega, upsilon) by one warp: R = I + A [w]x + B [w]x^2,
// t = (I + B [w]x + C [w]x^2) u, A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3,
// [w]x^2 = w w^T - th^2 I.  For th^2 < 0.01 lanes 0..2 evaluate the coefficients' Taylor series
// in th^2 (truncation error < 1e-21); larger angles use sincos.  Lanes 0..8 then write R and
// lanes 9..11 t into dT (row-major 3x4, shared); xi is in shared memory.
__device__ __forceinline__ void se3_exp_warp(const double* xi, double* dT) {
    const int lane = threadIdx.x & 31;
    const double w0 = xi[0], w1 = xi[1], w2 = xi[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double coef;
    if (th2 < 1e-2) {
        // coefficient tables of sum_k (-1)^k x^k / (2k+1)!, /(2k+2)!, /(2k+3)!
        constexpr double kA[8] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880, -1.0 / 39916800,
                                  1.0 / 6227020800.0, -1.0 / 1307674368000.0};
        constexpr double kB[8] = {1.0 / 2, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800, -1.0 / 479001600,
                                  1.0 / 87178291200.0, -1.0 / 20922789888000.0};
        constexpr double kC[8] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800,
                                  -1.0 / 6227020800.0, 1.0 / 1307674368000.0, -1.0 / 355687428096000.0};
        coef = lane == 0 ? kA[7] : (lane == 1 ? kB[7] : kC[7]);
#pragma unroll
        for (int k = 6; k >= 0; --k) coef = (lane == 0 ? kA[k] : (lane == 1 ? kB[k] : kC[k])) + th2 * coef;
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        coef = lane == 0 ? sn / th : (lane == 1 ? (1.0 - cs) / th2 : (th - sn) / (th2 * th));
    }
    const double A = __shfl_sync(0xffffffffu, coef, 0);
    const double B = __shfl_sync(0xffffffffu, coef, 1);
    const double C = __shfl_sync(0xffffffffu, coef, 2);
    // every lane evaluates one uniform expression  base + c1 X + c2 Y :
    //   lanes 0..8  (R entry (r, c)):  I_rc + A [w]x_rc + B ([w]x^2)_rc
    //   lanes 9..11 (t entry r):       u_r + B (w x u)_r + C (w_r (w.u) - th2 u_r)
    const int r = lane < 9 ? lane / 3 : (lane < 12 ? lane - 9 : 0);
    const int cc = lane < 9 ? lane - 3 * r : 0;
    const bool is_t = lane >= 9;
    const double u0 = xi[3], u1 = xi[4], u2 = xi[5];
    const double wr = r == 0 ? w0 : (r == 1 ? w1 : w2);
    const double wc = cc == 0 ? w0 : (cc == 1 ? w1 : w2);
    const double ur = r == 0 ? u0 : (r == 1 ? u1 : u2);
    // [w]x_rc for r != c: +-w_k with k the remaining index
    const int kk = 3 - r - cc;
    const double wk = kk == 0 ? w0 : (kk == 1 ? w1 : w2);
    const double kx = (r == cc) ? 0.0 : (((cc - r + 3) % 3 == 1) ? -wk : wk);
    // (w x u)_r = w_{r+1} u_{r+2} - w_{r+2} u_{r+1}
    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    const double wa = r1 == 0 ? w0 : (r1 == 1 ? w1 : w2), wb = r2 == 0 ? w0 : (r2 == 1 ? w1 : w2);
    const double ua = r1 == 0 ? u0 : (r1 == 1 ? u1 : u2), ub = r2 == 0 ? u0 : (r2 == 1 ? u1 : u2);
    const double wxu = fma(wa, ub, -(wb * ua));
    const double wu = fma(w0, u0, fma(w1, u1, w2 * u2));
    const double base = is_t ? ur : ((r == cc) ? 1.0 : 0.0);
    const double c1 = is_t ? B : A;
    const double c2 = is_t ? C : B;
    const double X = is_t ? wxu : kx;
    const double Y = is_t ? fma(wr, wu, -th2 * ur) : fma(wr, wc, (r == cc) ? -th2 : 0.0);
    const double v = fma(c2, Y, fma(c1, X, base));
    if (lane < 12) dT[is_t ? 4 * r + 3 : 4 * r + cc] = v;
    __syncwarp();
}

// ------------------------------------------------------------------------------------------
// exact fixed-point accumulation: a double x (|x| < 2^62) is rounded toward -inf to a multiple of
// 2^-64 and held as a 128-bit two's-complement integer, split into four 32-bit chunks; chunk k is
// added into 64-bit accumulator k.  Sums of up to 2^32 values are exact in any order.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ void fx_add(unsigned long long* acc4, double x) {
    const double fl = floor(x);
    const long long hi = (long long)fl;
    const unsigned long long lo = (unsigned long long)((x - fl) * 18446744073709551616.0);
    const unsigned long long uhi = (unsigned long long)hi;
    atomicAdd(acc4 + 0, lo & 0xffffffffull);
    atomicAdd(acc4 + 1, lo >> 32);
    atomicAdd(acc4 + 2, uhi & 0xffffffffull);
    atomicAdd(acc4 + 3, uhi >> 32);
}

// value of a fixed-point number given its four (possibly carry-laden) 64-bit chunk sums
__device__ __forceinline__ double fx_value(unsigned long long c0, unsigned long long c1,
                                          unsigned long long c2, unsigned long long c3) {
    // v = c0 + c1 2^32 + c2 2^64 + c3 2^96 (mod 2^128)
    const unsigned long long lo_a = c0 + (c1 << 32);
    const unsigned long long carry = (lo_a < c0) ? 1ull : 0ull;
    const unsigned long long hi = (c1 >> 32) + c2 + (c3 << 32) + carry;
    return (double)(long long)hi + (double)lo_a * 5.421010862427522e-20;  // lo * 2^-64
}

// Reduce-scatter of 32 per-lane values over a warp by butterfly exchange (31 shuffles instead of
// 160): afterwards lane l holds the warp sum of value l.
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int level = 0; level < 5; ++level) {
        const int half = 16 >> level;
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = upper ? v[j] : v[j + half];
            const float keep = upper ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0];
}

// ------------------------------------------------------------------------------------------
// per-pixel accumulation and the block / scene reductions
// ------------------------------------------------------------------------------------------

// Shared memory of a tracking CTA.
struct TrackShared {
    float Rt[12];  // R (row-major) and t rounded once to FP32
    double Tsh[16];
    double part[kTrackWarps][32];
    unsigned long long csum[kAccumCopies][32][4];
    double xi[6], dT[12];
    int flag;
};

// Load the FP64 pose into shared memory and round R, t once to FP32 (threads 0..15).  The caller
// synchronises afterwards.
__device__ __forceinline__ void load_pose(TrackShared& sh, const double* T_wc) {
    if (threadIdx.x < 16) {
        const double x = T_wc[threadIdx.x];
        sh.Tsh[threadIdx.x] = x;
        if (threadIdx.x < 12) {
            const int r = threadIdx.x >> 2, c = threadIdx.x & 3;
            sh.Rt[c < 3 ? 3 * r + c : 9 + r] = __double2float_rn(x);
        }
    }
}

// Residual and Jacobian of one pixel (Eq. (taylor)), Huber-weighted, added to the 30 terms:
// 21 of H = sum w J J^T, 6 of b = sum w J r, E = sum w r^2, n_valid, n_huber.
template <class Map>
__device__ __forceinline__ void track_pixel(const Map& map, const float* __restrict__ depth, const Intr& K,
                                            const float* R, const float* t, const Params& prm, int pix,
                                            float (&acc)[32]) {
    const float D = __ldg(depth + pix);
    if (!depth_ok(D, K.depth_max)) return;
    const int v = pix / K.width;
    const int u = pix - v * K.width;
    float dw[3], P[3];
    ray_world(K, R, u, v, dw);
#pragma unroll
    for (int i = 0; i < 3; ++i) P[i] = ray_coord(D, dw[i], t[i]);
    const int mx = round_voxel(P[0], prm.inv_vs);
    const int my = round_voxel(P[1], prm.inv_vs);
    const int mz = round_voxel(P[2], prm.inv_vs);
    const long long idx = map.find(mx, my, mz);
    if (idx < 0) return;
    float psi, g0, g1, g2;
    if (!map.voxel(idx, psi, g0, g1, g2)) return;
    const float gn2 = g0 * g0 + g1 * g1 + g2 * g2;
    if (!(gn2 > 0.0f)) return;
    const float inv_gn = rsqrtf(gn2);
    const float gx = g0 * inv_gn, gy = g1 * inv_gn, gz = g2 * inv_gn;
    // P - v_s m with a single rounding per component
    const float dx = fmaf(-(float)mx, prm.vs, P[0]);
    const float dy = fmaf(-(float)my, prm.vs, P[1]);
    const float dz = fmaf(-(float)mz, prm.vs, P[2]);
    const float r = psi + (gx * dx + gy * dy + gz * dz);
    const float J[6] = {P[1] * gz - P[2] * gy, P[2] * gx - P[0] * gz, P[0] * gy - P[1] * gx, gx, gy, gz};
    const float delta = prm.huber;
    const float ar = fabsf(r);
    const float w = ar <= delta ? 1.0f : __fdividef(delta, ar);
    int q = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float wJi = w * J[i];
#pragma unroll
        for (int j = i; j < 6; ++j) acc[q++] += wJi * J[j];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] += w * J[i] * r;
    acc[27] += w * r * r;
    acc[28] += 1.0f;
    acc[29] += ar > delta ? 1.0f : 0.0f;
}

// The direct SDF tracker the paper compares against (Eqs. dir_dist, dir_grad): psi interpolated
// trilinearly over the 8 voxels of the cell containing P -- 8 lookups per pixel -- with r = d(P)
// and J = (P x grad d, grad d), grad d the interpolant's exact gradient.  The cell's lowest corner
// is floor(P (1/v_s)) on the FP32 index path; a = (P - v_s b) / v_s with v_s b split exactly.
// Same Huber weighting and terms as track_pixel.
template <class Map>
__device__ __forceinline__ void track_pixel_trilinear(const Map& map, const float* __restrict__ depth,
                                                      const Intr& K, const float* R, const float* t,
                                                      const Params& prm, int pix, float (&acc)[32]) {
    const float D = __ldg(depth + pix);
    if (!depth_ok(D, K.depth_max)) return;
    const int v = pix / K.width;
    const int u = pix - v * K.width;
    float dw[3], P[3];
    ray_world(K, R, u, v, dw);
#pragma unroll
    for (int i = 0; i < 3; ++i) P[i] = ray_coord(D, dw[i], t[i]);
    int b[3];
    float a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        b[i] = (int)floorf(__fmul_rn(P[i], prm.inv_vs));
        const float bf = (float)b[i];
        const float vh = __fmul_rn(prm.vs, bf);
        const float vl = __fmaf_rn(prm.vs, bf, -vh);
        a[i] = __fsub_rn(__fsub_rn(P[i], vh), vl) * prm.inv_vs;
    }
    float d = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // each corner is accumulated as soon as it is read
        const long long idx = map.find(b[0] + (q & 1), b[1] + ((q >> 1) & 1), b[2] + ((q >> 2) & 1));
        if (idx < 0) return;
        float c, g0, g1, g2;
        if (!map.voxel(idx, c, g0, g1, g2)) return;
        const float wx = (q & 1) ? a[0] : 1.0f - a[0];
        const float wy = (q & 2) ? a[1] : 1.0f - a[1];
        const float wz = (q & 4) ? a[2] : 1.0f - a[2];
        d += c * wx * wy * wz;
        gx += ((q & 1) ? c : -c) * wy * wz;
        gy += ((q & 2) ? c : -c) * wx * wz;
        gz += ((q & 4) ? c : -c) * wx * wy;
    }
    gx *= prm.inv_vs;
    gy *= prm.inv_vs;
    gz *= prm.inv_vs;
    const float r = d;
    const float J[6] = {P[1] * gz - P[2] * gy, P[2] * gx - P[0] * gz, P[0] * gy - P[1] * gx, gx, gy, gz};
    const float delta = prm.huber;
    const float ar = fabsf(r);
    const float w = ar <= delta ? 1.0f : __fdividef(delta, ar);
    int q = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float wJi = w * J[i];
#pragma unroll
        for (int j = i; j < 6; ++j) acc[q++] += wJi * J[j];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] += w * J[i] * r;
    acc[27] += w * r * r;
    acc[28] += 1.0f;
    acc[29] += ar > delta ? 1.0f : 0.0f;
}

// Block reduction of the per-thread terms: warps reduce-scatter (lane l <- term l), then a fixed
// FP64 tree over the warps leaves the block totals in part[0][0..29].  All threads call it.
__device__ __forceinline__ void block_reduce_terms(TrackShared& sh, float (&acc)[32]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    sh.part[warp][lane] = (double)warp_reduce_scatter32(acc);
    __syncthreads();
#pragma unroll
    for (int h = kTrackWarps / 2; h > 0; h >>= 1) {
        if (warp < h) sh.part[warp][lane] += sh.part[warp + h][lane];
        __syncthreads();
    }
}

// Add the block totals to accumulator copy `copy` of a scene and take a ticket; returns (in
// every thread) whether this block was the scene's last of `n_parts`.
__device__ __forceinline__ bool add_partial_and_ticket(TrackShared& sh, unsigned long long* accum,
                                                       unsigned int* counter, int copy, unsigned n_parts) {
    if (threadIdx.x < kTerms) fx_add(accum + ((copy % kAccumCopies) * 32 + threadIdx.x) * 4, sh.part[0][threadIdx.x]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned ticket = atomicAdd(counter, 1u);
        sh.flag = (ticket == n_parts - 1) ? 1 : 0;
    }
    __syncthreads();
    return sh.flag != 0;
}

// Finish a scene's step (called by every thread of the block that took the last ticket): read
// and clear the exact sums, solve in FP64, update the pose (loaded in sh.Tsh) and write the
// statistics.  Ends with a block-wide barrier so the block may continue with other work.
__device__ __forceinline__ void finish_scene(TrackShared& sh, unsigned long long* accum, unsigned int* counter,
                                             const Params& prm, double* T_wc, gsdf_track_stats* stats) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __threadfence();
    {
        unsigned long long* src = accum + ((size_t)warp * 32 + lane) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sh.csum[warp][lane][q] = __ldcg(src + q);
            src[q] = 0ull;
        }
    }
    __syncthreads();
#pragma unroll
    for (int h = kAccumCopies / 2; h > 0; h >>= 1) {
        if (warp < h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) sh.csum[warp][lane][q] += sh.csum[warp + h][lane][q];
        }
        __syncthreads();
    }
    if (warp == 0) {
        sh.part[0][lane] = lane < kTerms ? fx_value(sh.csum[0][lane][0], sh.csum[0][lane][1], sh.csum[0][lane][2],
                                                    sh.csum[0][lane][3])
                                         : 0.0;
        __syncwarp();
        const double* total = sh.part[0];
        if (lane == 0) *counter = 0u;
        const long long n_valid = (long long)(total[28] + 0.5);
        const bool ok = solve6_warp(total, prm.damping, n_valid, sh.xi);
        if (ok) se3_exp_warp(sh.xi, sh.dT);
        // T <- dT * T: lanes 0..11 compute one entry each of the top three rows
        if (ok && lane < 12) {
            const int i = lane >> 2, j = lane & 3;
            double tn = (sh.dT[4 * i + 0] * sh.Tsh[j] + sh.dT[4 * i + 1] * sh.Tsh[4 + j]) + sh.dT[4 * i + 2] * sh.Tsh[8 + j];
            if (j == 3) tn += sh.dT[4 * i + 3];
            T_wc[lane] = tn;
        }
        if (stats) {
            if (lane < 21) stats->H[lane] = total[lane];
            else if (lane < 27) stats->b[lane - 21] = total[lane];
            if (lane < 6) stats->xi[lane] = ok ? sh.xi[lane] : 0.0;
            if (lane == 0) {
                stats->energy = total[27];
                stats->n_valid = n_valid;
                stats->n_huber = (long long)(total[29] + 0.5);
                stats->status = ok ? (int)GSDF_OK : (int)GSDF_ERR_DEGENERATE;
                stats->pad = 0;
            }
        }
    }
    __syncthreads();
}

}  // namespace gsdf
