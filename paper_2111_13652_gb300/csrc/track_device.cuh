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

// FP64 on this GPU: every FP64 warp instruction occupies the SM sub-partition's FP64 pipe for
// about 64 cycles, whatever the number of active lanes, and two independent FP64 instructions of
// one warp do not overlap; integer and FP32 instructions take a few cycles.  FP64 code is
// therefore costed in FP64 warp instructions on the critical path, and the finishing code keeps
// the method's FP64 arithmetic but issues few of them:
//   * the grid-wide sum is exact fixed-point integer arithmetic (associative, hence deterministic
//     in any order) and is converted to FP64 with integer instructions, rounded once;
//   * compares, maxima and power-of-two scalings of FP64 values act on their bit patterns;
//   * the 6x6 system is solved by one warp holding one entry of the augmented upper triangle
//     [H | -b] per lane (27 lanes), two FP64 instructions per elimination step, and the
//     exponential map evaluates its three coefficients and twelve entries side by side.

// 2^k as a double (k within the normal exponent range)
__device__ __forceinline__ double exp2i(int k) { return __hiloint2double((1023 + k) << 20, 0); }
// e such that x * 2^-e lies in [0.5, 1), for finite x > 0 with a normal exponent
__device__ __forceinline__ int exponent_of(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1022; }
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
// -x by an integer xor of the sign bit (kept opaque, so that it is not turned into an FP64
// negation; inside an fma operand write -x instead, which costs nothing)
__device__ __forceinline__ double neg_d(double x) {
    int hi = __double2hiint(x);
    asm("xor.b32 %0, %0, 0x80000000;" : "+r"(hi));
    return __hiloint2double(hi, __double2loint(x));
}
// x > 0 (false for zeros, negatives and NaN, true for +inf)
__device__ __forceinline__ bool pos_d(double x) {
    const long long b = dbits(x);
    return b > 0 && b <= 0x7ff0000000000000ll;
}
// x * 2^k, exact, as an exponent update on the bit pattern; zeros are returned unchanged.  Sets
// `slow` when x or the result is not a normal number (subnormal, overflow, inf, NaN), where the
// returned value is meaningless and the caller must take another path.
__device__ __forceinline__ double scale2(double x, int k, bool& slow) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int e = (hi >> 20) & 0x7ff;
    const bool zero = ((hi & 0x7fffffff) | lo) == 0;
    slow = !zero && ((unsigned)(e - 1) >= 2046u || (unsigned)(e + k - 1) >= 2046u);
    return zero ? x : __hiloint2double(hi + (int)((unsigned)k << 20), lo);
}

// lane of entry (i, k), i <= k <= 6, of the augmented upper triangle; index of (i, k), k < 6,
// among the 21 upper-triangle terms of H
__device__ __forceinline__ int aug_lane(int i, int k) { return i * 7 - i * (i - 1) / 2 + (k - i); }
__device__ __forceinline__ int h21_index(int i, int k) { return i * 6 - i * (i - 1) / 2 + (k - i); }

// The same solve by lane 0 alone: the damped matrix factorised in place by Cholesky (packed
// lower triangle, row i at i (i + 1) / 2) with the pivot test s_j > 1e-12 max diag, then the two
// triangular solves; every lane returns the outcome.  Taken only when the warp-parallel solve
// below meets a value outside the normal FP64 range.
static __device__ __noinline__ bool solve6_serial(const double* Hb, double tr, double lam_scale, long long n_valid,
                                           double* xi) {
    const int lane = threadIdx.x & 31;
    int ok = 0;
    if (lane == 0) {
        double L[21], y[6];
        const double lam = lam_scale != 0.0 ? lam_scale * tr : 0.0;
        double maxd = 0.0;
#pragma unroll 1
        for (int i = 0; i < 6; ++i) {
#pragma unroll 1
            for (int k = 0; k < i; ++k) L[i * (i + 1) / 2 + k] = Hb[h21_index(k, i)];
            const double dg = Hb[h21_index(i, i)] + lam;
            L[i * (i + 1) / 2 + i] = dg;
            maxd = dg > maxd ? dg : maxd;
        }
        ok = n_valid >= 6 && maxd > 0.0;
#pragma unroll 1
        for (int j = 0; j < 6 && ok; ++j) {
            double* Lj = L + j * (j + 1) / 2;
            double s = Lj[j];
#pragma unroll 1
            for (int k = 0; k < j; ++k) s -= Lj[k] * Lj[k];
            ok = s > 1e-12 * maxd;
            Lj[j] = sqrt(s);
#pragma unroll 1
            for (int i = j + 1; i < 6; ++i) {
                double* Li = L + i * (i + 1) / 2;
                double v = Li[j];
#pragma unroll 1
                for (int k = 0; k < j; ++k) v -= Li[k] * Lj[k];
                Li[j] = v / Lj[j];
            }
        }
        if (ok) {
#pragma unroll 1
            for (int i = 0; i < 6; ++i) {
                double v = -Hb[21 + i];
#pragma unroll 1
                for (int k = 0; k < i; ++k) v -= L[i * (i + 1) / 2 + k] * y[k];
                y[i] = v / L[i * (i + 1) / 2 + i];
            }
#pragma unroll 1
            for (int i = 5; i >= 0; --i) {
                double v = y[i];
#pragma unroll 1
                for (int k = i + 1; k < 6; ++k) v -= L[k * (k + 1) / 2 + i] * xi[k];
                xi[i] = v / L[i * (i + 1) / 2 + i];
            }
        }
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Solve (H + lambda I) xi = -b, lambda = damping * trace(H) / 6 = lam_scale * tr, with one warp
// (the damped Gauss-Newton step of Sec. 4.1).  Hb (shared): the 21 upper-triangle terms of H
// (row-major) then the 6 of b; tr = trace(H) as the caller has it; lam_scale = damping / 6.
// Degenerate (returns false, uniform across the warp) if fewer than 6 residuals, a diagonal
// entry of H + lambda I that is not positive, or an LDL^T pivot d_j <= 1e-12 max diag (the test
// of the Cholesky factorisation).  Otherwise writes xi (shared) and returns true.
//
// Method: rows and columns are scaled by powers of two s_i ~ diag_i^-1/2 (exact), then
// Gauss-Jordan elimination without division: step j replaces every row i != j by
//     n_j (p_j row_i - a_ij row_j),   p_j = current pivot, n_j = 2^-e with p_j n_j in [1/2, 1)
// (for i > j, a_ij = a_ji by symmetry of the trailing block, which holds exactly since the
// update is symmetric).  The rows below j are the Schur complement times sigma_{j+1} =
// prod_{k<=j} p_k n_k, so d_j (of the scaled matrix) = p_j / sigma_j and the pivot test is
// p_j > 1e-12 maxd s_j^2 sigma_j; lane 27, which holds no entry, forms c sigma_j (c = 1e-12
// maxd) inside the steps' own multiply instruction.  At the end row i reads d_i x_i = c_i, and the
// six quotients are formed at once from a hardware reciprocal estimate refined by Newton's
// iteration (relative error of order the square of the estimate's), then one correction of the
// quotient against its residual.  Powers of two are applied to the bit patterns; a value that
// leaves the normal range on the way sends the system to solve6_serial.
__device__ __forceinline__ bool solve6_warp(const double* Hb, double tr, double lam_scale, long long n_valid,
                                            double* xi) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    constexpr int kTestLane = 27;
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
    const bool test_lane = lane == kTestLane;

    // entries with the damping on the diagonal: one FP64 instruction for the warp
    double h = 0.0;
    if (active) h = ek < 6 ? Hb[h21_index(ei, ek)] : neg_d(Hb[21 + ei]);
    const double hl = fma(lam_scale, tr, h);
    double a = (active && ei == ek && (dbits(lam_scale) << 1) != 0) ? hl : h;

    // lane j < 6: damped diagonal d_j; positivity, maximum (on the bit patterns), scale 2^k_j
    const int dl = lane < 6 ? lane : 0;
    const double dj = __shfl_sync(full, a, aug_lane(dl, dl));
    const bool bad_diag = __any_sync(full, lane < 6 && !pos_d(dj));
    if (n_valid < 6 || bad_diag) return false;
    const long long djb = dbits(dj);
    const unsigned mhi = __reduce_max_sync(full, lane < 6 ? (unsigned)(djb >> 32) : 0u);
    const unsigned mlo = __reduce_max_sync(full, (lane < 6 && (unsigned)(djb >> 32) == mhi) ? (unsigned)djb : 0u);
    const double maxd = __longlong_as_double((long long)(((unsigned long long)mhi << 32) | mlo));
    const int my_k = -(exponent_of(lane < 6 ? dj : 1.0) >> 1);
    const int k_i = __shfl_sync(full, my_k, ei);
    const int k_k = __shfl_sync(full, my_k, ek < 6 ? ek : 0);
    bool slow = false, sl;
    a = scale2(a, k_i + (ek < 6 ? k_k : 0), sl);
    slow |= active && sl;

    double cs = maxd;       // test lane: c sigma_j once step j's multiply has run
    double mul = 1e-12;     // test lane: its factor in step j's multiply (then p_{j-1} n_{j-1})
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double p = __shfl_sync(full, a, aug_lane(j, j));
        const double m = __shfl_sync(full, a, ei > j ? aug_lane(j, ei) : aug_lane(ei < j ? ei : j, j));
        const double ajk = __shfl_sync(full, a, aug_lane(j, ek > j ? ek : j));
        const int kj = __shfl_sync(full, my_k, j);
        const bool upd_row = active && ei != j && ek > j;   // rows i != j, columns right of j
        const bool upd = upd_row || (active && ei == ek && ei < j);  // or the diagonal of an earlier pivot row
        const double pa = (test_lane ? mul : p) * (test_lane ? cs : a);
        const double t = fma(-m, upd_row ? ajk : 0.0, pa);
        const bool ppos = pos_d(p);
        const int ep = exponent_of(ppos ? p : 1.0);
        const double ts = scale2(t, -ep, sl);
        slow |= upd && sl;
        a = upd ? ts : a;
        // the pivot test of row j, meaningful on the test lane: p_j > c sigma_j s_j^2
        const double thr = scale2(pa, 2 * kj, sl);
        slow |= test_lane && sl;
        bad |= test_lane && !(ppos && dbits(p) > dbits(thr));
        cs = pa;
        mul = scale2(p, -ep, sl);
        slow |= test_lane && ppos && sl;
    }
    // lanes (i, 6): x_i = c_i / d_i, then unscaled by s_i
    const double d = __shfl_sync(full, a, aug_lane(ei, ei));
    double r0;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(d));
    const double r1 = fma(r0, fma(-d, r0, 1.0), r0);
    const double q0 = a * r1;
    const double x = scale2(fma(r1, fma(-d, q0, a), q0), k_i, sl);
    slow |= active && ek == 6 && sl;
    if (__any_sync(full, slow)) return solve6_serial(Hb, tr, lam_scale, n_valid, xi);
    if (__any_sync(full, bad)) return false;
    if (active && ek == 6) xi[ei] = x;
    __syncwarp();
    return true;
}

// exp of the twist xi = (omega, upsilon) by one warp (the update T <- exp(xi^) T of Sec. 4.1):
// R = I + A [w]x + B [w]x^2, t = (I + B [w]x + C [w]x^2) u with A = sin(th)/th,
// B = (1 - cos th)/th^2, C = (th - sin th)/th^3 and [w]x^2 = w w^T - th^2 I.  Lanes 0..8 write
// R (entry (lane / 3, lane % 3)) and lanes 9..11 t into dT (row-major 3x4, shared); xi is in
// shared memory.  For th^2 < 1e-2 lanes 12..14 evaluate the coefficients' Taylor series in th^2
// up to th^8 (truncation error below th^10 / 11! < 3e-18), while the entry lanes form their
// products in the same instructions: nine FP64 instructions in all.  Larger angles use sincos.
__device__ __forceinline__ void se3_exp_warp(const double* xi, double* dT) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const double w0 = xi[0], w1 = xi[1], w2 = xi[2], u0 = xi[3], u1 = xi[4], u2 = xi[5];
    const bool is_t = lane >= 9 && lane < 12;
    const int r = lane < 9 ? lane / 3 : (is_t ? lane - 9 : 0);
    const int c = lane < 9 ? lane - 3 * r : 0;
    const int r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
    auto pick = [](int k, double x0, double x1, double x2) { return k == 0 ? x0 : (k == 1 ? x1 : x2); };
    const double wr = pick(r, w0, w1, w2), wc = pick(c, w0, w1, w2), ur = pick(r, u0, u1, u2);
    // three-term dot products: (w x u)_r on the t lanes, w.u on lane 16, th^2 = w.w elsewhere
    double a0 = w0, b0 = w0, a1 = w1, b1 = w1, a2 = w2, b2 = w2;
    if (lane == 16) { b0 = u0; b1 = u1; b2 = u2; }
    if (is_t) {
        a0 = pick(r1, w0, w1, w2);
        b0 = pick(r2, u0, u1, u2);
        a1 = neg_d(pick(r2, w0, w1, w2));
        b1 = pick(r1, u0, u1, u2);
        a2 = 0.0;
        b2 = 0.0;
    }
    const double dot = fma(a0, b0, fma(a1, b1, a2 * b2));
    const double th2 = __shfl_sync(full, dot, 15);
    const double wu = __shfl_sync(full, dot, 16);
    // ([w]x^2)_rc = w_r w_c - [r == c] th2 on the R lanes, ([w]x^2 u)_r = w_r (w.u) - th2 u_r on
    // the t lanes; coefficient lanes 12..14 hold A, B, C
    double Y, coef;
    if (dbits(th2) < dbits(1e-2)) {
        constexpr double kA[5] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880};
        constexpr double kB[5] = {1.0 / 2, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800};
        constexpr double kC[5] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800};
        auto kcoef = [&](int k) { return lane == 12 ? kA[k] : (lane == 13 ? kB[k] : kC[k]); };
        const bool is_c = lane >= 12 && lane < 15;
        // step 1: Horner's first step | R lanes: Y | t lanes: th2 u_r
        const double s1 = fma(is_c ? kcoef(4) : (is_t ? ur : wr), is_c || is_t ? th2 : wc,
                              is_c ? kcoef(3) : ((!is_t && r == c) ? neg_d(th2) : 0.0));
        // step 2: Horner | t lanes: Y = w_r (w.u) - th2 u_r
        const double s2 = fma(is_c ? s1 : wr, is_c ? th2 : wu, is_c ? kcoef(2) : neg_d(s1));
        coef = fma(fma(s2, th2, kcoef(1)), th2, kcoef(0));
        Y = is_t ? s2 : s1;
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        coef = lane == 12 ? sn / th : (lane == 13 ? (1.0 - cs) / th2 : (th - sn) / (th2 * th));
        Y = is_t ? fma(wr, wu, -(th2 * ur)) : fma(wr, wc, r == c ? -th2 : 0.0);
    }
    const double A = __shfl_sync(full, coef, 12);
    const double B = __shfl_sync(full, coef, 13);
    const double C = __shfl_sync(full, coef, 14);
    // [w]x_rc for r != c: -w_k if c follows r cyclically, +w_k otherwise (k the third index)
    const double wk = pick(3 - r - c, w0, w1, w2);
    const double X = is_t ? dot : (r == c ? 0.0 : (c == r1 ? neg_d(wk) : wk));
    const double base = is_t ? ur : (r == c ? 1.0 : 0.0);
    const double v = fma(is_t ? C : B, Y, fma(is_t ? B : A, X, base));
    if (lane < 12) dT[is_t ? 4 * r + 3 : 4 * r + c] = v;
    __syncwarp();
}

// T <- dT T for the top three rows of a 4x4 rigid transform (row-major, shared), lanes 0..11
// one entry each; returns the new entry (lane i*4+j) in the calling lanes.
__device__ __forceinline__ double compose_entry(const double* dT, const double* T) {
    const int lane = threadIdx.x & 31;
    const int i = (lane >> 2) < 3 ? lane >> 2 : 0, j = lane & 3;
    const double* d = dT + 4 * i;
    return fma(d[2], T[8 + j], fma(d[1], T[4 + j], fma(d[0], T[j], j == 3 ? d[3] : 0.0)));
}

// ------------------------------------------------------------------------------------------
// exact fixed-point accumulation: a value x (|x| < 2^62) is rounded toward -inf to a multiple of
// 2^-64 and held as a 128-bit two's-complement integer, split into four 32-bit chunks; chunk k is
// added into 64-bit accumulator k.  Sums of up to 2^32 values are exact in any order.
// ------------------------------------------------------------------------------------------

// the four chunks of the fixed-point form of a float, with integer instructions only
__device__ __forceinline__ void fx_chunks(float v, unsigned (&c)[4]) {
    const unsigned b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xffu);
    const unsigned m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    // |v| 2^64 = m 2^p
    const int p = (e ? e : 1) - 150 + 64;
    unsigned long long lo = 0ull, hi = 0ull;
    bool inexact = false;
    if (p >= 64) {
        hi = p < 128 ? (unsigned long long)m << (p - 64) : 0ull;
    } else if (p >= 0) {
        lo = (unsigned long long)m << p;
        hi = p > 40 ? (unsigned long long)m >> (64 - p) : 0ull;
    } else {
        const int s = -p;
        lo = s < 32 ? (unsigned long long)(m >> s) : 0ull;
        inexact = s < 32 ? (m & ((1u << s) - 1u)) != 0u : m != 0u;
    }
    if (b >> 31) {  // floor(-|v| 2^64) = ~M + 1 - inexact
        lo = ~lo;
        hi = ~hi;
        if (!inexact) {
            ++lo;
            if (lo == 0ull) ++hi;
        }
    }
    c[0] = (unsigned)lo;
    c[1] = (unsigned)(lo >> 32);
    c[2] = (unsigned)hi;
    c[3] = (unsigned)(hi >> 32);
}

// the 128-bit value c0 + c1 2^32 + c2 2^64 + c3 2^96 (mod 2^128) of four chunk sums, as hi:lo
__device__ __forceinline__ void fx_join(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                        unsigned long long c3, unsigned long long& lo, unsigned long long& hi) {
    lo = c0 + (c1 << 32);
    hi = (c1 >> 32) + c2 + (c3 << 32) + (lo < c0 ? 1ull : 0ull);
}

// the two's-complement fixed-point number hi:lo * 2^-64 as the nearest double (ties to even),
// with integer instructions only
__device__ __forceinline__ double fx_to_double(unsigned long long lo, unsigned long long hi) {
    const bool neg = (long long)hi < 0;
    if (neg) {  // magnitude: ~v + 1
        lo = ~lo + 1ull;
        hi = ~hi + (lo == 0ull ? 1ull : 0ull);
    }
    if ((hi | lo) == 0ull) return 0.0;
    // top: the 64 leading bits of the magnitude (most significant bit set); rest: the bits below;
    // the magnitude lies in [2^(n-1), 2^n)
    int n;
    unsigned long long top, rest;
    if (hi != 0ull) {
        const int lz = __clzll((long long)hi);
        top = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
        rest = lo << lz;
        n = 128 - lz;
    } else {
        const int lz = __clzll((long long)lo);
        top = lo << lz;
        rest = 0ull;
        n = 64 - lz;
    }
    unsigned long long mant = top >> 11;  // 53 bits
    const bool half = (top >> 10) & 1ull;
    const bool sticky = (top & 0x3ffull) != 0ull || rest != 0ull;
    if (half && (sticky || (mant & 1ull))) ++mant;
    if (mant >> 53) {
        mant >>= 1;
        ++n;
    }
    // value = mant 2^(n - 53 - 64): biased exponent n - 65 + 1023
    const unsigned long long bits = ((unsigned long long)(n + 958) << 52) | (mant & 0x000fffffffffffffull) |
                                    (neg ? 0x8000000000000000ull : 0ull);
    return __longlong_as_double((long long)bits);
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
    unsigned wchunk[kTrackWarps][4][32];  // per-warp fixed-point chunks of the 32 term slots
    double total[32];                     // finishing block: the scene's sums in FP64
    unsigned long long tsum[4][32];  // chunk sums of the 32 term slots (finishing block)
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

// Pixels pix0, pix0 + stride, ... < n_px of a depth image of the given width, each handed with its
// depth value and column/row to f(D, pix, u, v); the next pixel's depth is loaded one iteration
// ahead, so that its latency overlaps the current pixel's lookups, and (u, v) advance by the
// stride's own (column, row) offset instead of a division per pixel.  d0 = depth[pix0] (loaded
// earlier by the caller if pix0 < n_px).
template <class F>
__device__ __forceinline__ void for_pixels(const float* __restrict__ depth, int width, int pix0, int n_px,
                                           int stride, float d0, F&& f) {
    int v = pix0 / width, u = pix0 - v * width;
    const int sv = stride / width, su = stride - sv * width;
    float Dn = d0;
    for (int pix = pix0; pix < n_px; pix += stride) {
        const float D = Dn;
        if (pix + stride < n_px) Dn = __ldg(depth + pix + stride);
        f(D, pix, u, v);
        u += su;
        v += sv;
        if (u >= width) {
            u -= width;
            ++v;
        }
    }
}

// Residual and Jacobian of one pixel (Eq. (taylor)), Huber-weighted, added to the 30 terms:
// 21 of H = sum w J J^T, 6 of b = sum w J r, E = sum w r^2, n_valid, n_huber.
template <class Map>
__device__ __forceinline__ void track_pixel(const Map& map, float D, const Intr& K, const float* R, const float* t,
                                            const Params& prm, int u, int v, float (&acc)[32]) {
    if (!depth_ok(D, K.depth_max)) return;
    float dw[3], P[3];
    ray_world(K, R, u, v, dw);
#pragma unroll
    for (int i = 0; i < 3; ++i) P[i] = ray_coord(D, dw[i], t[i]);
    const int mx = round_voxel(P[0], prm.inv_vs);
    const int my = round_voxel(P[1], prm.inv_vs);
    const int mz = round_voxel(P[2], prm.inv_vs);
    float psi, g0, g1, g2;
    if (!map.lookup(mx, my, mz, psi, g0, g1, g2)) return;
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
__device__ __forceinline__ void track_pixel_trilinear(const Map& map, float D, const Intr& K, const float* R,
                                                      const float* t, const Params& prm, int u, int v,
                                                      float (&acc)[32]) {
    if (!depth_ok(D, K.depth_max)) return;
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

// Block reduction of the per-thread terms into exact fixed-point sums: every warp reduce-
// scatters its terms in FP32 (lane l <- term l) and converts each warp sum to its four
// fixed-point chunks with integer instructions; warp q < 4 then sums chunk q of the 32 term
// slots over the warps.  Returns, in threads 0..127, chunk threadIdx.x / 32 of the block sum of
// term threadIdx.x % 32 (0 elsewhere).  All threads call it.
// kWarps: the block's warps (4 <= kWarps <= kTrackWarps).
template <int kWarps = kTrackWarps>
__device__ __forceinline__ unsigned long long block_reduce_terms(TrackShared& sh, float (&acc)[32]) {
    static_assert(kWarps >= 4 && kWarps <= kTrackWarps, "block size");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned c[4];
    fx_chunks(warp_reduce_scatter32(acc), c);
#pragma unroll
    for (int q = 0; q < 4; ++q) sh.wchunk[warp][q][lane] = c[q];
    __syncthreads();
    unsigned long long s = 0ull;
    if (warp < 4) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) s += sh.wchunk[w][warp][lane];
    }
    return s;
}

// Add a block's chunk sums (from block_reduce_terms) to accumulator copy `copy` of a scene and
// take a ticket; returns (in every thread) whether this block was the scene's last of
// `n_parts`.  Accumulator layout: word (copy * 4 + chunk) * 32 + term, so that the additions
// and the finishing reads are contiguous.  Only warps 0..3 write, so only they fence before the
// ticket.
__device__ __forceinline__ bool add_partial_and_ticket(TrackShared& sh, unsigned long long s,
                                                       unsigned long long* accum, unsigned int* counter, int copy,
                                                       unsigned n_parts) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 4) {
        if (lane < kTerms) atomicAdd(accum + (copy % kAccumCopies) * 128 + warp * 32 + lane, s);
        __threadfence();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (threadIdx.x == 0) sh.flag = (atomicAdd(counter, 1u) == n_parts - 1) ? 1 : 0;
    }
    __syncthreads();
    return sh.flag != 0;
}

// Warps 0..3 sum chunk (threadIdx.x / 32) of the 32 term slots of a scene's exact accumulators
// over their copies (one coalesced load per copy), zero the copies if `clear`, and leave the chunk
// sums in sh.tsum with the trace of H in the empty slot 30; they meet at a named barrier.  Other
// warps do nothing.
__device__ __forceinline__ void gather_sums(TrackShared& sh, unsigned long long* accum, bool clear) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    if (warp < 4) {
        unsigned long long* col = accum + warp * 32 + lane;
        unsigned long long s[kAccumCopies];
#pragma unroll
        for (int c = 0; c < kAccumCopies; ++c) s[c] = __ldcg(col + c * 128);
        if (clear) {
#pragma unroll
            for (int c = 0; c < kAccumCopies; ++c) col[c * 128] = 0ull;
        }
#pragma unroll
        for (int h = kAccumCopies / 2; h > 0; h >>= 1)
#pragma unroll
            for (int c = 0; c < h; ++c) s[c] += s[c + h];
        // slot 30 (empty otherwise): the trace of H, as the sum of the diagonal terms' chunks
        unsigned long long tr = 0ull;
#pragma unroll
        for (int i = 0; i < 6; ++i) tr += __shfl_sync(full, s[0], h21_index(i, i));
        sh.tsum[warp][lane] = lane == 30 ? tr : s[0];
        asm volatile("bar.sync 1, 128;" ::: "memory");
    }
}

// Warp 0, after gather_sums: the exact sums rounded once to FP64 (sh.total), the damped 6x6
// solve, the exponential map and T' = exp(xi^) T with T in sh.Tsh; writes the statistics if
// `stats`.  Returns whether the system was solved, and in lanes 0..11 the new pose entry
// (lane = 4 row + column; unchanged from sh.Tsh when the system is degenerate).
__device__ __forceinline__ bool solve_step_warp(TrackShared& sh, const Params& prm, gsdf_track_stats* stats,
                                                double& tn) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    // lanes 0..29 the terms, lane 30 the trace: exact sums rounded once to FP64
    unsigned long long lo, hi;
    fx_join(sh.tsum[0][lane], sh.tsum[1][lane], sh.tsum[2][lane], sh.tsum[3][lane], lo, hi);
    const double v = fx_to_double(lo, hi);
    sh.total[lane] = v;
    // the counts are whole numbers: their integer part is exact
    const long long n_valid = (long long)__shfl_sync(full, hi, 28);
    const long long n_huber = (long long)__shfl_sync(full, hi, 29);
    const double tr = __shfl_sync(full, v, 30);
    __syncwarp();
    const double* total = sh.total;
    const bool ok = solve6_warp(total, tr, prm.lam_scale, n_valid, sh.xi);
    tn = lane < 12 ? sh.Tsh[lane] : 0.0;
    if (ok) {
        se3_exp_warp(sh.xi, sh.dT);
        tn = compose_entry(sh.dT, sh.Tsh);  // T <- dT T, lanes 0..11
    }
    if (stats) {
        if (lane < 21) stats->H[lane] = total[lane];
        else if (lane < 27) stats->b[lane - 21] = total[lane];
        if (lane < 6) stats->xi[lane] = ok ? sh.xi[lane] : 0.0;
        if (lane == 0) {
            stats->energy = total[27];
            stats->n_valid = n_valid;
            stats->n_huber = n_huber;
            stats->status = ok ? (int)GSDF_OK : (int)GSDF_ERR_DEGENERATE;
            stats->pad = 0;
        }
    }
    return ok;
}

// Finish a scene's step (called by every thread of the block that took the last ticket): read
// and clear the exact sums, solve in FP64, update the pose (loaded in sh.Tsh) and write the
// statistics.  Ends with a block-wide barrier so the block may continue with other work.
__device__ __forceinline__ void finish_scene(TrackShared& sh, unsigned long long* accum, unsigned int* counter,
                                             const Params& prm, double* T_wc, gsdf_track_stats* stats) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 4) __threadfence();  // the other blocks' additions, ordered before their tickets
    gather_sums(sh, accum, true);
    if (warp == 0) {
        if (lane == 0) *counter = 0u;
        double tn;
        if (solve_step_warp(sh, prm, stats, tn) && lane < 12) T_wc[lane] = tn;
    }
    __syncthreads();
}

}  // namespace gsdf
