// Internal device-side definitions shared by the library's kernels (not part of the C ABI).
//
// Map layout in HBM
//   dense:  payload arrays indexed by the linear voxel index (x fastest) of the box;
//   hashed: an open-addressing table of 2^k slots of packed 64-bit block keys; slot s owns the
//           payload of one 8^3 block, voxels s * 512 + local (local = x + 8 y + 64 z).
//   payload per voxel: float4 A = (W psi, g.x, g.y, g.z) and float W -- 20 bytes, in two
//   arrays so that one 16-byte vector load/atomic covers A.  Storing W psi (not psi) makes the
//   running average of Eq. (sdf_update) a pure sum, order-independent and atomic-friendly:
//   psi = A.x / W when read.
#pragma once

#include <math.h>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsdf.h"

namespace gsdf {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kBlockVoxels = 512;
constexpr int kBias = 1 << 20;  // block coordinates are stored biased by 2^20 in 21 bits

// Device-side error word codes (first error wins).
constexpr int kErrNone = 0;

struct Intr {
    float fx, fy, cx, cy;
    int width, height;
    float depth_max;
    float ifx, ify;  // (float)(1 / fx) computed in FP64 then rounded once
};

struct Params {
    float vs, inv_vs, trunc, eps, half_vs, huber, cos_max;
    int band_half;  // K = ceil(T / (v_s / 2))
    double damping;
    double lam_scale;  // damping / 6: the Levenberg term is lam_scale * trace(H)
};

// The method parameters as the kernels use them, from the configuration values (the one place
// both gsdf_create and the allocation-free tracking step build them).
inline Params make_params(float voxel_size, float truncation, float weight_eps, float huber_delta,
                          float cos_max_angle, double damping) {
    Params p;
    p.vs = voxel_size;
    p.inv_vs = (float)(1.0 / (double)voxel_size);
    p.trunc = truncation;
    p.eps = weight_eps;
    p.half_vs = 0.5f * voxel_size;
    p.huber = huber_delta;
    p.cos_max = cos_max_angle;
    p.band_half = (int)ceil((double)truncation / (double)p.half_vs - 1e-6);
    p.damping = damping;
    p.lam_scale = damping / 6.0;
    return p;
}

// Pose rounded once from FP64: camera->world (R, t) and world->camera (R^T, -R^T t).
struct PoseF {
    float R[9], t[3], RT[9], tinv[3];
};

// ------------------------------------------------------------------------------------------
// block keys and hashing
// ------------------------------------------------------------------------------------------

__host__ __device__ inline int floor_div8(int m) { return m >> 3; }  // arithmetic shift = floor

__host__ __device__ inline unsigned long long pack_block(int bx, int by, int bz) {
    return ((unsigned long long)(unsigned)(bx + kBias) << 42) |
           ((unsigned long long)(unsigned)(by + kBias) << 21) |
           (unsigned long long)(unsigned)(bz + kBias);
}

__host__ __device__ inline void unpack_block(unsigned long long k, int* b) {
    b[0] = (int)((k >> 42) & 0x1FFFFF) - kBias;
    b[1] = (int)((k >> 21) & 0x1FFFFF) - kBias;
    b[2] = (int)(k & 0x1FFFFF) - kBias;
}

__host__ __device__ inline bool block_in_range(int bx, int by, int bz) {
    return bx >= -kBias && bx < kBias && by >= -kBias && by < kBias && bz >= -kBias && bz < kBias;
}

__host__ __device__ inline unsigned long long mix64(unsigned long long k) {
    k ^= k >> 31;
    k *= 0x7FB5D329728EA185ull;
    k ^= k >> 27;
    k *= 0x81DADEF4BC2DD44Dull;
    k ^= k >> 33;
    return k;
}

// Read-only loads issued where they are written (volatile asm is neither moved nor dropped), for
// loads that are issued speculatively before the branch that decides whether they are used.
__device__ __forceinline__ unsigned long long ld_nc_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.global.nc.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_nc_f32(const float* p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float4 ld_nc_f4(const float4* p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ ushort4 ld_nc_h4(const ushort4* p) {
    ushort4 v;
    asm volatile("ld.global.nc.v4.u16 {%0, %1, %2, %3}, [%4];" : "=h"(v.x), "=h"(v.y), "=h"(v.z), "=h"(v.w) : "l"(p));
    return v;
}

// ------------------------------------------------------------------------------------------
// maps
// ------------------------------------------------------------------------------------------

struct DenseMap {
    float4* A;
    float* W;
    int dims[3];
    int origin[3];

    __device__ __forceinline__ long long find(int mx, int my, int mz) const {
        int x = mx - origin[0], y = my - origin[1], z = mz - origin[2];
        if ((unsigned)x >= (unsigned)dims[0] || (unsigned)y >= (unsigned)dims[1] ||
            (unsigned)z >= (unsigned)dims[2])
            return -1;
        return ((long long)z * dims[1] + y) * dims[0] + x;
    }
    // Dense voxels always exist inside the box.
    __device__ __forceinline__ long long find_or_insert(int mx, int my, int mz, int* /*err*/,
                                                        unsigned int* /*n_new*/) const {
        return find(mx, my, mz);
    }
    // psi and the (unnormalised) gradient of voxel idx; false if unobserved (W = 0)
    __device__ __forceinline__ bool voxel(long long idx, float& psi, float& gx, float& gy, float& gz) const {
        const float w = __ldg(W + idx);
        const float4 a = __ldg(A + idx);  // issued with W: both loads in flight at once
        if (!(w > 0.0f)) return false;
        psi = __fdividef(a.x, w);
        gx = a.y;
        gy = a.z;
        gz = a.w;
        return true;
    }
    // find and voxel in one call (the tracking lookup of Eq. (taylor))
    __device__ __forceinline__ bool lookup(int mx, int my, int mz, float& psi, float& gx, float& gy, float& gz) const {
        const long long idx = find(mx, my, mz);
        return idx >= 0 && voxel(idx, psi, gx, gy, gz);
    }
};

struct HashMap {
    unsigned long long* keys;
    float4* A;
    float* W;
    unsigned long long mask;  // slots - 1
    int max_probe;

    __device__ __forceinline__ long long find(int mx, int my, int mz) const {
        int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
        if (!block_in_range(bx, by, bz)) return -1;
        unsigned long long key = pack_block(bx, by, bz);
        unsigned long long s = mix64(key) & mask;
        for (int p = 0; p < max_probe; ++p) {
            unsigned long long k = __ldg(keys + s);
            if (k == key) {
                int local = (mx & 7) + 8 * (my & 7) + 64 * (mz & 7);
                return (long long)s * kBlockVoxels + local;
            }
            if (k == kEmptyKey) return -1;
            s = (s + 1) & mask;
        }
        return -1;
    }

    // Lookup-or-insert used while other threads insert concurrently.  Keys are never removed,
    // so a stale read can only show an empty slot, which the compare-and-swap then resolves.
    __device__ __forceinline__ long long find_or_insert(int mx, int my, int mz, int* err,
                                                        unsigned int* n_new) const {
        int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
        if (!block_in_range(bx, by, bz)) {
            atomicCAS(err, kErrNone, (int)GSDF_ERR_CAPACITY);
            return -1;
        }
        unsigned long long key = pack_block(bx, by, bz);
        unsigned long long s = mix64(key) & mask;
        for (int p = 0; p < max_probe; ++p) {
            unsigned long long k = __ldcg(keys + s);
            if (k == kEmptyKey) {
                unsigned long long prev = atomicCAS(keys + s, kEmptyKey, key);
                if (prev == kEmptyKey) {
                    atomicAdd(n_new, 1u);
                    k = key;
                } else {
                    k = prev;
                }
            }
            if (k == key) {
                int local = (mx & 7) + 8 * (my & 7) + 64 * (mz & 7);
                return (long long)s * kBlockVoxels + local;
            }
            s = (s + 1) & mask;
        }
        atomicCAS(err, kErrNone, (int)GSDF_ERR_CAPACITY);
        return -1;
    }
    __device__ __forceinline__ bool voxel(long long idx, float& psi, float& gx, float& gy, float& gz) const {
        const float w = __ldg(W + idx);
        const float4 a = __ldg(A + idx);  // issued with W: both loads in flight at once
        if (!(w > 0.0f)) return false;
        psi = __fdividef(a.x, w);
        gx = a.y;
        gy = a.z;
        gz = a.w;
        return true;
    }
    // Slot of `key` probing from slot s + 1 on (s itself held another key), or -1: the rest of
    // find's probe sequence.
    __device__ __forceinline__ long long probe_on(unsigned long long key, unsigned long long s) const {
        for (int p = 1; p < max_probe; ++p) {
            s = (s + 1) & mask;
            const unsigned long long k = __ldg(keys + s);
            if (k == key) return (long long)s;
            if (k == kEmptyKey) return -1;
        }
        return -1;
    }
    // find and voxel in one call (the tracking lookup of Eq. (taylor)), with the same result.  The
    // voxel's payload in the key's home slot is loaded together with that slot's key, so that a
    // block found where it hashes to -- nearly every block at the tables' load factors -- costs one
    // round trip to memory instead of two; the loads of a block found further on are repeated.
    __device__ __forceinline__ bool lookup(int mx, int my, int mz, float& psi, float& gx, float& gy, float& gz) const {
        const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
        if (!block_in_range(bx, by, bz)) return false;
        const unsigned long long key = pack_block(bx, by, bz);
        const unsigned long long s = mix64(key) & mask;
        const int local = (mx & 7) + 8 * (my & 7) + 64 * (mz & 7);
        long long idx = (long long)s * kBlockVoxels + local;
        const unsigned long long k = ld_nc_u64(keys + s);
        float w = ld_nc_f32(W + idx);
        float4 a = ld_nc_f4(A + idx);
        if (k != key) {
            if (k == kEmptyKey || max_probe < 2) return false;
            const long long slot = probe_on(key, s);
            if (slot < 0) return false;
            idx = slot * kBlockVoxels + local;
            w = __ldg(W + idx);
            a = __ldg(A + idx);
        }
        if (!(w > 0.0f)) return false;
        psi = __fdividef(a.x, w);
        gx = a.y;
        gy = a.z;
        gz = a.w;
        return true;
    }
};

// FP16 payload on the same 8^3-block hash table.  Per voxel: half4 (psi / sigma_b, gbar) with
// gbar = g / W (|gbar| <= 1, same direction as g), and W in FP32; per block: sigma_b, a scale that
// only grows (the largest |psi| the block has held).  A frame is fused in two passes: the ray march
// adds (w d, w n, w) into FP32 accumulators of the blocks it touches, kept in a small
// open-addressing table keyed by hash slot; the occupied entries are listed, then one CTA per
// listed entry folds them in with Eq. (sdf_update) / (gradient_update) and re-encodes (round to
// nearest).
struct HashMap16 {
    HashMap base;      // keys, mask, probe limit (its A and W are unused)
    ushort4* H;        // [slots * 512] half bits of (psi / sigma_b, gbar_x, gbar_y, gbar_z)
    float* W;          // [slots * 512]
    float* scale;      // [slots] sigma_b
    int* akeys;        // [acap] hash slot owning each accumulator entry, -1 = free
    unsigned int amask;  // acap - 1 (acap a power of two)
    float4* accA;      // [acap * 512] (sum w d, sum w n)
    float* accW;       // [acap * 512] sum w
    int* alist;        // [2 acap] (entry, hash slot) of the occupied entries, listed after the march
    unsigned int* acount;  // number of listed entries (cleared once the apply pass is done)

    __device__ __forceinline__ long long find(int mx, int my, int mz) const { return base.find(mx, my, mz); }
    __device__ __forceinline__ bool voxel(long long idx, float& psi, float& gx, float& gy, float& gz) const {
        const float w = __ldg(W + idx);
        const ushort4 h = __ldg(H + idx);  // issued with W and the block scale
        const float sb = __ldg(scale + (idx >> 9));
        if (!(w > 0.0f)) return false;
        psi = __half2float(__ushort_as_half(h.x)) * sb;
        gx = __half2float(__ushort_as_half(h.y));
        gy = __half2float(__ushort_as_half(h.z));
        gz = __half2float(__ushort_as_half(h.w));
        return true;
    }
    // find and voxel in one call, the home slot's payload and scale loaded with its key (as
    // HashMap::lookup)
    __device__ __forceinline__ bool lookup(int mx, int my, int mz, float& psi, float& gx, float& gy, float& gz) const {
        const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
        if (!block_in_range(bx, by, bz)) return false;
        const unsigned long long key = pack_block(bx, by, bz);
        const unsigned long long s = mix64(key) & base.mask;
        const int local = (mx & 7) + 8 * (my & 7) + 64 * (mz & 7);
        long long idx = (long long)s * kBlockVoxels + local;
        const unsigned long long k = ld_nc_u64(base.keys + s);
        float w = ld_nc_f32(W + idx);
        ushort4 h = ld_nc_h4(H + idx);
        float sb = ld_nc_f32(scale + s);
        if (k != key) {
            if (k == kEmptyKey || base.max_probe < 2) return false;
            const long long slot = base.probe_on(key, s);
            if (slot < 0) return false;
            idx = slot * kBlockVoxels + local;
            w = __ldg(W + idx);
            h = __ldg(H + idx);
            sb = __ldg(scale + slot);
        }
        if (!(w > 0.0f)) return false;
        psi = __half2float(__ushort_as_half(h.x)) * sb;
        gx = __half2float(__ushort_as_half(h.y));
        gy = __half2float(__ushort_as_half(h.z));
        gz = __half2float(__ushort_as_half(h.w));
        return true;
    }
};

constexpr int kAccProbeLimit = 64;

// Accumulator entry of hash slot `slot` for this frame, inserted on first use with one
// compare-and-swap (entries are only freed by the apply pass, so no reader ever waits).  -1 when
// the probe limit is reached (recorded as GSDF_ERR_CAPACITY).
__device__ __forceinline__ int acc_entry(const HashMap16& m, long long slot, int* err) {
    unsigned int p = (unsigned int)mix64((unsigned long long)slot) & m.amask;
    for (int k = 0; k < kAccProbeLimit; ++k) {
        int v = __ldcg(m.akeys + p);
        if (v == -1) {
            v = atomicCAS(m.akeys + p, -1, (int)slot);
            if (v == -1) return (int)p;
        }
        if (v == (int)slot) return (int)p;
        p = (p + 1) & m.amask;
    }
    atomicCAS(err, kErrNone, (int)GSDF_ERR_CAPACITY);
    return -1;
}

// ------------------------------------------------------------------------------------------
// FP32 index path: correctly rounded operations in a fixed order, no contraction, so that every
// discrete decision (validity, voxel rounding, normal test, band test) is reproducible.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ bool depth_ok(float D, float dmax) { return D > 0.0f && D <= dmax; }

__device__ __forceinline__ void backproject(const Intr& K, int u, int v, float z, float p[3]) {
    float xn = __fmul_rn(__fsub_rn((float)u, K.cx), K.ifx);
    float yn = __fmul_rn(__fsub_rn((float)v, K.cy), K.ify);
    p[0] = __fmul_rn(z, xn);
    p[1] = __fmul_rn(z, yn);
    p[2] = z;
}

__device__ __forceinline__ float dot_row(const float* r, const float p[3]) {
    float s = __fadd_rn(__fmul_rn(r[0], p[0]), __fmul_rn(r[1], p[1]));
    return __fadd_rn(s, __fmul_rn(r[2], p[2]));
}

// World direction of pixel (u, v): d = R ray, ray = ((u - cx)/fx, (v - cy)/fy, 1),
// d_i = (R_i0 ray_0 + R_i1 ray_1) + R_i2.  The world point at depth z is P_i = z d_i + t_i.
__device__ __forceinline__ void ray_world(const Intr& K, const float* R, int u, int v, float d[3]) {
    const float xn = __fmul_rn(__fsub_rn((float)u, K.cx), K.ifx);
    const float yn = __fmul_rn(__fsub_rn((float)v, K.cy), K.ify);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = __fadd_rn(__fadd_rn(__fmul_rn(R[3 * i], xn), __fmul_rn(R[3 * i + 1], yn)), R[3 * i + 2]);
}

__device__ __forceinline__ float ray_coord(float z, float d, float t) { return __fadd_rn(__fmul_rn(z, d), t); }

__device__ __forceinline__ int round_voxel(float x, float inv_vs) {
    return (int)floorf(__fadd_rn(__fmul_rn(x, inv_vs), 0.5f));
}

__device__ __forceinline__ float dot3_rn(const float a[3], const float b[3]) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a[0], b[0]), __fmul_rn(a[1], b[1])), __fmul_rn(a[2], b[2]));
}

// Round an FP64 camera->world pose once to FP32 (R, t) and (R^T, -R^T t); -R^T t is formed in
// FP64 as ((R_0i t_0 + R_1i t_1) + R_2i t_2) without fused multiply-adds, then rounded.
__device__ inline void round_pose(const double* T, PoseF& q) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            q.R[3 * i + j] = __double2float_rn(T[4 * i + j]);
            q.RT[3 * i + j] = __double2float_rn(T[4 * j + i]);
        }
        q.t[i] = __double2float_rn(T[4 * i + 3]);
        double s = __dmul_rn(T[0 * 4 + i], T[3]);
        s = __dadd_rn(s, __dmul_rn(T[1 * 4 + i], T[7]));
        s = __dadd_rn(s, __dmul_rn(T[2 * 4 + i], T[11]));
        q.tinv[i] = __double2float_rn(-s);
    }
}

// The same rounding by the 24 lanes of one warp, one output value each (R: lanes 0..8, R^T:
// 9..17, t: 18..20, -R^T t: 21..23), with the operations and their order of round_pose: a block
// then waits for a few FP64 operations instead of thirty in one thread.  Called by the whole
// warp; the caller synchronises before reading q.
__device__ __forceinline__ void round_pose_warp(const double* T, PoseF& q) {
    const int lane = threadIdx.x & 31;
    if (lane < 9) {
        q.R[lane] = __double2float_rn(T[4 * (lane / 3) + lane % 3]);
    } else if (lane < 18) {
        const int k = lane - 9, i = k / 3, j = k % 3;  // (R^T)_ij = R_ji
        q.RT[k] = __double2float_rn(T[4 * j + i]);
    } else if (lane < 21) {
        q.t[lane - 18] = __double2float_rn(T[4 * (lane - 18) + 3]);
    } else if (lane < 24) {
        const int i = lane - 21;
        double s = __dmul_rn(T[0 * 4 + i], T[3]);
        s = __dadd_rn(s, __dmul_rn(T[1 * 4 + i], T[7]));
        s = __dadd_rn(s, __dmul_rn(T[2 * 4 + i], T[11]));
        q.tinv[i] = __double2float_rn(-s);
    }
}

// ------------------------------------------------------------------------------------------
// launchers (defined in the kernel translation units)
// ------------------------------------------------------------------------------------------

struct Scratch {
    unsigned long long* accum;  // [kAccumWords] fixed-point grid accumulators of the tracking terms
    unsigned int* counter;      // last-block-done ticket
    int* err;                   // sticky device error word
    unsigned int* n_blocks;     // number of allocated hash blocks
    int max_track_blocks;
    unsigned long long* chain;  // [kChainWords] chained tracking steps: 3 accumulator sets, 2 poses
};

constexpr int kAccumCopies = 16;  // grid accumulators are replicated to spread atomic traffic
constexpr int kAccumWords = kAccumCopies * 32 * 4;  // copies x 30 terms (21 H, 6 b, E, n_valid, n_huber, padded to 32) x 4 chunks
constexpr int kChainWords = 3 * kAccumWords + 32;     // three accumulator sets, then two 16-double poses

// n >= 2 Gauss-Newton steps as one chain of launches (track.cu; requires sc.chain)
cudaError_t launch_track_chain(const DenseMap* dm, const HashMap* hm, const HashMap16* hm16, bool trilinear,
                               const float* depth, const Intr& K, const Params& prm, double* T_wc,
                               gsdf_track_stats* stats, const Scratch& sc, int num_sms, int n, cudaStream_t st);

cudaError_t launch_track(const DenseMap* dm, const HashMap* hm, const float* depth, const Intr& K,
                         const Params& prm, double* T_wc, gsdf_track_stats* stats,
                         const Scratch& sc, int num_sms, cudaStream_t st);

cudaError_t launch_track_trilinear(const DenseMap* dm, const HashMap* hm, const float* depth, const Intr& K,
                                   const Params& prm, double* T_wc, gsdf_track_stats* stats, const Scratch& sc,
                                   int num_sms, cudaStream_t st);

cudaError_t launch_track16(const HashMap16& hm, const float* depth, const Intr& K, const Params& prm, double* T_wc,
                           gsdf_track_stats* stats, const Scratch& sc, int num_sms, cudaStream_t st);

cudaError_t launch_integrate16(const HashMap16& hm, const float* depth, const Intr& K, const Params& prm,
                               const double* T_wc, gsdf_integrate_stats* stats, const Scratch& sc, int num_sms,
                               cudaStream_t st);

cudaError_t launch_integrate(const DenseMap* dm, const HashMap* hm, const float* depth,
                             const Intr& K, const Params& prm, const double* T_wc,
                             gsdf_integrate_stats* stats, const Scratch& sc, cudaStream_t st);

}  // namespace gsdf

namespace gsdf {
// extraction / checkpoint (extract.cu).  *out_dev is allocated with cudaMalloc; caller frees.
cudaError_t extract_voxels(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                           cudaStream_t st, int num_sms, gsdf_voxel** out_dev, long long* n_out);
cudaError_t extract_points(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                           float voxel_size, int level, cudaStream_t st, int num_sms, gsdf_point** out_dev,
                           long long* n_out);
cudaError_t extract_mesh(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                         float voxel_size, cudaStream_t st, int num_sms, gsdf_triangle** out_dev, long long* n_out);
cudaError_t load_voxels(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, float trunc,
                        const gsdf_voxel* in_dev, long long n, int* err, unsigned int* n_blocks, cudaStream_t st,
                        int num_sms);
}  // namespace gsdf

// A map handle (the C ABI's opaque gsdf_handle).
struct gsdf_handle {
    gsdf_config cfg;
    bool fp16;
    gsdf::HashMap16 hm16;  // FP16 payload (hashed maps with GSDF_PAYLOAD_F16)
    cudaStream_t stream;
    int device;
    int num_sms;
    bool hashed;
    long long n_voxels;  // payload entries (dense box or slots * 512)
    gsdf::DenseMap dm;
    gsdf::HashMap hm;
    gsdf::Params prm;
    gsdf::Scratch sc;
    // cached CUDA graph of gsdf_track's launches, keyed by its arguments
    cudaStream_t capture_stream;
    cudaGraphExec_t track_exec;
    const float* g_depth;
    double* g_pose;
    gsdf_track_stats* g_stats;
    int g_iters;
    gsdf_intrinsics g_K;
};
