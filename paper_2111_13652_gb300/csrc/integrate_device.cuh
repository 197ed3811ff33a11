// Device building blocks of depth fusion (Eqs. (sdf_update), (gradient_update), pixel-driven as
// in Sec. 5.3), shared by the single-scene kernel (integrate.cu) and the batched persistent kernel
// (batch.cu).
#pragma once

#include "gsdf_internal.cuh"

namespace gsdf {

constexpr int kIntThreads = 256;

// Normal of pixel (u, v) from its 4-neighbours (FP32 index path).  Returns false if the pixel
// is rejected: image border, invalid neighbour, depth jump > T, zero cross product, or an angle
// to the viewing ray of 75 degrees or more (cos < cos_max).
__device__ __forceinline__ bool pixel_normal(const float* __restrict__ depth, const Intr& K,
                                             const Params& prm, int u, int v, float D, float n[3]) {
    if (u < 1 || u >= K.width - 1 || v < 1 || v >= K.height - 1) return false;
    const size_t row = (size_t)v * K.width;
    const float Dl = __ldg(depth + row + u - 1), Dr = __ldg(depth + row + u + 1);
    const float Du = __ldg(depth + row - K.width + u), Dd = __ldg(depth + row + K.width + u);
    const float nb[4] = {Dl, Dr, Du, Dd};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!depth_ok(nb[i], K.depth_max)) return false;
        const float diff = __fsub_rn(nb[i], D);
        if (diff > prm.trunc || diff < -prm.trunc) return false;
    }
    float pl[3], pr[3], pu[3], pd[3], p[3];
    backproject(K, u - 1, v, Dl, pl);
    backproject(K, u + 1, v, Dr, pr);
    backproject(K, u, v - 1, Du, pu);
    backproject(K, u, v + 1, Dd, pd);
    backproject(K, u, v, D, p);
    const float a[3] = {__fsub_rn(pr[0], pl[0]), __fsub_rn(pr[1], pl[1]), __fsub_rn(pr[2], pl[2])};
    const float b[3] = {__fsub_rn(pd[0], pu[0]), __fsub_rn(pd[1], pu[1]), __fsub_rn(pd[2], pu[2])};
    n[0] = __fsub_rn(__fmul_rn(a[1], b[2]), __fmul_rn(a[2], b[1]));
    n[1] = __fsub_rn(__fmul_rn(a[2], b[0]), __fmul_rn(a[0], b[2]));
    n[2] = __fsub_rn(__fmul_rn(a[0], b[1]), __fmul_rn(a[1], b[0]));
    const float nn = dot3_rn(n, n);
    if (!(nn > 0.0f)) return false;
    // The 75 degree test is a discrete decision and is taken exactly as specified: n normalised by
    // correctly rounded divisions, oriented so that n . p > 0, and c = (n . p) / sqrt(p . p)
    // compared with cos_max.  Most pixels are decided by a cheap evaluation of the same cosine,
    // |n . p| rsqrt(n . n) rsqrt(p . p): both evaluations are within 3e-6 (relative) of the true
    // cosine near the threshold (a dozen roundings of at most 2^-24, reciprocal square roots within
    // 2 ulp, cancellation in n . p at most 1 / c <= 4), so outside a margin of 4e-5 cos_max they take
    // the same decision; inside it the exact evaluation decides.  The normal returned feeds sums
    // only (Eq. gradient_update), so it is scaled by the reciprocal square root.
    const float pp = dot3_rn(p, p);
    const float dpr = dot3_rn(n, p);
    const float rn = rsqrtf(nn);
    const float cf = fabsf(dpr) * rn * rsqrtf(pp);
    const float margin = 4e-5f * fabsf(prm.cos_max) + 1e-7f;
    const bool fast = nn > 1e-30f && pp > 1e-30f && fabsf(cf - prm.cos_max) > margin;
    bool keep = cf > prm.cos_max;
    // the sign of the raw n . p orients the normal whenever |n . p| is clearly above rounding
    // (cf > 1e-4); a kept normal nearly perpendicular to its ray (possible only for cos_max < 1e-4)
    // takes the orientation of the exact evaluation too
    bool neg = dpr < 0.0f;
    if (!fast || (keep && !(cf > 1e-4f))) {
        const float s = __fsqrt_rn(nn);
        const float e[3] = {__fdiv_rn(n[0], s), __fdiv_rn(n[1], s), __fdiv_rn(n[2], s)};
        float dp = dot3_rn(e, p);
        neg = dp < 0.0f;
        if (neg) dp = -dp;
        keep = __fdiv_rn(dp, __fsqrt_rn(pp)) >= prm.cos_max;
    }
    if (!keep) return false;
    const float k = neg ? -rn : rn;
    n[0] *= k;
    n[1] *= k;
    n[2] *= k;
    return true;
}

// Per-ray cache of the last block looked up (consecutive voxels of a ray mostly share a block),
// and of one block found ahead: the block of the ray's last sample.  The first lookups of a warp's
// rays happen at about the same step and run together; finding the far block in the same pass
// spares each ray a second lookup later, which the lanes would reach at different steps.
struct BlockCache {
    int bx = 0x7fffffff, by = 0, bz = 0;
    long long base = -1;  // payload index of local voxel 0, or -1 when the block is unusable
    int fx = 0x7fffffff, fy = 0, fz = 0;
    long long fbase = -1;  // the far block's payload index, -1 if unknown
    bool ahead = false;    // the far block has been looked for
};

template <class Map>
__device__ __forceinline__ long long voxel_index(const Map& map, int mx, int my, int mz, BlockCache& bc,
                                                 int* err, unsigned int* n_new, const int* far);

// The far block is only found, never inserted: a block is created by a weighted update to one of
// its voxels (allocation stays exactly the set of updated blocks).  Not yet allocated, it is
// looked up (and inserted) when the ray reaches it, as any block.
template <>
__device__ __forceinline__ long long voxel_index<HashMap>(const HashMap& map, int mx, int my, int mz, BlockCache& bc,
                                                          int* err, unsigned int* n_new, const int* far) {
    const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
    if (bx != bc.bx || by != bc.by || bz != bc.bz) {
        if (bc.fbase >= 0 && bx == bc.fx && by == bc.fy && bz == bc.fz) {
            bc.base = bc.fbase;
            bc.fbase = -1;
        } else {
            bc.base = map.find_or_insert(bx * 8, by * 8, bz * 8, err, n_new);
            if (!bc.ahead) {
                bc.ahead = true;
                const int fx = floor_div8(far[0]), fy = floor_div8(far[1]), fz = floor_div8(far[2]);
                if (fx != bx || fy != by || fz != bz) {
                    bc.fbase = map.find(fx * 8, fy * 8, fz * 8);
                    bc.fx = fx;
                    bc.fy = fy;
                    bc.fz = fz;
                }
            }
        }
        bc.bx = bx;
        bc.by = by;
        bc.bz = bz;
    }
    if (bc.base < 0) return -1;
    return bc.base + ((mx & 7) + 8 * (my & 7) + 64 * (mz & 7));
}

// FP16 maps: the index returned addresses the frame's accumulators (entry * 512 + local)
template <>
__device__ __forceinline__ long long voxel_index<HashMap16>(const HashMap16& map, int mx, int my, int mz,
                                                            BlockCache& bc, int* err, unsigned int* n_new,
                                                            const int* far) {
    const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
    if (bx != bc.bx || by != bc.by || bz != bc.bz) {
        if (bc.fbase >= 0 && bx == bc.fx && by == bc.fy && bz == bc.fz) {
            bc.base = bc.fbase;
            bc.fbase = -1;
        } else {
            const long long idx = map.base.find_or_insert(bx * 8, by * 8, bz * 8, err, n_new);
            bc.base = -1;
            if (idx >= 0) {
                const int ci = acc_entry(map, idx >> 9, err);
                if (ci >= 0) bc.base = (long long)ci * kBlockVoxels;
            }
            // the far block (found, not inserted) and its frame accumulator entry, as for FP32 maps;
            // an entry that then receives no sums is read and freed by the apply pass unchanged
            if (!bc.ahead) {
                bc.ahead = true;
                const int fx = floor_div8(far[0]), fy = floor_div8(far[1]), fz = floor_div8(far[2]);
                if (fx != bx || fy != by || fz != bz) {
                    const long long fidx = map.base.find(fx * 8, fy * 8, fz * 8);
                    if (fidx >= 0) {
                        const int fci = acc_entry(map, fidx >> 9, err);
                        if (fci >= 0) {
                            bc.fbase = (long long)fci * kBlockVoxels;
                            bc.fx = fx;
                            bc.fy = fy;
                            bc.fz = fz;
                        }
                    }
                }
            }
        }
        bc.bx = bx;
        bc.by = by;
        bc.bz = bz;
    }
    if (bc.base < 0) return -1;
    return bc.base + ((mx & 7) + 8 * (my & 7) + 64 * (mz & 7));
}

// (w d, w n) and w of one visit
__device__ __forceinline__ void scatter(const DenseMap& m, long long i, float4 v, float w) {
    atomicAdd(m.A + i, v);
    atomicAdd(m.W + i, w);
}
__device__ __forceinline__ void scatter(const HashMap& m, long long i, float4 v, float w) {
    atomicAdd(m.A + i, v);
    atomicAdd(m.W + i, w);
}
__device__ __forceinline__ void scatter(const HashMap16& m, long long i, float4 v, float w) {
    atomicAdd(m.accA + i, v);
    atomicAdd(m.accW + i, w);
}

template <>
__device__ __forceinline__ long long voxel_index<DenseMap>(const DenseMap& map, int mx, int my, int mz, BlockCache&,
                                                           int*, unsigned int*, const int*) {
    return map.find(mx, my, mz);
}

// FP16 maps, second pass: fold listed accumulator entry q (of *m.acount) into its block, with
// Eqs. (sdf_update) and (gradient_update) in FP32 for the voxels that received updates:
//   W' = W + S_w,  psi' = (W psi + S_d) / W',  gbar' = (W gbar + S_n) / W',
// re-encoded (psi' / sigma_b, gbar') to FP16 with round-to-nearest.  The block scale becomes
// max(sigma_b, max |psi'| over the updated voxels); the other voxels already satisfy
// |psi| <= sigma_b, so only when the scale grows are they re-encoded too.  kApplyThreads threads
// fold one entry, thread t taking voxels t + kApplyThreads k: every thread first reads its
// voxels' weight sums, then issues the payload and sum loads of all its updated voxels together;
// a voxel without updates costs that one 4-byte read (its payload is read only when the scale
// grows).  The entry's sums are cleared and the entry freed for the next frame.  Called by all
// threads of the block, uniformly; red: kApplyThreads / 32 floats of shared memory.
constexpr int kApplyThreads = 128;
constexpr int kApplyPer = kBlockVoxels / kApplyThreads;

// FP16 maps, between the passes: list the occupied accumulator entries of the frame as (entry,
// hash slot) pairs, with one atomic per warp that finds any.  Entries e = first, first + stride,
// ...; called by whole warps (the loop runs to the table size rounded up to 32).
__device__ __forceinline__ void list16_entries(const HashMap16& m, unsigned first, unsigned stride) {
    const unsigned n = m.amask + 1u;
    const unsigned nr = (n + 31u) & ~31u;
    const int lane = threadIdx.x & 31;
    for (unsigned e = first; e < nr; e += stride) {
        const int slot = e < n ? __ldcg(m.akeys + e) : -1;
        const unsigned b = __ballot_sync(0xffffffffu, slot >= 0);
        unsigned base = 0u;
        if (lane == 0 && b) base = atomicAdd(m.acount, (unsigned)__popc(b));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (slot >= 0)
            reinterpret_cast<int2*>(m.alist)[base + __popc(b & ((1u << lane) - 1u))] = make_int2((int)e, slot);
    }
}

__device__ __forceinline__ void apply16_entry(const HashMap16& m, unsigned q, float trunc, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int2 e = __ldcg(reinterpret_cast<const int2*>(m.alist) + q);  // (entry, hash slot)
    const unsigned ci = (unsigned)e.x;
    const int slot = e.y;
    const float sigma = __ldcg(m.scale + slot);
    const long long gbase = (long long)slot * kBlockVoxels, abase = (long long)ci * kBlockVoxels;
    float sw[kApplyPer];
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) sw[k] = __ldcg(m.accW + abase + threadIdx.x + k * kApplyThreads);
    float4 sa[kApplyPer];
    ushort4 h[kApplyPer];
    float w[kApplyPer];
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) {
        const int v = threadIdx.x + k * kApplyThreads;
        const bool upd = sw[k] > 0.0f;
        sa[k] = upd ? __ldcg(m.accA + abase + v) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        h[k] = upd ? __ldcg(m.H + gbase + v) : make_ushort4(0, 0, 0, 0);
        w[k] = upd ? __ldcg(m.W + gbase + v) : 0.0f;
    }
    float psi[kApplyPer], g0[kApplyPer], g1[kApplyPer], g2[kApplyPer];
    float amax = 0.0f;
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) {
        const float wn = w[k] + sw[k];
        psi[k] = (w[k] * (__half2float(__ushort_as_half(h[k].x)) * sigma) + sa[k].x) / wn;
        g0[k] = (w[k] * __half2float(__ushort_as_half(h[k].y)) + sa[k].y) / wn;
        g1[k] = (w[k] * __half2float(__ushort_as_half(h[k].z)) + sa[k].z) / wn;
        g2[k] = (w[k] * __half2float(__ushort_as_half(h[k].w)) + sa[k].w) / wn;
        w[k] = wn;
        if (sw[k] > 0.0f) amax = fmaxf(amax, fabsf(psi[k]));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) red[warp] = amax;
    __syncthreads();
    float bmax = red[0];
#pragma unroll
    for (int k = 1; k < kApplyThreads / 32; ++k) bmax = fmaxf(bmax, red[k]);
    float sig = fmaxf(sigma, bmax);
    if (!(sig > 0.0f)) sig = trunc;  // nothing observed yet: any positive scale encodes zeros
    const bool rescale = sig != sigma && sigma > 0.0f;
#pragma unroll
    for (int k = 0; k < kApplyPer; ++k) {
        const int v = threadIdx.x + k * kApplyThreads;
        if (sw[k] > 0.0f) {
            ushort4 o4;
            o4.x = __half_as_ushort(__float2half_rn(psi[k] / sig));
            o4.y = __half_as_ushort(__float2half_rn(g0[k]));
            o4.z = __half_as_ushort(__float2half_rn(g1[k]));
            o4.w = __half_as_ushort(__float2half_rn(g2[k]));
            m.H[gbase + v] = o4;
            m.W[gbase + v] = w[k];
            m.accA[abase + v] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            m.accW[abase + v] = 0.0f;
        } else if (rescale) {
            ushort4 hh = __ldcg(m.H + gbase + v);
            hh.x = __half_as_ushort(__float2half_rn((__half2float(__ushort_as_half(hh.x)) * sigma) / sig));
            m.H[gbase + v] = hh;
        }
    }
    if (threadIdx.x == 0) {
        m.scale[slot] = sig;
        m.akeys[ci] = -1;
    }
    __syncthreads();
}

// Fuse the ray of pixel `pix` (Eqs. (sdf_update), (gradient_update), Sec. 5.3) into the map:
// validity and normal test, then every distinct voxel of the ray's samples inside the band
// receives (w d, w n_w) and w.  `pose` is the FP32-rounded pose; counts go to rays / visits.
template <class Map>
__device__ __forceinline__ void integrate_ray(const Map& map, const float* __restrict__ depth, const Intr& K,
                                              const Params& prm, const PoseF& pose, int pix, int* err,
                                              unsigned int* n_new, unsigned int& rays, unsigned int& visits) {
    const float D = __ldg(depth + pix);
    if (!depth_ok(D, K.depth_max)) return;
    const int v = pix / K.width;
    const int u = pix - v * K.width;
    float n[3];
    if (!pixel_normal(depth, K, prm, u, v, D, n)) return;
    ++rays;
    // world normal R n (value path)
    const float nwx = pose.R[0] * n[0] + pose.R[1] * n[1] + pose.R[2] * n[2];
    const float nwy = pose.R[3] * n[0] + pose.R[4] * n[1] + pose.R[5] * n[2];
    const float nwz = pose.R[6] * n[0] + pose.R[7] * n[1] + pose.R[8] * n[2];
    float dw[3];
    ray_world(K, pose.R, u, v, dw);
    const int Kb = prm.band_half;
    const float inv_band = 1.0f / (prm.trunc - prm.eps);
    // voxel of the ray's last sample (for the block found ahead)
    int far[3];
    {
        const float z = __fadd_rn(D, __fmul_rn((float)Kb, prm.half_vs));
        far[0] = round_voxel(ray_coord(z, dw[0], pose.t[0]), prm.inv_vs);
        far[1] = round_voxel(ray_coord(z, dw[1], pose.t[1]), prm.inv_vs);
        far[2] = round_voxel(ray_coord(z, dw[2], pose.t[2]), prm.inv_vs);
    }
    int k = 0;
    int pmx = 0x7fffffff, pmy = 0, pmz = 0;
    BlockCache bc;
    // Outer loop over the ray's distinct voxels; the inner loop advances through samples
    // that round to the voxel already visited, so that a warp runs the visit body about
    // once per distinct voxel rather than once per sample.
    while (true) {
        bool found = false;
        int mx = 0, my = 0, mz = 0;
        while (k <= 2 * Kb) {
            const float z = __fadd_rn(D, __fmul_rn((float)(k - Kb), prm.half_vs));
            ++k;
            mx = round_voxel(ray_coord(z, dw[0], pose.t[0]), prm.inv_vs);
            my = round_voxel(ray_coord(z, dw[1], pose.t[1]), prm.inv_vs);
            mz = round_voxel(ray_coord(z, dw[2], pose.t[2]), prm.inv_vs);
            if (mx != pmx || my != pmy || mz != pmz) {
                found = true;
                break;
            }
        }
        if (!found) break;
        pmx = mx;
        pmy = my;
        pmz = mz;
        const float vc[3] = {__fmul_rn((float)mx, prm.vs), __fmul_rn((float)my, prm.vs),
                             __fmul_rn((float)mz, prm.vs)};
        const float zv = __fadd_rn(dot_row(pose.RT + 6, vc), pose.tinv[2]);
        const float d = __fsub_rn(zv, D);
        if (d > prm.trunc || d < -prm.trunc) continue;
        const float w = d <= prm.eps ? 1.0f : (prm.trunc - d) * inv_band;
        if (!(w > 0.0f)) continue;
        const long long idx = voxel_index(map, mx, my, mz, bc, err, n_new, far);
        if (idx < 0) continue;
        scatter(map, idx, make_float4(w * d, w * nwx, w * nwy, w * nwz), w);
        ++visits;
    }
}

}  // namespace gsdf
