// Photometric + geometric voxel energy and its adjoint over an explicit voxel list (Sec. 4.2:
// Eqs. rgb_cost, intensity_proj, mean_color, variance; Eq. tracking with Eq. taylor; the surface
// point of Eq. grad_sdf_project).  See include/gsdf.h for the definition and the C ABI.
//
// Voxel index (built once by gsdf_energy_create): the list's voxels grouped by 8^3 block -- a
// compact open-addressing hash of block keys (16-byte slots) gives a block id, and a dense
// int32[512] array per block gives the list position of each of its voxels (-1 if absent).  The
// 32 pixels of a warp usually fall into two or three blocks, so their lookups share sectors.
//
// One evaluation, all on the handle's stream:
//   geo_kernel     thread per pixel of a keyframe (grid.y = keyframe): FP32 index path of the
//                  tracking step, nearest voxel through the index, the residual of Eq. taylor;
//                  the hit voxel's (dE/dpsi, dE/dg) go to an internal float4 accumulator (one red
//                  atomic), the keyframe's pose terms to per-thread registers;
//   merge_kernel   thread per voxel: writes dE/dpsi, dE/dg from the accumulator and dE/drho = 0
//                  (every output element once), and clears the accumulator (by red atomics of
//                  the negated values);
//   pairs_kernel   reads the visibility bit set (one word per voxel) and writes, per keyframe,
//                  the list of voxels it sees (one reservation per 1024 voxels and keyframe);
//   photo_kernel   thread per visible (voxel, keyframe) pair (grid.y = keyframe): projects the
//                  surface point, samples the keyframe's RGB bilinearly, adds its terms to the
//                  voxel's gradient with red atomics (coalesced: list order is voxel order), pose
//                  terms to per-thread registers;
//   finish_kernel  one block: energies, dE/dT and the left-perturbation gradient per keyframe,
//                  then clears the accumulators and list counters for the next evaluation.
// Per-keyframe accumulator (16 FP64): dE/dR (9, row-major), dE/dt (3), E_p, E_g, 2 spare.  A block
// reduces its threads' FP32 pose terms with a 16-value warp reduce-scatter and adds the block
// total to the accumulator with FP64 atomics.
#include <math.h>
#include <string.h>

#include <new>

#include "gsdf_internal.cuh"
#include "track_device.cuh"  // FP64 6x6 solve, SE(3) exponential and the 32-term warp reduce-scatter

using namespace gsdf;

namespace {

constexpr int kEThreads = 256;
constexpr int kEWarps = kEThreads / 32;
constexpr int kMaxFrames = 64;
constexpr int kSlots = 16;
constexpr int kSlotEp = 12, kSlotEg = 13;
constexpr unsigned kFull = 0xffffffffu;

struct EFrame {  // keyframe pose, camera -> world, rounded once to FP32
    float R[9], t[3];
};

struct __align__(16) IndexSlot {  // one probe = one 16-byte load
    unsigned long long key;
    int val;
    int pad;
};

struct IndexTable {  // voxel coordinate -> position in the list
    IndexSlot* slots;  // block key -> block id
    unsigned long long mask;
    int* vox;  // block id * 512 + local index -> list position, -1 if absent
};

struct EnergyArgs {
    long long n;
    int F;
    int nw;  // visibility words per voxel, ceil(F / 32)
    Intr K;
    float vs, inv_vs;
    const int* m;
    const float* psi;
    const float* g;
    const float* rho;
    const double* T;
    const unsigned* nu;  // n x nw words, bit i of voxel j = nu_ij
    const float4* rgb;   // F x H x W, (r, g, b, 0)
    const float* depth;  // F x H x W
    IndexTable tab;
    double lambda;
    const double* grad_scale;
    double* acc;               // F x kSlots
    float4* vacc;              // n: geometric (dE/dpsi, dE/dg) of each voxel, cleared by merge_kernel
    bool geo_grads;            // vacc holds this evaluation's geometric voxel gradients
    float4* cacc;              // n: colour sums and pair count of each voxel (bundle adjustment)
    double* bacc;              // F x 32: Gauss-Newton terms per keyframe (bundle adjustment)
    int* pairs;                // F x n: voxels keyframe i sees, pair_count[i] of them
    unsigned int* pair_count;  // F
    float* dpsi;
    float* dg;
    float* drho;
};

// ------------------------------------------------------------------------------------------
// index of the voxel list
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long first_slot(unsigned long long key, unsigned long long mask) {
    return mix64(key) & mask;
}

__device__ __forceinline__ int local_index(int mx, int my, int mz) { return (mx & 7) + 8 * (my & 7) + 64 * (mz & 7); }

// List position of voxel m, -1 if it is not in the list.
__device__ __forceinline__ int index_find(const IndexTable& t, int mx, int my, int mz) {
    const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
    if (!block_in_range(bx, by, bz)) return -1;
    const unsigned long long key = pack_block(bx, by, bz);
    unsigned long long s = first_slot(key, t.mask);
    for (unsigned long long probe = 0; probe <= t.mask; ++probe) {
        const IndexSlot e = t.slots[s];
        if (e.key == key) return t.vox[(long long)e.val * kBlockVoxels + local_index(mx, my, mz)];
        if (e.key == kEmptyKey) return -1;
        s = (s + 1) & t.mask;
    }
    return -1;
}

// Insert block key with a fresh id (from *count) unless present; returns the slot or -1 if the
// table is full (it never is: it has at least twice as many slots as keys).
__device__ __forceinline__ long long block_insert(IndexSlot* slots, unsigned long long mask, unsigned long long key,
                                                  unsigned int* count) {
    unsigned long long s = first_slot(key, mask);
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&slots[s].key, kEmptyKey, key);
        if (prev == kEmptyKey) {
            if (count) slots[s].val = (int)atomicAdd(count, 1u);
            return (long long)s;
        }
        if (prev == key) return (long long)s;
        s = (s + 1) & mask;
    }
    return -1;
}

__device__ __forceinline__ int block_id(const IndexSlot* slots, unsigned long long mask, unsigned long long key) {
    unsigned long long s = first_slot(key, mask);
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const IndexSlot e = slots[s];
        if (e.key == key) return e.val;
        if (e.key == kEmptyKey) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// Pass 1 of the index build: every voxel's block key into a table sized for n keys, ids 0.. in
// order of first insertion.  A voxel outside the block range sets *err.
__global__ void index_blocks_kernel(IndexSlot* slots, unsigned long long mask, const int* m, long long n,
                                    unsigned int* count, int* err) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int bx = floor_div8(m[3 * j]), by = floor_div8(m[3 * j + 1]), bz = floor_div8(m[3 * j + 2]);
        if (!block_in_range(bx, by, bz)) {
            atomicCAS(err, 0, (int)GSDF_ERR_INVALID_ARG);
            continue;
        }
        if (block_insert(slots, mask, pack_block(bx, by, bz), count) < 0) atomicCAS(err, 0, (int)GSDF_ERR_CAPACITY);
    }
}

// Pass 2: list positions into the per-block arrays (a voxel listed twice sets *err), and the
// block keys into the compact table with their ids.
__global__ void index_fill_kernel(const IndexSlot* big, unsigned long long big_mask, IndexTable t, const int* m,
                                  long long n, int* err) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        const int mx = m[3 * j], my = m[3 * j + 1], mz = m[3 * j + 2];
        const int bx = floor_div8(mx), by = floor_div8(my), bz = floor_div8(mz);
        if (!block_in_range(bx, by, bz)) continue;
        const unsigned long long key = pack_block(bx, by, bz);
        const int id = block_id(big, big_mask, key);
        if (id < 0) continue;
        if (atomicCAS(t.vox + (long long)id * kBlockVoxels + local_index(mx, my, mz), -1, (int)j) != -1)
            atomicCAS(err, 0, (int)GSDF_ERR_INVALID_ARG);  // the same voxel twice in the list
    }
}

__global__ void index_compact_kernel(const IndexSlot* big, unsigned long long big_mask, IndexTable t, int* err) {
    for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s <= big_mask;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const IndexSlot e = big[s];
        if (e.key == kEmptyKey) continue;
        const long long c = block_insert(t.slots, t.mask, e.key, nullptr);
        if (c < 0)
            atomicCAS(err, 0, (int)GSDF_ERR_CAPACITY);
        else
            t.slots[c].val = e.val;
    }
}

__global__ void pack_rgb_kernel(const float* rgb, float4* out, long long n_px) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_px; p += (long long)gridDim.x * blockDim.x)
        out[p] = make_float4(rgb[3 * p], rgb[3 * p + 1], rgb[3 * p + 2], 0.0f);
}

// ------------------------------------------------------------------------------------------
// FP32 index path of the pixel decisions (the same correctly rounded operations, in the same
// order, as the oracle): surface point, camera coordinates, projection.
// ------------------------------------------------------------------------------------------

struct SurfPt {
    float s[3];   // psi ghat
    float gh[3];  // ghat
    float p[3];   // v_s m - psi ghat
    float nr;     // |g|
};

__device__ __forceinline__ bool surface_point32(int mx, int my, int mz, float psi, float g0, float g1, float g2, float vs,
                                                SurfPt& o) {
    float n2 = __fmul_rn(g0, g0);
    n2 = __fadd_rn(n2, __fmul_rn(g1, g1));
    n2 = __fadd_rn(n2, __fmul_rn(g2, g2));
    if (!(n2 > 0.0f)) return false;
    o.nr = __fsqrt_rn(n2);
    const float gv[3] = {g0, g1, g2};
    const int mv[3] = {mx, my, mz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.gh[k] = __fdiv_rn(gv[k], o.nr);
        o.s[k] = __fmul_rn(psi, o.gh[k]);
        o.p[k] = __fsub_rn(__fmul_rn(vs, (float)mv[k]), o.s[k]);
    }
    return true;
}

// d = p - t and x = R^T d, x_i = (R_0i d_0 + R_1i d_1) + R_2i d_2; false unless x_2 > 0
__device__ __forceinline__ bool project32(const SurfPt& sp, const EFrame& f, const Intr& K, float d[3], float x[3],
                                          float& u, float& v) {
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = __fsub_rn(sp.p[k], f.t[k]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        x[i] = __fadd_rn(__fadd_rn(__fmul_rn(f.R[i], d[0]), __fmul_rn(f.R[3 + i], d[1])), __fmul_rn(f.R[6 + i], d[2]));
    if (!(x[2] > 0.0f)) return false;
    u = __fadd_rn(__fdiv_rn(__fmul_rn(K.fx, x[0]), x[2]), K.cx);
    v = __fadd_rn(__fdiv_rn(__fmul_rn(K.fy, x[1]), x[2]), K.cy);
    return true;
}

// threads 0..12*F-1 round the F poses to FP32
__device__ __forceinline__ void load_frames(EFrame* fr, const double* T, int F) {
    for (int k = threadIdx.x; k < 12 * F; k += blockDim.x) {
        const int i = k / 12, e = k % 12, r = e >> 2, c = e & 3;
        const float x = __double2float_rn(T[16 * i + 4 * r + c]);
        if (c < 3)
            fr[i].R[3 * r + c] = x;
        else
            fr[i].t[r] = x;
    }
}

// Sum 16 values over the warp: on return lane L holds the warp total of value L >> 1 (16 shuffles).
__device__ __forceinline__ float warp_reduce_scatter16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int level = 0; level < 4; ++level) {
        const int half = 8 >> level;  // values kept after this level
        const int bit = 16 >> level;  // lane bit that selects the half
        const bool upper = (lane & bit) != 0;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = upper ? v[j] : v[j + half];
            const float keep = upper ? v[j + half] : v[j];
            v[j] = keep + __shfl_xor_sync(kFull, send, bit);
        }
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

// Adds the block's per-thread pose terms acc[16] to a keyframe's FP64 accumulator.
__device__ __forceinline__ void block_add_terms(float (&acc)[16], double* out) {
    __shared__ double part[kEWarps][kSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float s = warp_reduce_scatter16(acc);
    if ((lane & 1) == 0) part[warp][lane >> 1] = (double)s;
    __syncthreads();
    if (threadIdx.x < kSlots) {
        double t = 0.0;
        for (int w = 0; w < kEWarps; ++w) t += part[w][threadIdx.x];
        if (t != 0.0) atomicAdd(out + threadIdx.x, t);
    }
}

// Adds the block's FP64 per-thread energies to *out.
__device__ __forceinline__ void block_add_energy(double x, double* out) {
    __shared__ double part[kEWarps];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kEWarps; ++w) s += part[w];
        if (s != 0.0) atomicAdd(out, s);
    }
}

// ------------------------------------------------------------------------------------------
// visibility
// ------------------------------------------------------------------------------------------

constexpr int kVisBatch = 8;  // keyframes whose depth gathers are issued together

__global__ void __launch_bounds__(kEThreads) visibility_kernel(EnergyArgs a, unsigned* nu) {
    __shared__ EFrame fr[kMaxFrames];
    load_frames(fr, a.T, a.F);
    __syncthreads();
    const float half = 0.5f * a.vs;
    const long long npx = (long long)a.K.width * a.K.height;
    for (long long j = (long long)blockIdx.x * kEThreads + threadIdx.x; j < a.n; j += (long long)gridDim.x * kEThreads) {
        SurfPt sp;
        const bool ok = surface_point32(a.m[3 * j], a.m[3 * j + 1], a.m[3 * j + 2], a.psi[j], a.g[3 * j],
                                        a.g[3 * j + 1], a.g[3 * j + 2], a.vs, sp) &&
                        fabsf(sp.s[0]) <= half && fabsf(sp.s[1]) <= half && fabsf(sp.s[2]) <= half;
        for (int w = 0; w < a.nw; ++w) {
            unsigned bits = 0u;
            const int i_end = a.F < 32 * (w + 1) ? a.F : 32 * (w + 1);
            for (int i0 = 32 * w; ok && i0 < i_end; i0 += kVisBatch) {
                long long at[kVisBatch];
                float z[kVisBatch], D[kVisBatch];
#pragma unroll
                for (int k = 0; k < kVisBatch; ++k) {
                    const int i = i0 + k;
                    at[k] = -1;
                    z[k] = 0.0f;
                    float d[3], x[3], u, v;
                    if (i < i_end && project32(sp, fr[i], a.K, d, x, u, v) && u >= 1.0f &&
                        u <= (float)(a.K.width - 2) && v >= 1.0f && v <= (float)(a.K.height - 2)) {
                        const int iu = (int)floorf(__fadd_rn(u, 0.5f)), iv = (int)floorf(__fadd_rn(v, 0.5f));
                        at[k] = (long long)i * npx + (long long)iv * a.K.width + iu;
                        z[k] = x[2];
                    }
                }
#pragma unroll
                for (int k = 0; k < kVisBatch; ++k) D[k] = at[k] >= 0 ? a.depth[at[k]] : 0.0f;
#pragma unroll
                for (int k = 0; k < kVisBatch; ++k)
                    if (at[k] >= 0 && depth_ok(D[k], a.K.depth_max) && fabsf(__fsub_rn(z[k], D[k])) <= a.vs)
                        bits |= 1u << (i0 + k - 32 * w);
            }
            nu[j * a.nw + w] = bits;
        }
    }
}

// ------------------------------------------------------------------------------------------
// per-keyframe lists of visible voxels
// ------------------------------------------------------------------------------------------

constexpr int kPairWords = 32;               // ballot words per block step
constexpr int kPairChunk = 32 * kPairWords;  // voxels per block step

__global__ void __launch_bounds__(kEThreads) pairs_kernel(EnergyArgs a) {
    __shared__ unsigned masks[kMaxFrames][kPairWords];  // ballot of keyframe i over word w
    __shared__ unsigned wofs[kMaxFrames][kPairWords];   // list offset of word w in keyframe i's list
    __shared__ unsigned long long fany;                  // keyframes seen anywhere in the step
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c0 = (long long)blockIdx.x * kPairChunk; c0 < a.n; c0 += (long long)gridDim.x * kPairChunk) {
        for (int k = threadIdx.x; k < a.F * kPairWords; k += kEThreads) masks[k / kPairWords][k % kPairWords] = 0u;
        if (threadIdx.x == 0) fany = 0ull;
        __syncthreads();
        for (int w = warp; w < kPairWords; w += kEWarps) {
            const long long j = c0 + 32 * w + lane;
            unsigned long long vb = 0ull;
            if (j < a.n)
                vb = a.nw == 1 ? (unsigned long long)a.nu[j]
                               : ((unsigned long long)a.nu[2 * j] | ((unsigned long long)a.nu[2 * j + 1] << 32));
            unsigned long long wb = __reduce_or_sync(kFull, (unsigned)vb);
            wb |= (unsigned long long)__reduce_or_sync(kFull, (unsigned)(vb >> 32)) << 32;
            if (wb != 0ull && lane == 0) atomicOr(&fany, wb);
            while (wb != 0ull) {  // warp-uniform
                const int i = __ffsll((long long)wb) - 1;
                wb &= wb - 1ull;
                const unsigned m = __ballot_sync(kFull, (vb >> i) & 1ull);
                if (lane == 0) masks[i][w] = m;
            }
        }
        __syncthreads();
        const unsigned long long fa = fany;
        for (int i = warp; i < a.F; i += kEWarps) {  // one warp per keyframe: scan, one reservation
            if (!((fa >> i) & 1ull)) continue;
            const unsigned c = __popc(masks[i][lane]);
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            unsigned base = 0u;
            if (lane == 31) base = atomicAdd(a.pair_count + i, incl);
            base = __shfl_sync(kFull, base, 31);
            wofs[i][lane] = base + incl - c;
        }
        __syncthreads();
        for (int w = warp; w < kPairWords; w += kEWarps) {
            const int j = (int)(c0 + 32 * w + lane);
            const unsigned lt = (1u << lane) - 1u;
            unsigned long long f = fa;
            while (f != 0ull) {
                const int i = __ffsll((long long)f) - 1;
                f &= f - 1ull;
                const unsigned m = masks[i][w];
                if ((m >> lane) & 1u) a.pairs[(long long)i * a.n + wofs[i][w] + __popc(m & lt)] = j;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// photometric term
// ------------------------------------------------------------------------------------------

template <bool kGrad>
__global__ void __launch_bounds__(kEThreads) photo_kernel(EnergyArgs a) {
    __shared__ EFrame fr[1];
    const int i = blockIdx.y;
    load_frames(fr, a.T + 16 * i, 1);
    __syncthreads();
    const float scale = (kGrad && a.grad_scale) ? (float)*a.grad_scale : 1.0f;
    const int W = a.K.width, H = a.K.height;
    const long long npx = (long long)W * H;
    const float4* rgb = a.rgb + (long long)i * npx;
    const int* list = a.pairs + (long long)i * a.n;
    const unsigned cnt = a.pair_count[i];
    float acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
    double e_tot = 0.0;
    for (unsigned k = blockIdx.x * kEThreads + threadIdx.x; k < cnt; k += gridDim.x * kEThreads) {
        const long long j = list[k];
        const float psi = a.psi[j];
        const float rho[3] = {a.rho[3 * j], a.rho[3 * j + 1], a.rho[3 * j + 2]};
        SurfPt sp;
        if (!surface_point32(a.m[3 * j], a.m[3 * j + 1], a.m[3 * j + 2], psi, a.g[3 * j], a.g[3 * j + 1],
                             a.g[3 * j + 2], a.vs, sp))
            continue;
        float d[3], x[3], u, v;
        if (!(project32(sp, fr[0], a.K, d, x, u, v) && u >= 0.0f && u <= (float)(W - 1) && v >= 0.0f &&
              v <= (float)(H - 1)))
            continue;
        int x0 = (int)floorf(u), y0 = (int)floorf(v);
        if (x0 > W - 2) x0 = W - 2;
        if (y0 > H - 2) y0 = H - 2;
        const float al = u - (float)x0, be = v - (float)y0;
        const float4* img = rgb + (long long)y0 * W + x0;
        const float4 I00 = img[0], I01 = img[1], I10 = img[W], I11 = img[W + 1];
        const float c00 = (1.0f - al) * (1.0f - be), c01 = al * (1.0f - be), c10 = (1.0f - al) * be, c11 = al * be;
        const float i00[3] = {I00.x, I00.y, I00.z}, i01[3] = {I01.x, I01.y, I01.z};
        const float i10[3] = {I10.x, I10.y, I10.z}, i11[3] = {I11.x, I11.y, I11.z};
        float e = 0.0f, dEdu = 0.0f, dEdv = 0.0f, r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float I = c00 * i00[c] + c01 * i01[c] + c10 * i10[c] + c11 * i11[c];
            r[c] = I - rho[c];
            e += r[c] * r[c];
            if (kGrad) {
                dEdu += 2.0f * r[c] * ((1.0f - be) * (i01[c] - i00[c]) + be * (i11[c] - i10[c]));
                dEdv += 2.0f * r[c] * ((1.0f - al) * (i10[c] - i00[c]) + al * (i11[c] - i01[c]));
            }
        }
        if (!kGrad) {
            e_tot += (double)e;
            continue;
        }
        // chain rule: (u, v) <- x (pinhole) <- p (x = R^T (p - t)) <- (psi, g) and the pose
        const float iz = 1.0f / x[2];
        const float dx[3] = {dEdu * a.K.fx * iz, dEdv * a.K.fy * iz, -(dEdu * a.K.fx * x[0] + dEdv * a.K.fy * x[1]) * iz * iz};
        const float* R = fr[0].R;
        float q[3];  // dE/dp = R dE/dx
#pragma unroll
        for (int r_ = 0; r_ < 3; ++r_) q[r_] = R[3 * r_] * dx[0] + R[3 * r_ + 1] * dx[1] + R[3 * r_ + 2] * dx[2];
        const float qg = q[0] * sp.gh[0] + q[1] * sp.gh[1] + q[2] * sp.gh[2];
        if (a.dpsi) {
            atomicAdd(a.dpsi + j, -scale * qg);  // dp/dpsi = -ghat
            const float c = -scale * psi / sp.nr;
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) {
                atomicAdd(a.dg + 3 * j + k2, c * (q[k2] - sp.gh[k2] * qg));  // dghat/dg
                atomicAdd(a.drho + 3 * j + k2, -2.0f * scale * r[k2]);
            }
        }
#pragma unroll
        for (int a_ = 0; a_ < 3; ++a_) {
#pragma unroll
            for (int b_ = 0; b_ < 3; ++b_) acc[3 * a_ + b_] += d[a_] * dx[b_];  // dE/dR_ab
            acc[9 + a_] -= q[a_];                                               // dE/dt
        }
        acc[kSlotEp] += e;
    }
    if (kGrad)
        block_add_terms(acc, a.acc + i * kSlots);
    else
        block_add_energy(e_tot, a.acc + i * kSlots + kSlotEp);
}

// ------------------------------------------------------------------------------------------
// geometric term
// ------------------------------------------------------------------------------------------

template <bool kGrad>
__global__ void __launch_bounds__(kEThreads) geo_kernel(EnergyArgs a) {
    __shared__ EFrame fr[1];
    const int i = blockIdx.y;
    load_frames(fr, a.T + 16 * i, 1);
    __syncthreads();
    const float scale = (kGrad && a.grad_scale) ? (float)*a.grad_scale : 1.0f;
    const float two_lambda = (float)(2.0 * a.lambda);
    const unsigned W = (unsigned)a.K.width;
    const unsigned npx = W * (unsigned)a.K.height;  // <= 2^30
    const float* depth = a.depth + (long long)i * npx;
    float acc[16];  // this thread's share of the keyframe's pose terms and E_g
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0f;
    double e_tot = 0.0;
    // pixel (u, v) of px, stepped by the grid stride without a division per pixel
    const unsigned stride = gridDim.x * kEThreads, sv = stride / W, su = stride - sv * W;
    unsigned px = blockIdx.x * kEThreads + threadIdx.x;
    int v = (int)(px / W), u = (int)(px - (unsigned)v * W);
    for (; px < npx; px += stride, u += (int)su, v += (int)sv) {
        if (u >= (int)W) {
            u -= (int)W;
            ++v;
        }
        const float D = depth[px];
        if (!depth_ok(D, a.K.depth_max)) continue;
        float dw[3], P[3];
        int mv[3];
        ray_world(a.K, fr[0].R, u, v, dw);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P[k] = ray_coord(D, dw[k], fr[0].t[k]);
            mv[k] = round_voxel(P[k], a.inv_vs);
        }
        const int j = index_find(a.tab, mv[0], mv[1], mv[2]);
        if (j < 0) continue;
        const float g0 = a.g[3 * j], g1 = a.g[3 * j + 1], g2 = a.g[3 * j + 2];
        if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
        const float psi = a.psi[j];
        const float n2 = g0 * g0 + g1 * g1 + g2 * g2;
        const float inr = n2 >= 1e-30f ? rsqrtf(n2) : 1.0f / norm3df(g0, g1, g2);  // no underflow for tiny g
        const float gh[3] = {g0 * inr, g1 * inr, g2 * inr};
        // P - v with v = v_s m split exactly into vh + vl, so d carries no rounding of v
        float dd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float mf = (float)mv[k];
            const float vh = __fmul_rn(a.vs, mf);
            const float vl = __fmaf_rn(a.vs, mf, -vh);
            dd[k] = __fsub_rn(__fsub_rn(P[k], vh), vl);
        }
        const float gd = gh[0] * dd[0] + gh[1] * dd[1] + gh[2] * dd[2];
        const float r = psi + gd;
        if (!kGrad) {
            e_tot += (double)(r * r);
            continue;
        }
        const float sr = two_lambda * r;
        if (a.geo_grads) {
            const float c = scale * sr * inr;
            atomicAdd(a.vacc + j, make_float4(scale * sr, c * (dd[0] - gh[0] * gd), c * (dd[1] - gh[1] * gd),
                                              c * (dd[2] - gh[2] * gd)));
        }
        float pc[3];  // camera point D ((u - c_x)/f_x, (v - c_y)/f_y, 1)
        backproject(a.K, u, v, D, pc);
#pragma unroll
        for (int a_ = 0; a_ < 3; ++a_) {
#pragma unroll
            for (int b_ = 0; b_ < 3; ++b_) acc[3 * a_ + b_] += sr * gh[a_] * pc[b_];
            acc[9 + a_] += sr * gh[a_];
        }
        acc[kSlotEg] += r * r;
    }
    if (kGrad)
        block_add_terms(acc, a.acc + i * kSlots);
    else
        block_add_energy(e_tot, a.acc + i * kSlots + kSlotEg);
}

// Every voxel's output gradient starts from its geometric part (zero unless geo_grads), and the
// accumulator is cleared for the next evaluation.  A warp covers 32 consecutive voxels; their
// (n, 3) rows of dE/dg and dE/drho are written as three coalesced 128-byte runs (staged through
// shared memory), so no store writes part of a sector.
__global__ void __launch_bounds__(kEThreads) merge_kernel(EnergyArgs a) {
    __shared__ float stage[kEWarps][96];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = (long long)blockIdx.x * kEThreads + warp * 32; base < a.n;
         base += (long long)gridDim.x * kEThreads) {
        const long long j = base + lane;
        const bool in = j < a.n;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (in && a.geo_grads) {
            v = a.vacc[j];
            // clear by adding -v (exact: x + (-x) = +0).  On GB300 a plain store right after a plain
            // load of a line that red atomics last modified costs about three times a red.
            if (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f)
                atomicAdd(a.vacc + j, make_float4(-v.x, -v.y, -v.z, -v.w));
        }
        if (in) a.dpsi[j] = v.x;
        stage[warp][3 * lane] = v.y;
        stage[warp][3 * lane + 1] = v.z;
        stage[warp][3 * lane + 2] = v.w;
        __syncwarp();
        const long long rows = a.n - base < 32 ? a.n - base : 32;  // voxels of this warp
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int e = 32 * k + lane;
            if (e < 3 * rows) {
                a.dg[3 * base + e] = stage[warp][e];
                a.drho[3 * base + e] = 0.0f;
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// photometric bundle adjustment (one Gauss-Newton iteration; see gsdf_energy_ba_step)
// ------------------------------------------------------------------------------------------

// Colour (and its image gradient, when dIdu != null) of the projection of voxel j's surface point
// into keyframe f, if the pair counts (FP32 index path of the decisions, as the energy).
__device__ __forceinline__ bool pair_colour(const EnergyArgs& a, const EFrame& f, const float4* rgb, long long j,
                                            SurfPt& sp, float d[3], float x[3], float I[3], float* dIdu,
                                            float* dIdv) {
    const int W = a.K.width, H = a.K.height;
    if (!surface_point32(a.m[3 * j], a.m[3 * j + 1], a.m[3 * j + 2], a.psi[j], a.g[3 * j], a.g[3 * j + 1],
                         a.g[3 * j + 2], a.vs, sp))
        return false;
    float u, v;
    if (!(project32(sp, f, a.K, d, x, u, v) && u >= 0.0f && u <= (float)(W - 1) && v >= 0.0f && v <= (float)(H - 1)))
        return false;
    int x0 = (int)floorf(u), y0 = (int)floorf(v);
    if (x0 > W - 2) x0 = W - 2;
    if (y0 > H - 2) y0 = H - 2;
    const float al = u - (float)x0, be = v - (float)y0;
    const float4* img = rgb + (long long)y0 * W + x0;
    const float4 I00 = img[0], I01 = img[1], I10 = img[W], I11 = img[W + 1];
    const float i00[3] = {I00.x, I00.y, I00.z}, i01[3] = {I01.x, I01.y, I01.z};
    const float i10[3] = {I10.x, I10.y, I10.z}, i11[3] = {I11.x, I11.y, I11.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        I[c] = (1.0f - al) * (1.0f - be) * i00[c] + al * (1.0f - be) * i01[c] + (1.0f - al) * be * i10[c] +
               al * be * i11[c];
        if (dIdu) {
            dIdu[c] = (1.0f - be) * (i01[c] - i00[c]) + be * (i11[c] - i10[c]);
            dIdv[c] = (1.0f - al) * (i10[c] - i00[c]) + al * (i11[c] - i01[c]);
        }
    }
    return true;
}

// Eq. (mean_color), pass 1: colour sums and counts of every voxel over the pairs that count.
__global__ void __launch_bounds__(kEThreads) colour_sum_kernel(EnergyArgs a) {
    __shared__ EFrame fr[1];
    const int i = blockIdx.y;
    load_frames(fr, a.T + 16 * i, 1);
    __syncthreads();
    const float4* rgb = a.rgb + (long long)i * a.K.width * a.K.height;
    const int* list = a.pairs + (long long)i * a.n;
    const unsigned cnt = a.pair_count[i];
    for (unsigned k = blockIdx.x * kEThreads + threadIdx.x; k < cnt; k += gridDim.x * kEThreads) {
        const long long j = list[k];
        SurfPt sp;
        float d[3], x[3], I[3];
        if (pair_colour(a, fr[0], rgb, j, sp, d, x, I, nullptr, nullptr))
            atomicAdd(a.cacc + j, make_float4(I[0], I[1], I[2], 1.0f));
    }
}

// Pass 2: rho = sums / count (0 for a voxel no pair counts); the sums are cleared by negated reds.
__global__ void __launch_bounds__(kEThreads) colour_mean_kernel(EnergyArgs a, float* rho) {
    for (long long j = (long long)blockIdx.x * kEThreads + threadIdx.x; j < a.n; j += (long long)gridDim.x * kEThreads) {
        const float4 s = a.cacc[j];
        const float inv = s.w > 0.0f ? 1.0f / s.w : 0.0f;
        rho[3 * j] = s.x * inv;
        rho[3 * j + 1] = s.y * inv;
        rho[3 * j + 2] = s.z * inv;
        if (s.w != 0.0f) atomicAdd(a.cacc + j, make_float4(-s.x, -s.y, -s.z, -s.w));
    }
}

// Adds J J^T (21 terms), J r (6), r^2 and one residual to the per-thread terms, weighted by w.
__device__ __forceinline__ void add_gn_terms(float (&acc)[32], const float J[6], float r, float w) {
    int q = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const float wJi = w * J[i];
#pragma unroll
        for (int k = i; k < 6; ++k) acc[q++] += wJi * J[k];
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] += w * J[i] * r;
    acc[27] += w * r * r;
    acc[28] += 1.0f;
}

// The keyframe's 29 Gauss-Newton terms of this block, added to its FP64 accumulator.
__device__ __forceinline__ void block_add_gn(float (&acc)[32], double* out) {
    __shared__ double part[kEWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    part[warp][lane] = (double)warp_reduce_scatter32(acc);
    __syncthreads();
    if (threadIdx.x < 29) {
        double t = 0.0;
        for (int w = 0; w < kEWarps; ++w) t += part[w][threadIdx.x];
        if (t != 0.0) atomicAdd(out + threadIdx.x, t);
    }
}

// Photometric Gauss-Newton terms with rho fixed (the decoupled energies of Eq. rgb_cost_pose):
// per pair and channel r = I - rho, J = (q x p, -q) with q = R dI/dx; per voxel (dr/dpsi)^2 and
// dr/dpsi r with dr/dpsi = -q . ghat, added to vacc.x, vacc.y.
__global__ void __launch_bounds__(kEThreads) ba_photo_kernel(EnergyArgs a) {
    __shared__ EFrame fr[1];
    const int i = blockIdx.y;
    load_frames(fr, a.T + 16 * i, 1);
    __syncthreads();
    const float4* rgb = a.rgb + (long long)i * a.K.width * a.K.height;
    const int* list = a.pairs + (long long)i * a.n;
    const unsigned cnt = a.pair_count[i];
    float acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
    for (unsigned k = blockIdx.x * kEThreads + threadIdx.x; k < cnt; k += gridDim.x * kEThreads) {
        const long long j = list[k];
        SurfPt sp;
        float d[3], x[3], I[3], du[3], dv[3];
        if (!pair_colour(a, fr[0], rgb, j, sp, d, x, I, du, dv)) continue;
        const float iz = 1.0f / x[2];
        const float* R = fr[0].R;
        float hp = 0.0f, bp = 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float r = I[c] - a.rho[3 * j + c];
            const float dx[3] = {du[c] * a.K.fx * iz, dv[c] * a.K.fy * iz,
                                 -(du[c] * a.K.fx * x[0] + dv[c] * a.K.fy * x[1]) * iz * iz};
            float q[3];
#pragma unroll
            for (int r_ = 0; r_ < 3; ++r_) q[r_] = R[3 * r_] * dx[0] + R[3 * r_ + 1] * dx[1] + R[3 * r_ + 2] * dx[2];
            const float J[6] = {q[1] * sp.p[2] - q[2] * sp.p[1], q[2] * sp.p[0] - q[0] * sp.p[2],
                                q[0] * sp.p[1] - q[1] * sp.p[0], -q[0], -q[1], -q[2]};
            add_gn_terms(acc, J, r, 1.0f);
            const float jp = -(q[0] * sp.gh[0] + q[1] * sp.gh[1] + q[2] * sp.gh[2]);
            hp += jp * jp;
            bp += jp * r;
        }
        atomicAdd(a.vacc + j, make_float4(hp, bp, 0.0f, 0.0f));
    }
    block_add_gn(acc, a.bacc + 32 * i);
}

// lambda times the tracking terms of every keyframe pixel (Eq. tracking with Eq. taylor); per
// voxel dr/dpsi = 1.
__global__ void __launch_bounds__(kEThreads) ba_geo_kernel(EnergyArgs a) {
    __shared__ EFrame fr[1];
    const int i = blockIdx.y;
    load_frames(fr, a.T + 16 * i, 1);
    __syncthreads();
    const float lam = (float)a.lambda;
    const unsigned W = (unsigned)a.K.width;
    const unsigned npx = W * (unsigned)a.K.height;
    const float* depth = a.depth + (long long)i * npx;
    float acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0f;
    for (unsigned px = blockIdx.x * kEThreads + threadIdx.x; px < npx; px += gridDim.x * kEThreads) {
        const float D = depth[px];
        if (!depth_ok(D, a.K.depth_max)) continue;
        const int v = (int)(px / W), u = (int)(px - (unsigned)v * W);
        float dw[3], P[3];
        int mv[3];
        ray_world(a.K, fr[0].R, u, v, dw);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            P[k] = ray_coord(D, dw[k], fr[0].t[k]);
            mv[k] = round_voxel(P[k], a.inv_vs);
        }
        const int j = index_find(a.tab, mv[0], mv[1], mv[2]);
        if (j < 0) continue;
        const float g0 = a.g[3 * j], g1 = a.g[3 * j + 1], g2 = a.g[3 * j + 2];
        if (g0 == 0.0f && g1 == 0.0f && g2 == 0.0f) continue;
        const float n2 = g0 * g0 + g1 * g1 + g2 * g2;
        const float inr = n2 >= 1e-30f ? rsqrtf(n2) : 1.0f / norm3df(g0, g1, g2);
        const float gh[3] = {g0 * inr, g1 * inr, g2 * inr};
        float dd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float mf = (float)mv[k];
            const float vh = __fmul_rn(a.vs, mf);
            const float vl = __fmaf_rn(a.vs, mf, -vh);
            dd[k] = __fsub_rn(__fsub_rn(P[k], vh), vl);
        }
        const float r = a.psi[j] + (gh[0] * dd[0] + gh[1] * dd[1] + gh[2] * dd[2]);
        const float J[6] = {P[1] * gh[2] - P[2] * gh[1], P[2] * gh[0] - P[0] * gh[2], P[0] * gh[1] - P[1] * gh[0],
                            gh[0], gh[1], gh[2]};
        add_gn_terms(acc, J, r, lam);
        atomicAdd(a.vacc + j, make_float4(lam, lam * r, 0.0f, 0.0f));
    }
    block_add_gn(acc, a.bacc + 32 * i);
}

// One warp per keyframe: damped FP64 solve of its 6x6 system, left update exp(xi^) T, statistics;
// clears the keyframe's accumulator and pair count for the next call.
__global__ void __launch_bounds__(32) ba_solve_kernel(double* bacc, unsigned int* pair_count, double* T,
                                                      double lam_scale, int update, gsdf_track_stats* stats) {
    __shared__ double tot[32], xi[6], dT[16], Ts[16];
    const int i = blockIdx.x, lane = threadIdx.x;
    tot[lane] = bacc[32 * i + lane];
    bacc[32 * i + lane] = 0.0;
    if (lane < 16) Ts[lane] = T[16 * i + lane];
    if (lane == 0) pair_count[i] = 0u;
    __syncwarp();
    const long long n_valid = (long long)(tot[28] + 0.5);
    bool ok = false;
    if (update) {
        const double tr = ((tot[0] + tot[6]) + (tot[11] + tot[15])) + (tot[18] + tot[20]);
        ok = solve6_warp(tot, tr, lam_scale, n_valid, xi);
        if (ok) {
            se3_exp_warp(xi, dT);
            const double tn = compose_entry(dT, Ts);
            if (lane < 12) T[16 * i + lane] = tn;
        }
    }
    if (stats) {
        gsdf_track_stats* s = stats + i;
        if (lane < 21)
            s->H[lane] = tot[lane];
        else if (lane < 27)
            s->b[lane - 21] = tot[lane];
        if (lane < 6) s->xi[lane] = ok ? xi[lane] : 0.0;
        if (lane == 0) {
            s->energy = tot[27];
            s->n_valid = n_valid;
            s->n_huber = 0;
            s->status = (!update || ok) ? (int)GSDF_OK : (int)GSDF_ERR_DEGENERATE;
            s->pad = 0;
        }
    }
}

// psi_j -= psi_b / ((1 + damping) psi_H) where psi_H > 0 (if update), and vacc cleared.
__global__ void __launch_bounds__(kEThreads) ba_psi_kernel(EnergyArgs a, float* psi, double damping, int update) {
    for (long long j = (long long)blockIdx.x * kEThreads + threadIdx.x; j < a.n; j += (long long)gridDim.x * kEThreads) {
        const float4 v = a.vacc[j];
        if (v.x == 0.0f && v.y == 0.0f) continue;
        if (update && v.x > 0.0f) psi[j] -= (float)((double)v.y / ((1.0 + damping) * (double)v.x));
        atomicAdd(a.vacc + j, make_float4(-v.x, -v.y, 0.0f, 0.0f));
    }
}

// ------------------------------------------------------------------------------------------
// finish: energies, pose gradients, accumulator reset
// ------------------------------------------------------------------------------------------

// One block of kMaxFrames * kSlots threads: thread (i, k) moves accumulator slot k of keyframe i
// to shared memory and clears it; thread i < F then forms keyframe i's outputs.
__global__ void __launch_bounds__(kMaxFrames * kSlots) finish_kernel(double* acc, unsigned int* pair_count, int F,
                                                                    double lambda, const double* T,
                                                                    const double* grad_scale, double* E, double* dT,
                                                                    double* dxi) {
    __shared__ double G[kMaxFrames][kSlots];
    __shared__ double Ts[kMaxFrames][12];
    const int t = threadIdx.x;
    if (t < F * kSlots) {
        G[t / kSlots][t % kSlots] = acc[t];
        acc[t] = 0.0;
    }
    if (t < F * 12) Ts[t / 12][t % 12] = T[16 * (t / 12) + t % 12];
    if (t < F) pair_count[t] = 0u;
    const double sc = grad_scale ? *grad_scale : 1.0;
    __syncthreads();
    const int i = t;
    if (i < F) {
        if (dT) {
            double* o = dT + 16 * i;
            for (int a_ = 0; a_ < 3; ++a_) {
                for (int b_ = 0; b_ < 3; ++b_) o[4 * a_ + b_] = sc * G[i][3 * a_ + b_];
                o[4 * a_ + 3] = sc * G[i][9 + a_];
            }
            for (int k = 12; k < 16; ++k) o[k] = 0.0;
        }
        if (dxi) {
            // exp(eps^) T: dR = [omega]x R, dt = [omega]x t + upsilon, so
            // dE/domega = sum_b R_{:,b} x G_{:,b} + t x dE/dt and dE/dupsilon = dE/dt
            double w[3] = {0.0, 0.0, 0.0};
            for (int b_ = 0; b_ < 4; ++b_) {
                const double c[3] = {Ts[i][b_], Ts[i][4 + b_], Ts[i][8 + b_]};  // column b of R, or t for b = 3
                const double gcol[3] = {b_ < 3 ? G[i][b_] : G[i][9], b_ < 3 ? G[i][3 + b_] : G[i][10],
                                        b_ < 3 ? G[i][6 + b_] : G[i][11]};
                w[0] += c[1] * gcol[2] - c[2] * gcol[1];
                w[1] += c[2] * gcol[0] - c[0] * gcol[2];
                w[2] += c[0] * gcol[1] - c[1] * gcol[0];
            }
            double* o = dxi + 6 * i;
            for (int k = 0; k < 3; ++k) {
                o[k] = sc * w[k];
                o[3 + k] = sc * G[i][9 + k];
            }
        }
    }
    if (t == 0) {
        double sp = 0.0, sg = 0.0;
        for (int k = 0; k < F; ++k) {
            sp += G[k][kSlotEp];
            sg += G[k][kSlotEg];
        }
        E[0] = sp + lambda * sg;
        E[1] = sp;
        E[2] = sg;
    }
}

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

gsdf_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return GSDF_OK;
    if (e == cudaErrorMemoryAllocation) return GSDF_ERR_OOM;
    return GSDF_ERR_CUDA;
}

}  // namespace

struct gsdf_energy {
    int device = 0, num_sms = 0;
    cudaStream_t stream = nullptr;
    long long n = 0;
    int F = 0;
    Intr K{};
    float vs = 0.0f, inv_vs = 0.0f;
    int* m = nullptr;
    IndexTable tab{};
    float4* rgb = nullptr;
    float* depth = nullptr;
    float4* vacc = nullptr;  // n
    float4* cacc = nullptr;  // n: colour sums (bundle adjustment)
    double* bacc = nullptr;  // kMaxFrames x 32: Gauss-Newton terms (bundle adjustment)
    int* pairs = nullptr;    // F x n
    unsigned int* pair_count = nullptr;
    double* acc = nullptr;
    int* err = nullptr;
    int vis_blocks = 0, pairs_blocks = 0, merge_blocks = 0;
    long long n_blocks = 0;  // 8^3 blocks holding the list's voxels
    int photo_blocks[2] = {0, 0};  // resident grid of photo_kernel<false>, <true>
    int geo_blocks[2] = {0, 0};
    int ba_photo_blocks = 0, ba_geo_blocks = 0;
};

namespace {

void free_energy(gsdf_energy* e) {
    cudaFree(e->m);
    cudaFree(e->tab.slots);
    cudaFree(e->tab.vox);
    cudaFree(e->vacc);
    cudaFree(e->cacc);
    cudaFree(e->bacc);
    cudaFree(e->pairs);
    cudaFree(e->pair_count);
    cudaFree(e->rgb);
    cudaFree(e->depth);
    cudaFree(e->acc);
    cudaFree(e->err);
    delete e;
}

EnergyArgs make_args(const gsdf_energy* e) {
    EnergyArgs a{};
    a.n = e->n;
    a.F = e->F;
    a.nw = (e->F + 31) / 32;
    a.K = e->K;
    a.vs = e->vs;
    a.inv_vs = e->inv_vs;
    a.m = e->m;
    a.rgb = e->rgb;
    a.depth = e->depth;
    a.tab = e->tab;
    a.acc = e->acc;
    a.vacc = e->vacc;
    a.cacc = e->cacc;
    a.bacc = e->bacc;
    a.pairs = e->pairs;
    a.pair_count = e->pair_count;
    return a;
}

int grid_for(long long work, int resident) {
    const long long need = (work + kEThreads - 1) / kEThreads;
    return (int)(need < resident ? (need > 0 ? need : 1) : resident);
}

// columns of a (columns x F) grid that keeps `resident` blocks busy, at most `need` columns
int columns_for(int resident, int F, long long need) {
    long long gx = (resident + F - 1) / F;
    if (gx > need) gx = need;
    return (int)(gx < 1 ? 1 : gx);
}

template <typename Kern>
cudaError_t resident(Kern k, int num_sms, int* out) {
    int occ = 0;
    cudaError_t ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kEThreads, 0);
    *out = (occ > 0 ? occ : 1) * num_sms;
    return ce;
}

}  // namespace

extern "C" {

gsdf_status gsdf_energy_create(int64_t n_voxels, const int32_t* m_dev, float voxel_size, int32_t n_frames,
                               const gsdf_intrinsics* K, const float* rgb_dev, const float* depth_dev, void* cuda_stream,
                               gsdf_energy** out) {
    if (!out) return GSDF_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_voxels < 0 || n_voxels > 0x7fffffffll || (n_voxels > 0 && !m_dev)) return GSDF_ERR_INVALID_ARG;
    if (n_frames < 1 || n_frames > kMaxFrames || !rgb_dev || !depth_dev || !K) return GSDF_ERR_INVALID_ARG;
    if (!finite_pos(voxel_size) || !finite_pos(K->fx) || !finite_pos(K->fy) || !isfinite(K->cx) ||
        !isfinite(K->cy) || !finite_pos(K->depth_max))
        return GSDF_ERR_INVALID_ARG;
    if (K->width < 2 || K->height < 2 || K->width > 32768 || K->height > 32768) return GSDF_ERR_INVALID_ARG;
    gsdf_energy* e = new (std::nothrow) gsdf_energy();
    if (!e) return GSDF_ERR_OOM;
    e->stream = (cudaStream_t)cuda_stream;
    e->n = n_voxels;
    e->F = n_frames;
    e->K.fx = K->fx;
    e->K.fy = K->fy;
    e->K.cx = K->cx;
    e->K.cy = K->cy;
    e->K.width = K->width;
    e->K.height = K->height;
    e->K.depth_max = K->depth_max;
    e->K.ifx = (float)(1.0 / (double)K->fx);
    e->K.ify = (float)(1.0 / (double)K->fy);
    e->vs = voxel_size;
    e->inv_vs = (float)(1.0 / (double)voxel_size);
    const size_t nv = (size_t)(n_voxels > 0 ? n_voxels : 1);
    const long long npx = (long long)K->width * K->height * n_frames;
    cudaError_t ce = cudaGetDevice(&e->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->m, sizeof(int) * 3 * nv);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->vacc, sizeof(float4) * nv);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->cacc, sizeof(float4) * nv);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->bacc, sizeof(double) * 32 * kMaxFrames);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->pairs, sizeof(int) * nv * (size_t)n_frames);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->pair_count, sizeof(unsigned int) * kMaxFrames);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->rgb, sizeof(float4) * (size_t)npx);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->depth, sizeof(float) * (size_t)npx);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->acc, sizeof(double) * kSlots * kMaxFrames);
    if (ce == cudaSuccess) ce = cudaMalloc(&e->err, sizeof(int));
    if (ce == cudaSuccess) ce = resident(visibility_kernel, e->num_sms, &e->vis_blocks);
    if (ce == cudaSuccess) ce = resident(pairs_kernel, e->num_sms, &e->pairs_blocks);
    if (ce == cudaSuccess) ce = resident(merge_kernel, e->num_sms, &e->merge_blocks);
    if (ce == cudaSuccess) ce = resident(photo_kernel<false>, e->num_sms, &e->photo_blocks[0]);
    if (ce == cudaSuccess) ce = resident(photo_kernel<true>, e->num_sms, &e->photo_blocks[1]);
    if (ce == cudaSuccess) ce = resident(geo_kernel<false>, e->num_sms, &e->geo_blocks[0]);
    if (ce == cudaSuccess) ce = resident(geo_kernel<true>, e->num_sms, &e->geo_blocks[1]);
    if (ce == cudaSuccess) ce = resident(ba_photo_kernel, e->num_sms, &e->ba_photo_blocks);
    if (ce == cudaSuccess) ce = resident(ba_geo_kernel, e->num_sms, &e->ba_geo_blocks);
    cudaStream_t st = e->stream;
    if (n_voxels > 0 && ce == cudaSuccess)
        ce = cudaMemcpyAsync(e->m, m_dev, sizeof(int) * 3 * (size_t)n_voxels, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->vacc, 0, sizeof(float4) * nv, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->cacc, 0, sizeof(float4) * nv, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->bacc, 0, sizeof(double) * 32 * kMaxFrames, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->acc, 0, sizeof(double) * kSlots * kMaxFrames, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->pair_count, 0, sizeof(unsigned int) * kMaxFrames, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->err, 0, sizeof(int), st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(e->depth, depth_dev, sizeof(float) * (size_t)npx, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess) {
        pack_rgb_kernel<<<grid_for(npx, 8 * e->num_sms), kEThreads, 0, st>>>(rgb_dev, e->rgb, npx);
        ce = cudaGetLastError();
    }
    // voxel index: (1) block keys into a table sized for n keys, counting blocks; (2) per-block
    // voxel arrays and a compact block table of twice the block count
    IndexSlot* big = nullptr;
    unsigned long long big_slots = 1024;
    while (big_slots < 2ull * (unsigned long long)nv) big_slots <<= 1;
    unsigned int* count = nullptr;
    if (ce == cudaSuccess) ce = cudaMalloc(&big, sizeof(IndexSlot) * big_slots);
    if (ce == cudaSuccess) ce = cudaMalloc(&count, sizeof(unsigned int));
    if (ce == cudaSuccess) ce = cudaMemsetAsync(big, 0xff, sizeof(IndexSlot) * big_slots, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
    if (ce == cudaSuccess && n_voxels > 0) {
        index_blocks_kernel<<<grid_for(n_voxels, 4 * e->num_sms), kEThreads, 0, st>>>(big, big_slots - 1, e->m,
                                                                                      n_voxels, count, e->err);
        ce = cudaGetLastError();
    }
    unsigned int nb = 0;
    int err = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&nb, count, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&err, e->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce == cudaSuccess && err == 0) {
        e->n_blocks = nb;
        unsigned long long slots = 1024;
        while (slots < 2ull * nb) slots <<= 1;
        e->tab.mask = slots - 1;
        ce = cudaMalloc(&e->tab.slots, sizeof(IndexSlot) * slots);
        if (ce == cudaSuccess) ce = cudaMalloc(&e->tab.vox, sizeof(int) * kBlockVoxels * (size_t)(nb > 0 ? nb : 1));
        if (ce == cudaSuccess) ce = cudaMemsetAsync(e->tab.slots, 0xff, sizeof(IndexSlot) * slots, st);
        if (ce == cudaSuccess)
            ce = cudaMemsetAsync(e->tab.vox, 0xff, sizeof(int) * kBlockVoxels * (size_t)(nb > 0 ? nb : 1), st);
        if (ce == cudaSuccess && n_voxels > 0) {
            index_fill_kernel<<<grid_for(n_voxels, 4 * e->num_sms), kEThreads, 0, st>>>(big, big_slots - 1, e->tab,
                                                                                        e->m, n_voxels, e->err);
            index_compact_kernel<<<grid_for((long long)big_slots, 4 * e->num_sms), kEThreads, 0, st>>>(
                big, big_slots - 1, e->tab, e->err);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&err, e->err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    }
    cudaFree(big);
    cudaFree(count);
    if (ce != cudaSuccess || err != 0) {
        gsdf_status s = ce != cudaSuccess ? from_cuda(ce) : (gsdf_status)err;
        cudaGetLastError();
        free_energy(e);
        return s;
    }
    *out = e;
    return GSDF_OK;
}

gsdf_status gsdf_energy_destroy(gsdf_energy* e) {
    if (!e) return GSDF_ERR_INVALID_ARG;
    cudaError_t ce = cudaStreamSynchronize(e->stream);
    free_energy(e);
    return from_cuda(ce);
}

gsdf_status gsdf_energy_set_stream(gsdf_energy* e, void* cuda_stream) {
    if (!e) return GSDF_ERR_INVALID_ARG;
    e->stream = (cudaStream_t)cuda_stream;
    return GSDF_OK;
}

gsdf_status gsdf_energy_visibility(gsdf_energy* e, const float* psi_dev, const float* g_dev, const double* T_dev,
                                   uint32_t* nu_dev) {
    if (!e || !T_dev || (e->n > 0 && (!psi_dev || !g_dev || !nu_dev))) return GSDF_ERR_INVALID_ARG;
    if (e->n == 0) return GSDF_OK;
    EnergyArgs a = make_args(e);
    a.psi = psi_dev;
    a.g = g_dev;
    a.T = T_dev;
    visibility_kernel<<<grid_for(e->n, e->vis_blocks), kEThreads, 0, e->stream>>>(a, (unsigned*)nu_dev);
    return from_cuda(cudaGetLastError());
}

gsdf_status gsdf_energy_eval(gsdf_energy* e, const float* psi_dev, const float* g_dev, const float* rho_dev,
                             const double* T_dev, const uint32_t* nu_dev, double lambda_geo,
                             const double* grad_scale_dev, double* E_dev, float* dpsi_dev, float* dg_dev,
                             float* drho_dev, double* dT_dev, double* dxi_dev) {
    if (!e || !T_dev || !E_dev || !isfinite(lambda_geo)) return GSDF_ERR_INVALID_ARG;
    if (e->n > 0 && (!psi_dev || !g_dev || !rho_dev || !nu_dev)) return GSDF_ERR_INVALID_ARG;
    const bool voxel_grads = dpsi_dev != nullptr;
    if (voxel_grads != (dg_dev != nullptr) || voxel_grads != (drho_dev != nullptr)) return GSDF_ERR_INVALID_ARG;
    const bool grad = voxel_grads || dT_dev || dxi_dev;
    EnergyArgs a = make_args(e);
    a.psi = psi_dev;
    a.g = g_dev;
    a.rho = rho_dev;
    a.T = T_dev;
    a.nu = (const unsigned*)nu_dev;
    a.lambda = lambda_geo;
    a.grad_scale = grad_scale_dev;
    a.dpsi = dpsi_dev;
    a.dg = dg_dev;
    a.drho = drho_dev;
    cudaStream_t st = e->stream;
    const long long npx = (long long)e->K.width * e->K.height;
    cudaError_t ce = cudaSuccess;
    a.geo_grads = voxel_grads && lambda_geo != 0.0 && e->n > 0;
    if (lambda_geo != 0.0) {  // at lambda = 0 the geometric term is not evaluated and E_g = 0
        const long long need = (npx + kEThreads - 1) / kEThreads;
        const dim3 grid(columns_for(e->geo_blocks[grad ? 1 : 0], e->F, need), e->F);
        if (grad)
            geo_kernel<true><<<grid, kEThreads, 0, st>>>(a);
        else
            geo_kernel<false><<<grid, kEThreads, 0, st>>>(a);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return from_cuda(ce);
    }
    if (e->n > 0) {
        if (voxel_grads) merge_kernel<<<grid_for(e->n, e->merge_blocks), kEThreads, 0, st>>>(a);
        const long long chunks = (e->n + kPairChunk - 1) / kPairChunk;
        pairs_kernel<<<(int)(chunks < e->pairs_blocks ? chunks : e->pairs_blocks), kEThreads, 0, st>>>(a);
        const long long need = (e->n + kEThreads - 1) / kEThreads;
        const dim3 grid(columns_for(e->photo_blocks[grad ? 1 : 0], e->F, need), e->F);
        if (grad)
            photo_kernel<true><<<grid, kEThreads, 0, st>>>(a);
        else
            photo_kernel<false><<<grid, kEThreads, 0, st>>>(a);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return from_cuda(ce);
    }
    finish_kernel<<<1, kMaxFrames * kSlots, 0, st>>>(e->acc, e->pair_count, e->F, lambda_geo, T_dev, grad_scale_dev, E_dev,
                                            dT_dev, dxi_dev);
    return from_cuda(cudaGetLastError());
}

gsdf_status gsdf_energy_ba_step(gsdf_energy* e, float* psi_dev, const float* g_dev, float* rho_dev, double* T_dev,
                                const uint32_t* nu_dev, double lambda_geo, double damping, int32_t flags,
                                gsdf_track_stats* stats_dev) {
    if (!e || !T_dev || !isfinite(lambda_geo) || !isfinite(damping) || damping < 0.0 || (flags & ~3)) return GSDF_ERR_INVALID_ARG;
    if (e->n > 0 && (!psi_dev || !g_dev || !rho_dev || !nu_dev)) return GSDF_ERR_INVALID_ARG;
    EnergyArgs a = make_args(e);
    a.psi = psi_dev;
    a.g = g_dev;
    a.rho = rho_dev;
    a.T = T_dev;
    a.nu = (const unsigned*)nu_dev;
    a.lambda = lambda_geo;
    cudaStream_t st = e->stream;
    const long long npx = (long long)e->K.width * e->K.height;
    const long long need = (e->n + kEThreads - 1) / kEThreads;
    if (e->n > 0) {
        const long long chunks = (e->n + kPairChunk - 1) / kPairChunk;
        pairs_kernel<<<(int)(chunks < e->pairs_blocks ? chunks : e->pairs_blocks), kEThreads, 0, st>>>(a);
        const dim3 pgrid(columns_for(e->ba_photo_blocks, e->F, need), e->F);
        colour_sum_kernel<<<pgrid, kEThreads, 0, st>>>(a);
        colour_mean_kernel<<<grid_for(e->n, e->vis_blocks), kEThreads, 0, st>>>(a, rho_dev);
        ba_photo_kernel<<<pgrid, kEThreads, 0, st>>>(a);
    }
    if (lambda_geo != 0.0) {
        const long long pneed = (npx + kEThreads - 1) / kEThreads;
        ba_geo_kernel<<<dim3(columns_for(e->ba_geo_blocks, e->F, pneed), e->F), kEThreads, 0, st>>>(a);
    }
    ba_solve_kernel<<<e->F, 32, 0, st>>>(e->bacc, e->pair_count, T_dev, damping / 6.0, (flags & GSDF_BA_POSES) ? 1 : 0,
                                         stats_dev);
    if (e->n > 0)
        ba_psi_kernel<<<grid_for(e->n, e->vis_blocks), kEThreads, 0, st>>>(a, psi_dev, damping,
                                                                             (flags & GSDF_BA_PSI) ? 1 : 0);
    return from_cuda(cudaGetLastError());
}

}  // extern "C"
