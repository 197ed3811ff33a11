// Extraction of every voxel with W > 0 in a canonical order, the oriented point cloud of Sec. 4.3
// (and its 2x2x2 Taylor upsampling) and the marching-cubes mesh in the same order, and checkpoint
// loading.
//
// Hashed maps: the occupied slots' block keys are collected, sorted (a bitonic network whose steps
// within 4096-key chunks run in shared memory; keys are unique, so the order is total), counted,
// prefix-summed, and each block's voxels with W > 0 are written in local-index order.  Dense maps are processed as chunks of
// 512 consecutive linear voxels.  Output order therefore never depends on insertion order.
#include "gsdf_internal.cuh"

namespace gsdf {

__global__ void collect_keys_kernel(const unsigned long long* __restrict__ keys, long long n_slots,
                                    unsigned long long* out, unsigned int* count) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n_slots;
         s += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[s];
        if (k != kEmptyKey) out[atomicAdd(count, 1u)] = k;
    }
}

__global__ void bitonic_step_kernel(unsigned long long* a, long long n, long long j, long long k) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long l = i ^ j;
        if (l <= i) continue;
        const unsigned long long x = a[i], y = a[l];
        const bool up = (i & k) == 0;
        if ((x > y) == up) {
            a[i] = y;
            a[l] = x;
        }
    }
}

// The same bitonic network, its steps with j < kSortChunk run in shared memory: chunks of
// kSortChunk consecutive elements are independent for those steps.  Each pair (i, i ^ j) is ordered
// ascending when (i & k) == 0, descending otherwise, with i the element's global index.
constexpr int kSortChunk = 4096;
constexpr int kSortThreads = 1024;

__device__ __forceinline__ void sort_pairs_shared(unsigned long long* c, long long base, long long k, long long j) {
    for (int t = threadIdx.x; t < kSortChunk / 2; t += blockDim.x) {
        const int lo = ((t & ~(int)(j - 1)) << 1) | (t & (int)(j - 1));
        const int hi = lo | (int)j;
        const unsigned long long x = c[lo], y = c[hi];
        const bool up = ((base + lo) & k) == 0;
        if ((x > y) == up) {
            c[lo] = y;
            c[hi] = x;
        }
    }
}

// Every chunk through all stages k = 2 .. kSortChunk (N a multiple of kSortChunk).
__global__ void __launch_bounds__(kSortThreads) bitonic_chunks_kernel(unsigned long long* a) {
    __shared__ unsigned long long c[kSortChunk];
    const long long base = (long long)blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) c[i] = a[base + i];
    __syncthreads();
    for (long long k = 2; k <= kSortChunk; k <<= 1)
        for (long long j = k >> 1; j > 0; j >>= 1) {
            sort_pairs_shared(c, base, k, j);
            __syncthreads();
        }
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) a[base + i] = c[i];
}

// Stage k > kSortChunk, its steps j = kSortChunk / 2 .. 1, for every chunk.
__global__ void __launch_bounds__(kSortThreads) bitonic_merge_chunks_kernel(unsigned long long* a, long long k) {
    __shared__ unsigned long long c[kSortChunk];
    const long long base = (long long)blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) c[i] = a[base + i];
    __syncthreads();
    for (long long j = kSortChunk / 2; j > 0; j >>= 1) {
        sort_pairs_shared(c, base, k, j);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) a[base + i] = c[i];
}

// Per chunk (hashed: sorted block i; dense: linear chunk i) the voxel base index and the number
// of voxels with W > 0.
__global__ void chunk_count_kernel(HashMap hm, const unsigned long long* __restrict__ sorted,
                                   long long n_chunks, long long dense_voxels, const float* __restrict__ W,
                                   long long* base, unsigned int* counts) {
    __shared__ unsigned int cnt;
    __shared__ long long b0;
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        if (threadIdx.x == 0) {
            cnt = 0;
            if (sorted) {
                int b[3];
                unpack_block(sorted[c], b);
                b0 = hm.find(b[0] * 8, b[1] * 8, b[2] * 8);  // local 0 of the block
            } else {
                b0 = c * kBlockVoxels;
            }
            base[c] = b0;
        }
        __syncthreads();
        const long long i = b0 + threadIdx.x;
        const bool in = (sorted != nullptr) || (i < dense_voxels);
        const bool occ = b0 >= 0 && in && W[i] > 0.0f;
        const unsigned int wc = __popc(__ballot_sync(0xffffffffu, occ));
        if ((threadIdx.x & 31) == 0 && wc) atomicAdd(&cnt, wc);
        __syncthreads();
        if (threadIdx.x == 0) counts[c] = cnt;
        __syncthreads();
    }
}

// Exclusive scan of counts into offsets by one block; offsets[n] = total.
__global__ void scan_kernel(const unsigned int* __restrict__ counts, long long n, long long* offsets) {
    __shared__ long long part[1024];
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long lo = threadIdx.x * per;
    const long long hi = lo + per < n ? lo + per : n;
    long long s = 0;
    for (long long i = lo; i < hi; ++i) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const long long x = part[t];
            part[t] = run;
            run += x;
        }
        offsets[n] = run;
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (long long i = lo; i < hi; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
}

__global__ void chunk_write_kernel(const unsigned long long* __restrict__ sorted, long long n_chunks,
                                   const long long* __restrict__ base, const long long* __restrict__ offsets,
                                   const float4* __restrict__ A, const float* __restrict__ W,
                                   long long dense_voxels, int dx, int dy, int ox, int oy, int oz,
                                   const ushort4* __restrict__ H16, const float* __restrict__ scale16,
                                   gsdf_voxel* out) {
    __shared__ unsigned int warp_off[kBlockVoxels / 32];
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const long long b0 = base[c];
        const long long i = b0 + threadIdx.x;
        const bool in = (sorted != nullptr) || (i < dense_voxels);
        const bool occ = b0 >= 0 && in && W[i] > 0.0f;
        const unsigned int bal = __ballot_sync(0xffffffffu, occ);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0) warp_off[warp] = __popc(bal);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned int run = 0;
            for (int w = 0; w < kBlockVoxels / 32; ++w) {
                const unsigned int x = warp_off[w];
                warp_off[w] = run;
                run += x;
            }
        }
        __syncthreads();
        if (occ) {
            const long long pos = offsets[c] + warp_off[warp] + __popc(bal & ((1u << lane) - 1u));
            gsdf_voxel o;
            if (sorted) {
                int b[3];
                unpack_block(sorted[c], b);
                o.m[0] = b[0] * 8 + (threadIdx.x & 7);
                o.m[1] = b[1] * 8 + ((threadIdx.x >> 3) & 7);
                o.m[2] = b[2] * 8 + (threadIdx.x >> 6);
            } else {
                const long long x = i % dx, y = (i / dx) % dy, z = i / ((long long)dx * dy);
                o.m[0] = ox + (int)x;
                o.m[1] = oy + (int)y;
                o.m[2] = oz + (int)z;
            }
            const float w = W[i];
            if (H16) {  // FP16 payload: psi = sigma_b * psi~, g = W * gbar
                const ushort4 h = H16[i];
                o.psi = __half2float(__ushort_as_half(h.x)) * scale16[i >> 9];
                o.g[0] = __half2float(__ushort_as_half(h.y)) * w;
                o.g[1] = __half2float(__ushort_as_half(h.z)) * w;
                o.g[2] = __half2float(__ushort_as_half(h.w)) * w;
            } else {
                const float4 a = A[i];
                o.psi = a.x / w;
                o.g[0] = a.y;
                o.g[1] = a.z;
                o.g[2] = a.w;
            }
            o.w = w;
            out[pos] = o;
        }
        __syncthreads();
    }
}

// Checkpoint restore: psi, g, W of each voxel written (not added) into the map.
__global__ void load_kernel_hashed(HashMap hm, const gsdf_voxel* __restrict__ in, long long n,
                                   int* err, unsigned int* n_new) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const gsdf_voxel v = in[i];
        const long long idx = hm.find_or_insert(v.m[0], v.m[1], v.m[2], err, n_new);
        if (idx < 0) continue;
        hm.A[idx] = make_float4(v.w * v.psi, v.g[0], v.g[1], v.g[2]);
        hm.W[idx] = v.w;
    }
}

// FP16 maps: blocks receive the scale sigma_b = T, voxels (psi / T, g / W) rounded to nearest
__global__ void load_kernel_hashed16(HashMap16 hm, const gsdf_voxel* __restrict__ in, long long n, float trunc,
                                     int* err, unsigned int* n_new) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const gsdf_voxel v = in[i];
        const long long idx = hm.base.find_or_insert(v.m[0], v.m[1], v.m[2], err, n_new);
        if (idx < 0) continue;
        ushort4 o;
        o.x = __half_as_ushort(__float2half_rn(v.psi / trunc));
        o.y = __half_as_ushort(__float2half_rn(v.g[0] / v.w));
        o.z = __half_as_ushort(__float2half_rn(v.g[1] / v.w));
        o.w = __half_as_ushort(__float2half_rn(v.g[2] / v.w));
        hm.H[idx] = o;
        hm.W[idx] = v.w;
        hm.scale[idx >> 9] = trunc;
    }
}

__global__ void load_kernel_dense(DenseMap dm, const gsdf_voxel* __restrict__ in, long long n, int* err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const gsdf_voxel v = in[i];
        const long long idx = dm.find(v.m[0], v.m[1], v.m[2]);
        if (idx < 0) {
            atomicCAS(err, kErrNone, (int)GSDF_ERR_INVALID_ARG);
            continue;
        }
        dm.A[idx] = make_float4(v.w * v.psi, v.g[0], v.g[1], v.g[2]);
        dm.W[idx] = v.w;
    }
}

// ------------------------------------------------------------------------------------------

static long long next_pow2(long long n) {
    long long p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Device buffer freed when it goes out of scope.
template <class T>
struct DevBuf {
    T* p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * (n > 0 ? n : 1)); }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

#define GSDF_CK(x)                            \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) return e_;     \
    } while (0)

// The occupied slots' block keys, sorted ascending into keys (a power-of-two buffer padded with
// the empty key); *n_keys receives their number.  Synchronises the stream.
static cudaError_t sorted_block_keys(const HashMap& hm, long long n_slots, cudaStream_t st, unsigned grid,
                                     DevBuf<unsigned long long>& keys, long long* n_keys_out) {
    DevBuf<unsigned int> cnt;
    DevBuf<unsigned long long> tmp;
    GSDF_CK(cnt.alloc(1));
    GSDF_CK(tmp.alloc((size_t)n_slots));
    GSDF_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int), st));
    collect_keys_kernel<<<grid, 256, 0, st>>>(hm.keys, n_slots, tmp.p, cnt.p);
    GSDF_CK(cudaGetLastError());
    unsigned int n_keys = 0;
    GSDF_CK(cudaMemcpyAsync(&n_keys, cnt.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
    GSDF_CK(cudaStreamSynchronize(st));
    // padded to a power of two no smaller than one shared-memory chunk
    const long long N = next_pow2(n_keys > kSortChunk ? n_keys : kSortChunk);
    GSDF_CK(keys.alloc((size_t)N));
    GSDF_CK(cudaMemsetAsync(keys.p, 0xFF, sizeof(unsigned long long) * (size_t)N, st));
    if (n_keys)
        GSDF_CK(cudaMemcpyAsync(keys.p, tmp.p, sizeof(unsigned long long) * n_keys, cudaMemcpyDeviceToDevice, st));
    // stages up to one chunk in shared memory; each larger stage: its steps j >= kSortChunk in
    // global memory, the rest in shared memory
    const unsigned chunks = (unsigned)(N / kSortChunk);
    bitonic_chunks_kernel<<<chunks, kSortThreads, 0, st>>>(keys.p);
    GSDF_CK(cudaGetLastError());
    for (long long k = 2 * (long long)kSortChunk; k <= N; k <<= 1) {
        for (long long j = k >> 1; j >= kSortChunk; j >>= 1) {
            bitonic_step_kernel<<<grid, 256, 0, st>>>(keys.p, N, j, k);
            GSDF_CK(cudaGetLastError());
        }
        bitonic_merge_chunks_kernel<<<chunks, kSortThreads, 0, st>>>(keys.p, k);
        GSDF_CK(cudaGetLastError());
    }
    GSDF_CK(cudaStreamSynchronize(st));
    *n_keys_out = n_keys;
    return cudaSuccess;
}

cudaError_t extract_voxels(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                           cudaStream_t st, int num_sms, gsdf_voxel** out_dev, long long* n_out) {
    *out_dev = nullptr;
    *n_out = 0;
    const unsigned grid = (unsigned)(num_sms * 8);
    DevBuf<unsigned long long> keys;
    long long n_chunks = 0, dense_voxels = 0;
    if (hm) {
        GSDF_CK(sorted_block_keys(*hm, n_slots, st, grid, keys, &n_chunks));
    } else {
        dense_voxels = (long long)dm->dims[0] * dm->dims[1] * dm->dims[2];
        n_chunks = (dense_voxels + kBlockVoxels - 1) / kBlockVoxels;
    }
    if (n_chunks == 0) return cudaSuccess;
    DevBuf<long long> base, offsets;
    DevBuf<unsigned int> counts;
    GSDF_CK(base.alloc((size_t)n_chunks));
    GSDF_CK(counts.alloc((size_t)n_chunks));
    GSDF_CK(offsets.alloc((size_t)n_chunks + 1));
    const HashMap hmv = hm ? *hm : HashMap{};
    const float* W = h16 ? h16->W : (hm ? hm->W : dm->W);
    const float4* A = hm ? hm->A : dm->A;
    const unsigned long long* sorted = hm ? keys.p : nullptr;
    const unsigned cgrid = (unsigned)(n_chunks < (long long)num_sms * 16 ? n_chunks : (long long)num_sms * 16);
    chunk_count_kernel<<<cgrid, kBlockVoxels, 0, st>>>(hmv, sorted, n_chunks, dense_voxels, W, base.p, counts.p);
    GSDF_CK(cudaGetLastError());
    scan_kernel<<<1, 1024, 0, st>>>(counts.p, n_chunks, offsets.p);
    GSDF_CK(cudaGetLastError());
    long long total = 0;
    GSDF_CK(cudaMemcpyAsync(&total, offsets.p + n_chunks, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GSDF_CK(cudaStreamSynchronize(st));
    if (total == 0) return cudaSuccess;
    DevBuf<gsdf_voxel> out;
    GSDF_CK(out.alloc((size_t)total));
    const int dx = dm ? dm->dims[0] : 0, dy = dm ? dm->dims[1] : 0;
    const int ox = dm ? dm->origin[0] : 0, oy = dm ? dm->origin[1] : 0, oz = dm ? dm->origin[2] : 0;
    chunk_write_kernel<<<cgrid, kBlockVoxels, 0, st>>>(sorted, n_chunks, base.p, offsets.p, A, W, dense_voxels,
                                                       dx, dy, ox, oy, oz, h16 ? h16->H : nullptr,
                                                       h16 ? h16->scale : nullptr, out.p);
    GSDF_CK(cudaGetLastError());
    GSDF_CK(cudaStreamSynchronize(st));
    *out_dev = out.release();
    *n_out = total;
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------------
// oriented point cloud (Sec. 4.3)
// ------------------------------------------------------------------------------------------

struct PointSrc {  // where a chunk's voxels live and how to decode them
    const unsigned long long* sorted;  // hashed: sorted block keys (chunk c = block c); dense: null
    const long long* base;             // first payload index of each chunk (-1: none)
    const float4* A;
    const float* W;
    const ushort4* H16;
    const float* scale16;
    long long dense_voxels;
    int dx, dy, ox, oy, oz;
    float vs;
    int level;
};

// Voxel coordinate of thread t (local index) in chunk c.
__device__ __forceinline__ void chunk_voxel_m(const PointSrc& s, long long c, long long i, int t, int m[3]) {
    if (s.sorted) {
        int b[3];
        unpack_block(s.sorted[c], b);
        m[0] = b[0] * 8 + (t & 7);
        m[1] = b[1] * 8 + ((t >> 3) & 7);
        m[2] = b[2] * 8 + (t >> 6);
    } else {
        m[0] = s.ox + (int)(i % s.dx);
        m[1] = s.oy + (int)((i / s.dx) % s.dy);
        m[2] = s.oz + (int)(i / ((long long)s.dx * s.dy));
    }
}

// The points of one voxel on the FP32 index path: bit q of the result keeps point q (level 0: q = 0;
// level 1: subvoxel q = sx + 2 sy + 4 sz).  gh receives ghat, psi the voxel's distance.
__device__ __forceinline__ unsigned voxel_point_mask(const PointSrc& s, long long i, float gh[3], float& psi) {
    const float w = s.W[i];
    if (!(w > 0.0f)) return 0u;
    float g[3];
    if (s.H16) {  // FP16 payload: psi = sigma_b psi~, g = W gbar
        const ushort4 h = s.H16[i];
        psi = __half2float(__ushort_as_half(h.x)) * s.scale16[i >> 9];
        g[0] = __half2float(__ushort_as_half(h.y)) * w;
        g[1] = __half2float(__ushort_as_half(h.z)) * w;
        g[2] = __half2float(__ushort_as_half(h.w)) * w;
    } else {
        const float4 a = s.A[i];
        psi = __fdiv_rn(a.x, w);
        g[0] = a.y;
        g[1] = a.z;
        g[2] = a.w;
    }
    float n2 = __fmul_rn(g[0], g[0]);
    n2 = __fadd_rn(n2, __fmul_rn(g[1], g[1]));
    n2 = __fadd_rn(n2, __fmul_rn(g[2], g[2]));
    if (!(n2 > 0.0f)) return 0u;
    const float nr = __fsqrt_rn(n2);
#pragma unroll
    for (int k = 0; k < 3; ++k) gh[k] = __fdiv_rn(g[k], nr);
    if (s.level == 0) {
        const float half = 0.5f * s.vs;
        bool keep = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) keep &= fabsf(__fmul_rn(psi, gh[k])) <= half;
        return keep ? 1u : 0u;
    }
    const float quarter = 0.25f * s.vs;
    unsigned mask = 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float d0 = (q & 1) ? quarter : -quarter, d1 = (q & 2) ? quarter : -quarter;
        const float d2 = (q & 4) ? quarter : -quarter;
        // Taylor distance of the subvoxel centre, Eq. (taylor): psi + ghat . delta
        const float t = __fadd_rn(__fadd_rn(__fmul_rn(gh[0], d0), __fmul_rn(gh[1], d1)), __fmul_rn(gh[2], d2));
        const float pc = __fadd_rn(psi, t);
        const bool keep = fabsf(__fmul_rn(pc, gh[0])) <= quarter && fabsf(__fmul_rn(pc, gh[1])) <= quarter &&
                          fabsf(__fmul_rn(pc, gh[2])) <= quarter;
        mask |= keep ? (1u << q) : 0u;
    }
    return mask;
}

__device__ __forceinline__ long long chunk_index(const PointSrc& s, long long c, int t, bool& in) {
    const long long b0 = s.base[c];
    const long long i = b0 + t;
    in = b0 >= 0 && ((s.sorted != nullptr) || (i < s.dense_voxels));
    return i;
}

__global__ void points_count_kernel(PointSrc s, long long n_chunks, unsigned int* counts) {
    __shared__ unsigned int cnt;
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        bool in;
        const long long i = chunk_index(s, c, threadIdx.x, in);
        float gh[3], psi;
        const unsigned k = in ? __popc(voxel_point_mask(s, i, gh, psi)) : 0u;
        unsigned w = k;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&cnt, w);
        __syncthreads();
        if (threadIdx.x == 0) counts[c] = cnt;
        __syncthreads();
    }
}

__global__ void points_write_kernel(PointSrc s, long long n_chunks, const long long* __restrict__ offsets,
                                    gsdf_point* out) {
    __shared__ unsigned int warp_off[kBlockVoxels / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        bool in;
        const long long i = chunk_index(s, c, threadIdx.x, in);
        float gh[3], psi = 0.0f;
        const unsigned mask = in ? voxel_point_mask(s, i, gh, psi) : 0u;
        const unsigned k = __popc(mask);
        unsigned incl = k;  // inclusive scan of the points per thread within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_off[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (int w = 0; w < kBlockVoxels / 32; ++w) {
                const unsigned x = warp_off[w];
                warp_off[w] = run;
                run += x;
            }
        }
        __syncthreads();
        if (mask) {
            long long pos = offsets[c] + warp_off[warp] + incl - k;
            int m[3];
            chunk_voxel_m(s, c, i, threadIdx.x, m);
            const float vm[3] = {__fmul_rn(s.vs, (float)m[0]), __fmul_rn(s.vs, (float)m[1]), __fmul_rn(s.vs, (float)m[2])};
            const float quarter = 0.25f * s.vs;
            for (int q = 0; q < 8; ++q) {
                if (!((mask >> q) & 1u)) continue;
                gsdf_point o;
                o.m[0] = m[0];
                o.m[1] = m[1];
                o.m[2] = m[2];
                o.sub = s.level == 0 ? -1 : q;
                float pc = psi;
                float cpos[3] = {vm[0], vm[1], vm[2]};
                if (s.level != 0) {
                    const float d[3] = {(q & 1) ? quarter : -quarter, (q & 2) ? quarter : -quarter,
                                        (q & 4) ? quarter : -quarter};
                    const float t =
                        __fadd_rn(__fadd_rn(__fmul_rn(gh[0], d[0]), __fmul_rn(gh[1], d[1])), __fmul_rn(gh[2], d[2]));
                    pc = __fadd_rn(psi, t);
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk) cpos[kk] = __fadd_rn(vm[kk], d[kk]);
                }
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    o.p[kk] = __fsub_rn(cpos[kk], __fmul_rn(pc, gh[kk]));
                    o.n[kk] = -gh[kk];
                }
                out[pos++] = o;
            }
        }
        __syncthreads();
    }
}

cudaError_t extract_points(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                           float voxel_size, int level, cudaStream_t st, int num_sms, gsdf_point** out_dev,
                           long long* n_out) {
    *out_dev = nullptr;
    *n_out = 0;
    const unsigned grid = (unsigned)(num_sms * 8);
    DevBuf<unsigned long long> keys;
    long long n_chunks = 0, dense_voxels = 0;
    if (hm) {
        GSDF_CK(sorted_block_keys(*hm, n_slots, st, grid, keys, &n_chunks));
    } else {
        dense_voxels = (long long)dm->dims[0] * dm->dims[1] * dm->dims[2];
        n_chunks = (dense_voxels + kBlockVoxels - 1) / kBlockVoxels;
    }
    if (n_chunks == 0) return cudaSuccess;
    DevBuf<long long> base, offsets;
    DevBuf<unsigned int> counts;
    GSDF_CK(base.alloc((size_t)n_chunks));
    GSDF_CK(counts.alloc((size_t)n_chunks));
    GSDF_CK(offsets.alloc((size_t)n_chunks + 1));
    const HashMap hmv = hm ? *hm : HashMap{};
    const float* W = h16 ? h16->W : (hm ? hm->W : dm->W);
    const unsigned long long* sorted = hm ? keys.p : nullptr;
    const unsigned cgrid = (unsigned)(n_chunks < (long long)num_sms * 16 ? n_chunks : (long long)num_sms * 16);
    // chunk bases (the voxel counts of chunk_count_kernel are not needed here)
    chunk_count_kernel<<<cgrid, kBlockVoxels, 0, st>>>(hmv, sorted, n_chunks, dense_voxels, W, base.p, counts.p);
    GSDF_CK(cudaGetLastError());
    PointSrc src{};
    src.sorted = sorted;
    src.base = base.p;
    src.A = hm ? hm->A : dm->A;
    src.W = W;
    src.H16 = h16 ? h16->H : nullptr;
    src.scale16 = h16 ? h16->scale : nullptr;
    src.dense_voxels = dense_voxels;
    src.dx = dm ? dm->dims[0] : 0;
    src.dy = dm ? dm->dims[1] : 0;
    src.ox = dm ? dm->origin[0] : 0;
    src.oy = dm ? dm->origin[1] : 0;
    src.oz = dm ? dm->origin[2] : 0;
    src.vs = voxel_size;
    src.level = level;
    points_count_kernel<<<cgrid, kBlockVoxels, 0, st>>>(src, n_chunks, counts.p);
    GSDF_CK(cudaGetLastError());
    scan_kernel<<<1, 1024, 0, st>>>(counts.p, n_chunks, offsets.p);
    GSDF_CK(cudaGetLastError());
    long long total = 0;
    GSDF_CK(cudaMemcpyAsync(&total, offsets.p + n_chunks, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GSDF_CK(cudaStreamSynchronize(st));
    if (total == 0) return cudaSuccess;
    DevBuf<gsdf_point> out;
    GSDF_CK(out.alloc((size_t)total));
    points_write_kernel<<<cgrid, kBlockVoxels, 0, st>>>(src, n_chunks, offsets.p, out.p);
    GSDF_CK(cudaGetLastError());
    GSDF_CK(cudaStreamSynchronize(st));
    *out_dev = out.release();
    *n_out = total;
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------------
// marching cubes (Sec. 4.3)
// ------------------------------------------------------------------------------------------

// The triangulation of each of the 256 cube cases, generated at compile time from the rule stated
// in include/gsdf.h (gsdf_extract_mesh): per face, crossing edges joined in pairs (an ambiguous
// face separates its inside corners), the joins closed into loops walked from the smallest edge
// id toward its smaller neighbour, each loop fanned from its first edge.
struct McTable {
    unsigned char count[256];
    unsigned char tri[256][12][3];
};

__host__ __device__ constexpr int mc_edge_lo(int e) {  // corner of edge e with the edge's axis bit clear
    const int axis = e >> 2, k = e & 3;
    return axis == 0 ? (((k & 1) << 1) | ((k >> 1) << 2)) : axis == 1 ? ((k & 1) | ((k >> 1) << 2)) : ((k & 1) | ((k >> 1) << 1));
}

constexpr int mc_edge_between(int c0, int c1) {  // edge joining two corners that differ in one bit
    const int diff = c0 ^ c1;
    const int axis = diff == 1 ? 0 : diff == 2 ? 1 : 2;
    const int lo = c0 & ~diff;
    const int k = axis == 0 ? (((lo >> 1) & 1) | (((lo >> 2) & 1) << 1))
                            : axis == 1 ? ((lo & 1) | (((lo >> 2) & 1) << 1)) : ((lo & 1) | (((lo >> 1) & 1) << 1));
    return 4 * axis + k;
}

constexpr McTable make_mc_table() {
    McTable t{};
    for (int cs = 0; cs < 256; ++cs) {
        int nb[12][2] = {};
        int deg[12] = {};
        for (int axis = 0; axis < 3; ++axis) {
            for (int side = 0; side < 2; ++side) {
                const int u = (axis + 1) % 3, w = (axis + 2) % 3;
                const int du[4] = {0, 1, 1, 0}, dw[4] = {0, 0, 1, 1};
                int corner[4] = {}, edge[4] = {};
                for (int q = 0; q < 4; ++q) corner[q] = (side << axis) | (du[q] << u) | (dw[q] << w);
                for (int q = 0; q < 4; ++q) edge[q] = mc_edge_between(corner[q], corner[(q + 1) % 4]);
                int crossings = 0, first = -1, second = -1;
                for (int q = 0; q < 4; ++q) {
                    if (((cs >> corner[q]) & 1) != ((cs >> corner[(q + 1) % 4]) & 1)) {
                        ++crossings;
                        if (first < 0)
                            first = edge[q];
                        else
                            second = edge[q];
                    }
                }
                int join[2][2] = {};
                int nj = 0;
                if (crossings == 2) {
                    join[0][0] = first;
                    join[0][1] = second;
                    nj = 1;
                } else if (crossings == 4) {
                    for (int q = 0; q < 4; ++q)
                        if ((cs >> corner[q]) & 1) {  // cut off the inside corner q
                            join[nj][0] = edge[(q + 3) % 4];
                            join[nj][1] = edge[q];
                            ++nj;
                        }
                }
                for (int j = 0; j < nj; ++j) {
                    nb[join[j][0]][deg[join[j][0]]++] = join[j][1];
                    nb[join[j][1]][deg[join[j][1]]++] = join[j][0];
                }
            }
        }
        bool used[12] = {};
        int nt = 0;
        for (int start = 0; start < 12; ++start) {
            if (deg[start] != 2 || used[start]) continue;
            int loop[12] = {};
            int len = 0, prev = -1, cur = start;
            int next = nb[start][0] < nb[start][1] ? nb[start][0] : nb[start][1];
            while (true) {
                loop[len++] = cur;
                used[cur] = true;
                if (prev >= 0) next = nb[cur][0] == prev ? nb[cur][1] : nb[cur][0];
                prev = cur;
                cur = next;
                if (cur == start) break;
            }
            for (int k = 1; k + 1 < len; ++k) {
                t.tri[cs][nt][0] = (unsigned char)loop[0];
                t.tri[cs][nt][1] = (unsigned char)loop[k];
                t.tri[cs][nt][2] = (unsigned char)loop[k + 1];
                ++nt;
            }
        }
        t.count[cs] = (unsigned char)nt;
    }
    return t;
}

__constant__ McTable c_mc = make_mc_table();

// psi of the 8 corners of the cube with lowest corner m; false unless all are observed
template <class Map>
__device__ __forceinline__ bool cube_corners(const Map& map, const int m[3], float psi[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const long long idx = map.find(m[0] + (c & 1), m[1] + ((c >> 1) & 1), m[2] + ((c >> 2) & 1));
        if (idx < 0) return false;
        float g0, g1, g2;
        if (!map.voxel(idx, psi[c], g0, g1, g2)) return false;
    }
    return true;
}

__device__ __forceinline__ int cube_case(const float psi[8]) {
    int cs = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) cs |= (psi[c] > 0.0f ? 1 : 0) << c;
    return cs;
}

struct MeshSrc {
    const unsigned long long* sorted;
    const long long* base;
    long long dense_voxels;
    int dx, dy, ox, oy, oz;
    float vs;
};

__device__ __forceinline__ bool mesh_cube(const MeshSrc& s, long long c, int t, int m[3]) {
    const long long b0 = s.base[c];
    if (b0 < 0) return false;
    if (s.sorted) {
        int b[3];
        unpack_block(s.sorted[c], b);
        m[0] = b[0] * 8 + (t & 7);
        m[1] = b[1] * 8 + ((t >> 3) & 7);
        m[2] = b[2] * 8 + (t >> 6);
        return true;
    }
    const long long i = b0 + t;
    if (i >= s.dense_voxels) return false;
    m[0] = s.ox + (int)(i % s.dx);
    m[1] = s.oy + (int)((i / s.dx) % s.dy);
    m[2] = s.oz + (int)(i / ((long long)s.dx * s.dy));
    return true;
}

template <class Map>
__global__ void mesh_count_kernel(Map map, MeshSrc s, long long n_chunks, unsigned int* counts) {
    __shared__ unsigned int cnt;
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        int m[3];
        float psi[8];
        unsigned k = 0;
        if (mesh_cube(s, c, threadIdx.x, m) && cube_corners(map, m, psi)) k = c_mc.count[cube_case(psi)];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
        if ((threadIdx.x & 31) == 0 && k) atomicAdd(&cnt, k);
        __syncthreads();
        if (threadIdx.x == 0) counts[c] = cnt;
        __syncthreads();
    }
}

template <class Map>
__global__ void mesh_write_kernel(Map map, MeshSrc s, long long n_chunks, const long long* __restrict__ offsets,
                                  gsdf_triangle* out) {
    __shared__ unsigned int warp_off[kBlockVoxels / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        int m[3];
        float psi[8];
        int cs = 0;
        unsigned k = 0;
        if (mesh_cube(s, c, threadIdx.x, m) && cube_corners(map, m, psi)) {
            cs = cube_case(psi);
            k = c_mc.count[cs];
        }
        unsigned incl = k;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_off[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (int w = 0; w < kBlockVoxels / 32; ++w) {
                const unsigned x = warp_off[w];
                warp_off[w] = run;
                run += x;
            }
        }
        __syncthreads();
        long long pos = offsets[c] + warp_off[warp] + incl - k;
        for (unsigned q = 0; q < k; ++q) {
            gsdf_triangle o;
            o.m[0] = m[0];
            o.m[1] = m[1];
            o.m[2] = m[2];
            o.edges = 0;
#pragma unroll
            for (int v = 0; v < 3; ++v) {
                const int e = c_mc.tri[cs][q][v];
                o.edges |= e << (4 * v);
                const int a = mc_edge_lo(e), b = a | (1 << (e >> 2));
                const float t = psi[a] / (psi[a] - psi[b]);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float va = s.vs * (float)(m[d] + ((a >> d) & 1));
                    const float vb = s.vs * (float)(m[d] + ((b >> d) & 1));
                    o.v[3 * v + d] = va + t * (vb - va);
                }
            }
            out[pos++] = o;
        }
        __syncthreads();
    }
}

template <class Map>
static cudaError_t mesh_passes(const Map& map, const MeshSrc& src, long long n_chunks, unsigned cgrid,
                               unsigned int* counts, long long* offsets, cudaStream_t st, gsdf_triangle** out_dev,
                               long long* n_out) {
    mesh_count_kernel<Map><<<cgrid, kBlockVoxels, 0, st>>>(map, src, n_chunks, counts);
    GSDF_CK(cudaGetLastError());
    scan_kernel<<<1, 1024, 0, st>>>(counts, n_chunks, offsets);
    GSDF_CK(cudaGetLastError());
    long long total = 0;
    GSDF_CK(cudaMemcpyAsync(&total, offsets + n_chunks, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GSDF_CK(cudaStreamSynchronize(st));
    if (total == 0) return cudaSuccess;
    DevBuf<gsdf_triangle> out;
    GSDF_CK(out.alloc((size_t)total));
    mesh_write_kernel<Map><<<cgrid, kBlockVoxels, 0, st>>>(map, src, n_chunks, offsets, out.p);
    GSDF_CK(cudaGetLastError());
    GSDF_CK(cudaStreamSynchronize(st));
    *out_dev = out.release();
    *n_out = total;
    return cudaSuccess;
}

cudaError_t extract_mesh(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                         float voxel_size, cudaStream_t st, int num_sms, gsdf_triangle** out_dev, long long* n_out) {
    *out_dev = nullptr;
    *n_out = 0;
    const unsigned grid = (unsigned)(num_sms * 8);
    DevBuf<unsigned long long> keys;
    long long n_chunks = 0, dense_voxels = 0;
    if (hm) {
        GSDF_CK(sorted_block_keys(*hm, n_slots, st, grid, keys, &n_chunks));
    } else {
        dense_voxels = (long long)dm->dims[0] * dm->dims[1] * dm->dims[2];
        n_chunks = (dense_voxels + kBlockVoxels - 1) / kBlockVoxels;
    }
    if (n_chunks == 0) return cudaSuccess;
    DevBuf<long long> base, offsets;
    DevBuf<unsigned int> counts;
    GSDF_CK(base.alloc((size_t)n_chunks));
    GSDF_CK(counts.alloc((size_t)n_chunks));
    GSDF_CK(offsets.alloc((size_t)n_chunks + 1));
    const HashMap hmv = hm ? *hm : HashMap{};
    const float* W = h16 ? h16->W : (hm ? hm->W : dm->W);
    const unsigned long long* sorted = hm ? keys.p : nullptr;
    const unsigned cgrid = (unsigned)(n_chunks < (long long)num_sms * 16 ? n_chunks : (long long)num_sms * 16);
    chunk_count_kernel<<<cgrid, kBlockVoxels, 0, st>>>(hmv, sorted, n_chunks, dense_voxels, W, base.p, counts.p);
    GSDF_CK(cudaGetLastError());
    MeshSrc src{};
    src.sorted = sorted;
    src.base = base.p;
    src.dense_voxels = dense_voxels;
    src.dx = dm ? dm->dims[0] : 0;
    src.dy = dm ? dm->dims[1] : 0;
    src.ox = dm ? dm->origin[0] : 0;
    src.oy = dm ? dm->origin[1] : 0;
    src.oz = dm ? dm->origin[2] : 0;
    src.vs = voxel_size;
    if (h16) return mesh_passes(*h16, src, n_chunks, cgrid, counts.p, offsets.p, st, out_dev, n_out);
    if (hm) return mesh_passes(*hm, src, n_chunks, cgrid, counts.p, offsets.p, st, out_dev, n_out);
    return mesh_passes(*dm, src, n_chunks, cgrid, counts.p, offsets.p, st, out_dev, n_out);
}

cudaError_t load_voxels(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, float trunc,
                        const gsdf_voxel* in_dev, long long n, int* err, unsigned int* n_blocks, cudaStream_t st,
                        int num_sms) {
    const unsigned grid = (unsigned)(num_sms * 8);
    if (h16)
        load_kernel_hashed16<<<grid, 256, 0, st>>>(*h16, in_dev, n, trunc, err, n_blocks);
    else if (hm)
        load_kernel_hashed<<<grid, 256, 0, st>>>(*hm, in_dev, n, err, n_blocks);
    else
        load_kernel_dense<<<grid, 256, 0, st>>>(*dm, in_dev, n, err);
    return cudaGetLastError();
}

}  // namespace gsdf
