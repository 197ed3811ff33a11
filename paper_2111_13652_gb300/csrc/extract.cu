// Extraction of every voxel with W > 0 in a canonical order, and checkpoint loading.
//
// Hashed maps: the occupied slots' block keys are collected, sorted (bitonic sort in global
// memory; keys are unique, so the order is total), counted, prefix-summed, and each block's
// voxels with W > 0 are written in local-index order.  Dense maps are processed as chunks of
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

cudaError_t extract_voxels(const DenseMap* dm, const HashMap* hm, const HashMap16* h16, long long n_slots,
                           cudaStream_t st, int num_sms, gsdf_voxel** out_dev, long long* n_out) {
    *out_dev = nullptr;
    *n_out = 0;
    const unsigned grid = (unsigned)(num_sms * 8);
    DevBuf<unsigned long long> keys;
    long long n_chunks = 0, dense_voxels = 0;
    if (hm) {
        DevBuf<unsigned int> cnt;
        DevBuf<unsigned long long> tmp;
        GSDF_CK(cnt.alloc(1));
        GSDF_CK(tmp.alloc((size_t)n_slots));
        GSDF_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int), st));
        collect_keys_kernel<<<grid, 256, 0, st>>>(hm->keys, n_slots, tmp.p, cnt.p);
        GSDF_CK(cudaGetLastError());
        unsigned int n_keys = 0;
        GSDF_CK(cudaMemcpyAsync(&n_keys, cnt.p, sizeof(unsigned int), cudaMemcpyDeviceToHost, st));
        GSDF_CK(cudaStreamSynchronize(st));
        const long long N = next_pow2(n_keys > 0 ? n_keys : 1);
        GSDF_CK(keys.alloc((size_t)N));
        GSDF_CK(cudaMemsetAsync(keys.p, 0xFF, sizeof(unsigned long long) * (size_t)N, st));
        if (n_keys)
            GSDF_CK(cudaMemcpyAsync(keys.p, tmp.p, sizeof(unsigned long long) * n_keys, cudaMemcpyDeviceToDevice, st));
        for (long long k = 2; k <= N; k <<= 1)
            for (long long j = k >> 1; j > 0; j >>= 1) {
                bitonic_step_kernel<<<grid, 256, 0, st>>>(keys.p, N, j, k);
                GSDF_CK(cudaGetLastError());
            }
        GSDF_CK(cudaStreamSynchronize(st));
        n_chunks = n_keys;
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
