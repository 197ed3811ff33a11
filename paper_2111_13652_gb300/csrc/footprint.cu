// Measurement utility: the distinct voxels and 8^3 blocks that one tracking step or one fusion of a
// frame touches, counted on the device.  These are the compulsory payload and table accesses of
// the two passes (each distinct voxel and block read once), the denominator-free counterpart of
// their per-access byte counts.  Not part of the per-frame loop: every call allocates two bitmaps,
// runs, copies the counts back and frees them.
//
//   tracking: a pixel with valid depth whose nearest voxel (Eq. taylor: m* = round(P / v_s) on the
//             FP32 index path) exists, is observed (W > 0) and has g != 0 marks that voxel and its
//             block -- exactly the pixels gsdf_track_step uses;
//   fusion:   every ray that passes the depth and normal tests marks the distinct voxels of its band
//             samples that receive a weight > 0 (Eqs. sdf_update, gradient_update), as gsdf_integrate
//             visits them; blocks are looked up, not inserted, so the call is made after the fusion
//             of the same frame at the same pose, when every updated block exists.
#include <algorithm>

#include "integrate_device.cuh"

namespace gsdf {

// A map that only marks: voxel_index finds (never inserts) and scatter sets the voxel's and its
// block's bits.  `Inner` provides find (a DenseMap, or the key table of a hashed map).
template <class Inner>
struct MarkMap {
    Inner inner;
    unsigned int* vbits;  // one bit per payload index
    unsigned int* bbits;  // one bit per block (payload index / 512)
};

template <class Inner>
__device__ __forceinline__ void mark(const MarkMap<Inner>& m, long long idx) {
    atomicOr(m.vbits + (idx >> 5), 1u << (idx & 31));
    const long long b = idx >> 9;
    atomicOr(m.bbits + (b >> 5), 1u << (b & 31));
}

template <>
__device__ __forceinline__ long long voxel_index<MarkMap<DenseMap>>(const MarkMap<DenseMap>& map, int mx, int my,
                                                                    int mz, BlockCache&, int*, unsigned int*,
                                                                    const int*) {
    return map.inner.find(mx, my, mz);
}
template <>
__device__ __forceinline__ long long voxel_index<MarkMap<HashMap>>(const MarkMap<HashMap>& map, int mx, int my,
                                                                   int mz, BlockCache&, int*, unsigned int*,
                                                                   const int*) {
    return map.inner.find(mx, my, mz);
}
template <class Inner>
__device__ __forceinline__ void scatter(const MarkMap<Inner>& m, long long i, float4, float) {
    mark(m, i);
}

template <class Inner>
__global__ void fuse_footprint_kernel(MarkMap<Inner> map, const float* __restrict__ depth, Intr K, Params prm,
                                      const double* __restrict__ T_wc) {
    __shared__ PoseF pose;
    if (threadIdx.x < 32) round_pose_warp(T_wc, pose);
    __syncthreads();
    unsigned int rays = 0, visits = 0, n_new = 0;
    int err = 0;
    const int n_px = K.width * K.height;
    for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < n_px; pix += gridDim.x * blockDim.x)
        integrate_ray(map, depth, K, prm, pose, pix, &err, &n_new, rays, visits);
}

// Voxel payloads as the tracking kernel reads them: a usable voxel is observed with g != 0.
template <class Map>
__global__ void track_footprint_kernel(Map map, unsigned int* vbits, unsigned int* bbits,
                                       const float* __restrict__ depth, Intr K, Params prm,
                                       const double* __restrict__ T_wc) {
    __shared__ PoseF pose;
    if (threadIdx.x < 32) round_pose_warp(T_wc, pose);
    __syncthreads();
    const int n_px = K.width * K.height;
    for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < n_px; pix += gridDim.x * blockDim.x) {
        const float D = __ldg(depth + pix);
        if (!depth_ok(D, K.depth_max)) continue;
        const int v = pix / K.width, u = pix - v * K.width;
        float dw[3];
        ray_world(K, pose.R, u, v, dw);
        const int mx = round_voxel(ray_coord(D, dw[0], pose.t[0]), prm.inv_vs);
        const int my = round_voxel(ray_coord(D, dw[1], pose.t[1]), prm.inv_vs);
        const int mz = round_voxel(ray_coord(D, dw[2], pose.t[2]), prm.inv_vs);
        const long long idx = map.find(mx, my, mz);
        if (idx < 0) continue;
        float psi, g0, g1, g2;
        if (!map.voxel(idx, psi, g0, g1, g2)) continue;
        if (!(g0 * g0 + g1 * g1 + g2 * g2 > 0.0f)) continue;
        atomicOr(vbits + (idx >> 5), 1u << (idx & 31));
        const long long b = idx >> 9;
        atomicOr(bbits + (b >> 5), 1u << (b & 31));
    }
}

__global__ void popcount_kernel(const unsigned int* __restrict__ bits, long long n_words,
                                unsigned long long* out) {
    unsigned long long c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_words;
         i += (long long)gridDim.x * blockDim.x)
        c += (unsigned long long)__popc(__ldg(bits + i));
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace gsdf

using namespace gsdf;

extern "C" gsdf_status gsdf_footprint(gsdf_handle* h, int32_t what, const float* depth_dev, const gsdf_intrinsics* K,
                                      const double* T_wc_dev, int64_t out[2]) {
    if (!h || !depth_dev || !K || !T_wc_dev || !out || (what != GSDF_FOOTPRINT_TRACK && what != GSDF_FOOTPRINT_FUSE))
        return GSDF_ERR_INVALID_ARG;
    if (!(K->fx > 0.0f) || !(K->fy > 0.0f) || !isfinite(K->cx) || !isfinite(K->cy) || K->width <= 0 ||
        K->height <= 0 || K->width > 32768 || K->height > 32768 || !(K->depth_max > 0.0f))
        return GSDF_ERR_INVALID_ARG;
    Intr ki;
    ki.fx = K->fx;
    ki.fy = K->fy;
    ki.cx = K->cx;
    ki.cy = K->cy;
    ki.width = K->width;
    ki.height = K->height;
    ki.depth_max = K->depth_max;
    ki.ifx = (float)(1.0 / (double)K->fx);
    ki.ify = (float)(1.0 / (double)K->fy);
    const long long n_vox = h->n_voxels;
    const long long vwords = (n_vox + 31) / 32, bwords = ((n_vox + 511) / 512 + 31) / 32;
    unsigned int *vbits = nullptr, *bbits = nullptr;
    unsigned long long* cnt = nullptr;
    cudaStream_t st = h->stream;
    cudaError_t e = cudaMalloc(&vbits, sizeof(unsigned int) * (size_t)vwords);
    if (e == cudaSuccess) e = cudaMalloc(&bbits, sizeof(unsigned int) * (size_t)bwords);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(vbits, 0, sizeof(unsigned int) * (size_t)vwords, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bbits, 0, sizeof(unsigned int) * (size_t)bwords, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st);
    const int threads = 256;
    const unsigned grid = (unsigned)std::min<long long>(((long long)ki.width * ki.height + threads - 1) / threads,
                                                        (long long)8 * h->num_sms);
    if (e == cudaSuccess) {
        const HashMap keys = h->fp16 ? h->hm16.base : h->hm;
        if (what == GSDF_FOOTPRINT_TRACK) {
            if (!h->hashed)
                track_footprint_kernel<<<grid, threads, 0, st>>>(h->dm, vbits, bbits, depth_dev, ki, h->prm, T_wc_dev);
            else if (h->fp16)
                track_footprint_kernel<<<grid, threads, 0, st>>>(h->hm16, vbits, bbits, depth_dev, ki, h->prm,
                                                                 T_wc_dev);
            else
                track_footprint_kernel<<<grid, threads, 0, st>>>(h->hm, vbits, bbits, depth_dev, ki, h->prm, T_wc_dev);
        } else if (!h->hashed) {
            fuse_footprint_kernel<<<grid, threads, 0, st>>>(MarkMap<DenseMap>{h->dm, vbits, bbits}, depth_dev, ki,
                                                            h->prm, T_wc_dev);
        } else {
            fuse_footprint_kernel<<<grid, threads, 0, st>>>(MarkMap<HashMap>{keys, vbits, bbits}, depth_dev, ki,
                                                            h->prm, T_wc_dev);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        popcount_kernel<<<4 * h->num_sms, 256, 0, st>>>(vbits, vwords, cnt);
        popcount_kernel<<<h->num_sms, 256, 0, st>>>(bbits, bwords, cnt + 1);
        e = cudaGetLastError();
    }
    unsigned long long host[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, cnt, sizeof(host), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(vbits);
    cudaFree(bbits);
    cudaFree(cnt);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GSDF_ERR_OOM : GSDF_ERR_CUDA;
    }
    out[0] = (int64_t)host[0];
    out[1] = (int64_t)host[1];
    return GSDF_OK;
}
