// Fusion of one depth frame: Eqs. (sdf_update) and (gradient_update), pixel-driven as in
// Sec. 5.3 ("for each pixel, update all voxels along the viewing ray within the truncation
// distance"), with block allocation fused in (hashed maps allocate the block of every voxel
// that receives an update).
//
// One thread per pixel.  The FP32 index path decides validity, the normal and its 75 degree test,
// the voxels of the ray's samples and the band test, exactly as specified; the world point of a
// sample at depth z is t + z (R ray), with the rotated ray formed once per pixel.  Each distinct
// voxel of the ray then receives (w d, w n_w) with one 16-byte vector atomic and w with one scalar
// atomic.  Because the payload stores W psi, the per-voxel sums equal the sequential running
// average of Eq. (sdf_update) up to summation order.  The loop runs over distinct voxels, not
// samples, so the lanes of a warp stay converged on the expensive visit body, and the last block
// looked up is cached per ray.
#include "integrate_device.cuh"

namespace gsdf {

template <class Map>
__global__ void __launch_bounds__(kIntThreads, 4)
integrate_kernel(Map map, const float* __restrict__ depth, Intr K, Params prm,
                 const double* __restrict__ T_wc, gsdf_integrate_stats* stats, Scratch sc) {
    __shared__ PoseF pose;
    __shared__ unsigned int s_rays, s_visits, s_new;
    if (threadIdx.x < 32) round_pose_warp(T_wc, pose);
    if (threadIdx.x == 0) s_rays = s_visits = s_new = 0u;
    __syncthreads();

    const int n_px = K.width * K.height;
    unsigned int my_rays = 0, my_visits = 0;
    for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < n_px; pix += gridDim.x * blockDim.x)
        integrate_ray(map, depth, K, prm, pose, pix, sc.err, &s_new, my_rays, my_visits);
    // block-aggregated statistics
    for (int o = 16; o > 0; o >>= 1) {
        my_rays += __shfl_xor_sync(0xffffffffu, my_rays, o);
        my_visits += __shfl_xor_sync(0xffffffffu, my_visits, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_rays, my_rays);
        atomicAdd(&s_visits, my_visits);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_new) atomicAdd(sc.n_blocks, s_new);
        if (stats) {
            atomicAdd((unsigned long long*)&stats->n_rays, (unsigned long long)s_rays);
            atomicAdd((unsigned long long*)&stats->n_visits, (unsigned long long)s_visits);
            atomicAdd((unsigned long long*)&stats->n_blocks_new, (unsigned long long)s_new);
        }
    }
}

// FP16 maps: the frame's occupied accumulator entries (list16_entries).  blockDim.x is a
// multiple of 32.
__global__ void list16_kernel(HashMap16 m) {
    list16_entries(m, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// FP16 maps, second pass: one block per listed accumulator entry (apply16_entry).
__global__ void __launch_bounds__(kApplyThreads) apply16_kernel(HashMap16 m, float trunc) {
    __shared__ float red[kApplyThreads / 32];
    const unsigned cnt = __ldcg(m.acount);
    for (unsigned q = blockIdx.x; q < cnt; q += gridDim.x) apply16_entry(m, q, trunc, red);
}

__global__ void integrate_stats_total(gsdf_integrate_stats* stats, const unsigned int* n_blocks) {
    stats->n_blocks_total = (long long)*n_blocks;
}

cudaError_t launch_integrate16(const HashMap16& hm, const float* depth, const Intr& K, const Params& prm,
                               const double* T_wc, gsdf_integrate_stats* stats, const Scratch& sc, int num_sms,
                               cudaStream_t st) {
    if (stats) {
        cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(gsdf_integrate_stats), st);
        if (e != cudaSuccess) return e;
    }
    const long long n_px = (long long)K.width * K.height;
    const unsigned blocks = (unsigned)((n_px + kIntThreads - 1) / kIntThreads);
    integrate_kernel<HashMap16><<<blocks, kIntThreads, 0, st>>>(hm, depth, K, prm, T_wc, stats, sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    list16_kernel<<<2 * num_sms, 256, 0, st>>>(hm);
    apply16_kernel<<<16 * num_sms, kApplyThreads, 0, st>>>(hm, prm.trunc);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(hm.acount, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    if (stats) integrate_stats_total<<<1, 1, 0, st>>>(stats, sc.n_blocks);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const DenseMap* dm, const HashMap* hm, const float* depth,
                             const Intr& K, const Params& prm, const double* T_wc,
                             gsdf_integrate_stats* stats, const Scratch& sc, cudaStream_t st) {
    if (stats) {
        cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(gsdf_integrate_stats), st);
        if (e != cudaSuccess) return e;
    }
    const long long n_px = (long long)K.width * K.height;
    const unsigned blocks = (unsigned)((n_px + kIntThreads - 1) / kIntThreads);
    if (dm)
        integrate_kernel<DenseMap><<<blocks, kIntThreads, 0, st>>>(*dm, depth, K, prm, T_wc, stats, sc);
    else
        integrate_kernel<HashMap><<<blocks, kIntThreads, 0, st>>>(*hm, depth, K, prm, T_wc, stats, sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (stats) integrate_stats_total<<<1, 1, 0, st>>>(stats, sc.n_blocks);
    return cudaGetLastError();
}

}  // namespace gsdf
