// Fusion of one depth frame: Eqs. (sdf_update) and (gradient_update), pixel-driven as in
// Sec. 5.3 ("for each pixel, update all voxels along the viewing ray within the truncation
// distance"), with block allocation fused in (hashed maps allocate the block of every voxel
// that receives an update).
//
// One thread per pixel: the FP32 index path decides validity, the normal and its 75 degree
// test, the ray samples' voxels and the band test exactly as specified; each distinct voxel of
// the ray then receives (w d, w n_w) with one 16-byte vector atomic and w with one scalar
// atomic.  Because the payload stores W psi, the per-voxel sums equal the sequential running
// average of Eq. (sdf_update) up to summation order.
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
    const float s = __fsqrt_rn(nn);
    n[0] = __fdiv_rn(n[0], s);
    n[1] = __fdiv_rn(n[1], s);
    n[2] = __fdiv_rn(n[2], s);
    float dp = dot3_rn(n, p);
    if (dp < 0.0f) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
        dp = -dp;
    }
    const float c = __fdiv_rn(dp, __fsqrt_rn(dot3_rn(p, p)));
    return c >= prm.cos_max;
}

template <class Map>
__global__ void __launch_bounds__(kIntThreads)
integrate_kernel(Map map, const float* __restrict__ depth, Intr K, Params prm,
                 const double* __restrict__ T_wc, gsdf_integrate_stats* stats, Scratch sc) {
    __shared__ PoseF pose;
    __shared__ unsigned int s_rays, s_visits, s_new;
    if (threadIdx.x == 0) {
        double T[16];
        for (int i = 0; i < 16; ++i) T[i] = T_wc[i];
        round_pose(T, pose);
        s_rays = s_visits = s_new = 0u;
    }
    __syncthreads();

    const int n_px = K.width * K.height;
    unsigned int my_rays = 0, my_visits = 0;
    for (int pix = blockIdx.x * blockDim.x + threadIdx.x; pix < n_px; pix += gridDim.x * blockDim.x) {
        const float D = __ldg(depth + pix);
        if (!depth_ok(D, K.depth_max)) continue;
        const int v = pix / K.width;
        const int u = pix - v * K.width;
        float n[3];
        if (!pixel_normal(depth, K, prm, u, v, D, n)) continue;
        ++my_rays;
        // world normal R n (value path)
        const float nwx = pose.R[0] * n[0] + pose.R[1] * n[1] + pose.R[2] * n[2];
        const float nwy = pose.R[3] * n[0] + pose.R[4] * n[1] + pose.R[5] * n[2];
        const float nwz = pose.R[6] * n[0] + pose.R[7] * n[1] + pose.R[8] * n[2];
        const float xn = __fmul_rn(__fsub_rn((float)u, K.cx), K.ifx);
        const float yn = __fmul_rn(__fsub_rn((float)v, K.cy), K.ify);
        int pmx = 0, pmy = 0, pmz = 0;
        bool have_prev = false;
        const int Kb = prm.band_half;
        for (int k = 0; k <= 2 * Kb; ++k) {
            const float z = __fadd_rn(D, __fmul_rn((float)(k - Kb), prm.half_vs));
            const float p[3] = {__fmul_rn(z, xn), __fmul_rn(z, yn), z};
            float P[3];
            xform(pose.R, pose.t, p, P);
            const int mx = round_voxel(P[0], prm.inv_vs);
            const int my = round_voxel(P[1], prm.inv_vs);
            const int mz = round_voxel(P[2], prm.inv_vs);
            if (have_prev && mx == pmx && my == pmy && mz == pmz) continue;
            pmx = mx;
            pmy = my;
            pmz = mz;
            have_prev = true;
            const float vc[3] = {__fmul_rn((float)mx, prm.vs), __fmul_rn((float)my, prm.vs),
                                 __fmul_rn((float)mz, prm.vs)};
            const float zv = __fadd_rn(dot_row(pose.RT + 6, vc), pose.tinv[2]);
            const float d = __fsub_rn(zv, D);
            if (d > prm.trunc || d < -prm.trunc) continue;
            const float w = d <= prm.eps ? 1.0f : (prm.trunc - d) / (prm.trunc - prm.eps);
            if (!(w > 0.0f)) continue;
            const long long idx = map.find_or_insert(mx, my, mz, sc.err, &s_new);
            if (idx < 0) continue;
            atomicAdd(map.A + idx, make_float4(w * d, w * nwx, w * nwy, w * nwz));
            atomicAdd(map.W + idx, w);
            ++my_visits;
        }
    }
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

__global__ void integrate_stats_total(gsdf_integrate_stats* stats, const unsigned int* n_blocks) {
    stats->n_blocks_total = (long long)*n_blocks;
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
