// Tracking: one Gauss-Newton step of Eq. (tracking) with the first-order model Eq. (taylor)
// (Sec. 4.1), reduced and solved on the device (Sec. 5.1: Gauss-Newton + Cholesky).  The same
// kernel, instantiated with kTrilinear, is the trilinear 8-lookup baseline of Eqs. (dir_dist),
// (dir_grad).
//
// One kernel per step.  Each thread walks pixels with a grid stride, evaluates the one-lookup
// Taylor residual and its Jacobian and accumulates the 30 unique terms (21 of H, 6 of b, E,
// n_valid, n_huber) in FP32 registers; a warp reduce-scatters them by butterfly exchange, a
// block combines its warps in FP64 with a fixed tree, and each block adds its row to exact
// fixed-point grid accumulators.  The last block to finish (ticket counter, no waiting) reads
// the sums -- identical whatever the order blocks finished in -- solves the 6x6 system in FP64,
// applies exp(xi^) to the device pose and writes the statistics.  No host round trip per step.
#include "track_device.cuh"

namespace gsdf {

template <class Map, bool kTrilinear = false>
__global__ void __launch_bounds__(kTrackThreads, kTrackBlocksPerSM)
track_kernel(Map map, const float* __restrict__ depth, Intr K, Params prm, double* T_wc,
             gsdf_track_stats* stats, Scratch sc) {
    __shared__ TrackShared sh;
    const int n_px = K.width * K.height;
    const int pix0 = blockIdx.x * blockDim.x + threadIdx.x;
    const float d0 = pix0 < n_px ? __ldg(depth + pix0) : 0.0f;  // in flight with the pose load
    load_pose(sh, T_wc);
    __syncthreads();
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
    for_pixels(depth, K.width, pix0, n_px, gridDim.x * blockDim.x, d0, [&](float D, int, int u, int v) {
        if (kTrilinear)
            track_pixel_trilinear(map, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc);
        else
            track_pixel(map, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc);
    });
    const unsigned long long s = block_reduce_terms(sh, acc);
    // block b adds into accumulator copy b mod kAccumCopies (spreads same-address atomics)
    if (!add_partial_and_ticket(sh, s, sc.accum, sc.counter, blockIdx.x, gridDim.x)) return;
    finish_scene(sh, sc.accum, sc.counter, prm, T_wc, stats);
}

// ------------------------------------------------------------------------------------------
// Chained steps (gsdf_track with n >= 2): step j's normal equations are solved at the start of
// step j + 1 by every block, from the exact sums step j left in memory, instead of by the last
// block of step j after a ticket.  The kernel boundary is then the only grid-wide
// synchronisation of a step: no fence, ticket or single-block tail, and no pose round trip
// through memory before the pixels.  Each block computes the identical FP64 solve, exponential
// and product (the same operations on the same exact sums), so poses and statistics are bit for
// bit those of n single steps.
//
// Scratch (sc.chain): three accumulator sets and two pose buffers.  Step j adds into set j % 3
// and reads set (j - 1) % 3; its block 0 writes the pose T_j into buffer j % 2, the statistics of
// step j - 1, and zeroes set (j + 1) % 3, the one step j + 1 adds into (last read by step j - 1).
// A final one-block kernel solves step n - 1, writes T_n and its statistics, and zeroes the sets
// it read, so that all three are zero again for the next call.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long* chain_set(const Scratch& sc, int k) {
    return sc.chain + (size_t)(k % 3) * kAccumWords;
}
__device__ __forceinline__ double* chain_pose(const Scratch& sc, int k) {
    return reinterpret_cast<double*>(sc.chain + 3 * (size_t)kAccumWords) + 16 * (k & 1);
}

// Every block: the pose of step j into sh (FP64 in sh.Tsh, rounded in sh.Rt).  For j >= 1 it is
// exp(xi_{j-1}^) T_{j-1}, solved here from set (j - 1) % 3; block 0 publishes it and the
// statistics of step j - 1 and zeroes set (j + 1) % 3.  Ends with a block-wide barrier.
__device__ __forceinline__ void chain_pose_in(TrackShared& sh, const double* T_wc, const Params& prm,
                                              gsdf_track_stats* stats, const Scratch& sc, int j) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (j == 0) {
        load_pose(sh, T_wc);
        __syncthreads();
        return;
    }
    const double* T_prev = j == 1 ? T_wc : chain_pose(sc, j - 1);
    if (threadIdx.x < 16) sh.Tsh[threadIdx.x] = threadIdx.x < 12 ? __ldcg(T_prev + threadIdx.x) : 0.0;
    gather_sums(sh, chain_set(sc, j + 2), false);  // set (j - 1) % 3
    if (blockIdx.x == 0) {
        unsigned long long* z = chain_set(sc, j + 1);
        for (int i = threadIdx.x; i < kAccumWords; i += blockDim.x) z[i] = 0ull;
    }
    __syncthreads();
    if (warp == 0) {
        double tn;
        solve_step_warp(sh, prm, (blockIdx.x == 0 && stats) ? stats + (j - 1) : nullptr, tn);
        __syncwarp();
        if (lane < 12) {
            sh.Tsh[lane] = tn;
            const int r = lane >> 2, c = lane & 3;
            sh.Rt[c < 3 ? 3 * r + c : 9 + r] = __double2float_rn(tn);
            if (blockIdx.x == 0) chain_pose(sc, j)[lane] = tn;
        }
    }
    __syncthreads();
}

template <class Map, bool kTrilinear>
__global__ void __launch_bounds__(kTrackThreads, kTrackBlocksPerSM)
track_chain_kernel(Map map, const float* __restrict__ depth, Intr K, Params prm, const double* T_wc,
                   gsdf_track_stats* stats, Scratch sc, int j) {
    __shared__ TrackShared sh;
    const int n_px = K.width * K.height;
    const int pix0 = blockIdx.x * blockDim.x + threadIdx.x;
    const float d0 = pix0 < n_px ? __ldg(depth + pix0) : 0.0f;  // in flight with the sums and pose
    chain_pose_in(sh, T_wc, prm, stats, sc, j);
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
    for_pixels(depth, K.width, pix0, n_px, gridDim.x * blockDim.x, d0, [&](float D, int, int u, int v) {
        if (kTrilinear)
            track_pixel_trilinear(map, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc);
        else
            track_pixel(map, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc);
    });
    const unsigned long long s = block_reduce_terms(sh, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < 4 && lane < kTerms)
        atomicAdd(chain_set(sc, j) + (blockIdx.x % kAccumCopies) * 128 + warp * 32 + lane, s);
}

// The last step's solve: T_n into T_wc, the statistics of step n - 1, sets (n - 1) % 3 and
// (n + 1) % 3 zeroed.  One block of 128 threads.
__global__ void __launch_bounds__(128) track_chain_final_kernel(Params prm, double* T_wc, gsdf_track_stats* stats,
                                                                Scratch sc, int n) {
    __shared__ TrackShared sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double* T_prev = chain_pose(sc, n - 1);
    if (threadIdx.x < 16) sh.Tsh[threadIdx.x] = threadIdx.x < 12 ? __ldcg(T_prev + threadIdx.x) : 0.0;
    gather_sums(sh, chain_set(sc, n - 1), true);
    {
        unsigned long long* z = chain_set(sc, n + 1);
        for (int i = threadIdx.x; i < kAccumWords; i += blockDim.x) z[i] = 0ull;
    }
    __syncthreads();
    if (warp == 0) {
        double tn;
        solve_step_warp(sh, prm, stats ? stats + (n - 1) : nullptr, tn);
        if (lane < 12) T_wc[lane] = tn;
    }
}

static long long track_blocks(const Intr& K, const Scratch& sc, int num_sms) {
    const long long n_px = (long long)K.width * K.height;
    long long blocks = (n_px + kTrackThreads - 1) / kTrackThreads;
    long long cap = (long long)kTrackBlocksPerSM * num_sms;
    if (cap > sc.max_track_blocks) cap = sc.max_track_blocks;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

template <class Map, bool kTri>
static cudaError_t launch_step(const Map& map, const float* depth, const Intr& K, const Params& prm, double* T_wc,
                               gsdf_track_stats* stats, const Scratch& sc, int num_sms, cudaStream_t st) {
    const unsigned blocks = (unsigned)track_blocks(K, sc, num_sms);
    track_kernel<Map, kTri><<<blocks, kTrackThreads, 0, st>>>(map, depth, K, prm, T_wc, stats, sc);
    return cudaGetLastError();
}

template <class Map, bool kTri>
static cudaError_t launch_chain(const Map& map, const float* depth, const Intr& K, const Params& prm, double* T_wc,
                               gsdf_track_stats* stats, const Scratch& sc, int num_sms, int n, cudaStream_t st) {
    const unsigned blocks = (unsigned)track_blocks(K, sc, num_sms);
    for (int j = 0; j < n; ++j) {
        track_chain_kernel<Map, kTri><<<blocks, kTrackThreads, 0, st>>>(map, depth, K, prm, T_wc, stats, sc, j);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    track_chain_final_kernel<<<1, 128, 0, st>>>(prm, T_wc, stats, sc, n);
    return cudaGetLastError();
}

cudaError_t launch_track_chain(const DenseMap* dm, const HashMap* hm, const HashMap16* hm16, bool trilinear,
                               const float* depth, const Intr& K, const Params& prm, double* T_wc,
                               gsdf_track_stats* stats, const Scratch& sc, int num_sms, int n, cudaStream_t st) {
    if (!sc.chain || n < 2) return cudaErrorInvalidValue;
    if (hm16) return launch_chain<HashMap16, false>(*hm16, depth, K, prm, T_wc, stats, sc, num_sms, n, st);
    if (trilinear) {
        if (dm) return launch_chain<DenseMap, true>(*dm, depth, K, prm, T_wc, stats, sc, num_sms, n, st);
        return launch_chain<HashMap, true>(*hm, depth, K, prm, T_wc, stats, sc, num_sms, n, st);
    }
    if (dm) return launch_chain<DenseMap, false>(*dm, depth, K, prm, T_wc, stats, sc, num_sms, n, st);
    return launch_chain<HashMap, false>(*hm, depth, K, prm, T_wc, stats, sc, num_sms, n, st);
}

cudaError_t launch_track16(const HashMap16& hm, const float* depth, const Intr& K, const Params& prm, double* T_wc,
                           gsdf_track_stats* stats, const Scratch& sc, int num_sms, cudaStream_t st) {
    return launch_step<HashMap16, false>(hm, depth, K, prm, T_wc, stats, sc, num_sms, st);
}

cudaError_t launch_track(const DenseMap* dm, const HashMap* hm, const float* depth, const Intr& K,
                         const Params& prm, double* T_wc, gsdf_track_stats* stats,
                         const Scratch& sc, int num_sms, cudaStream_t st) {
    if (dm) return launch_step<DenseMap, false>(*dm, depth, K, prm, T_wc, stats, sc, num_sms, st);
    return launch_step<HashMap, false>(*hm, depth, K, prm, T_wc, stats, sc, num_sms, st);
}

cudaError_t launch_track_trilinear(const DenseMap* dm, const HashMap* hm, const float* depth, const Intr& K,
                                   const Params& prm, double* T_wc, gsdf_track_stats* stats, const Scratch& sc,
                                   int num_sms, cudaStream_t st) {
    if (dm) return launch_step<DenseMap, true>(*dm, depth, K, prm, T_wc, stats, sc, num_sms, st);
    return launch_step<HashMap, true>(*hm, depth, K, prm, T_wc, stats, sc, num_sms, st);
}

}  // namespace gsdf

// ------------------------------------------------------------------------------------------
// Allocation-free tracking step.
//
// Some callers cannot call cudaMalloc: code that must run inside a fixed device-memory budget
// handed to it by a host framework (which owns every allocation), or a real-time loop in which
// an allocation, with the device-wide synchronisation it may imply, is not allowed.  For them
// gsdf_track_step_dense_noalloc runs the tracking kernel above on a caller-owned dense grid and
// takes its scratch (the fixed-point accumulators and the last-block ticket) from a file-scope
// device array instead of a handle's allocations.
// ------------------------------------------------------------------------------------------

#include <mutex>

namespace gsdf {
namespace {

// kAccumWords accumulator words, then one word for the ticket counter, padded: 16640 bytes.  The
// scratch a tracking step needs does not depend on the image or grid size (the accumulators are
// replicated a fixed number of times), so its fit is checked here, at compile time.
constexpr size_t kStaticScratchWords = kAccumWords + 32;
constexpr size_t kStaticScratchNeeded = kAccumWords + 1;
static_assert(kStaticScratchNeeded <= kStaticScratchWords, "static scratch too small");
static __device__ __align__(256) unsigned long long g_static_scratch[kStaticScratchWords];

constexpr int kMaxStaticDevices = 64;
std::mutex g_static_mu;
unsigned long long* g_static_ptr[kMaxStaticDevices];  // device address of the array, per device
int g_static_sms[kMaxStaticDevices];

bool finite_positive(float x) { return isfinite(x) && x > 0.0f; }

}  // namespace
}  // namespace gsdf

extern "C" gsdf_status gsdf_track_step_dense_noalloc(const float* depth_dev, const gsdf_intrinsics* K,
                                                     const void* A_dev, const float* W_dev,
                                                     const int32_t dims[3], const int32_t origin[3],
                                                     float voxel_size, float huber_delta, double damping,
                                                     double* T_wc_dev, gsdf_track_stats* stats_dev,
                                                     void* cuda_stream) {
    using namespace gsdf;
    if (!depth_dev || !K || !A_dev || !W_dev || !dims || !origin || !T_wc_dev) return GSDF_ERR_INVALID_ARG;
    if (!finite_positive(voxel_size) || !finite_positive(huber_delta) || !isfinite(damping) || damping < 0.0)
        return GSDF_ERR_INVALID_ARG;
    if (!finite_positive(K->fx) || !finite_positive(K->fy) || !isfinite(K->cx) || !isfinite(K->cy) ||
        K->width <= 0 || K->height <= 0 || K->width > 32768 || K->height > 32768 || !finite_positive(K->depth_max))
        return GSDF_ERR_INVALID_ARG;
    long long n = 1;
    for (int i = 0; i < 3; ++i) {
        if (dims[i] <= 0 || dims[i] > (1 << 16)) return GSDF_ERR_INVALID_ARG;
        n *= dims[i];
        if ((long long)origin[i] < -(1ll << 23) || (long long)origin[i] + dims[i] > (1ll << 23)) return GSDF_ERR_INVALID_ARG;
    }
    if (n > (1ll << 34)) return GSDF_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GSDF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxStaticDevices) return GSDF_ERR_INVALID_ARG;
    unsigned long long* scratch = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_ptr[dev]) {  // once per device, with that device current
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return GSDF_ERR_CUDA;
            int count = 0;
            if (cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GSDF_ERR_CUDA;
            g_static_ptr[dev] = (unsigned long long*)p;
            g_static_sms[dev] = count;
        }
        scratch = g_static_ptr[dev];
        sms = g_static_sms[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the array keeps the previous call's contents: clear the accumulators and the ticket
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * kStaticScratchNeeded, st) != cudaSuccess)
        return GSDF_ERR_CUDA;

    DenseMap dm;
    dm.A = (float4*)const_cast<void*>(A_dev);
    dm.W = const_cast<float*>(W_dev);
    for (int i = 0; i < 3; ++i) {
        dm.dims[i] = dims[i];
        dm.origin[i] = origin[i];
    }
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
    // the tracking kernel reads v_s, 1 / v_s, the Huber threshold and the damping; the fusion-only
    // fields take the library's defaults (T = 5 v_s, eps = v_s, 75 degrees), as gsdf_create would
    const Params prm = make_params(voxel_size, 5.0f * voxel_size, voxel_size, huber_delta, 0.25881904f, damping);
    Scratch sc = {};
    sc.accum = scratch;
    sc.counter = (unsigned int*)(scratch + kAccumWords);
    sc.max_track_blocks = 2 * sms;
    const cudaError_t e = launch_track(&dm, nullptr, depth_dev, ki, prm, T_wc_dev, stats_dev, sc, sms, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? GSDF_ERR_OOM : GSDF_ERR_CUDA;
    return GSDF_OK;
}

// ------------------------------------------------------------------------------------------
// Gauss-Newton update from given normal equations (the last stage of a tracking step on its
// own): one warp per system, the same device solve and exponential map as the tracking kernels.
// ------------------------------------------------------------------------------------------

namespace gsdf {
namespace {

__global__ void __launch_bounds__(32) gn_update_kernel(const double* __restrict__ Hb,
                                                       const int64_t* __restrict__ n_valid, double lam_scale,
                                                       double* T, double* xi_out, int32_t* status) {
    __shared__ double hb[32], xi[6], dT[12], Ts[16];
    const size_t s = blockIdx.x;
    const int lane = threadIdx.x;
    hb[lane] = lane < 27 ? Hb[27 * s + lane] : 0.0;
    if (lane < 16) Ts[lane] = T[16 * s + lane];
    __syncwarp();
    const double tr = hb[0] + hb[6] + hb[11] + hb[15] + hb[18] + hb[20];
    const bool ok = solve6_warp(hb, tr, lam_scale, (long long)n_valid[s], xi);
    if (ok) {
        se3_exp_warp(xi, dT);
        const double tn = compose_entry(dT, Ts);
        if (lane < 12) T[16 * s + lane] = tn;
    }
    if (xi_out && lane < 6) xi_out[6 * s + lane] = ok ? xi[lane] : 0.0;
    if (status && lane == 0) status[s] = ok ? (int32_t)GSDF_OK : (int32_t)GSDF_ERR_DEGENERATE;
}

}  // namespace
}  // namespace gsdf

extern "C" gsdf_status gsdf_gn_update(int32_t n, const double* Hb_dev, const int64_t* n_valid_dev, double damping,
                                      double* T_dev, double* xi_dev, int32_t* status_dev, void* cuda_stream) {
    using namespace gsdf;
    if (n < 0 || !isfinite(damping) || damping < 0.0) return GSDF_ERR_INVALID_ARG;
    if (n == 0) return GSDF_OK;
    if (!Hb_dev || !n_valid_dev || !T_dev) return GSDF_ERR_INVALID_ARG;
    gn_update_kernel<<<(unsigned)n, 32, 0, (cudaStream_t)cuda_stream>>>(Hb_dev, n_valid_dev, damping / 6.0, T_dev,
                                                                        xi_dev, status_dev);
    return cudaGetLastError() == cudaSuccess ? GSDF_OK : GSDF_ERR_CUDA;
}
