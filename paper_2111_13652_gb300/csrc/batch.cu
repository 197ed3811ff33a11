// Batched tracking and fusion of many independent scenes.
//
// A batch groups existing handles (dense, hashed FP32 or hashed FP16 maps of any voxel size) with
// one depth frame per scene (any resolution).  The pixels of all scenes are cut into tiles.
// For batches within the limits of a parameter table (64 scenes, 4096 tiles), tracking runs one
// thread block per tile and fusion one per fusion item (batch_track_grid_kernel,
// batch_integrate_grid_kernel), with the scenes' fixed values and the tile table in the launch's
// parameters (only the depth pointers, which the device advances between frames, and the fusion
// poses rounded on the device are read from the descriptor table); larger batches run persistent
// kernels whose resident CTAs pull (scene, tile) items from a device counter until none are left.
//   * Tracking: a tile's 30 normal-equation terms go into its scene's exact fixed-point
//     accumulators (the same accumulators and arithmetic as the single-scene kernel), and the
//     CTA that takes a scene's last ticket solves that scene's 6x6 system and updates its pose
//     while the other CTAs keep working on other scenes, so the serial FP64 tail of every scene
//     is hidden behind the others' pixel work.  One launch is one Gauss-Newton step of every
//     scene.
//   * Fusion: a prologue rounds every scene's pose once, the persistent kernel fuses all
//     scenes' rays (FP16 scenes into their frame accumulators), one persistent pass folds the
//     FP16 scenes' accumulators into their payload, and an epilogue writes the per-scene block
//     totals.
//   * A frame: gsdf_batch_frame replays one CUDA graph holding n tracking launches, the fusion
//     launches and, when strides are set, a kernel that advances every scene's depth pointer to
//     its next frame on the device.  Nothing is uploaded from the host between frames.
// The tile size and the number of resident CTAs per SM come from gsdf_batch_autotune, which
// times the candidates on the batch's own frames (tracking only, on scratch copies of the poses)
// and caches the choice per shape class (the multiset of image sizes).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "integrate_device.cuh"
#include "track_device.cuh"

namespace gsdf {

constexpr int kSceneDense = 0, kSceneHashed = 1, kSceneHashed16 = 2;
// The persistent kernels are instantiated for the set of scene kinds a batch holds (bit k set when
// kind k is present), so that each carries only the map code it needs.
constexpr int kAllKinds = 7;

struct SceneDesc {
    int kind;        // kSceneDense, kSceneHashed or kSceneHashed16
    int n_px;        // pixels of the scene's frame
    int tile_begin;  // first global tile index of the scene
    int n_tiles;
    DenseMap dm;
    HashMap hm;
    HashMap16 hm16;
    Params prm;
    Intr K;
    const float* depth;
    long long depth_stride;  // elements the depth pointer advances after each gsdf_batch_frame
    double* pose;
    gsdf_track_stats* tstats;
    gsdf_integrate_stats* istats;
    unsigned long long* accum;
    unsigned int* ticket;
    int* err;
    unsigned int* n_blocks;
    PoseF pose32;  // the pose rounded once, written by the fusion prologue
};

// An FP16 map whose tracking lookup resolves the key before it loads the payload.  In the
// persistent kernel, whose registers are capped for two CTAs of 512 threads per SM, loading the
// home slot's payload and scale together with the key (HashMap16::lookup) costs more in spills
// than it saves in latency.
struct HashMap16TwoStep {
    HashMap16 m;
    __device__ __forceinline__ bool lookup(int mx, int my, int mz, float& psi, float& gx, float& gy,
                                           float& gz) const {
        const long long idx = m.find(mx, my, mz);
        return idx >= 0 && m.voxel(idx, psi, gx, gy, gz);
    }
};

// The per-scene values of a tracking step that stay fixed from frame to frame, and the scene of
// every tile, passed to batch_track_grid_kernel as a kernel parameter.  Read from the launch's
// parameter space with a block-uniform index, they need no registers across the pixel loop (the
// persistent kernel holds its descriptor's values in registers capped at 64 per thread, and
// spills).  The depth pointers, which the device advances between frames, and the fusion's
// rounded poses stay in the descriptor table in global memory.
struct SceneConst {
    int kind, n_px, tile_begin, n_tiles;
    Intr K;
    Params prm;
    DenseMap dm;
    HashMap hm;
    HashMap16 hm16;
    unsigned long long* accum;
    unsigned int* ticket;
    int* err;
    unsigned int* n_blocks;
    double* pose;  // the scene's pose (fixed pointer; its value is updated on the device)
    gsdf_track_stats* tstats;
    gsdf_integrate_stats* istats;
};
constexpr int kParamScenes = 64;   // batches of up to this many scenes
constexpr int kParamTiles = 4096;  // and tiles use the grid kernels
struct BatchTrackParams {
    SceneConst s[kParamScenes];
    unsigned short tile_scene[kParamTiles];
};
static_assert(sizeof(BatchTrackParams) <= 32000, "kernel parameters are limited to 32,764 bytes");

// counters: [0] tracking work, [1] tracking exits, [2] fusion work, [3] fusion exits
constexpr int kBatchCounters = 4;

__device__ __forceinline__ void batch_exit(unsigned int* work, unsigned int* exited) {
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned e = atomicAdd(exited, 1u);
        if (e == gridDim.x - 1) {  // every CTA has taken its last item: reset for the next launch
            *work = 0u;
            *exited = 0u;
        }
    }
}

template <int KINDS>
__global__ void __launch_bounds__(kTrackThreads, kTrackBlocksPerSM)
batch_track_kernel(SceneDesc* descs, const int* __restrict__ tile_scene, int total_tiles, int tile_px,
                   unsigned int* counters) {
    __shared__ TrackShared sh;
    __shared__ int s_item;
    while (true) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counters + 0, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= total_tiles) break;
        SceneDesc* d = descs + __ldg(tile_scene + item);
        load_pose(sh, d->pose);
        const int lt = item - d->tile_begin;
        const int p0 = lt * tile_px;
        const int p1 = min(p0 + tile_px, d->n_px);
        const Params prm = d->prm;
        const Intr K = d->K;
        const float* depth = d->depth;
        __syncthreads();
        float acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
        const int pix0 = p0 + threadIdx.x;
        const float d0 = pix0 < p1 ? __ldg(depth + pix0) : 0.0f;
        const int kind = d->kind;
        if ((KINDS & (1 << kSceneDense)) && kind == kSceneDense) {
            const DenseMap m = d->dm;
            for_pixels(depth, K.width, pix0, p1, blockDim.x, d0,
                       [&](float D, int, int u, int v) { track_pixel(m, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc); });
        } else if ((KINDS & (1 << kSceneHashed)) && kind == kSceneHashed) {
            const HashMap m = d->hm;
            for_pixels(depth, K.width, pix0, p1, blockDim.x, d0,
                       [&](float D, int, int u, int v) { track_pixel(m, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc); });
        } else if ((KINDS & (1 << kSceneHashed16)) && kind == kSceneHashed16) {
            const HashMap16TwoStep m{d->hm16};
            for_pixels(depth, K.width, pix0, p1, blockDim.x, d0,
                       [&](float D, int, int u, int v) { track_pixel(m, D, K, sh.Rt, sh.Rt + 9, prm, u, v, acc); });
        }
        const unsigned long long s = block_reduce_terms(sh, acc);
        if (add_partial_and_ticket(sh, s, d->accum, d->ticket, lt, (unsigned)d->n_tiles))
            finish_scene(sh, d->accum, d->ticket, prm, d->pose, d->tstats);
        __syncthreads();
    }
    batch_exit(counters + 0, counters + 1);
}

// One Gauss-Newton step of every scene as a grid of tiles (block b tracks tile b), for batches
// within the parameter table's limits; otherwise the persistent kernel above runs.  The same
// per-tile work, reductions, tickets and finishing as batch_track_kernel.
constexpr int kGridTrackThreads = 256;  // threads per tile block of batch_track_grid_kernel

template <int KINDS>
__global__ void __launch_bounds__(kGridTrackThreads, 2 * kTrackBlocksPerSM)
batch_track_grid_kernel(const SceneDesc* descs, int tile_px, const __grid_constant__ BatchTrackParams p) {
    __shared__ TrackShared sh;
    const int item = blockIdx.x;
    const int si = p.tile_scene[item];
    const SceneConst& c = p.s[si];
    const SceneDesc* d = descs + si;
    load_pose(sh, c.pose);
    const int lt = item - c.tile_begin;
    const int p0 = lt * tile_px;
    const int p1 = min(p0 + tile_px, c.n_px);
    const float* depth = d->depth;
    __syncthreads();
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.0f;
    const int pix0 = p0 + threadIdx.x;
    const float d0 = pix0 < p1 ? __ldg(depth + pix0) : 0.0f;
    const int kind = c.kind;
    if ((KINDS & (1 << kSceneDense)) && kind == kSceneDense) {
        for_pixels(depth, c.K.width, pix0, p1, blockDim.x, d0,
                   [&](float D, int, int u, int v) { track_pixel(c.dm, D, c.K, sh.Rt, sh.Rt + 9, c.prm, u, v, acc); });
    } else if ((KINDS & (1 << kSceneHashed)) && kind == kSceneHashed) {
        for_pixels(depth, c.K.width, pix0, p1, blockDim.x, d0,
                   [&](float D, int, int u, int v) { track_pixel(c.hm, D, c.K, sh.Rt, sh.Rt + 9, c.prm, u, v, acc); });
    } else if ((KINDS & (1 << kSceneHashed16)) && kind == kSceneHashed16) {
        for_pixels(depth, c.K.width, pix0, p1, blockDim.x, d0,
                   [&](float D, int, int u, int v) { track_pixel(c.hm16, D, c.K, sh.Rt, sh.Rt + 9, c.prm, u, v, acc); });
    }
    const unsigned long long s = block_reduce_terms<kGridTrackThreads / 32>(sh, acc);
    if (add_partial_and_ticket(sh, s, c.accum, c.ticket, lt, (unsigned)c.n_tiles))
        finish_scene(sh, c.accum, c.ticket, c.prm, c.pose, c.tstats);
}

// Fusion prologue: round every pose once and clear the per-scene statistics.
__global__ void batch_prologue_kernel(SceneDesc* descs, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SceneDesc* d = descs + s;
    double T[16];
    for (int i = 0; i < 16; ++i) T[i] = d->pose[i];
    round_pose(T, d->pose32);
    if (d->istats) {
        d->istats->n_rays = 0;
        d->istats->n_visits = 0;
        d->istats->n_blocks_new = 0;
        d->istats->n_blocks_total = 0;
    }
}

// Fusion epilogue: the per-scene block totals; FP16 scenes' accumulator lists are emptied (their
// entries were folded and freed by the apply pass).
__global__ void batch_epilogue_kernel(SceneDesc* descs, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SceneDesc* d = descs + s;
    if (d->istats) d->istats->n_blocks_total = d->kind != kSceneDense ? (long long)*d->n_blocks : 0;
    if (d->kind == kSceneHashed16) *d->hm16.acount = 0u;
}

// FP16 scenes, second pass of fusion: every CTA walks the FP16 scenes in order and folds the
// listed accumulator entries q = blockIdx.x, blockIdx.x + gridDim.x, ... of each.
__global__ void __launch_bounds__(kApplyThreads)
batch_apply16_kernel(const SceneDesc* descs, const int* __restrict__ fp16_scenes, int n_fp16) {
    __shared__ float red[kApplyThreads / 32];
    for (int i = 0; i < n_fp16; ++i) {
        const SceneDesc* d = descs + __ldg(fp16_scenes + i);
        const HashMap16 m = d->hm16;
        const float trunc = d->prm.trunc;
        const unsigned cnt = __ldcg(m.acount);
        for (unsigned q = blockIdx.x; q < cnt; q += gridDim.x) apply16_entry(m, q, trunc, red);
    }
}

// FP16 scenes, between the passes: list every FP16 scene's occupied accumulator entries (blockDim.x
// a multiple of 32).
__global__ void batch_list16_kernel(const SceneDesc* descs, const int* __restrict__ fp16_scenes, int n_fp16) {
    for (int i = 0; i < n_fp16; ++i)
        list16_entries(descs[__ldg(fp16_scenes + i)].hm16, blockIdx.x * blockDim.x + threadIdx.x,
                       gridDim.x * blockDim.x);
}

// Advance every scene's depth pointer to its next frame (after a frame's fusion).
__global__ void batch_advance_kernel(SceneDesc* descs, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) descs[s].depth += descs[s].depth_stride;
}

constexpr int kBatchIntThreads = 256;
constexpr int kFusePx = 4096;  // pixels per fusion work item (16 per thread)

// Fusion cuts its own work items, smaller than tracking tiles (which the autotuner sizes for the
// tracking step): item i is part i % split of tracking tile i / split, fuse_px pixels.
template <int KINDS>
__global__ void __launch_bounds__(kBatchIntThreads, 4)
batch_integrate_kernel(SceneDesc* descs, const int* __restrict__ tile_scene, int total_items, int tile_px,
                       int split, int fuse_px, unsigned int* counters) {
    __shared__ PoseF pose;
    __shared__ int s_item;
    __shared__ unsigned int s_rays, s_visits, s_new;
    while (true) {
        if (threadIdx.x == 0) {
            s_item = (int)atomicAdd(counters + 2, 1u);
            s_rays = s_visits = s_new = 0u;
        }
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        const int tile = item / split;
        SceneDesc* d = descs + __ldg(tile_scene + tile);
        if (threadIdx.x < (int)(sizeof(PoseF) / sizeof(float)))
            reinterpret_cast<float*>(&pose)[threadIdx.x] = reinterpret_cast<const float*>(&d->pose32)[threadIdx.x];
        const int lt = tile - d->tile_begin;
        const int p0 = min(lt * tile_px + (item - tile * split) * fuse_px, d->n_px);
        const int p1 = min(p0 + fuse_px, d->n_px);
        const Params prm = d->prm;
        const Intr K = d->K;
        const float* depth = d->depth;
        __syncthreads();
        unsigned int rays = 0, visits = 0;
        const int kind = d->kind;
        if ((KINDS & (1 << kSceneDense)) && kind == kSceneDense) {
            const DenseMap m = d->dm;
            for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
                integrate_ray(m, depth, K, prm, pose, pix, d->err, &s_new, rays, visits);
        } else if ((KINDS & (1 << kSceneHashed)) && kind == kSceneHashed) {
            const HashMap m = d->hm;
            for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
                integrate_ray(m, depth, K, prm, pose, pix, d->err, &s_new, rays, visits);
        } else if ((KINDS & (1 << kSceneHashed16)) && kind == kSceneHashed16) {
            const HashMap16 m = d->hm16;
            for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
                integrate_ray(m, depth, K, prm, pose, pix, d->err, &s_new, rays, visits);
        }
        for (int o = 16; o > 0; o >>= 1) {
            rays += __shfl_xor_sync(0xffffffffu, rays, o);
            visits += __shfl_xor_sync(0xffffffffu, visits, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_rays, rays);
            atomicAdd(&s_visits, visits);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_new) atomicAdd(d->n_blocks, s_new);
            if (d->istats) {
                atomicAdd((unsigned long long*)&d->istats->n_rays, (unsigned long long)s_rays);
                atomicAdd((unsigned long long*)&d->istats->n_visits, (unsigned long long)s_visits);
                atomicAdd((unsigned long long*)&d->istats->n_blocks_new, (unsigned long long)s_new);
            }
        }
        __syncthreads();
    }
    batch_exit(counters + 2, counters + 3);
}

// Fusion of every scene's frame as a grid of work items (block b fuses item b: part b % split of
// tracking tile b / split), the scenes' fixed values read from the launch's parameters (as
// batch_track_grid_kernel); the same per-item work as batch_integrate_kernel.
template <int KINDS>
__global__ void __launch_bounds__(kBatchIntThreads, 4)
batch_integrate_grid_kernel(const SceneDesc* descs, int tile_px, int split, int fuse_px,
                            const __grid_constant__ BatchTrackParams p) {
    __shared__ PoseF pose;
    __shared__ unsigned int s_rays, s_visits, s_new;
    const int item = blockIdx.x;
    const int tile = item / split;
    const int si = p.tile_scene[tile];
    const SceneConst& c = p.s[si];
    const SceneDesc* d = descs + si;
    if (threadIdx.x < (int)(sizeof(PoseF) / sizeof(float)))
        reinterpret_cast<float*>(&pose)[threadIdx.x] = reinterpret_cast<const float*>(&d->pose32)[threadIdx.x];
    if (threadIdx.x == 0) s_rays = s_visits = s_new = 0u;
    const int lt = tile - c.tile_begin;
    const int p0 = min(lt * tile_px + (item - tile * split) * fuse_px, c.n_px);
    const int p1 = min(p0 + fuse_px, c.n_px);
    const float* depth = d->depth;
    __syncthreads();
    unsigned int rays = 0, visits = 0;
    const int kind = c.kind;
    if ((KINDS & (1 << kSceneDense)) && kind == kSceneDense) {
        for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
            integrate_ray(c.dm, depth, c.K, c.prm, pose, pix, c.err, &s_new, rays, visits);
    } else if ((KINDS & (1 << kSceneHashed)) && kind == kSceneHashed) {
        for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
            integrate_ray(c.hm, depth, c.K, c.prm, pose, pix, c.err, &s_new, rays, visits);
    } else if ((KINDS & (1 << kSceneHashed16)) && kind == kSceneHashed16) {
        for (int pix = p0 + threadIdx.x; pix < p1; pix += blockDim.x)
            integrate_ray(c.hm16, depth, c.K, c.prm, pose, pix, c.err, &s_new, rays, visits);
    }
    for (int o = 16; o > 0; o >>= 1) {
        rays += __shfl_xor_sync(0xffffffffu, rays, o);
        visits += __shfl_xor_sync(0xffffffffu, visits, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&s_rays, rays);
        atomicAdd(&s_visits, visits);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_new) atomicAdd(c.n_blocks, s_new);
        gsdf_integrate_stats* is = c.istats;
        if (is) {
            atomicAdd((unsigned long long*)&is->n_rays, (unsigned long long)s_rays);
            atomicAdd((unsigned long long*)&is->n_visits, (unsigned long long)s_visits);
            atomicAdd((unsigned long long*)&is->n_blocks_new, (unsigned long long)s_new);
        }
    }
}

}  // namespace gsdf

using namespace gsdf;

struct gsdf_batch {
    int n = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int num_sms = 0;
    std::vector<gsdf_handle*> h;
    SceneDesc* d_desc = nullptr;
    SceneDesc* h_desc = nullptr;  // pinned staging of the descriptor table
    cudaEvent_t desc_copied = nullptr;
    bool desc_pending = false;
    bool frames_set = false;
    bool strided = false;  // some scene's depth pointer advances after each gsdf_batch_frame
    unsigned int* d_counters = nullptr;
    double* d_scratch_pose = nullptr;  // autotuning works on copies of the poses
    int* d_fp16_scenes = nullptr;      // indices of the FP16 scenes
    int n_fp16 = 0;
    int kinds = 0;                     // bit k set when a scene of kind k is present
    int* d_tile_scene = nullptr;
    int tile_cap = 0;
    int total_tiles = 0;
    int tile_px = 2048;
    int ctas_per_sm = 1;
    std::vector<int> n_px;  // frame size per scene in the current tile table
    std::map<std::vector<int>, std::pair<int, int>> tuned;  // shape class -> (tile_px, ctas/SM)
    // cached graphs: n tracking steps (gsdf_batch_track) and a whole frame (gsdf_batch_frame),
    // each with the launch configuration it was recorded with
    struct Cached {
        cudaGraphExec_t exec = nullptr;
        int iters = 0, tiles = 0, tile_px = 0, ctas = 0;
        bool strided = false;
        const int* tile_ptr = nullptr;
        unsigned params_version = 0;
    };
    Cached track_graph, frame_graph;
    // parameters of batch_track_grid_kernel (valid when grid_ok), rebuilt whenever the descriptor
    // table or the tiles change; graphs recorded with another version are recorded again
    BatchTrackParams* params = nullptr;
    std::vector<int> scene_of;  // scene of every tile
    bool grid_ok = false;
    unsigned params_version = 1;
};

namespace {

gsdf_status batch_status(cudaError_t e) {
    if (e == cudaSuccess) return GSDF_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GSDF_ERR_OOM : GSDF_ERR_CUDA;
}

bool intr_ok(const gsdf_intrinsics& K) {
    auto pos = [](float x) { return std::isfinite(x) && x > 0.0f; };
    return pos(K.fx) && pos(K.fy) && std::isfinite(K.cx) && std::isfinite(K.cy) && K.width > 0 && K.height > 0 &&
           K.width <= 32768 && K.height <= 32768 && pos(K.depth_max);
}

void free_batch(gsdf_batch* b) {
    if (b->track_graph.exec) cudaGraphExecDestroy(b->track_graph.exec);
    if (b->frame_graph.exec) cudaGraphExecDestroy(b->frame_graph.exec);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->desc_copied) cudaEventDestroy(b->desc_copied);
    cudaFree(b->d_desc);
    cudaFreeHost(b->h_desc);
    cudaFree(b->d_counters);
    cudaFree(b->d_scratch_pose);
    cudaFree(b->d_fp16_scenes);
    cudaFree(b->d_tile_scene);
    delete b->params;
    delete b;
}

// Rebuild the grid kernel's parameters from the host descriptor table and the tile table.
void fill_params(gsdf_batch* b, const std::vector<int>& scene_of) {
    b->grid_ok = b->n <= kParamScenes && b->total_tiles <= kParamTiles;
    if (!b->grid_ok) return;
    BatchTrackParams next;
    memset(&next, 0, sizeof(next));
    for (int s = 0; s < b->n; ++s) {
        const SceneDesc& d = b->h_desc[s];
        SceneConst& c = next.s[s];
        c.kind = d.kind;
        c.n_px = d.n_px;
        c.tile_begin = d.tile_begin;
        c.n_tiles = d.n_tiles;
        c.K = d.K;
        c.prm = d.prm;
        c.dm = d.dm;
        c.hm = d.hm;
        c.hm16 = d.hm16;
        c.accum = d.accum;
        c.ticket = d.ticket;
        c.err = d.err;
        c.n_blocks = d.n_blocks;
        c.pose = d.pose;
        c.tstats = d.tstats;
        c.istats = d.istats;
    }
    for (int t = 0; t < b->total_tiles; ++t) next.tile_scene[t] = (unsigned short)scene_of[t];
    if (memcmp(&next, b->params, sizeof(next)) != 0) {
        memcpy(b->params, &next, sizeof(next));
        ++b->params_version;
    }
}

// (Re)build the tile table for the current frame sizes and tile size; host-synchronous (only when
// sizes or the tile size change).
cudaError_t build_tiles(gsdf_batch* b) {
    std::vector<int> scene_of;
    int t = 0;
    for (int s = 0; s < b->n; ++s) {
        const int nt = (b->n_px[s] + b->tile_px - 1) / b->tile_px;
        b->h_desc[s].tile_begin = t;
        b->h_desc[s].n_tiles = nt;
        for (int k = 0; k < nt; ++k) scene_of.push_back(s);
        t += nt;
    }
    b->total_tiles = t;
    if (t > b->tile_cap) {
        cudaFree(b->d_tile_scene);
        b->d_tile_scene = nullptr;
        cudaError_t e = cudaMalloc(&b->d_tile_scene, sizeof(int) * (size_t)t);
        if (e != cudaSuccess) return e;
        b->tile_cap = t;
    }
    b->scene_of = scene_of;
    fill_params(b, scene_of);
    return cudaMemcpy(b->d_tile_scene, scene_of.data(), sizeof(int) * (size_t)t, cudaMemcpyHostToDevice);
}

cudaError_t upload_desc(gsdf_batch* b) {
    fill_params(b, b->scene_of);
    cudaError_t e = cudaMemcpyAsync(b->d_desc, b->h_desc, sizeof(SceneDesc) * (size_t)b->n, cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->desc_copied, b->stream);
    b->desc_pending = true;
    return e;
}

cudaError_t wait_desc(gsdf_batch* b) {
    if (!b->desc_pending) return cudaSuccess;
    b->desc_pending = false;
    return cudaEventSynchronize(b->desc_copied);
}

// the instantiation of a persistent kernel for a batch's set of scene kinds
template <int K>
void launch_track_for(gsdf_batch* b, int grid, cudaStream_t st) {
    if (b->grid_ok) {
        batch_track_grid_kernel<K><<<b->total_tiles, kGridTrackThreads, 0, st>>>(b->d_desc, b->tile_px, *b->params);
        return;
    }
    batch_track_kernel<K><<<grid, kTrackThreads, 0, st>>>(b->d_desc, b->d_tile_scene, b->total_tiles, b->tile_px,
                                                           b->d_counters);
}
template <int K>
void launch_fusion_for(gsdf_batch* b, int grid, int items, int split, int fuse_px, cudaStream_t st) {
    if (b->grid_ok) {
        batch_integrate_grid_kernel<K><<<items, kBatchIntThreads, 0, st>>>(b->d_desc, b->tile_px, split, fuse_px,
                                                                            *b->params);
        return;
    }
    batch_integrate_kernel<K><<<grid, kBatchIntThreads, 0, st>>>(b->d_desc, b->d_tile_scene, items, b->tile_px,
                                                                  split, fuse_px, b->d_counters);
}

cudaError_t launch_batch_track(gsdf_batch* b, cudaStream_t st) {
    const int grid = std::max(1, std::min(b->total_tiles, b->ctas_per_sm * b->num_sms));
    switch (b->kinds) {
        case 1: launch_track_for<1>(b, grid, st); break;
        case 2: launch_track_for<2>(b, grid, st); break;
        case 3: launch_track_for<3>(b, grid, st); break;
        case 4: launch_track_for<4>(b, grid, st); break;
        case 5: launch_track_for<5>(b, grid, st); break;
        case 6: launch_track_for<6>(b, grid, st); break;
        default: launch_track_for<kAllKinds>(b, grid, st); break;
    }
    return cudaGetLastError();
}

// Fusion of every scene's frame at its current pose: prologue, ray march, FP16 apply pass (if
// the batch holds FP16 scenes), epilogue.
cudaError_t launch_batch_fusion(gsdf_batch* b, cudaStream_t st) {
    const int pro = (b->n + 127) / 128;
    batch_prologue_kernel<<<pro, 128, 0, st>>>(b->d_desc, b->n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int fuse_px = std::min(b->tile_px, kFusePx);
    const int split = b->tile_px / fuse_px;  // tile sizes are powers of two
    const int items = b->total_tiles * split;
    const int grid = std::max(1, std::min(items, 6 * b->num_sms));
    switch (b->kinds) {
        case 1: launch_fusion_for<1>(b, grid, items, split, fuse_px, st); break;
        case 2: launch_fusion_for<2>(b, grid, items, split, fuse_px, st); break;
        case 3: launch_fusion_for<3>(b, grid, items, split, fuse_px, st); break;
        case 4: launch_fusion_for<4>(b, grid, items, split, fuse_px, st); break;
        case 5: launch_fusion_for<5>(b, grid, items, split, fuse_px, st); break;
        case 6: launch_fusion_for<6>(b, grid, items, split, fuse_px, st); break;
        default: launch_fusion_for<kAllKinds>(b, grid, items, split, fuse_px, st); break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (b->n_fp16 > 0) {
        batch_list16_kernel<<<2 * b->num_sms, 256, 0, st>>>(b->d_desc, b->d_fp16_scenes, b->n_fp16);
        batch_apply16_kernel<<<16 * b->num_sms, kApplyThreads, 0, st>>>(b->d_desc, b->d_fp16_scenes, b->n_fp16);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    batch_epilogue_kernel<<<pro, 128, 0, st>>>(b->d_desc, b->n);
    return cudaGetLastError();
}

// One frame: n_iters tracking steps, fusion, and the depth pointers' advance.
cudaError_t launch_batch_frame(gsdf_batch* b, int n_iters, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < n_iters && e == cudaSuccess; ++it) e = launch_batch_track(b, st);
    if (e == cudaSuccess) e = launch_batch_fusion(b, st);
    if (e == cudaSuccess && b->strided) {
        batch_advance_kernel<<<(b->n + 127) / 128, 128, 0, st>>>(b->d_desc, b->n);
        e = cudaGetLastError();
    }
    return e;
}

std::vector<int> shape_class(const gsdf_batch* b) {
    std::vector<int> k = b->n_px;
    std::sort(k.begin(), k.end());
    return k;
}

// Replay the cached graph `g` of `record` (which launches into the stream it is given), recording
// it again if the launch configuration changed.  When the caller's stream is itself being
// captured, the launches go straight into the caller's graph.
template <class F>
cudaError_t replay(gsdf_batch* b, gsdf_batch::Cached& g, int iters, F&& record) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(b->stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return record(b->stream);
    const bool same = g.exec && g.iters == iters && g.tiles == b->total_tiles && g.tile_px == b->tile_px &&
                      g.ctas == b->ctas_per_sm && g.tile_ptr == b->d_tile_scene && g.strided == b->strided &&
                      g.params_version == b->params_version;
    if (!same) {
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t le = record(b->capture_stream);
        e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return e;
        }
        g.iters = iters;
        g.tiles = b->total_tiles;
        g.tile_px = b->tile_px;
        g.ctas = b->ctas_per_sm;
        g.tile_ptr = b->d_tile_scene;
        g.strided = b->strided;
        g.params_version = b->params_version;
    }
    return cudaGraphLaunch(g.exec, b->stream);
}

}  // namespace

extern "C" {

gsdf_status gsdf_batch_create(gsdf_handle* const* handles, int32_t n, void* cuda_stream, gsdf_batch** out) {
    if (!out || !handles || n < 1 || n > 65536) return GSDF_ERR_INVALID_ARG;
    *out = nullptr;
    for (int s = 0; s < n; ++s)
        if (!handles[s] || handles[s]->cfg.tracker != GSDF_TRACKER_TAYLOR) return GSDF_ERR_INVALID_ARG;
    gsdf_batch* b = new (std::nothrow) gsdf_batch();
    if (!b) return GSDF_ERR_OOM;
    b->params = new (std::nothrow) BatchTrackParams();
    if (!b->params) {
        delete b;
        return GSDF_ERR_OOM;
    }
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->h.assign(handles, handles + n);
    b->n_px.assign(n, 0);
    std::vector<int> fp16;
    for (int s = 0; s < n; ++s)
        if (handles[s]->fp16) fp16.push_back(s);
    b->n_fp16 = (int)fp16.size();
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_desc, sizeof(SceneDesc) * (size_t)n);
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_desc, sizeof(SceneDesc) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(unsigned int) * kBatchCounters);
    if (e == cudaSuccess) e = cudaMemset(b->d_counters, 0, sizeof(unsigned int) * kBatchCounters);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_scratch_pose, sizeof(double) * 16 * (size_t)n);
    if (e == cudaSuccess && b->n_fp16 > 0) e = cudaMalloc(&b->d_fp16_scenes, sizeof(int) * fp16.size());
    if (e == cudaSuccess && b->n_fp16 > 0)
        e = cudaMemcpy(b->d_fp16_scenes, fp16.data(), sizeof(int) * fp16.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->desc_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        gsdf_status st = batch_status(e);
        free_batch(b);
        return st;
    }
    for (int s = 0; s < n; ++s) {
        SceneDesc& d = b->h_desc[s];
        memset(&d, 0, sizeof(d));
        const gsdf_handle* hh = handles[s];
        d.kind = !hh->hashed ? kSceneDense : (hh->fp16 ? kSceneHashed16 : kSceneHashed);
        b->kinds |= 1 << d.kind;
        d.dm = hh->dm;
        d.hm = hh->hm;
        d.hm16 = hh->hm16;
        d.prm = hh->prm;
        d.accum = hh->sc.accum;
        d.ticket = hh->sc.counter;
        d.err = hh->sc.err;
        d.n_blocks = hh->sc.n_blocks;
    }
    *out = b;
    return GSDF_OK;
}

gsdf_status gsdf_batch_destroy(gsdf_batch* b) {
    if (!b) return GSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    free_batch(b);
    return batch_status(e);
}

gsdf_status gsdf_batch_set_frames(gsdf_batch* b, const float* const* depth_dev, const gsdf_intrinsics* K,
                                  double* const* T_wc_dev, gsdf_track_stats* track_stats_dev,
                                  gsdf_integrate_stats* integrate_stats_dev) {
    if (!b || !depth_dev || !K || !T_wc_dev) return GSDF_ERR_INVALID_ARG;
    for (int s = 0; s < b->n; ++s)
        if (!depth_dev[s] || !T_wc_dev[s] || !intr_ok(K[s])) return GSDF_ERR_INVALID_ARG;
    cudaError_t e = wait_desc(b);  // the pinned table may still be in flight from the last call
    if (e != cudaSuccess) return batch_status(e);
    bool resized = !b->frames_set;
    for (int s = 0; s < b->n; ++s) {
        SceneDesc& d = b->h_desc[s];
        const int npx = K[s].width * K[s].height;
        resized = resized || npx != b->n_px[s];
        b->n_px[s] = npx;
        d.n_px = npx;
        d.K.fx = K[s].fx;
        d.K.fy = K[s].fy;
        d.K.cx = K[s].cx;
        d.K.cy = K[s].cy;
        d.K.width = K[s].width;
        d.K.height = K[s].height;
        d.K.depth_max = K[s].depth_max;
        d.K.ifx = (float)(1.0 / (double)K[s].fx);
        d.K.ify = (float)(1.0 / (double)K[s].fy);
        d.depth = depth_dev[s];
        d.pose = T_wc_dev[s];
        d.tstats = track_stats_dev ? track_stats_dev + s : nullptr;
        d.istats = integrate_stats_dev ? integrate_stats_dev + s : nullptr;
    }
    if (resized) {
        auto it = b->tuned.find(shape_class(b));
        if (it != b->tuned.end()) {
            b->tile_px = it->second.first;
            b->ctas_per_sm = it->second.second;
        } else {
            // untuned: 2048-px tiles, larger while the tiles would not fit the grid kernels' table
            b->tile_px = 2048;
            if (b->n <= kParamScenes) {
                auto tiles = [&](int px) {
                    long long t = 0;
                    for (int q = 0; q < b->n; ++q) t += (b->n_px[q] + px - 1) / px;
                    return t;
                };
                while (b->tile_px < 16384 && tiles(b->tile_px) > kParamTiles) b->tile_px *= 2;
            }
        }
        e = build_tiles(b);
        if (e != cudaSuccess) return batch_status(e);
    }
    b->frames_set = true;
    return batch_status(upload_desc(b));
}

gsdf_status gsdf_batch_set_depth_stride(gsdf_batch* b, const int64_t* stride) {
    if (!b || !stride || !b->frames_set) return GSDF_ERR_INVALID_ARG;
    cudaError_t e = wait_desc(b);
    if (e != cudaSuccess) return batch_status(e);
    bool any = false;
    for (int s = 0; s < b->n; ++s) {
        b->h_desc[s].depth_stride = (long long)stride[s];
        any = any || stride[s] != 0;
    }
    b->strided = any;
    return batch_status(upload_desc(b));
}

gsdf_status gsdf_batch_track_step(gsdf_batch* b) {
    if (!b || !b->frames_set) return GSDF_ERR_INVALID_ARG;
    return batch_status(launch_batch_track(b, b->stream));
}

gsdf_status gsdf_batch_track(gsdf_batch* b, int32_t n_iters) {
    if (!b || !b->frames_set || n_iters < 1 || n_iters > 1024) return GSDF_ERR_INVALID_ARG;
    return batch_status(replay(b, b->track_graph, n_iters, [&](cudaStream_t st) {
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < n_iters && e == cudaSuccess; ++it) e = launch_batch_track(b, st);
        return e;
    }));
}

gsdf_status gsdf_batch_integrate(gsdf_batch* b) {
    if (!b || !b->frames_set) return GSDF_ERR_INVALID_ARG;
    return batch_status(launch_batch_fusion(b, b->stream));
}

gsdf_status gsdf_batch_frame(gsdf_batch* b, int32_t n_iters) {
    if (!b || !b->frames_set || n_iters < 0 || n_iters > 1024) return GSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    if (b->strided) e = wait_desc(b);  // the host copy of the pointers is advanced below
    if (e == cudaSuccess)
        e = replay(b, b->frame_graph, n_iters, [&](cudaStream_t st) { return launch_batch_frame(b, n_iters, st); });
    if (e == cudaSuccess && b->strided)  // keep the host copy of the table in step with the device's
        for (int s = 0; s < b->n; ++s) b->h_desc[s].depth += b->h_desc[s].depth_stride;
    return batch_status(e);
}

gsdf_status gsdf_batch_autotune(gsdf_batch* b, int32_t* tile_px_out, int32_t* ctas_per_sm_out) {
    if (!b || !b->frames_set) return GSDF_ERR_INVALID_ARG;
    const std::vector<int> key = shape_class(b);
    auto it = b->tuned.find(key);
    if (it == b->tuned.end()) {
        cudaError_t e = wait_desc(b);
        if (e != cudaSuccess) return batch_status(e);
        // time one Gauss-Newton step of every scene per candidate, on scratch copies of the poses
        // and without statistics, so that the maps, poses and statistics are left untouched
        std::vector<SceneDesc> saved(b->h_desc, b->h_desc + b->n);
        for (int s = 0; s < b->n; ++s) {
            e = cudaMemcpyAsync(b->d_scratch_pose + 16 * s, saved[s].pose, sizeof(double) * 16,
                                cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return batch_status(e);
            b->h_desc[s].pose = b->d_scratch_pose + 16 * s;
            b->h_desc[s].tstats = nullptr;
        }
        const int tiles[] = {512, 1024, 2048, 4096, 8192, 16384};
        const int ctas[] = {1, 2};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_tile = b->tile_px, best_ctas = b->ctas_per_sm;
        for (int tp : tiles) {
            b->tile_px = tp;
            e = build_tiles(b);
            if (e == cudaSuccess) e = upload_desc(b);
            if (e == cudaSuccess) e = wait_desc(b);
            for (int c : ctas) {
                if (e != cudaSuccess) break;
                b->ctas_per_sm = c;
                e = launch_batch_track(b, b->stream);  // warm-up
                float ms_sum = 0.0f;
                for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
                    cudaEventRecord(e0, b->stream);
                    e = launch_batch_track(b, b->stream);
                    cudaEventRecord(e1, b->stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms_sum += ms;
                }
                if (e == cudaSuccess && ms_sum < best) {
                    best = ms_sum;
                    best_tile = tp;
                    best_ctas = c;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (int s = 0; s < b->n; ++s) b->h_desc[s] = saved[s];
        b->tile_px = best_tile;
        b->ctas_per_sm = best_ctas;
        cudaError_t e2 = build_tiles(b);
        if (e2 == cudaSuccess) e2 = upload_desc(b);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return batch_status(e);
        b->tuned[key] = {best_tile, best_ctas};
    } else {
        if (it->second.first != b->tile_px || it->second.second != b->ctas_per_sm) {
            cudaError_t e = wait_desc(b);
            b->tile_px = it->second.first;
            b->ctas_per_sm = it->second.second;
            if (e == cudaSuccess) e = build_tiles(b);
            if (e == cudaSuccess) e = upload_desc(b);
            if (e != cudaSuccess) return batch_status(e);
        }
    }
    if (tile_px_out) *tile_px_out = b->tile_px;
    if (ctas_per_sm_out) *ctas_per_sm_out = b->ctas_per_sm;
    return GSDF_OK;
}

}  // extern "C"
