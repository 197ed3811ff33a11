// C ABI of libgsdf: handle management, argument checking, launches.  See include/gsdf.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "gsdf_internal.cuh"

using namespace gsdf;


namespace {

bool finite_pos(float x) { return isfinite(x) && x > 0.0f; }

gsdf_status check_config(const gsdf_config* c) {
    if (!c) return GSDF_ERR_INVALID_ARG;
    if (!finite_pos(c->voxel_size)) return GSDF_ERR_INVALID_ARG;
    if (!isfinite(c->truncation) || c->truncation < 0.5f * c->voxel_size) return GSDF_ERR_INVALID_ARG;
    if (!isfinite(c->weight_eps) || c->weight_eps < 0.0f || c->weight_eps >= c->truncation) return GSDF_ERR_INVALID_ARG;
    if (!finite_pos(c->huber_delta)) return GSDF_ERR_INVALID_ARG;
    if (!isfinite(c->cos_max_angle) || c->cos_max_angle < -1.0f || c->cos_max_angle > 1.0f) return GSDF_ERR_INVALID_ARG;
    if (!isfinite(c->damping) || c->damping < 0.0) return GSDF_ERR_INVALID_ARG;
    const double h = (double)(0.5f * c->voxel_size);
    const double kb = ceil((double)c->truncation / h - 1e-6);
    if (kb > 4096.0) return GSDF_ERR_INVALID_ARG;
    if (c->grid_kind == GSDF_GRID_DENSE) {
        long long n = 1;
        for (int i = 0; i < 3; ++i) {
            if (c->dense_dims[i] <= 0 || c->dense_dims[i] > (1 << 16)) return GSDF_ERR_INVALID_ARG;
            n *= c->dense_dims[i];
            const long long lo = c->dense_origin[i], hi = lo + c->dense_dims[i];
            if (lo < -(1ll << 23) || hi > (1ll << 23)) return GSDF_ERR_INVALID_ARG;
        }
        if (n > (1ll << 34)) return GSDF_ERR_INVALID_ARG;
    } else if (c->grid_kind == GSDF_GRID_HASHED) {
        const long long s = c->hash_slots;
        if (s < 1 || s > (1ll << 28) || (s & (s - 1)) != 0) return GSDF_ERR_INVALID_ARG;
        if (c->max_probe < 1 || (long long)c->max_probe > s) return GSDF_ERR_INVALID_ARG;
    } else {
        return GSDF_ERR_INVALID_ARG;
    }
    if (c->payload != GSDF_PAYLOAD_F32 && c->payload != GSDF_PAYLOAD_F16) return GSDF_ERR_INVALID_ARG;
    if (c->payload == GSDF_PAYLOAD_F16) {
        if (c->grid_kind != GSDF_GRID_HASHED) return GSDF_ERR_INVALID_ARG;
        const long long a = c->max_touched_blocks;
        if (a < 1 || a > c->hash_slots || (a & (a - 1)) != 0) return GSDF_ERR_INVALID_ARG;
    }
    if (c->tracker != GSDF_TRACKER_TAYLOR && c->tracker != GSDF_TRACKER_TRILINEAR) return GSDF_ERR_INVALID_ARG;
    if (c->tracker == GSDF_TRACKER_TRILINEAR && c->payload != GSDF_PAYLOAD_F32) return GSDF_ERR_INVALID_ARG;
    return GSDF_OK;
}

gsdf_status check_intr(const gsdf_intrinsics* K, Intr* out) {
    if (!K) return GSDF_ERR_INVALID_ARG;
    if (!finite_pos(K->fx) || !finite_pos(K->fy) || !isfinite(K->cx) || !isfinite(K->cy)) return GSDF_ERR_INVALID_ARG;
    if (K->width <= 0 || K->height <= 0 || K->width > 32768 || K->height > 32768) return GSDF_ERR_INVALID_ARG;
    if (!finite_pos(K->depth_max)) return GSDF_ERR_INVALID_ARG;
    out->fx = K->fx;
    out->fy = K->fy;
    out->cx = K->cx;
    out->cy = K->cy;
    out->width = K->width;
    out->height = K->height;
    out->depth_max = K->depth_max;
    out->ifx = (float)(1.0 / (double)K->fx);
    out->ify = (float)(1.0 / (double)K->fy);
    return GSDF_OK;
}

cudaError_t track_once(const gsdf_handle* h, const float* depth, const Intr& ki, double* T_wc, gsdf_track_stats* stats,
                       cudaStream_t st) {
    if (h->fp16) return launch_track16(h->hm16, depth, ki, h->prm, T_wc, stats, h->sc, h->num_sms, st);
    if (h->cfg.tracker == GSDF_TRACKER_TRILINEAR)
        return launch_track_trilinear(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, depth, ki, h->prm,
                                      T_wc, stats, h->sc, h->num_sms, st);
    return launch_track(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, depth, ki, h->prm, T_wc, stats,
                        h->sc, h->num_sms, st);
}

// n Gauss-Newton steps: one launch for a single step, otherwise the chained launches (each step's
// solve at the start of the next, then a final solve)
cudaError_t track_n(const gsdf_handle* h, const float* depth, const Intr& ki, double* T_wc, gsdf_track_stats* stats,
                    int n, cudaStream_t st) {
    if (n == 1) return track_once(h, depth, ki, T_wc, stats, st);
    return launch_track_chain(h->hashed || h->fp16 ? nullptr : &h->dm, h->hashed && !h->fp16 ? &h->hm : nullptr,
                              h->fp16 ? &h->hm16 : nullptr, !h->fp16 && h->cfg.tracker == GSDF_TRACKER_TRILINEAR,
                              depth, ki, h->prm, T_wc, stats, h->sc, h->num_sms, n, st);
}

gsdf_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return GSDF_OK;
    if (e == cudaErrorMemoryAllocation) return GSDF_ERR_OOM;
    return GSDF_ERR_CUDA;
}

void free_handle(gsdf_handle* h) {
    if (h->fp16) {
        cudaFree(h->hm16.H);
        cudaFree(h->hm16.W);
        cudaFree(h->hm16.scale);
        cudaFree(h->hm16.akeys);
        cudaFree(h->hm16.alist);
        cudaFree(h->hm16.acount);
        cudaFree(h->hm16.accA);
        cudaFree(h->hm16.accW);
    }
    if (h->track_exec) cudaGraphExecDestroy(h->track_exec);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    cudaFree(h->hm.keys);
    cudaFree(h->hashed ? (void*)h->hm.A : (void*)h->dm.A);
    cudaFree(h->hashed ? (void*)h->hm.W : (void*)h->dm.W);
    cudaFree(h->sc.accum);
    cudaFree(h->sc.chain);
    cudaFree(h->sc.counter);
    cudaFree(h->sc.err);
    cudaFree(h->sc.n_blocks);
    delete h;
}

}  // namespace

extern "C" {

gsdf_status gsdf_create(const gsdf_config* cfg, void* cuda_stream, gsdf_handle** out) {
    if (!out) return GSDF_ERR_INVALID_ARG;
    *out = nullptr;
    gsdf_status s = check_config(cfg);
    if (s != GSDF_OK) return s;
    gsdf_handle* h = new (std::nothrow) gsdf_handle();
    if (!h) return GSDF_ERR_OOM;
    h->cfg = *cfg;
    h->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
        delete h;
        return GSDF_ERR_CUDA;
    }
    h->hashed = cfg->grid_kind == GSDF_GRID_HASHED;
    h->prm = make_params(cfg->voxel_size, cfg->truncation, cfg->weight_eps, cfg->huber_delta, cfg->cos_max_angle,
                         cfg->damping);

    cudaError_t e = cudaSuccess;
    float4* A = nullptr;
    float* W = nullptr;
    if (h->hashed) {
        h->n_voxels = cfg->hash_slots * (long long)kBlockVoxels;
        e = cudaMalloc(&h->hm.keys, sizeof(unsigned long long) * (size_t)cfg->hash_slots);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->hm.keys, 0xFF, sizeof(unsigned long long) * (size_t)cfg->hash_slots, h->stream);
    } else {
        h->n_voxels = (long long)cfg->dense_dims[0] * cfg->dense_dims[1] * cfg->dense_dims[2];
    }
    h->fp16 = cfg->payload == GSDF_PAYLOAD_F16;
    if (h->fp16) {
        HashMap16& m = h->hm16;
        const size_t slots = (size_t)cfg->hash_slots, cap = (size_t)cfg->max_touched_blocks;
        m.amask = (unsigned int)cap - 1u;
        if (e == cudaSuccess) e = cudaMalloc(&m.H, sizeof(ushort4) * (size_t)h->n_voxels);
        if (e == cudaSuccess) e = cudaMalloc(&m.W, sizeof(float) * (size_t)h->n_voxels);
        if (e == cudaSuccess) e = cudaMalloc(&m.scale, sizeof(float) * slots);
        if (e == cudaSuccess) e = cudaMalloc(&m.akeys, sizeof(int) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&m.alist, sizeof(int2) * cap);
        if (e == cudaSuccess) e = cudaMalloc(&m.acount, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(m.acount, 0, sizeof(unsigned int), h->stream);
        if (e == cudaSuccess) e = cudaMalloc(&m.accA, sizeof(float4) * cap * kBlockVoxels);
        if (e == cudaSuccess) e = cudaMalloc(&m.accW, sizeof(float) * cap * kBlockVoxels);
        if (e == cudaSuccess) e = cudaMemsetAsync(m.H, 0, sizeof(ushort4) * (size_t)h->n_voxels, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m.W, 0, sizeof(float) * (size_t)h->n_voxels, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m.scale, 0, sizeof(float) * slots, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m.akeys, 0xFF, sizeof(int) * cap, h->stream);  // -1 = free
        if (e == cudaSuccess) e = cudaMemsetAsync(m.accA, 0, sizeof(float4) * cap * kBlockVoxels, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(m.accW, 0, sizeof(float) * cap * kBlockVoxels, h->stream);
    } else {
        if (e == cudaSuccess) e = cudaMalloc(&A, sizeof(float4) * (size_t)h->n_voxels);
        if (e == cudaSuccess) e = cudaMalloc(&W, sizeof(float) * (size_t)h->n_voxels);
    }
    if (h->hashed) {
        h->hm.A = A;
        h->hm.W = W;
        h->hm.mask = (unsigned long long)cfg->hash_slots - 1ull;
        h->hm.max_probe = cfg->max_probe;
        h->hm16.base = h->hm;
    } else {
        h->dm.A = A;
        h->dm.W = W;
        for (int i = 0; i < 3; ++i) {
            h->dm.dims[i] = cfg->dense_dims[i];
            h->dm.origin[i] = cfg->dense_origin[i];
        }
    }
    if (!h->fp16 && e == cudaSuccess) e = cudaMemsetAsync(A, 0, sizeof(float4) * (size_t)h->n_voxels, h->stream);
    if (!h->fp16 && e == cudaSuccess) e = cudaMemsetAsync(W, 0, sizeof(float) * (size_t)h->n_voxels, h->stream);
    h->sc.max_track_blocks = 2 * h->num_sms;
    if (e == cudaSuccess) e = cudaMalloc(&h->sc.accum, sizeof(unsigned long long) * kAccumWords);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.accum, 0, sizeof(unsigned long long) * kAccumWords, h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&h->sc.chain, sizeof(unsigned long long) * kChainWords);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.chain, 0, sizeof(unsigned long long) * kChainWords, h->stream);
    if (e == cudaSuccess) e = cudaMalloc(&h->sc.counter, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&h->sc.err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&h->sc.n_blocks, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.counter, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.err, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->sc.n_blocks, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_handle(h);
        return from_cuda(e);
    }
    *out = h;
    return GSDF_OK;
}

gsdf_status gsdf_destroy(gsdf_handle* h) {
    if (!h) return GSDF_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    free_handle(h);
    return from_cuda(e);
}

gsdf_status gsdf_set_stream(gsdf_handle* h, void* cuda_stream) {
    if (!h) return GSDF_ERR_INVALID_ARG;
    h->stream = (cudaStream_t)cuda_stream;
    return GSDF_OK;
}

gsdf_status gsdf_upload_dense(gsdf_handle* h, const float* psi, const float* g, const float* w) {
    if (!h || h->hashed || !psi || !g || !w) return GSDF_ERR_INVALID_ARG;
    const size_t n = (size_t)h->n_voxels;
    float4* A = (float4*)malloc(sizeof(float4) * n);
    if (!A) return GSDF_ERR_OOM;
    for (size_t i = 0; i < n; ++i) A[i] = make_float4(w[i] * psi[i], g[3 * i], g[3 * i + 1], g[3 * i + 2]);
    cudaError_t e = cudaMemcpyAsync(h->dm.A, A, sizeof(float4) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->dm.W, w, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    free(A);
    return from_cuda(e);
}

gsdf_status gsdf_integrate(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K,
                           const double* T_wc_dev, gsdf_integrate_stats* stats_dev) {
    if (!h || !depth_dev || !T_wc_dev) return GSDF_ERR_INVALID_ARG;
    Intr ki;
    gsdf_status s = check_intr(K, &ki);
    if (s != GSDF_OK) return s;
    if (h->fp16)
        return from_cuda(launch_integrate16(h->hm16, depth_dev, ki, h->prm, T_wc_dev, stats_dev, h->sc, h->num_sms,
                                            h->stream));
    return from_cuda(launch_integrate(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, depth_dev, ki,
                                      h->prm, T_wc_dev, stats_dev, h->sc, h->stream));
}

gsdf_status gsdf_track_step(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K,
                            double* T_wc_dev, gsdf_track_stats* stats_dev) {
    if (!h || !depth_dev || !T_wc_dev) return GSDF_ERR_INVALID_ARG;
    Intr ki;
    gsdf_status s = check_intr(K, &ki);
    if (s != GSDF_OK) return s;
    return from_cuda(track_once(h, depth_dev, ki, T_wc_dev, stats_dev, h->stream));
}

gsdf_status gsdf_track(gsdf_handle* h, const float* depth_dev, const gsdf_intrinsics* K, double* T_wc_dev,
                       int32_t n_iters, gsdf_track_stats* stats_dev) {
    if (!h || !depth_dev || !T_wc_dev || n_iters < 1 || n_iters > 1024) return GSDF_ERR_INVALID_ARG;
    Intr ki;
    gsdf_status s = check_intr(K, &ki);
    if (s != GSDF_OK) return s;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(h->stream, &cs);
    if (e != cudaSuccess) return from_cuda(e);
    if (cs != cudaStreamCaptureStatusNone)  // the caller is capturing: launch into its graph
        return from_cuda(track_n(h, depth_dev, ki, T_wc_dev, stats_dev, n_iters, h->stream));
    const bool same = h->track_exec && h->g_depth == depth_dev && h->g_pose == T_wc_dev && h->g_stats == stats_dev &&
                      h->g_iters == n_iters && memcmp(&h->g_K, K, sizeof(gsdf_intrinsics)) == 0;
    if (!same) {
        if (h->track_exec) {
            cudaGraphExecDestroy(h->track_exec);
            h->track_exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return from_cuda(e);
        const cudaError_t le = track_n(h, depth_dev, ki, T_wc_dev, stats_dev, n_iters, h->capture_stream);
        e = cudaStreamEndCapture(h->capture_stream, &graph);
        if (le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->track_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->track_exec = nullptr;
            return from_cuda(e);
        }
        h->g_depth = depth_dev;
        h->g_pose = T_wc_dev;
        h->g_stats = stats_dev;
        h->g_iters = n_iters;
        h->g_K = *K;
    }
    return from_cuda(cudaGraphLaunch(h->track_exec, h->stream));
}

gsdf_status gsdf_extract_voxels(gsdf_handle* h, gsdf_voxel* host_out, size_t capacity, size_t* count_out) {
    if (!h || !count_out || (capacity > 0 && !host_out)) return GSDF_ERR_INVALID_ARG;
    gsdf_voxel* dev = nullptr;
    long long n = 0;
    cudaError_t e = extract_voxels(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, h->fp16 ? &h->hm16 : nullptr,
                                   h->hashed ? h->cfg.hash_slots : 0, h->stream, h->num_sms, &dev, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    *count_out = (size_t)n;
    const size_t k = (size_t)n < capacity ? (size_t)n : capacity;
    if (k > 0) e = cudaMemcpyAsync(host_out, dev, sizeof(gsdf_voxel) * k, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dev);
    if (e != cudaSuccess) return from_cuda(e);
    return (size_t)n > capacity ? GSDF_ERR_CAPACITY : GSDF_OK;
}

gsdf_status gsdf_extract_points(gsdf_handle* h, int32_t level, gsdf_point* host_out, size_t capacity,
                                size_t* count_out) {
    if (!h || !count_out || (capacity > 0 && !host_out) || (level != 0 && level != 1)) return GSDF_ERR_INVALID_ARG;
    gsdf_point* dev = nullptr;
    long long n = 0;
    cudaError_t e = extract_points(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, h->fp16 ? &h->hm16 : nullptr,
                                   h->hashed ? h->cfg.hash_slots : 0, h->cfg.voxel_size, level, h->stream, h->num_sms,
                                   &dev, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    *count_out = (size_t)n;
    const size_t k = (size_t)n < capacity ? (size_t)n : capacity;
    if (k > 0) e = cudaMemcpyAsync(host_out, dev, sizeof(gsdf_point) * k, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dev);
    if (e != cudaSuccess) return from_cuda(e);
    return (size_t)n > capacity ? GSDF_ERR_CAPACITY : GSDF_OK;
}

gsdf_status gsdf_extract_mesh(gsdf_handle* h, gsdf_triangle* host_out, size_t capacity, size_t* count_out) {
    if (!h || !count_out || (capacity > 0 && !host_out)) return GSDF_ERR_INVALID_ARG;
    gsdf_triangle* dev = nullptr;
    long long n = 0;
    cudaError_t e = extract_mesh(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, h->fp16 ? &h->hm16 : nullptr,
                                 h->hashed ? h->cfg.hash_slots : 0, h->cfg.voxel_size, h->stream, h->num_sms, &dev, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    *count_out = (size_t)n;
    const size_t k = (size_t)n < capacity ? (size_t)n : capacity;
    if (k > 0) e = cudaMemcpyAsync(host_out, dev, sizeof(gsdf_triangle) * k, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dev);
    if (e != cudaSuccess) return from_cuda(e);
    return (size_t)n > capacity ? GSDF_ERR_CAPACITY : GSDF_OK;
}

gsdf_status gsdf_load_voxels(gsdf_handle* h, const gsdf_voxel* host_in, size_t n) {
    if (!h || (n > 0 && !host_in)) return GSDF_ERR_INVALID_ARG;
    for (size_t i = 0; i < n; ++i)
        if (!(host_in[i].w > 0.0f) || !isfinite(host_in[i].w) || !isfinite(host_in[i].psi)) return GSDF_ERR_INVALID_ARG;
    if (n == 0) return GSDF_OK;
    gsdf_voxel* dev = nullptr;
    cudaError_t e = cudaMalloc(&dev, sizeof(gsdf_voxel) * n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev, host_in, sizeof(gsdf_voxel) * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = load_voxels(h->hashed ? nullptr : &h->dm, h->hashed ? &h->hm : nullptr, h->fp16 ? &h->hm16 : nullptr,
                        h->prm.trunc, dev, (long long)n, h->sc.err, h->sc.n_blocks, h->stream, h->num_sms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
    }
    return gsdf_sync(h);
}

gsdf_status gsdf_num_blocks(gsdf_handle* h, int64_t* n_out) {
    if (!h || !n_out) return GSDF_ERR_INVALID_ARG;
    if (!h->hashed) {
        *n_out = (h->n_voxels + kBlockVoxels - 1) / kBlockVoxels;
        return GSDF_OK;
    }
    unsigned int n = 0;
    cudaError_t e = cudaMemcpyAsync(&n, h->sc.n_blocks, sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    *n_out = (int64_t)n;
    return from_cuda(e);
}

gsdf_status gsdf_sync(gsdf_handle* h) {
    if (!h) return GSDF_ERR_INVALID_ARG;
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, h->sc.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return from_cuda(e);
    if (err != 0) {
        e = cudaMemsetAsync(h->sc.err, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return from_cuda(e);
        return (gsdf_status)err;
    }
    return GSDF_OK;
}

const char* gsdf_status_string(gsdf_status s) {
    switch (s) {
        case GSDF_OK: return "ok";
        case GSDF_ERR_INVALID_ARG: return "invalid argument";
        case GSDF_ERR_CUDA: return "CUDA runtime error";
        case GSDF_ERR_OOM: return "out of device memory";
        case GSDF_ERR_CAPACITY: return "hash table capacity exhausted";
        case GSDF_ERR_DEGENERATE: return "degenerate tracking system";
        case GSDF_ERR_TIMEOUT: return "bounded device wait timed out";
        case GSDF_ERR_NO_VALID_PIXELS: return "no valid pixels";
    }
    return "unknown status";
}

}  // extern "C"
