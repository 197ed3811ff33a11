"""Python binding of libgsdf (include/gsdf.h): argument marshalling only.

Every C entry point is exposed under its own name (gsdf_create, gsdf_integrate, ...); `Map` wraps
a handle for convenience.  PyTorch supplies device memory and streams: depth images, poses and
statistics are torch CUDA tensors whose data pointers are passed straight to the library.  All
computation runs in the library's CUDA kernels; if the library cannot be loaded this module
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GSDF_OK = 0
GSDF_ERR_INVALID_ARG = 1
GSDF_ERR_CUDA = 2
GSDF_ERR_OOM = 3
GSDF_ERR_CAPACITY = 4
GSDF_ERR_DEGENERATE = 5
GSDF_ERR_TIMEOUT = 6
GSDF_ERR_NO_VALID_PIXELS = 7
GSDF_GRID_DENSE = 0
GSDF_GRID_HASHED = 1
GSDF_PAYLOAD_F32 = 0
GSDF_PAYLOAD_F16 = 1
GSDF_TRACKER_TAYLOR = 0
GSDF_TRACKER_TRILINEAR = 1
GSDF_FOOTPRINT_TRACK = 0
GSDF_FOOTPRINT_FUSE = 1
GSDF_BA_POSES = 1
GSDF_BA_PSI = 2


class gsdf_intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("depth_max", C.c_float)]


class gsdf_config(C.Structure):
    _fields_ = [("grid_kind", C.c_int32), ("dense_dims", C.c_int32 * 3), ("dense_origin", C.c_int32 * 3),
                ("voxel_size", C.c_float), ("truncation", C.c_float), ("weight_eps", C.c_float),
                ("huber_delta", C.c_float), ("cos_max_angle", C.c_float), ("damping", C.c_double),
                ("hash_slots", C.c_int64), ("max_probe", C.c_int32), ("payload", C.c_int32),
                ("max_touched_blocks", C.c_int32), ("tracker", C.c_int32)]


class gsdf_track_stats(C.Structure):
    _fields_ = [("H", C.c_double * 21), ("b", C.c_double * 6), ("energy", C.c_double),
                ("n_valid", C.c_int64), ("n_huber", C.c_int64), ("status", C.c_int32), ("pad", C.c_int32),
                ("xi", C.c_double * 6)]


class gsdf_integrate_stats(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("n_visits", C.c_int64), ("n_blocks_new", C.c_int64),
                ("n_blocks_total", C.c_int64)]


class gsdf_voxel(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("psi", C.c_float), ("g", C.c_float * 3), ("w", C.c_float)]


VOXEL_DTYPE = np.dtype([("m", "<i4", 3), ("psi", "<f4"), ("g", "<f4", 3), ("w", "<f4")])


class gsdf_point(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("sub", C.c_int32), ("p", C.c_float * 3), ("n", C.c_float * 3)]


POINT_DTYPE = np.dtype([("m", "<i4", 3), ("sub", "<i4"), ("p", "<f4", 3), ("n", "<f4", 3)])


class gsdf_triangle(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("edges", C.c_int32), ("v", C.c_float * 9)]


TRIANGLE_DTYPE = np.dtype([("m", "<i4", 3), ("edges", "<i4"), ("v", "<f4", 9)])
TRACK_STATS_BYTES = C.sizeof(gsdf_track_stats)
INTEGRATE_STATS_BYTES = C.sizeof(gsdf_integrate_stats)

# every entry point declared in include/gsdf.h, with (restype, argtypes)
_P = C.POINTER
_SIGS = {
    "gsdf_create": (C.c_int, [_P(gsdf_config), C.c_void_p, _P(C.c_void_p)]),
    "gsdf_destroy": (C.c_int, [C.c_void_p]),
    "gsdf_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gsdf_upload_dense": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gsdf_integrate": (C.c_int, [C.c_void_p, C.c_void_p, _P(gsdf_intrinsics), C.c_void_p, C.c_void_p]),
    "gsdf_track_step": (C.c_int, [C.c_void_p, C.c_void_p, _P(gsdf_intrinsics), C.c_void_p, C.c_void_p]),
    "gsdf_track": (C.c_int, [C.c_void_p, C.c_void_p, _P(gsdf_intrinsics), C.c_void_p, C.c_int32, C.c_void_p]),
    "gsdf_extract_voxels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, _P(C.c_size_t)]),
    "gsdf_load_voxels": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "gsdf_num_blocks": (C.c_int, [C.c_void_p, _P(C.c_int64)]),
    "gsdf_extract_points": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t, _P(C.c_size_t)]),
    "gsdf_extract_mesh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, _P(C.c_size_t)]),
    "gsdf_sync": (C.c_int, [C.c_void_p]),
    "gsdf_status_string": (C.c_char_p, [C.c_int]),
    "gsdf_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, _P(C.c_void_p)]),
    "gsdf_batch_destroy": (C.c_int, [C.c_void_p]),
    "gsdf_batch_set_frames": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), _P(gsdf_intrinsics),
                                        C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]),
    "gsdf_batch_track_step": (C.c_int, [C.c_void_p]),
    "gsdf_batch_track": (C.c_int, [C.c_void_p, C.c_int32]),
    "gsdf_batch_integrate": (C.c_int, [C.c_void_p]),
    "gsdf_batch_autotune": (C.c_int, [C.c_void_p, _P(C.c_int32), _P(C.c_int32)]),
    "gsdf_batch_set_depth_stride": (C.c_int, [C.c_void_p, _P(C.c_int64)]),
    "gsdf_footprint": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, _P(gsdf_intrinsics), C.c_void_p, _P(C.c_int64)]),
    "gsdf_batch_frame": (C.c_int, [C.c_void_p, C.c_int32]),
    "gsdf_track_step_dense_noalloc": (C.c_int, [C.c_void_p, _P(gsdf_intrinsics), C.c_void_p, C.c_void_p,
                                                _P(C.c_int32), _P(C.c_int32), C.c_float, C.c_float, C.c_double,
                                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "gsdf_gn_update": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "gsdf_energy_create": (C.c_int, [C.c_int64, C.c_void_p, C.c_float, C.c_int32, _P(gsdf_intrinsics), C.c_void_p,
                                     C.c_void_p, C.c_void_p, _P(C.c_void_p)]),
    "gsdf_energy_destroy": (C.c_int, [C.c_void_p]),
    "gsdf_energy_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "gsdf_energy_visibility": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gsdf_energy_ba_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_double, C.c_double, C.c_int32, C.c_void_p]),
    "gsdf_energy_eval": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p]),
}

_lib = None


def load_library(path: str | None = None):
    """Load libgsdf.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if path is None:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgsdf not found at {path}")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GsdfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {load_library().gsdf_status_string(status).decode()} (status {status})")


def _check(status: int, where: str):
    if status != GSDF_OK:
        raise GsdfError(status, where)


# -------------------------------------------------------------------------------------------
# thin wrappers with the C names
# -------------------------------------------------------------------------------------------


def gsdf_create(cfg: gsdf_config, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load_library().gsdf_create(C.byref(cfg), C.c_void_p(stream), C.byref(h)), "gsdf_create")
    return h.value


def gsdf_destroy(h: int) -> int:
    return load_library().gsdf_destroy(C.c_void_p(h))


def gsdf_set_stream(h: int, stream: int) -> int:
    return load_library().gsdf_set_stream(C.c_void_p(h), C.c_void_p(stream))


def gsdf_upload_dense(h: int, psi: np.ndarray, g: np.ndarray, w: np.ndarray) -> int:
    psi = np.ascontiguousarray(psi, np.float32)
    g = np.ascontiguousarray(g, np.float32)
    w = np.ascontiguousarray(w, np.float32)
    return load_library().gsdf_upload_dense(C.c_void_p(h), psi.ctypes.data, g.ctypes.data, w.ctypes.data)


def gsdf_integrate(h: int, depth_ptr: int, K: gsdf_intrinsics, pose_ptr: int, stats_ptr: int = 0) -> int:
    return load_library().gsdf_integrate(C.c_void_p(h), C.c_void_p(depth_ptr), C.byref(K), C.c_void_p(pose_ptr),
                                         C.c_void_p(stats_ptr or None))


def gsdf_track_step(h: int, depth_ptr: int, K: gsdf_intrinsics, pose_ptr: int, stats_ptr: int = 0) -> int:
    return load_library().gsdf_track_step(C.c_void_p(h), C.c_void_p(depth_ptr), C.byref(K), C.c_void_p(pose_ptr),
                                          C.c_void_p(stats_ptr or None))


def gsdf_track(h: int, depth_ptr: int, K: gsdf_intrinsics, pose_ptr: int, n_iters: int, stats_ptr: int = 0) -> int:
    return load_library().gsdf_track(C.c_void_p(h), C.c_void_p(depth_ptr), C.byref(K), C.c_void_p(pose_ptr),
                                     n_iters, C.c_void_p(stats_ptr or None))


def gsdf_extract_voxels(h: int, out: np.ndarray | None, capacity: int):
    n = C.c_size_t()
    ptr = out.ctypes.data if out is not None else None
    st = load_library().gsdf_extract_voxels(C.c_void_p(h), C.c_void_p(ptr), capacity, C.byref(n))
    return st, n.value


def gsdf_extract_points(h: int, level: int, out: np.ndarray | None, capacity: int):
    n = C.c_size_t()
    ptr = out.ctypes.data if out is not None else None
    st = load_library().gsdf_extract_points(C.c_void_p(h), level, C.c_void_p(ptr), capacity, C.byref(n))
    return st, n.value


def gsdf_extract_mesh(h: int, out: np.ndarray | None, capacity: int):
    n = C.c_size_t()
    ptr = out.ctypes.data if out is not None else None
    st = load_library().gsdf_extract_mesh(C.c_void_p(h), C.c_void_p(ptr), capacity, C.byref(n))
    return st, n.value


def gsdf_load_voxels(h: int, vox: np.ndarray) -> int:
    vox = np.ascontiguousarray(vox, VOXEL_DTYPE)
    return load_library().gsdf_load_voxels(C.c_void_p(h), C.c_void_p(vox.ctypes.data), len(vox))


def gsdf_num_blocks(h: int) -> int:
    n = C.c_int64()
    _check(load_library().gsdf_num_blocks(C.c_void_p(h), C.byref(n)), "gsdf_num_blocks")
    return n.value


def gsdf_sync(h: int) -> int:
    return load_library().gsdf_sync(C.c_void_p(h))


def gsdf_track_step_dense_noalloc(depth_ptr: int, K: gsdf_intrinsics, A_ptr: int, W_ptr: int, dims, origin,
                                  voxel_size: float, huber_delta: float, damping: float, pose_ptr: int,
                                  stats_ptr: int = 0, stream: int = 0) -> int:
    """One tracking step on a caller-owned dense grid; allocates nothing (see include/gsdf.h)."""
    d = (C.c_int32 * 3)(*dims)
    o = (C.c_int32 * 3)(*origin)
    return load_library().gsdf_track_step_dense_noalloc(
        C.c_void_p(depth_ptr), C.byref(K), C.c_void_p(A_ptr), C.c_void_p(W_ptr), d, o, voxel_size, huber_delta,
        damping, C.c_void_p(pose_ptr), C.c_void_p(stats_ptr or None), C.c_void_p(stream or None))


def gsdf_gn_update(n: int, Hb_ptr: int, n_valid_ptr: int, damping: float, T_ptr: int, xi_ptr: int = 0,
                   status_ptr: int = 0, stream: int = 0) -> int:
    v = lambda x: C.c_void_p(x or None)  # noqa: E731
    return load_library().gsdf_gn_update(n, v(Hb_ptr), v(n_valid_ptr), damping, v(T_ptr), v(xi_ptr), v(status_ptr),
                                         v(stream))


def gn_update(Hb, n_valid, damping: float, T, xi=None, status=None, stream=None):
    """Damped Gauss-Newton updates T <- exp(xi^) T of n poses from given normal equations
    (gsdf_gn_update): Hb (n, 27) float64 (21 upper-triangle terms of H, then b), n_valid (n,)
    int64, T (n, 4, 4) float64 updated in place, optional outputs xi (n, 6) float64 and status
    (n,) int32; all contiguous CUDA tensors."""
    import torch

    n = int(Hb.shape[0])
    want = [("Hb", Hb, torch.float64, (n, 27)), ("n_valid", n_valid, torch.int64, (n,)),
            ("T", T, torch.float64, (n, 4, 4))]
    if xi is not None:
        want.append(("xi", xi, torch.float64, (n, 6)))
    if status is not None:
        want.append(("status", status, torch.int32, (n,)))
    for name, x, dt, shape in want:
        if not (x.is_cuda and x.dtype == dt and x.is_contiguous() and tuple(x.shape) == shape):
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of shape {shape}")
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(gsdf_gn_update(n, Hb.data_ptr(), n_valid.data_ptr(), damping, T.data_ptr(), _ptr(xi), _ptr(status),
                          s.cuda_stream), "gsdf_gn_update")


def gsdf_status_string(s: int) -> str:
    return load_library().gsdf_status_string(s).decode()


def gsdf_energy_create(n_voxels: int, m_ptr: int, voxel_size: float, n_frames: int, K: gsdf_intrinsics,
                       rgb_ptr: int, depth_ptr: int, stream: int = 0) -> int:
    e = C.c_void_p()
    _check(load_library().gsdf_energy_create(n_voxels, C.c_void_p(m_ptr or None), voxel_size, n_frames, C.byref(K),
                                             C.c_void_p(rgb_ptr), C.c_void_p(depth_ptr), C.c_void_p(stream or None),
                                             C.byref(e)), "gsdf_energy_create")
    return e.value


def gsdf_energy_destroy(e: int) -> int:
    return load_library().gsdf_energy_destroy(C.c_void_p(e))


def gsdf_energy_set_stream(e: int, stream: int) -> int:
    return load_library().gsdf_energy_set_stream(C.c_void_p(e), C.c_void_p(stream or None))


def gsdf_energy_visibility(e: int, psi_ptr: int, g_ptr: int, T_ptr: int, nu_ptr: int) -> int:
    return load_library().gsdf_energy_visibility(C.c_void_p(e), C.c_void_p(psi_ptr or None), C.c_void_p(g_ptr or None),
                                                 C.c_void_p(T_ptr), C.c_void_p(nu_ptr or None))


def gsdf_energy_ba_step(e: int, psi_ptr: int, g_ptr: int, rho_ptr: int, T_ptr: int, nu_ptr: int, lambda_geo: float,
                        damping: float, flags: int, stats_ptr: int = 0) -> int:
    v = lambda x: C.c_void_p(x or None)  # noqa: E731
    return load_library().gsdf_energy_ba_step(C.c_void_p(e), v(psi_ptr), v(g_ptr), v(rho_ptr), v(T_ptr), v(nu_ptr),
                                              lambda_geo, damping, flags, v(stats_ptr))


def gsdf_energy_eval(e: int, psi_ptr: int, g_ptr: int, rho_ptr: int, T_ptr: int, nu_ptr: int, lambda_geo: float,
                     grad_scale_ptr: int, E_ptr: int, dpsi_ptr: int = 0, dg_ptr: int = 0, drho_ptr: int = 0,
                     dT_ptr: int = 0, dxi_ptr: int = 0) -> int:
    v = lambda x: C.c_void_p(x or None)  # noqa: E731
    return load_library().gsdf_energy_eval(C.c_void_p(e), v(psi_ptr), v(g_ptr), v(rho_ptr), v(T_ptr), v(nu_ptr),
                                           lambda_geo, v(grad_scale_ptr), v(E_ptr), v(dpsi_ptr), v(dg_ptr),
                                           v(drho_ptr), v(dT_ptr), v(dxi_ptr))


# -------------------------------------------------------------------------------------------
# convenience
# -------------------------------------------------------------------------------------------


def intrinsics(cam) -> gsdf_intrinsics:
    return gsdf_intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.depth_max)


def make_config(voxel_size, *, dense_dims=None, dense_origin=(0, 0, 0), truncation=None, weight_eps=None,
                huber_delta=None, cos_max_angle=0.25881904, damping=0.0, hash_slots=1 << 16,
                max_probe=128, fp16=False, max_touched_blocks=None, tracker=0) -> gsdf_config:
    vs = float(voxel_size)
    c = gsdf_config()
    c.grid_kind = GSDF_GRID_HASHED if dense_dims is None else GSDF_GRID_DENSE
    if dense_dims is not None:
        c.dense_dims[:] = list(dense_dims)
        c.dense_origin[:] = list(dense_origin)
    c.voxel_size = vs
    c.truncation = 5 * vs if truncation is None else truncation
    c.weight_eps = vs if weight_eps is None else weight_eps
    c.huber_delta = vs if huber_delta is None else huber_delta
    c.cos_max_angle = cos_max_angle
    c.damping = damping
    c.hash_slots = hash_slots
    c.max_probe = max_probe
    c.payload = GSDF_PAYLOAD_F16 if fp16 else GSDF_PAYLOAD_F32
    c.max_touched_blocks = max(1, hash_slots // 4) if max_touched_blocks is None else max_touched_blocks  # power of 2
    c.tracker = tracker
    return c


def track_stats_from_bytes(buf) -> gsdf_track_stats:
    b = bytes(np.asarray(buf, np.uint8).tobytes())
    return gsdf_track_stats.from_buffer_copy(b[:TRACK_STATS_BYTES])


def integrate_stats_from_bytes(buf) -> gsdf_integrate_stats:
    b = bytes(np.asarray(buf, np.uint8).tobytes())
    return gsdf_integrate_stats.from_buffer_copy(b[:INTEGRATE_STATS_BYTES])


class Map:
    """A gsdf map on the current CUDA device, issuing work on a torch stream.

    Device buffers (depth, pose, statistics) are torch CUDA tensors owned by the caller."""

    def __init__(self, cfg: gsdf_config, stream=None):
        import torch

        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.cfg = cfg
        self.h = gsdf_create(cfg, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            gsdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_dense(self, psi, g, w):
        _check(gsdf_upload_dense(self.h, psi, g, w), "gsdf_upload_dense")

    def integrate(self, depth, K: gsdf_intrinsics, pose, stats=None):
        _check(gsdf_integrate(self.h, depth.data_ptr(), K, pose.data_ptr(), stats.data_ptr() if stats is not None else 0),
               "gsdf_integrate")

    def track_step(self, depth, K: gsdf_intrinsics, pose, stats=None):
        _check(gsdf_track_step(self.h, depth.data_ptr(), K, pose.data_ptr(), stats.data_ptr() if stats is not None else 0),
               "gsdf_track_step")

    def track(self, depth, K: gsdf_intrinsics, pose, n_iters: int, stats=None):
        """n_iters Gauss-Newton steps (replayed from a cached CUDA graph); stats: None or a
        device uint8 tensor of n_iters * TRACK_STATS_BYTES."""
        _check(gsdf_track(self.h, depth.data_ptr(), K, pose.data_ptr(), n_iters,
                          stats.data_ptr() if stats is not None else 0), "gsdf_track")

    def new_track_stats(self, n: int | None = None):
        if n is not None:
            return self.torch.zeros((n, TRACK_STATS_BYTES), dtype=self.torch.uint8, device="cuda")
        return self.torch.zeros(TRACK_STATS_BYTES, dtype=self.torch.uint8, device="cuda")

    def new_integrate_stats(self):
        return self.torch.zeros(INTEGRATE_STATS_BYTES, dtype=self.torch.uint8, device="cuda")

    def sync(self):
        _check(gsdf_sync(self.h), "gsdf_sync")

    def num_blocks(self) -> int:
        return gsdf_num_blocks(self.h)

    def extract(self) -> np.ndarray:
        """All voxels with W > 0 as a structured array (m, psi, g, w), in the library's order."""
        st, n = gsdf_extract_voxels(self.h, None, 0)
        if st not in (GSDF_OK, GSDF_ERR_CAPACITY):
            _check(st, "gsdf_extract_voxels")
        out = np.zeros(n, VOXEL_DTYPE)
        if n:
            st, n2 = gsdf_extract_voxels(self.h, out, n)
            _check(st, "gsdf_extract_voxels")
            assert n2 == n
        return out

    def extract_points(self, level: int = 0, capacity: int | None = None) -> np.ndarray:
        """Oriented surface points (m, sub, p, n) of the map, level 0 or 1 (2x2x2 upsampling).  With a
        capacity large enough the library runs once; otherwise it is asked for the count first."""
        if capacity is None:
            st, capacity = gsdf_extract_points(self.h, level, None, 0)
            if st not in (GSDF_OK, GSDF_ERR_CAPACITY):
                _check(st, "gsdf_extract_points")
        out = np.zeros(capacity, POINT_DTYPE)
        st, n = gsdf_extract_points(self.h, level, out, capacity)
        if st == GSDF_ERR_CAPACITY:
            return self.extract_points(level, n)
        _check(st, "gsdf_extract_points")
        return out[:n]

    def extract_mesh(self, capacity: int | None = None) -> np.ndarray:
        """Marching-cubes triangles (m, edges, v) of the map; one library call when capacity suffices."""
        if capacity is None:
            st, capacity = gsdf_extract_mesh(self.h, None, 0)
            if st not in (GSDF_OK, GSDF_ERR_CAPACITY):
                _check(st, "gsdf_extract_mesh")
        out = np.zeros(capacity, TRIANGLE_DTYPE)
        st, n = gsdf_extract_mesh(self.h, out, capacity)
        if st == GSDF_ERR_CAPACITY:
            return self.extract_mesh(n)
        _check(st, "gsdf_extract_mesh")
        return out[:n]

    def footprint(self, what: int, depth, K: gsdf_intrinsics, pose):
        """(distinct voxels, distinct blocks) one tracking step (GSDF_FOOTPRINT_TRACK) or one fusion
        (GSDF_FOOTPRINT_FUSE, after fusing that frame at that pose) touches (gsdf_footprint)."""
        out = (C.c_int64 * 2)()
        _check(load_library().gsdf_footprint(C.c_void_p(self.h), what, C.c_void_p(depth.data_ptr()), C.byref(K),
                                              C.c_void_p(pose.data_ptr()), out), "gsdf_footprint")
        return int(out[0]), int(out[1])

    def load(self, vox: np.ndarray):
        _check(gsdf_load_voxels(self.h, vox), "gsdf_load_voxels")


class Batch:
    """Many scenes (Map objects) tracked and fused together in persistent launches."""

    def __init__(self, maps, stream=None):
        import torch

        self.torch = torch
        self.maps = list(maps)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (C.c_void_p * len(self.maps))(*[m.h for m in self.maps])
        h = C.c_void_p()
        _check(load_library().gsdf_batch_create(arr, len(self.maps), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "gsdf_batch_create")
        self.b = h.value

    def close(self):
        if getattr(self, "b", None):
            load_library().gsdf_batch_destroy(C.c_void_p(self.b))
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_frames(self, depths, Ks, poses, track_stats=None, integrate_stats=None):
        n = len(self.maps)
        d = (C.c_void_p * n)(*[x.data_ptr() for x in depths])
        p = (C.c_void_p * n)(*[x.data_ptr() for x in poses])
        k = (gsdf_intrinsics * n)(*Ks)
        _check(load_library().gsdf_batch_set_frames(
            C.c_void_p(self.b), d, k, p,
            C.c_void_p(track_stats.data_ptr() if track_stats is not None else None),
            C.c_void_p(integrate_stats.data_ptr() if integrate_stats is not None else None)), "gsdf_batch_set_frames")

    def track_step(self):
        _check(load_library().gsdf_batch_track_step(C.c_void_p(self.b)), "gsdf_batch_track_step")

    def track(self, n_iters: int):
        _check(load_library().gsdf_batch_track(C.c_void_p(self.b), n_iters), "gsdf_batch_track")

    def integrate(self):
        _check(load_library().gsdf_batch_integrate(C.c_void_p(self.b)), "gsdf_batch_integrate")

    def set_depth_stride(self, strides):
        """Per-scene depth strides in floats (gsdf_batch_set_depth_stride)."""
        arr = (C.c_int64 * len(self.maps))(*[int(x) for x in strides])
        _check(load_library().gsdf_batch_set_depth_stride(C.c_void_p(self.b), arr), "gsdf_batch_set_depth_stride")

    def frame(self, n_iters: int):
        """One frame of every scene: n_iters Gauss-Newton steps, fusion, depth advance (one graph)."""
        _check(load_library().gsdf_batch_frame(C.c_void_p(self.b), n_iters), "gsdf_batch_frame")

    def autotune(self):
        t, c = C.c_int32(), C.c_int32()
        _check(load_library().gsdf_batch_autotune(C.c_void_p(self.b), C.byref(t), C.byref(c)), "gsdf_batch_autotune")
        return t.value, c.value


def _ptr(t) -> int:
    return t.data_ptr() if t is not None and t.numel() > 0 else 0


class Energy:
    """The photometric + geometric voxel energy over a fixed voxel list and keyframe set (see
    include/gsdf.h, gsdf_energy_*).  Tensors are CUDA tensors: m (n, 3) int32, rgb (F, H, W, 3)
    float32, depth (F, H, W) float32; later calls take psi (n,) and g, rho (n, 3) float32 and
    poses (F, 4, 4) float64 (camera -> world)."""

    def __init__(self, m, voxel_size: float, K: gsdf_intrinsics, rgb, depth, stream=None):
        import torch

        self.torch = torch
        self.n = int(m.shape[0])
        self.F = int(rgb.shape[0])
        for name, t, dt in (("m", m, torch.int32), ("rgb", rgb, torch.float32), ("depth", depth, torch.float32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor")
        if tuple(rgb.shape) != (self.F, K.height, K.width, 3) or tuple(depth.shape) != (self.F, K.height, K.width):
            raise ValueError("rgb / depth shapes do not match the intrinsics")
        self.K = K
        st = stream if stream is not None else torch.cuda.current_stream()
        self.e = gsdf_energy_create(self.n, _ptr(m), voxel_size, self.F, K, rgb.data_ptr(), depth.data_ptr(),
                                    st.cuda_stream)

    def close(self):
        if getattr(self, "e", None):
            gsdf_energy_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        _check(gsdf_energy_set_stream(self.e, self.torch.cuda.current_stream().cuda_stream), "gsdf_energy_set_stream")

    def visibility(self, psi, g, poses):
        """nu (n, ceil(F / 32)) int32 on the device: bit i mod 32 of word i // 32 of voxel j is nu_ij."""
        self._stream()
        nu = self.torch.empty((self.n, (self.F + 31) // 32), dtype=self.torch.int32, device=poses.device)
        _check(gsdf_energy_visibility(self.e, _ptr(psi), _ptr(g), poses.data_ptr(), _ptr(nu)), "gsdf_energy_visibility")
        return nu

    def eval(self, psi, g, rho, poses, nu, lambda_geo: float, grad: bool = True, grad_scale=None):
        """E (3,) float64 = (E, E_p, E_g); with grad also dpsi, dg, drho (float32), dT (F, 4, 4) and
        dxi (F, 6) (float64)."""
        torch = self.torch
        self._stream()
        dev = poses.device
        E = torch.empty(3, dtype=torch.float64, device=dev)
        if not grad:
            _check(gsdf_energy_eval(self.e, _ptr(psi), _ptr(g), _ptr(rho), poses.data_ptr(), _ptr(nu), lambda_geo,
                                    _ptr(grad_scale), E.data_ptr()), "gsdf_energy_eval")
            return E
        dpsi = torch.empty((self.n,), dtype=torch.float32, device=dev)
        dg = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        drho = torch.empty((self.n, 3), dtype=torch.float32, device=dev)
        dT = torch.empty((self.F, 4, 4), dtype=torch.float64, device=dev)
        dxi = torch.empty((self.F, 6), dtype=torch.float64, device=dev)
        _check(gsdf_energy_eval(self.e, _ptr(psi), _ptr(g), _ptr(rho), poses.data_ptr(), _ptr(nu), lambda_geo,
                                _ptr(grad_scale), E.data_ptr(), _ptr(dpsi), _ptr(dg), _ptr(drho), dT.data_ptr(),
                                dxi.data_ptr()), "gsdf_energy_eval")
        return E, dpsi, dg, drho, dT, dxi


def _energy_ba_step(self, psi, g, rho, poses, nu, lambda_geo: float, damping: float, flags: int, stats=None):
    """One photometric bundle-adjustment iteration (gsdf_energy_ba_step): psi (n,) float32 and poses
    (F, 4, 4) float64 are updated in place as flags select; rho (n, 3) float32 receives the mean
    colours; stats: None or a (F, TRACK_STATS_BYTES) uint8 CUDA tensor."""
    self._stream()
    _check(gsdf_energy_ba_step(self.e, _ptr(psi), _ptr(g), _ptr(rho), poses.data_ptr(), _ptr(nu), lambda_geo,
                               damping, flags, _ptr(stats)), "gsdf_energy_ba_step")


Energy.ba_step = _energy_ba_step


def _voxel_energy_function():
    import torch

    class VoxelEnergy(torch.autograd.Function):
        """E(psi, g, rho, poses) as a differentiable scalar.  The forward pass evaluates the energy
        only; the backward pass re-runs the kernels with gradients (every per-pixel lookup is
        recomputed, nothing per pixel is kept), scaled on the device by the incoming gradient."""

        @staticmethod
        def forward(ctx, psi, g, rho, poses, energy, nu, lambda_geo):
            ctx.energy, ctx.nu, ctx.lambda_geo = energy, nu, float(lambda_geo)
            ctx.save_for_backward(psi, g, rho, poses)
            return energy.eval(psi, g, rho, poses, nu, ctx.lambda_geo, grad=False)[0]

        @staticmethod
        def backward(ctx, gE):
            psi, g, rho, poses = ctx.saved_tensors
            gE = gE.to(torch.float64).contiguous()
            _, dpsi, dg, drho, dT, _ = ctx.energy.eval(psi, g, rho, poses, ctx.nu, ctx.lambda_geo, grad=True,
                                                       grad_scale=gE)
            return dpsi, dg, drho, dT, None, None, None

    return VoxelEnergy


_VoxelEnergy = None


def voxel_energy(psi, g, rho, poses, energy: Energy, nu, lambda_geo: float):
    """Differentiable E = E_p + lambda E_g (torch.autograd.Function around gsdf_energy_eval).
    The gradient of poses is dE/dT for the entries of each 4 x 4 matrix (last row 0)."""
    global _VoxelEnergy
    if _VoxelEnergy is None:
        _VoxelEnergy = _voxel_energy_function()
    return _VoxelEnergy.apply(psi, g, rho, poses, energy, nu, lambda_geo)
