"""ctypes wrapper of the C oracle (gsdf_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg import this module;
the product path never does.  `build()` compiles the C source with gcc
(-O2 -ffp-contract=off, no fast-math) into oracle/liboracle.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gsdf_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gsdf_oracle.h"))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int), ("height", C.c_int), ("depth_max", C.c_float)]


class Params(C.Structure):
    _fields_ = [("voxel_size", C.c_float), ("truncation", C.c_float), ("weight_eps", C.c_float),
                ("huber_delta", C.c_float), ("cos_max_angle", C.c_float), ("damping", C.c_double),
                ("tracker", C.c_int)]


class VoxelOut(C.Structure):
    _fields_ = [("m", C.c_int32 * 3), ("psi", C.c_double), ("g", C.c_double * 3), ("w", C.c_double)]


class TrackStats(C.Structure):
    _fields_ = [("H", C.c_double * 21), ("b", C.c_double * 6), ("energy", C.c_double),
                ("n_valid", C.c_int64), ("n_huber", C.c_int64), ("status", C.c_int),
                ("xi", C.c_double * 6)]


class IntegrateStats(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("n_visits", C.c_int64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.POINTER
        L.orc_map_new.restype = C.c_void_p
        L.orc_map_new.argtypes = [P(Params)]
        L.orc_map_new_dense.restype = C.c_void_p
        L.orc_map_new_dense.argtypes = [P(Params), P(C.c_int), P(C.c_int)]
        L.orc_map_free.argtypes = [C.c_void_p]
        L.orc_map_count.restype = C.c_size_t
        L.orc_map_count.argtypes = [C.c_void_p]
        L.orc_map_set_dense.argtypes = [C.c_void_p, P(C.c_float), P(C.c_float), P(C.c_float)]
        L.orc_integrate.argtypes = [C.c_void_p, P(C.c_float), P(Intrinsics), P(C.c_double), P(IntegrateStats)]
        L.orc_track_reduce.argtypes = [C.c_void_p, P(C.c_float), P(Intrinsics), P(C.c_double), P(TrackStats)]
        L.orc_track_step.argtypes = [C.c_void_p, P(C.c_float), P(Intrinsics), P(C.c_double), P(TrackStats)]
        L.orc_solve6.argtypes = [P(C.c_double), P(C.c_double), C.c_double, C.c_int64, P(C.c_double)]
        L.orc_se3_exp.argtypes = [P(C.c_double), P(C.c_double)]
        L.orc_taylor.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int32), P(C.c_double), P(C.c_double)]
        L.orc_trilinear.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int32), P(C.c_double), P(C.c_double)]
        L.orc_pixel_point.argtypes = [P(Intrinsics), P(C.c_double), C.c_int, C.c_int, C.c_float,
                                      P(C.c_float), P(C.c_int32), C.c_float]
        L.orc_normal.argtypes = [P(C.c_float), P(Intrinsics), P(Params), C.c_int, C.c_int, P(C.c_float)]
        L.orc_extract.restype = C.c_size_t
        L.orc_extract.argtypes = [C.c_void_p, P(VoxelOut), C.c_size_t]
        L.orc_block_of.argtypes = [P(C.c_int32), P(C.c_int32), P(C.c_int32)]
        L.orc_visibility.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double), C.c_float, C.c_int,
                                     P(Intrinsics), P(C.c_double), P(P(C.c_float)), P(C.c_uint8)]
        L.orc_energy.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double), C.c_float,
                                 C.c_int, P(Intrinsics), P(C.c_double), P(P(C.c_float)), P(P(C.c_float)),
                                 P(C.c_uint8), C.c_double, P(C.c_double), P(C.c_double), P(C.c_double),
                                 P(C.c_double), P(C.c_double), P(C.c_double)]
        L.orc_ba_step.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double), P(C.c_double), C.c_float,
                                  C.c_int, P(Intrinsics), P(C.c_double), P(P(C.c_float)), P(P(C.c_float)),
                                  P(C.c_uint8), C.c_double, C.c_double, C.c_int, P(TrackStats), P(C.c_double),
                                  P(C.c_double)]
        L.orc_marching_cubes.restype = C.c_size_t
        L.orc_marching_cubes.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), C.c_float, C.c_void_p, C.c_size_t]
        L.orc_points.restype = C.c_size_t
        L.orc_points.argtypes = [C.c_int64, P(C.c_int32), P(C.c_double), P(C.c_double), C.c_float, C.c_int,
                                 C.c_void_p, C.c_size_t]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def intrinsics(cam) -> Intrinsics:
    return Intrinsics(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.depth_max)


def params(voxel_size, truncation=None, weight_eps=None, huber_delta=None,
           cos_max_angle=0.25881904, damping=0.0, tracker=0) -> Params:
    """tracker 0: Eq. (taylor); 1: trilinear interpolation over the 8 voxels of the cell."""
    vs = float(voxel_size)
    return Params(vs, 5 * vs if truncation is None else truncation,
                  vs if weight_eps is None else weight_eps,
                  vs if huber_delta is None else huber_delta, cos_max_angle, damping, tracker)


def _pose(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, np.float64).reshape(16))


class OracleMap:
    """An oracle map (per-voxel hash map, FP64 values)."""

    def __init__(self, prm: Params, dense_dims=None, dense_origin=None):
        L = lib()
        self.prm = prm
        if dense_dims is None:
            self.h = L.orc_map_new(C.byref(prm))
        else:
            dims = (C.c_int * 3)(*dense_dims)
            org = (C.c_int * 3)(*dense_origin)
            self.h = L.orc_map_new_dense(C.byref(prm), dims, org)
        if not self.h:
            raise MemoryError("orc_map_new failed")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_map_free(self.h)
            self.h = None

    def set_dense(self, psi, g, w):
        psi = np.ascontiguousarray(psi, np.float32)
        g = np.ascontiguousarray(g, np.float32)
        w = np.ascontiguousarray(w, np.float32)
        if lib().orc_map_set_dense(self.h, _ptr(psi, C.c_float), _ptr(g, C.c_float), _ptr(w, C.c_float)):
            raise RuntimeError("orc_map_set_dense failed")

    def integrate(self, depth, cam, T_wc) -> IntegrateStats:
        d = np.ascontiguousarray(depth, np.float32)
        K = intrinsics(cam)
        st = IntegrateStats()
        if lib().orc_integrate(self.h, _ptr(d, C.c_float), C.byref(K), _ptr(_pose(T_wc), C.c_double), C.byref(st)):
            raise RuntimeError("orc_integrate failed")
        return st

    def track_reduce(self, depth, cam, T_wc) -> TrackStats:
        d = np.ascontiguousarray(depth, np.float32)
        K = intrinsics(cam)
        st = TrackStats()
        lib().orc_track_reduce(self.h, _ptr(d, C.c_float), C.byref(K), _ptr(_pose(T_wc), C.c_double), C.byref(st))
        return st

    def track_step(self, depth, cam, T_wc):
        """One Gauss-Newton step; returns (new pose, stats at the input pose)."""
        d = np.ascontiguousarray(depth, np.float32)
        K = intrinsics(cam)
        st = TrackStats()
        T = _pose(T_wc).copy()
        lib().orc_track_step(self.h, _ptr(d, C.c_float), C.byref(K), _ptr(T, C.c_double), C.byref(st))
        return T.reshape(4, 4), st

    def count(self) -> int:
        return int(lib().orc_map_count(self.h))

    def extract(self):
        """Voxels with W > 0 sorted by (x, y, z): dict of m (n,3) int32, psi, g (n,3), w (FP64)."""
        n = self.count()
        buf = (VoxelOut * max(n, 1))()
        k = lib().orc_extract(self.h, buf, n)
        assert k == n
        dt = np.dtype([("m", "<i4", 3), ("psi", "<f8"), ("g", "<f8", 3), ("w", "<f8")], align=True)
        assert dt.itemsize == C.sizeof(VoxelOut)
        raw = np.frombuffer(buf, dtype=dt, count=n)
        return {"m": raw["m"].copy(), "psi": raw["psi"].copy(), "g": raw["g"].copy(), "w": raw["w"].copy()}

    def taylor(self, P, m):
        """Eq. (taylor) residual and ghat at world point P using voxel m; None if unusable."""
        Pa = np.ascontiguousarray(P, np.float64)
        ma = np.ascontiguousarray(m, np.int32)
        r = C.c_double()
        gh = np.zeros(3)
        if lib().orc_taylor(self.h, _ptr(Pa, C.c_double), _ptr(ma, C.c_int32), C.byref(r), _ptr(gh, C.c_double)):
            return None
        return r.value, gh

    def trilinear(self, P, b):
        """Eqs. (dir_dist), (dir_grad): trilinear d and grad d at P over the cell with lowest corner
        voxel b; None unless all 8 corners are observed."""
        Pa = np.ascontiguousarray(P, np.float64)
        ba = np.ascontiguousarray(b, np.int32)
        d = C.c_double()
        gr = np.zeros(3)
        if lib().orc_trilinear(self.h, _ptr(Pa, C.c_double), _ptr(ba, C.c_int32), C.byref(d), _ptr(gr, C.c_double)):
            return None
        return d.value, gr


def stats_H(st: TrackStats) -> np.ndarray:
    """Full symmetric 6x6 from the 21 upper-triangle terms."""
    H = np.zeros((6, 6))
    k = 0
    for i in range(6):
        for j in range(i, 6):
            H[i, j] = H[j, i] = st.H[k]
            k += 1
    return H


def solve6(H21, b, damping=0.0, n_valid=1000):
    H21 = np.ascontiguousarray(H21, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    xi = np.zeros(6)
    bad = lib().orc_solve6(_ptr(H21, C.c_double), _ptr(b, C.c_double), damping, n_valid, _ptr(xi, C.c_double))
    return bad, xi


def se3_exp(xi) -> np.ndarray:
    xi = np.ascontiguousarray(xi, np.float64)
    T = np.zeros(16)
    lib().orc_se3_exp(_ptr(xi, C.c_double), _ptr(T, C.c_double))
    return T.reshape(4, 4)


def pixel_point(cam, T_wc, u, v, D, voxel_size):
    K = intrinsics(cam)
    P = np.zeros(3, np.float32)
    m = np.zeros(3, np.int32)
    lib().orc_pixel_point(C.byref(K), _ptr(_pose(T_wc), C.c_double), u, v, D, _ptr(P, C.c_float),
                          _ptr(m, C.c_int32), voxel_size)
    return P, m


def normal(depth, cam, prm: Params, u, v):
    d = np.ascontiguousarray(depth, np.float32)
    K = intrinsics(cam)
    n = np.zeros(3, np.float32)
    ok = lib().orc_normal(_ptr(d, C.c_float), C.byref(K), C.byref(prm), u, v, _ptr(n, C.c_float))
    return bool(ok), n


def block_of(m):
    ma = np.ascontiguousarray(m, np.int32)
    b = np.zeros(3, np.int32)
    loc = np.zeros(3, np.int32)
    lib().orc_block_of(_ptr(ma, C.c_int32), _ptr(b, C.c_int32), _ptr(loc, C.c_int32))
    return b, loc


def _frames_ptrs(frames):
    arrs = [np.ascontiguousarray(f, np.float32) for f in frames]
    ptrs = (C.POINTER(C.c_float) * len(arrs))(*[_ptr(a, C.c_float) for a in arrs])
    return arrs, ptrs


def visibility(m, psi, g, voxel_size, cam, poses, depths):
    """nu (F, n) uint8 of the photometric energy (surface voxel, inside with a 1 px margin, depth test)."""
    m = np.ascontiguousarray(m, np.int32)
    psi = np.ascontiguousarray(psi, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    n, F = len(psi), len(poses)
    P = np.ascontiguousarray(np.stack([np.asarray(T, np.float64).reshape(16) for T in poses]))
    keep, dptr = _frames_ptrs(depths)
    nu = np.zeros((F, n), np.uint8)
    K = intrinsics(cam)
    lib().orc_visibility(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), _ptr(g, C.c_double), voxel_size, F,
                         C.byref(K), _ptr(P, C.c_double), dptr, _ptr(nu, C.c_uint8))
    return nu


def energy(m, psi, g, rho, voxel_size, cam, poses, rgbs, depths, nu, lambda_geo, grad=True):
    """(E, E_p, E_g) and, if grad, (dpsi, dg (n,3), drho (n,3), dxi (F,6), dT (F,4,4)) of the voxel energy.

    dxi is the gradient for a left perturbation T <- exp(xi^) T, dT the gradient with respect to
    the entries of T = [R t] taken as free variables."""
    m = np.ascontiguousarray(m, np.int32)
    psi = np.ascontiguousarray(psi, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    nu = np.ascontiguousarray(nu, np.uint8)
    n, F = len(psi), len(poses)
    P = np.ascontiguousarray(np.stack([np.asarray(T, np.float64).reshape(16) for T in poses]))
    keep_r, rptr = _frames_ptrs(rgbs)
    keep_d, dptr = _frames_ptrs(depths)
    E = np.zeros(3)
    K = intrinsics(cam)
    if grad:
        dpsi, dg, drho, dxi = np.zeros(n), np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((F, 6))
        dT = np.zeros((F, 4, 4))
        gp = (_ptr(dpsi, C.c_double), _ptr(dg, C.c_double), _ptr(drho, C.c_double), _ptr(dxi, C.c_double),
              _ptr(dT, C.c_double))
    else:
        gp = (None, None, None, None, None)
    rc = lib().orc_energy(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), _ptr(g, C.c_double), _ptr(rho, C.c_double),
                          voxel_size, F, C.byref(K), _ptr(P, C.c_double), rptr, dptr, _ptr(nu, C.c_uint8),
                          lambda_geo, _ptr(E, C.c_double), *gp)
    if rc != 0:
        raise MemoryError("orc_energy failed")
    if grad:
        return E, dpsi, dg, drho, dxi, dT
    return E


POINT_DTYPE = np.dtype([("m", np.int32, 3), ("sub", np.int32), ("p", np.float64, 3), ("n", np.float64, 3)],
                       align=True)


def points(m, psi, g, voxel_size, level):
    """Oriented points of a voxel list (Sec. 4.3): level 0 the voxels' own points, level 1 the 2x2x2
    Taylor upsampling.  Structured array with fields m, sub, p, n."""
    m = np.ascontiguousarray(m, np.int32)
    psi = np.ascontiguousarray(psi, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    n = len(psi)
    cap = n * (8 if level else 1)
    out = np.zeros(max(cap, 1), POINT_DTYPE)
    k = lib().orc_points(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), _ptr(g, C.c_double), voxel_size, int(level),
                         out.ctypes.data, cap)
    return out[:k]


BA_POSES = 1
BA_PSI = 2


def ba_step(m, psi, g, voxel_size, cam, poses, rgbs, depths, nu, lambda_geo, damping, flags):
    """One photometric BA iteration (see orc_ba_step).  Returns (psi', rho, poses', stats, psi_H, psi_b):
    psi' and poses' after the updates selected by flags (BA_POSES | BA_PSI), rho the mean colours the
    step used, stats a list of per-keyframe TrackStats (H, b, energy, n_valid, status, xi)."""
    m = np.ascontiguousarray(m, np.int32)
    psi = np.array(psi, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    nu = np.ascontiguousarray(nu, np.uint8)
    n, F = len(psi), len(poses)
    P = np.ascontiguousarray(np.stack([np.asarray(T, np.float64).reshape(16) for T in poses]))
    keep_r, rptr = _frames_ptrs(rgbs)
    keep_d, dptr = _frames_ptrs(depths)
    rho = np.zeros((n, 3))
    hp, hb = np.zeros(n), np.zeros(n)
    st = (TrackStats * F)()
    K = intrinsics(cam)
    rc = lib().orc_ba_step(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), _ptr(g, C.c_double), _ptr(rho, C.c_double),
                           voxel_size, F, C.byref(K), _ptr(P, C.c_double), rptr, dptr, _ptr(nu, C.c_uint8),
                           lambda_geo, damping, int(flags), st, _ptr(hp, C.c_double), _ptr(hb, C.c_double))
    if rc != 0:
        raise MemoryError("orc_ba_step failed")
    return psi, rho, [P[i].reshape(4, 4).copy() for i in range(F)], list(st), hp, hb


TRIANGLE_DTYPE = np.dtype([("m", np.int32, 3), ("edges", np.int32), ("v", np.float64, 9)], align=True)


def marching_cubes(m, psi, voxel_size):
    """Layered marching cubes over a voxel list (every listed voxel counts as observed).
    Structured array (m, edges, v) of triangles."""
    m = np.ascontiguousarray(m, np.int32)
    psi = np.ascontiguousarray(psi, np.float64)
    n = len(psi)
    k = lib().orc_marching_cubes(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), voxel_size, None, 0)
    out = np.zeros(max(k, 1), TRIANGLE_DTYPE)
    k2 = lib().orc_marching_cubes(n, _ptr(m, C.c_int32), _ptr(psi, C.c_double), voxel_size, out.ctypes.data, k)
    assert k2 == k
    return out[:k]
