"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU needed).

Each test ties one oracle function to something other than itself: numbers the paper prints,
closed forms (planes, spheres), library routines (scipy's matrix exponential, numpy's solver),
finite differences, or invariants.  A plausible mistake in the oracle (a dropped term, a wrong
sign or index, a transposed operand) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


# ----------------------------------------------------------------------------------------------
# numbers printed in the paper
# ----------------------------------------------------------------------------------------------


def test_block_boundary_fraction_matches_paper():
    """Sec. 3.1: in an 8^3 block, 57.8 % of voxels have a face neighbour in another block.
    Counted with the oracle's block decomposition, including a block at negative coordinates
    (floor division), so a truncating division or a wrong block size fails."""
    for base in [(0, 0, 0), (-8, 16, -24)]:
        n_boundary = 0
        for lz in range(8):
            for ly in range(8):
                for lx in range(8):
                    m = np.array([base[0] + lx, base[1] + ly, base[2] + lz], np.int32)
                    b, loc = O.block_of(m)
                    assert np.all(b * 8 + loc == m) and np.all((loc >= 0) & (loc < 8))
                    assert np.all(b == np.array(base) // 8)
                    out = False
                    for ax in range(3):
                        for s in (-1, 1):
                            nb = m.copy()
                            nb[ax] += s
                            out |= bool(np.any(O.block_of(nb)[0] != b))
                    n_boundary += out
        assert round(n_boundary / 512, 3) == GOLD["block_boundary_fraction"]["value"]


def test_memory_arithmetic_matches_paper():
    """Sec. 5.3: 512^3 dense volume, 2 values per SDF voxel, 5 per Gradient-SDF voxel
    (psi, g in R^3, W: the voxel payload this library stores)."""
    dense_vox = 512**3
    assert round(dense_vox / 1e8, 2) == GOLD["dense_volume_voxels"]["value"] / 1e8
    assert round(2 * dense_vox / 1e8, 2) == GOLD["dense_volume_floats"]["value"] / 1e8
    n = GOLD["hashed_voxels"]["value"]
    assert 2 * n == GOLD["sdf_baseline_floats"]["value"]
    values_per_voxel = 1 + 3 + 1  # psi, g, W
    assert values_per_voxel * n == GOLD["gradient_sdf_floats"]["value"]
    assert values_per_voxel / 2 == GOLD["per_voxel_ratio"]["value"]
    assert 2 * dense_vox / (values_per_voxel * n) > GOLD["memory_ratio_min"]["value"]


def test_angle_and_cutoff_constants():
    """Sec. 5.3: 75 degree normal filter (as FP32 cosine) and 3.5 m cutoff."""
    assert np.float32(math.cos(math.radians(GOLD["max_normal_angle_deg"]["value"]))) == np.float32(0.25881904)
    assert O.params(0.01).cos_max_angle == pytest.approx(0.25881904, abs=1e-8)
    assert I.KINECT_640.depth_max == GOLD["depth_cutoff_m"]["value"]
    assert O.params(0.02).truncation == pytest.approx(GOLD["truncation_voxels"]["value"] * 0.02)


# ----------------------------------------------------------------------------------------------
# SE(3) exponential and Cholesky solve against library routines
# ----------------------------------------------------------------------------------------------


def _twist(xi):
    w, u = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = u
    return M


@pytest.mark.parametrize("scale", [0.0, 1e-7, 1e-5, 1e-3, 0.1, 1.0, 2.5])
def test_se3_exp_matches_matrix_exponential(scale):
    rng = np.random.default_rng(int(scale * 1e6) + 3)
    for _ in range(5):
        xi = rng.normal(size=6)
        xi[:3] *= scale / max(np.linalg.norm(xi[:3]), 1e-300)
        T = O.se3_exp(xi)
        ref = scipy.linalg.expm(_twist(xi))
        assert np.allclose(T, ref, atol=1e-12, rtol=1e-12)
        R = T[:3, :3]
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(R) - 1) < 1e-13


def test_solve6_matches_numpy_and_flags_degenerate():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(40, 6))
    H = A.T @ A
    b = rng.normal(size=6)
    H21 = H[np.triu_indices(6)]
    bad, xi = O.solve6(H21, b)
    assert bad == 0
    assert np.allclose(xi, -np.linalg.solve(H, b), rtol=1e-10, atol=1e-12)
    # damping: (H + lambda I) with lambda = d * mean(diag H)
    d = 1e-2
    bad, xi = O.solve6(H21, b, damping=d)
    lam = d * np.trace(H) / 6
    assert np.allclose(xi, -np.linalg.solve(H + lam * np.eye(6), b), rtol=1e-10)
    # rank-deficient H -> degenerate, increment zero
    A2 = rng.normal(size=(40, 3)) @ rng.normal(size=(3, 6))
    bad, xi = O.solve6((A2.T @ A2)[np.triu_indices(6)], b)
    assert bad == 1 and np.all(xi == 0)
    # fewer than six residuals -> degenerate
    bad, _ = O.solve6(H21, b, n_valid=5)
    assert bad == 1


# ----------------------------------------------------------------------------------------------
# FP32 index path: back-projection, rounding, normals
# ----------------------------------------------------------------------------------------------


def test_pixel_point_and_half_up_rounding():
    """Eq. (taylor): j* by rounding P / v_s; ties (exact half-voxels) round up."""
    cam = I.Camera(100.0, 100.0, 8.0, 6.0, 16, 12)
    T = np.eye(4)
    # principal ray at depth 1.25 with v_s = 0.5: P = (0, 0, 1.25) -> 2.5 voxels -> tie -> 3
    P, m = O.pixel_point(cam, T, 8, 6, 1.25, 0.5)
    assert np.all(P == np.float32([0, 0, 1.25])) and list(m) == [0, 0, 3]
    # negative tie: x = -1.25 -> -2.5 voxels -> floor(-2.0) = -2
    T[:3, 3] = [-1.25, 0.0, 0.0]
    P, m = O.pixel_point(cam, T, 8, 6, 0.75, 0.5)
    assert P[0] == np.float32(-1.25) and list(m) == [-2, 0, 2]
    # off-axis pixel and a rotation about z by 90 degrees: camera x maps to world y
    T = np.eye(4)
    T[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    P, m = O.pixel_point(cam, T, 12, 6, 2.0, 0.01)  # camera point (0.08, 0, 2)
    assert np.allclose(P, [0.0, 0.08, 2.0], atol=1e-7) and list(m) == [0, 8, 200]


def _plane_depth(cam, n_cam, dist):
    """Exact z-depth image of the plane {x : n.x = dist} seen from the camera origin."""
    d = cam.ray_dirs_cam()
    return (dist / (d @ n_cam)).reshape(cam.height, cam.width)


def test_normals_of_planes_and_75_degree_filter():
    """Normals of a plane seen head-on and tilted; the 75 degree test of Sec. 5.3."""
    cam = I.Camera(140.0, 140.0, 80.0, 60.0, 160, 120)
    prm = O.params(0.02)
    depth = np.full((120, 160), 1.5, np.float32)
    ok, n = O.normal(depth, cam, prm, 40, 30)
    assert ok and np.all(n == np.float32([0, 0, 1]))  # exactly, oriented away from the camera
    for tilt_deg in [30.0, 60.0]:
        a = math.radians(tilt_deg)
        n_pl = np.array([math.sin(a), 0.0, math.cos(a)])
        depth = _plane_depth(cam, n_pl, 1.5).astype(np.float32)
        dirs = cam.ray_dirs_cam().reshape(120, 160, 3)
        for (u, v) in [(20, 20), (80, 60), (140, 100), (150, 10)]:
            ok, n = O.normal(depth, cam, prm, u, v)
            ray = dirs[v, u] / np.linalg.norm(dirs[v, u])
            ang = math.degrees(math.acos(abs(ray @ n_pl)))
            if ang < 74.9:
                assert ok
                assert np.allclose(n, n_pl, atol=2e-4)
            elif ang > 75.1:
                assert not ok
    # a steep plane seen at ~80 degrees everywhere is rejected
    a = math.radians(80)
    depth = _plane_depth(cam, np.array([0.0, math.sin(a), math.cos(a)]), 0.3).astype(np.float32)
    assert not O.normal(depth, cam, prm, 80, 60)[0]
    # border pixels, missing neighbours and depth jumps > T are rejected
    depth = np.full((120, 160), 1.5, np.float32)
    assert not O.normal(depth, cam, prm, 0, 60)[0]
    depth[60, 81] = 0.0
    assert not O.normal(depth, cam, prm, 80, 60)[0]
    depth[60, 81] = 1.5 + 0.11
    assert not O.normal(depth, cam, prm, 80, 60)[0]
    depth[60, 81] = 1.5 + 0.005  # small step: tilted normal, still within 75 degrees
    assert O.normal(depth, cam, prm, 80, 60)[0]


# ----------------------------------------------------------------------------------------------
# fusion: Eqs. (sdf_update), (gradient_update) against closed forms
# ----------------------------------------------------------------------------------------------


def _linear_weight(d, T, eps):
    return np.where(d <= eps, 1.0, (T - d) / (T - eps))


@pytest.fixture(scope="module")
def plane_fusion():
    cam = I.Camera(140.0, 140.0, 80.0, 60.0, 160, 120)
    vs = 0.02
    z0 = 1.0
    depth = np.full((120, 160), z0, np.float32)
    m = O.OracleMap(O.params(vs))
    st = m.integrate(depth, cam, np.eye(4))
    return cam, vs, z0, depth, m, st


def test_fusion_of_fronto_parallel_plane_is_exact(plane_fusion):
    """Noise-free fronto-parallel plane: d = z_v - D is the exact signed distance, so fused psi
    equals it, ghat is the plane normal, and every voxel's W is an integer number of rays times
    the linear weight w(d) (Bylow-style: 1 up to eps, linear to 0 at T)."""
    cam, vs, z0, depth, m, st = plane_fusion
    ex = m.extract()
    assert st.n_rays == (cam.width - 2) * (cam.height - 2)
    assert len(ex["m"]) > 1000
    T = 5 * vs
    psi_true = ex["m"][:, 2] * np.float64(np.float32(vs)) - z0
    assert np.max(np.abs(ex["psi"] - psi_true)) < 1e-6
    assert np.all(np.abs(ex["psi"]) <= T + 1e-6)
    g = ex["g"] / np.linalg.norm(ex["g"], axis=1, keepdims=True)
    assert np.max(np.abs(g - [0, 0, 1])) < 1e-6
    # the weight is a function of the FP32 distance estimate d = z_v - D (index path)
    d32 = (ex["m"][:, 2].astype(np.float32) * np.float32(vs)) - np.float32(z0)
    w1 = _linear_weight(d32.astype(np.float64), np.float64(np.float32(T)), np.float64(np.float32(vs)))
    rays = ex["w"] / w1
    assert np.max(np.abs(rays - np.round(rays))) < 1e-9 and np.min(np.round(rays)) >= 1
    # both sides of the surface are present and the band is truncated at +-T
    assert ex["psi"].min() < -0.7 * T and ex["psi"].max() > 0.7 * T
    # the z-layers present are exactly those with -T <= d < T in FP32 (d = T has w = 0)
    f = np.float32
    cand = np.arange(int((z0 - 2 * T) / vs), int((z0 + 2 * T) / vs) + 1)
    d_c = cand.astype(np.float32) * f(vs) - f(z0)
    expect = set(cand[(d_c >= -f(T)) & (d_c < f(T))])
    assert set(np.unique(ex["m"][:, 2])) == expect


def test_fusion_of_plane_from_rotated_camera():
    """Fronto-parallel plane seen from a general pose: psi(v) = z-component of R^T (v - t)
    minus the plane depth, and ghat is the plane normal in world coordinates, R e_z."""
    cam = I.Camera(140.0, 140.0, 80.0, 60.0, 160, 120)
    vs, z0 = 0.02, 1.3
    T = I.look_at([0.3, -0.4, 0.7], [1.1, 0.5, 1.9], roll=0.4)
    m = O.OracleMap(O.params(vs))
    m.integrate(np.full((120, 160), z0, np.float32), cam, T)
    ex = m.extract()
    assert len(ex["m"]) > 1000
    v = ex["m"] * np.float64(np.float32(vs))
    z_v = (v - T[:3, 3]) @ T[:3, :3][:, 2]
    assert np.max(np.abs(ex["psi"] - (z_v - z0))) < 2e-6
    g = ex["g"] / np.linalg.norm(ex["g"], axis=1, keepdims=True)
    assert np.max(np.abs(g - T[:3, :3][:, 2])) < 1e-6


def test_fusion_weighted_mean_invariant(plane_fusion):
    """Integrating the same frame N times leaves psi, ghat unchanged and scales W and g by N."""
    cam, vs, z0, depth, m1, _ = plane_fusion
    mN = O.OracleMap(O.params(vs))
    for _ in range(3):
        mN.integrate(depth, cam, np.eye(4))
    a, b = m1.extract(), mN.extract()
    assert np.array_equal(a["m"], b["m"])
    assert np.allclose(b["psi"], a["psi"], atol=1e-12)
    assert np.allclose(b["w"], 3 * a["w"], rtol=1e-12)
    assert np.allclose(b["g"], 3 * a["g"], rtol=1e-12, atol=1e-12)


def test_fusion_running_average_of_two_depths():
    """Two fronto-parallel frames at depths z1, z2: psi is the W-weighted average of the two
    distance estimates, i.e. Eq. (sdf_update) applied twice."""
    cam = I.Camera(140.0, 140.0, 80.0, 60.0, 160, 120)
    vs = 0.02
    T = 5 * vs
    z1, z2 = 1.0, 1.03
    m = O.OracleMap(O.params(vs))
    m.integrate(np.full((120, 160), z1, np.float32), cam, np.eye(4))
    a = m.extract()
    m2 = O.OracleMap(O.params(vs))
    m2.integrate(np.full((120, 160), z2, np.float32), cam, np.eye(4))
    b = m2.extract()
    m.integrate(np.full((120, 160), z2, np.float32), cam, np.eye(4))
    c = m.extract()
    ia = {tuple(k): i for i, k in enumerate(a["m"])}
    ib = {tuple(k): i for i, k in enumerate(b["m"])}
    n_checked = 0
    for i, k in enumerate(map(tuple, c["m"])):
        wa = a["w"][ia[k]] if k in ia else 0.0
        wb = b["w"][ib[k]] if k in ib else 0.0
        pa = a["psi"][ia[k]] if k in ia else 0.0
        pb = b["psi"][ib[k]] if k in ib else 0.0
        assert c["w"][i] == pytest.approx(wa + wb, rel=1e-12)
        assert c["psi"][i] == pytest.approx((wa * pa + wb * pb) / (wa + wb), abs=1e-12)
        n_checked += (wa > 0) and (wb > 0)
    assert n_checked > 1000
    # with both estimates present, psi is the plain weighted mean of z_v - z1 and z_v - z2
    zv = c["m"][:, 2] * np.float64(np.float32(vs))
    both = np.array([(tuple(k) in ia) and (tuple(k) in ib) for k in c["m"]])
    w1 = _linear_weight(zv - z1, T, vs)
    w2 = _linear_weight(zv - z2, T, vs)
    mean = (a_w := np.array([a["w"][ia[tuple(k)]] if tuple(k) in ia else 0 for k in c["m"]])) * (zv - z1)
    mean = (mean + np.array([b["w"][ib[tuple(k)]] if tuple(k) in ib else 0 for k in c["m"]]) * (zv - z2))
    mean /= c["w"]
    assert np.max(np.abs(c["psi"][both] - mean[both])) < 1e-6
    assert np.all(w1[both] > 0) and np.all(w2[both] > 0)


# ----------------------------------------------------------------------------------------------
# Taylor model and tracking
# ----------------------------------------------------------------------------------------------


def _planes_room(half=1.0, height=2.0):
    normals = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
    offsets = np.array([half, half, half, half, height, 0.0])
    return I.PlanesScene(normals, offsets)


def _dense_from_sdf(sdf, vs, lo, hi, T):
    """Dense grid arrays of an analytic SDF (inside-positive), W = 1 inside the band."""
    mlo = np.floor(np.asarray(lo) / vs).astype(int)
    mhi = np.ceil(np.asarray(hi) / vs).astype(int)
    dims = tuple(int(x) for x in (mhi - mlo + 1))
    mz, my, mx = np.meshgrid(*[np.arange(mlo[i], mhi[i] + 1) for i in (2, 1, 0)], indexing="ij")
    pts = np.stack([mx, my, mz], -1).astype(np.float64) * np.float64(np.float32(vs))
    psi, g = sdf(pts)
    w = (np.abs(psi) <= T).astype(np.float32)
    return dims, tuple(int(x) for x in mlo), psi.astype(np.float32), np.nan_to_num(g).astype(np.float32), w


@pytest.fixture(scope="module")
def planes_map():
    vs = 0.02
    T = 5 * vs
    room = _planes_room()
    dims, origin, psi, g, w = _dense_from_sdf(room.sdf, vs, (-1.2, -1.2, -0.2), (1.2, 1.2, 2.2), T)
    prm = O.params(vs)
    m = O.OracleMap(prm, dims, origin)
    m.set_dense(psi, g, w)
    return room, vs, m


def test_taylor_model_is_exact_on_planes(planes_map):
    """Eq. (taylor) on a planar SDF: psi_j* + (p - v_j*).ghat_j* equals the plane distance."""
    room, vs, m = planes_map
    rng = np.random.default_rng(11)
    n = 0
    for _ in range(300):
        P = rng.uniform([-0.95, -0.95, 0.05], [0.95, 0.95, 1.95])
        k = rng.integers(6)
        P = P - (room.normals[k] @ P - room.offsets[k] + rng.uniform(-0.06, 0.06)) * room.normals[k]
        mm = np.floor(P / np.float32(vs) + 0.5).astype(np.int32)
        psi_true, _ = room.sdf(P[None])
        _, g_v = room.sdf((mm * np.float64(np.float32(vs)))[None])
        out = m.taylor(P, mm)
        if out is None or not np.allclose(g_v[0], room.normals[k]):
            continue  # voxel off the band or on another face
        r, gh = out
        assert abs(r - psi_true[0]) < 1e-6  # FP32 storage of psi
        assert np.allclose(gh, room.normals[k], atol=1e-7)
        n += 1
    assert n > 100


def test_taylor_error_bound_on_sphere():
    """On a sphere with exact psi, g at the voxel, the Taylor residual deviates from the true
    distance by at most |p - v|^2 / (2 rho), rho the distance of the segment to the centre."""
    c = I.dense_sphere_case(1)
    m = O.OracleMap(O.params(c.voxel_size), c.dims, c.origin)
    m.set_dense(c.psi, c.grad, c.weight)
    rng = np.random.default_rng(3)
    vs = np.float64(np.float32(c.voxel_size))
    checked = 0
    for _ in range(500):
        P = I._unit(rng.normal(size=3)) * rng.uniform(0.33, 0.47)
        mm = np.floor(P / np.float32(c.voxel_size) + 0.5).astype(np.int32)
        out = m.taylor(P, mm)
        if out is None:
            continue
        r, gh = out
        v = mm * vs
        true = 0.4 - np.linalg.norm(P)
        rho = min(np.linalg.norm(P), np.linalg.norm(v)) - np.linalg.norm(P - v)
        bound = np.linalg.norm(P - v) ** 2 / (2 * rho) + 1e-6
        assert abs(r - true) <= bound
        checked += 1
    assert checked > 300


def _single_pixel_J(m, cam, T, depth, u, v, r0):
    """Per-pixel J recovered from the oracle's normal equations of a one-pixel image:
    b = w J r with w = 1 (|r| <= delta), r = r0 from Eq. (taylor); H must equal J J^T."""
    img = np.zeros_like(depth)
    img[v, u] = depth[v, u]
    st = m.track_reduce(img, cam, T)
    if st.n_valid != 1 or st.n_huber != 0 or abs(r0) < 1e-6:
        return None
    assert st.energy == pytest.approx(r0 * r0, rel=1e-12)
    J = np.array(st.b) / r0
    assert np.allclose(np.outer(J, J), O.stats_H(st), rtol=1e-9, atol=1e-12)
    return J


def test_jacobian_matches_finite_differences():
    """J = (P x ghat, ghat) of the oracle's reduction vs central differences of Eq. (taylor)
    under T <- expm(xi^) T (scipy), with the voxel j* held fixed."""
    c = I.dense_sphere_case(4)
    m = O.OracleMap(O.params(c.voxel_size), c.dims, c.origin)
    m.set_dense(c.psi, c.grad, c.weight)
    T = c.T_init
    rng = np.random.default_rng(9)
    ys, xs = np.nonzero(c.depth > 0)
    done = 0
    for i in rng.permutation(len(xs))[:200]:
        u, v = int(xs[i]), int(ys[i])
        P, mm = O.pixel_point(c.cam, T, u, v, c.depth[v, u], c.voxel_size)
        P = P.astype(np.float64)
        tay = m.taylor(P, mm)
        if tay is None:
            continue
        J = _single_pixel_J(m, c.cam, T, c.depth, u, v, tay[0])
        if J is None:
            continue
        h = 1e-6
        Jfd = np.zeros(6)
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Pp = (scipy.linalg.expm(_twist(e)) @ np.append(P, 1))[:3]
            Pm = (scipy.linalg.expm(_twist(-e)) @ np.append(P, 1))[:3]
            Jfd[k] = (m.taylor(Pp, mm)[0] - m.taylor(Pm, mm)[0]) / (2 * h)
        assert np.allclose(J, Jfd, atol=1e-7, rtol=1e-6)
        done += 1
        if done >= 20:
            break
    assert done >= 20


def test_huber_weight_of_large_residuals():
    """Tracking weight w_k (Huber, threshold delta): a one-pixel image whose residual exceeds
    delta contributes w r^2 = delta |r| to the energy and w J r = delta sign(r) J to b."""
    c = I.dense_sphere_case(4)
    delta = 0.004
    m = O.OracleMap(O.params(c.voxel_size, huber_delta=delta), c.dims, c.origin)
    m.set_dense(c.psi, c.grad, c.weight)
    T = c.T_init
    ys, xs = np.nonzero(c.depth > 0)
    n_big = 0
    for i in range(0, len(xs), 97):
        u, v = int(xs[i]), int(ys[i])
        P, mm = O.pixel_point(c.cam, T, u, v, c.depth[v, u], c.voxel_size)
        tay = m.taylor(P.astype(np.float64), mm)
        if tay is None:
            continue
        r0, gh = tay
        img = np.zeros_like(c.depth)
        img[v, u] = c.depth[v, u]
        st = m.track_reduce(img, c.cam, T)
        J = np.concatenate([np.cross(P.astype(np.float64), gh), gh])
        if abs(r0) > delta:
            n_big += 1
            assert st.n_huber == 1
            df = float(np.float32(delta))  # the threshold is an FP32 parameter
            assert st.energy == pytest.approx(df * abs(r0), rel=1e-12)
            assert np.allclose(st.b, df * np.sign(r0) * J, rtol=1e-9, atol=1e-14)
        else:
            assert st.n_huber == 0 and st.energy == pytest.approx(r0 * r0, rel=1e-12)
    assert n_big > 5


def test_sign_flip_leaves_normal_equations_unchanged():
    """A global sign flip of (psi, g) flips r and J together: H, b, E are unchanged."""
    c = I.dense_sphere_case(1)
    a = O.OracleMap(O.params(c.voxel_size), c.dims, c.origin)
    a.set_dense(c.psi, c.grad, c.weight)
    b = O.OracleMap(O.params(c.voxel_size), c.dims, c.origin)
    b.set_dense(-c.psi, -c.grad, c.weight)
    sa = a.track_reduce(c.depth, c.cam, c.T_init)
    sb = b.track_reduce(c.depth, c.cam, c.T_init)
    assert sa.n_valid == sb.n_valid > 5000
    assert np.allclose(sa.H, sb.H, rtol=1e-12)
    assert np.allclose(sa.b, sb.b, rtol=1e-10, atol=1e-12)
    assert sa.energy == pytest.approx(sb.energy, rel=1e-12)


def _edge_masked_depth(room, cam, T_gt, margin):
    """Ray-cast depth with pixels whose hit point lies within `margin` of another wall removed."""
    depth = I.render_depth(room, cam, T_gt).astype(np.float64)
    dirs = cam.ray_dirs_cam() @ T_gt[:3, :3].T
    pts = T_gt[:3, 3] + dirs * depth.reshape(-1, 1)
    dist = np.stack([off - pts @ n for n, off in zip(room.normals, room.offsets)], -1)
    second = np.sort(np.abs(dist), axis=1)[:, 1]
    depth = np.where(second.reshape(depth.shape) > margin, depth, 0.0)
    return depth.astype(np.float32)


def test_gauss_newton_recovers_pure_translation_in_one_step(planes_map):
    """Three visible planes, exact planar SDF, Taylor model exact: the linearised system is
    consistent with omega = 0, upsilon = -delta, so one step returns the true pose."""
    room, vs, m = planes_map
    cam = I.TINY_160
    T_gt = I.look_at([0.1, -0.2, 1.0], [0.9, 0.8, 0.3])
    depth = _edge_masked_depth(room, cam, T_gt, 0.08)
    assert (depth > 0).sum() > 5000
    T0 = T_gt.copy()
    T0[:3, 3] += [0.015, -0.01, 0.012]
    T1, st = m.track_step(depth, cam, T0)
    assert st.status == 0 and st.n_huber == 0
    assert np.abs(T1 - T_gt).max() < 2e-6


def test_gauss_newton_recovers_pose_on_planes(planes_map):
    """5 deg / 5 cm perturbation; Gauss-Newton on Eq. (tracking) converges to the true pose."""
    room, vs, m = planes_map
    cam = I.TINY_160
    rng = np.random.default_rng(21)
    T_gt = I.look_at([-0.1, 0.2, 1.1], [-0.9, -0.8, 0.4])
    depth = _edge_masked_depth(room, cam, T_gt, 0.12)
    T = I.perturb_pose(T_gt, rng, 5.0, 0.05)
    for _ in range(20):
        T, st = m.track_step(depth, cam, T)
    dR = T[:3, :3].T @ T_gt[:3, :3]
    ang = math.acos(min(1.0, (np.trace(dR) - 1) / 2))
    assert ang < 1e-5 and np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) < 1e-5


def test_sphere_tracking_recovers_observable_centre():
    """Dense sphere: only the camera-frame sphere centre R^T (c - t) is observable; damped
    Gauss-Newton brings it to the true value within the Taylor-model bias."""
    c = I.dense_sphere_case(1)
    prm = O.params(c.voxel_size, damping=1e-4)
    m = O.OracleMap(prm, c.dims, c.origin)
    m.set_dense(c.psi, c.grad, c.weight)
    T = c.T_init
    for _ in range(c.n_iters):
        T, st = m.track_step(c.depth, c.cam, T)
    cc_gt = c.T_gt[:3, :3].T @ (-c.T_gt[:3, 3])
    cc = T[:3, :3].T @ (-T[:3, 3])
    c0 = c.T_init[:3, :3].T @ (-c.T_init[:3, 3])
    assert np.linalg.norm(c0 - cc_gt) > 0.02
    assert np.linalg.norm(cc - cc_gt) < 5e-4


# ----------------------------------------------------------------------------------------------
# Sec. 5.2 (shape only): stored gradients beat central finite differences on noisy spheres
# ----------------------------------------------------------------------------------------------


@pytest.mark.slow
def test_stored_gradients_beat_central_differences():
    vs = 0.01
    T = 10 * vs
    cam = I.TINY_160
    sphere = I.SphereScene(np.array([0.0, 0.0, 0.0]), 0.3)
    rng = np.random.default_rng(17)
    m = O.OracleMap(O.params(vs, truncation=T))
    for i in range(24):
        d = I._unit(rng.normal(size=3))
        Tp = I.look_at(0.9 * d, np.zeros(3), roll=rng.uniform(-3, 3))
        depth = I.add_depth_noise(I.render_depth(sphere, cam, Tp), rng, k=0.004)
        m.integrate(depth, cam, Tp)
    ex = m.extract()
    key = {tuple(k): i for i, k in enumerate(ex["m"])}
    vsd = np.float64(np.float32(vs))
    err_ours, err_fd = [], []
    for i, k in enumerate(ex["m"]):
        p = k * vsd
        if abs(0.3 - np.linalg.norm(p)) > 10 * vs or ex["w"][i] < 5:
            continue
        gt = -p / np.linalg.norm(p)
        fd = np.zeros(3)
        ok = True
        for ax in range(3):
            kp, km = list(k), list(k)
            kp[ax] += 1
            km[ax] -= 1
            if tuple(kp) not in key or tuple(km) not in key:
                ok = False
                break
            fd[ax] = ex["psi"][key[tuple(kp)]] - ex["psi"][key[tuple(km)]]
        if not ok or np.linalg.norm(fd) == 0:
            continue
        g = ex["g"][i] / np.linalg.norm(ex["g"][i])
        err_ours.append(math.degrees(math.acos(np.clip(g @ gt, -1, 1))))
        err_fd.append(math.degrees(math.acos(np.clip(fd @ gt / np.linalg.norm(fd), -1, 1))))
    assert len(err_ours) > 1000
    assert np.mean(err_ours) < np.mean(err_fd)
