"""Pins of the oracle's direct SDF tracker baseline: trilinear interpolation of psi over the 8
voxels of a cell, Eqs. (dir_dist) and (dir_grad) (the paper's hash-map SDF tracker, Sec. 6).

* Trilinear interpolation reproduces every function in span{1, x, y, z, xy, yz, xz, xyz} exactly,
  so on such a field d(P) and grad d(P) equal the field's value and analytic gradient (up to the
  FP32 storage of the corner values).
* The reduction's Jacobian (P x grad d, grad d) against central differences of d under the left
  perturbation expm(xi^) (scipy), the cell held fixed.
* On exact planar SDFs (affine in the band) one Gauss-Newton step recovers a pure translation and
  20 steps recover a 5 deg / 5 cm perturbation, as for the Taylor model.
* A cell with an unobserved corner is unusable.
* The cell is the one containing P (lowest corner floor(P / v_s)): on a curved field (a sphere,
  where extrapolating from another cell gives another value) the reduction's residual equals the
  interpolant over that cell, and its error against the true distance stays within the
  interpolation bound.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I
from test_oracle_pins import _dense_from_sdf, _edge_masked_depth, _planes_room, _twist

VS = 0.02


def _cubic_field(x):
    """psi in span{1, x, y, z, xy, yz, xz, xyz} and its gradient (x: (..., 3), metres)."""
    c = np.array([0.2, -0.3, 0.25])
    x0, y0, z0 = 0.013, -0.021, 0.007
    X, Y, Z = x[..., 0] - x0, x[..., 1] - y0, x[..., 2] - z0
    psi = 0.01 + x @ c + 0.6 * X * Y - 0.4 * Y * Z + 0.3 * X * Z + 1.5 * X * Y * Z
    gx = c[0] + 0.6 * Y + 0.3 * Z + 1.5 * Y * Z
    gy = c[1] + 0.6 * X - 0.4 * Z + 1.5 * X * Z
    gz = c[2] - 0.4 * Y + 0.3 * X + 1.5 * X * Y
    return psi, np.stack([gx, gy, gz], -1)


@pytest.fixture(scope="module")
def cubic_map():
    dims, origin = (24, 24, 24), (-12, -12, -12)
    r = [np.arange(origin[i], origin[i] + dims[i]) for i in range(3)]
    mz, my, mx = np.meshgrid(r[2], r[1], r[0], indexing="ij")
    v = np.stack([mx, my, mz], -1).astype(np.float64) * np.float64(np.float32(VS))
    psi, g = _cubic_field(v)
    m = O.OracleMap(O.params(VS, tracker=1), dims, origin)
    m.set_dense(psi.astype(np.float32), g.astype(np.float32), np.ones(psi.shape, np.float32))
    return m


def test_trilinear_is_exact_on_its_function_space(cubic_map):
    rng = np.random.default_rng(5)
    vs = np.float64(np.float32(VS))
    for _ in range(300):
        P = rng.uniform(-0.2, 0.2, size=3)
        b = np.floor(P / vs).astype(np.int32)
        d, gr = cubic_map.trilinear(P, b)
        psi, g = _cubic_field(P)
        assert d == pytest.approx(psi, abs=2e-7)  # corner values stored in FP32
        assert np.allclose(gr, g, atol=5e-6)
    # at a grid node the interpolant is the node's value
    b = np.array([3, -4, 5], np.int32)
    d, _ = cubic_map.trilinear(b * vs, b)
    assert d == pytest.approx(float(np.float32(_cubic_field(b * vs)[0])), abs=1e-12)


def test_unobserved_corner_makes_the_cell_unusable():
    dims, origin = (4, 4, 4), (0, 0, 0)
    w = np.ones((4, 4, 4), np.float32)
    w[1, 1, 1] = 0.0  # voxel (1, 1, 1) (z, y, x order)
    m = O.OracleMap(O.params(VS, tracker=1), dims, origin)
    m.set_dense(np.zeros((4, 4, 4), np.float32), np.tile([0, 0, 1.0], (4, 4, 4, 1)).astype(np.float32), w)
    vs = np.float64(np.float32(VS))
    assert m.trilinear(np.array([1.5, 1.5, 1.5]) * vs, np.array([1, 1, 1], np.int32)) is None
    assert m.trilinear(np.array([0.5, 0.5, 0.5]) * vs, np.array([0, 0, 0], np.int32)) is None
    assert m.trilinear(np.array([2.5, 2.5, 2.5]) * vs, np.array([2, 2, 2], np.int32)) is not None


@pytest.fixture(scope="module")
def planes_tri():
    T = 5 * VS
    room = _planes_room()
    dims, origin, psi, g, w = _dense_from_sdf(room.sdf, VS, (-1.2, -1.2, -0.2), (1.2, 1.2, 2.2), T)
    m = O.OracleMap(O.params(VS, tracker=1), dims, origin)
    m.set_dense(psi, g, w)
    return room, m


def test_jacobian_matches_finite_differences(planes_tri):
    room, m = planes_tri
    cam = I.TINY_160
    T_gt = I.look_at([0.1, -0.2, 1.0], [0.9, 0.8, 0.3])
    depth = _edge_masked_depth(room, cam, T_gt, 0.12)
    T = T_gt.copy()
    T[:3, 3] += [0.006, -0.004, 0.005]  # away from the true pose, so residuals are not zero
    ys, xs = np.nonzero(depth > 0)
    rng = np.random.default_rng(2)
    inv_vs = np.float32(1.0 / np.float64(np.float32(VS)))
    done = 0
    for i in rng.permutation(len(xs))[:400]:
        u, v = int(xs[i]), int(ys[i])
        P, _ = O.pixel_point(cam, T, u, v, depth[v, u], VS)
        b = np.floor(P * inv_vs).astype(np.int32)  # FP32 product, as the index path
        P = P.astype(np.float64)
        out = m.trilinear(P, b)
        if out is None or abs(out[0]) < 1e-4:
            continue
        img = np.zeros_like(depth)
        img[v, u] = depth[v, u]
        st = m.track_reduce(img, cam, T)
        assert st.n_valid == 1 and st.energy == pytest.approx(out[0] ** 2, rel=1e-12)
        J = np.array(st.b) / out[0]
        h = 1e-6
        Jfd = np.zeros(6)
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Pp = (scipy.linalg.expm(_twist(e)) @ np.append(P, 1))[:3]
            Pm = (scipy.linalg.expm(_twist(-e)) @ np.append(P, 1))[:3]
            Jfd[k] = (m.trilinear(Pp, b)[0] - m.trilinear(Pm, b)[0]) / (2 * h)
        assert np.allclose(J, Jfd, atol=1e-7, rtol=1e-6)
        done += 1
        if done >= 20:
            break
    assert done >= 20


def test_gauss_newton_recovers_pure_translation_in_one_step(planes_tri):
    room, m = planes_tri
    cam = I.TINY_160
    T_gt = I.look_at([0.1, -0.2, 1.0], [0.9, 0.8, 0.3])
    depth = _edge_masked_depth(room, cam, T_gt, 0.12)
    T0 = T_gt.copy()
    T0[:3, 3] += [0.015, -0.01, 0.012]
    T1, st = m.track_step(depth, cam, T0)
    assert st.status == 0 and st.n_huber == 0 and st.n_valid > 5000
    assert np.abs(T1 - T_gt).max() < 2e-6


def test_gauss_newton_recovers_pose_on_planes(planes_tri):
    room, m = planes_tri
    cam = I.TINY_160
    rng = np.random.default_rng(21)
    T_gt = I.look_at([-0.1, 0.2, 1.1], [-0.9, -0.8, 0.4])
    depth = _edge_masked_depth(room, cam, T_gt, 0.15)
    T = I.perturb_pose(T_gt, rng, 5.0, 0.05)
    for _ in range(20):
        T, st = m.track_step(depth, cam, T)
    dR = T[:3, :3].T @ T_gt[:3, :3]
    ang = math.acos(min(1.0, (np.trace(dR) - 1) / 2))
    assert ang < 1e-5 and np.linalg.norm(T[:3, 3] - T_gt[:3, 3]) < 1e-5


def test_cell_contains_the_point_on_a_curved_field():
    c = I.dense_sphere_case(2)
    m = O.OracleMap(O.params(c.voxel_size, tracker=1, huber_delta=1e9), c.dims, c.origin)
    m.set_dense(c.psi, c.grad, c.weight)
    vs = np.float64(np.float32(c.voxel_size))
    inv_vs = np.float32(1.0 / vs)
    T = c.T_init
    ys, xs = np.nonzero(c.depth > 0)
    rng = np.random.default_rng(4)
    done = 0
    for i in rng.permutation(len(xs))[:300]:
        u, v = int(xs[i]), int(ys[i])
        P, _ = O.pixel_point(c.cam, T, u, v, c.depth[v, u], c.voxel_size)
        b = np.floor(P * inv_vs).astype(np.int32)
        out = m.trilinear(P.astype(np.float64), b)
        img = np.zeros_like(c.depth)
        img[v, u] = c.depth[v, u]
        st = m.track_reduce(img, c.cam, T)
        if out is None:
            assert st.n_valid == 0
            continue
        assert st.n_valid == 1 and st.energy == pytest.approx(out[0] ** 2, rel=1e-12, abs=1e-30)
        # interpolation error of r - |x| over a cell: at most (3 / 8) v_s^2 max |d2 psi| <= 3 v_s^2 / (8 rho)
        rho = np.linalg.norm(P) - np.sqrt(3) * vs
        assert abs(out[0] - (0.4 - np.linalg.norm(P.astype(np.float64)))) <= 3 * vs**2 / (8 * rho) + 1e-6
        done += 1
    assert done > 100
