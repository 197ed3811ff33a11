"""Pins of the oracle's oriented point cloud and its 2x2x2 Taylor upsampling (Sec. 4.3).

Analytic voxel fields stand in for fused maps, so every expected value is a closed form:
* a plane n.x = d sampled with psi = d - n.v, ghat = -n (the Taylor model of Eq. taylor is exact on
  it): every point lies on the plane with normal n, and the selection |psi ghat| <= v_s/2 per axis
  keeps the voxel centres of a slab of thickness v_s / max|n_k|, so the points have an area density
  of 1 / (v_s^2 max|n_k|); the upsampled cloud has four times that;
* an axis-aligned plane: exactly one point per voxel column (four after upsampling), at the
  column's (x, y) and the plane's height;
* a sphere with psi = r - |v|, ghat = -v/|v|: level-0 points lie on the sphere with radial normals;
  upsampled points lie on the tangent plane of their voxel's point, offset tangentially by at most
  sqrt(3) v_s / 4, so 0 <= |p| - r <= 3 v_s^2 / (32 r);
* the geometric meaning of the selection: a kept voxel's point lies in the voxel's cube
  (|p - v| <= v_s/2 per axis), a kept subvoxel's point in the subvoxel's cube (|p - c| <= v_s/4), and
  on an axis-aligned plane the kept subvoxel layer is the one within v_s/4 of the plane.
"""
import numpy as np
import pytest

from oracle import oracle as O

VS = 0.02


def _grid(lo, hi):
    r = np.arange(lo, hi)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)
    return m


def _centres(pts):
    """Centre of each point's voxel (level 0) or subvoxel (level 1)."""
    vs = np.float64(np.float32(VS))
    c = pts["m"] * vs
    sub = pts["sub"][:, None]
    bits = np.stack([(pts["sub"] >> k) & 1 for k in range(3)], -1)
    return np.where(sub >= 0, c + np.where(bits == 1, 1.0, -1.0) * vs / 4, c)


def _in_own_cube(pts, level):
    half = (VS / 2) if level == 0 else (VS / 4)
    return np.max(np.abs(pts["p"] - _centres(pts))) <= half * (1 + 1e-6)


def _plane(normal, d, lo=-40, hi=40):
    n = np.asarray(normal, float)
    n /= np.linalg.norm(n)
    m = _grid(lo, hi)
    v = m * np.float64(np.float32(VS))
    psi = d - v @ n
    g = np.broadcast_to(-n, v.shape).copy()
    keep = np.abs(psi) < 3 * VS  # a band around the surface, like a fused map
    return m[keep], psi[keep], g[keep], n


@pytest.mark.parametrize("normal", [(0.3, 0.5, 0.81), (1.0, 1.0, 1.0), (0.1, -0.9, 0.4)])
def test_tilted_plane_points_and_density(normal):
    m, psi, g, n = _plane(normal, 0.0123)
    for level, spacing in ((0, VS), (1, VS / 2)):
        pts = O.points(m, psi, g, VS, level)
        assert len(pts) > 1000
        assert np.max(np.abs(pts["p"] @ n - 0.0123)) < 1e-12  # on the plane
        assert np.allclose(pts["n"], n, atol=1e-12)
        assert _in_own_cube(pts, level)
        # density inside a disk of radius R around the plane's centre point, away from the grid edges
        c = 0.0123 * n
        R = 0.5
        inside = np.linalg.norm(pts["p"] - c, axis=1) < R
        expected = np.pi * R**2 / (spacing**2 * np.max(np.abs(n)))
        assert inside.sum() == pytest.approx(expected, rel=0.02), (level, inside.sum(), expected)


def test_axis_aligned_plane_gives_one_point_per_column():
    z0 = 0.3 * VS + 0.0011
    m, psi, g, n = _plane((0, 0, 1), z0)
    cols = {tuple(x) for x in m[:, :2]}
    p0 = O.points(m, psi, g, VS, 0)
    assert len(p0) == len(cols)
    assert len({tuple(x) for x in p0["m"][:, :2]}) == len(cols)
    vs = np.float64(np.float32(VS))
    assert np.allclose(p0["p"][:, :2], p0["m"][:, :2] * vs, atol=1e-15)
    assert np.allclose(p0["p"][:, 2], z0, atol=1e-15)
    p1 = O.points(m, psi, g, VS, 1)
    assert len(p1) == 4 * len(cols)
    sub = p1["sub"]
    dx = np.where(sub & 1, 1, -1) * vs / 4
    dy = np.where(sub & 2, 1, -1) * vs / 4
    assert np.allclose(p1["p"][:, 0], p1["m"][:, 0] * vs + dx, atol=1e-15)
    assert np.allclose(p1["p"][:, 1], p1["m"][:, 1] * vs + dy, atol=1e-15)
    assert np.allclose(p1["p"][:, 2], z0, atol=1e-15)
    cz = _centres(p1)[:, 2]
    assert np.all(np.abs(cz - z0) <= vs / 4)  # the kept layer straddles the plane


def test_sphere_points_and_upsampling_bound():
    r = 0.4
    m = _grid(-32, 32)
    v = m * np.float64(np.float32(VS))
    nv = np.linalg.norm(v, axis=1)
    keep = (np.abs(r - nv) < 3 * VS) & (nv > 0)
    m, v, nv = m[keep], v[keep], nv[keep]
    psi = r - nv
    g = -v / nv[:, None]
    p0 = O.points(m, psi, g, VS, 0)
    rad = np.linalg.norm(p0["p"], axis=1)
    assert len(p0) > 1000
    assert np.max(np.abs(rad - r)) < 1e-12
    assert np.allclose(p0["n"], p0["p"] / rad[:, None], atol=1e-12)
    assert _in_own_cube(p0, 0)
    p1 = O.points(m, psi, g, VS, 1)
    assert _in_own_cube(p1, 1)
    rad1 = np.linalg.norm(p1["p"], axis=1)
    assert np.min(rad1 - r) > -1e-12
    assert np.max(rad1 - r) <= 3 * VS**2 / (32 * r) + 1e-12
    # the upsampled cloud is about four times denser
    assert 3.5 < len(p1) / len(p0) < 4.5
    # every sphere direction has a level-0 point within one voxel
    rng = np.random.default_rng(0)
    u = rng.normal(size=(2000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    dmin = np.min(np.linalg.norm((r * u)[:, None, :] - p0["p"][None, :, :], axis=2), axis=1)
    assert dmin.max() <= VS


def test_zero_gradient_and_empty_list():
    m = np.array([[0, 0, 0]], np.int32)
    assert len(O.points(m, np.array([0.0]), np.zeros((1, 3)), VS, 0)) == 0
    assert len(O.points(m, np.array([0.0]), np.zeros((1, 3)), VS, 1)) == 0
    assert len(O.points(np.zeros((0, 3), np.int32), np.zeros(0), np.zeros((0, 3)), VS, 1)) == 0
