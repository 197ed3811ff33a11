"""Pins of the oracle's layered marching cubes (Sec. 4.3).

* The triangulation rule on all 256 cases: the triangles of a case use exactly its crossing edges,
  and every join is made once (each crossing edge lies on two faces).
* On a sphere (psi = r - |v|): the mesh is a closed 2-manifold -- every mesh edge, identified by the
  two grid edges its vertices lie on, belongs to exactly two triangles -- with Euler characteristic
  V - E + F = 2, vertices within the linear-interpolation error of r - |x| along a grid edge of the
  sphere, and area within 1.5 % of 4 pi r^2.
* On planes (linear psi, so interpolation is exact): vertices on the plane; an axis-aligned plane
  gives two triangles per straddling cube and exactly the covered area.
* A cube with a corner missing from the list gives nothing.
"""
import numpy as np
import pytest

from oracle import oracle as O

VS = 0.02


def _grid(lo, hi):
    r = np.arange(lo, hi)
    return np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3).astype(np.int32)


def _cube_list(inside_bits):
    m = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int32)
    psi = np.array([1.0 if (inside_bits >> c) & 1 else -1.0 for c in range(8)])
    return m, psi


def _edge_corners(e):
    axis, k = e >> 2, e & 3
    lo = [0, 0, 0]
    others = [a for a in range(3) if a != axis]
    lo[others[0]], lo[others[1]] = k & 1, k >> 1
    a = lo[0] + 2 * lo[1] + 4 * lo[2]
    return a, a | (1 << axis)


def test_every_case_uses_exactly_its_crossing_edges():
    for case in range(256):
        m, psi = _cube_list(case)
        tri = O.marching_cubes(m, psi, 1.0)
        crossing = {e for e in range(12) if ((case >> _edge_corners(e)[0]) & 1) != ((case >> _edge_corners(e)[1]) & 1)}
        used = set()
        for t in tri:
            used |= {(t["edges"] >> (4 * k)) & 15 for k in range(3)}
        assert used == crossing, case
        if case in (0, 255):
            assert len(tri) == 0
        # a fan over loops: triangles = crossings - 2 * loops, at least one loop if anything crosses
        if crossing:
            assert len(tri) <= len(crossing) - 2 and (len(crossing) - len(tri)) % 2 == 0


def _global_edge(mc, e):
    a, b = _edge_corners(e)
    ca = tuple(mc + np.array([a & 1, (a >> 1) & 1, (a >> 2) & 1]))
    cb = tuple(mc + np.array([b & 1, (b >> 1) & 1, (b >> 2) & 1]))
    return (ca, cb)


def test_sphere_mesh_is_a_closed_manifold_near_the_sphere():
    r = 0.4
    m = _grid(-26, 26)
    v = m * np.float64(np.float32(VS))
    nv = np.linalg.norm(v, axis=1)
    keep = np.abs(r - nv) < 3 * VS
    m, v, nv = m[keep], v[keep], nv[keep]
    tri = O.marching_cubes(m, r - nv, VS)
    assert len(tri) > 1000
    verts = {}
    faces = []
    for t in tri:
        ids = []
        for k in range(3):
            key = _global_edge(t["m"], (t["edges"] >> (4 * k)) & 15)
            ids.append(verts.setdefault(key, len(verts)))
        faces.append(ids)
    faces = np.array(faces)
    edges = {}
    for f in faces:
        for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0])):
            key = (min(a, b), max(a, b))
            edges[key] = edges.get(key, 0) + 1
    assert set(edges.values()) == {2}
    assert len(verts) - len(edges) + len(faces) == 2
    P = tri["v"].reshape(-1, 3)
    rad = np.linalg.norm(P, axis=1)
    assert np.max(np.abs(rad - r)) <= VS**2 / (8 * (r - VS))
    area = 0.5 * np.linalg.norm(np.cross(P[1::3] - P[0::3], P[2::3] - P[0::3]), axis=1).sum()
    assert area == pytest.approx(4 * np.pi * r**2, rel=0.015)


@pytest.mark.parametrize("normal", [(0.0, 0.0, 1.0), (0.3, -0.5, 0.81)])
def test_planes(normal):
    n = np.asarray(normal) / np.linalg.norm(normal)
    d = 0.0123
    m = _grid(-15, 15)
    v = m * np.float64(np.float32(VS))
    psi = d - v @ n
    keep = np.abs(psi) < 3 * VS
    tri = O.marching_cubes(m[keep], psi[keep], VS)
    P = tri["v"].reshape(-1, 3)
    assert np.max(np.abs(P @ n - d)) < 1e-12
    if normal == (0.0, 0.0, 1.0):
        cols = len({tuple(x) for x in tri["m"][:, :2]})
        assert len(tri) == 2 * cols and cols == 29 * 29
        area = 0.5 * np.linalg.norm(np.cross(P[1::3] - P[0::3], P[2::3] - P[0::3]), axis=1).sum()
        assert area == pytest.approx(29 * 29 * np.float64(np.float32(VS)) ** 2, rel=1e-12)


def test_cube_with_a_missing_corner_gives_nothing():
    m, psi = _cube_list(1)
    assert len(O.marching_cubes(m[1:], psi[1:], 1.0)) == 0
    assert len(O.marching_cubes(m, psi, 1.0)) == 1
