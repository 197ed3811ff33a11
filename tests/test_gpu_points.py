"""Oriented point cloud extraction and its 2x2x2 Taylor upsampling (gsdf_extract_points) against
the FP64 oracle.

The voxel list comes from the oracle's fusion of the room; psi and g are rounded to FP32 and W is
set to 1, so the map's stored (W psi, g, W) give back exactly those values and both sides decide
on the same FP32 inputs.  Bars: the set of (voxel, subvoxel) entries is identical and in the
library's documented order; points within 2e-6 m (FP32 rounding of coordinates up to ~4 m, one
subtraction) and normals within 1e-6 of the oracle's FP64 values.  The full-size case is the room
fused from 10 frames of 640x480 at 1 cm, the map size of the benchmark.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


def _room_voxels(n_frames, vs):
    s = I.room_sequence(seed=2, n_frames=n_frames, voxel_size=vs)
    om = O.OracleMap(O.params(vs))
    for f in range(n_frames):
        om.integrate(s.depths[f], s.cam, s.poses[f])
    ex = om.extract()
    return ex["m"].astype(np.int32), ex["psi"].astype(np.float32), ex["g"].astype(np.float32)


def _as_map_input(G, m, psi, g):
    vox = np.zeros(len(m), G.VOXEL_DTYPE)
    vox["m"], vox["psi"], vox["g"], vox["w"] = m, psi, g, 1.0
    return vox


def _key(pts):
    return np.lexsort((pts["sub"], pts["m"][:, 2], pts["m"][:, 1], pts["m"][:, 0]))


def _block_order(pts):
    """Sort key of the library's order: block (lexicographic), local index x + 8 y + 64 z, sub."""
    b = pts["m"] >> 3
    loc = (pts["m"][:, 0] & 7) + 8 * (pts["m"][:, 1] & 7) + 64 * (pts["m"][:, 2] & 7)
    return np.lexsort((pts["sub"], loc, b[:, 2], b[:, 1], b[:, 0]))


def _compare(gp, op):
    assert len(gp) == len(op), (len(gp), len(op))
    assert np.array_equal(_block_order(gp), np.arange(len(gp))), "not in the documented order"
    g2, o2 = gp[_key(gp)], op[_key(op)]
    assert np.array_equal(g2["m"], o2["m"]) and np.array_equal(g2["sub"], o2["sub"]), "point sets differ"
    dp = np.abs(g2["p"].astype(np.float64) - o2["p"]).max()
    dn = np.abs(g2["n"].astype(np.float64) - o2["n"]).max()
    print(f"points: {len(gp)}, max |dp| = {dp:.2e} m, max |dn| = {dn:.2e}")
    assert dp <= 2e-6 and dn <= 1e-6


@pytest.mark.parametrize("n_frames,vs", [(2, 0.02), (10, 0.01)])
def test_points_match_oracle_on_hashed_room(G, n_frames, vs):
    m, psi, g = _room_voxels(n_frames, vs)
    gm = G.Map(G.make_config(vs, hash_slots=1 << 18))
    gm.load(_as_map_input(G, m, psi, g))
    for level in (0, 1):
        gp = gm.extract_points(level)
        op = O.points(m, psi.astype(np.float64), g.astype(np.float64), vs, level)
        assert len(op) > (1000 if vs > 0.015 else 50000)
        _compare(gp, op)
    gm.close()


def test_points_match_oracle_on_dense_sphere(G):
    vs, r = 0.02, 0.4
    dims, origin = (64, 64, 64), (-32, -32, -32)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1)
    m = (idx + np.array(origin)).transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.int32)  # x fastest
    v = m * np.float64(np.float32(vs))
    nv = np.maximum(np.linalg.norm(v, axis=1), 1e-9)
    psi = (r - nv).astype(np.float32)
    g = (-v / nv[:, None]).astype(np.float32)
    w = (np.abs(r - nv) <= 5 * vs).astype(np.float32)
    gm = G.Map(G.make_config(vs, dense_dims=dims, dense_origin=origin))
    gm.upload_dense(psi, g.reshape(-1), w)
    keep = w > 0
    for level in (0, 1):
        gp = gm.extract_points(level)
        op = O.points(m[keep], psi[keep].astype(np.float64), g[keep].astype(np.float64), vs, level)
        assert len(gp) == len(op) > 1000
        g2, o2 = gp[_key(gp)], op[_key(op)]
        assert np.array_equal(g2["m"], o2["m"]) and np.array_equal(g2["sub"], o2["sub"])
        assert np.abs(g2["p"] - o2["p"]).max() <= 2e-6 and np.abs(g2["n"] - o2["n"]).max() <= 1e-6
    gm.close()


def test_capacity_and_arguments(G):
    m, psi, g = _room_voxels(1, 0.02)
    gm = G.Map(G.make_config(0.02, hash_slots=1 << 16))
    gm.load(_as_map_input(G, m, psi, g))
    st, n = G.gsdf_extract_points(gm.h, 1, None, 0)
    assert st == G.GSDF_ERR_CAPACITY and n > 100
    small = np.zeros(10, G.POINT_DTYPE)
    st, n2 = G.gsdf_extract_points(gm.h, 1, small, 10)
    assert st == G.GSDF_ERR_CAPACITY and n2 == n
    full = gm.extract_points(1)
    assert np.array_equal(small, full[:10])
    st, _ = G.gsdf_extract_points(gm.h, 2, None, 0)
    assert st == G.GSDF_ERR_INVALID_ARG
    empty = G.Map(G.make_config(0.02, hash_slots=1 << 10))
    assert len(empty.extract_points(0)) == 0 and len(empty.extract_points(1)) == 0
    gm.close()
    empty.close()
