"""Marching-cubes mesh (gsdf_extract_mesh) against the oracle's layered marching cubes.

As for the point cloud, the voxel list comes from the oracle's fusion of the room with psi rounded
to FP32 and W = 1, so both sides take the same inside/outside decisions.  The two triangulation
tables are generated independently from the same stated rule.  Bars: the set of (cube, edge
triple) entries is identical and in the library's documented order; vertices within 2e-6 m (FP32
interpolation of coordinates up to ~4 m).
"""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_points import _as_map_input, _room_voxels  # noqa: E402


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


def _key(t):
    return np.lexsort((t["edges"], t["m"][:, 2], t["m"][:, 1], t["m"][:, 0]))


def _block_order(t):
    b = t["m"] >> 3
    loc = (t["m"][:, 0] & 7) + 8 * (t["m"][:, 1] & 7) + 64 * (t["m"][:, 2] & 7)
    return np.lexsort((loc, b[:, 2], b[:, 1], b[:, 0]))


def _compare(gt, ot, ordered=True):
    assert len(gt) == len(ot), (len(gt), len(ot))
    if ordered:  # cubes in the library's voxel order (a stable sort keeps each cube's triangles together)
        o = _block_order(gt)
        assert np.array_equal(gt["m"][o], gt["m"]), "not in the documented order"
    g2, o2 = gt[_key(gt)], ot[_key(ot)]
    assert np.array_equal(g2["m"], o2["m"]) and np.array_equal(g2["edges"], o2["edges"]), "triangle sets differ"
    dv = np.abs(g2["v"].astype(np.float64) - o2["v"]).max()
    print(f"triangles: {len(gt)}, max |dv| = {dv:.2e} m")
    assert dv <= 2e-6


@pytest.mark.parametrize("n_frames,vs", [(2, 0.02), (10, 0.01)])
def test_mesh_matches_oracle_on_hashed_room(G, n_frames, vs):
    m, psi, g = _room_voxels(n_frames, vs)
    gm = G.Map(G.make_config(vs, hash_slots=1 << 18))
    gm.load(_as_map_input(G, m, psi, g))
    gt = gm.extract_mesh()
    ot = O.marching_cubes(m, psi.astype(np.float64), vs)
    assert len(ot) > (1000 if vs > 0.015 else 100000)
    _compare(gt, ot)
    gm.close()


def test_mesh_of_dense_sphere(G):
    vs, r = 0.02, 0.4
    dims, origin = (64, 64, 64), (-32, -32, -32)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1)
    m = (idx + np.array(origin)).transpose(2, 1, 0, 3).reshape(-1, 3).astype(np.int32)
    v = m * np.float64(np.float32(vs))
    nv = np.maximum(np.linalg.norm(v, axis=1), 1e-9)
    psi = (r - nv).astype(np.float32)
    g = (-v / nv[:, None]).astype(np.float32)
    w = (np.abs(r - nv) <= 5 * vs).astype(np.float32)
    gm = G.Map(G.make_config(vs, dense_dims=dims, dense_origin=origin))
    gm.upload_dense(psi, g.reshape(-1), w)
    gt = gm.extract_mesh()
    keep = w > 0
    ot = O.marching_cubes(m[keep], psi[keep].astype(np.float64), vs)
    _compare(gt, ot, ordered=False)
    gm.close()


def test_mesh_capacity_and_empty(G):
    m, psi, g = _room_voxels(1, 0.02)
    gm = G.Map(G.make_config(0.02, hash_slots=1 << 16))
    gm.load(_as_map_input(G, m, psi, g))
    st, n = G.gsdf_extract_mesh(gm.h, None, 0)
    assert st == G.GSDF_ERR_CAPACITY and n > 100
    small = np.zeros(7, G.TRIANGLE_DTYPE)
    st, n2 = G.gsdf_extract_mesh(gm.h, small, 7)
    assert st == G.GSDF_ERR_CAPACITY and n2 == n
    assert np.array_equal(small, gm.extract_mesh()[:7])
    empty = G.Map(G.make_config(0.02, hash_slots=1 << 10))
    assert len(empty.extract_mesh()) == 0
    gm.close()
    empty.close()
