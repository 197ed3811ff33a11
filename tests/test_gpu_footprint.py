"""gsdf_footprint: the distinct voxels and blocks that a tracking step or a fusion touches.

Fusion: into an empty map, the footprint of the first frame is the whole map (every voxel with
W > 0 and every allocated block); for a later frame it is exactly the set of voxels whose weight
that fusion raised, read off two extractions.  Tracking: the oracle's own FP32 index path gives
each valid pixel's nearest voxel (Eq. taylor); the footprint is the number of distinct such voxels
that the map holds with g != 0, and of their blocks.
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


@pytest.fixture(scope="module")
def room():
    return I.room_sequence(seed=2, n_frames=3, cam=I.scaled_camera(160, 120), voxel_size=0.02)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _keys(vox):
    return {tuple(int(c) for c in m): i for i, m in enumerate(vox["m"])}


@pytest.mark.parametrize("fp16", [False, True])
def test_fusion_footprint_counts_the_updated_voxels(G, room, fp16):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 14, fp16=fp16, max_touched_blocks=1 << 12))
    K = G.intrinsics(s.cam)
    d0, p0 = _dev(s.depths[0]), _dev(s.poses[0])
    m.integrate(d0, K, p0)
    v0 = m.extract()
    assert m.footprint(G.GSDF_FOOTPRINT_FUSE, d0, K, p0) == (len(v0), m.num_blocks())
    d1, p1 = _dev(s.depths[1]), _dev(s.poses[1])
    m.integrate(d1, K, p1)
    v1 = m.extract()
    k0 = _keys(v0)
    changed = [i for i, mm in enumerate(v1["m"])
               if tuple(int(c) for c in mm) not in k0 or v1["w"][i] != v0["w"][k0[tuple(int(c) for c in mm)]]]
    blocks = {tuple(int(c) for c in np.floor_divide(v1["m"][i], 8)) for i in changed}
    assert m.footprint(G.GSDF_FOOTPRINT_FUSE, d1, K, p1) == (len(changed), len(blocks))
    m.sync()
    m.close()


def test_tracking_footprint_matches_the_oracles_pixel_voxels(G, room):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 14))
    K = G.intrinsics(s.cam)
    for f in range(2):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
    vox = m.extract()
    usable = {tuple(int(c) for c in mm) for mm, g in zip(vox["m"], vox["g"]) if np.any(g != 0)}
    T = s.poses[1]
    D = s.depths[2]
    seen = set()
    for v in range(s.cam.height):
        for u in range(s.cam.width):
            z = float(D[v, u])
            if not (0.0 < z <= s.cam.depth_max):
                continue
            _, mm = O.pixel_point(s.cam, T, u, v, np.float32(z), s.voxel_size)
            key = tuple(int(c) for c in mm)
            if key in usable:
                seen.add(key)
    blocks = {tuple(c // 8 for c in k) for k in seen}
    assert len(seen) > 1000
    assert m.footprint(G.GSDF_FOOTPRINT_TRACK, _dev(D), K, _dev(T)) == (len(seen), len(blocks))
    m.close()


def test_footprint_arguments(G, room):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 10))
    d, p = _dev(s.depths[0]), _dev(s.poses[0])
    with pytest.raises(G.GsdfError):
        m.footprint(7, d, G.intrinsics(s.cam), p)
    empty = torch.zeros_like(d)
    assert m.footprint(G.GSDF_FOOTPRINT_TRACK, empty, G.intrinsics(s.cam), p) == (0, 0)
    m.close()
