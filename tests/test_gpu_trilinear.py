"""The trilinear 8-lookup tracker (the direct SDF baseline of Eqs. dir_dist, dir_grad;
GSDF_TRACKER_TRILINEAR) against the FP64 oracle with tracker = 1.

Both sides fuse the same frames (voxel sets equal bit for bit, so the "all 8 corners observed"
decision agrees) and take the interpolation cell on the FP32 index path, so the pixel counts are
exact; H, b and E carry the tolerances of the Taylor tracker's tests (sums of FP32 terms), and poses
agree within 1e-4.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_13652_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_gpu_parity import assert_device_solve_matches, assert_normal_equations_match  # noqa: E402

TRI = 1


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_13652_gb300 import gsdf

    gsdf.load_library()
    return gsdf


@pytest.fixture(scope="module")
def room():
    return I.room_sequence(seed=2, n_frames=12)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_trilinear_tracking_matches_oracle_on_room(G, room):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 16, tracker=TRI))
    om = O.OracleMap(O.params(s.voxel_size, tracker=TRI))
    K = G.intrinsics(s.cam)
    for f in range(2):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        om.integrate(s.depths[f], s.cam, s.poses[f])
    stats = m.new_track_stats()
    depth = _dev(s.depths[2])
    T = s.poses[1].copy()
    for _ in range(10):  # lockstep: the oracle's iterate is given to the GPU each step
        pose = _dev(T)
        m.track_step(depth, K, pose, stats)
        T, ost = om.track_step(s.depths[2], s.cam, T)
        st = G.track_stats_from_bytes(stats.cpu().numpy())
        assert st.status == ost.status == 0 and ost.n_valid > 100000
        assert_normal_equations_match(st, ost)
        assert_device_solve_matches(st, 0.0)
        assert np.abs(pose.cpu().numpy() - T).max() < 1e-4
    pose = _dev(s.poses[1])
    m.track(depth, K, pose, 10)  # free running, graph-replayed
    m.sync()
    assert np.abs(pose.cpu().numpy() - T).max() < 1e-4
    assert np.linalg.norm(T[:3, 3] - s.poses[2][:3, 3]) < np.linalg.norm(s.poses[1][:3, 3] - s.poses[2][:3, 3])


def test_trilinear_full_size_ten_frames(G, room):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 17, tracker=TRI))
    om = O.OracleMap(O.params(s.voxel_size, tracker=TRI))
    K = G.intrinsics(s.cam)
    for f in range(10):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        om.integrate(s.depths[f], s.cam, s.poses[f])
    pose = _dev(s.poses[9])
    T = s.poses[9].copy()
    d = _dev(s.depths[10])
    for _ in range(10):
        m.track_step(d, K, pose)
        T, _ = om.track_step(s.depths[10], s.cam, T)
    m.sync()
    assert np.abs(pose.cpu().numpy() - T).max() < 1e-4


def test_trilinear_on_dense_sphere_in_lockstep(G):
    c = I.dense_sphere_case(1)
    cfg = G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=1e-4, tracker=TRI)
    m = G.Map(cfg)
    m.upload_dense(c.psi, c.grad, c.weight)
    om = O.OracleMap(O.params(c.voxel_size, damping=1e-4, tracker=TRI), c.dims, c.origin)
    om.set_dense(c.psi, c.grad, c.weight)
    stats = m.new_track_stats()
    d = _dev(c.depth)
    T = c.T_init.copy()
    for _ in range(5):
        pose = _dev(T)
        m.track_step(d, G.intrinsics(c.cam), pose, stats)
        T, ost = om.track_step(c.depth, c.cam, T)
        st = G.track_stats_from_bytes(stats.cpu().numpy())
        assert ost.n_valid > 1000
        assert_normal_equations_match(st, ost)
        assert np.abs(pose.cpu().numpy() - T).max() < 1e-4


def test_trilinear_configuration_limits(G, room):
    L = G.load_library()
    import ctypes as C

    h = C.c_void_p()
    bad = G.make_config(0.01, hash_slots=1 << 12, fp16=True, max_touched_blocks=1 << 10, tracker=TRI)
    assert L.gsdf_create(C.byref(bad), None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    bad = G.make_config(0.01, hash_slots=1 << 12, tracker=2)
    assert L.gsdf_create(C.byref(bad), None, C.byref(h)) == G.GSDF_ERR_INVALID_ARG
    m = G.Map(G.make_config(0.01, hash_slots=1 << 12, tracker=TRI))
    with pytest.raises(G.GsdfError):
        G.Batch([m])  # batches run the Taylor tracker only
    m.close()
