"""gsdf_track's chained steps against single steps and the oracle.

gsdf_track with n >= 2 solves each step's normal equations at the start of the next launch
(every block, from the exact fixed-point sums) and the last one in a final one-block launch,
instead of in the last block of each step.  The operations on the same exact sums are the same,
so poses and statistics must equal those of n gsdf_track_step calls bit for bit, for every map
kind and tracker, call after call (the chain's accumulator sets are zeroed for the next call).
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
    return I.room_sequence(seed=2, n_frames=12)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _room_map(G, room, **kw):
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 17, **kw))
    K = G.intrinsics(s.cam)
    for f in range(3):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
    return m, K, _dev(s.depths[3]), s.poses[2]


def _sphere_map(G, **kw):
    c = I.dense_sphere_case(1)
    m = G.Map(G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=1e-4, **kw))
    m.upload_dense(c.psi, c.grad, c.weight)
    return m, G.intrinsics(c.cam), _dev(c.depth), c.T_init


def _compare_chain_with_steps(G, m, K, depth, T0, n, calls=2):
    """`calls` consecutive gsdf_track calls of n steps each against the same number of single
    steps: poses and statistics equal bit for bit after every call."""
    p_chain, p_step = _dev(T0), _dev(T0)
    for call in range(calls):
        s_chain, s_step = m.new_track_stats(n), m.new_track_stats(n)
        m.track(depth, K, p_chain, n, s_chain)
        for it in range(n):
            m.track_step(depth, K, p_step, s_step[it])
        torch.cuda.synchronize()
        assert np.array_equal(p_chain.cpu().numpy(), p_step.cpu().numpy()), (n, call)
        assert bytes(s_chain.cpu().numpy()) == bytes(s_step.cpu().numpy()), (n, call)
    m.sync()
    return p_chain.cpu().numpy(), [G.track_stats_from_bytes(x) for x in s_chain.cpu().numpy()]


@pytest.mark.parametrize("tracker", [0, 1])
@pytest.mark.parametrize("n", [2, 3, 10])
def test_chain_equals_single_steps_dense(G, n, tracker):
    m, K, depth, T0 = _sphere_map(G, tracker=tracker)
    _, st = _compare_chain_with_steps(G, m, K, depth, T0, n)
    assert all(s.status == G.GSDF_OK and s.n_valid > 5000 for s in st)
    m.close()


@pytest.mark.parametrize("kind", ["fp32", "fp16", "trilinear"])
def test_chain_equals_single_steps_hashed(G, room, kind):
    kw = {"fp16": True} if kind == "fp16" else ({"tracker": 1} if kind == "trilinear" else {})
    m, K, depth, T0 = _room_map(G, room, **kw)
    for n in (2, 10):
        _, st = _compare_chain_with_steps(G, m, K, depth, T0, n)
        assert all(s.status == G.GSDF_OK and s.n_valid > 100000 for s in st)
    m.close()


def test_chain_degenerate_steps_leave_pose(G):
    """An empty frame: every step of the chain is degenerate, the pose is left unchanged and
    every step's statistics say so; the next call on a real frame is unaffected."""
    m, K, depth, T0 = _sphere_map(G)
    empty = torch.zeros_like(depth)
    pose = _dev(T0)
    st = m.new_track_stats(4)
    m.track(empty, K, pose, 4, st)
    torch.cuda.synchronize()
    assert np.array_equal(pose.cpu().numpy(), T0)
    for s in st.cpu().numpy():
        s = G.track_stats_from_bytes(s)
        assert s.status == G.GSDF_ERR_DEGENERATE and s.n_valid == 0 and not np.any(s.xi)
    _compare_chain_with_steps(G, m, K, depth, T0, 5, calls=1)
    m.close()


def test_chain_in_a_caller_captured_graph(G):
    """When the caller is capturing the map's stream, gsdf_track launches the chain into the
    caller's graph; replaying that graph twice equals 2 n single steps."""
    c = I.dense_sphere_case(1)
    s = torch.cuda.Stream()
    m = G.Map(G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=1e-4), s)
    m.upload_dense(c.psi, c.grad, c.weight)
    K = G.intrinsics(c.cam)
    depth, pose = _dev(c.depth), _dev(c.T_init)
    st = m.new_track_stats(6)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        m.track(depth, K, pose, 6, st)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    p_step = _dev(c.T_init)
    for _ in range(12):
        m.track_step(depth, K, p_step)
    m.sync()
    assert np.array_equal(pose.cpu().numpy(), p_step.cpu().numpy())
    m.close()


def test_chain_full_size_against_oracle(G, room):
    """The benchmark's form: 10 frames fused at the true poses, then one gsdf_track call of 10
    steps on the next frame against 10 free-running oracle steps: the final poses within 1e-4, the
    first step's usable-pixel count equal (both sides start at the same pose), every step solved."""
    s = room
    m = G.Map(G.make_config(s.voxel_size, hash_slots=1 << 17))
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    for f in range(10):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        om.integrate(s.depths[f], s.cam, s.poses[f])
    pose = _dev(s.poses[9])
    st = m.new_track_stats(10)
    m.track(_dev(s.depths[10]), K, pose, 10, st)
    T = s.poses[9].copy()
    ost = []
    for _ in range(10):
        T, o = om.track_step(s.depths[10], s.cam, T)
        ost.append(o)
    m.sync()
    assert np.abs(pose.cpu().numpy() - T).max() < 1e-4
    gst = [G.track_stats_from_bytes(x) for x in st.cpu().numpy()]
    assert gst[0].n_valid == ost[0].n_valid  # the first step runs at the same pose on both sides
    assert all(g.status == o.status == 0 for g, o in zip(gst, ost))
    m.close()
