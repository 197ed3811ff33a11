"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerances (derived from the arithmetic; the GPU computes per-pixel values in FP32):
  * voxel sets, block sets, ray/visit counts and per-pixel index decisions: bit-exact (both sides
    take them on the same FP32 index path);
  * psi and ghat components: 1e-5 absolute; W: 1e-5 relative (FP32 sums of O(10^2) terms);
  * normal equations at the same pose: each H_ij within 1e-5 sqrt(H_ii H_jj), each b_i within
    1e-5 sqrt(H_ii E) + 1e-6 sqrt(H_ii n) (Cauchy-Schwarz bounds of sums of FP32 terms with
    relative error ~1e-6 and absolute residual error ~1e-7 m), E within 1e-5 relative + 1e-9;
  * tracked poses: 1e-4 per matrix entry (rad / m), the bar the method's FP32 evaluation allows.
"""
import math

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sorted(vox):
    m = vox["m"]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0]))
    return vox[order]


def _ghat(g):
    n = np.linalg.norm(g, axis=1, keepdims=True)
    return g / n


def assert_voxels_match(gv, ov, psi_tol=1e-5, g_tol=1e-5, w_rtol=1e-5):
    gv = _sorted(gv)
    assert len(gv) == len(ov["m"]), (len(gv), len(ov["m"]))
    assert np.array_equal(gv["m"], ov["m"]), "voxel sets differ"
    assert np.max(np.abs(gv["psi"] - ov["psi"])) <= psi_tol
    assert np.max(np.abs(_ghat(gv["g"].astype(np.float64)) - _ghat(ov["g"]))) <= g_tol
    assert np.max(np.abs(gv["w"] - ov["w"]) / ov["w"]) <= w_rtol


def assert_normal_equations_match(st, ost, exact_counts=True):
    n = ost.n_valid
    if exact_counts:
        assert st.n_valid == ost.n_valid
    else:
        assert abs(st.n_valid - ost.n_valid) <= max(2, 1e-3 * n)
    Ho, Hg = O.stats_H(ost), O.stats_H(st)
    d = np.sqrt(np.maximum(np.diag(Ho), 0))
    assert np.all(np.abs(Hg - Ho) <= 1e-5 * np.outer(d, d) + 1e-9), np.max(np.abs(Hg - Ho) / (np.outer(d, d) + 1e-30))
    E = ost.energy
    btol = 1e-5 * np.sqrt(np.diag(Ho) * E) + 1e-6 * np.sqrt(np.diag(Ho) * n) + 1e-9
    assert np.all(np.abs(np.array(st.b) - np.array(ost.b)) <= btol)
    assert abs(st.energy - E) <= 1e-5 * E + 1e-9


def assert_device_solve_matches(st, damping):
    """The increment the device applied solves the device's own normal equations: compared with
    the oracle's FP64 Cholesky solve of the same H and b (a pure check of the on-device solve)."""
    bad, xo = O.solve6(np.array(st.H), np.array(st.b), damping, st.n_valid)
    assert bad == (st.status != 0)
    if not bad:
        assert np.max(np.abs(np.array(st.xi) - xo)) <= 1e-10 * np.max(np.abs(xo)) + 1e-15


# ----------------------------------------------------------------------------------------------
# dense sphere grid (64^3, 2 cm voxels, 160x120 depth, 20 Gauss-Newton steps)
# ----------------------------------------------------------------------------------------------


@pytest.fixture(scope="module")
def sphere():
    return I.dense_sphere_case(1)


def _dense_maps(G, c, damping=1e-4):
    cfg = G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=damping)
    m = G.Map(cfg)
    m.upload_dense(c.psi, c.grad, c.weight)
    om = O.OracleMap(O.params(c.voxel_size, damping=damping), c.dims, c.origin)
    om.set_dense(c.psi, c.grad, c.weight)
    return m, om


def test_dense_sphere_tracking_matches_oracle_in_lockstep(G, sphere):
    """Every Gauss-Newton iterate of the oracle is fed to the GPU: at identical poses the
    normal equations match (counts exactly) and so does the updated pose."""
    c = sphere
    m, om = _dense_maps(G, c)
    K = G.intrinsics(c.cam)
    depth = _dev(c.depth)
    stats = m.new_track_stats()
    T = c.T_init.copy()
    worst = 0.0
    for it in range(c.n_iters):
        pose = _dev(T)
        m.track_step(depth, K, pose, stats)
        T_next, ost = om.track_step(c.depth, c.cam, T)
        st = G.track_stats_from_bytes(stats.cpu().numpy())
        assert st.status == ost.status == 0
        assert_normal_equations_match(st, ost)
        assert_device_solve_matches(st, 1e-4)
        worst = max(worst, np.abs(pose.cpu().numpy() - T_next).max())
        T = T_next
    print(f"dense sphere lockstep: max |T_gpu - T_oracle| after one step = {worst:.3e}")
    assert worst < 1e-4
    m.sync()


def test_dense_sphere_tracking_free_running(G, sphere):
    """20 free-running steps on each side.  A sphere leaves three pose directions (rotations
    about its centre) unobservable, so only the camera-frame sphere centre R^T (c - t) is
    compared; it matches the oracle and the ground truth within 1e-4 m / 5e-4 m."""
    c = sphere
    m, om = _dense_maps(G, c)
    K = G.intrinsics(c.cam)
    depth = _dev(c.depth)
    pose = _dev(c.T_init)
    T = c.T_init.copy()
    for it in range(c.n_iters):
        m.track_step(depth, K, pose)
        T, _ = om.track_step(c.depth, c.cam, T)
    m.sync()
    Tg = pose.cpu().numpy()
    centre = lambda X: X[:3, :3].T @ (-X[:3, 3])  # noqa: E731
    print(f"dense sphere free-running: |T_gpu - T_oracle| = {np.abs(Tg - T).max():.3e}, "
          f"centre diff = {np.linalg.norm(centre(Tg) - centre(T)):.3e}")
    assert np.linalg.norm(centre(Tg) - centre(T)) < 1e-4
    assert np.linalg.norm(centre(Tg) - centre(c.T_gt)) < 5e-4


def test_dense_tracking_is_deterministic(G, sphere):
    c = sphere
    m, _ = _dense_maps(G, c)
    K = G.intrinsics(c.cam)
    depth = _dev(c.depth)
    outs = []
    for _ in range(2):
        pose = _dev(c.T_init)
        stats = m.new_track_stats()
        for _ in range(3):
            m.track_step(depth, K, pose, stats)
        outs.append((pose.cpu().numpy(), stats.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_graph_replayed_track_equals_single_steps(G, sphere):
    """gsdf_track (n steps recorded once into a CUDA graph, then replayed) gives bit-identical
    poses and statistics to n separate gsdf_track_step calls; a change of arguments re-records."""
    c = sphere
    m, _ = _dense_maps(G, c)
    K = G.intrinsics(c.cam)
    depth = _dev(c.depth)
    n = 7
    p1 = _dev(c.T_init)
    s1 = m.new_track_stats(n)
    for it in range(n):
        m.track_step(depth, K, p1, s1[it])
    p2 = _dev(c.T_init)
    s2 = m.new_track_stats(n)
    m.track(depth, K, p2, n, s2)  # records
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    assert np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())
    p2.copy_(_dev(c.T_init))
    m.track(depth, K, p2, n, s2)  # replays
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())
    p3 = _dev(c.T_init)
    m.track(depth, K, p3, n)  # other arguments: records again
    assert np.array_equal(p1.cpu().numpy(), p3.cpu().numpy())
    m.sync()


def test_sign_flip_invariance_on_gpu(G, sphere):
    c = sphere
    m1, _ = _dense_maps(G, c)
    cfg = G.make_config(c.voxel_size, dense_dims=c.dims, dense_origin=c.origin, damping=1e-4)
    m2 = G.Map(cfg)
    m2.upload_dense(-c.psi, -c.grad, c.weight)
    K = G.intrinsics(c.cam)
    depth = _dev(c.depth)
    s1, s2 = m1.new_track_stats(), m2.new_track_stats()
    m1.track_step(depth, K, _dev(c.T_init), s1)
    m2.track_step(depth, K, _dev(c.T_init), s2)
    a, b = G.track_stats_from_bytes(s1.cpu().numpy()), G.track_stats_from_bytes(s2.cpu().numpy())
    assert np.allclose(a.H, b.H, rtol=1e-6) and np.allclose(a.b, b.b, rtol=1e-5, atol=1e-9)


def test_empty_depth_is_degenerate_and_leaves_pose(G, sphere):
    c = sphere
    m, _ = _dense_maps(G, c)
    K = G.intrinsics(c.cam)
    depth = torch.zeros((c.cam.height, c.cam.width), dtype=torch.float32, device="cuda")
    pose = _dev(c.T_init)
    stats = m.new_track_stats()
    m.track_step(depth, K, pose, stats)
    st = G.track_stats_from_bytes(stats.cpu().numpy())
    assert st.status == G.GSDF_ERR_DEGENERATE and st.n_valid == 0
    assert np.array_equal(pose.cpu().numpy(), c.T_init)
    m.sync()


def test_invalid_depth_values_are_ignored(G, sphere):
    """NaN, negative and beyond-cutoff depths count as missing, exactly like the oracle."""
    c = sphere
    rng = np.random.default_rng(0)
    d = c.depth.copy()
    idx = rng.choice(d.size, 400, replace=False)
    d.flat[idx[:100]] = np.nan
    d.flat[idx[100:200]] = -1.0
    d.flat[idx[200:300]] = 7.0
    d.flat[idx[300:]] = np.inf
    m, om = _dense_maps(G, c)
    stats = m.new_track_stats()
    m.track_step(_dev(d), G.intrinsics(c.cam), _dev(c.T_init), stats)
    ost = om.track_reduce(d, c.cam, c.T_init)
    assert_normal_equations_match(G.track_stats_from_bytes(stats.cpu().numpy()), ost)


# ----------------------------------------------------------------------------------------------
# hashed room (8^3 blocks, 1 cm voxels, 640x480 frames)
# ----------------------------------------------------------------------------------------------


@pytest.fixture(scope="module")
def room():
    return I.room_sequence(seed=2, n_frames=12)


def _hash_map(G, vs, slots=1 << 16, **kw):
    return G.Map(G.make_config(vs, hash_slots=slots, **kw))


def test_hashed_integration_matches_oracle(G, room):
    s = room
    m = _hash_map(G, s.voxel_size)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    st_dev = m.new_integrate_stats()
    for f in range(2):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]), st_dev)
        ost = om.integrate(s.depths[f], s.cam, s.poses[f])
        st = G.integrate_stats_from_bytes(st_dev.cpu().numpy())
        assert st.n_rays == ost.n_rays and st.n_visits == ost.n_visits
    m.sync()
    gv, ov = m.extract(), om.extract()
    assert_voxels_match(gv, ov)
    # block set: every allocated block holds a voxel with W > 0, and the sets agree
    gb = np.unique(np.floor_divide(gv["m"], 8), axis=0)
    ob = np.unique(np.floor_divide(ov["m"], 8), axis=0)
    assert np.array_equal(gb, ob)
    assert m.num_blocks() == len(ob) == st.n_blocks_total


def test_hashed_tracking_matches_oracle(G, room):
    """Room map from frame 0; 10 Gauss-Newton steps on frame 1.  Lockstep (the oracle's iterate
    fed to the GPU each step): normal equations match with exact counts.  Free-running: the final
    poses agree within 1e-4 and moved toward the true pose."""
    s = room
    m = _hash_map(G, s.voxel_size)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    m.integrate(_dev(s.depths[0]), K, _dev(s.poses[0]))
    om.integrate(s.depths[0], s.cam, s.poses[0])
    stats = m.new_track_stats()
    depth1 = _dev(s.depths[1])
    T = s.poses[0].copy()
    for it in range(10):
        pose = _dev(T)
        m.track_step(depth1, K, pose, stats)
        T, ost = om.track_step(s.depths[1], s.cam, T)
        st = G.track_stats_from_bytes(stats.cpu().numpy())
        assert st.status == ost.status == 0
        assert_normal_equations_match(st, ost)
        assert_device_solve_matches(st, 0.0)
        assert np.abs(pose.cpu().numpy() - T).max() < 1e-4
    pose = _dev(s.poses[0])
    for it in range(10):
        m.track_step(depth1, K, pose)
    m.sync()
    assert np.abs(pose.cpu().numpy() - T).max() < 1e-4
    assert np.linalg.norm(T[:3, 3] - s.poses[1][:3, 3]) < np.linalg.norm(s.poses[0][:3, 3] - s.poses[1][:3, 3])


def test_track_then_integrate_sequence(G, room):
    """The per-frame loop (10 Gauss-Newton steps, then fusion at the tracked pose) on both sides:
    tracked poses agree within 1e-4 and the maps stay nearly identical."""
    s = room
    n_frames = 4
    m = _hash_map(G, s.voxel_size)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    pose = _dev(s.poses[0])
    T = s.poses[0].copy()
    m.integrate(_dev(s.depths[0]), K, pose)
    om.integrate(s.depths[0], s.cam, T)
    for f in range(1, n_frames):
        d = _dev(s.depths[f])
        for _ in range(10):
            m.track_step(d, K, pose)
            T, _ = om.track_step(s.depths[f], s.cam, T)
        Tg = pose.cpu().numpy()
        assert np.abs(Tg - T).max() < 1e-4
        m.integrate(d, K, pose)
        om.integrate(s.depths[f], s.cam, T)
    m.sync()
    gv, ov = _sorted(m.extract()), om.extract()
    gset = set(map(tuple, gv["m"]))
    oset = set(map(tuple, ov["m"]))
    jac = len(gset & oset) / len(gset | oset)
    assert jac > 0.999


def test_full_size_ten_frames(G, room):
    """Full 640x480 frames in the benchmark's launch configuration: 10 frames fused at the true
    poses, then 10 Gauss-Newton steps on the next frame; voxel set exact, fields and poses within
    tolerance."""
    s = room
    m = _hash_map(G, s.voxel_size, slots=1 << 17)
    om = O.OracleMap(O.params(s.voxel_size))
    K = G.intrinsics(s.cam)
    for f in range(10):
        m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        om.integrate(s.depths[f], s.cam, s.poses[f])
    m.sync()
    assert_voxels_match(m.extract(), om.extract())
    pose = _dev(s.poses[9])
    T = s.poses[9].copy()
    d = _dev(s.depths[10])
    for _ in range(10):
        m.track_step(d, K, pose)
        T, _ = om.track_step(s.depths[10], s.cam, T)
    assert np.abs(pose.cpu().numpy() - T).max() < 1e-4


def test_ragged_image_and_dense_integration(G):
    """Odd image sizes (ragged tails in every launch) on a dense grid, integration and tracking."""
    cam = I.Camera(90.0, 90.0, 48.3, 30.7, 97, 61)
    vs = 0.02
    sphere = I.SphereScene(np.array([0.05, -0.02, 0.0]), 0.35)
    T_gt = I.look_at([0.2, -1.1, 0.3], [0.0, 0.0, 0.0], roll=0.3)
    depth = I.render_depth(sphere, cam, T_gt)
    dims, origin = (40, 40, 40), (-20, -20, -20)
    cfg = G.make_config(vs, dense_dims=dims, dense_origin=origin)
    m = G.Map(cfg)
    om = O.OracleMap(O.params(vs), dims, origin)
    K = G.intrinsics(cam)
    m.integrate(_dev(depth), K, _dev(T_gt))
    om.integrate(depth, cam, T_gt)
    m.sync()
    assert_voxels_match(m.extract(), om.extract())
    T0 = I.perturb_pose(T_gt, np.random.default_rng(1), 2.0, 0.02)
    stats = m.new_track_stats()
    m.track_step(_dev(depth), K, _dev(T0), stats)
    ost = om.track_reduce(depth, cam, T0)
    assert_normal_equations_match(G.track_stats_from_bytes(stats.cpu().numpy()), ost)


def test_extract_load_roundtrip(G, room):
    s = room
    m = _hash_map(G, s.voxel_size)
    K = G.intrinsics(s.cam)
    m.integrate(_dev(s.depths[0]), K, _dev(s.poses[0]))
    a = m.extract()
    m2 = _hash_map(G, s.voxel_size, slots=1 << 15)
    m2.load(a)
    b = m2.extract()
    assert np.array_equal(a["m"], b["m"])
    assert np.array_equal(a["g"], b["g"]) and np.array_equal(a["w"], b["w"])
    assert np.max(np.abs(a["psi"] - b["psi"]) / np.maximum(np.abs(a["psi"]), 1e-30)) <= 2.4e-7
    assert m2.num_blocks() == m.num_blocks()


def test_extraction_order_is_canonical_for_many_blocks(G, room):
    """Ten frames fused at 5 mm (more than 4096 blocks, so the block-key sort crosses several
    shared-memory chunks): the extracted voxels come in ascending block order (x, then y, then z of
    the block) and, within a block, ascending local index, whatever the table size that held them."""
    s = room
    K = G.intrinsics(s.cam)
    outs = []
    for slots in (1 << 17, 1 << 16):
        m = _hash_map(G, 0.005, slots=slots)
        for f in range(10):
            m.integrate(_dev(s.depths[f]), K, _dev(s.poses[f]))
        assert m.num_blocks() > 4096
        outs.append(m.extract())
        m.close()
    a, b = outs
    assert np.array_equal(a["m"], b["m"])
    blk = np.floor_divide(a["m"], 8).astype(np.int64)
    loc = (a["m"][:, 0] & 7) + 8 * (a["m"][:, 1] & 7) + 64 * (a["m"][:, 2] & 7)
    key = ((blk[:, 0] + (1 << 20)) << 42) | ((blk[:, 1] + (1 << 20)) << 21) | (blk[:, 2] + (1 << 20))
    assert np.all((key[1:] > key[:-1]) | ((key[1:] == key[:-1]) & (loc[1:] > loc[:-1])))


def test_capacity_exhaustion_is_reported(G, room):
    """A table far too small fills up: the frame is partially fused, the sticky error word
    reports GSDF_ERR_CAPACITY, and the handle keeps working."""
    s = room
    m = _hash_map(G, s.voxel_size, slots=8, max_probe=8)
    K = G.intrinsics(s.cam)
    m.integrate(_dev(s.depths[0]), K, _dev(s.poses[0]))
    assert G.gsdf_sync(m.h) == G.GSDF_ERR_CAPACITY
    assert G.gsdf_sync(m.h) == G.GSDF_OK  # cleared
    assert m.num_blocks() == 8
    stats = m.new_track_stats()
    m.track_step(_dev(s.depths[0]), K, _dev(s.poses[0]), stats)
    m.sync()
